// Ladder (Bethe-Salpeter) solves of Eq. lin_alg_inv, FP64 path, and the
// leading-eigenvalue check of gamma chi~ (the convergence-radius condition
// stated after Eq. lin_alg_inv).
//
// For every (q, W) and channel: D = 1 - gamma_W diag(chi~_W(q)), solve
// D Gamma = gamma_W, keep only diag Gamma, and write the Eq. sd bracket
//     kc = c (Gamma_ww - Gamma^(2)_ww / 2),  Gamma^(2)_ww = sum_x gamma_wx chi~_x gamma_xw,
// with c = 1 (density) or 3 (magnetic).
//
// Design: one CTA per system (persistent grid, systems strided by
// gridDim.x), D factorised in place by right-looking LU with partial
// pivoting (pivot = largest |re|+|im| in the column, first on ties), the
// right-hand sides P gamma processed in column chunks.  Because only the
// diagonal of Gamma is needed, the back substitution for column j stops at
// row j: LU (n^3/3) + forward (n^3/2) + truncated back substitution (n^3/6)
// = n^3 complex multiply-adds per system instead of 4n^3/3.  U's columns are
// pre-scaled by 1/U_kk so that neither substitution divides.
#include "df_bse_dev.cuh"

namespace df {

// gg[c][a][i][j] = gamma[c][a][i][j] * gamma[c][a][j][i]  (for Gamma^(2))
__global__ void gamma_gt_kernel(int n, int count, const double2* __restrict__ gam, double2* __restrict__ gg) {
  const size_t total = (size_t)count * n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t mat = idx / ((size_t)n * n);
    const int rem = (int)(idx - mat * n * n);
    const int i = rem / n, j = rem - i * n;
    const double2* G = gam + mat * n * n;
    gg[idx] = cmul(G[i * n + j], G[j * n + i]);
  }
}

template <bool LU_SMEM>
__global__ void __launch_bounds__(kBseThreads)
bse_f64_kernel(Dims dm, int ch0, int nch, int nc, const double2* __restrict__ gam,
               const double2* __restrict__ gg, const double2* __restrict__ chi,
               double2* __restrict__ kc, double2* __restrict__ ws, int* __restrict__ flags, int radius_K,
               const double2* __restrict__ lam, const int* __restrict__ list, int spread) {
  extern __shared__ double2 sm[];
  __shared__ BseF64Shared sh;
  const int n = dm.n_w, N = dm.N, nb = dm.nb, na = dm.na;
  const BseSmem L = bse_layout(n, nc, LU_SMEM);
  double2* LU = LU_SMEM ? sm + L.lu : ws + (size_t)blockIdx.x * n * n;
  // the handle's planes of channels ch0 .. ch0 + nch - 1, or with `list` the
  // list[0] systems (c N_W + a) N + q that follow it (ladders the mixed-precision
  // kernels handed back).  A short list is spread over up to `spread` blocks:
  // each ladder's right-hand-side chunks are split into `parts` column ranges,
  // one block per range, each factorising the ladder itself (the FP64 pipe of
  // one SM bounds a lone ladder's latency)
  const int chunks = (n + nc - 1) / nc;
  long count = list ? (long)list[0] : 0;
  int parts = 1;
  if (list && count > 0 && spread > count) {
    const long p = spread / count;
    parts = (int)(p < chunks ? p : chunks);
  }
  const int cpp = (chunks + parts - 1) / parts;      // chunks per part
  const long systems = list ? count * parts : (long)nch * na * N;
  for (long s = blockIdx.x; s < systems; s += gridDim.x) {
    int c, a, q, jb = 0, je = n;
    if (list) {
      const int part = (int)(s % parts);
      jb = part * cpp * nc;
      je = jb + cpp * nc < n ? jb + cpp * nc : n;
      if (jb >= je) continue;                         // the same in the whole block
      const long sys = list[1 + s / parts];
      c = (int)(sys / ((long)nb * N));
      const int rem = (int)(sys - (long)c * nb * N);
      a = rem / N;
      q = rem - a * N;
    } else {
      c = ch0 + (int)(s / ((long)na * N));
      const int rem = (int)(s - (long)(c - ch0) * na * N);
      a = dm.a0 + rem / N;
      q = rem - (a - dm.a0) * N;
    }
    bse_f64_system(dm, c, a, q, nc, gam, gg, chi, kc, LU, sm + L.y, sm + L.xs, sm + L.invu, sh, flags, radius_K,
                   lam, jb, je);
  }
}

// The ladder term of the susceptibilities (section "Resulting observables"):
// for one (q, W, channel), sum_{w,w'} L_w Gamma_{w,w'} L_w' with
// Gamma = D^-1 gamma (Eq. lin_alg_inv) = L . x, D x = gamma L, D in LU
// (bse_f64_factor, FP64); out = chi0 + L . x.  Y holds [n][2]: the permuted
// right-hand side, then L.
__device__ __forceinline__ void chi_ladder_system(const Dims& dm, int c, int a, int q,
                                                  const double2* __restrict__ gam, const double2* __restrict__ chi,
                                                  const double2* __restrict__ Lb, const double2* __restrict__ chi0,
                                                  double2* __restrict__ out, double2* LU, double2* Y, double2* xs,
                                                  double2* invu, BseF64Shared& sh, int* __restrict__ flags) {
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double2* G = gam + ((size_t)c * nb + a) * n * n;
  double2* y = Y;
  double2* lv = Y + n;
  bse_f64_factor(dm, c, a, q, gam, chi, LU, xs, invu, sh, flags);
  for (int i = tid; i < n; i += blockDim.x) lv[i] = Lb[((size_t)a * n + i) * N + q];
  __syncthreads();
  for (int r = tid; r < n; r += blockDim.x) {      // y = P (gamma L)
    const double2* gr = G + (size_t)sh.perm[r] * n;
    double2 b = mk(0.0, 0.0);
    for (int j = 0; j < n; ++j) b = cfma(gr[j], lv[j], b);
    y[r] = b;
  }
  __syncthreads();
  if (warp == 0) {
    for (int k = 0; k < n - 1; ++k) {              // unit-lower forward substitution
      const double2 yk = y[k];
      for (int r = k + 1 + lane; r < n; r += 32) y[r] = cfms(LU[r * n + k], yk, y[r]);
      __syncwarp();
    }
    for (int k = n - 1; k > 0; --k) {              // unit-upper back substitution (V = U diag(1/U_kk))
      const double2 yk = y[k];
      for (int r = lane; r < k; r += 32) y[r] = cfms(LU[r * n + k], yk, y[r]);
      __syncwarp();
    }
    double2 s2 = mk(0.0, 0.0);                     // L . x, x = y / U_kk
    for (int i = lane; i < n; i += 32) s2 = cfma(lv[i], cmul(y[i], invu[i]), s2);
    for (int o = 16; o > 0; o >>= 1) {
      s2.x += __shfl_xor_sync(0xffffffffu, s2.x, o);
      s2.y += __shfl_xor_sync(0xffffffffu, s2.y, o);
    }
    if (lane == 0) {
      const double2 c0 = chi0[(size_t)a * N + q];
      out[((size_t)c * nb + a) * N + q] = mk(c0.x + s2.x, c0.y + s2.y);
    }
  }
  __syncthreads();
}

// All 2 nb N systems, or with `list` non-null the list[0] systems whose
// indices follow it (the ones the refinement kernel below handed back).
template <bool LU_SMEM>
__global__ void __launch_bounds__(kBseThreads)
chi_ladder_kernel(Dims dm, const double2* __restrict__ gam, const double2* __restrict__ chi,
                  const double2* __restrict__ Lb, const double2* __restrict__ chi0, double2* __restrict__ out,
                  double2* __restrict__ ws, int* __restrict__ flags, const int* __restrict__ list) {
  extern __shared__ double2 sm[];
  __shared__ BseF64Shared sh;
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  const BseSmem L = bse_layout(n, 2, LU_SMEM);
  double2* LU = LU_SMEM ? sm + L.lu : ws + (size_t)blockIdx.x * n * n;
  const long systems = list ? (long)list[0] : 2L * nb * N;
  for (long s = blockIdx.x; s < systems; s += gridDim.x) {
    const long sys = list ? (long)list[1 + s] : s;
    const int c = (int)(sys / ((long)nb * N));
    const int rem = (int)(sys - (long)c * nb * N);
    const int a = rem / N, q = rem - a * N;
    chi_ladder_system(dm, c, a, q, gam, chi, Lb, chi0, out, LU, sm + L.y, sm + L.xs, sm + L.invu, sh, flags);
  }
}

// ---------------------------------------------------------------------------
// The same ladder term under DF_FP32_IR (n_w <= 64): x = D^-1 gamma L by
// mixed-precision iterative refinement.  D = 1 - gamma_W diag(chi~_W(q)) is
// factorised once in FP32 (complex64 in shared memory, row stride n + 1,
// partial pivoting on |re| + |im|); then, from x = 0 and r = gamma L,
//     D d = r / |r|   (the FP32 factors),   x += |r| d,   r = gamma L - D x
// with x, r and the products gamma v in FP64 (D x = x - gamma (chi~ o x)).
// Each step shrinks the error by about cond(D) 2^-24.  A system stops when
// its correction d is below ir_tol |x| (max norms of |re| + |im|), or when
// d times its ratio to the previous correction is (the error left after a
// contracting step); it is handed back to the FP64 LU kernel (appended to
// `redo`, count in redo[0], output not written here) on an exactly zero FP32
// pivot, a non-finite value, a correction that did not halve, or after
// max_steps solves.  128 threads: all of them run the rank-1 updates (one
// column each, rows split in 128 / n groups; the owners of the next column
// leave per-group pivot candidates, so that a column step takes two
// barriers) and the FP64 row products (128 / n rounded down to a power of
// two lanes per row; those of gamma L interleaved with the column steps);
// warp 0 runs the FP32 triangular solves (two rows per lane in registers).
// ---------------------------------------------------------------------------
constexpr int kChiIrThreads = 128;
constexpr int kChiIrMaxN = 64;

struct ChiIrShared {
  int perm[kChiIrMaxN];
  double2 xs[kChiIrMaxN], lv[kChiIrMaxN], b[kChiIrMaxN], x[kChiIrMaxN], v[kChiIrMaxN], r[kChiIrMaxN];
  float2 invd[kChiIrMaxN];
  // per row group: the largest |re| + |im| of the next pivot column among the
  // group's rows, its row (n when the group has none) and its value
  float pabs[kChiIrThreads];
  int prow[kChiIrThreads];
  float2 pval[kChiIrThreads];
  int bad, state;
};

// sum_j gamma_ij v_j for row i by `tpr` adjacent lanes (lane part of them
// takes j = part mod tpr); every lane of the warp must call it, rows i >= n
// contribute nothing.  The sum is complete in every lane of the group.
__device__ __forceinline__ double2 chi_ir_rowdot(const double2* __restrict__ G, const double2* v, int n, int i,
                                                 int part, int tpr) {
  double2 s0 = mk(0.0, 0.0), s1 = mk(0.0, 0.0);
  if (i < n) {
    const double2* g = G + (size_t)i * n;
    int j = part;
    for (; j + tpr < n; j += 2 * tpr) {
      s0 = cfma(__ldg(g + j), v[j], s0);
      s1 = cfma(__ldg(g + j + tpr), v[j + tpr], s1);
    }
    if (j < n) s0 = cfma(__ldg(g + j), v[j], s0);
  }
  s0 = s0 + s1;
  for (int o = tpr >> 1; o > 0; o >>= 1) {
    s0.x += __shfl_xor_sync(0xffffffffu, s0.x, o);
    s0.y += __shfl_xor_sync(0xffffffffu, s0.y, o);
  }
  return s0;
}

// 1/z in FP32 for the FP32 factorisation (a reciprocal of |z|^2: outside
// ~1e-19 < |z| < 1e19 it gives 0 or non-finite values, and the system is
// handed back by the refinement's checks)
__device__ __forceinline__ float2 cinv_f32(float2 z) {
  const float d = __frcp_rn(z.x * z.x + z.y * z.y);
  return make_float2(z.x * d, -z.y * d);
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(kChiIrThreads, 5)
chi_ladder_ir_kernel(Dims dm, const double2* __restrict__ gam, const float2* __restrict__ gam32,
                     const double2* __restrict__ chi, const double2* __restrict__ Lb,
                     const double2* __restrict__ chi0, double2* __restrict__ out, int* __restrict__ redo,
                     int max_steps, double tol) {
  extern __shared__ float2 A[];        // [n][n + 1]
  __shared__ ChiIrShared sh;
  const int n = dm.n_w, N = dm.N, nb = dm.nb, ld = n + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // rank-1 update / build map: column j, row group i0 of rpp
  const int rpp = kChiIrThreads / n, j = tid % n, i0 = tid / n;
  // row-product map: tpr lanes per row
  int tpr = 1;
  while (tpr < 32 && 2 * tpr * n <= kChiIrThreads) tpr *= 2;
  const int ri = tid / tpr, rpart = tid % tpr;
  const long systems = 2L * nb * N;
  for (long sys = blockIdx.x; sys < systems; sys += gridDim.x) {
    const int c = (int)(sys / ((long)nb * N));
    const int rem = (int)(sys - (long)c * nb * N);
    const int a = rem / N, q = rem - a * N;
    const double2* G = gam + ((size_t)c * nb + a) * n * n;
    const float2* G32 = gam32 + ((size_t)c * nb + a) * n * n;
    for (int i = tid; i < n; i += kChiIrThreads) {
      sh.xs[i] = chi[((size_t)a * n + i) * N + q];
      sh.lv[i] = Lb[((size_t)a * n + i) * N + q];
      sh.perm[i] = i;
    }
    if (tid == 0) sh.bad = 0;
    __syncthreads();
    // D in FP32 from gamma's leading FP32 words and FP32-rounded chi~ (only
    // the factorisation uses it; the residuals take D from FP64 gamma); the
    // threads of column 0 leave their row group's pivot candidate
    if (i0 < rpp) {
      const float2 xj = make_float2((float)sh.xs[j].x, (float)sh.xs[j].y);
      float best = -1.f;
      int brow = n;
      float2 bval = make_float2(0.f, 0.f);
      for (int i = i0; i < n; i += rpp) {
        float2 t = cmul(__ldg(G32 + (size_t)i * n + j), xj);
        t = make_float2((i == j ? 1.f : 0.f) - t.x, -t.y);
        A[i * ld + j] = t;
        if (j == 0 && cabs1(t) > best) { best = cabs1(t); brow = i; bval = t; }
      }
      if (j == 0) { sh.pabs[i0] = best; sh.prow[i0] = brow; sh.pval[i0] = bval; }
    }
    __syncthreads();
    // ---- FP32 LU with partial pivoting, two barriers per column; the FP64
    // row products b = gamma L run alongside, one term per column step, their
    // loads issued a step ahead ----
    double2 bacc = mk(0.0, 0.0), gnext = mk(0.0, 0.0);
    if (ri < n && rpart < n) gnext = __ldg(G + (size_t)ri * n + rpart);
    int npart = rpp < n ? rpp : n;         // row groups holding pivot candidates
    for (int k = 0; k < n; ++k) {
      // the pivot of column k from the row groups' candidates (every thread
      // takes the same one: largest, then lowest row)
      float best = -1.f;
      int p = n;
      float2 pv = make_float2(0.f, 0.f);
      for (int g = 0; g < npart; ++g) {
        const float v = sh.pabs[g];
        const int rr = sh.prow[g];
        if (v > best || (v == best && rr < p)) { best = v; p = rr; pv = sh.pval[g]; }
      }
      if (p >= n) { p = k; pv = make_float2(0.f, 0.f); }   // no candidate (NaN column): a zero pivot
      const bool zero = (pv.x == 0.f && pv.y == 0.f);
      const float2 inv = zero ? make_float2(0.f, 0.f) : cinv_f32(pv);
      if (tid == 0) {
        if (zero) sh.bad = 1;
        sh.invd[k] = inv;
        if (p != k) { const int t = sh.perm[k]; sh.perm[k] = sh.perm[p]; sh.perm[p] = t; }
      }
      // rows k and p exchanged (column k: the pivot on the diagonal, the old
      // A_kk scaled into row p), the other multipliers of column k scaled
      if (p != k && tid < n) {
        if (tid == k) {
          const float2 okk = A[k * ld + k];
          A[k * ld + k] = pv;
          A[p * ld + k] = cmul(okk, inv);
        } else {
          const float2 t = A[k * ld + tid];
          A[k * ld + tid] = A[p * ld + tid];
          A[p * ld + tid] = t;
        }
      }
      if (tid > k && tid < n && tid != p) A[tid * ld + k] = cmul(A[tid * ld + k], inv);
      __syncthreads();
      // rank-1 update of the trailing m x m block, spread over all threads:
      // thread = g m + jc takes column k + 1 + jc, rows k + 1 + g + ng t with
      // ng = floor(128 / m) groups (the quotients in FP32: exact here, every
      // true quotient is at least 0.5 / m from an integer); the threads of
      // column k + 1 leave the next pivot candidates
      const int m = n - k - 1;
      if (m > 0) {
        const float rcp = __frcp_rn((float)m);
        const int ng = __float2int_rz(128.f * rcp + 0.5f * rcp);
        const int g = __float2int_rz(((float)tid + 0.5f) * rcp);
        npart = ng < m ? ng : m;
        if (g < ng) {
          const int jcol = k + 1 + (tid - g * m);
          const bool cand = (jcol == k + 1);
          const float2 u = A[k * ld + jcol];
          float bb = -1.f;
          int br = n;
          float2 bv = make_float2(0.f, 0.f);
          int r = k + 1 + g;
          // rows in batches of four, all loads of a batch before its stores
          // (the compiler cannot order them otherwise: columns k and jcol share A)
          for (; r + 3 * ng < n; r += 4 * ng) {
            float2 l[4], t[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              l[e] = A[(r + e * ng) * ld + k];
              t[e] = A[(r + e * ng) * ld + jcol];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              t[e] = cfms(l[e], u, t[e]);
              A[(r + e * ng) * ld + jcol] = t[e];
            }
            if (cand) {
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (cabs1(t[e]) > bb) { bb = cabs1(t[e]); br = r + e * ng; bv = t[e]; }
            }
          }
          for (; r < n; r += ng) {
            const float2 t = cfms(A[r * ld + k], u, A[r * ld + jcol]);
            A[r * ld + jcol] = t;
            if (cand && cabs1(t) > bb) { bb = cabs1(t); br = r; bv = t; }
          }
          if (cand && g < m) {
            sh.pabs[g] = bb;
            sh.prow[g] = br;
            sh.pval[g] = bv;
          }
        }
      }
      {
        const int jj = rpart + tpr * k;
        if (ri < n && jj < n) {
          const double2 gv = gnext;
          if (jj + tpr < n) gnext = __ldg(G + (size_t)ri * n + jj + tpr);
          bacc = cfma(gv, sh.lv[jj], bacc);
        }
      }
      __syncthreads();
    }
    for (int o = tpr >> 1; o > 0; o >>= 1) {
      bacc.x += __shfl_xor_sync(0xffffffffu, bacc.x, o);
      bacc.y += __shfl_xor_sync(0xffffffffu, bacc.y, o);
    }
    if (rpart == 0 && ri < n) {
      sh.b[ri] = bacc;
      sh.r[ri] = bacc;
      sh.x[ri] = mk(0.0, 0.0);
    }
    __syncthreads();
    // ---- refinement: state 0 going on, 1 converged, 2 handed back; every
    // thread reads the state right after the barrier that follows its write,
    // and warp 0 writes it again only after the next barrier ----
    int state = sh.bad ? 2 : 0;
    double dprev = 0.0;
    for (int it = 0; state == 0; ++it) {
      if (warp == 0) {
        const bool h0 = lane < n, h1 = lane + 32 < n;
        double rm = fmax(h0 ? cabs1(sh.r[sh.perm[lane]]) : 0.0, h1 ? cabs1(sh.r[sh.perm[lane + 32]]) : 0.0);
        rm = warp_max(rm);
        const double sc = rm > 0.0 ? 1.0 / rm : 0.0;
        float2 y0 = make_float2(0.f, 0.f), y1 = y0;
        if (h0) { const double2 t = sh.r[sh.perm[lane]]; y0 = make_float2((float)(t.x * sc), (float)(t.y * sc)); }
        if (h1) { const double2 t = sh.r[sh.perm[lane + 32]]; y1 = make_float2((float)(t.x * sc), (float)(t.y * sc)); }
        for (int k = 0; k < n - 1; ++k) {          // unit-lower forward substitution
          const float2 src = k < 32 ? y0 : y1;
          const float2 yk = make_float2(__shfl_sync(0xffffffffu, src.x, k & 31), __shfl_sync(0xffffffffu, src.y, k & 31));
          if (lane > k && h0) y0 = cfms(A[lane * ld + k], yk, y0);
          if (lane + 32 > k && h1) y1 = cfms(A[(lane + 32) * ld + k], yk, y1);
        }
        for (int k = n - 1; k >= 0; --k) {         // upper back substitution
          const float2 src = k < 32 ? y0 : y1;
          const float2 yk = make_float2(__shfl_sync(0xffffffffu, src.x, k & 31), __shfl_sync(0xffffffffu, src.y, k & 31));
          const float2 xk = cmul(yk, sh.invd[k]);
          if (lane == k) y0 = xk;
          if (lane + 32 == k) y1 = xk;
          if (lane < k) y0 = cfms(A[lane * ld + k], xk, y0);
          if (lane + 32 < k) y1 = cfms(A[(lane + 32) * ld + k], xk, y1);
        }
        double dn = 0.0, xn = 0.0;
        if (h0) {
          const double2 d = mk((double)y0.x * rm, (double)y0.y * rm);
          const double2 xv = sh.x[lane] + d;
          sh.x[lane] = xv;
          sh.v[lane] = cmul(sh.xs[lane], xv);
          dn = cabs1(d);
          xn = cabs1(xv);
        }
        if (h1) {
          const double2 d = mk((double)y1.x * rm, (double)y1.y * rm);
          const double2 xv = sh.x[lane + 32] + d;
          sh.x[lane + 32] = xv;
          sh.v[lane + 32] = cmul(sh.xs[lane + 32], xv);
          dn = fmax(dn, cabs1(d));
          xn = fmax(xn, cabs1(xv));
        }
        // NaN compares false: a non-finite value hands the system back
        dn = warp_max(isfinite(dn) ? dn : INFINITY);
        xn = warp_max(isfinite(xn) ? xn : INFINITY);
        int st = 0;
        if (!(dn < INFINITY) || !(xn < INFINITY)) st = 2;
        else if (dn <= tol * xn) st = 1;
        else if (it > 0 && dn > 0.5 * dprev) st = 2;
        else if (it > 0 && dn * dn <= 0.5 * tol * xn * dprev) st = 1;
        else if (it + 1 >= max_steps) st = 2;
        dprev = dn;
        if (st == 1) {                              // out = chi0 + L . x
          double2 s2 = mk(0.0, 0.0);
          if (h0) s2 = cfma(sh.lv[lane], sh.x[lane], s2);
          if (h1) s2 = cfma(sh.lv[lane + 32], sh.x[lane + 32], s2);
          for (int o = 16; o > 0; o >>= 1) {
            s2.x += __shfl_xor_sync(0xffffffffu, s2.x, o);
            s2.y += __shfl_xor_sync(0xffffffffu, s2.y, o);
          }
          if (lane == 0) {
            const double2 c0 = chi0[(size_t)a * N + q];
            out[((size_t)c * nb + a) * N + q] = mk(c0.x + s2.x, c0.y + s2.y);
          }
        }
        if (lane == 0) sh.state = st;
      }
      __syncthreads();
      state = sh.state;
      if (state != 0) break;
      {   // r = gamma L - x + gamma (chi~ o x)
        const double2 s = chi_ir_rowdot(G, sh.v, n, ri, rpart, tpr);
        if (rpart == 0 && ri < n) sh.r[ri] = sh.b[ri] - sh.x[ri] + s;
      }
      __syncthreads();
    }
    if (tid == 0 && state == 2) {
      const int slot = atomicAdd(redo, 1);
      redo[1 + slot] = (int)sys;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// leading eigenvalue of A = gamma_W diag(chi~_W(q)): power iteration with a
// Rayleigh-quotient estimate, first in FP32 (gamma staged in shared memory
// as complex64) until the estimate settles to FP32 precision, then polished
// from that vector with FP64 vectors and Rayleigh quotients, the products
// gamma (chi~ o v) in double-float FP32 (gamma staged as (hi, lo) pairs;
// ~2^-46 relative, far below the 1e-12 stopping tolerance).  The reported
// value and its converged flag are those of the polish.  The polish runs only
// for the systems whose FP32 phase settled: one that still changes by more
// than 2e-6 per step after 64 steps converges at a geometric rate above 0.81,
// so 24 more steps cannot reach 1e-12; it reports its FP32 estimate, flagged
// not converged (a block whose systems all are skips the polish).  One CTA handles
// kEigQ systems that share (channel, W); each thread owns (row, system)
// pairs of y = A v.
// ---------------------------------------------------------------------------
constexpr int kEigQ = 8;
constexpr int kEigThreads = 1024;   // one (row, system) pair per thread up to n_w = 128
constexpr int kEigIter32 = 64;
constexpr int kEigIter64 = 24;

template <typename C, typename R>
__device__ __forceinline__ void eig_rayleigh(int n, int warp, int lane, const C* v, const C* y, C* lam_new, R* nrm) {
  if (warp < kEigQ) {
    const int t = warp;
    C rq = mk((R)0, (R)0);
    R yy = 0;
    for (int j = lane; j < n; j += 32) {
      const C vj = v[j * kEigQ + t], yj = y[j * kEigQ + t];
      rq = cfma(cconj(vj), yj, rq);
      yy += cabs2(yj);
    }
    for (int o = 16; o > 0; o >>= 1) {
      rq.x += __shfl_xor_sync(0xffffffffu, rq.x, o);
      rq.y += __shfl_xor_sync(0xffffffffu, rq.y, o);
      yy += __shfl_xor_sync(0xffffffffu, yy, o);
    }
    if (lane == 0) {
      lam_new[t] = rq;
      nrm[t] = yy > (R)0 ? (R)1 / sqrt(yy) : (R)0;
    }
  }
}

__global__ void __launch_bounds__(kEigThreads)
lambda_kernel(Dims dm, int ch0, int a0, int na, int lo_in_smem, double tol, const double2* __restrict__ gam,
              const double2* __restrict__ chi, double2* __restrict__ lam, int* __restrict__ ok,
              int* __restrict__ flags) {
  extern __shared__ double2 sm[];
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  double2* v = sm;                       // [n][kEigQ]
  double2* xq = v + n * kEigQ;
  double2* y = xq + n * kEigQ;
  float2* G32 = (float2*)(y + n * kEigQ);  // [n][n]
  float2* G32l = G32 + n * n;              // [n][n], gamma - G32 (when it fits; else formed on the fly)
  float2* v32 = G32l + (lo_in_smem ? n * n : 0);
  float2* x32 = v32 + n * kEigQ;
  float2* y32 = x32 + n * kEigQ;
  __shared__ double2 lam_old[kEigQ], lam_new[kEigQ];
  __shared__ float2 l32_old[kEigQ], l32_new[kEigQ];
  __shared__ double nrm[kEigQ];
  __shared__ float nrm32[kEigQ];
  __shared__ int done[kEigQ];
  __shared__ int conv[kEigQ];            // FP32 phase converged (the polish runs for these only)
  const int qtiles = (N + kEigQ - 1) / kEigQ;
  const int tile = blockIdx.x % qtiles;
  const int a = a0 + (blockIdx.x / qtiles) % na;
  const int c = ch0 + blockIdx.x / (qtiles * na);
  const int q0 = tile * kEigQ;
  const int nq = min(kEigQ, N - q0);
  const double2* Gg = gam + ((size_t)c * nb + a) * n * n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const double2 g = Gg[idx];
    const float hx = (float)g.x, hy = (float)g.y;
    G32[idx] = make_float2(hx, hy);
    if (lo_in_smem) G32l[idx] = make_float2((float)(g.x - (double)hx), (float)(g.y - (double)hy));
  }
  for (int idx = tid; idx < n * kEigQ; idx += blockDim.x) {
    const int j = idx / kEigQ, t = idx % kEigQ;
    const double2 x = (t < nq) ? chi[((size_t)a * n + j) * N + q0 + t] : mk(0.0, 0.0);
    xq[idx] = x;
    x32[idx] = make_float2((float)x.x, (float)x.y);
    v32[idx] = make_float2(rsqrtf((float)n), 0.f);
  }
  if (tid < kEigQ) {
    l32_old[tid] = make_float2(0.f, 0.f);
    l32_new[tid] = make_float2(0.f, 0.f);
    lam_old[tid] = mk(0.0, 0.0);
    lam_new[tid] = mk(0.0, 0.0);
    done[tid] = (tid < nq) ? 0 : 1;
  }
  __syncthreads();
  // ---- FP32 phase ----
  for (int it = 0; it < kEigIter32; ++it) {
    for (int p = tid; p < n * kEigQ; p += blockDim.x) {
      const int i = p / kEigQ, t = p % kEigQ;
      float2 acc = make_float2(0.f, 0.f);
      for (int j = 0; j < n; ++j) acc = cfma(G32[i * n + j], cmul(x32[j * kEigQ + t], v32[j * kEigQ + t]), acc);
      y32[p] = acc;
    }
    __syncthreads();
    eig_rayleigh<float2, float>(n, warp, lane, v32, y32, l32_new, nrm32);
    __syncthreads();
    for (int idx = tid; idx < n * kEigQ; idx += blockDim.x) v32[idx] = cscale(y32[idx], nrm32[idx % kEigQ]);
    if (tid < kEigQ && !done[tid]) {
      const float2 d = l32_new[tid] - l32_old[tid];
      if (sqrtf(cabs2(d)) <= 2e-6f * sqrtf(cabs2(l32_new[tid]))) done[tid] = 1;
      l32_old[tid] = l32_new[tid];
    }
    __syncthreads();
    int all = 1;
#pragma unroll
    for (int t = 0; t < kEigQ; ++t) all &= done[t];
    if (all) break;
  }
  // ---- FP64 polish from the FP32 vector ----
  for (int idx = tid; idx < n * kEigQ; idx += blockDim.x) v[idx] = mk((double)v32[idx].x, (double)v32[idx].y);
  // a system whose FP32 phase did not settle keeps its FP32 estimate (not converged)
  if (tid < kEigQ) {
    conv[tid] = tid < nq && done[tid];
    done[tid] = conv[tid] ? 0 : 1;
  }
  __syncthreads();
  int any = 0;
#pragma unroll
  for (int t = 0; t < kEigQ; ++t) any |= conv[t];
  float2* wh = x32;                        // chi~ o v as (hi, lo) pairs; x32, y32 are free now
  float2* wl = y32;
  for (int it = 0; it < (any ? kEigIter64 : 0); ++it) {
    for (int idx = tid; idx < n * kEigQ; idx += blockDim.x) {
      const double2 w = cmul(xq[idx], v[idx]);
      const float hx = (float)w.x, hy = (float)w.y;
      wh[idx] = make_float2(hx, hy);
      wl[idx] = make_float2((float)(w.x - (double)hx), (float)(w.y - (double)hy));
    }
    __syncthreads();
    for (int p = tid; p < n * kEigQ; p += blockDim.x) {
      const int i = p / kEigQ, t = p % kEigQ;
      float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
      for (int j = 0; j < n; ++j) {
        const float2 gh = G32[i * n + j];
        float2 gl;
        if (lo_in_smem) {
          gl = G32l[i * n + j];
        } else {
          const double2 g = Gg[(size_t)i * n + j];
          gl = make_float2((float)(g.x - (double)gh.x), (float)(g.y - (double)gh.y));
        }
        cdf_fma(sr, lr, si, li, gh, gl, wh[j * kEigQ + t], wl[j * kEigQ + t]);
      }
      y[p] = mk((double)sr + (double)lr, (double)si + (double)li);
    }
    __syncthreads();
    eig_rayleigh<double2, double>(n, warp, lane, v, y, lam_new, nrm);
    __syncthreads();
    for (int idx = tid; idx < n * kEigQ; idx += blockDim.x) v[idx] = cscale(y[idx], nrm[idx % kEigQ]);
    if (tid < kEigQ && !done[tid]) {
      const double2 d = lam_new[tid] - lam_old[tid];
      if (it > 0 && sqrt(cabs2(d)) <= tol * sqrt(cabs2(lam_new[tid]))) done[tid] = 1;
      lam_old[tid] = lam_new[tid];
    }
    __syncthreads();
    int all = 1;
#pragma unroll
    for (int t = 0; t < kEigQ; ++t) all &= done[t];
    if (all) break;
  }
  if (tid < nq) {
    const size_t o = ((size_t)c * nb + a) * N + q0 + tid;
    const double2 l = conv[tid] ? lam_new[tid] : mk((double)l32_new[tid].x, (double)l32_new[tid].y);
    lam[o] = l;
    ok[o] = conv[tid] && done[tid];
    if (cabs2(l) >= 1.0) atomicOr(flags, 2);
  }
}

// The same power iteration and polish for n_w <= 64 with gamma in registers:
// thread (i, jb) = (tid / 4, tid % 4) holds row i, columns 16 jb .. 16 jb + 15
// of gamma's hi parts (the lo parts, polish only, in shared memory as
// [jb][k][i]), reads u = chi~ o v (all kEigQ systems) as broadcast 16-byte
// loads, and the four column blocks of a row (consecutive lanes) are summed
// by shuffles.  Thread (i, jb) owns systems 2 jb, 2 jb + 1 of row i.  The
// polish keeps its vectors in double-float (FP32 pairs: the FP64 pipe is
// slow); only the per-system scalars (Rayleigh quotient, norm, stopping test)
// are FP64, in 8 threads.  Same stopping rules and outputs as lambda_kernel.
constexpr int kEigRegN = 64;                      // largest n_w of this kernel
constexpr int kEigUStride = 16 * kEigQ + 2;       // u block stride (float2): the 4 column blocks in distinct banks
constexpr int kEigLoStride = 16 * kEigRegN + 8;   // gamma-lo block stride (float2): a warp's 4 blocks in 2 wavefronts

// y = gamma u for the kEigQ systems (FP32, this thread's 16 columns), then
// summed over the 4 column blocks of the row (consecutive lanes)
__device__ __forceinline__ void eig_gemv32(const float2 (&gh)[16], const float2* __restrict__ ub2,
                                           float2 (&y)[kEigQ]) {
#pragma unroll
  for (int t = 0; t < kEigQ; ++t) y[t] = make_float2(0.f, 0.f);
  const float4* ub = reinterpret_cast<const float4*>(ub2);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
#pragma unroll
    for (int tp = 0; tp < kEigQ / 2; ++tp) {
      const float4 q = ub[(k * kEigQ) / 2 + tp];
      y[2 * tp] = cfma(gh[k], make_float2(q.x, q.y), y[2 * tp]);
      y[2 * tp + 1] = cfma(gh[k], make_float2(q.z, q.w), y[2 * tp + 1]);
    }
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1)
#pragma unroll
    for (int t = 0; t < kEigQ; ++t) {
      y[t].x += __shfl_xor_sync(0xffffffffu, y[t].x, o);
      y[t].y += __shfl_xor_sync(0xffffffffu, y[t].y, o);
    }
}

template <typename T, int M>
__device__ __forceinline__ T pick2(const T (&a)[M], int jb, int k) {   // a[2 jb + k], jb < 4
  T r = a[k];
#pragma unroll
  for (int q = 1; q < 4; ++q)
    if (q == jb) r = a[2 * q + k];
  return r;
}

// (hi, lo) * s for a double-float real s = (sh, sl): leading product exact
__device__ __forceinline__ void df_scale(float& hi, float& lo, float sh, float sl) {
  const float p = hi * sh;
  const float e = fmaf(hi, sh, -p);
  const float l = fmaf(hi, sl, fmaf(lo, sh, e));
  hi = p + l;
  lo = l - (hi - p);
}

__global__ void __launch_bounds__(256, 2)
lambda_reg_kernel(Dims dm, int ch0, int a0, int na, double tol, const double2* __restrict__ gam,
                  const double2* __restrict__ chi, double2* __restrict__ lam, int* __restrict__ ok,
                  int* __restrict__ flags) {
  static_assert(kEigQ == 8, "two systems per thread of a row");
  extern __shared__ float2 glo[];                // [4][16][kEigRegN], block stride kEigLoStride
  __shared__ __align__(16) float2 uh[4 * kEigUStride], ul[4 * kEigUStride];
  __shared__ float2 xh[kEigRegN][kEigQ], xl[kEigRegN][kEigQ];   // chi~ as (hi, lo) pairs
  __shared__ float redf[8][kEigQ][7];            // per warp: FP32 phase: u^H y, |y|^2, u_prev^H y, u_prev^H u;
                                                 // polish: u^H y and |y|^2 as df pairs
  __shared__ float2 pair_s[kEigQ][2];            // FP32 phase: the dominant pair's two estimates
  __shared__ float cprev_s[kEigQ];               // FP32 phase: |A u_prev|
  __shared__ int pconv_s[kEigQ];                 // FP32 phase: the pair estimate settled
  __shared__ int phave_s[kEigQ];                 // FP32 phase: pair_s holds an accepted estimate
  __shared__ float2 scal[kEigQ];                 // per system: 1 / |y| as a double-float (hi, lo)
  __shared__ double2 lold_s[kEigQ];              // previous (current, at the end) Rayleigh quotients
  __shared__ int done_s[kEigQ];
  __shared__ int conv_s[kEigQ];                  // FP32 phase converged (the polish runs for these only)
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  const int qtiles = (N + kEigQ - 1) / kEigQ;
  const int tile = blockIdx.x % qtiles;
  const int a = a0 + (blockIdx.x / qtiles) % na;
  const int c = ch0 + blockIdx.x / (qtiles * na);
  const int q0 = tile * kEigQ;
  const int nq = min(kEigQ, N - q0);
  const double2* Gg = gam + ((size_t)c * nb + a) * n * n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i = tid >> 2, jb = tid & 3;
  const int uo = (i >> 4) * kEigUStride + (i & 15) * kEigQ + 2 * jb;   // this thread's u slot (row i, t = 2 jb)
  float2 gh[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int j = 16 * jb + k;
    const double2 g = (i < n && j < n) ? Gg[(size_t)i * n + j] : mk(0.0, 0.0);
    gh[k] = make_float2((float)g.x, (float)g.y);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int t = 2 * jb + k;
    const double2 x = (i < n && t < nq) ? chi[((size_t)a * n + i) * N + q0 + t] : mk(0.0, 0.0);
    const float2 h = make_float2((float)x.x, (float)x.y);
    xh[i][t] = h;
    xl[i][t] = make_float2((float)(x.x - (double)h.x), (float)(x.y - (double)h.y));
  }
  if (tid < kEigQ) {
    done_s[tid] = tid < nq ? 0 : 1;
    lold_s[tid] = mk(0.0, 0.0);
    pair_s[tid][0] = pair_s[tid][1] = make_float2(0.f, 0.f);
    cprev_s[tid] = 0.f;
    pconv_s[tid] = 0;
    phave_s[tid] = 0;
  }

  // ---- FP32 phase ----
  // Alongside the Rayleigh quotient, the span of the last two iterates gives
  // the dominant pair when two eigenvalues share the largest modulus (a
  // complex-conjugate pair, where one vector cannot settle): with u_k = A
  // u_{k-1} / c, fit A u_k ~ alpha u_k + beta u_{k-1} (least squares); on that
  // span A acts as [[0, beta], [c, alpha]], whose eigenvalues solve
  // l^2 - alpha l - beta c = 0.
  float2 v32[2], vprev[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  const float v0 = i < n ? rsqrtf((float)n) : 0.f;
  v32[0] = v32[1] = make_float2(v0, 0.f);
  for (int it = 0; it < kEigIter32; ++it) {
    {
      const float2 u0 = cmul(xh[i][2 * jb], v32[0]), u1 = cmul(xh[i][2 * jb + 1], v32[1]);
      *reinterpret_cast<float4*>(uh + uo) = make_float4(u0.x, u0.y, u1.x, u1.y);
    }
    __syncthreads();
    float2 y[kEigQ];
    eig_gemv32(gh, uh + jb * kEigUStride, y);
    float2 yo[2];
    float pt[2][7];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      yo[k] = pick2(y, jb, k);
      const float2 rq = cmul(cconj(v32[k]), yo[k]);
      const float2 g = cmul(cconj(vprev[k]), yo[k]);
      const float2 h = cmul(cconj(vprev[k]), v32[k]);
      pt[k][0] = rq.x;
      pt[k][1] = rq.y;
      pt[k][2] = cabs2(yo[k]);
      pt[k][3] = g.x;
      pt[k][4] = g.y;
      pt[k][5] = h.x;
      pt[k][6] = h.y;
#pragma unroll
      for (int m = 0; m < 7; ++m)
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) pt[k][m] += __shfl_xor_sync(0xffffffffu, pt[k][m], o);
    }
    if (lane < 4) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int m = 0; m < 7; ++m) redf[warp][2 * jb + k][m] = pt[k][m];
    }
    __syncthreads();
    if (tid < kEigQ) {
      float r[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int w = 0; w < 8; ++w)
#pragma unroll
        for (int m = 0; m < 7; ++m) r[m] += redf[w][tid][m];
      const float yy = r[2];
      scal[tid] = make_float2(yy > 0.f ? 1.f / sqrtf(yy) : 0.f, 0.f);
      const float2 ln = make_float2(r[0], r[1]);
      const float2 lo = make_float2((float)lold_s[tid].x, (float)lold_s[tid].y);
      if (!done_s[tid]) {
        const float2 d = ln - lo;
        if (sqrtf(cabs2(d)) <= 2e-6f * sqrtf(cabs2(ln))) done_s[tid] = 1;
      }
      lold_s[tid] = mk((double)ln.x, (double)ln.y);
      // the pair from span{u_prev, u}: Gram [[1, conj h], [h, 1]], right side
      // (u^H y, u_prev^H y).  For a pair the two iterates' overlap oscillates;
      // a fit counts only when the Gram matrix is well conditioned (det > 0.1:
      // FP32 rounding amplified <= 10x), and is compared with the previous
      // counted fit (settled: both roots within 1e-4); ill-conditioned steps
      // leave the estimate as it was
      const float c = cprev_s[tid];
      const float2 g = make_float2(r[3], r[4]), h = make_float2(r[5], r[6]);
      const float det = 1.f - cabs2(h);
      if (it > 0 && c > 0.f && det > 0.1f) {
        const float2 al = cscale(ln - cmul(cconj(h), g), 1.f / det);
        const float2 be = cscale(g - cmul(h, ln), 1.f / det);
        const float2 disc = cmul(al, al) + cscale(be, 4.f * c);
        const float dm = sqrtf(cabs2(disc));
        float2 sq = make_float2(sqrtf(fmaxf(0.5f * (dm + disc.x), 0.f)), sqrtf(fmaxf(0.5f * (dm - disc.x), 0.f)));
        if (disc.y < 0.f) sq.y = -sq.y;
        const float2 l1 = cscale(al + sq, 0.5f), l2 = cscale(al - sq, 0.5f);
        // match the new roots to the previous ones (their order may swap)
        const float2 o1 = pair_s[tid][0], o2 = pair_s[tid][1];
        const bool sw = cabs2(l1 - o2) + cabs2(l2 - o1) < cabs2(l1 - o1) + cabs2(l2 - o2);
        const float2 d1 = (sw ? l2 : l1) - o1, d2 = (sw ? l1 : l2) - o2;
        const float sc = fmaxf(sqrtf(cabs2(l1)), sqrtf(cabs2(l2)));
        pconv_s[tid] = phave_s[tid] && sqrtf(cabs2(d1)) <= 1e-4f * sc && sqrtf(cabs2(d2)) <= 1e-4f * sc;
        pair_s[tid][0] = l1;
        pair_s[tid][1] = l2;
        phave_s[tid] = 1;
      }
      cprev_s[tid] = sqrtf(yy);
    }
    __syncthreads();
    int all = 1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      vprev[k] = v32[k];
      v32[k] = cscale(yo[k], scal[2 * jb + k].x);
    }
#pragma unroll
    for (int t = 0; t < kEigQ; ++t) all &= done_s[t];   // the pair is for systems that never settle
    if (all) break;
  }
  // ---- double-float polish from the FP32 vector ----
  float2* glt = glo + jb * kEigLoStride + i;     // this thread's lo parts, stride kEigRegN
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int j = 16 * jb + k;
    const double2 g = (i < n && j < n) ? Gg[(size_t)i * n + j] : mk(0.0, 0.0);
    glt[k * kEigRegN] = make_float2((float)(g.x - (double)gh[k].x), (float)(g.y - (double)gh[k].y));
  }
  float2 vh[2] = {v32[0], v32[1]}, vl[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  __syncthreads();
  // a system whose FP32 phase did not settle keeps its FP32 estimate (not converged)
  if (tid < kEigQ) {
    conv_s[tid] = tid < nq && done_s[tid];
    done_s[tid] = conv_s[tid] ? 0 : 1;
    if (conv_s[tid]) lold_s[tid] = mk(0.0, 0.0);
  }
  __syncthreads();
  int any = 0;
#pragma unroll
  for (int t = 0; t < kEigQ; ++t) any |= conv_s[t];
  for (int it = 0; it < (any ? kEigIter64 : 0); ++it) {
    {
      // w = chi~ o v in double-float
      float4 wh4, wl4;
      float* whp = &wh4.x;
      float* wlp = &wl4.x;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
        cdf_fma(sr, lr, si, li, xh[i][2 * jb + k], xl[i][2 * jb + k], vh[k], vl[k]);
        whp[2 * k] = sr + lr;
        wlp[2 * k] = lr - (whp[2 * k] - sr);
        whp[2 * k + 1] = si + li;
        wlp[2 * k + 1] = li - (whp[2 * k + 1] - si);
      }
      *reinterpret_cast<float4*>(uh + uo) = wh4;
      *reinterpret_cast<float4*>(ul + uo) = wl4;
    }
    __syncthreads();
    // y = gamma w in double-float, two systems at a time (register pressure);
    // systems 2 h2, 2 h2 + 1 belong to the threads with jb == h2
    float ys[2][4];                                   // this thread's two systems: sr, lr, si, li
#pragma unroll
    for (int h2 = 0; h2 < 4; ++h2) {
      float sr[2], lr[2], si[2], li[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) sr[t] = lr[t] = si[t] = li[t] = 0.f;
      const float4* bh = reinterpret_cast<const float4*>(uh + jb * kEigUStride) + h2;
      const float4* bl = reinterpret_cast<const float4*>(ul + jb * kEigUStride) + h2;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 h = bh[(k * kEigQ) / 2], l = bl[(k * kEigQ) / 2];
        const float2 gk = glt[k * kEigRegN];
        cdf_fma(sr[0], lr[0], si[0], li[0], gh[k], gk, make_float2(h.x, h.y), make_float2(l.x, l.y));
        cdf_fma(sr[1], lr[1], si[1], li[1], gh[k], gk, make_float2(h.z, h.w), make_float2(l.z, l.w));
      }
#pragma unroll
      for (int o = 1; o < 4; o <<= 1)
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const float a1 = __shfl_xor_sync(0xffffffffu, sr[t], o), a2 = __shfl_xor_sync(0xffffffffu, lr[t], o);
          const float b1 = __shfl_xor_sync(0xffffffffu, si[t], o), b2 = __shfl_xor_sync(0xffffffffu, li[t], o);
          df_add(sr[t], lr[t], a1);
          lr[t] += a2;
          df_add(si[t], li[t], b1);
          li[t] += b2;
        }
      if (jb == h2) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          ys[k][0] = sr[k];
          ys[k][1] = lr[k];
          ys[k][2] = si[k];
          ys[k][3] = li[k];
        }
      }
    }
    // row sums of conj(v) y and |y|^2 in double-float
    float pt[2][6];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float2 yh = make_float2(ys[k][0], ys[k][2]), yl = make_float2(ys[k][1], ys[k][3]);
      float a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
      cdf_fma(a1, a2, a3, a4, cconj(vh[k]), cconj(vl[k]), yh, yl);
      float b1 = 0.f, b2 = 0.f, b3 = 0.f, b4 = 0.f;
      cdf_fma(b1, b2, b3, b4, cconj(yh), cconj(yl), yh, yl);
      pt[k][0] = a1; pt[k][1] = a2; pt[k][2] = a3; pt[k][3] = a4; pt[k][4] = b1; pt[k][5] = b2;
#pragma unroll
      for (int o = 4; o < 32; o <<= 1)
#pragma unroll
        for (int m = 0; m < 6; m += 2) {
          const float oh = __shfl_xor_sync(0xffffffffu, pt[k][m], o), ol = __shfl_xor_sync(0xffffffffu, pt[k][m + 1], o);
          df_add(pt[k][m], pt[k][m + 1], oh);
          pt[k][m + 1] += ol;
        }
    }
    if (lane < 4) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int m = 0; m < 6; ++m) redf[warp][2 * jb + k][m] = pt[k][m];
    }
    __syncthreads();
    if (tid < kEigQ) {
      double r[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int w = 0; w < 8; ++w)
#pragma unroll
        for (int m = 0; m < 3; ++m) r[m] += (double)redf[w][tid][2 * m] + (double)redf[w][tid][2 * m + 1];
      const double nrm = r[2] > 0.0 ? 1.0 / sqrt(r[2]) : 0.0;
      const float nh = (float)nrm;
      scal[tid] = make_float2(nh, (float)(nrm - (double)nh));
      const double2 ln = mk(r[0], r[1]);
      if (!done_s[tid]) {
        const double2 d = ln - lold_s[tid];
        if (it > 0 && sqrt(cabs2(d)) <= tol * sqrt(cabs2(ln))) done_s[tid] = 1;
        lold_s[tid] = ln;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float2 sc = scal[2 * jb + k];
      float a1 = ys[k][0], a2 = ys[k][1], a3 = ys[k][2], a4 = ys[k][3];
      df_scale(a1, a2, sc.x, sc.y);
      df_scale(a3, a4, sc.x, sc.y);
      vh[k] = make_float2(a1, a3);
      vl[k] = make_float2(a2, a4);
    }
    int all = 1;
#pragma unroll
    for (int t = 0; t < kEigQ; ++t) all &= done_s[t];
    if (all) break;
  }
  if (tid < nq) {
    const size_t o = ((size_t)c * nb + a) * N + q0 + tid;
    double2 l = lold_s[tid];
    int okv = conv_s[tid] && done_s[tid];
    if (!conv_s[tid] && pconv_s[tid]) {
      // a settled dominant pair: the root of larger modulus (of equal moduli,
      // the one with the larger imaginary part), to FP32 accuracy
      const float2 l1 = pair_s[tid][0], l2 = pair_s[tid][1];
      const float m1 = cabs2(l1), m2 = cabs2(l2);
      const bool first = m1 > m2 * (1.f + 1e-5f) || (m2 <= m1 * (1.f + 1e-5f) && l1.y >= l2.y);
      const float2 lp = first ? l1 : l2;
      l = mk((double)lp.x, (double)lp.y);
      okv = 2;
    }
    lam[o] = l;
    ok[o] = okv;
    if (cabs2(l) >= 1.0) atomicOr(flags, 2);
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

static int bse_chunk(int n) { return n <= 32 ? n : (n <= 64 ? 32 : 16); }
static bool bse_lu_in_smem(int n) { return n <= kLuSmemOrder; }
static bool bse_lu_fits_smem(int n) { return n <= 96; }   // the allocation-free entry point's limit

size_t bse_workspace_bytes(const Dims& dm, int grid) {
  size_t b = (size_t)2 * dm.nb * dm.n_w * dm.n_w * sizeof(double2);      // gamma o gamma^T
  if (!bse_lu_in_smem(dm.n_w)) b += (size_t)grid * dm.n_w * dm.n_w * sizeof(double2);
  return b;
}

static size_t bse_smem_bytes(int n) {
  return sizeof(double2) * (size_t)bse_layout(n, bse_chunk(n), bse_lu_in_smem(n)).total;
}

int bse_default_grid(const Dims& dm, int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const size_t smem = bse_smem_bytes(dm.n_w);
  const void* fn = bse_lu_in_smem(dm.n_w) ? (const void*)bse_f64_kernel<true> : (const void*)bse_f64_kernel<false>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBseThreads, smem);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

static double2* gg_ptr(df_ctx* c) { return (double2*)c->bse_ws; }
const double2* gamma_gt_ptr(df_ctx* c) { return gg_ptr(c); }
static int* flag_ptr(df_ctx* c) { return bse_flags(c); }
static double2* lu_ws_ptr(df_ctx* c) {
  return (double2*)((char*)c->bse_ws + (size_t)2 * c->dm.nb * c->dm.n_w * c->dm.n_w * sizeof(double2));
}

cudaError_t launch_gamma_gt(df_ctx* c) {
  const Dims& dm = c->dm;
  gamma_gt_kernel<<<2 * dm.nb * 8, 256, 0, c->stream>>>(dm.n_w, 2 * dm.nb, c->gam, gg_ptr(c));
  return cudaGetLastError();
}

cudaError_t launch_bse(df_ctx* c, int channel_mask) {
  const Dims& dm = c->dm;
  const int n = dm.n_w;
  const int nc = bse_chunk(n);
  const size_t smem = bse_smem_bytes(n);
  cudaError_t e = cudaSuccess;
  if (c->opts.precision == DF_FP32_IR) return launch_bse_mixed(c, channel_mask, flag_ptr(c));
  const int K = c->opts.radius_order;
  const double2* lam = K > 0 ? c->lam : nullptr;
  // both channels in one launch of the grid-stride kernel when both are asked
  // for (one partial wave instead of two)
  const bool both = (channel_mask & 3) == 3;
  for (int ch = 0; ch < 2; ++ch) {
    if (!(channel_mask & (1 << ch))) continue;
    const int nch = both ? 2 : 1;
    const long systems = (long)nch * dm.na * dm.N;
    const int grid = (int)(systems < c->bse_grid ? systems : c->bse_grid);
    if (bse_lu_in_smem(n)) {
      bse_f64_kernel<true><<<grid, kBseThreads, smem, c->stream>>>(dm, ch, nch, nc, c->gam, gg_ptr(c), c->chi,
                                                                   c->kc, nullptr, flag_ptr(c), K, lam, nullptr, 0);
    } else {
      bse_f64_kernel<false><<<grid, kBseThreads, smem, c->stream>>>(dm, ch, nch, nc, c->gam, gg_ptr(c), c->chi,
                                                                    c->kc, lu_ws_ptr(c), flag_ptr(c), K, lam,
                                                                    nullptr, 0);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (both) break;
  }
  return cudaSuccess;
}

// the FP64 LU over the ladders the mixed-precision kernels handed back: list[0]
// (read on the device) systems (c N_W + a) N + q, on the persistent grid; a
// list shorter than the SM count is spread over the SMs by right-hand-side ranges
cudaError_t launch_bse_f64_list(df_ctx* c, const int* list) {
  const Dims& dm = c->dm;
  const int n = dm.n_w;
  const int nc = bse_chunk(n) < 16 ? bse_chunk(n) : 16;   // 16-column ranges to spread (fits the default layout)
  const size_t smem = bse_smem_bytes(n);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  cudaError_t e = cudaFuncSetAttribute(bse_lu_in_smem(n) ? (const void*)bse_f64_kernel<true>
                                                         : (const void*)bse_f64_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (bse_lu_in_smem(n))
    bse_f64_kernel<true><<<c->bse_grid, kBseThreads, smem, c->stream>>>(dm, 0, 2, nc, c->gam, gg_ptr(c), c->chi,
                                                                        c->kc, nullptr, flag_ptr(c), 0, nullptr, list,
                                                                        sms);
  else
    bse_f64_kernel<false><<<c->bse_grid, kBseThreads, smem, c->stream>>>(dm, 0, 2, nc, c->gam, gg_ptr(c), c->chi,
                                                                         c->kc, lu_ws_ptr(c), flag_ptr(c), 0, nullptr,
                                                                         list, sms);
  return cudaGetLastError();
}

// the ladder term of the susceptibilities for both channels: FP64 LU on the
// persistent grid and LU scratch of the FP64 ladder kernel, or under
// DF_FP32_IR the refinement kernel first (D from gamma's FP32 leading words,
// the first array of the mixed-precision workspace) and the FP64 LU only for
// the systems it hands back (redo: 1 + 2 nb N ints)
cudaError_t launch_chi_ladder(df_ctx* c, const double2* Lb, const double2* chi0, double2* out, int* redo) {
  const Dims& dm = c->dm;
  const int n = dm.n_w;
  const bool in_smem = bse_lu_in_smem(n);
  const size_t smem = sizeof(double2) * (size_t)bse_layout(n, 2, in_smem).total;
  const void* fn = in_smem ? (const void*)chi_ladder_kernel<true> : (const void*)chi_ladder_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long systems = 2L * dm.nb * dm.N;
  const int* list = nullptr;
  if (c->opts.precision == DF_FP32_IR && n <= kChiIrMaxN && c->mixed_ws) {
    const size_t ism = sizeof(float2) * (size_t)n * (n + 1);
    e = cudaFuncSetAttribute((const void*)chi_ladder_ir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void*)chi_ladder_ir_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)chi_ladder_ir_kernel, kChiIrThreads, ism);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long ig = (long)sms * per_sm;
    if ((e = cudaMemsetAsync(redo, 0, sizeof(int), c->stream)) != cudaSuccess) return e;
    chi_ladder_ir_kernel<<<(int)(systems < ig ? systems : ig), kChiIrThreads, ism, c->stream>>>(
        dm, c->gam, (const float2*)c->mixed_ws, c->chi, Lb, chi0, out, redo, c->opts.ir_max_steps, c->opts.ir_tol);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    list = redo;
  }
  const int grid = (int)(systems < c->bse_grid ? systems : c->bse_grid);
  if (in_smem)
    chi_ladder_kernel<true><<<grid, kBseThreads, smem, c->stream>>>(dm, c->gam, c->chi, Lb, chi0, out, nullptr,
                                                                    flag_ptr(c), list);
  else
    chi_ladder_kernel<false><<<grid, kBseThreads, smem, c->stream>>>(dm, c->gam, c->chi, Lb, chi0, out,
                                                                     lu_ws_ptr(c), flag_ptr(c), list);
  return cudaGetLastError();
}

cudaError_t launch_lambda(df_ctx* c, int channel_mask) {
  const Dims& dm = c->dm;
  if (c->opts.eig_mode == 0) return cudaSuccess;
  // W = 0 only (eig_mode 1) or every plane, within the handle's bosonic range
  if (c->opts.eig_mode == 1 && (dm.m_max < dm.a0 || dm.m_max >= dm.a0 + dm.na)) return cudaSuccess;
  const int a0 = (c->opts.eig_mode == 1) ? dm.m_max : dm.a0;
  const int na = (c->opts.eig_mode == 1) ? 1 : dm.na;
  const int qtiles = (dm.N + kEigQ - 1) / kEigQ;
  const int ch0 = (channel_mask & 1) ? 0 : 1;
  const int nch = (channel_mask & 1) && (channel_mask & 2) ? 2 : 1;
  if (!(channel_mask & 3)) return cudaSuccess;
  if (dm.n_w <= kEigRegN) {
    const size_t lsm = sizeof(float2) * 4 * kEigLoStride;
    cudaError_t e = cudaFuncSetAttribute((const void*)lambda_reg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)lsm);
    if (e != cudaSuccess) return e;
    lambda_reg_kernel<<<nch * na * qtiles, 256, lsm, c->stream>>>(dm, ch0, a0, na, 1e-12, c->gam, c->chi, c->lam,
                                                                  c->lam_ok, flag_ptr(c));
    return cudaGetLastError();
  }
  // gamma's (hi, lo) FP32 pairs in shared memory when they fit (n_w <= 96), the
  // lo parts formed from FP64 gamma on the fly above that
  const size_t base = sizeof(double2) * 3 * dm.n_w * kEigQ + sizeof(float2) * ((size_t)dm.n_w * dm.n_w + 3 * dm.n_w * kEigQ);
  const int lo_in_smem = base + sizeof(float2) * (size_t)dm.n_w * dm.n_w <= (size_t)200 * 1024 ? 1 : 0;
  const size_t smem = base + (lo_in_smem ? sizeof(float2) * (size_t)dm.n_w * dm.n_w : 0);
  cudaError_t e = cudaFuncSetAttribute((const void*)lambda_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // both channels in one launch when both are asked for
  lambda_kernel<<<nch * na * qtiles, kEigThreads, smem, c->stream>>>(dm, ch0, a0, na, lo_in_smem, 1e-12, c->gam,
                                                                     c->chi, c->lam, c->lam_ok, flag_ptr(c));
  return cudaGetLastError();
}

}  // namespace df

// ---------------------------------------------------------------------------
// launchers on caller-given buffers (no handle), used by the allocation-free
// entry point; the kernels are the ones above
// ---------------------------------------------------------------------------
namespace df {

cudaError_t launch_gamma_gt_raw(int n, int count, const double2* gam, double2* gg, cudaStream_t stream) {
  gamma_gt_kernel<<<count * 8, 256, 0, stream>>>(n, count, gam, gg);
  return cudaGetLastError();
}

cudaError_t launch_bse_both_raw(const Dims& dm, const double2* gam, const double2* gg, const double2* chi,
                                double2* kc, int* flags, int device, cudaStream_t stream) {
  if (!bse_lu_fits_smem(dm.n_w)) return cudaErrorInvalidValue;
  const int nc = bse_chunk(dm.n_w);
  const size_t smem = sizeof(double2) * (size_t)bse_layout(dm.n_w, nc, true).total;
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaFuncSetAttribute((const void*)bse_f64_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bse_f64_kernel<true>, kBseThreads, smem);
  const int grid_max = sms * (per_sm < 1 ? 1 : per_sm);
  const long systems = 2L * dm.nb * dm.N;
  const int grid = (int)(systems < grid_max ? systems : grid_max);
  bse_f64_kernel<true><<<grid, kBseThreads, smem, stream>>>(dm, 0, 2, nc, gam, gg, chi, kc, nullptr, flags, 0,
                                                            nullptr, nullptr, 0);
  return cudaGetLastError();
}

}  // namespace df
