// Device body of the DF_FP32_IR ladder solve of order 64 < n <= 128 (one
// (q, W, channel) system); used by the single-problem kernel
// (df_mixed_large.cu) and the batched one (df_batch.cu).  Must be called by
// every thread of a block of at least 2n threads (a multiple of 32), with
// gj_layout(n).total bytes of dynamic shared memory at smraw.
#pragma once
#include "df_internal.cuh"
#include "df_tcgj_dev.cuh"

namespace df {

constexpr int kGjNc = 8;            // right-hand-side columns per chunk
constexpr int kGjMaxN = 128;

struct GjLayout {
  // byte offsets inside the dynamic shared block
  int S, B, Y, Zh, Zl, colk, xh, xl, xs, total;
};

// tc: the tensor-core sweep's operand tiles share the S region (used before S is written)
__host__ __device__ inline GjLayout gj_layout(int n, bool tc = false) {
  GjLayout L;
  int off = 0;
  auto take = [&](int bytes) { const int o = off; off += (bytes + 15) & ~15; return o; };
  const int s_bytes = 8 * n * (n + 1);
  L.S = take(tc && tc_smem_bytes(n) > s_bytes ? tc_smem_bytes(n) : s_bytes);
  L.B = take(8 * n * kGjNc);
  L.Y = take(8 * n * kGjNc);
  L.Zh = take(8 * n * kGjNc);
  L.Zl = take(8 * n * kGjNc);
  L.colk = take(8 * n);
  L.xh = take(8 * n);
  L.xl = take(8 * n);
  L.xs = take(16 * n);
  L.total = off;
  return L;
}

__host__ __device__ inline int gj_threads(int n) { return (2 * n + 31) / 32 * 32; }

struct GjShared {
  int perm[kGjMaxN];
  int ipiv[kGjMaxN];      // tensor-core sweep: the position of each row in the pivot order
  float pabs[2];
  int prow[2];
  float2 pval[2];
  // per-ladder error control: max |correction|, max |Gamma_jj| (float bits), non-finite seen
  unsigned emax, gmax;
  int bad;
};

__device__ __forceinline__ float2 gj_cinv(float2 z) {   // 1/z in FP32 (|z|^2 in range here)
  const float d = __frcp_rn(z.x * z.x + z.y * z.y);
  return make_float2(z.x * d, -z.y * d);
}

// (S, L) += A o B exactly, elementwise: the product's rounding error by FMA
// (nA = -A gives p - A B = -error), the sum's by TwoSum
__device__ __forceinline__ void x2_acc(float2& S, float2& L, float2 A, float2 nA, float2 B) {
  const float2 p = x2_mul(A, B);
  const float2 ne = x2_fma(nA, B, p);
  const float2 s = x2_add(S, p);
  const float2 bb = x2_sub(s, S);
  const float2 e = x2_add(x2_sub(S, x2_sub(s, bb)), x2_sub(p, bb));
  S = s;
  L = x2_sub(x2_add(L, e), ne);
}

// Tensor-core state of a block running the TC variant (TC = true): TMEM base of
// its 256 columns, the MMA completion barrier and its parity.
struct GjTc {
  unsigned tmem;
  uint64_t* mbar;
  unsigned phase;
};

// ghi, glo: gamma's (hi, lo) FP32 words [2][nb][n][n]; gth, gtl: gamma^T's;
// gg: gamma o gamma^T (FP64); chi: chi~ [nb][n][N]; kc: the Eq. sd bracket
// [2][nb][n][N]; flags bit 0: a zero FP32 pivot.  TC: the Gauss-Jordan
// inversion on the tensor cores (df_tcgj_dev.cuh; kTcThreads threads, tc
// set up), else on the CUDA cores.  Returns false when a tensor-core wait
// gave up (the block must stop; the same value in every thread).
template <bool TC = false>
__device__ __forceinline__ bool gj_ir_system(const Dims& dm, int c, int a, int q, const float2* __restrict__ ghi,
                                             const float2* __restrict__ glo, const float2* __restrict__ gth,
                                             const float2* __restrict__ gtl, const double2* __restrict__ gg,
                                             const double2* __restrict__ chi, double2* __restrict__ kc,
                                             int* __restrict__ flags, unsigned char* smraw, GjShared& sh,
                                             const MixedCheck& mc, GjTc* tc = nullptr) {
  const int n = dm.n_w, N = dm.N, nb = dm.nb, ld = n + 1;
  const GjLayout L = gj_layout(n, TC);
  float2* S = (float2*)(smraw + L.S);      // [n][n + 1]: D, then (P D)^-1
  float2* B = (float2*)(smraw + L.B);      // [n][8]: P gamma, then R
  float2* Y = (float2*)(smraw + L.Y);      // [n][8]
  float2* Zh = (float2*)(smraw + L.Zh);    // [n][8]: chi~ o Y, leading words
  float2* Zl = (float2*)(smraw + L.Zl);    // [n][8]: trailing words
  float2* colk = (float2*)(smraw + L.colk);
  float2* xh = (float2*)(smraw + L.xh);
  float2* xl = (float2*)(smraw + L.xl);
  double2* xs = (double2*)(smraw + L.xs);
  const int tid = threadIdx.x, T = blockDim.x, warp = tid >> 5, lane = tid & 31, nwarp = T >> 5;
  const bool act = tid < 2 * n;
  // column (row in the products) and group: row group of two in the build and
  // the update, column half of four in the products
  const int j = tid % n, g = tid / n;
  const size_t mat = ((size_t)c * nb + a) * n * n;
  const float2* Gh = ghi + mat;
  const float2* Gl = glo + mat;
  const float2* GTh = gth + mat;
  const float2* GTl = gtl + mat;
  const double2* GG = gg + mat;
  for (int i = tid; i < n; i += T) {
    const double2 v = chi[((size_t)a * n + i) * N + q];
    xs[i] = v;
    const float hx = (float)v.x, hy = (float)v.y;
    xh[i] = make_float2(hx, hy);
    xl[i] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
    sh.perm[i] = i;
  }
  if (tid == 0) {
    sh.emax = 0u;
    sh.gmax = 0u;
    sh.bad = 0;
  }
  __syncthreads();
  if constexpr (TC) {
    // 1-2. D into tensor memory (lane j = column j, TMEM column 2i + c = row i), in
    // double-float rounded once, then the Gauss-Jordan sweep on the tensor cores
    const int np = tc_pad(n);
    const int qd = warp & 3, jl = 32 * qd + lane;
    const unsigned tq = tc->tmem + ((32u * qd) << 16);
    tc05_fence_after();
    {
      const float2 ah = jl < n ? xh[jl] : make_float2(0.f, 0.f), al = jl < n ? xl[jl] : make_float2(0.f, 0.f);
      for (int r = 8 * (warp >> 2); r < np; r += 16) {
        float v[16];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int i = r + e;
          float2 d = make_float2(0.f, 0.f);
          if (i < n && jl < n) {
            float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
            cdf_fma(sr, lr, si, li, __ldg(Gh + (size_t)i * n + jl), __ldg(Gl + (size_t)i * n + jl), ah, al);
            d = make_float2(((i == jl ? 1.f : 0.f) - sr) - lr, -si - li);
          }
          v[2 * e] = d.x;
          v[2 * e + 1] = d.y;
        }
        tmem_st16(tq + 2 * r, v);
      }
      tmem_wait_st();
    }
    tc05_fence_before();
    __syncthreads();
    tc05_fence_after();
    if (!tcgj_sweep(tc->tmem, n, n, tc_smem(smraw + L.S, n), sh.perm, tc->mbar, tc->phase, flags)) return false;
    for (int k = tid; k < n; k += T) sh.ipiv[sh.perm[k]] = k;
    __syncthreads();
    // S = (P D)^-1, S[k][l] = D^-1[k][p_l] = A[p_k][l]: row r of the swept A is row ipiv[r] of S
    for (int r = 8 * (warp >> 2); r < np; r += 16) {
      float v[16];
      tmem_ld16(tq + 2 * r, v);
      if (jl < n) {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (r + e < n) {
            const int rr = sh.ipiv[r + e];
            if ((unsigned)rr < (unsigned)n) S[rr * ld + jl] = make_float2(v[2 * e], v[2 * e + 1]);
          }
      }
    }
    tc05_fence_before();
    __syncthreads();
  } else {
  // 1. D in double-float, rounded once; column 0's pivot candidates
  if (act) {
    const float2 ah = xh[j], al = xl[j];
    float best = -1.f;
    int brow = n;
    float2 bval = make_float2(0.f, 0.f);
    for (int i = g; i < n; i += 2) {
      float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
      cdf_fma(sr, lr, si, li, __ldg(Gh + (size_t)i * n + j), __ldg(Gl + (size_t)i * n + j), ah, al);
      const float2 d = make_float2(((i == j ? 1.f : 0.f) - sr) - lr, -si - li);
      S[i * ld + j] = d;
      if (j == 0 && cabs1(d) > best) { best = cabs1(d); brow = i; bval = d; }
    }
    if (j == 0) { sh.pabs[g] = best; sh.prow[g] = brow; sh.pval[g] = bval; }
  }
  __syncthreads();
  // 2. Gauss-Jordan in place: S = (P D)^-1
  for (int k = 0; k < n; ++k) {
    float best = -1.f;
    int p = n;
    float2 pv = make_float2(0.f, 0.f);
#pragma unroll
    for (int gi = 0; gi < 2; ++gi) {
      const float v = sh.pabs[gi];
      const int rr = sh.prow[gi];
      if (v > best || (v == best && rr < p)) { best = v; p = rr; pv = sh.pval[gi]; }
    }
    if (p >= n) { p = k; pv = make_float2(0.f, 0.f); }   // no candidate (NaN column): a zero pivot
    const bool zero = (pv.x == 0.f && pv.y == 0.f);
    const float2 inv = zero ? make_float2(0.f, 0.f) : gj_cinv(pv);
    if (tid == 0) {
      if (zero) atomicOr(flags, kFlagSingular);
      if (p != k) { const int t = sh.perm[k]; sh.perm[k] = sh.perm[p]; sh.perm[p] = t; }
    }
    // rows k and p exchanged, row k scaled by 1/pivot (its column-k entry
    // becomes 1/pivot); column k's other entries moved to the multipliers
    // colk and zeroed (the update below then writes -colk_i / pivot there),
    // row k's multiplier 0
    if (tid < n) {
      const float2 t1 = S[k * ld + tid], t2 = S[p * ld + tid];
      if (p != k) S[p * ld + tid] = (tid == k) ? make_float2(0.f, 0.f) : t1;
      S[k * ld + tid] = (tid == k) ? inv : cmul(t2, inv);
      if (tid == k) {
        if (p != k) colk[p] = t1;
        colk[k] = make_float2(0.f, 0.f);
      }
      if (tid != k && tid != p) {
        colk[tid] = S[tid * ld + k];
        S[tid * ld + k] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    // every row: S_ij -= colk_i S_kj, the same code in every lane; rows in
    // batches of four, loads before stores; the lanes of column k + 1 keep
    // its pivot candidates among rows > k
    if (act) {
      const float2 u = S[k * ld + j];
      const bool cand = (j == k + 1);
      float bb = -1.f;
      int br = n;
      float2 bv = make_float2(0.f, 0.f);
      float2* col = S + j;
      int i = g;
      for (; i + 6 < n; i += 8) {
        float2 f[4], t[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          f[e] = colk[i + 2 * e];
          t[e] = col[(i + 2 * e) * ld];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          t[e] = cfms(f[e], u, t[e]);
          col[(i + 2 * e) * ld] = t[e];
        }
        if (cand) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (i + 2 * e > k && cabs1(t[e]) > bb) { bb = cabs1(t[e]); br = i + 2 * e; bv = t[e]; }
        }
      }
      for (; i < n; i += 2) {
        const float2 t = cfms(colk[i], u, col[i * ld]);
        col[i * ld] = t;
        if (cand && i > k && cabs1(t) > bb) { bb = cabs1(t); br = i; bv = t; }
      }
      if (cand) { sh.pabs[g] = bb; sh.prow[g] = br; sh.pval[g] = bv; }
    }
    __syncthreads();
  }
  }   // CUDA-core sweep
  // 3. right-hand sides in chunks of kGjNc columns
  for (int j0 = 0; j0 < n; j0 += kGjNc) {
    const int w = min(kGjNc, n - j0);
    for (int e = tid; e < n * kGjNc; e += T) {        // P gamma, leading words
      const int k = e / kGjNc, jj = e - k * kGjNc;
      B[e] = jj < w ? __ldg(Gh + (size_t)sh.perm[k] * n + j0 + jj) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (act) {                                        // Y = S (P gamma)
      float2 acc[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] = make_float2(0.f, 0.f);
      for (int k = 0; k < n; ++k) {
        const float2 s = S[j * ld + k];
        const float4 b01 = *reinterpret_cast<const float4*>(B + k * kGjNc + 4 * g);
        const float4 b23 = *reinterpret_cast<const float4*>(B + k * kGjNc + 4 * g + 2);
        acc[0] = cfma(s, make_float2(b01.x, b01.y), acc[0]);
        acc[1] = cfma(s, make_float2(b01.z, b01.w), acc[1]);
        acc[2] = cfma(s, make_float2(b23.x, b23.y), acc[2]);
        acc[3] = cfma(s, make_float2(b23.z, b23.w), acc[3]);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) Y[j * kGjNc + 4 * g + e] = acc[e];
    }
    __syncthreads();
    for (int e = tid; e < n * kGjNc; e += T) {        // Z = chi~ o Y, double-float
      const int k = e / kGjNc;
      float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
      cdf_fma(sr, lr, si, li, xh[k], xl[k], Y[e], make_float2(0.f, 0.f));
      Zh[e] = make_float2(sr, si);
      Zl[e] = make_float2(lr, li);
    }
    __syncthreads();
    if (act) {                                        // R = gamma - Y + gamma Z, double-float
      // per column two packed accumulators: S (re, im) takes gamma_re * Z and
      // the trailing-word terms with gamma_re; S2 (im, re), swapped, takes
      // gamma_im * Z, so that Z's words are used in their stored order
      float2 S1[4], L1[4], S2[4], L2[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) S1[e] = L1[e] = S2[e] = L2[e] = make_float2(0.f, 0.f);
      for (int k = 0; k < n; ++k) {
        const float2 gh = __ldg(GTh + (size_t)k * n + j), gl = __ldg(GTl + (size_t)k * n + j);
        const float2 A1 = make_float2(gh.x, gh.x), nA1 = make_float2(-gh.x, -gh.x);
        const float2 A2 = make_float2(gh.y, -gh.y), nA2 = make_float2(-gh.y, gh.y);
        const float2 AL1 = make_float2(gl.x, gl.x), AL2 = make_float2(gl.y, -gl.y);
        const float4 h01 = *reinterpret_cast<const float4*>(Zh + k * kGjNc + 4 * g);
        const float4 h23 = *reinterpret_cast<const float4*>(Zh + k * kGjNc + 4 * g + 2);
        const float4 l01 = *reinterpret_cast<const float4*>(Zl + k * kGjNc + 4 * g);
        const float4 l23 = *reinterpret_cast<const float4*>(Zl + k * kGjNc + 4 * g + 2);
        const float2 Bh[4] = {make_float2(h01.x, h01.y), make_float2(h01.z, h01.w), make_float2(h23.x, h23.y),
                              make_float2(h23.z, h23.w)};
        const float2 Bl[4] = {make_float2(l01.x, l01.y), make_float2(l01.z, l01.w), make_float2(l23.x, l23.y),
                              make_float2(l23.z, l23.w)};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          x2_acc(S1[e], L1[e], A1, nA1, Bh[e]);
          x2_acc(S2[e], L2[e], A2, nA2, Bh[e]);
          L1[e] = x2_fma(AL1, Bh[e], x2_fma(A1, Bl[e], L1[e]));
          L2[e] = x2_fma(AL2, Bh[e], x2_fma(A2, Bl[e], L2[e]));
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int jj = 4 * g + e;
        if (jj < w) {
          // re = S1.x + S2.y, im = S1.y + S2.x, each a double-float sum
          float sr, lr, si, li;
          two_sum(S1[e].x, S2[e].y, sr, lr);
          lr += L1[e].x + L2[e].y;
          two_sum(S1[e].y, S2[e].x, si, li);
          li += L1[e].y + L2[e].x;
          const float2 gh = __ldg(GTh + (size_t)(j0 + jj) * n + j), gl = __ldg(GTl + (size_t)(j0 + jj) * n + j);
          const float2 y = Y[j * kGjNc + jj];
          float s, e1;
          two_sum(sr, gh.x, s, e1);
          const float rx = (s - y.x) + (e1 + lr + gl.x);
          two_sum(si, gh.y, s, e1);
          const float ry = (s - y.y) + (e1 + li + gl.y);
          B[j * kGjNc + jj] = make_float2(rx, ry);
        }
      }
    }
    __syncthreads();
    // Gamma_jj = Y_jj + (S (P R))_jj, Gamma^(2)_jj in FP64, the Eq. sd bracket
    for (int jj = warp; jj < w; jj += nwarp) {
      const int jc = j0 + jj;
      float2 d = make_float2(0.f, 0.f);
      for (int k = lane; k < n; k += 32) d = cfma(S[jc * ld + k], B[sh.perm[k] * kGjNc + jj], d);
      double2 g2 = mk(0.0, 0.0);
      for (int x = lane; x < n; x += 32) g2 = cfma(__ldg(GG + (size_t)jc * n + x), xs[x], g2);
      for (int o = 16; o > 0; o >>= 1) {
        d.x += __shfl_xor_sync(0xffffffffu, d.x, o);
        d.y += __shfl_xor_sync(0xffffffffu, d.y, o);
        g2.x += __shfl_xor_sync(0xffffffffu, g2.x, o);
        g2.y += __shfl_xor_sync(0xffffffffu, g2.y, o);
      }
      if (lane == 0) {
        const float2 y = Y[jc * kGjNc + jj];
        const double gx = (double)y.x + (double)d.x, gy = (double)y.y + (double)d.y;
        const float ea = fabsf(d.x) + fabsf(d.y), ga = (float)(fabs(gx) + fabs(gy));
        if (isfinite(ea) && isfinite(ga)) {
          atomicMax(&sh.emax, __float_as_uint(ea));
          atomicMax(&sh.gmax, __float_as_uint(ga));
        } else {
          sh.bad = 1;
        }
        const double wgt = (c == 0) ? 1.0 : 3.0;
        kc[(((size_t)c * nb + a) * n + jc) * N + q] = mk(wgt * (gx - 0.5 * g2.x), wgt * (gy - 0.5 * g2.y));
      }
    }
    __syncthreads();
  }
  // per-ladder error control (the next system's reset is by this thread too)
  if (tid == 0)
    mixed_check_ladder(mc, __uint_as_float(sh.emax), __uint_as_float(sh.gmax), sh.bad == 0,
                       ((long)c * nb + a) * N + q, flags);
  return true;
}

}  // namespace df
