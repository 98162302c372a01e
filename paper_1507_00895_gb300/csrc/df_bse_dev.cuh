// Device body of the FP64 ladder solve (Eq. lin_alg_inv) of one
// (q, W, channel) system; used by the single-problem kernel (df_bse.cu) and
// the batched one (df_batch.cu).  Must be called by all threads of a
// 256-thread block.
#pragma once
#include "df_internal.cuh"

namespace df {

constexpr int kBseThreads = 256;
// FP64 ladders of order <= kLuSmemOrder factorise in shared memory, larger ones
// in a per-block slice of global (L2-resident) scratch: the shared-memory LU
// limits the blocks per SM (one at order 96, two at 64), the global one
// leaves room for several, which hides the per-pivot barrier latency better.
// Measured fractions of the FP64 peak (shared / global): order 40 64.6 / 63.8%,
// 48 67.4 / 70.2%, 64 71.4 / 78.4%, 96 57 / 83%.
constexpr int kLuSmemOrder = 40;

struct BseSmem {
  // offsets in double2 units inside the dynamic shared block
  int lu, y, xs, invu, total;
};

__host__ __device__ inline BseSmem bse_layout(int n, int nc, bool lu_in_smem) {
  BseSmem L;
  int off = 0;
  L.lu = off;
  if (lu_in_smem) off += n * n;
  L.y = off;
  off += n * nc;
  L.xs = off;
  off += n;
  L.invu = off;
  off += n;
  L.total = off;
  return L;
}

struct BseF64Shared {
  int perm[128];
  int piv;
  double2 pv, oldkk;
  // (row offset << 8) | column of the triangular part of a right-hand-side
  // chunk's back substitution, rows 0..nc-2 in order (row d has columns 0..d)
  unsigned short tri[32 * 31 / 2];
};

// D = 1 - gamma_W diag(chi~_W(q)) (Eq. lin_alg_inv) factorised in place in LU
// (n x n, row-major; shared or global memory) with partial pivoting:
// P D = L U, L unit lower (the multipliers), U's strictly upper columns
// scaled by 1/U_kk (so D = P^T L V diag(U_kk) with V unit upper), 1/U_kk in
// invu, the row order in sh.perm, chi~_W(q) in xs.  Zero pivots set flags bit 0.
__device__ __forceinline__ void bse_f64_factor(const Dims& dm, int c, int a, int q,
                                               const double2* __restrict__ gam, const double2* __restrict__ chi,
                                               double2* LU, double2* xs, double2* invu, BseF64Shared& sh,
                                               int* __restrict__ flags) {
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const double2* G = gam + ((size_t)c * nb + a) * n * n;

  for (int i = tid; i < n; i += blockDim.x) {
    xs[i] = chi[((size_t)a * n + i) * N + q];
    sh.perm[i] = i;
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    double2 v = cmul(G[idx], xs[j]);
    v = mk((i == j ? 1.0 : 0.0) - v.x, -v.y);
    LU[idx] = v;
  }
  __syncthreads();
  // ---- LU with partial pivoting ----
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int r = k + lane; r < n; r += 32) {
        const double v = cabs1(LU[r * n + k]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) {
        sh.piv = bi;
        const double2 pv = LU[bi * n + k];
        sh.pv = pv;
        sh.oldkk = LU[k * n + k];
        if (pv.x == 0.0 && pv.y == 0.0) {
          atomicOr(flags, 1);
          invu[k] = mk(0.0, 0.0);
        } else {
          invu[k] = cinv(pv);
        }
        if (bi != k) {
          const int t = sh.perm[k]; sh.perm[k] = sh.perm[bi]; sh.perm[bi] = t;
        }
      }
    }
    __syncthreads();
    const int p = sh.piv;
    const double2 inv = invu[k];
    // row swap of the columns != k, and the multipliers of column k
    if (p != k) {
      for (int col = tid; col < n; col += blockDim.x) {
        if (col == k) continue;
        const double2 t = LU[k * n + col];
        LU[k * n + col] = LU[p * n + col];
        LU[p * n + col] = t;
      }
    }
    for (int r = k + tid; r < n; r += blockDim.x) {
      if (r == k) {
        LU[k * n + k] = sh.pv;
      } else {
        const double2 v = (r == p) ? sh.oldkk : LU[r * n + k];
        LU[r * n + k] = cmul(v, inv);
      }
    }
    __syncthreads();
    // trailing rank-1 update
    const int m = n - k - 1;
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      const int r = k + 1 + idx / m, col = k + 1 + idx % m;
      LU[r * n + col] = cfms(LU[r * n + k], LU[k * n + col], LU[r * n + col]);
    }
    __syncthreads();
  }
  // scale U's strictly-upper columns by 1/U_kk (unit-diagonal V = U diag(1/U_kk))
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, col = idx - r * n;
    if (r < col) LU[idx] = cmul(LU[idx], invu[col]);
  }
  __syncthreads();
}

// D = 1 - gamma_W diag(chi~_W(q)) factorised in LU (n x n, row-major; shared
// or global memory), right-hand sides P gamma in chunks of nc columns in Y,
// writes kc[c][a][j][q] = w_c (Gamma_jj - Gamma^(2)_jj / 2) for the columns
// j in [j_begin, j_end) (multiples of nc but the last; default all).  With radius_K > 0
// and |lam[c][a][q]| >= 1 (outside the ladder's convergence radius) Gamma is
// instead the low-order iterative evaluation Gamma <- gamma + gamma chi~ Gamma,
// radius_K times from Gamma = gamma (the LU buffer holds the product).
__device__ __forceinline__ void bse_f64_system(const Dims& dm, int c, int a, int q, int nc,
                                               const double2* __restrict__ gam, const double2* __restrict__ gg,
                                               const double2* __restrict__ chi, double2* __restrict__ kc,
                                               double2* LU, double2* Y, double2* xs, double2* invu,
                                               BseF64Shared& sh, int* __restrict__ flags, int radius_K = 0,
                                               const double2* __restrict__ lam = nullptr, int j_begin = 0,
                                               int j_end = 1 << 30) {
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  const int tid = threadIdx.x;
  const double2* G = gam + ((size_t)c * nb + a) * n * n;
  const double2* GG = gg + ((size_t)c * nb + a) * n * n;

  bool series = false;
  if (radius_K > 0) {
    const double2 l = lam[((size_t)c * nb + a) * N + q];
    series = (l.x * l.x + l.y * l.y >= 1.0);
  }
  if (series) {
    for (int i = tid; i < n; i += blockDim.x) xs[i] = chi[((size_t)a * n + i) * N + q];
    __syncthreads();
  } else {
    for (int e = tid; e < nc * (nc - 1) / 2; e += blockDim.x) {
      int d = 0;
      while ((d + 1) * (d + 2) / 2 <= e) ++d;
      sh.tri[e] = (unsigned short)((d << 8) | (e - d * (d + 1) / 2));
    }
    bse_f64_factor(dm, c, a, q, gam, chi, LU, xs, invu, sh, flags);
  }

  // ---- diag(Gamma) by chunks of nc right-hand sides ----
  const int j_stop = j_end < n ? j_end : n;
  for (int j0 = j_begin; j0 < j_stop; j0 += nc) {
    const int w = min(nc, n - j0);
    if (series) {
      for (int idx = tid; idx < n * w; idx += blockDim.x) {
        const int r = idx / w, jj = idx - r * w;
        Y[r * nc + jj] = G[(size_t)r * n + j0 + jj];
      }
      __syncthreads();
      for (int it = 0; it < radius_K; ++it) {
        for (int idx = tid; idx < n * w; idx += blockDim.x) {
          const int r = idx / w, jj = idx - r * w;
          double2 t = G[(size_t)r * n + j0 + jj];
          for (int k = 0; k < n; ++k) t = cfma(cmul(G[(size_t)r * n + k], xs[k]), Y[k * nc + jj], t);
          LU[r * nc + jj] = t;
        }
        __syncthreads();
        for (int idx = tid; idx < n * w; idx += blockDim.x) {
          const int r = idx / w, jj = idx - r * w;
          Y[r * nc + jj] = LU[r * nc + jj];
        }
        __syncthreads();
      }
    } else {
    for (int idx = tid; idx < n * w; idx += blockDim.x) {
      const int r = idx / w, jj = idx - r * w;
      Y[r * nc + jj] = G[(size_t)sh.perm[r] * n + j0 + jj];
    }
    __syncthreads();
    for (int k = 0; k < n - 1; ++k) {           // unit-lower forward substitution
      const int m = n - k - 1;
      for (int idx = tid; idx < m * w; idx += blockDim.x) {
        const int r = k + 1 + idx / w, jj = idx % w;
        Y[r * nc + jj] = cfms(LU[r * n + k], Y[k * nc + jj], Y[r * nc + jj]);
      }
      __syncthreads();
    }
    for (int k = n - 1; k > j0; --k) {          // unit-upper back substitution, rows >= j0 only
      // column jj needs rows r >= j0 + jj: rows j0 .. j0+w-2 are the triangle
      // (table), rows from j0+w-1 on take all w columns
      const int m = k - j0;
      const int tr = m < w - 1 ? m : w - 1;
      const int ntri = tr * (tr + 1) / 2;
      const int nrect = m > w - 1 ? (m - (w - 1)) * w : 0;
      for (int idx = tid; idx < ntri + nrect; idx += blockDim.x) {
        int r, jj;
        if (idx < ntri) {
          const unsigned short e = sh.tri[idx];
          r = j0 + (e >> 8);
          jj = e & 0xff;
        } else {
          const int i2 = idx - ntri;
          r = j0 + (w - 1) + i2 / w;
          jj = i2 % w;
        }
        Y[r * nc + jj] = cfms(LU[r * n + k], Y[k * nc + jj], Y[r * nc + jj]);
      }
      __syncthreads();
    }
    }
    for (int jj = tid; jj < w; jj += blockDim.x) {
      const int j = j0 + jj;
      const double2 gdiag = series ? Y[j * nc + jj] : cmul(Y[j * nc + jj], invu[j]);
      double2 g2 = mk(0.0, 0.0);
      for (int x = 0; x < n; ++x) g2 = cfma(GG[(size_t)j * n + x], xs[x], g2);
      const double wgt = (c == 0) ? 1.0 : 3.0;
      kc[(((size_t)c * nb + a) * n + j) * N + q] =
          mk(wgt * (gdiag.x - 0.5 * g2.x), wgt * (gdiag.y - 0.5 * g2.y));
    }
    __syncthreads();
  }
}

}  // namespace df
