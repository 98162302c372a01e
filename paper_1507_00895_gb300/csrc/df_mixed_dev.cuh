// Mixed-precision ladder solves (DF_FP32_IR): Eq. lin_alg_inv factorised in
// FP32 (complex64) and corrected once with an FP64-accurate residual.
//
// Per (q, W, channel) system, with D = 1 - gamma diag(chi~):
//   1. LU with partial pivoting of D in FP32 on the augmented [D | gamma]
//      (forward substitution of the n right-hand sides fused into the
//      elimination), then back substitution: X0 ~ D^-1 gamma in FP32.
//   2. R = gamma - D X0 = gamma - X0 + gamma (chi o X0), evaluated with
//      gamma and chi~ split into FP32 (hi, lo) pairs, exact FP32 products
//      (fma) and double-float (TwoSum) accumulation: ~48-bit accurate.
//   3. E = D^-1 R with the same FP32 LU; diag Gamma = diag X0 + diag E in FP64.
// One correction step leaves an error ~(kappa u32)^2 |Gamma| plus kappa times
// the residual's own accuracy, i.e. FP64-level for the condition numbers of
// the ladder matrices met here (up to ~1e6).
//
// Layout: the whole [D | RHS] lives in registers.  The block is a P x P
// grid of threads, P = n_pad / 4; thread (tr, tc) owns rows tr + P i and
// columns tc + P j (i, j < 4) of D and of the right-hand sides (2D cyclic,
// so that the shrinking active part of the elimination stays balanced).
// Row pivoting is implicit: rows never move; pivot rows are marked used and
// their order is kept in piv[] (logical row k of the factorisation is
// physical row piv[k]).  Matrices of order n < n_pad are padded with an
// identity block (gamma = 0, chi~ = 0 there), which leaves the solution of
// the first n rows unchanged.
#pragma once
#include "df_internal.cuh"

namespace df {


constexpr int kTile = 4;          // rows / columns per thread
constexpr int kResChunk = 16;     // gamma columns staged per residual sweep

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfmsf(float2 a, float2 b, float2 c) {   // c - a b
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cinvf(float2 z) {
  const float s = fmaxf(fabsf(z.x), fabsf(z.y));
  const float a = z.x / s, b = z.y / s;
  const float d = 1.0f / ((a * a + b * b) * s);
  return make_float2(a * d, -b * d);
}

// double-float helpers (value = hi + lo, |lo| <= ulp(hi)/2 after renormalisation)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// acc (hi, lo) += p exactly-ish: hi absorbs p with its rounding error moved to lo
__device__ __forceinline__ void df_add(float& hi, float& lo, float p) {
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo += e;
}
// (hi, lo) += a * b with a renormalised double-float accumulator: the exact
// product p + pe (fma), TwoSum into hi, the error and lo folded back by
// FastTwoSum, so that |lo| <= ulp(hi)/2 after every step and the running
// error stays ~2^-48 |hi| per step (not ~step * 2^-48 max|hi|).
__device__ __forceinline__ void dd_fma(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  float s, e;
  two_sum(hi, p, s, e);
  e += lo + pe;
  hi = s + e;
  lo = e - (hi - s);
}
// acc += a * b exactly for FP32 a, b (the product error goes to lo)
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  df_add(hi, lo, p);
  lo += e;
}

struct MixedSmem {
  // offsets in float2 units
  int x0, chih, chil, ubuf, lbuf, invu, x0d, gt_h, gt_l, yh, yl, chi64, total;
};

__host__ __device__ inline MixedSmem mixed_layout(int np) {
  MixedSmem L;
  int o = 0;
  L.x0 = o;   o += np * np;        // X0 (logical rows), also the row broadcast of the solves
  L.chih = o; o += np;
  L.chil = o; o += np;
  L.ubuf = o; o += 2 * np;         // pivot-row broadcast (D part + RHS part)
  L.lbuf = o; o += 2 * np;         // column broadcast, double buffered
  L.invu = o; o += np;
  L.x0d = o;  o += np;             // diag X0 (FP32)
  L.gt_h = o; o += kResChunk * np; // gamma tile, [l][row], hi
  L.gt_l = o; o += kResChunk * np; // lo
  L.yh = o;   o += np * np;        // Y = chi o X0, hi
  L.yl = o;   o += np * np;        // lo
  L.chi64 = o; o += 2 * np;        // chi~ in FP64 (double2 = two float2 slots)
  L.total = o;
  return L;
}

// Shared-memory views of one mixed solve (layout from mixed_layout).
struct MixedPtrs {
  float2 *X0s, *chih, *chil, *ubuf, *lbuf, *invu, *x0d, *gth, *gtl, *Yh, *Yl;
  double2* chi64;
  int* piv_s;
};

__device__ __forceinline__ MixedPtrs mixed_ptrs(float2* smf, int np, int* piv_s) {
  const MixedSmem L = mixed_layout(np);
  MixedPtrs m;
  m.X0s = smf + L.x0;
  m.chih = smf + L.chih;
  m.chil = smf + L.chil;
  m.ubuf = smf + L.ubuf;
  m.lbuf = smf + L.lbuf;
  m.invu = smf + L.invu;
  m.x0d = smf + L.x0d;
  m.gth = smf + L.gt_h;
  m.gtl = smf + L.gt_l;
  m.Yh = smf + L.yh;
  m.Yl = smf + L.yl;
  m.chi64 = (double2*)(smf + L.chi64);
  m.piv_s = piv_s;
  return m;
}

// One (q, W, channel) ladder in mixed precision; all P*P threads of the
// block (P = np / 4) must call it.  Writes kc[c][a][:][q].
__device__ __forceinline__ void bse_mixed_system(const Dims& dm, int c, int a, int q, int np,
                                                 const double2* __restrict__ gam,
                                                 const float2* __restrict__ gam_hi,
                                                 const float2* __restrict__ gam_lo,
                                                 const double2* __restrict__ gg,
                                                 const double2* __restrict__ chi, double2* __restrict__ kc,
                                                 int* __restrict__ flags, const MixedPtrs& sp) {
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  const int P = np / kTile;
  float2* X0s = sp.X0s;
  float2* chih = sp.chih;
  float2* chil = sp.chil;
  float2* ubuf = sp.ubuf;
  float2* lbuf = sp.lbuf;
  float2* invu = sp.invu;
  float2* x0d = sp.x0d;
  float2* gth = sp.gth;
  float2* gtl = sp.gtl;
  float2* Yh = sp.Yh;
  float2* Yl = sp.Yl;
  int* piv_s = sp.piv_s;
  const int t = threadIdx.x;
  const int tr = t % P, tc = t / P;
  const size_t mat = ((size_t)c * nb + a) * n * n;
  const float2* Gh = gam_hi + mat;
  const float2* Gl = gam_lo + mat;

  for (int i = t; i < np; i += blockDim.x) {
    double2 x = (i < n) ? chi[((size_t)a * n + i) * N + q] : mk(0.0, 0.0);
    const float hx = (float)x.x, hy = (float)x.y;
    chih[i] = make_float2(hx, hy);
    chil[i] = make_float2((float)(x.x - (double)hx), (float)(x.y - (double)hy));
    sp.chi64[i] = x;
  }
  __syncthreads();

  // ---- load [D | gamma] (FP32) into registers ----
  float2 A[kTile][2 * kTile];
  int rowpos[kTile];
#pragma unroll
  for (int ii = 0; ii < kTile; ++ii) {
    const int r = tr + P * ii;
    rowpos[ii] = -1;
#pragma unroll
    for (int jj = 0; jj < kTile; ++jj) {
      const int col = tc + P * jj;
      // D = 1 - gamma chi~ formed in FP64 and rounded once: the diagonal
      // 1 - gamma_ww chi~_w cancels when |gamma chi~| >> |D|, and a product of
      // FP32-rounded factors would lose those digits
      const bool in = (r < n && col < n);
      const double2 g64 = in ? gam[mat + (size_t)r * n + col] : mk(0.0, 0.0);
      const double2 z = cmul(g64, sp.chi64[col]);
      A[ii][jj] = make_float2((float)((r == col ? 1.0 : 0.0) - z.x), (float)(-z.y));
      A[ii][kTile + jj] = in ? Gh[r * n + col] : make_float2(0.f, 0.f);
    }
  }

  // ---- elimination with implicit partial pivoting; RHS forward-substituted ----
  // k = jk P + kk: jk (the register column of pivot column k) is a
  // compile-time index after unrolling; the P owners of column k are the
  // consecutive, P-aligned threads tc == kk and reduce the pivot by shuffles.
  const unsigned gmask = (P >= 32) ? 0xffffffffu : (((1u << P) - 1u) << ((t & 31) & ~(P - 1)));
#pragma unroll
  for (int jk = 0; jk < kTile; ++jk) {
    for (int kk = 0; kk < P; ++kk) {
      const int k = jk * P + kk;
      const bool own_col = (tc == kk);
      if (own_col) {
        float best = -1.f;
        int br = 0x7fffffff;
        float2 bv = make_float2(0.f, 0.f);
#pragma unroll
        for (int ii = 0; ii < kTile; ++ii) {
          if (rowpos[ii] < 0) {
            const float2 v = A[ii][jk];
            const float m = fabsf(v.x) + fabsf(v.y);
            const int r = tr + P * ii;
            if (m > best || (m == best && r < br)) { best = m; br = r; bv = v; }
          }
        }
        for (int o = P >> 1; o > 0; o >>= 1) {
          const float ob = __shfl_xor_sync(gmask, best, o);
          const int orr = __shfl_xor_sync(gmask, br, o);
          const float ox = __shfl_xor_sync(gmask, bv.x, o);
          const float oy = __shfl_xor_sync(gmask, bv.y, o);
          if (ob > best || (ob == best && orr < br)) { best = ob; br = orr; bv = make_float2(ox, oy); }
        }
        if (tr == 0) {
          const bool singular = (bv.x == 0.f && bv.y == 0.f);
          piv_s[k] = br;
          invu[k] = singular ? make_float2(0.f, 0.f) : cinvf(bv);
          if (singular) atomicOr(flags, 1);
        }
      }
      __syncthreads();
      const int p = piv_s[k];
      const float2 inv = invu[k];
      if (tr == p % P) {
        const int ip = p / P;
#pragma unroll
        for (int ii = 0; ii < kTile; ++ii) {
          if (ii == ip) {
            rowpos[ii] = k;
#pragma unroll
            for (int jj = 0; jj < kTile; ++jj) {
              if (jj > jk || (jj == jk && tc > kk)) ubuf[tc + P * jj] = A[ii][jj];
              ubuf[np + tc + P * jj] = A[ii][kTile + jj];
            }
          }
        }
      }
      if (own_col) {
#pragma unroll
        for (int ii = 0; ii < kTile; ++ii) {
          if (rowpos[ii] < 0) {
            const float2 l = cmulf(A[ii][jk], inv);
            A[ii][jk] = l;
            lbuf[tr + P * ii] = l;
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int ii = 0; ii < kTile; ++ii) {
        if (rowpos[ii] < 0) {
          const float2 l = lbuf[tr + P * ii];
#pragma unroll
          for (int jj = 0; jj < kTile; ++jj) {
            if (jj > jk || (jj == jk && tc > kk)) A[ii][jj] = cfmsf(l, ubuf[tc + P * jj], A[ii][jj]);
            A[ii][kTile + jj] = cfmsf(l, ubuf[np + tc + P * jj], A[ii][kTile + jj]);
          }
        }
      }
    }
  }

  __syncthreads();   // the last elimination update still reads lbuf / ubuf

  // ---- back substitution: X0 row k (logical) from physical row piv[k] ----
#pragma unroll
  for (int jk = kTile - 1; jk >= 0; --jk) {
    for (int kk = P - 1; kk >= 0; --kk) {
      const int k = jk * P + kk;
      const int p = piv_s[k];
      float2* ucol = lbuf + (k & 1) * np;
      if (tc == kk) {
#pragma unroll
        for (int ii = 0; ii < kTile; ++ii) ucol[tr + P * ii] = A[ii][jk];
      }
      if (tr == p % P) {
        const int ip = p / P;
        const float2 inv = invu[k];
#pragma unroll
        for (int ii = 0; ii < kTile; ++ii)
          if (ii == ip)
#pragma unroll
            for (int jj = 0; jj < kTile; ++jj) X0s[k * np + tc + P * jj] = cmulf(A[ii][kTile + jj], inv);
      }
      __syncthreads();
#pragma unroll
      for (int ii = 0; ii < kTile; ++ii) {
        if (rowpos[ii] < k) {
          const float2 u = ucol[tr + P * ii];
#pragma unroll
          for (int jj = 0; jj < kTile; ++jj)
            A[ii][kTile + jj] = cfmsf(u, X0s[k * np + tc + P * jj], A[ii][kTile + jj]);
        }
      }
    }
  }
  __syncthreads();
  for (int j = t; j < np; j += blockDim.x) x0d[j] = X0s[j * np + j];
  // Y = chi o X0 as double-float pairs, once per system
  for (int idx = t; idx < np * np; idx += blockDim.x) {
    const int l = idx / np;
    const float2 xh = chih[l], xl = chil[l];
    const float2 x = X0s[idx];
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    df_fma(rh, rl, xh.x, x.x);
    df_fma(rh, rl, -xh.y, x.y);
    df_fma(ih, il, xh.x, x.y);
    df_fma(ih, il, xh.y, x.x);
    rl = fmaf(xl.x, x.x, fmaf(-xl.y, x.y, rl));
    il = fmaf(xl.x, x.y, fmaf(xl.y, x.x, il));
    float sv, ev;
    two_sum(rh, rl, sv, ev); rh = sv; rl = ev;
    two_sum(ih, il, sv, ev); ih = sv; il = ev;
    Yh[idx] = make_float2(rh, ih);
    Yl[idx] = make_float2(rl, il);
  }

  // ---- residual R = gamma - X0 + gamma (chi o X0), ~48-bit accurate ----
  const int lc = np < kResChunk ? np : kResChunk;   // gamma columns per staged tile (divides np)
  // two passes of 2 rows each keep the double-float accumulators in registers
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float acc[2][kTile][6];   // [row][col][re_hi, re_lo, im_hi, im_lo, re_small, im_small]
#pragma unroll
    for (int i2 = 0; i2 < 2; ++i2)
#pragma unroll
      for (int jj = 0; jj < kTile; ++jj)
#pragma unroll
        for (int e = 0; e < 6; ++e) acc[i2][jj][e] = 0.f;
    for (int l0 = 0; l0 < np; l0 += lc) {
      __syncthreads();
      for (int idx = t; idx < lc * np; idx += blockDim.x) {
        const int r = idx / lc, ll = idx - r * lc;
        const int l = l0 + ll;
        const bool in = (r < n && l < n);
        gth[ll * np + r] = in ? Gh[r * n + l] : make_float2(0.f, 0.f);
        gtl[ll * np + r] = in ? Gl[r * n + l] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      for (int ll = 0; ll < lc; ++ll) {
        const int l = l0 + ll;
        float2 yh[kTile], yl[kTile];
#pragma unroll
        for (int jj = 0; jj < kTile; ++jj) {
          yh[jj] = Yh[l * np + tc + P * jj];
          yl[jj] = Yl[l * np + tc + P * jj];
        }
#pragma unroll
        for (int i2 = 0; i2 < 2; ++i2) {
          const int r = tr + P * (2 * half + i2);
          const float2 gh = gth[ll * np + r], gl = gtl[ll * np + r];
#pragma unroll
          for (int jj = 0; jj < kTile; ++jj) {
            float* ac = acc[i2][jj];
            // real: gh.x yh.x - gh.y yh.y (+ cross terms in lo)
            dd_fma(ac[0], ac[1], gh.x, yh[jj].x);
            dd_fma(ac[0], ac[1], -gh.y, yh[jj].y);
            ac[4] = fmaf(gh.x, yl[jj].x, fmaf(-gh.y, yl[jj].y, ac[4]));
            ac[4] = fmaf(gl.x, yh[jj].x, fmaf(-gl.y, yh[jj].y, ac[4]));
            // imag: gh.x yh.y + gh.y yh.x
            dd_fma(ac[2], ac[3], gh.x, yh[jj].y);
            dd_fma(ac[2], ac[3], gh.y, yh[jj].x);
            ac[5] = fmaf(gh.x, yl[jj].y, fmaf(gh.y, yl[jj].x, ac[5]));
            ac[5] = fmaf(gl.x, yh[jj].y, fmaf(gl.y, yh[jj].x, ac[5]));
          }
        }
      }
    }
    // R = gamma - X0 + acc, in FP64, rounded to FP32 into the RHS registers
#pragma unroll
    for (int i2 = 0; i2 < 2; ++i2) {
      const int ii = 2 * half + i2;
      const int r = tr + P * ii;
#pragma unroll
      for (int jj = 0; jj < kTile; ++jj) {
        const int col = tc + P * jj;
        double2 g = (r < n && col < n) ? gam[mat + (size_t)r * n + col] : mk(0.0, 0.0);
        const float2 x = X0s[r * np + col];
        const double re = g.x - (double)x.x + (((double)acc[i2][jj][0] + (double)acc[i2][jj][1]) + (double)acc[i2][jj][4]);
        const double im = g.y - (double)x.y + (((double)acc[i2][jj][2] + (double)acc[i2][jj][3]) + (double)acc[i2][jj][5]);
        A[ii][kTile + jj] = make_float2((float)re, (float)im);
      }
    }
  }
  __syncthreads();

  // ---- correction E = D^-1 R: forward substitution over the pivot order ----
#pragma unroll
  for (int jk = 0; jk < kTile; ++jk) {
    for (int kk = 0; kk < P; ++kk) {
      const int k = jk * P + kk;
      const int p = piv_s[k];
      float2* yrow = ubuf + (k & 1) * np;
      float2* lcol = lbuf + (k & 1) * np;
      if (tr == p % P) {
        const int ip = p / P;
#pragma unroll
        for (int ii = 0; ii < kTile; ++ii)
          if (ii == ip)
#pragma unroll
            for (int jj = 0; jj < kTile; ++jj) yrow[tc + P * jj] = A[ii][kTile + jj];
      }
      if (tc == kk) {
#pragma unroll
        for (int ii = 0; ii < kTile; ++ii) lcol[tr + P * ii] = A[ii][jk];
      }
      __syncthreads();
#pragma unroll
      for (int ii = 0; ii < kTile; ++ii) {
        if (rowpos[ii] > k) {
          const float2 l = lcol[tr + P * ii];
#pragma unroll
          for (int jj = 0; jj < kTile; ++jj)
            A[ii][kTile + jj] = cfmsf(l, yrow[tc + P * jj], A[ii][kTile + jj]);
        }
      }
    }
  }
  __syncthreads();
  // back substitution (X0s reused as the row broadcast)
#pragma unroll
  for (int jk = kTile - 1; jk >= 0; --jk) {
    for (int kk = P - 1; kk >= 0; --kk) {
      const int k = jk * P + kk;
      const int p = piv_s[k];
      float2* ucol = lbuf + (k & 1) * np;
      if (tc == kk) {
#pragma unroll
        for (int ii = 0; ii < kTile; ++ii) ucol[tr + P * ii] = A[ii][jk];
      }
      if (tr == p % P) {
        const int ip = p / P;
        const float2 inv = invu[k];
#pragma unroll
        for (int ii = 0; ii < kTile; ++ii)
          if (ii == ip)
#pragma unroll
            for (int jj = 0; jj < kTile; ++jj) X0s[k * np + tc + P * jj] = cmulf(A[ii][kTile + jj], inv);
      }
      __syncthreads();
#pragma unroll
      for (int ii = 0; ii < kTile; ++ii) {
        if (rowpos[ii] < k) {
          const float2 u = ucol[tr + P * ii];
#pragma unroll
          for (int jj = 0; jj < kTile; ++jj)
            A[ii][kTile + jj] = cfmsf(u, X0s[k * np + tc + P * jj], A[ii][kTile + jj]);
        }
      }
    }
  }
  __syncthreads();

  // ---- diag Gamma = diag X0 + diag E (FP64), Gamma^(2), Eq. sd bracket ----
  const double2* GG = gg + mat;
  // four threads per output frequency j (consecutive lanes, shuffle-reduced)
  // when the block has whole warps; one thread per j otherwise
  const int per_j = (blockDim.x >= 32) ? 4 : 1;
  for (int base = 0; base < per_j * np; base += blockDim.x) {
    const int idx = base + t;
    const int j = idx / per_j, part = idx % per_j;
    double2 g2 = mk(0.0, 0.0);
    if (j < n) {
      for (int x = part; x < n; x += per_j) {
        const double2 cx = mk((double)chih[x].x + (double)chil[x].x, (double)chih[x].y + (double)chil[x].y);
        g2 = cfma(GG[(size_t)j * n + x], cx, g2);
      }
    }
    if (per_j == 4) {
      g2.x += __shfl_xor_sync(0xffffffffu, g2.x, 1);
      g2.y += __shfl_xor_sync(0xffffffffu, g2.y, 1);
      g2.x += __shfl_xor_sync(0xffffffffu, g2.x, 2);
      g2.y += __shfl_xor_sync(0xffffffffu, g2.y, 2);
    }
    if (j < n && part == 0) {
      const float2 x0 = x0d[j], e = X0s[j * np + j];
      const double2 gdiag = mk((double)x0.x + (double)e.x, (double)x0.y + (double)e.y);
      const double wgt = (c == 0) ? 1.0 : 3.0;
      kc[(((size_t)c * nb + a) * n + j) * N + q] =
          mk(wgt * (gdiag.x - 0.5 * g2.x), wgt * (gdiag.y - 0.5 * g2.y));
    }
  }
  __syncthreads();
}

}  // namespace df
