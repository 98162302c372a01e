// DF_FP32_IR ladder solve of order 64 < n <= 96 with both the Gauss-Jordan
// inversion and the residual on the tensor cores (one (q, W, channel) ladder
// per pass of a block; used by bse_tcr_kernel in df_mixed_large.cu).
//
// Eq. lin_alg_inv, D Gamma = gamma with D = 1 - gamma diag(chi~):
//   1. [D | gamma] into tensor memory, transposed (lane j = column j, TMEM
//      column 2i + c = row i): D in double-float rounded once to FP32,
//      gamma's FP32 leading words.  TMEM: D at columns [0, 2 np), gamma at
//      [2 np, 4 np), the residual's accumulators at [4 np, 4 np + 128)
//      (np = tc_pad(n) <= 96: 512 columns, one block per SM).
//   2. The tensor-core Gauss-Jordan sweep (df_tcgj_dev.cuh) over D with the
//      gamma columns as a second region: D becomes A with A[p_k][j] =
//      D^-1[k][p_j], gamma becomes G with G[p_k][m] = X0[k][m], X0 ~ D^-1 gamma
//      (FP32-accurate).
//   3. R = gamma - D X0 = gamma - X0 + gamma Y, Y = chi~ o X0, in column blocks
//      of kTcrCB = 8: Y in double-float, cut into 8 signed base-128 digits
//      relative to a power of two per column; gamma's digits (8 per value,
//      relative to a power of two per row, cut once per input upload) are
//      streamed from global memory one (row tile, slice) chunk at a time by
//      bulk asynchronous copies into two shared-memory buffers.  For gamma
//      slice s one MMA per K step of 16 takes A = the chunk ([gamma_re rows;
//      gamma_im rows] of a 64-row tile, M = 128) and B = the Y slices 0 .. 7-s
//      stacked along N (16 rows each: the block's Y_re then Y_im columns),
//      D at accumulator column 16 s, so that Y slice t lands in group d = s+t
//      (weight 2^-7(d+2)).  Each group's FP32 sum is exact (<= 8 pairs x 96 x
//      127^2 < 2^24); the 36 pairs with weight >= 2^-63 are formed.  The
//      groups are folded into a double-float sum, scaled by the row and column
//      powers of two, the gamma_im rows' products exchanged through shared
//      memory, and R = gamma - X0 + gamma Y assembled in double-float.
//   4. Gamma_mm = X0_mm + sum_j D^-1[m][j] R[j][m] (FP32 products with A's row
//      p_m read from TMEM), Gamma^(2)_mm in FP64, the Eq. sd bracket, and the
//      per-ladder error control of the correction's size.
#pragma once
#include "df_tcgj_dev.cuh"

namespace df {

constexpr int kTcrCB = 8;            // right-hand-side columns per residual block
constexpr int kTcrMaxNp = 96;        // largest padded order: 4 np + 128 TMEM columns <= 512
constexpr int kTcrChunk = 128 * 2 * 128;   // one gamma digit chunk: 128 rows x 2 K-atoms x 128 bytes

__host__ __device__ constexpr bool tcr_supported(int n) { return n > 64 && tc_pad(n) <= kTcrMaxNp; }

// bytes of gamma's digit chunks of one (channel, W) matrix: 2 row tiles x 8 slices
__host__ __device__ constexpr size_t tcr_gdig_bytes() { return (size_t)2 * kSlices * kTcrChunk; }

struct TcrLayout {
  int sweep, gbuf, ystk, x0b, rb, ex, xs, xh, xl, cole, rowe, red, g2, total;   // byte offsets
};
__host__ __device__ inline TcrLayout tcr_layout(int n) {
  TcrLayout L;
  int off = 0;
  auto take = [&](int bytes, int align) {
    off = (off + align - 1) / align * align;
    const int o = off;
    off += bytes;
    return o;
  };
  // the sweep's tiles, then (1024-aligned) the right-hand sides' A tile
  // (at least two gamma chunks: the residual's buffers 2 and 3 reuse it)
  const int sw = (tc_smem_bytes(n) + 1023) / 1024 * 1024 + 128 * 128;
  L.sweep = take(sw > 2 * kTcrChunk ? sw : 2 * kTcrChunk, 1024);
  L.gbuf = take(2 * kTcrChunk, 1024);                   // two gamma digit chunks
  L.ystk = take(128 * 2 * 128, 1024);                   // Y digits: 8 slices x 16 rows x 2 K-atoms
  L.x0b = take(8 * n * kTcrCB, 16);                     // X0 of the block's columns [n][8]
  L.rb = take(8 * n * kTcrCB, 16);                      // R of the block's columns [n][8]
  L.ex = take(4 * 2 * 64 * (kTcrCB + 1) * 2, 16);      // exchange of the gamma_im rows' products
  L.xs = take(16 * n, 16);
  L.xh = take(8 * n, 16);
  L.xl = take(8 * n, 16);
  L.cole = take(4 * kTcrCB, 16);
  L.rowe = take(4 * 128, 16);
  L.red = take(4 * 64, 16);
  L.g2 = take(16 * n, 16);                              // Gamma^(2)_mm of the ladder (FP64)
  L.total = off;
  return L;
}

constexpr int kTcrBufs = 4;          // gamma chunks in flight (two in their own space, two over the sweep's tiles)

struct TcrState {
  unsigned tmem;          // TMEM base (512 columns)
  uint64_t* mbar;         // sweep / fold completion barrier
  uint64_t* full;         // [kTcrBufs] gamma chunk arrived
  uint64_t* empty;        // [kTcrBufs] the MMAs that read a chunk completed
  unsigned phase, fphase[kTcrBufs], ephase[kTcrBufs];
};

__device__ __forceinline__ void bulk_copy_g2s(unsigned dst, const void* src, unsigned bytes, uint64_t* mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(unsigned taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "r"(taddr)
      : "memory");
}

// One ladder.  All kTcThreads threads call it; returns false when a bounded
// tensor-core wait gave up (the same in every thread).
// ghi, glo: gamma's FP32 (hi, lo) words [2][nb][n][n]; gg: gamma o gamma^T
// (FP64); gdig: gamma's digit chunks [2][nb][2 tiles][8 slices][kTcrChunk],
// growe: their row exponents [2][nb][2 tiles][128]; chi: chi~ [nb][n][N];
// kc: the Eq. sd bracket [2][nb][n][N]
__device__ __forceinline__ bool tcr_system(const Dims& dm, int c, int a, int q, const float2* __restrict__ ghi,
                                           const float2* __restrict__ glo, const double2* __restrict__ gg,
                                           const unsigned char* __restrict__ gdig, const int* __restrict__ growe,
                                           const double2* __restrict__ chi, double2* __restrict__ kc,
                                           int* __restrict__ flags, unsigned char* smem, int* piv, int* ipiv,
                                           TcrState& st, const MixedCheck& mc) {
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  const int np = tc_pad(n), ksteps = (n + 15) / 16;
  const TcrLayout L = tcr_layout(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, qd = warp & 3;
  const int jl = 32 * qd + lane;                 // this thread's TMEM lane
  const unsigned tA = st.tmem, tG = st.tmem + 2 * np, tR = st.tmem + 4 * np;
  const unsigned lq = (32u * qd) << 16;
  const size_t mat = ((size_t)c * nb + a) * n * n;
  const float2* Gh = ghi + mat;
  const float2* Gl = glo + mat;
  const unsigned char* GD = gdig + ((size_t)c * nb + a) * tcr_gdig_bytes();
  const int* GE = growe + ((size_t)c * nb + a) * 2 * 128;
  float2* x0b = reinterpret_cast<float2*>(smem + L.x0b);
  float2* rb = reinterpret_cast<float2*>(smem + L.rb);
  float2* ex = reinterpret_cast<float2*>(smem + L.ex);
  double2* xs = reinterpret_cast<double2*>(smem + L.xs);
  float2* xh = reinterpret_cast<float2*>(smem + L.xh);
  float2* xl = reinterpret_cast<float2*>(smem + L.xl);
  int* cole = reinterpret_cast<int*>(smem + L.cole);
  int* rowe = reinterpret_cast<int*>(smem + L.rowe);
  float* red = reinterpret_cast<float*>(smem + L.red);
  unsigned* yw = reinterpret_cast<unsigned*>(smem + L.ystk);
  const unsigned gbuf0 = smem_u32(smem + L.gbuf), ystk = smem_u32(smem + L.ystk);

  for (int i = tid; i < n; i += kTcThreads) {
    const double2 v = chi[((size_t)a * n + i) * N + q];
    xs[i] = v;
    const float hx = (float)v.x, hy = (float)v.y;
    xh[i] = make_float2(hx, hy);
    xl[i] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
  }
  if (tid < 4) red[tid] = 0.f;                   // [0] max |correction|, [1] max |Gamma_mm| (float bits), [2] bad
  __syncthreads();
  // 1. [D | gamma] into TMEM
  tc05_fence_after();
  {
    const float2 ah = jl < n ? xh[jl] : make_float2(0.f, 0.f), al = jl < n ? xl[jl] : make_float2(0.f, 0.f);
    for (int r = 8 * (warp >> 2); r < np; r += 16) {
      float v[16], g[16];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = r + e;
        float2 d = make_float2(0.f, 0.f), gv = make_float2(0.f, 0.f);
        if (i < n && jl < n) {
          const float2 h = __ldg(Gh + (size_t)i * n + jl);
          float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
          cdf_fma(sr, lr, si, li, h, __ldg(Gl + (size_t)i * n + jl), ah, al);
          d = make_float2(((i == jl ? 1.f : 0.f) - sr) - lr, -si - li);
          gv = h;
        }
        v[2 * e] = d.x;
        v[2 * e + 1] = d.y;
        g[2 * e] = gv.x;
        g[2 * e + 1] = gv.y;
      }
      tmem_st16(tA + lq + 2 * r, v);
      tmem_st16(tG + lq + 2 * r, g);
    }
    tmem_wait_st();
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  // 2. the sweep of [D | gamma]
  {
    const TcGjSmem sw = tc_smem(smem + L.sweep, n);
    __nv_bfloat16* atg = reinterpret_cast<__nv_bfloat16*>(smem + L.sweep + (tc_smem_bytes(n) + 1023) / 1024 * 1024);
    if (!tcgj_sweep(tA, n, n, sw, piv, st.mbar, st.phase, flags, tG, n, atg)) return false;
  }
  for (int k = tid; k < n; k += kTcThreads) ipiv[piv[k]] = k;
  __syncthreads();
  const int fh_half = warp >> 2;  // fold: warp w reads lane quadrant w % 4, column half w / 4
  double2* g2s = reinterpret_cast<double2*>(smem + L.g2);
  // Gamma^(2)_mm = sum_x gamma_mx gamma_xm chi~_x, every m of the ladder (warp w: m = w + 8 i),
  // in double-float from gamma's and chi~'s (hi, lo) words (the FP64 pipe runs at 1/64 of FP32)
  for (int m = warp; m < n; m += kTcThreads / 32) {
    float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
    for (int x = lane; x < n; x += 32) {
      float pr = 0.f, plr = 0.f, pi = 0.f, pli = 0.f;
      cdf_fma(pr, plr, pi, pli, __ldg(Gh + (size_t)m * n + x), __ldg(Gl + (size_t)m * n + x),
              __ldg(Gh + (size_t)x * n + m), __ldg(Gl + (size_t)x * n + m));
      cdf_fma(sr, lr, si, li, make_float2(pr, pi), make_float2(plr, pli), xh[x], xl[x]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float osr = __shfl_xor_sync(0xffffffffu, sr, o), olr = __shfl_xor_sync(0xffffffffu, lr, o);
      const float osi = __shfl_xor_sync(0xffffffffu, si, o), oli = __shfl_xor_sync(0xffffffffu, li, o);
      df_add(sr, lr, osr);
      lr += olr;
      df_add(si, li, osi);
      li += oli;
    }
    if (lane == 0) g2s[m] = mk((double)sr + (double)lr, (double)si + (double)li);
  }
  // gamma's digit chunks in the order (column block, row tile, slice), kTcrBufs
  // buffers in flight; thread 0 loads and issues (buffers 0, 1 own space; 2, 3
  // over the sweep's tiles, free from here to the end of the ladder)
  const int nblk = (n + kTcrCB - 1) / kTcrCB, total = nblk * 2 * kSlices;
  int gload = 0, gmma = 0, gfree = 0;
  auto buf_addr = [&](int g) -> unsigned {
    const int b = g % kTcrBufs;
    return b < 2 ? gbuf0 + b * kTcrChunk : smem_u32(smem + L.sweep) + (b - 2) * kTcrChunk;
  };
  // (thread 0) issue loads while fewer than `ahead` chunks past gmma are loaded;
  // a buffer is reused once the MMAs of the chunk before it completed
  auto load_ahead = [&](int ahead) -> bool {
    while (gload < total && gload < gmma + ahead) {
      if (gload >= kTcrBufs) {
        const int gb = gload - kTcrBufs;           // the chunk that last used this buffer
        while (gfree <= gb) {
          const int fb = gfree % kTcrBufs;
          if (!mbar_wait(&st.empty[fb], st.ephase[fb])) return false;
          st.ephase[fb] ^= 1u;
          ++gfree;
        }
      }
      const int blk = gload / (2 * kSlices), T = (gload / kSlices) & 1, sl = gload % kSlices;
      (void)blk;
      bulk_copy_g2s(buf_addr(gload), GD + ((size_t)T * kSlices + sl) * kTcrChunk, kTcrChunk,
                    &st.full[gload % kTcrBufs]);
      ++gload;
    }
    return true;
  };
  if (tid == 0) {
    tc05_fence_after();
    if (!load_ahead(kTcrBufs)) red[3] = 1.f;
  }
  // 3-4. residual and correction, kTcrCB columns at a time
  for (int m0 = 0; m0 < n; m0 += kTcrCB) {
    const int wcols = min(kTcrCB, n - m0);
    // X0 of the block: lanes m0 .. m0 + 7 of region G, row r of G is row ipiv[r] of X0
    if (qd == (m0 >> 5)) {
      const int r0 = warp < 4 ? 0 : np / 2, r1 = warp < 4 ? np / 2 : np;
      const int ml = jl - m0;
      for (int r = r0; r < r1; r += 8) {
        float v[16];
        tmem_ld16(tG + lq + 2 * r, v);
        if (ml >= 0 && ml < kTcrCB) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (r + e < n && (unsigned)ipiv[r + e] < (unsigned)n)
              x0b[ipiv[r + e] * kTcrCB + ml] = (m0 + ml < n) ? make_float2(v[2 * e], v[2 * e + 1])
                                                             : make_float2(0.f, 0.f);
        }
      }
    }
    if (tid < kTcrCB) cole[tid] = -1000;
    tc05_fence_before();
    __syncthreads();
    // Y = chi~ o X0 (double-float) for the item (k pair, column): its column exponent
    const int nitems = (n / 2) * kTcrCB;
    float y[2][2][4];                             // [item][row of the pair][re hi, re lo, im hi, im lo]
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int item = tid + kTcThreads * it;
      float mx = 0.f;
      if (item < nitems) {
        const int ml = item % kTcrCB, k = 2 * (item / kTcrCB);
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const float2 x = x0b[(k + rr) * kTcrCB + ml];
          y[it][rr][0] = y[it][rr][1] = y[it][rr][2] = y[it][rr][3] = 0.f;
          cdf_fma(y[it][rr][0], y[it][rr][1], y[it][rr][2], y[it][rr][3], xh[k + rr], xl[k + rr], x,
                  make_float2(0.f, 0.f));
          mx = fmaxf(mx, fmaxf(fabsf(y[it][rr][0]), fabsf(y[it][rr][2])));
        }
        mx *= 1.0001f;
        if (mx > 0.f) atomicMax(&cole[ml], exp_bound_f32(mx));
      }
    }
    __syncthreads();
    // Y's digits into the stacked B operand: slice t, row 16 t + (re: ml, im: 8 + ml), K = k
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int item = tid + kTcThreads * it;
      if (item < nitems) {
        const int ml = item % kTcrCB, k = 2 * (item / kTcrCB);
        const int e = cole[ml];
        unsigned r0d[kSlices], r1d[kSlices], i0d[kSlices], i1d[kSlices];
        if (e > -1000) {
          digits_pair_f(y[it][0][0], y[it][0][1], e, r0d);
          digits_pair_f(y[it][1][0], y[it][1][1], e, r1d);
          digits_pair_f(y[it][0][2], y[it][0][3], e, i0d);
          digits_pair_f(y[it][1][2], y[it][1][3], e, i1d);
        } else {
#pragma unroll
          for (int t = 0; t < kSlices; ++t) r0d[t] = r1d[t] = i0d[t] = i1d[t] = 0u;
        }
        const int atom = k >> 6, kk = k & 63;
#pragma unroll
        for (int t = 0; t < kSlices; ++t) {
          yw[(atom * 128 * 64 + swz(16 * t + ml, kk)) >> 1] = pack_bf16_hi(r0d[t], r1d[t]);
          yw[(atom * 128 * 64 + swz(16 * t + 8 + ml, kk)) >> 1] = pack_bf16_hi(i0d[t], i1d[t]);
        }
      }
    }
    fence_async_smem();
    tc05_fence_before();
    __syncthreads();
    // two row tiles of gamma: rows 64 T .. 64 T + 63 (re at lanes 0-63, im at 64-127)
    for (int T = 0; T < 2; ++T) {
      if (tid == 0 && red[3] == 0.f) {
        tc05_fence_after();
        bool ok = true;
        for (int sl = 0; sl < kSlices && ok; ++sl) {
          const int g = gmma, b = g % kTcrBufs;
          ok = mbar_wait(&st.full[b], st.fphase[b]);
          st.fphase[b] ^= 1u;
          if (!ok) break;
          tc05_fence_after();
          const unsigned abuf = buf_addr(g);
          const unsigned idesc = umma_idesc_bf16(128, 16 * (kSlices - sl));
          for (int ks = 0; ks < ksteps; ++ks) {
            const unsigned koff = (unsigned)((ks >> 2) * 128 * 128 + 32 * (ks & 3));
            umma_bf16(tR + 16 * sl, umma_desc_sw128(abuf + koff), umma_desc_sw128(ystk + koff), idesc,
                      (sl > 0 || ks > 0) ? 1u : 0u);
          }
          umma_commit(&st.empty[b]);
          ++gmma;
          ok = load_ahead(kTcrBufs - 1);         // the next chunks fly while these MMAs run
        }
        if (ok) umma_commit(st.mbar);
        else atomicOr(flags, kFlagTcTimeout);
        red[3] = ok ? 0.f : 1.f;
      }
      // the row exponents of this tile (lane order)
      if (tid < 128) rowe[tid] = GE[T * 128 + tid];
      __syncthreads();
      if (red[3] != 0.f) return false;
      const bool done = mbar_wait(st.mbar, st.phase);
      st.phase ^= 1u;
      tc05_fence_after();
      if (__syncthreads_or(!done)) {
        if (tid == 0) atomicOr(flags, kFlagTcTimeout);
        return false;
      }
      // fold: lane row i (gamma_re rows at quadrants 0-1, gamma_im at 2-3), half h = Y_re / Y_im
      {
        const unsigned tl = tR + lq + (unsigned)(8 * fh_half);
        float fh[kTcrCB], fl[kTcrCB], v[kTcrCB];
        tmem_ld8(tl + 16 * 7, fh);
#pragma unroll
        for (int d = 6; d >= 4; --d) {
          tmem_ld8(tl + 16 * d, v);
#pragma unroll
          for (int c2 = 0; c2 < kTcrCB; ++c2) fh[c2] = fmaf(fh[c2], 0.0078125f, v[c2]);
        }
#pragma unroll
        for (int c2 = 0; c2 < kTcrCB; ++c2) {
          fh[c2] *= 3.7252902984619141e-09f;      // 2^-28
          fl[c2] = 0.f;
        }
#pragma unroll
        for (int d = 3; d >= 0; --d) {
          tmem_ld8(tl + 16 * d, v);
          const float sc = __int_as_float((127 - 7 * d) << 23);     // 2^-7d
#pragma unroll
          for (int c2 = 0; c2 < kTcrCB; ++c2) dd_add(fh[c2], fl[c2], v[c2] * sc);
        }
        const int ei = rowe[jl];
#pragma unroll
        for (int c2 = 0; c2 < kTcrCB; ++c2) {
          const int ej = cole[c2];
          const float w = (ei > -1000 && ej > -1000) ? pow2f(ei + ej - 14) : 0.f;
          fh[c2] *= w;
          fl[c2] *= w;
        }
        // the gamma_im rows' products: (im x Y_re) -> imaginary part, (im x Y_im) -> real part, negated
        const bool zi = qd >= 2;
        const int il = jl & 63;
        if (zi) {
          const float sg = fh_half ? -1.f : 1.f;
          float2* eo = ex + ((1 - fh_half) * 64 + il) * (kTcrCB + 1);
#pragma unroll
          for (int c2 = 0; c2 < kTcrCB; ++c2) eo[c2] = make_float2(sg * fh[c2], sg * fl[c2]);
        }
        tc05_fence_before();
        __syncthreads();
        if (!zi) {
          float2* eo = ex + (fh_half * 64 + il) * (kTcrCB + 1);
#pragma unroll
          for (int c2 = 0; c2 < kTcrCB; ++c2) {
            const float2 o = eo[c2];
            float sh, se;
            two_sum(fh[c2], o.x, sh, se);
            eo[c2] = make_float2(sh, se + (fl[c2] + o.y));
          }
        }
        __syncthreads();
        // R = gamma - X0 + S in double-float, rows of this tile
        for (int e2 = tid; e2 < 64 * kTcrCB; e2 += kTcThreads) {
          const int il2 = e2 / kTcrCB, ml = e2 - il2 * kTcrCB, i = 64 * T + il2, m = m0 + ml;
          if (i < n) {
            float2 r = make_float2(0.f, 0.f);
            if (ml < wcols) {
              const float2 gh = __ldg(Gh + (size_t)i * n + m), gl2 = __ldg(Gl + (size_t)i * n + m);
              const float2 x = x0b[i * kTcrCB + ml];
              const float2 sr = ex[il2 * (kTcrCB + 1) + ml], si = ex[(64 + il2) * (kTcrCB + 1) + ml];
              float re = gh.x, rl = gl2.x, im = gh.y, imlo = gl2.y;
              df_add(re, rl, -x.x);
              df_add(re, rl, sr.x);
              df_add(im, imlo, -x.y);
              df_add(im, imlo, si.x);
              r = make_float2(re + (rl + sr.y), im + (imlo + si.y));
            }
            rb[i * kTcrCB + ml] = r;
          }
        }
        __syncthreads();
      }
    }
    // Gamma_mm = X0_mm + sum_j A[p_m][j] R[p_j][m] for the block's columns: warps
    // 0-3 columns 0-3, warps 4-7 columns 4-7; lane j of A's row p_m from TMEM
    {
      const int grp = warp >> 2;
      float2 part[4];
      float ax[4], ay[4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int ml = 4 * grp + cc;
        const int m = m0 + (ml < wcols ? ml : 0);
        tmem_ld_x2(tA + lq + 2 * piv[m], ax[cc], ay[cc]);
      }
      tmem_wait_ld();
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int ml = 4 * grp + cc;
        part[cc] = (jl < n && ml < wcols) ? cmulf(make_float2(ax[cc], ay[cc]), rb[piv[jl] * kTcrCB + ml])
                                          : make_float2(0.f, 0.f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          part[cc].x += __shfl_xor_sync(0xffffffffu, part[cc].x, o);
          part[cc].y += __shfl_xor_sync(0xffffffffu, part[cc].y, o);
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) ex[(4 * grp + cc) * 4 + qd] = part[cc];
      }
      tc05_fence_before();
      __syncthreads();
      if (tid < wcols) {
        const int ml = tid, m = m0 + ml;
        const float2 corr = (ex[ml * 4 + 0] + ex[ml * 4 + 1]) + (ex[ml * 4 + 2] + ex[ml * 4 + 3]);
        const float2 x0 = x0b[m * kTcrCB + ml];
        const double gx = (double)x0.x + (double)corr.x, gy = (double)x0.y + (double)corr.y;
        const double2 gs = g2s[m];
        const double wgt = (c == 0) ? 1.0 : 3.0;
        kc[(((size_t)c * nb + a) * n + m) * N + q] = mk(wgt * (gx - 0.5 * gs.x), wgt * (gy - 0.5 * gs.y));
        const float ea = fabsf(corr.x) + fabsf(corr.y), ga = (float)(fabs(gx) + fabs(gy));
        if (isfinite(ea) && isfinite(ga)) {
          atomicMax(reinterpret_cast<unsigned*>(&red[0]), __float_as_uint(ea));
          atomicMax(reinterpret_cast<unsigned*>(&red[1]), __float_as_uint(ga));
        } else {
          red[2] = 1.f;
        }
      }
    }
    __syncthreads();
  }
  // the last chunks' MMAs: keep the buffers' parities in step for the next ladder
  if (tid == 0) {
    while (gfree < total) {
      const int fb = gfree % kTcrBufs;
      if (!mbar_wait(&st.empty[fb], st.ephase[fb])) break;
      st.ephase[fb] ^= 1u;
      ++gfree;
    }
  }
  if (tid == 0)
    mixed_check_ladder(mc, red[0], red[1], red[2] == 0.f, ((long)c * nb + a) * N + q, flags);
  __syncthreads();
  return true;
}

}  // namespace df

namespace df {

// gamma's digit chunks for tcr_system, one warp per (matrix, row tile T,
// tile row il): row i = 64 T + il's exponent bound e_i over both parts
// (|gamma_ik| < 2^e_i, -1000 for a zero row) and the 8 digits of each part
// relative to 2^e_i at chunk rows il (real part) and 64 + il (imaginary part),
// K = k in two 64-wide atoms (zero for k >= n and for rows i >= n).
__device__ __forceinline__ void tcr_gamma_digits_rows(int n, int count, const double2* __restrict__ gam,
                                                      unsigned char* __restrict__ out, int* __restrict__ rowe_out,
                                                      int warp_id, int nwarps, int lane) {
  for (int w = warp_id; w < count * 2 * 64; w += nwarps) {
    const int mtx = w / 128, T = (w / 64) & 1, il = w & 63, i = 64 * T + il;
    const double2* G = gam + (size_t)mtx * n * n;
    unsigned char* O = out + (size_t)mtx * tcr_gdig_bytes() + (size_t)T * kSlices * kTcrChunk;
    double m = 0.0;
    if (i < n)
      for (int l = lane; l < n; l += 32) m = fmax(m, fmax(fabs(G[(size_t)i * n + l].x), fabs(G[(size_t)i * n + l].y)));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = -1000;
    if (m > 0.0) frexp(m, &e);
    if (lane == 0) {
      rowe_out[((size_t)mtx * 2 + T) * 128 + il] = e;
      rowe_out[((size_t)mtx * 2 + T) * 128 + 64 + il] = e;
    }
    for (int k = lane; k < 128; k += 32) {
      float dr[kSlices], di[kSlices];
      if (i < n && k < n && e > -1000) {
        digits_f64(G[(size_t)i * n + k].x, e, dr);
        digits_f64(G[(size_t)i * n + k].y, e, di);
      } else {
#pragma unroll
        for (int s = 0; s < kSlices; ++s) dr[s] = di[s] = 0.f;
      }
      const int atom = k >> 6, kk = k & 63;
#pragma unroll
      for (int s = 0; s < kSlices; ++s) {
        __nv_bfloat16* ch = reinterpret_cast<__nv_bfloat16*>(O + (size_t)s * kTcrChunk) + atom * 128 * 64;
        ch[swz(il, kk)] = __float2bfloat16_rn(dr[s]);
        ch[swz(64 + il, kk)] = __float2bfloat16_rn(di[s]);
      }
    }
  }
}

}  // namespace df
