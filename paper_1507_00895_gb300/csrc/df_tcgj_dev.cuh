// Gauss-Jordan inversion of a ladder matrix on the tensor cores (tcgen05):
// the in-place Gauss-Jordan sweep with partial pivoting of Eq. lin_alg_inv's
// D = 1 - gamma diag(chi~), in panels of kTcPanel pivot columns.
//
// The working matrix A (nr rows x nc columns, nc <= 128) lives in tensor
// memory, transposed: TMEM lane j holds column j, TMEM column 2i + c holds
// row i (c = 0 real, 1 imaginary part), FP32.  Rows never move (implicit
// pivoting).  One panel = pivot columns k0 .. k0 + 7:
//   1. the panel's columns (eight lanes) to shared memory;
//   2. the eight Gauss-Jordan steps on the panel alone, on the CUDA cores
//      (warps 0-3, one row per thread in registers; per step one warp max
//      of a pivot key and one 128-thread barrier), giving the panel's new
//      columns P' and its pivot rows p_0 .. p_7;
//   3. the eight steps compose to A <- A + W A[p, :] for every column, with
//      W = P' - [e_p0 .. e_p7]; on the panel's own columns the same product
//      plus W's column (a 1 added to the A operand at that column's own
//      pivot slot) gives P', the in-place storage of the inverse's columns.
//      So the whole update is one real matrix product
//         D[j][(i, c)] += sum_(s, c') Aop[j][(s, c')] Bop[(i, c)][(s, c')],
//      Aop[j] = (re, im) of A[p_s][j] (+1 at the panel's own slot), Bop the
//      2 x 2 real form of W ([re -im; im re]), M = 128, N = 2 n_pad, K = 16,
//      on tcgen05 with the accumulator in TMEM;
//   4. each operand value is split into three BF16 pieces (8 significant
//      bits each, 24 together) and the six products of pieces with weight
//      >= 2^-16 relative are accumulated (hi*hi, hi*mid, mid*hi, hi*lo,
//      mid*mid, lo*hi): the update is FP32-accurate like the CUDA-core sweep.
// At the end A holds D^-1 with rows and columns permuted by the pivots:
// D^-1[k][l] = A[p_k][m] with p_m = l... precisely A[p_k][j] = D^-1[k][p_j].
#pragma once
#include <cuda_bf16.h>

#include "df_mixed_dev.cuh"

namespace df {

constexpr int kTcPanel = 8;          // pivot columns per panel (K = 16 real per BF16 piece)
constexpr int kTcThreads = 256;      // warps 0-3: panel rows, B operand; warps 4-7: A operand
constexpr int kBarTcPanel = 1;       // named barrier of the 128 panel threads

// rows of the working matrix rounded up to 16 (TMEM columns 2 n_pad, a multiple of 32)
__host__ __device__ constexpr int tc_pad(int n) { return (n + 15) / 16 * 16; }

// ---- tensor-memory transfers (warp-collective; warp w reaches lanes 32 (w % 4) + 0..31) ----
__device__ __forceinline__ void tmem_ld_x2(unsigned taddr, float& a, float& b) {
  unsigned r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr) : "memory");
  a = __uint_as_float(r0);
  b = __uint_as_float(r1);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st16(unsigned taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}

// TMEM allocation of a fixed power-of-two column count (warp 0 calls alloc/dealloc)
template <int COLS>
__device__ __forceinline__ void tmem_alloc_cols(unsigned* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "n"(COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int COLS>
__device__ __forceinline__ void tmem_dealloc_cols(unsigned taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(COLS) : "memory");
}

// v ~ h + m + l, three BF16 pieces (round to nearest at each cut: |v - h - m - l| <= 2^-24 |v|)
__device__ __forceinline__ void split3(float v, float& h, float& m, float& l) {
  h = __bfloat162float(__float2bfloat16_rn(v));
  const float r = v - h;
  m = __bfloat162float(__float2bfloat16_rn(r));
  l = __bfloat162float(__float2bfloat16_rn(r - m));
}

// one operand row of 16 values as three BF16 pieces at K 0-15 (hi), 16-31 (mid),
// 32-47 (lo) of a 128-byte-swizzled row (the layout of swz())
__device__ __forceinline__ void put_split_row(__nv_bfloat16* tile, int row, const float* v) {
  unsigned* w = reinterpret_cast<unsigned*>(tile);
#pragma unroll
  for (int k = 0; k < 16; k += 2) {
    float h0, m0, l0, h1, m1, l1;
    split3(v[k], h0, m0, l0);
    split3(v[k + 1], h1, m1, l1);
    const __nv_bfloat162 ph = __floats2bfloat162_rn(h0, h1), pm = __floats2bfloat162_rn(m0, m1),
                         pl = __floats2bfloat162_rn(l0, l1);
    w[swz(row, k) >> 1] = *reinterpret_cast<const unsigned*>(&ph);
    w[swz(row, 16 + k) >> 1] = *reinterpret_cast<const unsigned*>(&pm);
    w[swz(row, 32 + k) >> 1] = *reinterpret_cast<const unsigned*>(&pl);
  }
}

struct TcGjSmem {
  __nv_bfloat16* atile;   // [128][64] 128-byte swizzled, 1024-aligned: the A operand (columns j)
  __nv_bfloat16* btile;   // [2 n_pad][64] the B operand (rows (i, c))
  float2* panel;          // [128][kTcPanel] the panel's columns, row-major
  unsigned* slot_key;     // [2][4] per-warp pivot candidates (step parity, warp)
  float2* slot_row;       // [2][4][kTcPanel] their panel rows
};

__host__ __device__ constexpr int tc_smem_bytes(int n) {
  return 128 * 128 + 2 * tc_pad(n) * 128 + 128 * kTcPanel * 8 + 2 * 4 * 4 + 2 * 4 * kTcPanel * 8;
}
__device__ __forceinline__ TcGjSmem tc_smem(unsigned char* base, int n) {
  TcGjSmem s;
  s.atile = reinterpret_cast<__nv_bfloat16*>(base);
  s.btile = reinterpret_cast<__nv_bfloat16*>(base + 128 * 128);
  s.panel = reinterpret_cast<float2*>(base + 128 * 128 + 2 * tc_pad(n) * 128);
  s.slot_key = reinterpret_cast<unsigned*>(base + 128 * 128 + 2 * tc_pad(n) * 128 + 128 * kTcPanel * 8);
  s.slot_row = reinterpret_cast<float2*>(base + 128 * 128 + 2 * tc_pad(n) * 128 + 128 * kTcPanel * 8 + 32);
  return s;
}

__device__ __forceinline__ void panel_bar() { asm volatile("bar.sync %0, 128;" ::"n"(kBarTcPanel) : "memory"); }

// The sweep over the nr pivot columns of the TMEM-resident matrix (see above).
// All kTcThreads threads call it.  tmem: TMEM base of the matrix (lane 0);
// nc <= 128 columns (lanes), nr <= nc rows; TMEM columns 0 .. 2 tc_pad(nr) - 1.
// With ng > 0 a second matrix of ng <= 128 columns at TMEM base tmem_g (the
// right-hand sides, same row layout) takes the same row operations: its
// columns are never pivot columns, so it ends as the rows of D^-1 times the
// original columns, row p_k holding row k (A operand tile atile_g).
// piv[k] receives the pivot row of column k.  mbar / phase: the MMA
// completion barrier and its parity (updated).  Zero pivots set
// kFlagSingular.  Returns false when a bounded completion wait gave up (then
// the block must stop issuing MMAs; the flag kFlagTcTimeout is set).
__device__ __forceinline__ bool tcgj_sweep(unsigned tmem, int nr, int nc, const TcGjSmem sm, int* piv, uint64_t* mbar,
                                           unsigned& phase, int* __restrict__ flags, unsigned tmem_g = 0u,
                                           int ng = 0, __nv_bfloat16* atile_g = nullptr) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp & 3;
  const int np = tc_pad(nr);
  const int j = 32 * q + lane;                  // the TMEM lane this thread reaches
  const unsigned tq = tmem + ((32u * q) << 16);  // this warp's lane quadrant
  const unsigned abase = smem_u32(sm.atile), bbase = smem_u32(sm.btile);
  const unsigned idesc = umma_idesc_bf16(128, 2 * np);
  bool used = tid >= nr;                        // warps 0-3: row tid; padding rows never pivot
  for (int k0 = 0; k0 < nr; k0 += kTcPanel) {
    const int nb = min(kTcPanel, nr - k0);
    // 1. the panel's columns: lanes k0 .. k0 + 7 of quadrant k0 / 32, all rows
    if (q == (k0 >> 5)) {
      const int r0 = warp < 4 ? 0 : np / 2, r1 = warp < 4 ? np / 2 : np;
      const int s = j - k0;
      // two 8-row groups (32 TMEM columns) per wait
      for (int r = r0; r < r1; r += 16) {
        float v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            "tcgen05.wait::ld.sync.aligned;\n"
            : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
              "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]),
              "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]),
              "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
            : "r"(tq + 2 * r)
            : "memory");
        if (s >= 0 && s < kTcPanel) {
#pragma unroll
          for (int e = 0; e < 16; ++e) sm.panel[(r + e) * kTcPanel + s] = make_float2(v[2 * e], v[2 * e + 1]);
        }
      }
    }
    tc05_fence_before();
    __syncthreads();
    // 2. the panel's Gauss-Jordan steps (warps 0-3, row tid in registers)
    int pivs[kTcPanel];
    float2 pv[kTcPanel];
    if (warp < 4) {
#pragma unroll
      for (int s = 0; s < kTcPanel; ++s) pv[s] = tid < np ? sm.panel[tid * kTcPanel + s] : make_float2(0.f, 0.f);
#pragma unroll
      for (int s = 0; s < kTcPanel; ++s) {
        pivs[s] = 0;
        if (s < nb) {
          const int par = (k0 + s) & 1;
          unsigned key = 0u;
          if (!used) {
            // |pivot| bits (+ one step, so that a zero or NaN candidate in row 127
            // still has a nonzero key) with the row in the low bits: the pivot
            // rows stay a permutation whatever the values
            const float m = fabsf(pv[s].x) + fabsf(pv[s].y);
            key = ((__float_as_uint(m) & ~0x7Fu) + 0x80u) | (unsigned)(127 - tid);
          }
          const unsigned wk = __reduce_max_sync(0xffffffffu, key);
          if (key == wk && wk != 0u) {
            sm.slot_key[par * 4 + warp] = wk;
#pragma unroll
            for (int t = 0; t < kTcPanel; ++t) sm.slot_row[(par * 4 + warp) * kTcPanel + t] = pv[t];
          }
          if (lane == 0 && wk == 0u) sm.slot_key[par * 4 + warp] = 0u;
          panel_bar();
          unsigned best = 0u;
          int bw = 0;
#pragma unroll
          for (int w2 = 0; w2 < 4; ++w2) {
            const unsigned k2 = sm.slot_key[par * 4 + w2];
            if (k2 > best) { best = k2; bw = w2; }
          }
          const int p = 127 - (int)(best & 0x7Fu);
          const float bm = __uint_as_float((best & ~0x7Fu) - 0x80u);
          const bool ok = bm > 0.f && best != 0u;
          float2 prow[kTcPanel];
#pragma unroll
          for (int t = 0; t < kTcPanel; ++t) prow[t] = sm.slot_row[(par * 4 + bw) * kTcPanel + t];
          float2 inv = make_float2(0.f, 0.f);
          if (ok) {                               // 1/z by a scaled reciprocal of |z|^2 (no division)
            const float sc = fmaxf(fabsf(prow[s].x), fabsf(prow[s].y));
            const float rs = __frcp_rn(sc), a = prow[s].x * rs, b = prow[s].y * rs;
            const float d = __frcp_rn(fmaf(a, a, b * b)) * rs;
            inv = make_float2(a * d, -b * d);
          }
          if (tid == p) {
            used = true;
#pragma unroll
            for (int t = 0; t < kTcPanel; ++t) pv[t] = (t == s) ? inv : cmulf(prow[t], inv);
          } else {
            const float2 mi = cmulf(pv[s], inv);
#pragma unroll
            for (int t = 0; t < kTcPanel; ++t) pv[t] = (t == s) ? make_float2(-mi.x, -mi.y) : cfmsf(mi, prow[t], pv[t]);
          }
          pivs[s] = best != 0u ? p : 0;
          if (tid == 0) {
            piv[k0 + s] = pivs[s];
            if (!ok) atomicOr(flags, kFlagSingular);
          }
        }
      }
      // 3a. B operand rows (2 tid, 2 tid + 1) from W = P' - unit columns at the pivot rows
      if (tid < np) {
        float wr[16], wi[16];
#pragma unroll
        for (int s = 0; s < kTcPanel; ++s) {
          float2 w = s < nb ? pv[s] : make_float2(0.f, 0.f);
          if (s < nb && pivs[s] == tid) w.x -= 1.f;
          wr[2 * s] = w.x;
          wr[2 * s + 1] = -w.y;
          wi[2 * s] = w.y;
          wi[2 * s + 1] = w.x;
        }
        put_split_row(sm.btile, 2 * tid, wr);
        put_split_row(sm.btile, 2 * tid + 1, wi);
      }
      if (ng > 0) {                             // A operand of the right-hand sides: row j = G[p_s][j]
        const unsigned tg = tmem_g + ((32u * q) << 16);
        float a[16];
#pragma unroll
        for (int s = 0; s < kTcPanel; ++s) {
          if (s < nb) {
            tmem_ld_x2(tg + 2 * pivs[s], a[2 * s], a[2 * s + 1]);
          } else {
            a[2 * s] = 0.f;
            a[2 * s + 1] = 0.f;
          }
        }
        tmem_wait_ld();
        if (j >= ng) {
#pragma unroll
          for (int t = 0; t < 16; ++t) a[t] = 0.f;
        }
        put_split_row(atile_g, j, a);
      }
    }
    __syncthreads();                            // the panel's pivots in piv[]
    // 3b. A operand (warps 4-7): row j = A[p_s][j] (+1 at the panel's own column's slot)
    if (warp >= 4) {
      float a[16];
#pragma unroll
      for (int s = 0; s < kTcPanel; ++s) {
        if (s < nb) {
          tmem_ld_x2(tq + 2 * piv[k0 + s], a[2 * s], a[2 * s + 1]);
        } else {
          a[2 * s] = 0.f;
          a[2 * s + 1] = 0.f;
        }
      }
      tmem_wait_ld();
#pragma unroll
      for (int s = 0; s < kTcPanel; ++s) {
        if (j == k0 + s) a[2 * s] += 1.f;
        if (j >= nc) a[2 * s] = a[2 * s + 1] = 0.f;
      }
      put_split_row(sm.atile, j, a);
    }
    fence_async_smem();
    tc05_fence_before();
    __syncthreads();
    // 4. the update on the tensor cores: six products of BF16 pieces, one commit
    if (tid == 0) {
      tc05_fence_after();
      const int ap[6] = {0, 0, 1, 0, 1, 2}, bp[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
      for (int t = 0; t < 6; ++t)
        umma_bf16(tmem, umma_desc_sw128(abase + 32 * ap[t]), umma_desc_sw128(bbase + 32 * bp[t]), idesc, 1u);
      if (ng > 0) {
        const unsigned gbase = smem_u32(atile_g);
#pragma unroll
        for (int t = 0; t < 6; ++t)
          umma_bf16(tmem_g, umma_desc_sw128(gbase + 32 * ap[t]), umma_desc_sw128(bbase + 32 * bp[t]), idesc, 1u);
      }
      umma_commit(mbar);
    }
    const bool done = mbar_wait(mbar, phase);
    phase ^= 1u;
    tc05_fence_after();
    if (__syncthreads_or(!done)) {
      if (tid == 0) atomicOr(flags, kFlagTcTimeout);
      return false;
    }
  }
  return true;
}

}  // namespace df
