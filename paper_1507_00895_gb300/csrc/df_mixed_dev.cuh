// Mixed-precision ladder solves (DF_FP32_IR): Eq. lin_alg_inv solved in
// FP32 (complex64) and corrected once with an FP64-accurate residual.
//
// Per (q, W, channel) system, with D = 1 - gamma diag(chi~):
//   1. Gauss-Jordan sweep with partial pivoting of the augmented [D | gamma]
//      in FP32: the D part becomes D^-1 in place (rows and columns permuted
//      by the pivot order), the gamma part X0 ~ D^-1 gamma.  The pivots are
//      those of LU with partial pivoting (the same unused-row maximum of the
//      same Schur complement column); one sweep, three block barriers per
//      panel of 8 pivots.
//   2. R = gamma - D X0 = gamma - X0 + Z X0, Z = gamma diag(chi~) formed in
//      FP64, with ~2^-49 accuracy relative to |Z| |X0| (exact BF16 digit
//      products on the tensor cores: tcgen05 with TMEM accumulators at
//      n_pad = 64, mma.sync at 32; double-float FP32 arithmetic below).
//   3. diag E = diag(D^-1 R) (n^2 work with the explicit inverse);
//      diag Gamma = diag X0 + diag E in FP64.
// One correction step leaves an error ~(kappa u32)^2 |Gamma| plus kappa times
// the residual's own accuracy.
//
// Layout: the whole [D | gamma] lives in registers.  The block is a P x P
// grid of threads, P = n_pad / 4; thread (tr, tc) = (t / P, t % P) owns rows
// tr + P i and columns tc + P j (i, j < 4) of D and of gamma (2D cyclic), so
// that the P threads of a thread row are consecutive lanes and every warp
// holds whole rows.  Row pivoting is implicit: rows never move.  The sweep
// goes by panels of 8 pivot columns factored by one or two warps (see the
// sweep below).  Matrices of order n < n_pad are padded with an identity
// block (gamma = 0, chi~ = 0 there), which leaves the solution of the first
// n rows unchanged.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "df_internal.cuh"

namespace df {


constexpr int kTile = 4;          // rows / columns per thread
constexpr int kResChunk = 16;     // gamma columns staged per residual sweep (SIMT residual)
constexpr int kSlices = 8;        // base-128 digits of the tensor-core residual (56 bits)
constexpr int kCB = 16;           // column block of the tensor-core residual
constexpr int kPanel = 8;         // pivot columns per Gauss-Jordan panel
constexpr int kPanelLd = kPanel + 1;   // panel row stride (float2): conflict-free lane-per-row access
constexpr int kPanelRows = 2;     // panel rows per lane of warp 0 (np / min(32, P^2) <= 2 for np >= 8)

// padded order of a mixed ladder: a power of two >= 8 (P = np / 4 >= 2 lanes per
// thread row; warp 0 then holds at most two panel rows per lane)
// bytes of one gamma matrix's digits for the tensor-core residual: 8 slices
// x (re, im) x np rows of 64 bf16 (swizzled as in shared memory), then the
// np row exponents (int)
__host__ __device__ constexpr int gdig_bytes(int np) { return 2 * kSlices * 2 * np * 64 + 4 * np; }

__host__ __device__ inline int mixed_pad(int n) {
  int np = 2 * kTile;
  while (np < n) np *= 2;
  return np;
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfmsf(float2 a, float2 b, float2 c) {   // c - a b
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfmaf2(float2 a, float2 b, float2 c) {   // c + a b
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cinvf(float2 z) {
  const float s = fmaxf(fabsf(z.x), fabsf(z.y));
  const float a = z.x / s, b = z.y / s;
  const float d = 1.0f / ((a * a + b * b) * s);
  return make_float2(a * d, -b * d);
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


// ---- tensor-core residual helpers --------------------------------------

// |v| < 2^e: the 8 signed base-128 digits d_s of v / 2^e, v ~ sum_s d_s 2^(e - 7(s+1)),
// truncated below 2^(e - 56).  Read from the FP64 bits (integer operations only).
__device__ __forceinline__ void digits_f64(double v, int e, float* d) {
  const long long bits = __double_as_longlong(v);
  int E = (int)((bits >> 52) & 0x7FF);
  unsigned long long M = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
  if (E == 0) {
    if (M == 0) {
#pragma unroll
      for (int s = 0; s < kSlices; ++s) d[s] = 0.f;
      return;
    }
    E = 1;
  } else {
    M |= (1ull << 52);
  }
  const int sh = e - (E - 1023) - 1;                 // >= 0
  const unsigned long long T = sh <= 3 ? (M << (3 - sh)) : (sh - 3 >= 64 ? 0ull : (M >> (sh - 3)));
  const float sg = bits < 0 ? -1.f : 1.f;
#pragma unroll
  for (int s = 0; s < kSlices; ++s) d[s] = sg * (float)(unsigned)((T >> (49 - 7 * s)) & 0x7Full);
}

// the same for an FP32 value
__device__ __forceinline__ void digits_f32(float v, int e, float* d) {
  const unsigned bits = __float_as_uint(v);
  int E = (int)((bits >> 23) & 0xFF);
  unsigned M = bits & 0x7FFFFFu;
  if (E == 0) {
    if (M == 0) {
#pragma unroll
      for (int s = 0; s < kSlices; ++s) d[s] = 0.f;
      return;
    }
    E = 1;
  } else {
    M |= 0x800000u;
  }
  const int sh = e - (E - 127) - 1;                  // >= 0
  const unsigned long long T = sh <= 32 ? ((unsigned long long)M << (32 - sh))
                                        : (sh - 32 >= 32 ? 0ull : (unsigned long long)(M >> (sh - 32)));
  const float sg = (bits >> 31) ? -1.f : 1.f;
#pragma unroll
  for (int s = 0; s < kSlices; ++s) d[s] = sg * (float)(unsigned)((T >> (49 - 7 * s)) & 0x7Full);
}

// 2^e as a float for e >= -126 (0 below: the terms it scales are < 2^-100 of the result)
__device__ __forceinline__ float pow2f(int e) {
  return e < -126 ? 0.f : __int_as_float((e + 127) << 23);
}

// exponent e with |v| < 2^e (v != 0): unbiased exponent + 1
__device__ __forceinline__ int exp_bound_f32(float v) {
  const unsigned bits = __float_as_uint(v) & 0x7FFFFFFFu;
  if (bits == 0) return -1000;
  const int E = (int)(bits >> 23);
  return (E == 0 ? -126 : E - 127) + 1;
}

// digit matrices: rows of 64 bf16 (32 words); word w of row r stored at
// w ^ ((r & 7) << 2), so that fragment loads (8 rows x 4 words) hit 32 banks
__device__ __forceinline__ int swz(int row, int k) {
  return row * 64 + ((((k >> 1) ^ ((row & 7) << 2))) << 1) + (k & 1);
}
__device__ __forceinline__ unsigned ld_frag(const __nv_bfloat16* base, int row, int k) {
  return *reinterpret_cast<const unsigned*>(base + swz(row, k));
}

__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, unsigned b0, unsigned b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---- tcgen05 (5th-generation tensor core) helpers for the np = 64 residual ----
// Operands are K-major bf16 tiles in shared memory with 128-byte rows in the
// 128-byte swizzle (16-byte chunk c of row r at chunk c ^ (r & 7); 8-row groups
// 1024 bytes apart, group base 1024-aligned) -- the layout swz() writes.  The
// FP32 accumulators live in tensor memory (TMEM): row i of D in TMEM lane i,
// column j in TMEM column (base + j).
constexpr int kTmemCols = 512;      // two buffers of 8 weight groups x 32 columns
constexpr unsigned kMbarSpin = 1u << 22;   // try_wait rounds before giving up

struct Tc05 {
  unsigned tmem;        // TMEM base address (lane 0, first allocated column)
  uint64_t* mbar;       // completion barrier of the MMA batches
  unsigned phase;       // parity of the next completion (the same in every thread)
  uint64_t* fin;        // the tear-down's barrier: every queued MMA done before TMEM is freed
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t umma_desc_sw128(unsigned saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor, kind::f16: bf16 A and B (K-major), FP32 D, M x N
__host__ __device__ constexpr unsigned umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(unsigned dtmem, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on mbar once every MMA issued so far by this thread has completed
__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
// bounded wait for the completion of the given parity; false if it gave up
// after `spins` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, unsigned parity, unsigned spins = kMbarSpin) {
  const unsigned a = smem_u32(mbar);
  for (unsigned it = 0; it < spins; ++it) {
    unsigned done;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tc05_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc05_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) ..)
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// block-level set-up / tear-down (all threads call; warp 0 owns the TMEM allocation);
// mbar: two barriers (the MMA batches', the tear-down's)
__device__ __forceinline__ void tc05_setup(Tc05& tc, uint64_t* mbar, unsigned* tslot) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "n"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  tc.tmem = *tslot;
  tc.mbar = mbar;
  tc.phase = 0;
  tc.fin = mbar + 1;
}
// issuer: the thread that issued the block's MMAs.  Its one more commit, to
// the tear-down's barrier, completes once every MMA it queued has (also after
// a completion wait that gave up earlier); the wait for it is bounded.
__device__ __forceinline__ void tc05_teardown(const Tc05& tc, int issuer) {
  if ((int)threadIdx.x == issuer) {
    tc05_fence_before();
    umma_commit(tc.fin);
    mbar_wait(tc.fin, 0u);
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "n"(kTmemCols) : "memory");
}

__device__ __forceinline__ void dd_add(float& hi, float& lo, float v) {
  float s, e;
  two_sum(hi, v, s, e);
  e += lo;
  hi = s + e;
  lo = e - (hi - s);
}

// b = pb in-place Gauss-Jordan steps on the panel pan[np][kPanelLd] (the pivot
// columns k0 .. k0 + pb - 1), run by warp 0 alone: lane l holds rows
// l + nlanes s (s < np / nlanes <= 2) in registers.  The pivot of each
// column is the warp maximum of a key (|re| + |im| bits with their low 7 bits
// replaced by 127 - row: the largest to 2^-16 relative, ties to the lowest
// row) over the rows not yet used; the pivot row is broadcast by shuffles
// from its owner lane.  The elimination is branch-free (the pivot row takes
// the scaled row by a select).  Writes the new panel to pan, after the pb
// steps the pivot rows to piv_s[k0 + i] and the steps to rowstep[row];
// used0 marks this lane's rows taken.
template <int NP>
__device__ __forceinline__ void gj_panel(float2* pan, int k0, int lane, unsigned& used0, int* piv_s, int* rowstep,
                                         int* flags) {
  constexpr int np = NP, P = NP / kTile;
  constexpr int nlanes = P * P < 32 ? P * P : 32;
  constexpr unsigned wmask = nlanes == 32 ? 0xffffffffu : ((1u << nlanes) - 1u);
  constexpr int pb = P < kPanel ? P : kPanel;
  constexpr int rows_per_lane = np / nlanes;
  static_assert(rows_per_lane <= kPanelRows, "panel rows per lane");
  float2 pv[kPanelRows][kPanel];
#pragma unroll
  for (int s2 = 0; s2 < kPanelRows; ++s2)
#pragma unroll
    for (int c2 = 0; c2 < kPanel; ++c2)
      pv[s2][c2] = (s2 < rows_per_lane && c2 < pb) ? pan[(lane + nlanes * s2) * kPanelLd + c2] : make_float2(0.f, 0.f);
  int pivs[kPanel];
  bool sing = false;
#pragma unroll
  for (int i = 0; i < kPanel; ++i) {
    if (i < pb) {
      unsigned key = 0u;
#pragma unroll
      for (int s2 = 0; s2 < rows_per_lane; ++s2) {
        const int r = lane + nlanes * s2;
        const float m = fabsf(pv[s2][i].x) + fabsf(pv[s2][i].y);
        const unsigned k2 = ((used0 >> s2) & 1u) ? 0u : ((__float_as_uint(m) & ~0x7Fu) | (unsigned)(127 - r));
        key = k2 > key ? k2 : key;
      }
      key = __reduce_max_sync(wmask, key);
      int p = 127 - (int)(key & 0x7Fu);
      const float bm = __uint_as_float(key & ~0x7Fu);
      const bool singular = !(bm > 0.f) || p >= np;
      if (p >= np) p = 0;
      const int owner = p % nlanes, sp2 = p / nlanes;
      float2 u[kPanel];
#pragma unroll
      for (int c2 = 0; c2 < kPanel; ++c2) {
        float2 v = pv[0][c2];
#pragma unroll
        for (int s2 = 1; s2 < rows_per_lane; ++s2)
          if (s2 == sp2) v = pv[s2][c2];
        u[c2].x = __shfl_sync(wmask, v.x, owner);
        u[c2].y = __shfl_sync(wmask, v.y, owner);
      }
      // 1 / pivot (approximate reciprocal: the FP32 sweep is corrected later)
      float2 ainv = make_float2(0.f, 0.f);
      if (!singular) {
        const float2 z = u[i];
        const float d = __fdividef(1.f, fmaf(z.x, z.x, z.y * z.y));
        ainv = make_float2(z.x * d, -z.y * d);
      }
#pragma unroll
      for (int c2 = 0; c2 < kPanel; ++c2) u[c2] = (c2 == i) ? ainv : cmulf(u[c2], ainv);
      pivs[i] = p;
      sing |= singular;
      used0 |= (lane == owner) ? (1u << sp2) : 0u;
#pragma unroll
      for (int s2 = 0; s2 < rows_per_lane; ++s2) {
        const bool isp = (lane + nlanes * s2 == p);
        const float2 m = pv[s2][i];
#pragma unroll
        for (int c2 = 0; c2 < kPanel; ++c2) {
          const float2 base = (c2 == i) ? make_float2(0.f, 0.f) : pv[s2][c2];
          const float2 e = cfmsf(m, u[c2], base);
          pv[s2][c2] = isp ? u[c2] : e;
        }
      }
    }
  }
#pragma unroll
  for (int s2 = 0; s2 < rows_per_lane; ++s2)
#pragma unroll
    for (int c2 = 0; c2 < kPanel; ++c2)
      if (c2 < pb) pan[(lane + nlanes * s2) * kPanelLd + c2] = pv[s2][c2];
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < kPanel; ++i) {
      if (i < pb) {
        piv_s[k0 + i] = pivs[i];
        rowstep[pivs[i]] = k0 + i;
      }
    }
    if (sing) atomicOr(flags, 1);
  }
}

// The same b = 8 steps for np = 64 on two warps (threads 0..63), one row per
// lane: each warp's best unused row (its warp max) goes to cand / ckey, a
// 64-thread named barrier, then both warps take the better of the two.  The
// candidate slots alternate between steps, so one barrier per step suffices.
__device__ __forceinline__ void gj_panel2(float2* pan, int k0, int w, int lane, unsigned& used0, int* piv_s,
                                          int* rowstep, int* flags, float4* cand, unsigned* ckey) {
  constexpr int np = 64;
  const int r = 32 * w + lane;
  float2 pv[kPanel];
#pragma unroll
  for (int c2 = 0; c2 < kPanel; ++c2) pv[c2] = pan[r * kPanelLd + c2];
  int pivs[kPanel];
  bool sing = false;
#pragma unroll
  for (int i = 0; i < kPanel; ++i) {
    const float m0 = fabsf(pv[i].x) + fabsf(pv[i].y);
    const unsigned key = (used0 & 1u) ? 0u : ((__float_as_uint(m0) & ~0x7Fu) | (unsigned)(127 - r));
    const unsigned kw = __reduce_max_sync(0xffffffffu, key);
    const int par = i & 1;
    if (key == kw && kw != 0u) {
      float4* cs = cand + (par * 2 + w) * (kPanel / 2);
#pragma unroll
      for (int c4 = 0; c4 < kPanel / 2; ++c4)
        cs[c4] = make_float4(pv[2 * c4].x, pv[2 * c4].y, pv[2 * c4 + 1].x, pv[2 * c4 + 1].y);
    }
    if (lane == 0) ckey[par * 2 + w] = kw;
    asm volatile("bar.sync 1, 64;" ::: "memory");
    const unsigned ka = ckey[par * 2], kb = ckey[par * 2 + 1];
    const int wb = kb > ka ? 1 : 0;
    const unsigned kbest = kb > ka ? kb : ka;
    int p = 127 - (int)(kbest & 0x7Fu);
    const float bm = __uint_as_float(kbest & ~0x7Fu);
    const bool singular = !(bm > 0.f) || p >= np;
    if (p >= np) p = 0;
    const float4* cb = cand + (par * 2 + wb) * (kPanel / 2);
    float2 u[kPanel];
#pragma unroll
    for (int c4 = 0; c4 < kPanel / 2; ++c4) {
      const float4 q = cb[c4];
      u[2 * c4] = make_float2(q.x, q.y);
      u[2 * c4 + 1] = make_float2(q.z, q.w);
    }
    float2 ainv = make_float2(0.f, 0.f);
    if (!singular) {
      const float2 z = u[i];
      const float d = __fdividef(1.f, fmaf(z.x, z.x, z.y * z.y));
      ainv = make_float2(z.x * d, -z.y * d);
    }
#pragma unroll
    for (int c2 = 0; c2 < kPanel; ++c2) u[c2] = (c2 == i) ? ainv : cmulf(u[c2], ainv);
    pivs[i] = p;
    sing |= singular;
    const bool isp = (r == p);
    used0 |= isp ? 1u : 0u;
    const float2 m = pv[i];
#pragma unroll
    for (int c2 = 0; c2 < kPanel; ++c2) {
      const float2 base = (c2 == i) ? make_float2(0.f, 0.f) : pv[c2];
      const float2 e = cfmsf(m, u[c2], base);
      pv[c2] = isp ? u[c2] : e;
    }
  }
#pragma unroll
  for (int c2 = 0; c2 < kPanel; ++c2) pan[r * kPanelLd + c2] = pv[c2];
  if (w == 0 && lane == 0) {
#pragma unroll
    for (int i = 0; i < kPanel; ++i) {
      piv_s[k0 + i] = pivs[i];
      rowstep[pivs[i]] = k0 + i;
    }
    if (sing) atomicOr(flags, 1);
  }
}

// bf16 bit pattern of the signed digit (sign16 = 0 or 0x8000, 0 <= d < 256),
// exact and without a conversion unit: the float 2^23 + d minus 2^23
__device__ __forceinline__ unsigned bf16_digit(unsigned d, unsigned sign16) {
  return (__float_as_uint(__uint_as_float(0x4B000000u | d) - 8388608.f) >> 16) | sign16;
}

// v 2^(56 - e), truncated toward zero, as a signed integer (|v| < 2^e;
// subnormal v count as 0)
__device__ __forceinline__ long long fixed56(float v, int e) {
  const unsigned bits = __float_as_uint(v);
  const int E = (int)((bits >> 23) & 0xFFu);
  if (E == 0) return 0;
  const unsigned long long M = (unsigned long long)((bits & 0x7FFFFFu) | 0x800000u);
  const int sh = E - 150 + 56 - e;                       // v = M 2^(E - 150), sh <= 32
  const unsigned long long m = sh >= 0 ? (M << sh) : (-sh >= 64 ? 0ull : (M >> -sh));
  return (bits >> 31) ? -(long long)m : (long long)m;
}

// the 8 base-128 digits of hi + lo relative to 2^e as bf16 patterns
__device__ __forceinline__ void digits_pair(float hi, float lo, int e, unsigned* d) {
  const long long T = fixed56(hi, e) + fixed56(lo, e);
  const unsigned sign16 = T < 0 ? 0x8000u : 0u;
  const unsigned long long m = (unsigned long long)(T < 0 ? -T : T);
#pragma unroll
  for (int s2 = 0; s2 < kSlices; ++s2) d[s2] = bf16_digit((unsigned)((m >> (49 - 7 * s2)) & 0x7Full), sign16);
}

// The same 8 digits as float bit patterns of the signed digit (+-d, d < 128,
// exact), for packing two rows' bf16 halves with one byte permute.  Digit s =
// bits [49 - 7s, 55 - 7s] of |T|, taken from the 32-bit word that holds it.
__device__ __forceinline__ unsigned bfe7(unsigned x, unsigned pos) {
  unsigned r;
  asm("bfe.u32 %0, %1, %2, 7;" : "=r"(r) : "r"(x), "r"(pos));
  return r;
}
__device__ __forceinline__ void digits_pair_f(float hi, float lo, int e, unsigned* f) {
  const long long T = fixed56(hi, e) + fixed56(lo, e);
  const unsigned sgn = T < 0 ? 0x80000000u : 0u;
  const unsigned long long m = (unsigned long long)(T < 0 ? -T : T);
  const unsigned mh = (unsigned)(m >> 32), ml = (unsigned)m;
  unsigned d[kSlices];
  d[0] = bfe7(mh, 17);
  d[1] = bfe7(mh, 10);
  d[2] = bfe7(mh, 3);
  d[3] = __funnelshift_r(ml, mh, 28) & 0x7Fu;
  d[4] = bfe7(ml, 21);
  d[5] = bfe7(ml, 14);
  d[6] = bfe7(ml, 7);
  d[7] = ml & 0x7Fu;
#pragma unroll
  for (int s2 = 0; s2 < kSlices; ++s2) f[s2] = __float_as_uint(__uint_as_float(0x4B000000u | d[s2]) - 8388608.f) | sgn;
}
// {bf16 of row l (low half), bf16 of row l + 1 (high half)} from their float patterns
__device__ __forceinline__ unsigned pack_bf16_hi(unsigned f0, unsigned f1) { return __byte_perm(f0, f1, 0x7632); }

// gamma's digits for the tensor-core residual, `count` n x n matrices (FP64)
// -> out[count][gdig_bytes(np)]: row i's exponent bound e_i (|gamma_il| < 2^e_i
// for both parts, -1000 for a zero row) and the 8 digits of each part
// relative to 2^e_i; rows and columns >= n are zero.  One warp per row.
__device__ __forceinline__ void gamma_digits_rows(int n, int np, int count, const double2* __restrict__ gam,
                                                  unsigned char* __restrict__ out, int warp_id, int nwarps,
                                                  int lane) {
  for (int w = warp_id; w < count * np; w += nwarps) {
    const int mtx = w / np, i = w - mtx * np;
    const double2* G = gam + (size_t)mtx * n * n;
    unsigned char* O = out + (size_t)mtx * gdig_bytes(np);
    __nv_bfloat16* dig = reinterpret_cast<__nv_bfloat16*>(O);
    int* rowe = reinterpret_cast<int*>(O + 2 * kSlices * 2 * np * 64);
    double m = 0.0;
    for (int l = lane; l < n; l += 32)
      if (i < n) m = fmax(m, fmax(fabs(G[(size_t)i * n + l].x), fabs(G[(size_t)i * n + l].y)));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = -1000;
    if (m > 0.0) frexp(m, &e);                           // m < 2^e
    if (lane == 0) rowe[i] = e;
    for (int l = lane; l < 64; l += 32) {
      float dr[kSlices], di[kSlices];
      if (i < n && l < n && e > -1000) {
        digits_f64(G[(size_t)i * n + l].x, e, dr);
        digits_f64(G[(size_t)i * n + l].y, e, di);
      } else {
#pragma unroll
        for (int s2 = 0; s2 < kSlices; ++s2) dr[s2] = di[s2] = 0.f;
      }
      const int o = swz(i, l);
#pragma unroll
      for (int s2 = 0; s2 < kSlices; ++s2) {
        dig[(size_t)(s2 * 2 + 0) * np * 64 + o] = __float2bfloat16_rn(dr[s2]);
        dig[(size_t)(s2 * 2 + 1) * np * 64 + o] = __float2bfloat16_rn(di[s2]);
      }
    }
  }
}

struct MixedSmem {
  // offsets in float2 units (8 bytes)
  int x0, chih, chil, invu, x0d, chi64, work, gt_h, gt_l, yh, yl, total;
};

__host__ __device__ constexpr bool use_tc_residual(int np) { return np == 32 || np == 64; }
// np = 64: the digit products run as tcgen05 MMAs (M = 128 = [Zr; Zi] rows)
__host__ __device__ constexpr bool use_umma_residual(int np) { return np == 64; }
// offset of the Y digits in the work area (1024-aligned for the tcgen05 operands)
__host__ __device__ constexpr int xs_offset(int np) {
  return use_umma_residual(np) ? ((gdig_bytes(np) + 1023) & ~1023) : gdig_bytes(np);
}
// bytes of the tensor-core residual's work area (n_pad in {32, 64}): the
// gamma digits of the current (channel, W) (kept across systems), then the
// Y digits of one column block and their column exponents
__host__ __device__ constexpr int tc_work_bytes(int np) {
  // np = 64 adds a second column-exponent slot, the re/im exchange
  // [2][np][kCB + 1] (double-float) and per-warp column exponents [8][kCB]
  return xs_offset(np) + 2 * kSlices * 2 * kCB * 64 + 4 * kCB +
         (use_umma_residual(np) ? 4 * kCB + 2 * np * (kCB + 1) * 8 + 4 * 8 * kCB : 0);
}

// row stride of X0 / R in shared memory (float2): np + 1 spreads a column
// read (16 rows, one column) over 16 banks
__host__ __device__ constexpr int x0_ld(int np) { return np + 1; }

__host__ __device__ inline MixedSmem mixed_layout(int np) {
  MixedSmem L;
  int o = 0;
  L.x0 = o;   o += np * x0_ld(np); // X0 (logical rows), then R in its place
  L.chih = o; o += np;
  L.chil = o; o += np;
  L.invu = o; o += np;
  L.x0d = o;  o += np;             // diag X0 (FP32)
  L.chi64 = o; o += 2 * np;        // chi~ in FP64 (double2 = two float2 slots)
  if (use_umma_residual(np)) o = (o + 127) & ~127;   // tcgen05 operand tiles: 1024-byte aligned
  L.work = o;                      // residual work area (one of the two layouts below)
  // SIMT residual: gamma tiles and Y = chi o X0 as double-float
  L.gt_h = o;
  L.gt_l = L.gt_h + kResChunk * np;
  L.yh = L.gt_l + kResChunk * np;
  L.yl = L.yh + np * np;
  const int simt = 2 * kResChunk * np + 2 * np * np;
  const int tc = (tc_work_bytes(np) + 7) / 8;
  // Gauss-Jordan panels [2][np][kPanelLd] and pivot rows [kPanel][2 np]; with
  // the tensor-core residual they sit in the Y-digit area, past gamma's digits
  const int gj = (use_tc_residual(np) ? gdig_bytes(np) / 8 : 0) + 2 * np * kPanelLd + kPanel * 2 * np +
                 2 * 2 * kPanel + 2;   // + the two-warp panel's candidate rows and keys
  const int res = use_tc_residual(np) ? tc : simt;
  o += res > gj ? res : gj;
  L.total = o;
  return L;
}

// Shared-memory views of one mixed solve (layout from mixed_layout).
struct MixedPtrs {
  float2 *X0s, *chih, *chil, *invu, *x0d, *gth, *gtl, *Yh, *Yl;
  double2* chi64;
  int* piv_s;
  unsigned char* work;
};

__device__ __forceinline__ MixedPtrs mixed_ptrs(float2* smf, int np, int* piv_s) {
  const MixedSmem L = mixed_layout(np);
  MixedPtrs m;
  m.X0s = smf + L.x0;
  m.chih = smf + L.chih;
  m.chil = smf + L.chil;
  m.invu = smf + L.invu;
  m.x0d = smf + L.x0d;
  m.gth = smf + L.gt_h;
  m.gtl = smf + L.gt_l;
  m.Yh = smf + L.yh;
  m.Yl = smf + L.yl;
  m.chi64 = (double2*)(smf + L.chi64);
  m.work = (unsigned char*)(smf + L.work);
  m.piv_s = piv_s;
  return m;
}

// n_pad = 64 runs 9 warps: warps 0-7 compute (their own 256-thread barrier),
// warp 8 issues the tensor-core MMAs.  Per column block the compute warps
// arrive on barrier kBarHandoff once the block's Y digits are in shared
// memory; the producer waits there, issues the block's MMAs and commits them
// to the mbarrier the compute warps wait on before they read TMEM.
constexpr int kBarCompute = 2;    // named barrier of the 256 compute threads
constexpr int kBarHandoff = 3;    // compute warps -> producer warp (288 threads)
__host__ __device__ constexpr int mixed_compute_threads(int np) { return (np / kTile) * (np / kTile); }
__host__ __device__ constexpr int mixed_block_threads(int np) {
  return mixed_compute_threads(np) + (use_umma_residual(np) ? 32 : 0);
}
template <int NP>
__device__ __forceinline__ void block_sync() {
  if constexpr (use_umma_residual(NP))
    asm volatile("bar.sync %0, %1;" ::"n"(kBarCompute), "n"(mixed_compute_threads(NP)) : "memory");
  else
    __syncthreads();
}
__device__ __forceinline__ void handoff_arrive() {
  asm volatile("bar.arrive %0, %1;" ::"n"(kBarHandoff), "n"(mixed_compute_threads(64) + 32) : "memory");
}
__device__ __forceinline__ void handoff_wait() {
  asm volatile("bar.sync %0, %1;" ::"n"(kBarHandoff), "n"(mixed_compute_threads(64) + 32) : "memory");
}

// One (q, W, channel) ladder in mixed precision; all P*P threads of the
// block (P = np / 4) must call it.  Writes kc[c][a][:][q].
template <int NP>
__device__ __forceinline__ void bse_mixed_system(const Dims& dm, int c, int a, int q,
                                                 const double2* __restrict__ gam,
                                                 const float2* __restrict__ gam_hi,
                                                 const float2* __restrict__ gam_lo,
                                                 const float2* __restrict__ gg_hi,
                                                 const float2* __restrict__ gg_lo,
                                                 const double2* __restrict__ chi, double2* __restrict__ kc,
                                                 int* __restrict__ flags, const MixedPtrs& sp,
                                                 const unsigned char* __restrict__ gdig, bool reload,
                                                 Tc05* umma, const MixedCheck& mc) {
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  constexpr int np = NP, P = NP / kTile;
  constexpr int kThr = mixed_compute_threads(NP);       // threads taking part (the producer warp does not)
  constexpr int ld = x0_ld(NP);
  float2* X0s = sp.X0s;
  float2* chih = sp.chih;
  float2* chil = sp.chil;
  float2* invu = sp.invu;
  float2* x0d = sp.x0d;
  float2* gth = sp.gth;
  float2* gtl = sp.gtl;
  float2* Yh = sp.Yh;
  float2* Yl = sp.Yl;
  int* piv_s = sp.piv_s;
  const int t = threadIdx.x;
  const int tr = t / P, tc = t % P;
  const size_t mat = ((size_t)c * nb + a) * n * n;
  const float2* Gh = gam_hi + mat;
  const float2* Gl = gam_lo + mat;

  if constexpr (use_tc_residual(NP)) {
    // gamma's digits of this (channel, W), kept in shared memory across systems
    if (reload) {
      const uint4* src = reinterpret_cast<const uint4*>(gdig);
      uint4* dst = reinterpret_cast<uint4*>(sp.work);
      for (int i = t; i < gdig_bytes(NP) / 16; i += kThr) dst[i] = __ldg(src + i);
      if constexpr (use_umma_residual(NP)) fence_async_smem();
    }
  }
  for (int i = t; i < np; i += kThr) {
    double2 x = (i < n) ? chi[((size_t)a * n + i) * N + q] : mk(0.0, 0.0);
    const float hx = (float)x.x, hy = (float)x.y;
    chih[i] = make_float2(hx, hy);
    chil[i] = make_float2((float)(x.x - (double)hx), (float)(x.y - (double)hy));
    sp.chi64[i] = x;
  }
  block_sync<NP>();

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
      // D = 1 - gamma chi~ formed in double-float and rounded once: the
      // diagonal 1 - gamma_ww chi~_w cancels when |gamma chi~| >> |D|, and a
      // product of FP32-rounded factors would lose those digits
      const bool in = (r < n && col < n);
      const float2 gh = in ? Gh[r * n + col] : make_float2(0.f, 0.f);
      const float2 gl = in ? Gl[r * n + col] : make_float2(0.f, 0.f);
      float sr = (r == col) ? 1.f : 0.f, lr = 0.f, si = 0.f, li = 0.f;
      cdf_fma(sr, lr, si, li, make_float2(-gh.x, -gh.y), make_float2(-gl.x, -gl.y), chih[col], chil[col]);
      A[ii][jj] = make_float2(sr + lr, si + li);
      A[ii][kTile + jj] = gh;
    }
  }

  // ---- Gauss-Jordan sweep of [D | gamma], implicit partial pivoting, in
  // panels of b = min(8, P) pivot columns ----
  // The b GJ steps of a panel change every other column j by a rank-b
  // update, A[:, j] += W A[piv, j], where W = (panel after its own in-place
  // GJ steps) - (unit columns at the pivot rows).  Per panel: (1) the owners
  // of the panel columns copy them to pan; (2) warp 0 (warps 0 and 1 for
  // np = 64, one row per lane) runs the b steps on pan in registers (pivot =
  // max of a (|a| bits, ~row) key); (3) the pivot rows' current values go to
  // prs; (4) every thread applies the rank-b update to its whole tile, then
  // the panel columns take the panel's new values (their updated ones are
  // dropped: no per-column test in the update).  Three block barriers per
  // panel instead of one or two per pivot.
  const int warp = t >> 5, lane = t & 31;
  constexpr int nlanes = P * P < 32 ? P * P : 32;
  constexpr unsigned wmask = nlanes == 32 ? 0xffffffffu : ((1u << nlanes) - 1u);
  constexpr int pb = P < kPanel ? P : kPanel;        // panel width b
  float2* panbuf = reinterpret_cast<float2*>(sp.work + (use_tc_residual(NP) ? gdig_bytes(NP) : 0));   // [2][np][kPanelLd]
  float2* prs = panbuf + 2 * np * kPanelLd;                      // [kPanel][2 np]
  float4* cand = reinterpret_cast<float4*>(prs + kPanel * 2 * np);  // two-warp panel: [2][2][kPanel / 2]
  unsigned* ckey = reinterpret_cast<unsigned*>(cand + 2 * kPanel);   // [2][2]
  int* rowstep = reinterpret_cast<int*>(invu);                   // pivot step of each row, -1 if none
  for (int i = t; i < np; i += kThr) rowstep[i] = -1;
  unsigned used0 = 0;                                            // panel warps: their rows already pivots
  // one copy of the loop body (the register column jk is selected at run time)
#pragma unroll 1
  for (int k0 = 0; k0 < np; k0 += pb) {
    const int jk = k0 / P, kc = k0 - jk * P;
    float2* pan = panbuf + ((k0 / pb) & 1) * np * kPanelLd;
    const bool pcol = (tc >= kc && tc < kc + pb);
    // (1) the panel columns
    if (pcol) {
#pragma unroll
      for (int ii = 0; ii < kTile; ++ii) {
        float2 v = A[ii][0];
#pragma unroll
        for (int jj = 1; jj < kTile; ++jj)
          if (jj == jk) v = A[ii][jj];
        pan[(tr + P * ii) * kPanelLd + (tc - kc)] = v;
      }
    }
    block_sync<NP>();
    // (2) b GJ steps on the panel: warps 0 and 1 for np = 64, else warp 0
    if constexpr (NP == 64) {
      if (warp < 2) gj_panel2(pan, k0, warp, lane, used0, piv_s, rowstep, flags, cand, ckey);
    } else {
      if (warp == 0) gj_panel<NP>(pan, k0, lane, used0, piv_s, rowstep, flags);
    }
    block_sync<NP>();
    // (3) current values of the pivot rows
#pragma unroll
    for (int ii = 0; ii < kTile; ++ii) {
      const int l = rowstep[tr + P * ii] - k0;
      if (l >= 0 && l < pb) {
#pragma unroll
        for (int jj = 0; jj < kTile; ++jj) {
          prs[l * 2 * np + tc + P * jj] = A[ii][jj];
          prs[l * 2 * np + np + tc + P * jj] = A[ii][kTile + jj];
        }
      }
    }
    block_sync<NP>();
    // (4) rank-b update (the panel columns too: they take their new values after)
    for (int l = 0; l < pb; ++l) {
      const int pl = piv_s[k0 + l];
      float2 pr[2 * kTile];
#pragma unroll
      for (int jj = 0; jj < kTile; ++jj) {
        pr[jj] = prs[l * 2 * np + tc + P * jj];
        pr[kTile + jj] = prs[l * 2 * np + np + tc + P * jj];
      }
#pragma unroll
      for (int ii = 0; ii < kTile; ++ii) {
        const int r = tr + P * ii;
        float2 w = pan[r * kPanelLd + l];
        if (r == pl) w.x -= 1.f;
#pragma unroll
        for (int jj = 0; jj < kTile; ++jj) {
          A[ii][jj] = cfmaf2(w, pr[jj], A[ii][jj]);
          A[ii][kTile + jj] = cfmaf2(w, pr[kTile + jj], A[ii][kTile + jj]);
        }
      }
    }
    if (pcol) {
#pragma unroll
      for (int ii = 0; ii < kTile; ++ii) {
        const float2 v = pan[(tr + P * ii) * kPanelLd + (tc - kc)];
#pragma unroll
        for (int jj = 0; jj < kTile; ++jj)
          if (jj == jk) A[ii][jj] = v;
      }
    }
  }
  block_sync<NP>();
#pragma unroll
  for (int ii = 0; ii < kTile; ++ii) rowpos[ii] = rowstep[tr + P * ii];
  // X0 in logical row order: row r of the sweep is X0 row rowpos (its pivot step)
#pragma unroll
  for (int ii = 0; ii < kTile; ++ii) {
    if (rowpos[ii] >= 0) {
#pragma unroll
      for (int jj = 0; jj < kTile; ++jj) X0s[rowpos[ii] * ld + tc + P * jj] = A[ii][kTile + jj];
    }
  }
  block_sync<NP>();
  for (int j = t; j < np; j += kThr) x0d[j] = X0s[j * ld + j];
  if constexpr (use_umma_residual(NP)) {
    // ---- residual R = gamma - X0 + gamma Y with tcgen05, Y = diag(chi~) X0 ----
    // gamma's digits (8 signed base-128 digits relative to per-row powers of
    // two, cut once per input upload) are in zs / rowe; Y is formed in
    // double-float and cut the same way relative to per-column powers of two,
    // kCB columns at a time.  For each gamma slice sa one MMA per K step of
    // 16: A = [Zr; Zi] of slice sa (M = 128), B = the Y slices 0 .. 7 - sa
    // stacked along N (32 rows each: the block's Yr then Yi columns), D at
    // TMEM column 32 sa, so that Y slice sb lands in accumulator d = sa + sb
    // (weight 2^-7(d+2)), columns 32 d .. 32 d + 31 = [Yr | Yi]; lanes 0-63
    // hold the Zr rows, 64-127 the Zi rows.  Every accumulator is exact (<= 8
    // pairs x 64 x 127^2 < 2^23), and the pairs with weight < 2^-63 are never
    // formed.  Column block b's MMAs run in TMEM buffer b & 1 while block
    // b - 1 is folded and assembled.
    __nv_bfloat16* zs = reinterpret_cast<__nv_bfloat16*>(sp.work);                       // [kSlices][2][np][64]
    const int* rowe = reinterpret_cast<const int*>(zs + (size_t)kSlices * 2 * np * 64);   // [np]
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(sp.work + xs_offset(NP));       // [kSlices][2][kCB][64]
    int* cole2 = reinterpret_cast<int*>(xs + (size_t)kSlices * 2 * kCB * 64);            // [2][kCB]
    float2* E = reinterpret_cast<float2*>(cole2 + 2 * kCB);                              // [2][np][kCB + 1]
    int* cw = reinterpret_cast<int*>(E + 2 * np * (kCB + 1));                            // [8][kCB]
    unsigned* xw = reinterpret_cast<unsigned*>(xs);
    const int warp = t >> 5, lane = t & 31;
    const int yc = t & (kCB - 1), yp = t >> 4;          // Y map: column yc, rows 2 yp (+1) (+32)
    // fold of column block bb (TMEM buffer bb & 1) and R = gamma - X0 + S for it
    auto finish = [&](int bb) {
      const int* ce = cole2 + (bb & 1) * kCB;
      // gamma (hi, lo) of this thread's four R entries, loaded ahead of the fold
      float2 ghv[4], glv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int row = yp + 16 * k, j = bb * kCB + yc;
        const bool in = (row < n && j < n);
        ghv[k] = in ? Gh[row * n + j] : make_float2(0.f, 0.f);
        glv[k] = in ? Gl[row * n + j] : make_float2(0.f, 0.f);
      }
      // warp w reads lane quadrant q = w % 4 (gamma row i; Zr or Zi) and column
      // half h = w / 4 (Yr or Yi) of the 8 accumulators.  Weights 2^-7d for
      // d = 4..7 are summed in FP32 (Horner; their sum is < 2^-4.9 of the
      // d = 0 scale, rounding error < 2^-27 of it), d = 0..3 in double-float.
      const int qd = warp & 3, h = warp >> 2;
      const int i = ((qd & 1) << 5) + lane;
      const bool zi = qd >= 2;
      const unsigned tl = umma->tmem + ((unsigned)(32 * qd) << 16) + (unsigned)(256 * (bb & 1) + 16 * h);
      float fh[kCB], fl[kCB];
      {
        float v[kCB];
        tmem_ld16(tl + 32 * 7, fh);
#pragma unroll
        for (int d = 6; d >= 4; --d) {
          tmem_ld16(tl + 32 * d, v);
#pragma unroll
          for (int c2 = 0; c2 < kCB; ++c2) fh[c2] = fmaf(fh[c2], 0.0078125f, v[c2]);
        }
#pragma unroll
        for (int c2 = 0; c2 < kCB; ++c2) {
          fh[c2] *= 3.7252902984619141e-09f;      // 2^-28
          fl[c2] = 0.f;
        }
#pragma unroll
        for (int d = 3; d >= 0; --d) {
          tmem_ld16(tl + 32 * d, v);
          const float sc = __int_as_float((127 - 7 * d) << 23);     // 2^-7d
#pragma unroll
          for (int c2 = 0; c2 < kCB; ++c2) dd_add(fh[c2], fl[c2], v[c2] * sc);
        }
      }
      tc05_fence_before();
      // scale by 2^(e_i + e_j - 14); the Zi rows' parts go to E first (ZiYi
      // negated: it enters the real part with a minus), then the Zr rows add
      // theirs: E[0] = S real, E[1] = S imaginary, row stride kCB + 1
      const int ei = rowe[i];
#pragma unroll
      for (int c2 = 0; c2 < kCB; ++c2) {
        const int ej = ce[c2];
        const float w = (ei > -1000 && ej > -1000) ? pow2f(ei + ej - 14) : 0.f;
        fh[c2] *= w;
        fl[c2] *= w;
      }
      if (zi) {
        const float sg = h ? -1.f : 1.f;
        float2* Eo = E + (1 - h) * np * (kCB + 1) + i * (kCB + 1);   // ZiYr -> imaginary, ZiYi -> real
#pragma unroll
        for (int c2 = 0; c2 < kCB; ++c2) Eo[c2] = make_float2(sg * fh[c2], sg * fl[c2]);
      }
      block_sync<NP>();
      if (!zi) {
        float2* Eo = E + h * np * (kCB + 1) + i * (kCB + 1);         // ZrYr -> real, ZrYi -> imaginary
#pragma unroll
        for (int c2 = 0; c2 < kCB; ++c2) {
          const float2 o = Eo[c2];
          float sh, se;
          two_sum(fh[c2], o.x, sh, se);
          Eo[c2] = make_float2(sh, se + (fl[c2] + o.y));
        }
      }
      block_sync<NP>();
      // R = gamma - X0 + S in double-float (it cancels to ~u32 |gamma|)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int row = yp + 16 * k, j = bb * kCB + yc;
        const float2 x = X0s[row * ld + j];
        const float2 sr = E[row * (kCB + 1) + yc], si = E[np * (kCB + 1) + row * (kCB + 1) + yc];
        float re = ghv[k].x, rl = glv[k].x, im = ghv[k].y, il = glv[k].y;
        df_add(re, rl, -x.x);
        df_add(re, rl, sr.x);
        df_add(im, il, -x.y);
        df_add(im, il, si.x);
        X0s[row * ld + j] = make_float2(re + (rl + sr.y), im + (il + si.y));   // R replaces X0
      }
    };
    for (int b = 0; b < np / kCB; ++b) {
      block_sync<NP>();
      // Y = chi~ o X0 in double-float for rows 2 yp, 2 yp + 1, 2 yp + 32, 2 yp + 33
      // of column yc; its column exponent e (|Y| < 2^e, -1000 for a zero
      // column): the thread's max, the warp's two row groups, the 8 warps
      float y[4][4];
      float m = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int l = 2 * yp + (k & 1) + 32 * (k >> 1);
        const float2 x = X0s[l * ld + b * kCB + yc];
        y[k][0] = y[k][1] = y[k][2] = y[k][3] = 0.f;
        cdf_fma(y[k][0], y[k][1], y[k][2], y[k][3], chih[l], chil[l], x, make_float2(0.f, 0.f));
        m = fmaxf(m, fmaxf(fabsf(y[k][0]), fabsf(y[k][2])));
      }
      m *= 1.0001f;
      int e = m > 0.f ? exp_bound_f32(m) : -1000;
      e = max(e, __shfl_xor_sync(0xffffffffu, e, 16));
      if (lane < kCB) cw[warp * kCB + lane] = e;
      block_sync<NP>();
      int ecol = cw[yc];
#pragma unroll
      for (int w2 = 1; w2 < 8; ++w2) ecol = max(ecol, cw[w2 * kCB + yc]);
      if (t < kCB) cole2[(b & 1) * kCB + t] = ecol;
      // digits of the two row pairs, two rows per 32-bit word
#pragma unroll
      for (int pr = 0; pr < 2; ++pr) {
        unsigned w0[kSlices], w1[kSlices], v0[kSlices], v1[kSlices];
        if (ecol > -1000) {
          digits_pair_f(y[2 * pr][0], y[2 * pr][1], ecol, w0);
          digits_pair_f(y[2 * pr][2], y[2 * pr][3], ecol, w1);
          digits_pair_f(y[2 * pr + 1][0], y[2 * pr + 1][1], ecol, v0);
          digits_pair_f(y[2 * pr + 1][2], y[2 * pr + 1][3], ecol, v1);
        } else {
#pragma unroll
          for (int s2 = 0; s2 < kSlices; ++s2) w0[s2] = w1[s2] = v0[s2] = v1[s2] = 0u;
        }
        const int wo = swz(yc, 2 * yp + 32 * pr) >> 1;
#pragma unroll
        for (int s2 = 0; s2 < kSlices; ++s2) {
          xw[(s2 * 2 + 0) * kCB * 32 + wo] = pack_bf16_hi(w0[s2], v0[s2]);
          xw[(s2 * 2 + 1) * kCB * 32 + wo] = pack_bf16_hi(w1[s2], v1[s2]);
        }
      }
      fence_async_smem();
      tc05_fence_before();
      handoff_arrive();                                 // the producer warp issues block b's MMAs
      if (b > 0) finish(b - 1);
      if (!mbar_wait(umma->mbar, umma->phase) && t == 0) atomicOr(flags, kFlagTcTimeout);
      umma->phase ^= 1;
      tc05_fence_after();
    }
    finish(np / kCB - 1);
    block_sync<NP>();
  } else if constexpr (use_tc_residual(NP)) {
    // ---- residual R = gamma - X0 + gamma Y on the tensor cores, Y = diag(chi~) X0 ----
    // gamma's digits (cut once per input upload: 8 signed base-128 digits
    // relative to per-row powers of two) are in zs / rowe; Y is formed in
    // double-float and cut the same way relative to per-column powers of two,
    // kCB columns at a time.  Each digit pair's product is exact in the FP32
    // accumulator of its weight, and the 36 pairs with weight >= 2^-63 are
    // folded, scaled, into a double-float sum.
    __nv_bfloat16* zs = reinterpret_cast<__nv_bfloat16*>(sp.work);                       // [kSlices][2][np][64]
    const int* rowe = reinterpret_cast<const int*>(zs + (size_t)kSlices * 2 * np * 64);   // [np]
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(sp.work + xs_offset(NP));       // [kSlices][2][kCB][64]
    int* cole = reinterpret_cast<int*>(xs + (size_t)kSlices * 2 * kCB * 64);             // [kCB]
    unsigned* xw = reinterpret_cast<unsigned*>(xs);
    const int nthr = kThr;
    const int warp = t >> 5, lane = t & 31, gq = lane >> 2, t4 = lane & 3;
    const int nwarp = nthr >> 5;
    const int tiles = (np / 16) * (kCB / 8);
    for (int b = 0; b < np / kCB; ++b) {
      block_sync<NP>();
      for (int c2 = t; c2 < kCB; c2 += nthr) cole[c2] = -1000;
      block_sync<NP>();
      // lanes take consecutive columns of a row of X0 (no bank conflicts)
      for (int idx = t; idx < kCB * np; idx += nthr) {
        const int l = idx / kCB, c2 = idx - l * kCB;
        const float2 x = X0s[l * ld + b * kCB + c2];
        float yr = 0.f, ylr = 0.f, yi = 0.f, yli = 0.f;
        cdf_fma(yr, ylr, yi, yli, chih[l], chil[l], x, make_float2(0.f, 0.f));
        const float m = fmaxf(fabsf(yr), fabsf(yi)) * 1.0001f;
        if (m > 0.f) atomicMax(&cole[c2], exp_bound_f32(m));
      }
      block_sync<NP>();
      // two consecutive l per thread: one 32-bit word per slice and part
      for (int idx = t; idx < kCB * np / 2; idx += nthr) {
        const int l = 2 * (idx / kCB), c2 = idx - (l / 2) * kCB;
        unsigned w0[kSlices], w1[kSlices], v0[kSlices], v1[kSlices];
        const int e = cole[c2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 x = X0s[(l + h) * ld + b * kCB + c2];
          float yr = 0.f, ylr = 0.f, yi = 0.f, yli = 0.f;
          cdf_fma(yr, ylr, yi, yli, chih[l + h], chil[l + h], x, make_float2(0.f, 0.f));
          unsigned* dr = h ? v0 : w0;
          unsigned* di = h ? v1 : w1;
          if (e > -1000) {
            digits_pair(yr, ylr, e, dr);
            digits_pair(yi, yli, e, di);
          } else {
#pragma unroll
            for (int s2 = 0; s2 < kSlices; ++s2) dr[s2] = di[s2] = 0u;
          }
        }
        const int wo = swz(c2, l) >> 1;
#pragma unroll
        for (int s2 = 0; s2 < kSlices; ++s2) {
          xw[(s2 * 2 + 0) * kCB * 32 + wo] = w0[s2] | (v0[s2] << 16);
          xw[(s2 * 2 + 1) * kCB * 32 + wo] = w1[s2] | (v1[s2] << 16);
        }
      }
      block_sync<NP>();
      for (int tile = warp; tile < tiles; tile += nwarp) {
        const int r16 = (tile / (kCB / 8)) * 16, c8 = (tile % (kCB / 8)) * 8;
        // acc[d][0 / 1][.]: re / im of all digit pairs with sa + sb = d (one
        // power-of-two weight; exact: at most 8 pairs x 2 x 64 x 127^2 < 2^24)
        float acc[kSlices][2][4];
#pragma unroll
        for (int d = 0; d < kSlices; ++d)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[d][0][e] = acc[d][1][e] = 0.f;
        for (int kk = 0; kk < np; kk += 16) {
#pragma unroll
          for (int sa = 0; sa < kSlices; ++sa) {
            const __nv_bfloat16* zr = zs + (size_t)(sa * 2 + 0) * np * 64;
            const __nv_bfloat16* zi = zs + (size_t)(sa * 2 + 1) * np * 64;
            unsigned fr[4], fi[4], fn[4];
            fr[0] = ld_frag(zr, r16 + gq, kk + 2 * t4);
            fr[1] = ld_frag(zr, r16 + gq + 8, kk + 2 * t4);
            fr[2] = ld_frag(zr, r16 + gq, kk + 2 * t4 + 8);
            fr[3] = ld_frag(zr, r16 + gq + 8, kk + 2 * t4 + 8);
            fi[0] = ld_frag(zi, r16 + gq, kk + 2 * t4);
            fi[1] = ld_frag(zi, r16 + gq + 8, kk + 2 * t4);
            fi[2] = ld_frag(zi, r16 + gq, kk + 2 * t4 + 8);
            fi[3] = ld_frag(zi, r16 + gq + 8, kk + 2 * t4 + 8);
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) fn[q2] = fi[q2] ^ 0x80008000u;   // -Zi
#pragma unroll
            for (int sb = 0; sa + sb < kSlices; ++sb) {
              const __nv_bfloat16* xr = xs + (size_t)(sb * 2 + 0) * kCB * 64;
              const __nv_bfloat16* xi = xs + (size_t)(sb * 2 + 1) * kCB * 64;
              const unsigned br0 = ld_frag(xr, c8 + gq, kk + 2 * t4), br1 = ld_frag(xr, c8 + gq, kk + 2 * t4 + 8);
              const unsigned bi0 = ld_frag(xi, c8 + gq, kk + 2 * t4), bi1 = ld_frag(xi, c8 + gq, kk + 2 * t4 + 8);
              mma_bf16(acc[sa + sb][0], fr, br0, br1);    // + Zr Xr
              mma_bf16(acc[sa + sb][1], fr, bi0, bi1);    // + Zr Xi
              mma_bf16(acc[sa + sb][0], fn, bi0, bi1);    // - Zi Xi
              mma_bf16(acc[sa + sb][1], fi, br0, br1);    // + Zi Xr
            }
          }
        }
        float hr[4] = {0.f, 0.f, 0.f, 0.f}, lr[4] = {0.f, 0.f, 0.f, 0.f};
        float hm[4] = {0.f, 0.f, 0.f, 0.f}, lm[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = r16 + gq + (e >= 2 ? 8 : 0), col = c8 + 2 * t4 + (e & 1);
          if (rowe[row] > -1000 && cole[col] > -1000) {
            const int ex = rowe[row] + cole[col];
#pragma unroll
            for (int d = kSlices - 1; d >= 0; --d) {      // smallest weights first
              const float w = pow2f(ex - 7 * (d + 2));
              dd_add(hr[e], lr[e], acc[d][0][e] * w);
              dd_add(hm[e], lm[e], acc[d][1][e] * w);
            }
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = r16 + gq + (e >= 2 ? 8 : 0), col = c8 + 2 * t4 + (e & 1);
          const int j = b * kCB + col;
          // R = gamma - X0 + S in double-float (it cancels to ~u32 |gamma|)
          const bool in = (row < n && j < n);
          const float2 gh = in ? Gh[row * n + j] : make_float2(0.f, 0.f);
          const float2 gl = in ? Gl[row * n + j] : make_float2(0.f, 0.f);
          const float2 x = X0s[row * ld + j];
          float re = gh.x, rl = gl.x, im = gh.y, il = gl.y;
          df_add(re, rl, -x.x);
          df_add(re, rl, hr[e]);
          df_add(im, il, -x.y);
          df_add(im, il, hm[e]);
          X0s[row * ld + j] = make_float2(re + (rl + lr[e]), im + (il + lm[e]));   // R replaces X0
        }
      }
    }
    block_sync<NP>();
  } else {
    // Y = chi o X0 as double-float pairs, once per system
    for (int idx = t; idx < np * np; idx += kThr) {
      const int l = idx / np;
      const float2 xh = chih[l], xl = chil[l];
      const float2 x = X0s[l * ld + (idx - l * np)];
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
        block_sync<NP>();
        for (int idx = t; idx < lc * np; idx += kThr) {
          const int r = idx / lc, ll = idx - r * lc;
          const int l = l0 + ll;
          const bool in = (r < n && l < n);
          gth[ll * np + r] = in ? Gh[r * n + l] : make_float2(0.f, 0.f);
          gtl[ll * np + r] = in ? Gl[r * n + l] : make_float2(0.f, 0.f);
        }
        block_sync<NP>();
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
          const float2 x = X0s[r * ld + col];
          const double re = g.x - (double)x.x + (((double)acc[i2][jj][0] + (double)acc[i2][jj][1]) + (double)acc[i2][jj][4]);
          const double im = g.y - (double)x.y + (((double)acc[i2][jj][2] + (double)acc[i2][jj][3]) + (double)acc[i2][jj][5]);
          A[ii][kTile + jj] = make_float2((float)re, (float)im);
        }
      }
    }
    block_sync<NP>();
    // R to shared memory (logical rows, in place of X0)
#pragma unroll
    for (int ii = 0; ii < kTile; ++ii)
#pragma unroll
      for (int jj = 0; jj < kTile; ++jj) X0s[(tr + P * ii) * ld + tc + P * jj] = A[ii][kTile + jj];
    block_sync<NP>();
  }

  // gamma o gamma^T (hi, lo) of this thread's first pass of the Gamma^(2)
  // sums below, loaded now so that their latency overlaps the diag correction
  constexpr int per_j = (P * P >= 32) ? 4 : 1;      // threads per output frequency j
  constexpr int nxj = (np + per_j - 1) / per_j;     // terms per thread
  const float2* GGh = gg_hi + mat;
  const float2* GGl = gg_lo + mat;
  float2 pgh[nxj], pgl[nxj];
  auto load_gg = [&](int idx) {
    const int j = idx / per_j, part = idx % per_j;
#pragma unroll
    for (int k = 0; k < nxj; ++k) {
      const int x = part + per_j * k;
      const bool ok = j < n && x < n;
      pgh[k] = ok ? GGh[j * n + x] : make_float2(0.f, 0.f);
      pgl[k] = ok ? GGl[j * n + x] : make_float2(0.f, 0.f);
    }
  };
  load_gg(t);

  // ---- diag E = diag(D^-1 R): the sweep's D part W holds D^-1 permuted,
  // D^-1[j][m] = W[piv[j]][ipiv[m]], so E_jj = sum_c W[r][c] R[piv[c]][j] with
  // j = ipiv[r]; the P threads of a thread row reduce by shuffles ----
  float2* ediag = invu;
  int pc[kTile];
#pragma unroll
  for (int jj = 0; jj < kTile; ++jj) pc[jj] = piv_s[tc + P * jj];
#pragma unroll
  for (int ii = 0; ii < kTile; ++ii) {
    const int j = rowpos[ii] < 0 ? 0 : rowpos[ii];
    float ex = 0.f, ey = 0.f;
#pragma unroll
    for (int jj = 0; jj < kTile; ++jj) {
      const float2 rv = X0s[pc[jj] * ld + j];
      const float2 w = A[ii][jj];
      ex = fmaf(w.x, rv.x, fmaf(-w.y, rv.y, ex));
      ey = fmaf(w.x, rv.y, fmaf(w.y, rv.x, ey));
    }
    for (int o = 1; o < P; o <<= 1) {
      ex += __shfl_xor_sync(wmask, ex, o);
      ey += __shfl_xor_sync(wmask, ey, o);
    }
    if (tc == 0 && rowpos[ii] >= 0) ediag[j] = make_float2(ex, ey);
  }
  block_sync<NP>();

  // ---- diag Gamma = diag X0 + diag E (FP64), Gamma^(2), Eq. sd bracket ----
  // Gamma^(2)_jj = sum_x (gamma_jx gamma_xj) chi~_x in double-float; four
  // threads per output frequency j (consecutive lanes, shuffle-reduced) when
  // the block has whole warps, one thread per j otherwise
  for (int base = 0; base < per_j * np; base += kThr) {
    const int idx = base + t;
    const int j = idx / per_j, part = idx % per_j;
    if (base > 0) load_gg(idx);
    float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
#pragma unroll
    for (int k = 0; k < nxj; ++k) {
      const int x = part + per_j * k;
      if (x < n) cdf_fma(sr, lr, si, li, pgh[k], pgl[k], chih[x], chil[x]);
    }
    if (per_j == 4) {
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        const float osr = __shfl_xor_sync(0xffffffffu, sr, o), olr = __shfl_xor_sync(0xffffffffu, lr, o);
        const float osi = __shfl_xor_sync(0xffffffffu, si, o), oli = __shfl_xor_sync(0xffffffffu, li, o);
        df_add(sr, lr, osr);
        lr += olr;
        df_add(si, li, osi);
        li += oli;
      }
    }
    const double2 g2 = mk((double)sr + (double)lr, (double)si + (double)li);
    if (j < n && part == 0) {
      const float2 x0 = x0d[j], e = ediag[j];
      const double2 gdiag = mk((double)x0.x + (double)e.x, (double)x0.y + (double)e.y);
      const double wgt = (c == 0) ? 1.0 : 3.0;
      kc[(((size_t)c * nb + a) * n + j) * N + q] =
          mk(wgt * (gdiag.x - 0.5 * g2.x), wgt * (gdiag.y - 0.5 * g2.y));
    }
  }
  // per-ladder error control: the size of the correction against diag Gamma
  if (t == 0) {
    float emax = 0.f, gmax = 0.f;
    bool fin = true;
    for (int j = 0; j < n; ++j) {
      const float2 x0 = x0d[j], e = ediag[j];
      const float ea = fabsf(e.x) + fabsf(e.y), ga = fabsf(x0.x + e.x) + fabsf(x0.y + e.y);
      fin = fin && isfinite(ea) && isfinite(ga);
      emax = fmaxf(emax, ea);
      gmax = fmaxf(gmax, ga);
    }
    mixed_check_ladder(mc, emax, gmax, fin, ((long)c * nb + a) * N + q, flags);
  }
  block_sync<NP>();
}

// The producer warp's side of bse_mixed_system<64> for one system: per
// column block, wait for the compute warps' handoff, then (lane 0) issue the
// 32 MMAs (gamma slice sa: A = [Zr; Zi] of slice sa, B = the Y slices 0 .. 7 - sa
// stacked along N, D at TMEM buffer b & 1, column 32 sa) and commit them.
__device__ __forceinline__ void mixed_producer(const MixedPtrs& sp, const Tc05* umma) {
  constexpr int np = 64;
  const unsigned za = smem_u32(sp.work), xa = smem_u32(sp.work + xs_offset(np));
  const int lane = threadIdx.x & 31;
  for (int b = 0; b < np / kCB; ++b) {
    handoff_wait();
    if (lane == 0) {
      tc05_fence_after();
      const unsigned dt = umma->tmem + (unsigned)(256 * (b & 1));
#pragma unroll 1
      for (int sa = 0; sa < kSlices; ++sa) {
        const unsigned idesc = umma_idesc_bf16(128, 32 * (kSlices - sa));
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          umma_bf16(dt + 32 * sa, umma_desc_sw128(za + sa * (2 * np * 128) + 32 * ks), umma_desc_sw128(xa + 32 * ks),
                    idesc, (sa > 0 || ks > 0) ? 1u : 0u);
      }
      umma_commit(umma->mbar);
    }
    __syncwarp();
  }
}

}  // namespace df
