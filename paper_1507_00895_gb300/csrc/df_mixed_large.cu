// Mixed-precision ladder solves (DF_FP32_IR) of order 64 < n <= 128, where the
// register tile of the n <= 64 kernel (df_mixed.cu) no longer fits: the same
// Eq. lin_alg_inv, D Gamma = gamma with D = 1 - gamma_W diag(chi~_W(q)), and
// the same output, kc = w_c (Gamma_jj - Gamma^(2)_jj / 2) (Eq. sd bracket).
//
// Per (q, W, channel), one CTA of 2n threads (rounded up to a warp):
//   1. D in double-float from gamma's and chi~'s (hi, lo) FP32 words, rounded
//      once to FP32 (the diagonal 1 - gamma_ww chi~_w cancels; rounded
//      factors would lose those digits), in shared memory, row stride n + 1.
//   2. S = (P D)^-1 in FP32 by Gauss-Jordan in place with partial pivoting
//      (largest |re| + |im|, lowest row on ties; full row exchanges), two
//      barriers per column: the threads of column k+1 leave per-row-group
//      pivot candidates during column k's update.
//   3. Right-hand sides in chunks of 8 columns j:
//        Y = S (P gamma)                       FP32 product, n^2 per column
//        R = gamma - Y + gamma (chi~ o Y)      double-float (packed f32x2), n^2 per column
//        Gamma_jj = Y_jj + (S (P R))_jj        one row of S: n per column
//      (D Y = Y - gamma diag(chi~) Y; D^-1 R = S (P R)).  One correction: the
//      error left is ~(cond(D) 2^-24)^2 plus cond(D) times the double-float
//      residual's ~2^-46 relative to sum_k |gamma_ik| |(chi~ o Y)_kj|.
//   4. Gamma^(2)_jj = sum_x (gamma o gamma^T)_jx chi~_x in FP64, n per column.
// gamma's words come from the mixed-precision workspace: the leading words
// row-major (slot 0) and, for these orders, the transpose's leading and
// trailing words (slots 2 and 3), so that a warp's 32 rows read one
// contiguous 256-byte line per k in the residual product.
#include "df_mixed_large_dev.cuh"
#include "df_tcr_dev.cuh"

namespace df {

// gamma^T's (hi, lo) FP32 words: out_hi[c][a][k][i] = hi(gamma[c][a][i][k])
__global__ void split_gamma_t_kernel(int n, size_t mats, const double2* __restrict__ g, float2* __restrict__ th,
                                     float2* __restrict__ tl) {
  const size_t count = mats * n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t m = e / ((size_t)n * n);
    const int r = (int)(e - m * n * n);
    const int k = r / n, i = r - k * n;
    const double2 v = g[m * n * n + (size_t)i * n + k];
    const float hx = (float)v.x, hy = (float)v.y;
    th[e] = make_float2(hx, hy);
    tl[e] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
  }
}

__global__ void __launch_bounds__(256, 1)
bse_gj_ir_kernel(Dims dm, int ch0, int nch, const float2* __restrict__ ghi, const float2* __restrict__ glo,
                 const float2* __restrict__ gth, const float2* __restrict__ gtl, const double2* __restrict__ gg,
                 const double2* __restrict__ chi, double2* __restrict__ kc, int* __restrict__ flags,
                 MixedCheck mc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ GjShared sh;
  const long systems = (long)nch * dm.na * dm.N;
  for (long sys = blockIdx.x; sys < systems; sys += gridDim.x) {
    const int c = ch0 + (int)(sys / ((long)dm.na * dm.N));
    const int rem = (int)(sys - (long)(c - ch0) * dm.na * dm.N);
    const int a = dm.a0 + rem / dm.N, q = rem - (a - dm.a0) * dm.N;
    gj_ir_system(dm, c, a, q, ghi, glo, gth, gtl, gg, chi, kc, flags, smraw, sh, mc);
  }
}

// The same ladders with the Gauss-Jordan inversion on the tensor cores
// (df_tcgj_dev.cuh): 256 threads, 256 TMEM columns per block, two blocks per
// SM (the launch asks for enough shared memory that no third fits), systems
// strided over the persistent grid.  A completion wait that gives up stops
// the block: it sets kFlagTcTimeout, waits (bounded) for its last MMAs and
// frees its tensor memory.
constexpr int kTcTmemCols = 256;

__global__ void __launch_bounds__(kTcThreads, 2)
bse_tc_ir_kernel(Dims dm, int ch0, int nch, const float2* __restrict__ ghi, const float2* __restrict__ glo,
                 const float2* __restrict__ gth, const float2* __restrict__ gtl, const double2* __restrict__ gg,
                 const double2* __restrict__ chi, double2* __restrict__ kc, int* __restrict__ flags,
                 MixedCheck mc) {
  extern __shared__ __align__(1024) unsigned char smtc[];
  __shared__ GjShared sh;
  __shared__ uint64_t mbar_s;
  __shared__ unsigned tslot_s;
  if (smem_u32(smtc) & 1023u) {                  // the swizzled operand tiles need 1024-byte alignment
    if (threadIdx.x == 0) atomicOr(flags, kFlagTcLayout);
    return;
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc_cols<kTcTmemCols>(&tslot_s);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_s)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  GjTc tc{tslot_s, &mbar_s, 0u};
  bool ok = true;
  const long systems = (long)nch * dm.na * dm.N;
  for (long sys = blockIdx.x; sys < systems && ok; sys += gridDim.x) {
    const int c = ch0 + (int)(sys / ((long)dm.na * dm.N));
    const int rem = (int)(sys - (long)(c - ch0) * dm.na * dm.N);
    const int a = dm.a0 + rem / dm.N, q = rem - (a - dm.a0) * dm.N;
    ok = gj_ir_system<true>(dm, c, a, q, ghi, glo, gth, gtl, gg, chi, kc, flags, smtc, sh, mc, &tc);
  }
  if (!ok && threadIdx.x == 0) mbar_wait(&mbar_s, tc.phase ^ 1u);   // the abandoned commit, bounded
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc_cols<kTcTmemCols>(tc.tmem);
}

// Orders 64 < n <= 96 with the residual on the tensor cores too
// (df_tcr_dev.cuh): 256 threads, all 512 TMEM columns, one block per SM.
__global__ void tcr_gamma_digits_kernel(int n, int count, const double2* __restrict__ gam,
                                        unsigned char* __restrict__ out, int* __restrict__ rowe) {
  tcr_gamma_digits_rows(n, count, gam, out, rowe, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                        (gridDim.x * blockDim.x) >> 5, threadIdx.x & 31);
}

__global__ void __launch_bounds__(kTcThreads, 1)
bse_tcr_kernel(Dims dm, int ch0, int nch, const float2* __restrict__ ghi, const float2* __restrict__ glo,
               const double2* __restrict__ gg, const unsigned char* __restrict__ gdig, const int* __restrict__ growe,
               const double2* __restrict__ chi, double2* __restrict__ kc, int* __restrict__ flags, MixedCheck mc) {
  extern __shared__ __align__(1024) unsigned char smtcr[];
  __shared__ int piv_s[128], ipiv_s[128];
  __shared__ uint64_t bars_s[1 + 2 * kTcrBufs];   // sweep / fold, full[kTcrBufs], empty[kTcrBufs]
  __shared__ unsigned tslot_s;
  if (smem_u32(smtcr) & 1023u) {
    if (threadIdx.x == 0) atomicOr(flags, kFlagTcLayout);
    return;
  }
  {                                    // Y digits: K beyond n stays zero for the whole launch
    const TcrLayout L = tcr_layout(dm.n_w);
    uint4* y = reinterpret_cast<uint4*>(smtcr + L.ystk);
    for (int i = threadIdx.x; i < 128 * 2 * 128 / 16; i += blockDim.x) y[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc_cols<512>(&tslot_s);
  if (threadIdx.x == 0) {
    for (int b = 0; b < 1 + 2 * kTcrBufs; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars_s[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  TcrState st;
  st.tmem = tslot_s;
  st.mbar = &bars_s[0];
  st.full = &bars_s[1];
  st.empty = &bars_s[1 + kTcrBufs];
  st.phase = 0u;
  for (int b = 0; b < kTcrBufs; ++b) st.fphase[b] = st.ephase[b] = 0u;
  bool ok = true;
  const long systems = (long)nch * dm.na * dm.N;
  for (long sys = blockIdx.x; sys < systems && ok; sys += gridDim.x) {
    const int c = ch0 + (int)(sys / ((long)dm.na * dm.N));
    const int rem = (int)(sys - (long)(c - ch0) * dm.na * dm.N);
    const int a = dm.a0 + rem / dm.N, q = rem - (a - dm.a0) * dm.N;
    ok = tcr_system(dm, c, a, q, ghi, glo, gg, gdig, growe, chi, kc, flags, smtcr, piv_s, ipiv_s, st, mc);
  }
  if (!ok && threadIdx.x == 0) {       // bounded waits for what may still be in flight
    mbar_wait(st.mbar, st.phase ^ 1u);
    for (int b = 0; b < kTcrBufs; ++b) mbar_wait(&st.full[b], st.fphase[b]);
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc_cols<512>(st.tmem);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

size_t gj_smem_bytes(int n_w) { return (size_t)gj_layout(n_w).total; }

// gamma's digit chunks of the tensor-core residual (orders 64 < n <= 96),
// after the mixed workspace's other parts
size_t tcr_workspace_bytes(const Dims& dm) {
  if (!tcr_supported(dm.n_w)) return 0;
  return (size_t)2 * dm.nb * (tcr_gdig_bytes() + 2 * 128 * sizeof(int));
}
static unsigned char* tcr_gdig_ptr(df_ctx* c) { return (unsigned char*)c->mixed_ws + c->tcr_off; }
static int* tcr_rowe_ptr(df_ctx* c) {
  return (int*)(tcr_gdig_ptr(c) + (size_t)2 * c->dm.nb * tcr_gdig_bytes());
}

// gamma^T's (hi, lo) words into workspace slots 2 and 3 (orders > 64); the
// tensor-core residual's digit chunks where that kernel takes the order
cudaError_t launch_split_gamma_t(df_ctx* c) {
  const Dims& dm = c->dm;
  const size_t count = (size_t)2 * dm.nb * dm.n_w * dm.n_w;
  float2* ws = (float2*)c->mixed_ws;
  split_gamma_t_kernel<<<256, 256, 0, c->stream>>>(dm.n_w, (size_t)2 * dm.nb, c->gam, ws + 2 * count, ws + 3 * count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !tcr_supported(dm.n_w)) return e;
  const int warps = 2 * dm.nb * 128;
  tcr_gamma_digits_kernel<<<(warps + 7) / 8, 256, 0, c->stream>>>(dm.n_w, 2 * dm.nb, c->gam, tcr_gdig_ptr(c),
                                                                  tcr_rowe_ptr(c));
  return cudaGetLastError();
}

// orders 64 < n <= 96: sweep and residual on the tensor cores, one block per SM
static cudaError_t launch_bse_tcr(df_ctx* c, int channel_mask, int* flags) {
  const Dims& dm = c->dm;
  const size_t smem = (size_t)tcr_layout(dm.n_w).total;
  cudaError_t e = cudaFuncSetAttribute((const void*)bse_tcr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) return e;
  const size_t count = (size_t)2 * dm.nb * dm.n_w * dm.n_w;
  const float2* ws = (const float2*)c->mixed_ws;
  const MixedCheck mc = mixed_check(c);
  for (int ch = 0; ch < 2; ++ch) {
    if (!(channel_mask & (1 << ch))) continue;
    const long systems = (long)dm.na * dm.N;
    bse_tcr_kernel<<<(int)(systems < sms ? systems : sms), kTcThreads, smem, c->stream>>>(
        dm, ch, 1, ws, ws + count, gamma_gt_ptr(c), tcr_gdig_ptr(c), tcr_rowe_ptr(c), c->chi, c->kc, flags, mc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// the tensor-core variant: at most two blocks per SM (256 TMEM columns each)
static cudaError_t launch_bse_tc_large(df_ctx* c, int channel_mask, int* flags) {
  const Dims& dm = c->dm;
  const int n = dm.n_w;
  size_t smem = (size_t)gj_layout(n, true).total;
  if (smem < 80 * 1024) smem = 80 * 1024;         // no third block per SM (its TMEM allocation would wait)
  cudaError_t e = cudaFuncSetAttribute((const void*)bse_tc_ir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)bse_tc_ir_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  // blocks per SM from shared memory alone (the register cap of the launch bounds
  // allows two; the occupancy calculator reports one for any kernel that
  // allocates tensor memory, while two 256-column allocations fit the SM's 512)
  int sms = 0, sm_smem = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device)) != cudaSuccess)
    return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, (const void*)bse_tc_ir_kernel)) != cudaSuccess) return e;
  int per_sm = (int)((size_t)sm_smem / (smem + fa.sharedSizeBytes + 1024));
  per_sm = per_sm < 1 ? 1 : (per_sm > 2 ? 2 : per_sm);
  const size_t count = (size_t)2 * dm.nb * n * n;
  const float2* ws = (const float2*)c->mixed_ws;
  const MixedCheck mc = mixed_check(c);
  for (int ch = 0; ch < 2; ++ch) {
    if (!(channel_mask & (1 << ch))) continue;
    const long systems = (long)dm.na * dm.N;
    const long grid = (long)sms * per_sm;
    bse_tc_ir_kernel<<<(int)(systems < grid ? systems : grid), kTcThreads, smem, c->stream>>>(
        dm, ch, 1, ws, ws + count, ws + 2 * count, ws + 3 * count, gamma_gt_ptr(c), c->chi, c->kc, flags, mc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_bse_mixed_large(df_ctx* c, int channel_mask, int* flags) {
  const Dims& dm = c->dm;
  const int n = dm.n_w;
  if (n > kGjMaxN) return cudaErrorInvalidValue;
  if (c->opts.mixed_sweep == 0)
    return tcr_supported(n) ? launch_bse_tcr(c, channel_mask, flags) : launch_bse_tc_large(c, channel_mask, flags);
  const size_t smem = gj_smem_bytes(n);
  const int threads = gj_threads(n);
  cudaError_t e = cudaFuncSetAttribute((const void*)bse_gj_ir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)bse_gj_ir_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int sms = 0, per_sm = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)bse_gj_ir_kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const size_t count = (size_t)2 * dm.nb * n * n;
  const float2* ws = (const float2*)c->mixed_ws;
  const MixedCheck mc = mixed_check(c);
  for (int ch = 0; ch < 2; ++ch) {
    if (!(channel_mask & (1 << ch))) continue;
    const long systems = (long)dm.na * dm.N;
    const long grid = (long)sms * per_sm;
    bse_gj_ir_kernel<<<(int)(systems < grid ? systems : grid), threads, smem, c->stream>>>(
        dm, ch, 1, ws, ws + count, ws + 2 * count, ws + 3 * count, gamma_gt_ptr(c), c->chi, c->kc, flags, mc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace df
