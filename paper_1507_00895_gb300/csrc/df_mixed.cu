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
#include "df_mixed_dev.cuh"

namespace df {

// gamma and gamma o gamma^T (FP64) -> (hi, lo) FP32 pairs, same layouts
__global__ void split_gamma_kernel(size_t count, const double2* __restrict__ g, const double2* __restrict__ gg,
                                   float2* __restrict__ hi, float2* __restrict__ lo, float2* __restrict__ gg_hi,
                                   float2* __restrict__ gg_lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = g[i];
    float hx = (float)v.x, hy = (float)v.y;
    hi[i] = make_float2(hx, hy);
    lo[i] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
    const double2 w = gg[i];
    hx = (float)w.x; hy = (float)w.y;
    gg_hi[i] = make_float2(hx, hy);
    gg_lo[i] = make_float2((float)(w.x - (double)hx), (float)(w.y - (double)hy));
  }
}

// gamma's digits for the tensor-core residual (once per input upload)
__global__ void gamma_digits_kernel(int n, int np, int count, const double2* __restrict__ gam,
                                    unsigned char* __restrict__ out) {
  gamma_digits_rows(n, np, count, gam, out, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                    (gridDim.x * blockDim.x) >> 5, threadIdx.x & 31);
}

// One contiguous range of systems per block (so that consecutive systems
// share (channel, W) and gamma's digits stay in shared memory).
template <int NP>
__global__ void __launch_bounds__(mixed_block_threads(NP), use_umma_residual(NP) ? 1 : 0)
bse_mixed_kernel(Dims dm, int ch0, int nch, const double2* __restrict__ gam,
                 const float2* __restrict__ gam_hi, const float2* __restrict__ gam_lo,
                 const float2* __restrict__ gg_hi, const float2* __restrict__ gg_lo,
                 const double2* __restrict__ chi, double2* __restrict__ kc,
                 const unsigned char* __restrict__ gdig, int* __restrict__ flags, MixedCheck mc) {
  extern __shared__ __align__(1024) float2 smf[];
  __shared__ int piv_s[128];
  __shared__ uint64_t mbar_s[2];
  __shared__ unsigned tslot_s;
  const MixedPtrs sp = mixed_ptrs(smf, NP, piv_s);
  Tc05 tc{};
  if constexpr (use_umma_residual(NP)) {
    // the swizzled operand tiles need a 1024-aligned work area
    if (smem_u32(sp.work) & 1023u) {
      if (threadIdx.x == 0) atomicOr(flags, kFlagTcLayout);
      return;
    }
    tc05_setup(tc, mbar_s, &tslot_s);
  }
  const int N = dm.N, nb = dm.nb, na = dm.na;
  const long systems = (long)nch * na * N;
  const long per = (systems + gridDim.x - 1) / gridDim.x;
  const long s0 = (long)blockIdx.x * per, s1 = s0 + per < systems ? s0 + per : systems;
  int cur = -1;
  for (long sys = s0; sys < s1; ++sys) {
    const int c = ch0 + (int)(sys / ((long)na * N));
    const int rem = (int)(sys - (long)(c - ch0) * na * N);
    const int a = dm.a0 + rem / N, q = rem - (a - dm.a0) * N;
    const int key = c * nb + a;
    if (use_umma_residual(NP) && (threadIdx.x >> 5) == mixed_compute_threads(NP) / 32)
      mixed_producer(sp, &tc);                        // warp 8: the tensor-core MMAs
    else
      bse_mixed_system<NP>(dm, c, a, q, gam, gam_hi, gam_lo, gg_hi, gg_lo, chi, kc, flags, sp,
                           gdig ? gdig + (size_t)key * gdig_bytes(NP) : nullptr, key != cur, &tc, mc);
    cur = key;
  }
  if constexpr (use_umma_residual(NP)) tc05_teardown(tc, mixed_compute_threads(NP));
}

// Self-test of the bounded wait the tensor-core residual uses: one warp
// initialises an mbarrier (one arrival expected), arrives on it only when
// `arrive` is set, and waits for its first phase with a limit of `spins`
// polls; a wait that gives up sets kFlagTcTimeout.  Nothing else runs.
__global__ void wait_selftest_kernel(int arrive, unsigned spins, int* __restrict__ flags) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&mbar)) : "memory");
  }
  if (!mbar_wait(&mbar, 0, spins) && threadIdx.x == 0) atomicOr(flags, kFlagTcTimeout);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

cudaError_t launch_wait_selftest(int arrive, unsigned spins, int* flags, cudaStream_t stream) {
  wait_selftest_kernel<<<1, 32, 0, stream>>>(arrive, spins, flags);
  return cudaGetLastError();
}

static int mixed_np(int n) { return mixed_pad(n); }

// the register-resident [D | RHS] tile limits this kernel to n_w <= 64; orders
// up to 128 take the shared-memory Gauss-Jordan kernel of df_mixed_large.cu
bool mixed_supported(int n_w) { return mixed_np(n_w) <= 128; }

// gamma hi, lo; gamma o gamma^T hi, lo (orders > 64: gamma^T hi, lo); gamma's
// digits (tensor-core residual); then the error control's words: the call's
// largest rho^2 and the hand-back list (count + 2 N_W N system indices)
static size_t mixed_check_offset(const Dims& dm) {
  const int np = mixed_np(dm.n_w);
  const size_t digits = use_tc_residual(np) ? (size_t)2 * dm.nb * gdig_bytes(np) : 0;
  return ((size_t)4 * 2 * dm.nb * dm.n_w * dm.n_w * sizeof(float2) + digits + 15) & ~(size_t)15;
}
size_t mixed_tcr_offset(const Dims& dm) {
  return (mixed_check_offset(dm) + sizeof(int) * (4 + (size_t)2 * dm.nb * dm.N) + 1023) & ~(size_t)1023;
}
size_t mixed_workspace_bytes(const Dims& dm) { return mixed_tcr_offset(dm) + tcr_workspace_bytes(dm); }
// [0] worst rho^2 (float bits), [1] unused, [2] hand-back count, [3 ..] list
unsigned* mixed_check_words(df_ctx* c) { return (unsigned*)((char*)c->mixed_ws + mixed_check_offset(c->dm)); }

MixedCheck mixed_check(df_ctx* c) {
  unsigned* w = mixed_check_words(c);
  MixedCheck mc;
  mc.worst = w;
  mc.redo = c->opts.ladder_fallback ? (int*)(w + 2) : nullptr;
  mc.rho2_max = (float)c->opts.ladder_tol;
  mc.base = 0;
  return mc;
}

static unsigned char* gdig_ptr(df_ctx* c) {
  const int np = mixed_np(c->dm.n_w);
  if (!use_tc_residual(np)) return nullptr;
  return (unsigned char*)c->mixed_ws + (size_t)4 * 2 * c->dm.nb * c->dm.n_w * c->dm.n_w * sizeof(float2);
}

cudaError_t launch_split_gamma(df_ctx* c, const double2* gg) {
  const Dims& dm = c->dm;
  const size_t count = (size_t)2 * dm.nb * dm.n_w * dm.n_w;
  float2* hi = (float2*)c->mixed_ws;
  split_gamma_kernel<<<256, 256, 0, c->stream>>>(count, c->gam, gg, hi, hi + count, hi + 2 * count, hi + 3 * count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (mixed_np(dm.n_w) > 64) return launch_split_gamma_t(c);   // slots 2, 3: gamma^T's words
  if (unsigned char* gd = gdig_ptr(c)) {
    const int np = mixed_np(dm.n_w), rows = 2 * dm.nb * np;
    gamma_digits_kernel<<<(rows + 7) / 8, 256, 0, c->stream>>>(dm.n_w, np, 2 * dm.nb, c->gam, gd);
    e = cudaGetLastError();
  }
  return e;
}

template <int NP>
static cudaError_t launch_bse_mixed_np(df_ctx* c, int channel_mask, int* flags) {
  const Dims& dm = c->dm;
  constexpr int threads = mixed_block_threads(NP);   // + the producer warp at n_pad = 64
  const size_t smem = sizeof(float2) * (size_t)mixed_layout(NP).total;
  cudaError_t e = cudaFuncSetAttribute((const void*)bse_mixed_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (c->mixed_grid == 0) {
    int per_sm = 0, sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bse_mixed_kernel<NP>, threads, smem);
    c->mixed_grid = sms * (per_sm < 1 ? 1 : per_sm);
  }
  const size_t count = (size_t)2 * dm.nb * dm.n_w * dm.n_w;
  const float2* hi = (const float2*)c->mixed_ws;
  const MixedCheck mc = mixed_check(c);
  // one launch per channel; both channels in one launch when a channel is only a
  // few waves of the grid (the reduced grids), where the last partial wave of
  // each launch would otherwise idle most blocks
  const long per_channel = (long)dm.na * dm.N;
  const bool both = (channel_mask & 3) == 3 && per_channel < 16L * c->mixed_grid;
  for (int ch = 0; ch < 2; ++ch) {
    if (!(channel_mask & (1 << ch))) continue;
    const int nch = both ? 2 : 1;
    const long systems = nch * per_channel;
    const int grid = (int)(systems < c->mixed_grid ? systems : c->mixed_grid);
    bse_mixed_kernel<NP><<<grid, threads, smem, c->stream>>>(dm, ch, nch, c->gam, hi, hi + count, hi + 2 * count,
                                                             hi + 3 * count, c->chi, c->kc, gdig_ptr(c), flags, mc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (both) break;
  }
  return cudaSuccess;
}

// the mixed-precision ladder solves of one df_bse call, then the FP64 LU over
// the ladders whose predicted error exceeded the bound (none: its blocks exit
// at once).  The caller zeroes the check words before (run_ladders).
cudaError_t launch_bse_mixed(df_ctx* c, int channel_mask, int* flags) {
  cudaError_t e;
  switch (mixed_np(c->dm.n_w)) {
    case 8: e = launch_bse_mixed_np<8>(c, channel_mask, flags); break;
    case 16: e = launch_bse_mixed_np<16>(c, channel_mask, flags); break;
    case 32: e = launch_bse_mixed_np<32>(c, channel_mask, flags); break;
    case 64: e = launch_bse_mixed_np<64>(c, channel_mask, flags); break;
    case 128: e = launch_bse_mixed_large(c, channel_mask, flags); break;   // df_mixed_large.cu
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess || !c->opts.ladder_fallback) return e;
  return launch_bse_f64_list(c, (const int*)(mixed_check_words(c) + 2));
}

}  // namespace df
