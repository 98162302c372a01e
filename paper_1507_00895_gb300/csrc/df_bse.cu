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
               double2* __restrict__ kc, double2* __restrict__ ws, int* __restrict__ flags) {
  extern __shared__ double2 sm[];
  __shared__ BseF64Shared sh;
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  const BseSmem L = bse_layout(n, nc, LU_SMEM);
  double2* LU = LU_SMEM ? sm + L.lu : ws + (size_t)blockIdx.x * n * n;
  const long systems = (long)nch * nb * N;
  for (long sys = blockIdx.x; sys < systems; sys += gridDim.x) {
    const int c = ch0 + (int)(sys / ((long)nb * N));
    const int rem = (int)(sys - (long)(c - ch0) * nb * N);
    const int a = rem / N, q = rem - a * N;
    bse_f64_system(dm, c, a, q, nc, gam, gg, chi, kc, LU, sm + L.y, sm + L.xs, sm + L.invu, sh, flags);
  }
}

// ---------------------------------------------------------------------------
// leading eigenvalue of A = gamma_W diag(chi~_W(q)) by FP64 power iteration
// with a Rayleigh-quotient estimate.  One CTA handles kEigQ systems that
// share (channel, W): gamma_W is staged in shared memory once (when it
// fits) and each thread owns (row, system) pairs of y = A v, so one
// iteration is n^2 complex multiply-adds per system with no reductions
// except the per-system Rayleigh quotient.  A system is "converged" when
// the estimate changes by less than tol relative; iterations stop when all
// kEigQ systems converged or after kEigMaxIter.
// ---------------------------------------------------------------------------
constexpr int kEigQ = 8;
constexpr int kEigThreads = 256;
constexpr int kEigMaxIter = 64;

__global__ void __launch_bounds__(kEigThreads)
lambda_kernel(Dims dm, int ch0, int a0, int na, int g_in_smem, double tol, const double2* __restrict__ gam,
              const double2* __restrict__ chi, double2* __restrict__ lam, int* __restrict__ ok,
              int* __restrict__ flags) {
  extern __shared__ double2 sm[];
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  double2* v = sm;                 // [n][kEigQ] current unit vector
  double2* xq = v + n * kEigQ;     // [n][kEigQ] chi~ of the kEigQ systems
  double2* y = xq + n * kEigQ;     // [n][kEigQ] A v
  double2* Gs = y + n * kEigQ;     // [n][n] gamma_W (if g_in_smem)
  __shared__ double2 lam_old[kEigQ], lam_new[kEigQ];
  __shared__ double nrm[kEigQ];
  __shared__ int done[kEigQ];
  const int qtiles = (N + kEigQ - 1) / kEigQ;
  const int tile = blockIdx.x % qtiles;
  const int a = a0 + blockIdx.x / qtiles;
  const int c = ch0;
  if (a >= a0 + na) return;
  const int q0 = tile * kEigQ;
  const int nq = min(kEigQ, N - q0);
  const double2* Gg = gam + ((size_t)c * nb + a) * n * n;
  const double2* G = g_in_smem ? Gs : Gg;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double inv_sqrt_n = rsqrt((double)n);

  if (g_in_smem)
    for (int idx = tid; idx < n * n; idx += blockDim.x) Gs[idx] = Gg[idx];
  for (int idx = tid; idx < n * kEigQ; idx += blockDim.x) {
    const int j = idx / kEigQ, t = idx % kEigQ;
    xq[idx] = (t < nq) ? chi[((size_t)a * n + j) * N + q0 + t] : mk(0.0, 0.0);
    v[idx] = mk(inv_sqrt_n, 0.0);
  }
  if (tid < kEigQ) {
    lam_old[tid] = mk(0.0, 0.0);
    lam_new[tid] = mk(0.0, 0.0);
    done[tid] = (tid < nq) ? 0 : 1;
  }
  __syncthreads();
  for (int it = 0; it < kEigMaxIter; ++it) {
    // y[i][t] = sum_j G[i][j] chi[j][t] v[j][t]
    for (int pidx = tid; pidx < n * kEigQ; pidx += blockDim.x) {
      const int i = pidx / kEigQ, t = pidx % kEigQ;
      double2 acc = mk(0.0, 0.0);
      for (int j = 0; j < n; ++j)
        acc = cfma(G[i * n + j], cmul(xq[j * kEigQ + t], v[j * kEigQ + t]), acc);
      y[pidx] = acc;
    }
    __syncthreads();
    // per system: Rayleigh quotient v^H y (|v| = 1) and 1/|y|
    if (warp < kEigQ) {
      const int t = warp;
      double2 rq = mk(0.0, 0.0);
      double yy = 0.0;
      for (int j = lane; j < n; j += 32) {
        const double2 vj = v[j * kEigQ + t], yj = y[j * kEigQ + t];
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
        nrm[t] = yy > 0.0 ? rsqrt(yy) : 0.0;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < n * kEigQ; idx += blockDim.x) v[idx] = cscale(y[idx], nrm[idx % kEigQ]);
    if (tid < kEigQ && !done[tid]) {
      const double2 d = lam_new[tid] - lam_old[tid];
      if (sqrt(cabs2(d)) <= tol * sqrt(cabs2(lam_new[tid]))) done[tid] = 1;
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
    lam[o] = lam_new[tid];
    ok[o] = done[tid];
    if (cabs2(lam_new[tid]) >= 1.0) atomicOr(flags, 2);
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

static int bse_chunk(int n) { return n <= 32 ? n : (n <= 64 ? 32 : 16); }
static bool bse_lu_in_smem(int n) { return n <= 96; }

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
  cudaError_t e = cudaMemsetAsync(flag_ptr(c), 0, sizeof(int) * 4, c->stream);
  if (e != cudaSuccess) return e;
  if (c->opts.precision == DF_FP32_IR) return launch_bse_mixed(c, channel_mask, gg_ptr(c), flag_ptr(c));
  for (int ch = 0; ch < 2; ++ch) {
    if (!(channel_mask & (1 << ch))) continue;
    const long systems = (long)dm.nb * dm.N;
    const int grid = (int)(systems < c->bse_grid ? systems : c->bse_grid);
    if (bse_lu_in_smem(n)) {
      bse_f64_kernel<true><<<grid, kBseThreads, smem, c->stream>>>(dm, ch, 1, nc, c->gam, gg_ptr(c), c->chi,
                                                                   c->kc, nullptr, flag_ptr(c));
    } else {
      bse_f64_kernel<false><<<grid, kBseThreads, smem, c->stream>>>(dm, ch, 1, nc, c->gam, gg_ptr(c), c->chi,
                                                                    c->kc, lu_ws_ptr(c), flag_ptr(c));
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_lambda(df_ctx* c, int channel_mask) {
  const Dims& dm = c->dm;
  if (c->opts.eig_mode == 0) return cudaSuccess;
  const int a0 = (c->opts.eig_mode == 1) ? dm.m_max : 0;
  const int na = (c->opts.eig_mode == 1) ? 1 : dm.nb;
  const int qtiles = (dm.N + kEigQ - 1) / kEigQ;
  const int g_in_smem = dm.n_w <= 96;
  const size_t smem = sizeof(double2) * (3 * dm.n_w * kEigQ + (g_in_smem ? dm.n_w * dm.n_w : 0));
  cudaError_t e = cudaFuncSetAttribute((const void*)lambda_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  for (int ch = 0; ch < 2; ++ch) {
    if (!(channel_mask & (1 << ch))) continue;
    lambda_kernel<<<qtiles * na, kEigThreads, smem, c->stream>>>(dm, ch, a0, na, g_in_smem, 1e-12, c->gam,
                                                                 c->chi, c->lam, c->lam_ok, flag_ptr(c));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
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
  if (!bse_lu_in_smem(dm.n_w)) return cudaErrorInvalidValue;
  const int nc = bse_chunk(dm.n_w);
  const size_t smem = bse_smem_bytes(dm.n_w);
  const int grid_max = bse_default_grid(dm, device);   // sets the shared-memory attribute
  const long systems = 2L * dm.nb * dm.N;
  const int grid = (int)(systems < grid_max ? systems : grid_max);
  bse_f64_kernel<true><<<grid, kBseThreads, smem, stream>>>(dm, 0, 2, nc, gam, gg, chi, kc, nullptr, flags);
  return cudaGetLastError();
}

}  // namespace df
