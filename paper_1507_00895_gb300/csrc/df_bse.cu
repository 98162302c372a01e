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
               const double2* __restrict__ lam) {
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
    bse_f64_system(dm, c, a, q, nc, gam, gg, chi, kc, LU, sm + L.y, sm + L.xs, sm + L.invu, sh, flags, radius_K,
                   lam);
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

template <bool LU_SMEM>
__global__ void __launch_bounds__(kBseThreads)
chi_ladder_kernel(Dims dm, const double2* __restrict__ gam, const double2* __restrict__ chi,
                  const double2* __restrict__ Lb, const double2* __restrict__ chi0, double2* __restrict__ out,
                  double2* __restrict__ ws, int* __restrict__ flags) {
  extern __shared__ double2 sm[];
  __shared__ BseF64Shared sh;
  const int n = dm.n_w, N = dm.N, nb = dm.nb;
  const BseSmem L = bse_layout(n, 2, LU_SMEM);
  double2* LU = LU_SMEM ? sm + L.lu : ws + (size_t)blockIdx.x * n * n;
  const long systems = 2L * nb * N;
  for (long sys = blockIdx.x; sys < systems; sys += gridDim.x) {
    const int c = (int)(sys / ((long)nb * N));
    const int rem = (int)(sys - (long)c * nb * N);
    const int a = rem / N, q = rem - a * N;
    chi_ladder_system(dm, c, a, q, gam, chi, Lb, chi0, out, LU, sm + L.y, sm + L.xs, sm + L.invu, sh, flags);
  }
}

// ---------------------------------------------------------------------------
// leading eigenvalue of A = gamma_W diag(chi~_W(q)): power iteration with a
// Rayleigh-quotient estimate, first in FP32 (gamma staged in shared memory
// as complex64) until the estimate settles to FP32 precision, then polished
// from that vector with FP64 vectors and Rayleigh quotients, the products
// gamma (chi~ o v) in double-float FP32 (gamma staged as (hi, lo) pairs;
// ~2^-46 relative, far below the 1e-12 stopping tolerance).  The reported
// value and its converged flag are those of the polish.  One CTA handles
// kEigQ systems that share (channel, W); each thread owns (row, system)
// pairs of y = A v.
// ---------------------------------------------------------------------------
constexpr int kEigQ = 8;
constexpr int kEigThreads = 256;
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
  if (tid < kEigQ) done[tid] = (tid < nq) ? 0 : 1;
  __syncthreads();
  float2* wh = x32;                        // chi~ o v as (hi, lo) pairs; x32, y32 are free now
  float2* wl = y32;
  for (int it = 0; it < kEigIter64; ++it) {
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
    lam[o] = lam_new[tid];
    ok[o] = done[tid];
    if (cabs2(lam_new[tid]) >= 1.0) atomicOr(flags, 2);
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
  for (int ch = 0; ch < 2; ++ch) {
    if (!(channel_mask & (1 << ch))) continue;
    const long systems = (long)dm.nb * dm.N;
    const int grid = (int)(systems < c->bse_grid ? systems : c->bse_grid);
    if (bse_lu_in_smem(n)) {
      bse_f64_kernel<true><<<grid, kBseThreads, smem, c->stream>>>(dm, ch, 1, nc, c->gam, gg_ptr(c), c->chi,
                                                                   c->kc, nullptr, flag_ptr(c), K, lam);
    } else {
      bse_f64_kernel<false><<<grid, kBseThreads, smem, c->stream>>>(dm, ch, 1, nc, c->gam, gg_ptr(c), c->chi,
                                                                    c->kc, lu_ws_ptr(c), flag_ptr(c), K, lam);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// the ladder term of the susceptibilities for both channels (FP64); the
// persistent grid and LU scratch of the FP64 ladder kernel
cudaError_t launch_chi_ladder(df_ctx* c, const double2* Lb, const double2* chi0, double2* out) {
  const Dims& dm = c->dm;
  const int n = dm.n_w;
  const bool in_smem = bse_lu_in_smem(n);
  const size_t smem = sizeof(double2) * (size_t)bse_layout(n, 2, in_smem).total;
  const void* fn = in_smem ? (const void*)chi_ladder_kernel<true> : (const void*)chi_ladder_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long systems = 2L * dm.nb * dm.N;
  const int grid = (int)(systems < c->bse_grid ? systems : c->bse_grid);
  if (in_smem)
    chi_ladder_kernel<true><<<grid, kBseThreads, smem, c->stream>>>(dm, c->gam, c->chi, Lb, chi0, out, nullptr,
                                                                    flag_ptr(c));
  else
    chi_ladder_kernel<false><<<grid, kBseThreads, smem, c->stream>>>(dm, c->gam, c->chi, Lb, chi0, out,
                                                                     lu_ws_ptr(c), flag_ptr(c));
  return cudaGetLastError();
}

cudaError_t launch_lambda(df_ctx* c, int channel_mask) {
  const Dims& dm = c->dm;
  if (c->opts.eig_mode == 0) return cudaSuccess;
  const int a0 = (c->opts.eig_mode == 1) ? dm.m_max : 0;
  const int na = (c->opts.eig_mode == 1) ? 1 : dm.nb;
  const int qtiles = (dm.N + kEigQ - 1) / kEigQ;
  // gamma's (hi, lo) FP32 pairs in shared memory when they fit (n_w <= 96), the
  // lo parts formed from FP64 gamma on the fly above that
  const size_t base = sizeof(double2) * 3 * dm.n_w * kEigQ + sizeof(float2) * ((size_t)dm.n_w * dm.n_w + 3 * dm.n_w * kEigQ);
  const int lo_in_smem = base + sizeof(float2) * (size_t)dm.n_w * dm.n_w <= (size_t)200 * 1024 ? 1 : 0;
  const size_t smem = base + (lo_in_smem ? sizeof(float2) * (size_t)dm.n_w * dm.n_w : 0);
  cudaError_t e = cudaFuncSetAttribute((const void*)lambda_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // both channels in one launch when both are asked for
  const int ch0 = (channel_mask & 1) ? 0 : 1;
  const int nch = (channel_mask & 1) && (channel_mask & 2) ? 2 : 1;
  if (!(channel_mask & 3)) return cudaSuccess;
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
                                                            nullptr);
  return cudaGetLastError();
}

}  // namespace df
