// Batched ladder dual-fermion loop over many uneven parameter points.
//
// Every stage of one loop pass is ONE launch over all points: the FFT
// stages map blocks to (point, plane) through prefix tables; the FP64
// ladder solves run in a persistent kernel whose CTAs pull chunks of
// systems from an atomic counter over an index space sorted by cost
// (largest ladder order first); the mixed-precision ladders run one
// persistent launch per padded-order class.  The pass is captured once in a
// CUDA graph and replayed; a final kernel computes each point's residual
// and clears its `active` flag when it has converged, after which every
// stage skips that point.  A self-timed autotuner picks the FP64 chunk
// width and the scheduler's chunk size.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "df_bse_dev.cuh"
#include "df_fft_dev.cuh"
#include "df_mixed_dev.cuh"
#include "df_mixed_large_dev.cuh"

namespace df {

// Per-ladder error control of the batch's mixed ladders: a ladder whose
// predicted error rho^2 exceeds kBatchLadderTol goes to one batch-wide list,
// entries (point << 24) | ((c N_W + a) N + q), solved again by the FP64 LU
// (batch_bse_f64_list_kernel) in the same pass.
constexpr float kBatchLadderTol = 1e-9f;
__device__ __forceinline__ MixedCheck batch_check(int* redo, int point) {
  return MixedCheck{redo, nullptr, kBatchLadderTol, point << 24};
}


struct PointDev {
  Dims dm;
  // the ladder stage's view: dm, chi and kc, or with the point-group reduction
  // (sym) the compact grid of one momentum per orbit (ldm.N = n_orb) and its
  // arrays; with the frequency reflection (refl) only the planes W >= 0
  // (ldm.a0 = m_max, ldm.na = m_max + 1)
  Dims ldm;
  double2 *lchi, *lkc;
  int sym, refl, n_orb;
  int *qmap, *qrep;
  int nc;        // FP64 ladder right-hand-side chunk
  int mixed;     // ladders of this point run in DF_FP32_IR
  int active;    // 1 until converged
  double mix, tol, resid;
  double2 *g, *delta, *gam, *gg, *g0, *gk, *gr, *chi, *kc, *prod, *sigma;
  float2 *gam_hi, *gam_lo, *gg_hi, *gg_lo;   // mixed: FP32 (hi, lo) of gam and gg (orders > 64: of gam^T)
  unsigned char* gdig;                         // mixed, n_pad 32 / 64: gamma's digits
  double* red;   // [2 n_w + 4]
  int* flags;    // [4]
};

// the FP64 right-hand-side chunk of an order (as default_nc on the host)
__device__ __forceinline__ int default_nc_dev(int n) { return n <= 32 ? n : (n <= 64 ? 32 : 16); }

__device__ __forceinline__ int find_segment(const long* start, int nseg, long x) {
  // largest k with start[k] <= x (start[0] = 0, start[nseg] = total)
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---- FFT stages ------------------------------------------------------------

__global__ void __launch_bounds__(kFftThreads)
batch_bubble_kernel(const PointDev* __restrict__ pts, const long* __restrict__ start, int npts) {
  extern __shared__ double2 sm[];
  const int p = find_segment(start, npts, blockIdx.x);
  const PointDev& P = pts[p];
  if (!P.active) return;
  const int local = (int)(blockIdx.x - start[p]);
  const int a = local / P.dm.n_w, i = local - a * P.dm.n_w;
  if (P.refl && a < P.dm.m_max) return;             // W < 0: not needed under the reflection
  bubble_plane(P.dm, a, i, P.gr, P.chi, sm, sm + P.dm.nk / 2);
}

__global__ void __launch_bounds__(kFftThreads)
batch_sigma_prod_kernel(const PointDev* __restrict__ pts, const long* __restrict__ start, int npts) {
  extern __shared__ double2 sm[];
  const int p = find_segment(start, npts, blockIdx.x);
  const PointDev& P = pts[p];
  if (!P.active) return;
  const int local = (int)(blockIdx.x - start[p]);
  const int a = local / P.dm.n_w, i = local - a * P.dm.n_w;
  if (P.refl && a < P.dm.m_max) return;             // W < 0: summed by the reflection
  sigma_prod_plane(P.dm, a, i, P.kc, P.gr, P.prod, sm, sm + P.dm.nk / 2);
}

__global__ void __launch_bounds__(kFftThreads)
batch_sigma_dyson_kernel(const PointDev* __restrict__ pts, const long* __restrict__ start, int npts) {
  extern __shared__ double2 sm[];
  __shared__ double red_sm[32];
  const int p = find_segment(start, npts, blockIdx.x);
  const PointDev& P = pts[p];
  if (!P.active) return;
  const int i = (int)(blockIdx.x - start[p]);
  sigma_dyson_plane(P.dm, i, P.mix, P.prod, P.g0, P.sigma, P.gk, P.gr, P.red, sm, sm + P.dm.nk / 2,
                    sm + P.dm.nk / 2 + P.dm.N, red_sm, P.refl);
}

// one block per point: residual, convergence flag, result copy
__global__ void __launch_bounds__(kFftThreads)
batch_residual_kernel(PointDev* __restrict__ pts, double* __restrict__ out) {
  __shared__ double red_sm[32];
  PointDev& P = pts[blockIdx.x];
  if (P.active) {
    residual_reduce_block(P.dm.n_w, P.red, red_sm);
    if (threadIdx.x == 0) {
      const double num = P.red[2 * P.dm.n_w], den = P.red[2 * P.dm.n_w + 1];
      const double r = den > 0.0 ? num / den : 0.0;
      P.resid = r;
      if (P.tol > 0.0 && r <= P.tol) P.active = 0;
    }
  }
  if (threadIdx.x == 0) {
    out[3 * blockIdx.x] = P.resid;
    out[3 * blockIdx.x + 1] = (double)P.active;
    out[3 * blockIdx.x + 2] = (double)P.flags[0];
  }
}

// per-point set-up: Eq. gd0, gamma o gamma^T, gamma (hi, lo), Dyson + FFT
__global__ void batch_setup_elem_kernel(const PointDev* __restrict__ pts, int p) {
  const PointDev& P = pts[p];
  const int total = P.dm.ne * P.dm.N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x)
    init_g0_elem(P.dm, idx, P.g, P.delta, P.g0, P.gk);
  const int n = P.dm.n_w;
  const size_t nv = (size_t)2 * P.dm.nb * n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < nv; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t mat = idx / ((size_t)n * n);
    const int rem = (int)(idx - mat * n * n);
    const int i = rem / n, j = rem - i * n;
    const double2* G = P.gam + mat * n * n;
    const double2 w = cmul(G[i * n + j], G[j * n + i]);
    P.gg[idx] = w;
    if (P.gam_hi) {
      const double2 v = P.gam[idx];
      float hx = (float)v.x, hy = (float)v.y;
      P.gam_hi[idx] = make_float2(hx, hy);
      P.gam_lo[idx] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
      // orders > 64 keep gamma^T's words in these slots (the large-order kernel's residual)
      const double2 t = mixed_pad(n) > 64 ? G[j * n + i] : w;
      hx = (float)t.x; hy = (float)t.y;
      P.gg_hi[idx] = make_float2(hx, hy);
      P.gg_lo[idx] = make_float2((float)(t.x - (double)hx), (float)(t.y - (double)hy));
    }
  }
  if (P.gdig)
    gamma_digits_rows(n, mixed_pad(n), 2 * P.dm.nb, P.gam, P.gdig, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                      (gridDim.x * blockDim.x) >> 5, threadIdx.x & 31);
}

__global__ void __launch_bounds__(kFftThreads)
batch_setup_dyson_kernel(const PointDev* __restrict__ pts, int p) {
  extern __shared__ double2 sm[];
  const PointDev& P = pts[p];
  dyson_ifft_plane(P.dm, blockIdx.x, P.g0, P.sigma, P.gk, P.gr, sm, sm + P.dm.nk / 2);
}

// ---- ladder stages ---------------------------------------------------------

__global__ void __launch_bounds__(kBseThreads)
batch_bse_f64_kernel(const PointDev* __restrict__ pts, const int* __restrict__ order, const long* __restrict__ start,
                     int nseg, int chunk, unsigned long long* __restrict__ counter, double2* __restrict__ ws,
                     size_t ws_stride) {
  extern __shared__ double2 sm[];
  __shared__ BseF64Shared sh;
  __shared__ unsigned long long item_s;
  const long total = start[nseg];
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, (unsigned long long)chunk);
    __syncthreads();
    const long item = (long)item_s;
    __syncthreads();
    if (item >= total) break;
    const long end = min(item + (long)chunk, total);
    for (long s = item; s < end; ++s) {
      const int k = find_segment(start, nseg, s);
      const PointDev& P = pts[order[k]];
      if (!P.active) continue;
      const Dims& dm = P.ldm;
      const long local = s - start[k];
      const long per_ch = (long)dm.na * dm.N;      // the view's planes a0 .. a0 + na - 1
      const int c = (int)(local / per_ch);
      const int rem = (int)(local - (long)c * per_ch);
      const int a = dm.a0 + rem / dm.N, q = rem - (a - dm.a0) * dm.N;
      const bool lu_smem = dm.n_w <= kLuSmemOrder;
      const BseSmem L = bse_layout(dm.n_w, P.nc, lu_smem);
      double2* LU = lu_smem ? sm + L.lu : ws + blockIdx.x * ws_stride;
      bse_f64_system(dm, c, a, q, P.nc, P.gam, P.gg, P.lchi, P.lkc, LU, sm + L.y, sm + L.xs, sm + L.invu, sh,
                     P.flags);
    }
  }
}

// the FP64 LU over the mixed ladders handed back this pass (redo[0] entries)
__global__ void __launch_bounds__(kBseThreads)
batch_bse_f64_list_kernel(const PointDev* __restrict__ pts, const int* __restrict__ redo, double2* __restrict__ ws,
                          size_t ws_stride) {
  extern __shared__ double2 sm[];
  __shared__ BseF64Shared sh;
  const int count = redo[0];
  for (int s = blockIdx.x; s < count; s += gridDim.x) {
    const int code = redo[1 + s];
    const PointDev& P = pts[code >> 24];
    const Dims& dm = P.ldm;
    const int sys = code & 0xFFFFFF;
    const int c = sys / (dm.nb * dm.N), rem = sys - c * dm.nb * dm.N;
    const int a = rem / dm.N, q = rem - a * dm.N;
    const int nc = default_nc_dev(dm.n_w);
    const bool lu_smem = dm.n_w <= kLuSmemOrder;
    const BseSmem L = bse_layout(dm.n_w, nc, lu_smem);
    double2* LU = lu_smem ? sm + L.lu : ws + blockIdx.x * ws_stride;
    bse_f64_system(dm, c, a, q, nc, P.gam, P.gg, P.lchi, P.lkc, LU, sm + L.y, sm + L.xs, sm + L.invu, sh, P.flags);
  }
}

// the point-group reduction (df_point.symmetry): per reduced point (blockIdx.y),
// chi~'s orbit representatives into the compact array before the ladders, the
// compact brackets back to every momentum after them
__global__ void batch_wedge_gather_kernel(const PointDev* __restrict__ pts) {
  const PointDev& P = pts[blockIdx.y];
  if (!P.sym || !P.active) return;
  const Dims& dm = P.dm;
  const long total = (long)P.ldm.na * dm.n_w * P.n_orb;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int o = (int)(idx % P.n_orb);
    const long row = (long)P.ldm.a0 * dm.n_w + idx / P.n_orb;   // a * n_w + i
    P.lchi[row * P.n_orb + o] = P.chi[row * dm.N + P.qrep[o]];
  }
}

__global__ void batch_wedge_scatter_kernel(const PointDev* __restrict__ pts) {
  const PointDev& P = pts[blockIdx.y];
  if (!P.sym || !P.active) return;
  const Dims& dm = P.dm;
  const long total = 2L * dm.nb * dm.n_w * dm.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx % dm.N);
    const long row = idx / dm.N;                   // (c nb + a) n_w + i
    const int i = (int)(row % dm.n_w);
    const long ca = row / dm.n_w;
    const int a = (int)(ca % dm.nb);
    if (P.refl && a < dm.m_max) {                  // W < 0: the reflection of 2 m_max - a
      const long src = (ca + 2 * (dm.m_max - a)) * dm.n_w + (dm.n_w - 1 - i);
      const double2 v = P.lkc[src * P.n_orb + P.qmap[q]];
      P.kc[idx] = make_double2(v.x, -v.y);
    } else {
      P.kc[idx] = P.lkc[row * P.n_orb + P.qmap[q]];
    }
  }
}

template <int NP>
__global__ void __launch_bounds__(mixed_block_threads(NP), use_umma_residual(NP) ? 1 : 0)
batch_bse_mixed_kernel(const PointDev* __restrict__ pts, const int* __restrict__ order, const long* __restrict__ start,
                       int nseg, int chunk, unsigned long long* __restrict__ counter, int* __restrict__ redo) {
  extern __shared__ __align__(1024) float2 smf[];
  __shared__ int piv_s[128];
  __shared__ unsigned long long item_s;
  __shared__ uint64_t mbar_s[2];
  __shared__ unsigned tslot_s;
  const MixedPtrs sp = mixed_ptrs(smf, NP, piv_s);
  Tc05 tc{};
  if constexpr (use_umma_residual(NP)) {
    // the swizzled operand tiles need a 1024-aligned work area
    if (smem_u32(sp.work) & 1023u) {
      if (threadIdx.x == 0) atomicOr(pts[0].flags, kFlagTcLayout);
      return;
    }
    tc05_setup(tc, mbar_s, &tslot_s);
  }
  const long total = start[nseg];
  long cur = -1;                       // (point, channel, W) whose gamma digits are in shared memory
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, (unsigned long long)chunk);
    __syncthreads();
    const long item = (long)item_s;
    __syncthreads();
    if (item >= total) break;
    const long end = min(item + (long)chunk, total);
    for (long s = item; s < end; ++s) {
      const int k = find_segment(start, nseg, s);
      const PointDev& P = pts[order[k]];
      if (!P.active) continue;
      const Dims& dm = P.ldm;
      const long local = s - start[k];
      const long per_ch = (long)dm.na * dm.N;      // the view's planes a0 .. a0 + na - 1
      const int c = (int)(local / per_ch);
      const int rem = (int)(local - (long)c * per_ch);
      const int a = dm.a0 + rem / dm.N, q = rem - (a - dm.a0) * dm.N;
      const long key = (long)k * 256 + c * dm.nb + a;
      if (use_umma_residual(NP) && (threadIdx.x >> 5) == mixed_compute_threads(NP) / 32)
        mixed_producer(sp, &tc);                      // warp 8: the tensor-core MMAs
      else
        bse_mixed_system<NP>(dm, c, a, q, P.gam, P.gam_hi, P.gam_lo, P.gg_hi, P.gg_lo, P.lchi, P.lkc, P.flags, sp,
                             P.gdig ? P.gdig + (size_t)(c * dm.nb + a) * gdig_bytes(NP) : nullptr, key != cur, &tc,
                             batch_check(redo, order[k]));
      cur = key;
    }
  }
  if constexpr (use_umma_residual(NP)) tc05_teardown(tc, mixed_compute_threads(NP));
}

// mixed ladders of order 64 < n <= 128 (the shared-memory Gauss-Jordan body),
// 256 threads, the same chunked queue over the class's cost-sorted points
__global__ void __launch_bounds__(256, 1)
batch_bse_gj_kernel(const PointDev* __restrict__ pts, const int* __restrict__ order, const long* __restrict__ start,
                    int nseg, int chunk, unsigned long long* __restrict__ counter, int* __restrict__ redo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ GjShared sh;
  __shared__ unsigned long long item_s;
  const long total = start[nseg];
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, (unsigned long long)chunk);
    __syncthreads();
    const long item = (long)item_s;
    __syncthreads();
    if (item >= total) break;
    const long end = min(item + (long)chunk, total);
    for (long s = item; s < end; ++s) {
      const int k = find_segment(start, nseg, s);
      const PointDev& P = pts[order[k]];
      if (!P.active) continue;
      const Dims& dm = P.ldm;
      const long local = s - start[k];
      const long per_ch = (long)dm.na * dm.N;      // the view's planes a0 .. a0 + na - 1
      const int c = (int)(local / per_ch);
      const int rem = (int)(local - (long)c * per_ch);
      const int a = dm.a0 + rem / dm.N, q = rem - (a - dm.a0) * dm.N;
      gj_ir_system(dm, c, a, q, P.gam_hi, P.gam_lo, P.gg_hi, P.gg_lo, P.gg, P.lchi, P.lkc, P.flags, smraw, sh,
                   batch_check(redo, order[k]));
    }
  }
}

}  // namespace df

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

using namespace df;

namespace {

int mixed_np_of(int n) { return mixed_pad(n); }

using MixedKernel = void (*)(const PointDev*, const int*, const long*, int, int, unsigned long long*, int*);

// the ladder kernel instance of a padded order (8, 16, 32 or 64)
MixedKernel mixed_kernel_of(int np) {
  switch (np) {
    case 8: return batch_bse_mixed_kernel<8>;
    case 16: return batch_bse_mixed_kernel<16>;
    case 32: return batch_bse_mixed_kernel<32>;
    default: return batch_bse_mixed_kernel<64>;
  }
}

struct LadderGroup {          // one persistent ladder launch
  bool mixed = false;
  int np = 0;                 // mixed: padded order (block = (np/4)^2 threads)
  std::vector<int> order;     // points, cost-sorted
  long* d_start = nullptr;    // [nseg + 1]
  int* d_order = nullptr;
  int nseg = 0;
  long total = 0;
  size_t smem = 0;
  int threads = 0;
  int grid = 0;
  int counter_slot = 0;
};

}  // namespace

struct df_batch {
  int npts = 0;
  int precision = DF_FP64;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;
  std::string err;
  std::vector<PointDev> host_pts;
  PointDev* d_pts = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  // FFT-stage tables
  long *d_plane_start = nullptr, *d_box_start = nullptr;
  long total_planes = 0, total_box = 0;
  size_t fft_smem1 = 0, fft_smem2 = 0;
  std::vector<LadderGroup> groups;
  unsigned long long* d_counters = nullptr;   // one per ladder group
  double2* ws = nullptr;                       // global LU scratch (FP64, n > 96)
  size_t ws_stride = 0;
  int* d_redo = nullptr;                       // mixed ladders handed back to the FP64 LU: count, list
  int redo_grid = 0;
  size_t redo_smem = 0;
  double* d_out = nullptr;                     // [3 npts] residual, active, flags
  bool any_sym = false;                        // some point uses the point-group reduction
  double* h_out = nullptr;
  int chunk = 1;                               // scheduler chunk (autotuned)
  int nc_override = 0;                         // FP64 RHS chunk (autotuned; 0 = per-point default)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int passes = 0;
  bool own_stream = false;
};

namespace {

df_status bfail(df_batch* b, df_status s, const char* what, cudaError_t e = cudaSuccess) {
  if (b) {
    char buf[512];
    if (e != cudaSuccess)
      snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    else
      snprintf(buf, sizeof buf, "%s", what);
    b->err = buf;
  }
  return s;
}

#define B_CUDA(b, call, what)                                                               \
  do {                                                                                      \
    cudaError_t e__ = (call);                                                               \
    if (e__ != cudaSuccess)                                                                 \
      return bfail((b), e__ == cudaErrorMemoryAllocation ? DF_ERR_OOM : DF_ERR_CUDA, (what), e__); \
  } while (0)

int default_nc(int n) { return n <= 32 ? n : (n <= 64 ? 32 : 16); }

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kLuScratchPerSm = 4;   // global LU slices per SM (FP64 ladders of order > kLuSmemOrder)
constexpr int kWedgeBlocks = 32;     // blocks per point of the orbit gather and scatter

// the pass: all stages, captured into b->graph
df_status record_pass(df_batch* b) {
  cudaStream_t s = b->stream;
  const int ng = (int)b->groups.size();
  B_CUDA(b, cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned long long) * (ng ? ng : 1), s), "counter reset");
  if (b->d_redo) B_CUDA(b, cudaMemsetAsync(b->d_redo, 0, sizeof(int), s), "hand-back count reset");
  batch_bubble_kernel<<<(unsigned)b->total_planes, kFftThreads, b->fft_smem1, s>>>(b->d_pts, b->d_plane_start, b->npts);
  B_CUDA(b, cudaGetLastError(), "batch bubble");
  if (b->any_sym) {
    batch_wedge_gather_kernel<<<dim3(kWedgeBlocks, b->npts), 256, 0, s>>>(b->d_pts);
    B_CUDA(b, cudaGetLastError(), "batch orbit gather");
  }
  for (auto& g : b->groups) {
    if (g.total == 0) continue;
    if (!g.mixed) {
      batch_bse_f64_kernel<<<g.grid, kBseThreads, g.smem, s>>>(b->d_pts, g.d_order, g.d_start, g.nseg, b->chunk,
                                                               b->d_counters + g.counter_slot, b->ws, b->ws_stride);
    } else if (g.np > 64) {
      batch_bse_gj_kernel<<<g.grid, g.threads, g.smem, s>>>(b->d_pts, g.d_order, g.d_start, g.nseg, b->chunk,
                                                            b->d_counters + g.counter_slot, b->d_redo);
    } else {
      mixed_kernel_of(g.np)<<<g.grid, g.threads, g.smem, s>>>(b->d_pts, g.d_order, g.d_start, g.nseg, b->chunk,
                                                              b->d_counters + g.counter_slot, b->d_redo);
    }
    B_CUDA(b, cudaGetLastError(), "batch ladder");
  }
  if (b->d_redo) {
    batch_bse_f64_list_kernel<<<b->redo_grid, kBseThreads, b->redo_smem, s>>>(b->d_pts, b->d_redo, b->ws,
                                                                              b->ws_stride);
    B_CUDA(b, cudaGetLastError(), "batch hand-back ladders");
  }
  if (b->any_sym) {
    batch_wedge_scatter_kernel<<<dim3(kWedgeBlocks, b->npts), 256, 0, s>>>(b->d_pts);
    B_CUDA(b, cudaGetLastError(), "batch orbit scatter");
  }
  batch_sigma_prod_kernel<<<(unsigned)b->total_planes, kFftThreads, b->fft_smem1, s>>>(b->d_pts, b->d_plane_start,
                                                                                      b->npts);
  B_CUDA(b, cudaGetLastError(), "batch Sigma~ stage 1");
  batch_sigma_dyson_kernel<<<(unsigned)b->total_box, kFftThreads, b->fft_smem2, s>>>(b->d_pts, b->d_box_start,
                                                                                    b->npts);
  B_CUDA(b, cudaGetLastError(), "batch Sigma~ stage 2");
  batch_residual_kernel<<<b->npts, kFftThreads, 0, s>>>(b->d_pts, b->d_out);
  B_CUDA(b, cudaGetLastError(), "batch residual");
  B_CUDA(b, cudaMemcpyAsync(b->h_out, b->d_out, sizeof(double) * 3 * b->npts, cudaMemcpyDeviceToHost, s),
         "batch residual copy");
  return DF_OK;
}

df_status build_graph(df_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  B_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  df_status st = record_pass(b);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (st != DF_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  B_CUDA(b, e, "end capture");
  b->graph = g;
  B_CUDA(b, cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
  return DF_OK;
}

df_status configure_groups(df_batch* b) {
  // kernel attributes and persistent grids for the current nc / chunk; the
  // mixed classes share one kernel, whose shared-memory limit is set once to
  // the largest class
  for (auto& g : b->groups) {
    if (g.mixed && g.np > 64) {
      g.threads = 256;
      g.smem = (size_t)gj_layout(kGjMaxN).total;       // the largest order's layout serves every order
      B_CUDA(b, cudaFuncSetAttribute((const void*)batch_bse_gj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)g.smem),
             "large-order mixed smem attribute");
      int per = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_bse_gj_kernel, g.threads, g.smem);
      g.grid = b->sms * std::max(1, per);
    } else if (g.mixed) {
      g.threads = mixed_block_threads(g.np);
      g.smem = sizeof(float2) * (size_t)mixed_layout(g.np).total;
      B_CUDA(b, cudaFuncSetAttribute((const void*)mixed_kernel_of(g.np), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)g.smem),
             "mixed smem attribute");
      int per = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mixed_kernel_of(g.np), g.threads, g.smem);
      g.grid = b->sms * std::max(1, per);
    } else {
      size_t sm = 0;
      for (int p : g.order) {
        PointDev& P = b->host_pts[p];
        P.nc = b->nc_override ? std::min(b->nc_override, P.dm.n_w) : default_nc(P.dm.n_w);
        sm = std::max(sm, sizeof(double2) * (size_t)bse_layout(P.dm.n_w, P.nc, P.dm.n_w <= kLuSmemOrder).total);
      }
      g.smem = sm;
      g.threads = kBseThreads;
      B_CUDA(b, cudaFuncSetAttribute((const void*)batch_bse_f64_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem),
             "FP64 smem attribute");
      int per = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_bse_f64_kernel, kBseThreads, g.smem);
      g.grid = b->sms * std::max(1, per);
      if (b->ws) g.grid = std::min(g.grid, b->sms * kLuScratchPerSm);   // one LU slice per CTA
    }
  }
  B_CUDA(b, cudaMemcpyAsync(b->d_pts, b->host_pts.data(), sizeof(PointDev) * b->npts, cudaMemcpyHostToDevice,
                            b->stream), "point table");
  return DF_OK;
}

}  // namespace

extern "C" {

// df_point.symmetry = 2: g(-w) = g(w)*, Delta(-w) = Delta(w)* and gamma(-W; w, w')
// = gamma(W; -w, -w')* for both channels, within 1e-12 of each array's largest entry
static bool reflection_holds(const df_point& q) {
  const int ne = q.n_w + 2 * q.m_max, nb = 2 * q.m_max + 1, n = q.n_w;
  auto dev = [](const double* x, size_t i, size_t j) {   // |x_i - conj(x_j)|, x interleaved (re, im)
    return fabs(x[2 * i] - x[2 * j]) + fabs(x[2 * i + 1] + x[2 * j + 1]);
  };
  auto mag = [](const double* x, size_t i) { return fabs(x[2 * i]) + fabs(x[2 * i + 1]); };
  const double* vec[2] = {q.g, q.delta};
  for (const double* x : vec) {
    double top = 0.0, d = 0.0;
    for (int e = 0; e < ne; ++e) {
      top = std::max(top, mag(x, e));
      d = std::max(d, dev(x, e, ne - 1 - e));
    }
    if (!(d <= 1e-12 * top)) return false;
  }
  const double* mats[2] = {q.gamma_d, q.gamma_m};
  for (const double* x : mats) {
    double top = 0.0, d = 0.0;
    for (int a = 0; a < nb; ++a)
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          const size_t u = ((size_t)a * n + i) * n + j, v = ((size_t)(nb - 1 - a) * n + (n - 1 - i)) * n + (n - 1 - j);
          top = std::max(top, mag(x, u));
          d = std::max(d, dev(x, u, v));
        }
    if (!(d <= 1e-12 * top)) return false;
  }
  return true;
}

df_status df_batch_init(df_batch** out, int npts, const df_point* pts, int precision, double mix, double tol,
                        void* stream) {
  if (!out || !pts || npts < 1 || npts > 4096) return DF_ERR_ARG;
  if (precision == DF_FP32_IR && npts > 127) return DF_ERR_ARG;   // the hand-back list's point field
  if (precision != DF_FP64 && precision != DF_FP32_IR) return DF_ERR_ARG;
  if (!(mix > 0.0 && mix <= 1.0)) return DF_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < npts; ++i) {
    const df_point& q = pts[i];
    int N = 1;
    if (q.dim < 1 || q.dim > 4 || q.nk < 2 || q.nk > 64 || (q.nk & (q.nk - 1))) return DF_ERR_ARG;
    for (int d = 0; d < q.dim; ++d) N *= q.nk;
    if (N > 4096 || (q.tp != 0.0 && q.dim != 2)) return DF_ERR_ARG;
    if (q.n_w < 2 || q.n_w > 128 || (q.n_w & 1) || q.m_max < 0 || q.m_max > 31 || !(q.beta > 0.0)) return DF_ERR_ARG;
    if (!q.g || !q.delta || !q.gamma_d || !q.gamma_m) return DF_ERR_ARG;
    if (q.symmetry < 0 || q.symmetry > 2) return DF_ERR_ARG;
    if (q.symmetry == 2 && !reflection_holds(q)) return DF_ERR_ARG;
  }
  df_batch* b = new (std::nothrow) df_batch();
  if (!b) return DF_ERR_OOM;
  b->npts = npts;
  b->precision = precision;
  b->stream = (cudaStream_t)stream;
  int ndev = 0;
  if (!b->stream) {
    // graph capture needs a stream other than the legacy default one
    cudaError_t es = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (es != cudaSuccess) {
      delete b;
      fprintf(stderr, "libdf: df_batch_init: cudaStreamCreate: %s\n", cudaGetErrorString(es));
      return DF_ERR_CUDA;
    }
    b->own_stream = true;
  }
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    delete b;
    fprintf(stderr, "libdf: df_batch_init: no CUDA device\n");
    return DF_ERR_CUDA;
  }
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);

  // ---- sizes and the arena ----
  b->host_pts.resize(npts);
  std::vector<size_t> off(npts);
  std::vector<std::vector<int>> qmaps(npts), qreps(npts);
  size_t total = 0;
  int nmax = 0;
  for (int i = 0; i < npts; ++i) {
    const df_point& q = pts[i];
    PointDev& P = b->host_pts[i];
    memset(&P, 0, sizeof P);
    Dims& dm = P.dm;
    dm.D = q.dim;
    dm.nk = q.nk;
    dm.p = 0;
    while ((1 << dm.p) < q.nk) ++dm.p;
    dm.N = 1;
    for (int d = 0; d < q.dim; ++d) dm.N *= q.nk;
    dm.n_w = q.n_w;
    dm.m_max = q.m_max;
    dm.nb = 2 * q.m_max + 1;
    dm.a0 = 0;
    dm.na = dm.nb;
    dm.ne = q.n_w + 2 * q.m_max;
    dm.beta = q.beta;
    dm.T = 1.0 / q.beta;
    dm.mu = q.mu;
    dm.t = q.t;
    dm.tp = q.tp;
    P.mixed = (precision == DF_FP32_IR && mixed_np_of(q.n_w) <= kGjMaxN) ? 1 : 0;
    P.sym = q.symmetry ? 1 : 0;
    P.refl = q.symmetry == 2 ? 1 : 0;
    P.n_orb = P.sym ? build_wedge(q.dim, q.nk, qmaps[i], qreps[i]) : dm.N;
    P.ldm = dm;
    P.ldm.N = P.n_orb;
    if (P.refl) {
      P.ldm.a0 = dm.m_max;
      P.ldm.na = dm.m_max + 1;
    }
    b->any_sym = b->any_sym || P.sym;
    P.active = 1;
    P.mix = mix;
    P.tol = tol;
    P.resid = -1.0;
    nmax = std::max(nmax, q.n_w);
    const size_t nv = (size_t)2 * dm.nb * dm.n_w * dm.n_w;
    const size_t plane = (size_t)dm.ne * dm.N;
    const size_t nchi = (size_t)dm.nb * dm.n_w * dm.N;
    off[i] = total;
    total += align_up(sizeof(double2) * dm.ne) * 2;               // g, delta
    total += align_up(sizeof(double2) * nv) * 2;                  // gam, gg
    total += align_up(sizeof(double2) * plane) * 3;               // g0, gk, gr
    total += align_up(sizeof(double2) * nchi) * 4;                // chi, kc (2), prod
    total += align_up(sizeof(double2) * (size_t)dm.n_w * dm.N);  // sigma
    total += align_up(sizeof(double) * (2 * dm.n_w + 4));
    total += align_up(sizeof(int) * 4);
    if (P.mixed) total += align_up(sizeof(float2) * nv) * 4;      // gam hi, lo; gg hi, lo
    if (P.mixed && use_tc_residual(mixed_pad(dm.n_w)))
      total += align_up((size_t)2 * dm.nb * gdig_bytes(mixed_pad(dm.n_w)));   // gamma's digits
    if (P.sym) {
      const size_t nw = (size_t)dm.nb * dm.n_w * P.n_orb;
      total += align_up(sizeof(double2) * nw) * 3;                // compact chi, kc (2)
      total += align_up(sizeof(int) * dm.N) + align_up(sizeof(int) * P.n_orb);   // orbit map, representatives
    }
  }
  b->arena_bytes = total;
  df_status st = DF_OK;
  cudaError_t e;
#define BALLOC(ptr, bytes, what)                                                    \
  do {                                                                              \
    e = cudaMalloc((void**)&(ptr), (bytes));                                        \
    if (e != cudaSuccess) { st = bfail(b, DF_ERR_OOM, what, e); goto bad; }         \
  } while (0)
  BALLOC(b->arena, total, "batch arena");
  for (int i = 0; i < npts; ++i) {
    PointDev& P = b->host_pts[i];
    const Dims& dm = P.dm;
    const size_t nv = (size_t)2 * dm.nb * dm.n_w * dm.n_w;
    const size_t plane = (size_t)dm.ne * dm.N;
    const size_t nchi = (size_t)dm.nb * dm.n_w * dm.N;
    char* cur = b->arena + off[i];
    auto take = [&](size_t bytes) { char* r = cur; cur += align_up(bytes); return r; };
    P.g = (double2*)take(sizeof(double2) * dm.ne);
    P.delta = (double2*)take(sizeof(double2) * dm.ne);
    P.gam = (double2*)take(sizeof(double2) * nv);
    P.gg = (double2*)take(sizeof(double2) * nv);
    P.g0 = (double2*)take(sizeof(double2) * plane);
    P.gk = (double2*)take(sizeof(double2) * plane);
    P.gr = (double2*)take(sizeof(double2) * plane);
    P.chi = (double2*)take(sizeof(double2) * nchi);
    P.kc = (double2*)take(sizeof(double2) * 2 * nchi);
    P.prod = (double2*)take(sizeof(double2) * nchi);
    P.sigma = (double2*)take(sizeof(double2) * (size_t)dm.n_w * dm.N);
    P.red = (double*)take(sizeof(double) * (2 * dm.n_w + 4));
    P.flags = (int*)take(sizeof(int) * 4);
    if (P.mixed) {
      P.gam_hi = (float2*)take(sizeof(float2) * nv);
      P.gam_lo = (float2*)take(sizeof(float2) * nv);
      P.gg_hi = (float2*)take(sizeof(float2) * nv);
      P.gg_lo = (float2*)take(sizeof(float2) * nv);
      if (use_tc_residual(mixed_pad(dm.n_w)))
        P.gdig = (unsigned char*)take((size_t)2 * dm.nb * gdig_bytes(mixed_pad(dm.n_w)));
    }
    if (P.sym) {
      const size_t nw = (size_t)dm.nb * dm.n_w * P.n_orb;
      P.lchi = (double2*)take(sizeof(double2) * nw);
      P.lkc = (double2*)take(sizeof(double2) * 2 * nw);
      P.qmap = (int*)take(sizeof(int) * dm.N);
      P.qrep = (int*)take(sizeof(int) * P.n_orb);
    } else {
      P.lchi = P.chi;
      P.lkc = P.kc;
    }
    const char* limit = b->arena + (i + 1 < npts ? off[i + 1] : total);
    if (cur > limit) {
      st = bfail(b, DF_ERR_ARG, "internal: point buffers exceed their arena slice");
      goto bad;
    }
  }
  BALLOC(b->d_pts, sizeof(PointDev) * npts, "point table");
  BALLOC(b->d_out, sizeof(double) * 3 * npts, "residual array");
  e = cudaMallocHost((void**)&b->h_out, sizeof(double) * 3 * npts);
  if (e != cudaSuccess) { st = bfail(b, DF_ERR_OOM, "pinned residuals", e); goto bad; }
  for (int i = 0; i < npts; ++i) {
    b->h_out[3 * i] = -1.0;
    b->h_out[3 * i + 1] = 1.0;
    b->h_out[3 * i + 2] = 0.0;
  }

  // ---- inputs ----
  for (int i = 0; i < npts; ++i) {
    PointDev& P = b->host_pts[i];
    const Dims& dm = P.dm;
    const size_t nvc = (size_t)dm.nb * dm.n_w * dm.n_w;
    cudaStream_t s = b->stream;
    if ((e = cudaMemcpyAsync(P.g, pts[i].g, sizeof(double2) * dm.ne, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P.delta, pts[i].delta, sizeof(double2) * dm.ne, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P.gam, pts[i].gamma_d, sizeof(double2) * nvc, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P.gam + nvc, pts[i].gamma_m, sizeof(double2) * nvc, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(P.sigma, 0, sizeof(double2) * dm.n_w * dm.N, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(P.red, 0, sizeof(double) * (2 * dm.n_w + 4), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(P.flags, 0, sizeof(int) * 4, s)) != cudaSuccess) {
      st = bfail(b, DF_ERR_CUDA, "batch inputs", e);
      goto bad;
    }
    if (P.sym && ((e = cudaMemcpyAsync(P.qmap, qmaps[i].data(), sizeof(int) * dm.N, cudaMemcpyHostToDevice, s)) !=
                      cudaSuccess ||
                  (e = cudaMemcpyAsync(P.qrep, qreps[i].data(), sizeof(int) * P.n_orb, cudaMemcpyHostToDevice, s)) !=
                      cudaSuccess)) {
      st = bfail(b, DF_ERR_CUDA, "batch orbit tables", e);
      goto bad;
    }
  }
  if ((e = cudaMemcpyAsync(b->d_pts, b->host_pts.data(), sizeof(PointDev) * npts, cudaMemcpyHostToDevice,
                           b->stream)) != cudaSuccess) {
    st = bfail(b, DF_ERR_CUDA, "point table", e);
    goto bad;
  }
  {
    size_t fs = 0;
    for (int i = 0; i < npts; ++i)
      fs = std::max(fs, fft_smem_bytes(b->host_pts[i].dm.nk, b->host_pts[i].dm.N, 1));
    cudaFuncSetAttribute((const void*)batch_setup_dyson_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs);
    for (int i = 0; i < npts; ++i) {
      const Dims& dm = b->host_pts[i].dm;
      batch_setup_elem_kernel<<<64, 256, 0, b->stream>>>(b->d_pts, i);
      batch_setup_dyson_kernel<<<dm.ne, kFftThreads, fft_smem_bytes(dm.nk, dm.N, 1), b->stream>>>(b->d_pts, i);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) { st = bfail(b, DF_ERR_CUDA, "batch set-up", e); goto bad; }
  }

  // ---- work tables ----
  {
    std::vector<long> ps(npts + 1, 0), bs(npts + 1, 0);
    size_t f1 = 0, f2 = 0;
    for (int i = 0; i < npts; ++i) {
      const Dims& dm = b->host_pts[i].dm;
      ps[i + 1] = ps[i] + (long)dm.nb * dm.n_w;
      bs[i + 1] = bs[i] + dm.n_w;
      f1 = std::max(f1, fft_smem_bytes(dm.nk, dm.N, 1));
      f2 = std::max(f2, fft_smem_bytes(dm.nk, dm.N, 2));
    }
    b->total_planes = ps[npts];
    b->total_box = bs[npts];
    b->fft_smem1 = f1;
    b->fft_smem2 = f2;
    BALLOC(b->d_plane_start, sizeof(long) * (npts + 1), "plane table");
    BALLOC(b->d_box_start, sizeof(long) * (npts + 1), "box table");
    cudaMemcpy(b->d_plane_start, ps.data(), sizeof(long) * (npts + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_box_start, bs.data(), sizeof(long) * (npts + 1), cudaMemcpyHostToDevice);
    cudaFuncSetAttribute((const void*)batch_bubble_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f1);
    cudaFuncSetAttribute((const void*)batch_sigma_prod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f1);
    cudaFuncSetAttribute((const void*)batch_sigma_dyson_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f2);

    // ladder groups: FP64 (all non-mixed points) + one per mixed padded order
    std::vector<int> idx(npts);
    for (int i = 0; i < npts; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
      return b->host_pts[x].dm.n_w > b->host_pts[y].dm.n_w;   // largest ladders first
    });
    LadderGroup f64;
    std::vector<LadderGroup> mixed_groups(6);   // padded orders 4 .. 128
    for (int k = 0; k < 6; ++k) {
      mixed_groups[k].mixed = true;
      mixed_groups[k].np = 4 << k;
    }
    for (int i : idx) {
      if (b->host_pts[i].mixed) {
        int k = 0;
        while ((4 << k) < mixed_np_of(b->host_pts[i].dm.n_w)) ++k;
        mixed_groups[k].order.push_back(i);
      } else {
        f64.order.push_back(i);
      }
    }
    if (!f64.order.empty()) b->groups.push_back(f64);
    for (int k = 5; k >= 0; --k)
      if (!mixed_groups[k].order.empty()) b->groups.push_back(mixed_groups[k]);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
      LadderGroup& g = b->groups[gi];
      g.counter_slot = (int)gi;
      g.nseg = (int)g.order.size();
      std::vector<long> st_(g.nseg + 1, 0);
      for (int k = 0; k < g.nseg; ++k) {
        const Dims& dm = b->host_pts[g.order[k]].ldm;
        st_[k + 1] = st_[k] + 2L * dm.na * dm.N;
      }
      g.total = st_[g.nseg];
      BALLOC(g.d_start, sizeof(long) * (g.nseg + 1), "ladder table");
      BALLOC(g.d_order, sizeof(int) * g.nseg, "ladder order");
      cudaMemcpy(g.d_start, st_.data(), sizeof(long) * (g.nseg + 1), cudaMemcpyHostToDevice);
      cudaMemcpy(g.d_order, g.order.data(), sizeof(int) * g.nseg, cudaMemcpyHostToDevice);
    }
    BALLOC(b->d_counters, sizeof(unsigned long long) * std::max<size_t>(1, b->groups.size()), "counters");
    // global LU scratch for FP64 ladders of order > kLuSmemOrder
    // (mixed points: their hand-back ladders use the same scratch, one slice per block)
    int big = 0;
    long mixed_ladders = 0;
    for (auto& g : b->groups)
      for (int p : g.order) {
        const Dims& dm = b->host_pts[p].ldm;
        big = std::max(big, dm.n_w > kLuSmemOrder ? dm.n_w : 0);
        if (g.mixed) mixed_ladders += 2L * dm.na * dm.N;
      }
    if (big) {
      b->ws_stride = (size_t)big * big;
      BALLOC(b->ws, sizeof(double2) * b->ws_stride * (size_t)b->sms * kLuScratchPerSm, "LU scratch");
    }
    if (mixed_ladders > 0) {
      BALLOC(b->d_redo, sizeof(int) * (1 + (size_t)mixed_ladders), "hand-back list");
      size_t sm_max = 0;
      for (auto& g : b->groups)
        if (g.mixed)
          for (int p : g.order) {
            const int n = b->host_pts[p].dm.n_w;
            sm_max = std::max(sm_max, sizeof(double2) * (size_t)bse_layout(n, default_nc(n), n <= kLuSmemOrder).total);
          }
      b->redo_smem = sm_max;
      b->redo_grid = b->sms * kLuScratchPerSm;   // blocks beyond the list's count exit at once
      e = cudaFuncSetAttribute((const void*)batch_bse_f64_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sm_max);
      if (e != cudaSuccess) { st = bfail(b, DF_ERR_CUDA, "hand-back kernel", e); goto bad; }
    }
  }
#undef BALLOC
  if ((st = configure_groups(b)) != DF_OK) goto bad;
  if ((st = build_graph(b)) != DF_OK) goto bad;
  if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) { st = bfail(b, DF_ERR_CUDA, "batch init", e); goto bad; }
  *out = b;
  return DF_OK;
bad:
  fprintf(stderr, "libdf: df_batch_init failed: %s\n", b->err.c_str());
  df_batch_destroy(b);
  return st;
}

void df_batch_destroy(df_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& g : b->groups) {
    cudaFree(g.d_start);
    cudaFree(g.d_order);
  }
  cudaFree(b->arena);
  cudaFree(b->d_pts);
  cudaFree(b->d_out);
  cudaFree(b->d_plane_start);
  cudaFree(b->d_box_start);
  cudaFree(b->d_counters);
  cudaFree(b->ws);
  cudaFree(b->d_redo);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

df_status df_batch_iterate(df_batch* b, int max_iter, int* passes_done, double* resid, int* active) {
  if (!b || max_iter < 0) return DF_ERR_ARG;
  int it = 0;
  bool any = true;
  for (; it < max_iter && any; ++it) {
    B_CUDA(b, cudaGraphLaunch(b->exec, b->stream), "graph launch");
    B_CUDA(b, cudaStreamSynchronize(b->stream), "batch pass");
    any = false;
    for (int i = 0; i < b->npts; ++i) any |= (b->h_out[3 * i + 1] != 0.0);
    ++b->passes;
  }
  int fl = 0;
  for (int i = 0; i < b->npts; ++i) {
    if (resid) resid[i] = b->h_out[3 * i];
    if (active) active[i] = (int)b->h_out[3 * i + 1];
    fl |= (int)b->h_out[3 * i + 2];
  }
  if (passes_done) *passes_done = it;
  if (fl & kFlagSingular) return bfail(b, DF_ERR_SINGULAR, "exactly zero pivot in a ladder solve");
  if (fl & kFlagTcTimeout)
    return bfail(b, DF_ERR_TIMEOUT, "a tensor-core completion wait in the mixed ladder kernel gave up");
  if (fl & kFlagTcLayout) return bfail(b, DF_ERR_CUDA, "mixed ladder kernel: shared-memory operands not 1024-byte aligned");
  return any ? DF_ERR_NOT_CONVERGED : DF_OK;
}

df_status df_batch_get_sigma(df_batch* b, int point, double* out, int is_device) {
  if (!b || !out || point < 0 || point >= b->npts) return DF_ERR_ARG;
  const PointDev& P = b->host_pts[point];
  B_CUDA(b, cudaMemcpyAsync(out, P.sigma, sizeof(double2) * P.dm.n_w * P.dm.N,
                            is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream),
         "df_batch_get_sigma");
  if (!is_device) B_CUDA(b, cudaStreamSynchronize(b->stream), "df_batch_get_sigma");
  return DF_OK;
}

df_status df_batch_reset(df_batch* b) {
  if (!b) return DF_ERR_ARG;
  for (int i = 0; i < b->npts; ++i) {
    PointDev& P = b->host_pts[i];
    P.active = 1;
    P.resid = -1.0;
    B_CUDA(b, cudaMemsetAsync(P.sigma, 0, sizeof(double2) * P.dm.n_w * P.dm.N, b->stream), "reset");
    B_CUDA(b, cudaMemsetAsync(P.flags, 0, sizeof(int) * 4, b->stream), "reset");
  }
  B_CUDA(b, cudaMemcpyAsync(b->d_pts, b->host_pts.data(), sizeof(PointDev) * b->npts, cudaMemcpyHostToDevice,
                            b->stream), "reset");
  for (int i = 0; i < b->npts; ++i) {
    const Dims& dm = b->host_pts[i].dm;
    batch_setup_dyson_kernel<<<dm.ne, kFftThreads, fft_smem_bytes(dm.nk, dm.N, 1), b->stream>>>(b->d_pts, i);
  }
  B_CUDA(b, cudaGetLastError(), "reset");
  B_CUDA(b, cudaStreamSynchronize(b->stream), "reset");
  b->passes = 0;
  return DF_OK;
}

df_status df_batch_autotune(df_batch* b, const char* cache_path, int* chosen) {
  if (!b) return DF_ERR_ARG;
  // signature of the batch: every point's (D, N_k, n_w, N_W, reduced) and the precision
  std::string sig = "v1 p" + std::to_string(b->precision);
  for (auto& P : b->host_pts)
    sig += " " + std::to_string(P.dm.D) + "," + std::to_string(P.dm.nk) + "," + std::to_string(P.dm.n_w) + "," +
           std::to_string(P.dm.nb) + (P.sym ? "s" : "");
  const int nc_c[] = {0, 8, 16, 32};
  const int ch_c[] = {1, 4};
  int best_nc = 0, best_ch = 1;
  bool cached = false;
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[1 << 16];
      while (fgets(line, sizeof line, f)) {
        int nc = 0, ch = 0, pos = 0;
        if (sscanf(line, "%d %d %n", &nc, &ch, &pos) == 2) {
          std::string rest(line + pos);
          while (!rest.empty() && (rest.back() == '\n' || rest.back() == '\r')) rest.pop_back();
          if (rest == sig) {
            best_nc = nc;
            best_ch = ch;
            cached = true;
          }
        }
      }
      fclose(f);
    }
  }
  if (!cached) {
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    B_CUDA(b, cudaEventCreate(&e0), "event");
    B_CUDA(b, cudaEventCreate(&e1), "event");
    for (int nc : nc_c) {
      for (int ch : ch_c) {
        b->nc_override = nc;
        b->chunk = ch;
        df_status st = df_batch_reset(b);
        if (st != DF_OK) return st;
        if ((st = configure_groups(b)) != DF_OK) return st;
        if ((st = build_graph(b)) != DF_OK) return st;
        B_CUDA(b, cudaGraphLaunch(b->exec, b->stream), "tune warm-up");
        B_CUDA(b, cudaEventRecord(e0, b->stream), "event");
        B_CUDA(b, cudaGraphLaunch(b->exec, b->stream), "tune pass");
        B_CUDA(b, cudaEventRecord(e1, b->stream), "event");
        B_CUDA(b, cudaEventSynchronize(e1), "event");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best_nc = nc;
          best_ch = ch;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cache_path) {
      FILE* f = fopen(cache_path, "a");
      if (f) {
        fprintf(f, "%d %d %s\n", best_nc, best_ch, sig.c_str());
        fclose(f);
      }
    }
  }
  b->nc_override = best_nc;
  b->chunk = best_ch;
  df_status st = df_batch_reset(b);
  if (st != DF_OK) return st;
  if ((st = configure_groups(b)) != DF_OK) return st;
  if ((st = build_graph(b)) != DF_OK) return st;
  B_CUDA(b, cudaStreamSynchronize(b->stream), "autotune");
  if (chosen) {
    chosen[0] = best_nc;
    chosen[1] = best_ch;
    chosen[2] = cached ? 1 : 0;
  }
  return DF_OK;
}

const char* df_batch_last_error(const df_batch* b) { return b ? b->err.c_str() : "NULL handle"; }

}  // extern "C"
