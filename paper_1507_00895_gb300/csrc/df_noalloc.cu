// df_bse_noalloc: the FP64 ladder solves of df_bse on caller-given device
// buffers, with the kernel's scratch memory in a fixed file-scope device
// array, so that the call itself allocates nothing.
//
// Who needs it: callers that cannot allocate device memory at the point of
// the call, for instance code embedded in a host application that owns the
// whole device-memory budget and forbids other allocations, or a
// latency-critical loop where cudaMalloc's implicit device synchronisation
// is not acceptable.  They pass the inputs and the output; the only scratch
// (gamma o gamma^T for the Gamma^(2) term, and the zero-pivot flags) lives
// in g_bse_scratch below, which every GPU that loads libdf holds until the
// process exits.
#include <cstdio>
#include <mutex>

#include "df_internal.cuh"

namespace df {
cudaError_t launch_gamma_gt_raw(int n, int count, const double2* gam, double2* gg, cudaStream_t stream);
cudaError_t launch_bse_both_raw(const Dims& dm, const double2* gam, const double2* gg, const double2* chi,
                                double2* kc, int* flags, int device, cudaStream_t stream);
}  // namespace df

namespace {

// 2^19 complex128 = 8 MiB for gamma o gamma^T of both channels
// (2 * n_bos * n_w^2 complex), plus 256 bytes for the flags.
constexpr size_t kScratchComplex = size_t(1) << 19;
constexpr size_t kFlagComplex = 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_bse_scratch[kScratchComplex + kFlagComplex];

std::mutex g_mu;
double2* g_scratch_ptr[kMaxDevices] = {};

df_status reject(const char* why) {
  fprintf(stderr, "libdf: df_bse_noalloc: %s\n", why);
  return DF_ERR_ARG;
}

}  // namespace

extern "C" df_status df_bse_noalloc(const double* gamma, const double* chi, int n_w, int n_bos, int n_k_total,
                                    double* kernel, void* stream) {
  if (!gamma || !chi || !kernel) return reject("NULL pointer");
  if (n_w < 2 || n_w > 96 || (n_w & 1)) return reject("n_w must be even and in [2, 96]");
  if (n_bos < 1 || n_bos > 63 || !(n_bos & 1)) return reject("n_bos must be odd and in [1, 63]");
  if (n_k_total < 1 || n_k_total > 4096) return reject("n_k_total must be in [1, 4096]");
  if ((size_t)2 * n_bos * n_w * n_w > kScratchComplex)
    return reject("2 * n_bos * n_w^2 exceeds the 2^19 complex (8 MiB) scratch array");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    fprintf(stderr, "libdf: df_bse_noalloc: cudaGetDevice: %s\n", cudaGetErrorString(e));
    return DF_ERR_CUDA;
  }
  if (dev >= kMaxDevices) return reject("device ordinal >= 64");
  double2* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the
    // array (its host-side name is only a stand-in, not a device address)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_bse_scratch);
      if (e != cudaSuccess) {
        fprintf(stderr, "libdf: df_bse_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
        return DF_ERR_CUDA;
      }
      g_scratch_ptr[dev] = (double2*)p;
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  int* flags = (int*)(scratch + kScratchComplex);
  df::Dims dm{};
  dm.N = n_k_total;
  dm.n_w = n_w;
  dm.nb = n_bos;
  dm.a0 = 0;
  dm.na = n_bos;
  dm.m_max = (n_bos - 1) / 2;
  dm.ne = n_w + 2 * dm.m_max;
  // the flags must start at zero; gamma o gamma^T is fully rewritten below
  if ((e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), s)) != cudaSuccess ||
      (e = df::launch_gamma_gt_raw(n_w, 2 * n_bos, (const double2*)gamma, scratch, s)) != cudaSuccess ||
      (e = df::launch_bse_both_raw(dm, (const double2*)gamma, scratch, (const double2*)chi, (double2*)kernel,
                                   flags, dev, s)) != cudaSuccess) {
    fprintf(stderr, "libdf: df_bse_noalloc: %s\n", cudaGetErrorString(e));
    return DF_ERR_CUDA;
  }
  return DF_OK;
}
