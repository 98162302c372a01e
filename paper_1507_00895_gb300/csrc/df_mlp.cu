// Learned warm start of the dual self-energy: a dense network (4 layers,
// n_in -> W -> W -> W -> n_out, tanh between, linear output) evaluated and
// trained with this file's kernels.  Operands of every matrix product are
// rounded to BF16 and multiplied on the tensor cores (tcgen05, FP32
// accumulate in tensor memory); master weights, biases, Adam moments and
// activations are FP32.  The network's output is Sigma~ on the irreducible wedge of the
// square lattice's point group at positive Matsubara frequencies;
// df_warmstart_sigma expands it to the whole grid (D4 images and
// Sigma~(k, -w) = conj Sigma~(k, w)) and sets it as the loop's Sigma~.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include <cuda_bf16.h>

#include "df_tcgj_dev.cuh"

namespace df {

constexpr int kGm = 128, kGn = 128, kGk = 64;  // block tile: M x N outputs, K per stage
constexpr int kGemmThreads = 256;               // 8 warps: staging, epilogue; thread 0 issues the MMAs
constexpr int kGemmTmemCols = 128;              // the FP32 accumulator tile (N = 128 columns)
constexpr int kGemmStage = kGm * kGk * 2;       // bytes of one operand tile (128 rows x 64 bf16)
constexpr int kGemmSmem = 4 * kGemmStage + 1024;   // two stages of (A, B) + alignment slack

// C[m][n] = act(sum_k bf16(A(m,k)) bf16(B(k,n)) + bias[n]) (+ C[m][n] if accumulate)
// A(m,k) = A[m sam + k sak], B(k,n) = B[k sbk + n sbn], C row-major with ldc.
// act: 0 identity, 1 tanh.  One 128 x 128 output tile per block on the tensor
// cores (tcgen05, M = 128, N = 128, K = 16 per MMA, FP32 accumulator in tensor
// memory): per stage of 64 k the block rounds its A and B tiles to BF16 into
// shared memory (K-major, 128-byte swizzle), thread 0 issues 4 MMAs and commits
// them to the stage buffer's barrier, and the next stage is staged into the
// other buffer meanwhile.  The epilogue reads the accumulator from tensor
// memory (warp w: lanes 32 (w % 4) .., columns 64 (w / 4) ..).  Waits are
// bounded; one that gives up sets *err.
__global__ void __launch_bounds__(kGemmThreads)
gemm_tc_kernel(int M, int N, int K, const float* __restrict__ A, long sam, long sak, const float* __restrict__ B,
               long sbk, long sbn, float* __restrict__ C, long ldc, const float* __restrict__ bias, int act,
               int accumulate, int* __restrict__ err) {
  extern __shared__ unsigned char gsm_raw[];
  __shared__ uint64_t bar_s[2];
  __shared__ unsigned tslot_s;
  unsigned char* gsm = reinterpret_cast<unsigned char*>(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);
  const int m0 = blockIdx.y * kGm, n0 = blockIdx.x * kGn;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc_cols<kGemmTmemCols>(&tslot_s);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_s[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_s[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  const unsigned tmem = tslot_s;
  const unsigned idesc = umma_idesc_bf16(kGm, kGn);
  unsigned ph = 0u;                                  // bit b: the phase of buffer b's barrier
  bool ok = true;
  const int nst = (K + kGk - 1) / kGk;
  for (int st = 0; st < nst; ++st) {
    const int b = st & 1, k0 = st * kGk;
    if (st >= 2) {                                   // the MMAs that read this buffer are done
      ok = ok && mbar_wait(&bar_s[b], (ph >> b) & 1u);
      ph ^= 1u << b;
    }
    if (__syncthreads_or(!ok)) break;
    __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(gsm + b * 2 * kGemmStage);
    __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(gsm + b * 2 * kGemmStage + kGemmStage);
    // A tile [m][k]: k fastest when A's rows are contiguous, m fastest otherwise
    for (int idx = tid; idx < kGm * kGk; idx += kGemmThreads) {
      const int r = sak == 1 ? idx / kGk : idx % kGm, k = sak == 1 ? idx % kGk : idx / kGm;
      const int gm = m0 + r, gk = k0 + k;
      const float v = (gm < M && gk < K) ? A[gm * sam + gk * sak] : 0.f;
      As[swz(r, k)] = __float2bfloat16_rn(v);
    }
    // B tile [n][k]: n fastest when B's rows (over n) are contiguous, k fastest otherwise
    for (int idx = tid; idx < kGn * kGk; idx += kGemmThreads) {
      const int nn = sbn == 1 ? idx % kGn : idx / kGk, k = sbn == 1 ? idx / kGn : idx % kGk;
      const int gn = n0 + nn, gk = k0 + k;
      const float v = (gn < N && gk < K) ? B[gk * sbk + gn * sbn] : 0.f;
      Bs[swz(nn, k)] = __float2bfloat16_rn(v);
    }
    fence_async_smem();
    tc05_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc05_fence_after();
      const unsigned a = smem_u32(As), bb = smem_u32(Bs);
#pragma unroll
      for (int ks = 0; ks < kGk / 16; ++ks)
        umma_bf16(tmem, umma_desc_sw128(a + 32 * ks), umma_desc_sw128(bb + 32 * ks), idesc,
                  (st > 0 || ks > 0) ? 1u : 0u);
      umma_commit(&bar_s[b]);
    }
  }
  // the last one or two commits: every MMA done before the epilogue
  for (int st = nst - 2 < 0 ? 0 : nst - 2; ok && st < nst; ++st) {
    const int b = st & 1;
    ok = mbar_wait(&bar_s[b], (ph >> b) & 1u);
    ph ^= 1u << b;
  }
  tc05_fence_after();
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(err, 1);
  } else {
    const int q = warp & 3, half = warp >> 2;
    const int r = m0 + 32 * q + lane;
    const unsigned tl = tmem + ((32u * q) << 16) + (unsigned)(64 * half);
#pragma unroll
    for (int c16 = 0; c16 < 4; ++c16) {
      float v[16];
      tmem_ld16(tl + 16 * c16, v);
      if (r < M) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int cn = n0 + 64 * half + 16 * c16 + e;
          if (cn < N) {
            float x = v[e];
            if (bias) x += bias[cn];
            if (act == 1) x = tanhf(x);
            float* dst = C + (long)r * ldc + cn;
            *dst = accumulate ? *dst + x : x;
          }
        }
      }
    }
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  if (warp == 0) tmem_dealloc_cols<kGemmTmemCols>(tmem);
}

// dY = 2 (Y - T) / (B n_out); per-block partial sums of (Y - T)^2
__global__ void mse_grad_kernel(long count, const float* __restrict__ y, const float* __restrict__ t,
                                float* __restrict__ dy, float scale, float* __restrict__ partial) {
  __shared__ float sred[32];
  float s = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d * scale;
    s += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < blockDim.x / 32) ? sred[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// dZ = dA (1 - A^2)  (tanh layers)
__global__ void tanh_back_kernel(long count, const float* __restrict__ a, float* __restrict__ dz) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    dz[i] = dz[i] * (1.f - a[i] * a[i]);
}

// db[n] = sum_m dZ[m][n]
__global__ void colsum_kernel(int M, int N, const float* __restrict__ dz, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += dz[(long)m * N + n];
  db[n] = s;
}

__global__ void adam_kernel(long count, float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m1,
                            float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const float gv = gr[i];
    const float a = b1 * m1[i] + (1.f - b1) * gv;
    const float b = b2 * m2[i] + (1.f - b2) * gv * gv;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

// Sigma~[i][r] from the wedge output y [n_wedge][n_w/2][2]: w = kmap[r],
// n = i - n_w/2 >= 0 -> y[w][n], n < 0 -> conj y[w][-n-1]; y de-normalised
// with mean / std of the same layout.
__global__ void warmstart_expand_kernel(int n_w, int N, const int* __restrict__ kmap, const float* __restrict__ y,
                                        const float* __restrict__ mean, const float* __restrict__ sd,
                                        double2* __restrict__ sigma) {
  const int total = n_w * N;
  const int half = n_w / 2;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int i = idx / N, r = idx - i * N;
    const int n = i - half;
    const int f = n >= 0 ? n : -n - 1;
    const long o = ((long)kmap[r] * half + f) * 2;
    const double re = (double)y[o] * sd[o] + mean[o];
    const double im = (double)y[o + 1] * sd[o + 1] + mean[o + 1];
    sigma[idx] = mk(re, n >= 0 ? im : -im);
  }
}

}  // namespace df

using namespace df;

struct df_mlp {
  int dims[5];
  int max_batch = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  float* params = nullptr;   // W1 b1 W2 b2 W3 b3 W4 b4 (W_l row-major [in][out])
  float* grads = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  long nparam = 0;
  long off_w[4], off_b[4];
  float* act[5] = {};        // act[0] = input copy, act[l] = layer-l output
  float* dact = nullptr;     // scratch for dA / dZ (max width)
  float* dact2 = nullptr;
  float* partial = nullptr;
  int* d_timeout = nullptr;  // set by a tensor-core GEMM whose bounded wait gave up
  float* h_loss = nullptr;
  long step = 0;
};

namespace {

df_status mfail(df_mlp* m, df_status s, const char* what, cudaError_t e = cudaSuccess) {
  if (m) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s%s%s", what, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
    m->err = buf;
  }
  return s;
}

#define M_CUDA(m, call, what)                                                                  \
  do {                                                                                         \
    cudaError_t e__ = (call);                                                                  \
    if (e__ != cudaSuccess)                                                                    \
      return mfail((m), e__ == cudaErrorMemoryAllocation ? DF_ERR_OOM : DF_ERR_CUDA, (what), e__); \
  } while (0)

// err: the handle's device flag a GEMM sets when a bounded tensor-core wait gave up
cudaError_t gemm(cudaStream_t s, int* err, int M, int N, int K, const float* A, long sam, long sak, const float* B,
                 long sbk, long sbn, float* C, long ldc, const float* bias, int act, int accumulate) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute((const void*)gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               kGemmSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((N + kGn - 1) / kGn, (M + kGm - 1) / kGm);
  gemm_tc_kernel<<<grid, kGemmThreads, kGemmSmem, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, act, accumulate,
                                                       err);
  return cudaGetLastError();
}

int blocks_for(long n) { return (int)std::min<long>(1024, (n + 255) / 256); }

df_status forward(df_mlp* m, const float* x, int B) {
  M_CUDA(m, cudaMemcpyAsync(m->act[0], x, sizeof(float) * B * m->dims[0], cudaMemcpyDeviceToDevice, m->stream),
         "copy input");
  for (int l = 0; l < 4; ++l) {
    const int in = m->dims[l], out = m->dims[l + 1];
    M_CUDA(m, gemm(m->stream, m->d_timeout, B, out, in, m->act[l], in, 1, m->params + m->off_w[l], out, 1, m->act[l + 1], out,
                   m->params + m->off_b[l], l < 3 ? 1 : 0, 0),
           "forward GEMM");
  }
  return DF_OK;
}

df_status backward(df_mlp* m, const float* target, int B, float* loss_host) {
  const int nout = m->dims[4];
  const long count = (long)B * nout;
  const int nb = blocks_for(count);
  mse_grad_kernel<<<nb, 256, 0, m->stream>>>(count, m->act[4], target, m->dact, 1.f / (float)count, m->partial);
  M_CUDA(m, cudaGetLastError(), "loss");
  float* dz = m->dact;      // dZ of the current layer [B][out]
  float* da = m->dact2;     // dA of the layer below
  for (int l = 3; l >= 0; --l) {
    const int in = m->dims[l], out = m->dims[l + 1];
    // dW_l[in][out] = A_{l}^T dZ   (M = in, N = out, K = B)
    M_CUDA(m, gemm(m->stream, m->d_timeout, in, out, B, m->act[l], 1, in, dz, out, 1, m->grads + m->off_w[l], out, nullptr, 0, 0),
           "weight gradient");
    colsum_kernel<<<(out + 255) / 256, 256, 0, m->stream>>>(B, out, dz, m->grads + m->off_b[l]);
    M_CUDA(m, cudaGetLastError(), "bias gradient");
    if (l == 0) break;
    // dA_{l} [B][in] = dZ W_l^T   (M = B, N = in, K = out; B(k, n) = W[n][k])
    M_CUDA(m, gemm(m->stream, m->d_timeout, B, in, out, dz, out, 1, m->params + m->off_w[l], 1, out, da, in, nullptr, 0, 0),
           "activation gradient");
    tanh_back_kernel<<<blocks_for((long)B * in), 256, 0, m->stream>>>((long)B * in, m->act[l], da);
    M_CUDA(m, cudaGetLastError(), "tanh backward");
    float* t = dz;
    dz = da;
    da = t;
  }
  if (loss_host) {
    std::vector<float> part(nb);
    M_CUDA(m, cudaMemcpyAsync(part.data(), m->partial, sizeof(float) * nb, cudaMemcpyDeviceToHost, m->stream),
           "loss copy");
    int timeout = 0;
    M_CUDA(m, cudaMemcpyAsync(&timeout, m->d_timeout, sizeof(int), cudaMemcpyDeviceToHost, m->stream), "flag copy");
    M_CUDA(m, cudaStreamSynchronize(m->stream), "loss");
    if (timeout) return mfail(m, DF_ERR_TIMEOUT, "a tensor-core GEMM's completion wait gave up");
    double s = 0.0;
    for (float v : part) s += v;
    *loss_host = (float)(s / (double)count);
  }
  return DF_OK;
}

}  // namespace

extern "C" {

df_status df_mlp_create(df_mlp** out, int n_in, int width, int n_out, int max_batch, unsigned long long seed,
                        void* stream) {
  if (!out || n_in < 1 || width < 1 || n_out < 1 || max_batch < 1) return DF_ERR_ARG;
  *out = nullptr;
  df_mlp* m = new (std::nothrow) df_mlp();
  if (!m) return DF_ERR_OOM;
  const int d[5] = {n_in, width, width, width, n_out};
  memcpy(m->dims, d, sizeof d);
  m->max_batch = max_batch;
  m->stream = (cudaStream_t)stream;
  long o = 0;
  for (int l = 0; l < 4; ++l) {
    m->off_w[l] = o;
    o += (long)d[l] * d[l + 1];
    m->off_b[l] = o;
    o += d[l + 1];
  }
  m->nparam = o;
  // Glorot-uniform weights, zero biases (host RNG, seeded)
  std::vector<float> h(o, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < 4; ++l) {
    const float lim = std::sqrt(6.f / (float)(d[l] + d[l + 1]));
    std::uniform_real_distribution<float> U(-lim, lim);
    for (long i = 0; i < (long)d[l] * d[l + 1]; ++i) h[m->off_w[l] + i] = U(rng);
  }
  int maxw = std::max(std::max(n_in, width), n_out);
  cudaError_t e;
  df_status st = DF_OK;
  if ((e = cudaMalloc(&m->params, sizeof(float) * o)) != cudaSuccess ||
      (e = cudaMalloc(&m->grads, sizeof(float) * o)) != cudaSuccess ||
      (e = cudaMalloc(&m->m1, sizeof(float) * o)) != cudaSuccess ||
      (e = cudaMalloc(&m->m2, sizeof(float) * o)) != cudaSuccess ||
      (e = cudaMalloc(&m->dact, sizeof(float) * (long)max_batch * maxw)) != cudaSuccess ||
      (e = cudaMalloc(&m->dact2, sizeof(float) * (long)max_batch * maxw)) != cudaSuccess ||
      (e = cudaMalloc(&m->partial, sizeof(float) * 1024)) != cudaSuccess ||
      (e = cudaMalloc(&m->d_timeout, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(m->d_timeout, 0, sizeof(int))) != cudaSuccess) {
    st = mfail(m, DF_ERR_OOM, "cudaMalloc", e);
  }
  for (int l = 0; l < 5 && st == DF_OK; ++l)
    if ((e = cudaMalloc(&m->act[l], sizeof(float) * (long)max_batch * d[l])) != cudaSuccess)
      st = mfail(m, DF_ERR_OOM, "cudaMalloc activations", e);
  if (st == DF_OK &&
      ((e = cudaMemcpy(m->params, h.data(), sizeof(float) * o, cudaMemcpyHostToDevice)) != cudaSuccess ||
       (e = cudaMemset(m->m1, 0, sizeof(float) * o)) != cudaSuccess ||
       (e = cudaMemset(m->m2, 0, sizeof(float) * o)) != cudaSuccess ||
       (e = cudaMemset(m->grads, 0, sizeof(float) * o)) != cudaSuccess))
    st = mfail(m, DF_ERR_CUDA, "initialise parameters", e);
  if (st != DF_OK) {
    fprintf(stderr, "libdf: df_mlp_create: %s\n", m->err.c_str());
    df_mlp_destroy(m);
    return st;
  }
  *out = m;
  return DF_OK;
}

void df_mlp_destroy(df_mlp* m) {
  if (!m) return;
  cudaFree(m->params);
  cudaFree(m->grads);
  cudaFree(m->m1);
  cudaFree(m->m2);
  cudaFree(m->dact);
  cudaFree(m->dact2);
  cudaFree(m->partial);
  cudaFree(m->d_timeout);
  for (auto* a : m->act) cudaFree(a);
  delete m;
}

df_status df_mlp_param_count(const df_mlp* m, long* count) {
  if (!m || !count) return DF_ERR_ARG;
  *count = m->nparam;
  return DF_OK;
}

df_status df_mlp_forward(df_mlp* m, const float* x, int batch, float* y) {
  if (!m || !x || !y || batch < 1 || batch > m->max_batch) return DF_ERR_ARG;
  df_status s = forward(m, x, batch);
  if (s != DF_OK) return s;
  M_CUDA(m, cudaMemcpyAsync(y, m->act[4], sizeof(float) * batch * m->dims[4], cudaMemcpyDeviceToDevice, m->stream),
         "copy output");
  return DF_OK;
}

df_status df_mlp_gradients(df_mlp* m, const float* x, const float* target, int batch, float* loss_host) {
  if (!m || !x || !target || batch < 1 || batch > m->max_batch) return DF_ERR_ARG;
  df_status s = forward(m, x, batch);
  if (s != DF_OK) return s;
  return backward(m, target, batch, loss_host);
}

df_status df_mlp_adam_step(df_mlp* m, float lr, float beta1, float beta2, float eps) {
  if (!m) return DF_ERR_ARG;
  ++m->step;
  const float c1 = 1.f - std::pow(beta1, (float)m->step), c2 = 1.f - std::pow(beta2, (float)m->step);
  adam_kernel<<<blocks_for(m->nparam), 256, 0, m->stream>>>(m->nparam, m->params, m->grads, m->m1, m->m2, lr, beta1,
                                                           beta2, eps, c1, c2);
  M_CUDA(m, cudaGetLastError(), "adam");
  return DF_OK;
}

df_status df_mlp_train_step(df_mlp* m, const float* x, const float* target, int batch, float lr, float* loss_host) {
  df_status s = df_mlp_gradients(m, x, target, batch, loss_host);
  if (s != DF_OK) return s;
  return df_mlp_adam_step(m, lr, 0.9f, 0.999f, 1e-8f);
}

df_status df_mlp_params(df_mlp* m, float* buf, int set, int is_device) {
  if (!m || !buf) return DF_ERR_ARG;
  const cudaMemcpyKind k = set ? (is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)
                               : (is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  M_CUDA(m, cudaMemcpyAsync(set ? m->params : buf, set ? buf : m->params, sizeof(float) * m->nparam, k, m->stream),
         "params");
  M_CUDA(m, cudaStreamSynchronize(m->stream), "params");
  return DF_OK;
}

df_status df_mlp_grads(df_mlp* m, float* buf, int is_device) {
  if (!m || !buf) return DF_ERR_ARG;
  M_CUDA(m, cudaMemcpyAsync(buf, m->grads, sizeof(float) * m->nparam,
                            is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream),
         "grads");
  M_CUDA(m, cudaStreamSynchronize(m->stream), "grads");
  return DF_OK;
}

const char* df_mlp_last_error(const df_mlp* m) { return m ? m->err.c_str() : "NULL handle"; }

df_status df_warmstart_sigma(df_ctx* c, const float* y, const float* mean, const float* sd, const int* kmap) {
  if (!c || !y || !mean || !sd || !kmap) return DF_ERR_ARG;
  if (c->dm.n_w & 1) return DF_ERR_ARG;
  const int total = c->dm.n_w * c->dm.N;
  warmstart_expand_kernel<<<(total + 255) / 256, 256, 0, c->stream>>>(c->dm.n_w, c->dm.N, kmap, y, mean, sd, c->sigma);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_dyson_ifft(c, c->dm.m_max, c->dm.n_w);
  if (e != cudaSuccess) {
    c->err = std::string("df_warmstart_sigma: ") + cudaGetErrorString(e);
    return DF_ERR_CUDA;
  }
  return DF_OK;
}

}  // extern "C"
