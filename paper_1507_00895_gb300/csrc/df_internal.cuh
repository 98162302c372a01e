// Internal declarations of libdf: device helpers shared by the kernels and
// the context layout used by the host code.  Not part of the public ABI
// (that is include/df.h).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/df.h"

namespace df {

// bits of the ladder kernels' flags word
constexpr int kFlagSingular = 1;    // an exactly zero pivot
constexpr int kFlagRadius = 2;      // a ladder outside the radius of convergence
constexpr int kFlagTcTimeout = 4;   // a bounded tensor-core completion wait gave up
constexpr int kFlagTcLayout = 8;    // tensor-core operands not 1024-byte aligned (no MMA issued)
constexpr int kFlagRefine = 16;     // a mixed-precision ladder missed its error bound and was not re-solved

// Per-ladder error control of the mixed-precision ladder solves.  After the
// one correction E of X0 ~ D^-1 gamma, rho = max_j |E_jj| / max_j |Gamma_jj|
// (|re| + |im|) is the relative size of the correction; with a fixed FP32
// factorisation each correction shrinks the error by about the same factor,
// so the error left in diag Gamma is about rho^2 of its largest entry.  A
// ladder with rho^2 above rho2_max (or a non-finite value) is appended to
// the hand-back list (redo[0] = count, redo[1 + i] = (c N_W + a) N + q) for
// the FP64 LU, or, without a list, flagged kFlagRefine.  worst receives the
// call's largest rho^2 (float bits; non-negative floats order as integers).
struct MixedCheck {
  int* redo;
  unsigned* worst;
  float rho2_max;
  int base;       // added to the system index in the list (the batch: point << 24)
};

__device__ __forceinline__ void mixed_check_ladder(const MixedCheck& mc, float emax, float gmax, bool finite,
                                                   long sys, int* flags) {
  float rho2;
  if (!finite) rho2 = __int_as_float(0x7f800000);
  else if (gmax > 0.f) rho2 = (emax / gmax) * (emax / gmax);
  else rho2 = emax > 0.f ? __int_as_float(0x7f800000) : 0.f;
  if (mc.worst) atomicMax(mc.worst, __float_as_uint(rho2));
  if (!(rho2 <= mc.rho2_max)) {
    if (mc.redo) {
      const int i = atomicAdd(mc.redo, 1);
      mc.redo[1 + i] = mc.base + (int)sys;
    } else {
      atomicOr(flags, kFlagRefine);
    }
  }
}

// ---------------------------------------------------------------------------
// complex arithmetic on double2 / float2 (x = real, y = imag)
// ---------------------------------------------------------------------------

template <typename R> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <typename R> using cplx = typename cplx_t<R>::type;

__host__ __device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
__host__ __device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }

__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return mk(a.x - b.x, a.y - b.y); }

template <typename C>
__host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// c - a*b
template <typename C>
__host__ __device__ __forceinline__ C cfms(C a, C b, C c) {
  return mk(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c) {
  return mk(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
// c + a*b
template <typename C>
__host__ __device__ __forceinline__ C cfma(C a, C b, C c) {
  return mk(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return mk(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
template <typename C>
__host__ __device__ __forceinline__ C cscale(C a, decltype(a.x) s) { return mk(a.x * s, a.y * s); }
template <typename C>
__host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <typename C>
__host__ __device__ __forceinline__ decltype(C().x) cabs1(C a) { return fabs(a.x) + fabs(a.y); }
template <typename C>
__host__ __device__ __forceinline__ decltype(C().x) cabs2(C a) { return a.x * a.x + a.y * a.y; }
// 1/z with a scaling step so that |z|^2 cannot overflow or underflow
template <typename C>
__host__ __device__ __forceinline__ C cinv(C z) {
  using R = decltype(z.x);
  R s = fabs(z.x) > fabs(z.y) ? fabs(z.x) : fabs(z.y);
  R inv_s = R(1) / s;
  R a = z.x * inv_s, b = z.y * inv_s;
  R d = R(1) / ((a * a + b * b) * s);
  return mk(a * d, -b * d);
}

// ---------------------------------------------------------------------------
// lattice helpers: the grid is N_k^D points, flattened with the last axis
// fastest; axis d occupies bits [(D-1-d) p, (D-d) p) of the flat index,
// N_k = 2^p.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int reflect_index(int r, int D, int p) {
  // flat index of -r (each axis j -> (N_k - j) mod N_k)
  const int mask = (1 << p) - 1;
  int out = 0;
  for (int d = 0; d < D; ++d) {
    int j = (r >> (d * p)) & mask;
    out |= ((-j) & mask) << (d * p);
  }
  return out;
}

__device__ __forceinline__ int bitrev_axes(int r, int D, int p) {
  // reverse the p bits of every axis digit (an involution)
  if (p == 0) return r;
  const int mask = (1 << p) - 1;
  int out = 0;
  for (int d = 0; d < D; ++d) {
    int j = (r >> (d * p)) & mask;
    out |= (int)(__brev((unsigned)j) >> (32 - p)) << (d * p);
  }
  return out;
}

// Twiddles w[m] = exp(-2 pi i m / N_k), m < N_k/2, into shared memory.
template <typename C>
__device__ __forceinline__ void load_twiddles(C* tw, int nk) {
  using R = decltype(C().x);
  for (int m = threadIdx.x; m < nk / 2; m += blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)m / (double)nk, &s, &c);
    tw[m] = mk((R)c, (R)s);
  }
}

// In-place D-dimensional radix-2 decimation-in-time DFT of the N = 2^(D p)
// points in shared memory s.  The input must be stored in per-axis
// bit-reversed order (see bitrev_axes); the output is in natural order.
// sign: forward (-1) computes X(k) = sum_r exp(-i k.r) x(r); inverse (+1)
// computes sum_k exp(+i k.r) X(k) (no 1/N).  All threads of the block must
// call it; it ends with __syncthreads().
template <typename C>
__device__ void fft_dit_smem(C* s, int D, int p, const C* tw, bool inverse) {
  const int half = 1 << (D * p - 1);
  for (int d = 0; d < D; ++d) {
    const int base = d * p;  // axis bits [base, base+p)
    for (int st = 0; st < p; ++st) {
      const int h = 1 << st;
      const int bit = base + st;
      const int lowmask = (1 << bit) - 1;
      for (int t = threadIdx.x; t < half; t += blockDim.x) {
        const int i0 = ((t >> bit) << (bit + 1)) | (t & lowmask);
        const int i1 = i0 | (1 << bit);
        const int j = (i0 >> base) & (h - 1);
        C w = tw[j << (p - 1 - st)];
        if (inverse) w.y = -w.y;
        C a = s[i0];
        C b = cmul(s[i1], w);
        s[i0] = a + b;
        s[i1] = a - b;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

struct Dims {
  int D, nk, p, N;       // lattice
  int n_w, m_max, nb, ne;
  int a0, na;            // the bosonic planes a0 .. a0 + na - 1 this problem owns (the Omega split)
  double beta, T, mu, t, tp;
};

}  // namespace df

// ---- double-float (FP32 pair) arithmetic ----
// double-float helpers (value = hi + lo, |lo| <= ulp(hi)/2 after renormalisation)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// acc (hi, lo) += p exactly-ish: hi absorbs p with its rounding error moved to lo
__device__ __forceinline__ void df_add(float& hi, float& lo, float p) {
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo += e;
}
// (sr + lr, si + li) += (ah + al)(bh + bl) for complex double-float operands:
// the four leading products exactly (product + fma error), summed by TwoSum
// into the leading words; their errors and the four cross products go to
// the trailing words.  ~2^-46 relative to the largest partial sum.
__device__ __forceinline__ void cdf_fma(float& sr, float& lr, float& si, float& li, float2 ah, float2 al, float2 bh,
                                        float2 bl) {
  float p, e;
  p = ah.x * bh.x; e = fmaf(ah.x, bh.x, -p); df_add(sr, lr, p); lr += e;
  p = -ah.y * bh.y; e = fmaf(-ah.y, bh.y, -p); df_add(sr, lr, p); lr += e;
  lr += fmaf(ah.x, bl.x, fmaf(al.x, bh.x, fmaf(-ah.y, bl.y, -al.y * bh.y)));
  p = ah.x * bh.y; e = fmaf(ah.x, bh.y, -p); df_add(si, li, p); li += e;
  p = ah.y * bh.x; e = fmaf(ah.y, bh.x, -p); df_add(si, li, p); li += e;
  li += fmaf(ah.x, bl.y, fmaf(al.x, bh.y, fmaf(ah.y, bl.x, al.y * bh.x)));
}

// ---- packed FP32 pairs: the sm_100+ f32x2 instructions, elementwise and
// rounded to nearest like their scalar forms (a complex value's two halves,
// or two lanes of the same step, in one instruction) ----
__device__ __forceinline__ float2 x2_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 x2_add(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 x2_sub(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 x2_mul(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
struct df_ctx {
  df::Dims dm;
  df_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;
  // device buffers (complex arrays are double2 = interleaved re, im)
  double2* g = nullptr;        // [ne]
  double2* delta = nullptr;    // [ne]
  double2* gam = nullptr;      // [2][nb][n_w][n_w]  (channel 0 = d, 1 = m)
  double2* g0 = nullptr;       // [ne][N]  bare dual G0~(k)
  double2* gk = nullptr;       // [ne][N]  G~(k)
  double2* gr = nullptr;       // [ne][N]  G~(r)
  double2* chi = nullptr;      // [nb][n_w][N]
  double2* kc = nullptr;       // [2][nb][n_w][N] Eq. sd bracket per channel (weights 1, 3)
  double2* prod = nullptr;     // [nb][n_w][N] K(-r) G~_{w+W}(r)
  double2* sigma = nullptr;    // [n_w][N]
  double2* lat = nullptr;      // [2][n_w][N] lattice observables staged for host copies
  double2* sus = nullptr;      // susceptibility buffers, allocated by the first df_susceptibility
  double2* lam = nullptr;      // [2][nb][N] leading eigenvalue of gamma chi
  int* lam_ok = nullptr;       // [2][nb][N] power iteration converged flag
  double* red = nullptr;       // [2 n_w] residual partials, [2] final, [2] solve flags (ints)
  double* h_red = nullptr;     // pinned host mirror of the final residual
  void* bse_ws = nullptr;      // global scratch of the BSE kernel (large n)
  void* mixed_ws = nullptr;    // DF_FP32_IR: gamma as FP32 (hi, lo) pairs
  size_t tcr_off = 0;          // byte offset of the tensor-core residual's digits in mixed_ws (fixed at
                               // df_init: the hand-back list before it is sized for the full grid)
  int mixed_grid = 0;
  size_t bse_ws_bytes = 0;
  int bse_grid = 0;
  int iter_done = 0;
  int sigma_valid = 0;         // gk/gr reflect sigma
  double last_resid = -1.0;
  int radius_flag = 0;         // |lambda| >= 1 seen on the last df_bse
  // point-group reduction (opts.symmetry): orbit map, representatives and the compact arrays
  int n_orb = 0;
  int* qmap = nullptr;         // [N] orbit of each momentum
  int* qrep = nullptr;         // [n_orb] smallest momentum of each orbit
  double2* chi_w = nullptr;    // [nb][n_w][n_orb]
  double2* kc_w = nullptr;     // [2][nb][n_w][n_orb]
  double2* lam_w = nullptr;    // [2][nb][n_orb]
  int* lam_ok_w = nullptr;     // [2][nb][n_orb]
  unsigned long long* sym_chk = nullptr;   // [2] invariance check of df_set_sigma
  // per-kernel-group timing (df_set_timing)
  int timing = 0;
  struct Mark { int slot; int launches; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> event_pool;
  double t_ms[DF_T_COUNT] = {0, 0, 0, 0};
  int t_launches[DF_T_COUNT] = {0, 0, 0, 0};
};

// host-side launchers (kernels live in df_fft.cu and df_bse.cu)
namespace df {
cudaError_t launch_init_g0(df_ctx* c);
cudaError_t launch_wait_selftest(int arrive, unsigned spins, int* flags, cudaStream_t stream);
cudaError_t launch_dyson_ifft(df_ctx* c, int first_plane, int n_planes);
cudaError_t launch_bubble(df_ctx* c, int all_planes = 0);   // all_planes: every W even under the reflection
cudaError_t launch_sigma(df_ctx* c, double mix);
cudaError_t launch_sigma_partial(df_ctx* c, double2* out);
cudaError_t launch_sigma_finish(df_ctx* c, const double2* total, double mix);
cudaError_t launch_gamma_gt(df_ctx* c);
cudaError_t launch_bse(df_ctx* c, int channel_mask);
cudaError_t launch_lambda(df_ctx* c, int channel_mask);
size_t bse_workspace_bytes(const Dims& dm, int grid);
int bse_default_grid(const Dims& dm, int device);
int* bse_flags(df_ctx* c);   // [0]: bit 0 zero pivot, bit 1 |lambda| >= 1
// mixed precision (df_mixed.cu)
bool mixed_supported(int n_w);
size_t mixed_workspace_bytes(const Dims& dm);
cudaError_t launch_split_gamma(df_ctx* c, const double2* gg);
cudaError_t launch_lattice(df_ctx* c, double2* s_out, double2* g_out);
cudaError_t launch_obs_bubbles(df_ctx* c, double2* planes, double2* P, double2* L, double2* chi0);
cudaError_t launch_chi_ladder(df_ctx* c, const double2* Lb, const double2* chi0, double2* out, int* redo);
const double2* gamma_gt_ptr(df_ctx* c);   // gamma o gamma^T, written by launch_gamma_gt
cudaError_t launch_bse_mixed(df_ctx* c, int channel_mask, int* flags);
// orders 64 < n_w <= 128 (df_mixed_large.cu)
cudaError_t launch_bse_mixed_large(df_ctx* c, int channel_mask, int* flags);
MixedCheck mixed_check(df_ctx* c);
size_t mixed_tcr_offset(const Dims& dm);      // byte offset of the tensor-core residual's gamma digits
size_t tcr_workspace_bytes(const Dims& dm);
unsigned* mixed_check_words(df_ctx* c);   // [0] worst rho^2, [2] hand-back count, [3 ..] list
cudaError_t launch_bse_f64_list(df_ctx* c, const int* list);
cudaError_t launch_split_gamma_t(df_ctx* c);
// point-group reduction (df_sym.cu)
int build_wedge(int dim, int nk, std::vector<int>& qmap, std::vector<int>& qrep);
cudaError_t launch_wedge_gather(df_ctx* c, const Dims& ladder_dims);
cudaError_t launch_wedge_scatter(df_ctx* c, bool with_lambda);
cudaError_t launch_sigma_invariance(df_ctx* c, unsigned long long* out);
cudaError_t launch_chi_reflect(df_ctx* c);   // chi~ of W < 0 from W > 0 (df_opts.symmetry = 2)
}  // namespace df
