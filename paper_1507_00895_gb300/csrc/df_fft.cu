// Lattice-FFT kernels of the dual-fermion loop for one problem: bare dual
// propagator (Eq. gd0), Dyson + transform to real space (Eq. dyson), the
// dual bubble (Eq. dual_bubble) and the Schwinger-Dyson convolution
// (Eq. sd).
//
// Every momentum sum over the N = N_k^D grid is a cyclic correlation and is
// done exactly with D-dimensional FFTs held in shared memory: one CTA per
// (frequency, frequency) plane, N <= 4096 points (64 KB in complex128).
#include <math_constants.h>

#include "df_fft_dev.cuh"

namespace df {

__global__ void init_g0_kernel(Dims dm, const double2* __restrict__ g, const double2* __restrict__ delta,
                               double2* __restrict__ g0, double2* __restrict__ gk) {
  const int total = dm.ne * dm.N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x)
    init_g0_elem(dm, idx, g, delta, g0, gk);
}

__global__ void __launch_bounds__(kFftThreads)
dyson_ifft_kernel(Dims dm, int first, const double2* __restrict__ g0, const double2* __restrict__ sigma,
                  double2* __restrict__ gk, double2* __restrict__ gr) {
  extern __shared__ double2 sm[];
  dyson_ifft_plane(dm, first + blockIdx.x, g0, sigma, gk, gr, sm, sm + dm.nk / 2);
}

__global__ void __launch_bounds__(kFftThreads)
bubble_kernel(Dims dm, const double2* __restrict__ gr, double2* __restrict__ chi) {
  extern __shared__ double2 sm[];
  const int b = blockIdx.x / dm.n_w, i = blockIdx.x - b * dm.n_w, a = dm.a0 + b;
  bubble_plane(dm, a, i, gr, chi, sm, sm + dm.nk / 2);
}

__global__ void __launch_bounds__(kFftThreads)
sigma_prod_kernel(Dims dm, const double2* __restrict__ kc, const double2* __restrict__ gr,
                  double2* __restrict__ prod) {
  extern __shared__ double2 sm[];
  const int b = blockIdx.x / dm.n_w, i = blockIdx.x - b * dm.n_w, a = dm.a0 + b;
  sigma_prod_plane(dm, a, i, kc, gr, prod, sm, sm + dm.nk / 2);
}

__global__ void __launch_bounds__(kFftThreads)
sigma_dyson_kernel(Dims dm, double mix, const double2* __restrict__ prod, const double2* __restrict__ g0,
                   double2* __restrict__ sigma, double2* __restrict__ gk, double2* __restrict__ gr,
                   double* __restrict__ red, int refl) {
  extern __shared__ double2 sm[];
  __shared__ double red_sm[32];
  sigma_dyson_plane(dm, blockIdx.x, mix, prod, g0, sigma, gk, gr, red, sm, sm + dm.nk / 2,
                    sm + dm.nk / 2 + dm.N, red_sm, refl);
}

// The Omega split: this problem's share of Eq. sd, out[i][k] = (T/2) FFT[sum over
// its bosonic planes of prod[W][i]](k), before mixing and Dyson
__global__ void __launch_bounds__(kFftThreads)
sigma_partial_kernel(Dims dm, const double2* __restrict__ prod, double2* __restrict__ out, int refl) {
  extern __shared__ double2 sm[];
  const int i = blockIdx.x;
  double2* s = sm + dm.nk / 2;
  sigma_sum_plane(dm, i, prod, sm, s, refl);
  const double pref = 0.5 * dm.T;
  for (int k = threadIdx.x; k < dm.N; k += blockDim.x) out[(size_t)i * dm.N + k] = cscale(s[k], pref);
}

// ... and the rest of the pass from the sum of every share: mixing, residual
// partials, Eq. dyson, G~(r)
__global__ void __launch_bounds__(kFftThreads)
sigma_finish_kernel(Dims dm, double mix, const double2* __restrict__ total, const double2* __restrict__ g0,
                    double2* __restrict__ sigma, double2* __restrict__ gk, double2* __restrict__ gr,
                    double* __restrict__ red) {
  extern __shared__ double2 sm[];
  __shared__ double red_sm[32];
  const int i = blockIdx.x;
  double2* s = sm + dm.nk / 2;
  load_twiddles(sm, dm.nk);
  for (int k = threadIdx.x; k < dm.N; k += blockDim.x) s[k] = total[(size_t)i * dm.N + k];
  __syncthreads();
  sigma_finish_plane(dm, i, mix, 1.0, s, g0, sigma, gk, gr, red, sm, s + dm.N, red_sm);
}

// Section "Resulting observables", per box element (w, k): Eq. sigma_lat
// (denominator 1 + g Sigma~) and Eq. glat, with G~ from Eq. dyson.
__global__ void lattice_kernel(Dims dm, const double2* __restrict__ g, const double2* __restrict__ delta,
                               const double2* __restrict__ g0, const double2* __restrict__ sigma,
                               double2* __restrict__ s_out, double2* __restrict__ g_out) {
  const int total = dm.n_w * dm.N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int i = idx / dm.N, r = idx - i * dm.N, e = i + dm.m_max;
    const double2 ge = g[e], de = delta[e], st = sigma[idx];
    const double2 gi = cinv(ge);
    if (g_out) {
      const double eps = eps_of(r, dm.D, dm.p, dm.t, dm.tp);
      const double2 y = cinv(g0[(size_t)e * dm.N + r]);
      const double2 gt = cinv(mk(y.x - st.x, y.y - st.y));
      const double2 a = cinv(mk(de.x - eps, de.y));
      const double2 v = cmul(cmul(a, gi), cmul(gt, cmul(gi, a)));
      g_out[idx] = mk(a.x + v.x, a.y + v.y);
    }
    if (s_out) {
      const double2 den = cmul(ge, st);
      const double2 f = cmul(st, cinv(mk(1.0 + den.x, den.y)));
      const double w = (double)(2 * (i - dm.n_w / 2) + 1) * CUDART_PI * dm.T;
      s_out[idx] = mk(f.x + dm.mu - de.x - gi.x, f.y + w - de.y - gi.y);
    }
  }
}

// Planes of the susceptibilities (section "Resulting observables") on the
// extended grid: G (Eq. glat) and frakG = G~ (G0~ + g) / G0~, with G~ from
// Eq. dyson inside the box and G0~ outside.
__global__ void obs_planes_kernel(Dims dm, const double2* __restrict__ g, const double2* __restrict__ delta,
                                  const double2* __restrict__ g0, const double2* __restrict__ sigma,
                                  double2* __restrict__ Gk, double2* __restrict__ Fk) {
  const int total = dm.ne * dm.N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int e = idx / dm.N, r = idx - e * dm.N, i = e - dm.m_max;
    const double2 ge = g[e], de = delta[e], g0v = g0[idx];
    double2 gt = g0v;
    if (i >= 0 && i < dm.n_w) {
      const double2 y = cinv(g0v), st = sigma[(size_t)i * dm.N + r];
      gt = cinv(mk(y.x - st.x, y.y - st.y));
    }
    const double eps = eps_of(r, dm.D, dm.p, dm.t, dm.tp);
    const double2 a = cinv(mk(de.x - eps, de.y)), gi = cinv(ge);
    const double2 v = cmul(cmul(a, gi), cmul(gt, cmul(gi, a)));
    Gk[idx] = mk(a.x + v.x, a.y + v.y);
    Fk[idx] = cmul(gt, cmul(mk(g0v.x + ge.x, g0v.y + ge.y), cinv(g0v)));
  }
}

// chi0[a][q] = sum_i P[a][i][q] (the bare term's sum over the box frequencies)
__global__ void sum_w_kernel(Dims dm, const double2* __restrict__ P, double2* __restrict__ chi0) {
  const int total = dm.nb * dm.N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int a = idx / dm.N, q = idx - a * dm.N;
    double2 s = mk(0.0, 0.0);
    for (int i = 0; i < dm.n_w; ++i) {
      const double2 v = P[((size_t)a * dm.n_w + i) * dm.N + q];
      s = mk(s.x + v.x, s.y + v.y);
    }
    chi0[idx] = s;
  }
}

__global__ void residual_reduce_kernel(int n, double* red) {
  __shared__ double red_sm[32];
  residual_reduce_block(n, red, red_sm);
}

static size_t fft_smem(const Dims& dm, int planes) { return fft_smem_bytes(dm.nk, dm.N, planes); }

static cudaError_t set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_init_g0(df_ctx* c) {
  const Dims& dm = c->dm;
  const int total = dm.ne * dm.N;
  const int blocks = (total + 255) / 256;
  init_g0_kernel<<<blocks, 256, 0, c->stream>>>(dm, c->g, c->delta, c->g0, c->gk);
  return cudaGetLastError();
}

cudaError_t launch_dyson_ifft(df_ctx* c, int first_plane, int n_planes) {
  const Dims& dm = c->dm;
  const size_t sm = fft_smem(dm, 1);
  cudaError_t e = set_smem((const void*)dyson_ifft_kernel, sm);
  if (e != cudaSuccess) return e;
  dyson_ifft_kernel<<<n_planes, kFftThreads, sm, c->stream>>>(dm, first_plane, c->g0, c->sigma, c->gk, c->gr);
  return cudaGetLastError();
}

// The planes the pass needs: with the frequency reflection (df_opts.symmetry = 2)
// only W >= 0 (the ladder stage reads those; chi~ of W < 0 is their reflection).
static Dims pass_planes(const df_ctx* c) {
  Dims d = c->dm;
  if (c->opts.symmetry == 2) {
    d.a0 = d.m_max;
    d.na = d.m_max + 1;
  }
  return d;
}

cudaError_t launch_bubble(df_ctx* c, int all_planes) {
  const Dims dm = all_planes ? c->dm : pass_planes(c);
  const size_t sm = fft_smem(dm, 1);
  cudaError_t e = set_smem((const void*)bubble_kernel, sm);
  if (e != cudaSuccess) return e;
  bubble_kernel<<<dm.na * dm.n_w, kFftThreads, sm, c->stream>>>(dm, c->gr, c->chi);
  return cudaGetLastError();
}

cudaError_t launch_lattice(df_ctx* c, double2* s_out, double2* g_out) {
  const Dims& dm = c->dm;
  const int total = dm.n_w * dm.N;
  lattice_kernel<<<(total + 255) / 256, 256, 0, c->stream>>>(dm, c->g, c->delta, c->g0, c->sigma, s_out, g_out);
  return cudaGetLastError();
}

// The lattice parts of the susceptibilities: G and frakG planes (planes[0..1],
// k space), to real space (planes[2..3]), their bubbles; writes
// L [N_W][n_w][N] and chi0 [N_W][N], P [N_W][n_w][N] is scratch.
cudaError_t launch_obs_bubbles(df_ctx* c, double2* planes, double2* P, double2* L, double2* chi0) {
  const Dims& dm = c->dm;
  const size_t plane = (size_t)dm.ne * dm.N;
  double2* Gp = planes;
  double2* Fp = planes + plane;
  double2* Gr = planes + 2 * plane;
  double2* Fr = planes + 3 * plane;
  const int total = dm.ne * dm.N;
  obs_planes_kernel<<<(total + 255) / 256, 256, 0, c->stream>>>(dm, c->g, c->delta, c->g0, c->sigma, Gp, Fp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  size_t sm = fft_smem(dm, 1);
  if ((e = set_smem((const void*)dyson_ifft_kernel, sm)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)bubble_kernel, sm)) != cudaSuccess) return e;
  dyson_ifft_kernel<<<dm.ne, kFftThreads, sm, c->stream>>>(dm, 0, Gp, nullptr, nullptr, Gr);
  dyson_ifft_kernel<<<dm.ne, kFftThreads, sm, c->stream>>>(dm, 0, Fp, nullptr, nullptr, Fr);
  bubble_kernel<<<dm.nb * dm.n_w, kFftThreads, sm, c->stream>>>(dm, Gr, P);
  bubble_kernel<<<dm.nb * dm.n_w, kFftThreads, sm, c->stream>>>(dm, Fr, L);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nq = dm.nb * dm.N;
  sum_w_kernel<<<(nq + 255) / 256, 256, 0, c->stream>>>(dm, P, chi0);
  return cudaGetLastError();
}

// the Omega split: this problem's planes of Eq. sd into out [n_w][N] (device)
cudaError_t launch_sigma_partial(df_ctx* c, double2* out) {
  const Dims& dm = c->dm;
  const Dims pp = pass_planes(c);
  size_t sm = fft_smem(dm, 1);
  cudaError_t e = set_smem((const void*)sigma_prod_kernel, sm);
  if (e != cudaSuccess) return e;
  sigma_prod_kernel<<<pp.na * pp.n_w, kFftThreads, sm, c->stream>>>(pp, c->kc, c->gr, c->prod);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = set_smem((const void*)sigma_partial_kernel, sm)) != cudaSuccess) return e;
  sigma_partial_kernel<<<dm.n_w, kFftThreads, sm, c->stream>>>(dm, c->prod, out, c->opts.symmetry == 2);
  return cudaGetLastError();
}

// ... and the rest of the pass from the summed shares total [n_w][N] (device)
cudaError_t launch_sigma_finish(df_ctx* c, const double2* total, double mix) {
  const Dims& dm = c->dm;
  const size_t sm = fft_smem(dm, 2);
  cudaError_t e = set_smem((const void*)sigma_finish_kernel, sm);
  if (e != cudaSuccess) return e;
  sigma_finish_kernel<<<dm.n_w, kFftThreads, sm, c->stream>>>(dm, mix, total, c->g0, c->sigma, c->gk, c->gr, c->red);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  residual_reduce_kernel<<<1, kFftThreads, 0, c->stream>>>(dm.n_w, c->red);
  return cudaGetLastError();
}

cudaError_t launch_sigma(df_ctx* c, double mix) {
  const Dims& dm = c->dm;
  const Dims pp = pass_planes(c);
  size_t sm = fft_smem(dm, 1);
  cudaError_t e = set_smem((const void*)sigma_prod_kernel, sm);
  if (e != cudaSuccess) return e;
  sigma_prod_kernel<<<pp.na * pp.n_w, kFftThreads, sm, c->stream>>>(pp, c->kc, c->gr, c->prod);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  sm = fft_smem(dm, 2);
  if ((e = set_smem((const void*)sigma_dyson_kernel, sm)) != cudaSuccess) return e;
  sigma_dyson_kernel<<<dm.n_w, kFftThreads, sm, c->stream>>>(dm, mix, c->prod, c->g0, c->sigma, c->gk,
                                                             c->gr, c->red, c->opts.symmetry == 2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  residual_reduce_kernel<<<1, kFftThreads, 0, c->stream>>>(dm.n_w, c->red);
  return cudaGetLastError();
}

}  // namespace df
