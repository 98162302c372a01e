// Device bodies of the lattice-FFT stages (Eq. gd0, Eq. dyson,
// Eq. dual_bubble, Eq. sd), one (frequency, frequency) plane per CTA.  Used
// by the single-problem kernels (df_fft.cu) and by the batched ones
// (df_batch.cu).  Every function must be called by all threads of the block.
#pragma once
#include "df_internal.cuh"

namespace df {

constexpr int kFftThreads = 256;

__device__ __forceinline__ double eps_of(int r, int D, int p, double t, double tp) {
  const int mask = (1 << p) - 1;
  const double inv_nk = 1.0 / (double)(1 << p);
  double c[4] = {0, 0, 0, 0};
  double e = 0.0;
  for (int d = 0; d < D; ++d) {
    const int j = (r >> ((D - 1 - d) * p)) & mask;   // coordinate along axis d
    c[d] = cospi(2.0 * (double)j * inv_nk);
    e += c[d];
  }
  e *= -2.0 * t;
  if (D == 2) e -= 4.0 * tp * c[0] * c[1];
  return e;
}

// Eq. gd0 for one element idx = e N + r of the extended grid; G~ = G0~.
__device__ __forceinline__ void init_g0_elem(const Dims& dm, int idx, const double2* __restrict__ g,
                                             const double2* __restrict__ delta, double2* __restrict__ g0,
                                             double2* __restrict__ gk) {
  const int e = idx / dm.N, r = idx - e * dm.N;
  const double2 ge = g[e];
  const double eps = eps_of(r, dm.D, dm.p, dm.t, dm.tp);
  double2 den = cinv(ge) + delta[e];
  den.x -= eps;
  const double2 v = cinv(den) - ge;
  g0[idx] = v;
  gk[idx] = v;
}

// Plane e: G~(k) = Dyson(G0~, Sigma~) inside the box (G0~ outside), then
// G~(r) = (1/N) sum_k exp(ik.r) G~(k).  With sigma == nullptr the plane is
// transformed as given; with gk == nullptr the k-space copy is skipped.
__device__ __forceinline__ void dyson_ifft_plane(const Dims& dm, int e, const double2* __restrict__ g0,
                                                 const double2* __restrict__ sigma, double2* __restrict__ gk,
                                                 double2* __restrict__ gr, double2* tw, double2* s) {
  const int i = e - dm.m_max;        // box index or outside
  const bool in_box = (i >= 0 && i < dm.n_w);
  load_twiddles(tw, dm.nk);
  for (int r = threadIdx.x; r < dm.N; r += blockDim.x) {
    double2 v = g0[(size_t)e * dm.N + r];
    if (in_box && sigma) v = cinv(cinv(v) - sigma[(size_t)i * dm.N + r]);
    if (gk) gk[(size_t)e * dm.N + r] = v;
    s[bitrev_axes(r, dm.D, dm.p)] = v;
  }
  __syncthreads();
  fft_dit_smem(s, dm.D, dm.p, tw, true);
  const double invN = 1.0 / (double)dm.N;
  for (int r = threadIdx.x; r < dm.N; r += blockDim.x) gr[(size_t)e * dm.N + r] = cscale(s[r], invN);
  __syncthreads();
}

// Eq. dual_bubble for plane (a, i): chi~(q) = -T FFT[G~_w(-r) G~_{w+W}(r)](q).
__device__ __forceinline__ void bubble_plane(const Dims& dm, int a, int i, const double2* __restrict__ gr,
                                             double2* __restrict__ chi, double2* tw, double2* s) {
  const double2* A = gr + (size_t)(i + dm.m_max) * dm.N;   // G~_w
  const double2* B = gr + (size_t)(i + a) * dm.N;          // G~_{w+W}
  load_twiddles(tw, dm.nk);
  for (int r = threadIdx.x; r < dm.N; r += blockDim.x)
    s[bitrev_axes(r, dm.D, dm.p)] = cmul(A[reflect_index(r, dm.D, dm.p)], B[r]);
  __syncthreads();
  fft_dit_smem(s, dm.D, dm.p, tw, false);
  double2* out = chi + ((size_t)a * dm.n_w + i) * dm.N;
  for (int q = threadIdx.x; q < dm.N; q += blockDim.x) out[q] = cscale(s[q], -dm.T);
  __syncthreads();
}

// Eq. sd, stage 1, plane (a, i): K(r) = (1/N) sum_q exp(iq.r) K(q),
// K = kernel_d + kernel_m, then prod(r) = K(-r) G~_{w+W}(r).
__device__ __forceinline__ void sigma_prod_plane(const Dims& dm, int a, int i, const double2* __restrict__ kc,
                                                 const double2* __restrict__ gr, double2* __restrict__ prod,
                                                 double2* tw, double2* s) {
  const size_t plane = ((size_t)a * dm.n_w + i) * dm.N;
  const size_t chstride = (size_t)dm.nb * dm.n_w * dm.N;
  load_twiddles(tw, dm.nk);
  for (int q = threadIdx.x; q < dm.N; q += blockDim.x)
    s[bitrev_axes(q, dm.D, dm.p)] = kc[plane + q] + kc[chstride + plane + q];
  __syncthreads();
  fft_dit_smem(s, dm.D, dm.p, tw, true);
  const double invN = 1.0 / (double)dm.N;
  const double2* B = gr + (size_t)(i + a) * dm.N;
  for (int r = threadIdx.x; r < dm.N; r += blockDim.x)
    prod[plane + r] = cmul(cscale(s[reflect_index(r, dm.D, dm.p)], invN), B[r]);
  __syncthreads();
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* red_sm) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red_sm[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < NT / 32) ? red_sm[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) red_sm[0] = v;
  }
  __syncthreads();
  v = red_sm[0];
  __syncthreads();
  return v;
}

// Eq. sd, stage 2a, box frequency i: acc(r) = sum_W prod[W][i](r) over the
// problem's bosonic planes, s = FFT[acc] (natural order; the T/2 is applied by
// the caller).  Loads the twiddles into tw.
// With refl (the frequency reflection, full range) only the planes W >= 0 of
// prod are formed: the term of -W at w is that of W at -w, conjugated and taken
// at -r (prod_{-W,w}(r) = prod_{W,-w}(-r)*, from bracket_{-W}(w) = bracket_W(-w)*
// and G~(-w) = G~(w)*).
__device__ __forceinline__ void sigma_sum_plane(const Dims& dm, int i, const double2* __restrict__ prod, double2* tw,
                                                double2* s, int refl = 0) {
  load_twiddles(tw, dm.nk);
  const int ir = dm.n_w - 1 - i;
  for (int r = threadIdx.x; r < dm.N; r += blockDim.x) {
    double2 acc = mk(0.0, 0.0);
    if (refl) {
      const int rr = reflect_index(r, dm.D, dm.p);
      for (int a = dm.m_max; a < dm.nb; ++a) acc = acc + prod[((size_t)a * dm.n_w + i) * dm.N + r];
      for (int a = dm.m_max + 1; a < dm.nb; ++a) acc = acc + cconj(prod[((size_t)a * dm.n_w + ir) * dm.N + rr]);
    } else {
      for (int a = dm.a0; a < dm.a0 + dm.na; ++a) acc = acc + prod[((size_t)a * dm.n_w + i) * dm.N + r];
    }
    s[bitrev_axes(r, dm.D, dm.p)] = acc;
  }
  __syncthreads();
  fft_dit_smem(s, dm.D, dm.p, tw, false);
}

// Eq. sd, stage 2b, fused with mixing, the residual partials and Eq. dyson,
// for box frequency i: Sigma~_new(k) = pref s(k); Sigma~ <- mix new +
// (1-mix) old; G~ = 1/(1/G0~ - Sigma~); G~(r) = IFFT[G~(k)] / N.
// red[i], red[n_w + i] = max|dSigma~|, max|Sigma~|.  Needs the twiddles in tw.
__device__ __forceinline__ void sigma_finish_plane(const Dims& dm, int i, double mix, double pref, const double2* s,
                                                   const double2* __restrict__ g0, double2* __restrict__ sigma,
                                                   double2* __restrict__ gk, double2* __restrict__ gr,
                                                   double* __restrict__ red, const double2* tw, double2* s2,
                                                   double* red_sm) {
  const int e = i + dm.m_max;
  double dmax = 0.0, smax = 0.0;
  for (int k = threadIdx.x; k < dm.N; k += blockDim.x) {
    const size_t idx = (size_t)i * dm.N + k;
    const double2 old = sigma[idx];
    const double2 nw = cscale(s[k], pref);
    const double2 sg = mk(mix * nw.x + (1.0 - mix) * old.x, mix * nw.y + (1.0 - mix) * old.y);
    const double2 d = sg - old;
    dmax = fmax(dmax, sqrt(cabs2(d)));
    smax = fmax(smax, sqrt(cabs2(sg)));
    sigma[idx] = sg;
    const double2 gnew = cinv(cinv(g0[(size_t)e * dm.N + k]) - sg);
    gk[(size_t)e * dm.N + k] = gnew;
    s2[bitrev_axes(k, dm.D, dm.p)] = gnew;
  }
  dmax = block_max<kFftThreads>(dmax, red_sm);
  smax = block_max<kFftThreads>(smax, red_sm);
  if (threadIdx.x == 0) {
    red[i] = dmax;
    red[dm.n_w + i] = smax;
  }
  fft_dit_smem(s2, dm.D, dm.p, tw, true);
  const double invN = 1.0 / (double)dm.N;
  for (int r = threadIdx.x; r < dm.N; r += blockDim.x) gr[(size_t)e * dm.N + r] = cscale(s2[r], invN);
  __syncthreads();
}

// Eq. sd (stages 2a and 2b) for box frequency i: Sigma~_new = (T/2) FFT[sum_W prod]
__device__ __forceinline__ void sigma_dyson_plane(const Dims& dm, int i, double mix, const double2* __restrict__ prod,
                                                  const double2* __restrict__ g0, double2* __restrict__ sigma,
                                                  double2* __restrict__ gk, double2* __restrict__ gr,
                                                  double* __restrict__ red, double2* tw, double2* s, double2* s2,
                                                  double* red_sm, int refl = 0) {
  sigma_sum_plane(dm, i, prod, tw, s, refl);
  sigma_finish_plane(dm, i, mix, 0.5 * dm.T, s, g0, sigma, gk, gr, red, tw, s2, red_sm);
}

// max over red[0..n) and red[n..2n) into red[2n], red[2n+1] (one block)
__device__ __forceinline__ void residual_reduce_block(int n, double* red, double* red_sm) {
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    a = fmax(a, red[j]);
    b = fmax(b, red[n + j]);
  }
  a = block_max<kFftThreads>(a, red_sm);
  b = block_max<kFftThreads>(b, red_sm);
  if (threadIdx.x == 0) {
    red[2 * n] = a;
    red[2 * n + 1] = b;
  }
}

// shared memory of one FFT plane kernel: twiddles + `planes` lattice planes
__host__ __device__ inline size_t fft_smem_bytes(int nk, int N, int planes) {
  return sizeof(double2) * ((size_t)nk / 2 + (size_t)planes * N);
}

}  // namespace df
