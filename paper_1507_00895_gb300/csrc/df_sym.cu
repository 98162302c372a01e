// Point-group reduction of the ladder stage (df_opts.symmetry).  The ladder
// of (q, W, channel) depends on q only through the column chi~(q, W; .) of
// the bubble (Eq. dual_bubble), and chi~ inherits every symmetry R of G~:
// G~(Rk) = G~(k) for all k gives chi~(Rq) = chi~(q).  On the hypercubic
// grid the group is generated by axis permutations and sign flips, and
// eps_k (with t' on the square lattice) is invariant under it, so with
// local g, Delta, gamma and an invariant Sigma~, the solutions of Eq.
// lin_alg_inv, their Eq. sd brackets and the leading eigenvalues of gamma
// chi~ are equal across each momentum orbit.  The handle then solves one
// representative per orbit: chi~ is gathered into a compact [nb][n_w][n_orb]
// array, the unchanged ladder kernels run on it as on a grid of n_orb
// momenta, and the results are copied back to every momentum of the orbit.
//
// The frequency reflection (df_opts.symmetry = 2) halves the bosonic planes
// too.  With g(-w) = g(w)*, Delta(-w) = Delta(w)* and a real eps_k, G~(k,-w)
// = G~(k,w)* (Eqs. gd0 and dyson, given the same of Sigma~), so Eq.
// dual_bubble gives chi~(q,-W;w) = chi~(q,W;-w)*; with gamma(-W;w,w') =
// gamma(W;-w,-w')* the ladder matrix of -W is the frequency-reversed complex
// conjugate of that of W, and so are its solution, Gamma^(2), the bracket and
// the eigenvalues.  Only the planes W >= 0 are solved; index-wise W -> -W is
// a -> N_W - 1 - a and w -> -w is i -> n_w - 1 - i.
#include <algorithm>
#include <vector>

#include "df_internal.cuh"

namespace df {

// host: orbit index of every flat momentum and the smallest member of each orbit
int build_wedge(int dim, int nk, std::vector<int>& qmap, std::vector<int>& qrep) {
  int p = 0;
  while ((1 << p) < nk) ++p;
  const int N = 1 << (p * dim), h = nk / 2, base = h + 1;
  int cells = 1;
  for (int d = 0; d < dim; ++d) cells *= base;
  std::vector<int> slot(cells, -1);
  qmap.assign(N, 0);
  qrep.clear();
  for (int q = 0; q < N; ++q) {
    int a[4];
    for (int d = 0; d < dim; ++d) {
      const int j = (q >> ((dim - 1 - d) * p)) & (nk - 1);
      a[d] = std::min(j, nk - j);
    }
    std::sort(a, a + dim);
    int key = 0;
    for (int d = 0; d < dim; ++d) key = key * base + a[d];
    if (slot[key] < 0) {
      slot[key] = (int)qrep.size();
      qrep.push_back(q);
    }
    qmap[q] = slot[key];
  }
  return (int)qrep.size();
}

namespace {

// chi_w[a][i][o] = chi[a][i][qrep[o]] for the planes a in [a0, a0 + na) of dm
// (the ladder stage's planes; dm.N the full grid's momenta)
__global__ void wedge_gather_kernel(Dims dm, int n_orb, const int* __restrict__ qrep, const double2* __restrict__ chi,
                                    double2* __restrict__ chi_w) {
  const long total = (long)dm.na * dm.n_w * n_orb;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int o = (int)(idx % n_orb);
    const long row = (long)dm.a0 * dm.n_w + idx / n_orb;   // a * n_w + i
    chi_w[row * n_orb + o] = chi[row * dm.N + qrep[o]];
  }
}

// kc[c][a][i][q] = kc_w[c][a][i][qmap[q]] for a in the handle's range; the
// leading eigenvalue and its flag likewise ([c][a][q]) when lam_w is given
// (eigenvalues computed this pass).  With refl, the planes a < m_max are the
// reflections of a' = 2 m_max - a: kc_w[c][a'][n_w - 1 - i][o]*, lam_w[c][a'][o]*.
__global__ void wedge_scatter_kernel(Dims dm, int n_orb, int refl, const int* __restrict__ qmap,
                                     const double2* __restrict__ kc_w, double2* __restrict__ kc,
                                     const double2* __restrict__ lam_w, const int* __restrict__ ok_w,
                                     double2* __restrict__ lam, int* __restrict__ ok) {
  const long rows = 2L * dm.na * dm.n_w;                    // (c, a - a0, i)
  const long total = rows * dm.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx % dm.N);
    const long r = idx / dm.N;
    const int i = (int)(r % dm.n_w);
    const long ca = r / dm.n_w;
    const int c = (int)(ca / dm.na), a = dm.a0 + (int)(ca % dm.na);
    const bool mirror = refl && a < dm.m_max;
    const int as = mirror ? 2 * dm.m_max - a : a, is = mirror ? dm.n_w - 1 - i : i;
    const long row = ((long)c * dm.nb + a) * dm.n_w + i;
    const long srow = ((long)c * dm.nb + as) * dm.n_w + is;
    const int o = qmap[q];
    const double2 v = kc_w[srow * n_orb + o];
    kc[row * dm.N + q] = mirror ? make_double2(v.x, -v.y) : v;
    if (lam_w && i == 0) {
      const long lr = (long)c * dm.nb + a, ls = (long)c * dm.nb + as;
      const double2 l = lam_w[ls * n_orb + o];
      // the eigenvalues of -W are the conjugates of those of W (of a dominant pair
      // of equal moduli, flag 2, the reflection may report the other member than
      // the plane's own solve, whose tie-break is by imaginary part)
      lam[lr * dm.N + q] = mirror ? make_double2(l.x, -l.y) : l;
      ok[lr * dm.N + q] = ok_w[ls * n_orb + o];
    }
  }
}

// out[0] = max |sigma(k) - sigma(qrep[qmap[k]])| (with refl also
// max |sigma(w, k) - sigma(-w, k)*|), out[1] = max |sigma| (|re| + |im|;
// non-negative doubles order as their bit patterns)
__global__ void sigma_invariance_kernel(Dims dm, int refl, const int* __restrict__ qmap, const int* __restrict__ qrep,
                                        const double2* __restrict__ sigma, unsigned long long* __restrict__ out) {
  double dev = 0.0, mag = 0.0;
  const long total = (long)dm.n_w * dm.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx % dm.N);
    const long row = idx / dm.N;
    const double2 s = sigma[idx], r = sigma[row * dm.N + qrep[qmap[q]]];
    double d = fabs(s.x - r.x) + fabs(s.y - r.y);
    bool bad = !(d == d);                      // a NaN counts as an infinite deviation
    const double m = fabs(s.x) + fabs(s.y);
    if (refl) {
      const double2 t = sigma[(dm.n_w - 1 - row) * dm.N + q];
      const double d2 = fabs(s.x - t.x) + fabs(s.y + t.y);
      bad = bad || !(d2 == d2);
      d = fmax(d, d2);
    }
    if (bad) d = __longlong_as_double(0x7ff0000000000000LL);
    dev = fmax(dev, d);
    mag = fmax(mag, m);
  }
  for (int o = 16; o > 0; o >>= 1) {
    dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    mag = fmax(mag, __shfl_xor_sync(0xffffffffu, mag, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(dev));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(mag));
  }
}

// chi~ of the planes W < 0 (a < m_max), which the pass does not form under the
// frequency reflection: chi[a][i][q] = chi[2 m_max - a][n_w - 1 - i][q]*
__global__ void chi_reflect_kernel(Dims dm, double2* __restrict__ chi) {
  const long total = (long)dm.m_max * dm.n_w * dm.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx % dm.N);
    const long row = idx / dm.N;
    const int i = (int)(row % dm.n_w), a = (int)(row / dm.n_w);
    const double2 v = chi[(((size_t)(2 * dm.m_max - a)) * dm.n_w + (dm.n_w - 1 - i)) * dm.N + q];
    chi[idx] = make_double2(v.x, -v.y);
  }
}

int grid_for(long total) { return (int)std::min<long>(4096, (total + 255) / 256); }

}  // namespace

// the ladder stage's planes (ladder_dims.a0, .na) of the full-grid chi~ (c->dm)
cudaError_t launch_wedge_gather(df_ctx* c, const Dims& ladder_dims) {
  Dims dm = c->dm;
  dm.a0 = ladder_dims.a0;
  dm.na = ladder_dims.na;
  const long total = (long)dm.na * dm.n_w * c->n_orb;
  wedge_gather_kernel<<<grid_for(total), 256, 0, c->stream>>>(dm, c->n_orb, c->qrep, c->chi, c->chi_w);
  return cudaGetLastError();
}

cudaError_t launch_wedge_scatter(df_ctx* c, bool with_lambda) {
  const Dims& dm = c->dm;
  const long total = 2L * dm.na * dm.n_w * dm.N;
  wedge_scatter_kernel<<<grid_for(total), 256, 0, c->stream>>>(dm, c->n_orb, c->opts.symmetry == 2, c->qmap,
                                                               c->kc_w, c->kc,
                                                               with_lambda ? c->lam_w : nullptr,
                                                               with_lambda ? c->lam_ok_w : nullptr, c->lam, c->lam_ok);
  return cudaGetLastError();
}

cudaError_t launch_chi_reflect(df_ctx* c) {
  const Dims& dm = c->dm;
  const long total = (long)dm.m_max * dm.n_w * dm.N;
  if (total == 0) return cudaSuccess;
  chi_reflect_kernel<<<grid_for(total), 256, 0, c->stream>>>(dm, c->chi);
  return cudaGetLastError();
}

cudaError_t launch_sigma_invariance(df_ctx* c, unsigned long long* out) {
  const Dims& dm = c->dm;
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return e;
  sigma_invariance_kernel<<<grid_for((long)dm.n_w * dm.N), 256, 0, c->stream>>>(dm, c->opts.symmetry == 2, c->qmap,
                                                                                c->qrep, c->sigma, out);
  return cudaGetLastError();
}

}  // namespace df

extern "C" df_status df_wedge(int dim, int nk, int* qmap, int* qrep, int* n_orbits) {
  if (!n_orbits || dim < 1 || dim > 4 || nk < 2 || nk > 64 || (nk & (nk - 1))) return DF_ERR_ARG;
  long N = 1;
  for (int d = 0; d < dim; ++d) N *= nk;
  if (N > 4096) return DF_ERR_ARG;
  std::vector<int> m, r;
  *n_orbits = df::build_wedge(dim, nk, m, r);
  if (qmap) std::copy(m.begin(), m.end(), qmap);
  if (qrep) std::copy(r.begin(), r.end(), qrep);
  return DF_OK;
}
