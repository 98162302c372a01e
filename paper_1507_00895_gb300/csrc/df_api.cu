// C ABI of libdf (include/df.h): handle, validation, buffers and the
// sequence of launches of one pass of the ladder dual-fermion loop.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "df_internal.cuh"

namespace df {
int* bse_flags(df_ctx* c) { return (int*)(c->red + 2 * c->dm.n_w + 2); }
}  // namespace df

using namespace df;

namespace {

df_status fail(df_ctx* c, df_status s, const char* what, cudaError_t e = cudaSuccess) {
  if (c) {
    char buf[512];
    if (e != cudaSuccess)
      snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    else
      snprintf(buf, sizeof buf, "%s", what);
    c->err = buf;
  }
  return s;
}

#define DF_CUDA(c, call, what)                                                          \
  do {                                                                                  \
    cudaError_t e__ = (call);                                                           \
    if (e__ != cudaSuccess)                                                             \
      return fail((c), e__ == cudaErrorMemoryAllocation ? DF_ERR_OOM : DF_ERR_CUDA, (what), e__); \
  } while (0)

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

cudaMemcpyKind kind_to_dev(int is_device) {
  return is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_from_dev(int is_device) {
  return is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

df_status copy_out(df_ctx* c, void* dst, const void* src, size_t bytes, int is_device, const char* what) {
  if (!c) return DF_ERR_ARG;
  if (!dst) return fail(c, DF_ERR_ARG, "output pointer is NULL");
  DF_CUDA(c, cudaMemcpyAsync(dst, src, bytes, kind_from_dev(is_device), c->stream), what);
  if (!is_device) DF_CUDA(c, cudaStreamSynchronize(c->stream), what);
  return DF_OK;
}

// The conditions of the frequency reflection (df_opts.symmetry = 2) on the
// inputs: g(-w) = g(w)*, Delta(-w) = Delta(w)* on the extended grid (index
// e -> n_e - 1 - e) and gamma(-W; w, w') = gamma(W; -w, -w')* for both
// channels, each within 1e-12 of its array's largest |re| + |im|.
df_status check_reflection(df_ctx* c, const double* g, const double* delta, const double* gd, const double* gm,
                           int is_device) {
  const Dims& dm = c->dm;
  const size_t nv = (size_t)dm.nb * dm.n_w * dm.n_w;
  auto host = [&](const double* p, size_t count, std::vector<double2>& v) -> cudaError_t {
    v.resize(count);
    if (!is_device) {
      memcpy(v.data(), p, sizeof(double2) * count);
      return cudaSuccess;
    }
    cudaError_t e = cudaMemcpyAsync(v.data(), p, sizeof(double2) * count, cudaMemcpyDeviceToHost, c->stream);
    return e == cudaSuccess ? cudaStreamSynchronize(c->stream) : e;
  };
  auto mag = [](double2 z) { return fabs(z.x) + fabs(z.y); };
  auto dconj = [](double2 a, double2 b) { return fabs(a.x - b.x) + fabs(a.y + b.y); };   // |a - b*|
  std::vector<double2> v;
  const double* vec[2] = {g, delta};
  for (const double* p : vec) {
    DF_CUDA(c, host(p, dm.ne, v), "read inputs for the reflection check");
    double top = 0.0, dev = 0.0;
    for (int e = 0; e < dm.ne; ++e) {
      top = std::max(top, mag(v[e]));
      dev = std::max(dev, dconj(v[e], v[dm.ne - 1 - e]));
    }
    if (!(dev <= 1e-12 * top)) return fail(c, DF_ERR_ARG, "g or Delta breaks g(-w) = g(w)* (df_opts.symmetry = 2)");
  }
  const double* mats[2] = {gd, gm};
  const int n = dm.n_w;
  for (const double* p : mats) {
    DF_CUDA(c, host(p, nv, v), "read gamma for the reflection check");
    double top = 0.0, dev = 0.0;
    for (int a = 0; a < dm.nb; ++a)
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          const double2 x = v[((size_t)a * n + i) * n + j];
          const double2 y = v[((size_t)(dm.nb - 1 - a) * n + (n - 1 - i)) * n + (n - 1 - j)];
          top = std::max(top, mag(x));
          dev = std::max(dev, dconj(x, y));
        }
    if (!(dev <= 1e-12 * top))
      return fail(c, DF_ERR_ARG, "gamma breaks gamma(-W;w,w') = gamma(W;-w,-w')* (df_opts.symmetry = 2)");
  }
  return DF_OK;
}

df_status upload_inputs(df_ctx* c, const double* g, const double* delta, const double* gd, const double* gm,
                        int is_device) {
  const Dims& dm = c->dm;
  const size_t nv = (size_t)dm.nb * dm.n_w * dm.n_w;
  const cudaMemcpyKind k = kind_to_dev(is_device);
  DF_CUDA(c, cudaMemcpyAsync(c->g, g, sizeof(double2) * dm.ne, k, c->stream), "copy g");
  DF_CUDA(c, cudaMemcpyAsync(c->delta, delta, sizeof(double2) * dm.ne, k, c->stream), "copy delta");
  DF_CUDA(c, cudaMemcpyAsync(c->gam, gd, sizeof(double2) * nv, k, c->stream), "copy gamma_d");
  DF_CUDA(c, cudaMemcpyAsync(c->gam + nv, gm, sizeof(double2) * nv, k, c->stream), "copy gamma_m");
  DF_CUDA(c, launch_gamma_gt(c), "gamma o gamma^T");
  if (c->mixed_ws) DF_CUDA(c, launch_split_gamma(c, gamma_gt_ptr(c)), "gamma -> FP32 (hi, lo)");
  DF_CUDA(c, launch_init_g0(c), "bare dual propagator (Eq. gd0)");
  DF_CUDA(c, launch_dyson_ifft(c, 0, dm.ne), "Dyson + FFT to real space");
  return DF_OK;
}

cudaEvent_t take_event(df_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Records CUDA events around one kernel group when timing is on.
struct Timed {
  df_ctx* c;
  df_ctx::Mark m;
  Timed(df_ctx* c_, int slot, int launches) : c(c_) {
    m.slot = slot;
    m.launches = launches;
    m.a = m.b = nullptr;
    if (c->timing) {
      m.a = take_event(c);
      m.b = take_event(c);
      cudaEventRecord(m.a, c->stream);
    }
  }
  ~Timed() {
    if (m.a) {
      cudaEventRecord(m.b, c->stream);
      c->marks.push_back(m);
    }
  }
};

int n_channels(int mask) { return (mask & 1) + ((mask >> 1) & 1); }

cudaError_t run_bubble(df_ctx* c) {
  Timed t(c, DF_T_BUBBLE, 1);
  return launch_bubble(c);
}
cudaError_t run_bse(df_ctx* c, int mask) {
  Timed t(c, DF_T_BSE, n_channels(mask));
  return launch_bse(c, mask);
}
cudaError_t run_lambda(df_ctx* c, int mask) {
  if (c->opts.eig_mode == 0) return cudaSuccess;
  Timed t(c, DF_T_LAMBDA, n_channels(mask));
  return launch_lambda(c, mask);
}
// both ladder stages of a pass: the solves and the leading eigenvalue; with the
// radius extension the eigenvalue goes first (the solves read it)
cudaError_t run_ladders_on(df_ctx* c, int mask) {
  cudaError_t e;
  if (c->opts.radius_order > 0) {
    if ((e = run_lambda(c, mask)) != cudaSuccess) return e;
    return run_bse(c, mask);
  }
  if ((e = run_bse(c, mask)) != cudaSuccess) return e;
  return run_lambda(c, mask);
}
// With the point-group reduction the ladder kernels run on the compact
// arrays of the orbit representatives, seen as a grid of n_orb momenta.
// With the frequency reflection only the planes W >= 0 (a >= m_max) are in
// the view.
Dims wedge_dims(const df_ctx* c) {
  Dims d = c->dm;
  d.N = c->n_orb;
  if (c->opts.symmetry == 2) {
    d.a0 = d.m_max;
    d.na = d.m_max + 1;
  }
  return d;
}
struct WedgeView {
  df_ctx* c;
  Dims dm;
  double2 *chi, *kc, *lam;
  int* ok;
  explicit WedgeView(df_ctx* cc) : c(cc), dm(cc->dm), chi(cc->chi), kc(cc->kc), lam(cc->lam), ok(cc->lam_ok) {
    c->dm = wedge_dims(c);
    c->chi = c->chi_w;
    c->kc = c->kc_w;
    c->lam = c->lam_w;
    c->lam_ok = c->lam_ok_w;
  }
  ~WedgeView() {
    c->dm = dm;
    c->chi = chi;
    c->kc = kc;
    c->lam = lam;
    c->lam_ok = ok;
  }
};
cudaError_t run_ladders(df_ctx* c, int mask) {
  cudaError_t e = cudaMemsetAsync(bse_flags(c), 0, sizeof(int) * 4, c->stream);
  if (e != cudaSuccess) return e;
  // the mixed path's error-control words: worst rho^2 and the hand-back count
  if (c->mixed_ws && (e = cudaMemsetAsync(mixed_check_words(c), 0, sizeof(unsigned) * 4, c->stream)) != cudaSuccess)
    return e;
  if (!c->opts.symmetry) return run_ladders_on(c, mask);
  {
    Timed t(c, DF_T_BSE, 1);
    if ((e = launch_wedge_gather(c, wedge_dims(c))) != cudaSuccess) return e;
  }
  {
    WedgeView view(c);
    if ((e = run_ladders_on(c, mask)) != cudaSuccess) return e;
  }
  Timed t(c, DF_T_BSE, 1);
  return launch_wedge_scatter(c, c->opts.eig_mode != 0);
}
cudaError_t run_sigma(df_ctx* c) {
  Timed t(c, DF_T_SIGMA, 3);
  return launch_sigma(c, c->opts.mix);
}

df_status read_scalars(df_ctx* c, double* resid, int* flags) {
  // one 32-byte copy: residual max-norms and the solve flags
  double* h = c->h_red;
  DF_CUDA(c, cudaMemcpyAsync(h, c->red + 2 * c->dm.n_w, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
          "read residual");
  DF_CUDA(c, cudaStreamSynchronize(c->stream), "synchronise");
  if (resid) *resid = (h[1] > 0.0) ? h[0] / h[1] : 0.0;
  if (flags) memcpy(flags, h + 2, sizeof(int));
  return DF_OK;
}

}  // namespace

extern "C" {

df_status df_default_opts(df_opts* o) {
  if (!o) return DF_ERR_ARG;
  o->n_w = 0;
  o->m_max = 0;
  o->mix = 1.0;
  o->precision = DF_FP64;
  o->eig_mode = 1;
  o->ir_max_steps = 8;
  o->ir_tol = 1e-13;
  o->radius_order = 0;
  o->ladder_tol = 1e-9;
  o->ladder_fallback = 1;
  o->mixed_sweep = 0;
  o->w_lo = 0;
  o->w_hi = 0;
  o->symmetry = 0;
  return DF_OK;
}

const char* df_status_string(df_status s) {
  switch (s) {
    case DF_OK: return "DF_OK";
    case DF_ERR_ARG: return "DF_ERR_ARG";
    case DF_ERR_CUDA: return "DF_ERR_CUDA";
    case DF_ERR_OOM: return "DF_ERR_OOM";
    case DF_ERR_SINGULAR: return "DF_ERR_SINGULAR";
    case DF_ERR_REFINE_STALL: return "DF_ERR_REFINE_STALL";
    case DF_ERR_NOT_CONVERGED: return "DF_ERR_NOT_CONVERGED";
    case DF_ERR_TIMEOUT: return "DF_ERR_TIMEOUT";
    case DF_WARN_LADDER_RADIUS: return "DF_WARN_LADDER_RADIUS";
  }
  return "unknown df_status";
}

const char* df_last_error(const df_ctx* c) { return c ? c->err.c_str() : "NULL handle"; }

df_status df_vertex_from_spin(const double* uu, const double* ud, double* d, double* m, size_t count) {
  if (!uu || !ud || !d || !m) return DF_ERR_ARG;
  for (size_t i = 0; i < 2 * count; ++i) {
    const double a = uu[i], b = ud[i];
    d[i] = a + b;
    m[i] = a - b;
  }
  return DF_OK;
}

void df_destroy(df_ctx* c) {
  if (!c) return;
  cudaFree(c->g);
  cudaFree(c->delta);
  cudaFree(c->gam);
  cudaFree(c->g0);
  cudaFree(c->gk);
  cudaFree(c->gr);
  cudaFree(c->chi);
  cudaFree(c->kc);
  cudaFree(c->prod);
  cudaFree(c->sigma);
  cudaFree(c->lat);
  cudaFree(c->sus);
  cudaFree(c->lam);
  cudaFree(c->lam_ok);
  cudaFree(c->red);
  cudaFree(c->bse_ws);
  cudaFree(c->mixed_ws);
  cudaFree(c->qmap);
  cudaFree(c->qrep);
  cudaFree(c->chi_w);
  cudaFree(c->kc_w);
  cudaFree(c->lam_w);
  cudaFree(c->lam_ok_w);
  cudaFree(c->sym_chk);
  if (c->h_red) cudaFreeHost(c->h_red);
  for (auto& m : c->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  delete c;
}

df_status df_init(df_ctx** out, const df_lattice* lat, double beta, double mu, double t, const double* g,
                  const double* delta, const double* gamma_d, const double* gamma_m, const df_opts* opts,
                  void* stream) {
  if (!out || !lat || !opts || !g || !delta || !gamma_d || !gamma_m) return DF_ERR_ARG;
  *out = nullptr;
  if (lat->dim < 1 || lat->dim > 4 || !is_pow2(lat->nk) || lat->nk < 2 || lat->nk > 64) return DF_ERR_ARG;
  int N = 1;
  for (int d = 0; d < lat->dim; ++d) N *= lat->nk;
  if (N > 4096) return DF_ERR_ARG;
  if (lat->tp != 0.0 && lat->dim != 2) return DF_ERR_ARG;
  if (opts->n_w < 2 || opts->n_w > 128 || (opts->n_w & 1)) return DF_ERR_ARG;
  if (opts->m_max < 0 || opts->m_max > 31) return DF_ERR_ARG;
  if (!(beta > 0.0) || !(opts->mix > 0.0 && opts->mix <= 1.0)) return DF_ERR_ARG;
  if (opts->precision != DF_FP64 && opts->precision != DF_FP32_IR) return DF_ERR_ARG;
  if (opts->eig_mode < 0 || opts->eig_mode > 2) return DF_ERR_ARG;
  if (opts->radius_order < 0 || opts->radius_order > 16) return DF_ERR_ARG;
  if (opts->ir_max_steps < 1 || opts->ir_max_steps > 64 || !(opts->ir_tol > 0.0 && opts->ir_tol < 1.0))
    return DF_ERR_ARG;
  if (opts->radius_order > 0 && (opts->precision != DF_FP64 || opts->eig_mode != 2)) return DF_ERR_ARG;
  if (!(opts->ladder_tol > 0.0 && opts->ladder_tol < 1.0) || (opts->ladder_fallback != 0 && opts->ladder_fallback != 1))
    return DF_ERR_ARG;
  if (opts->mixed_sweep != 0 && opts->mixed_sweep != 1) return DF_ERR_ARG;
  if (opts->symmetry < 0 || opts->symmetry > 2) return DF_ERR_ARG;
  if (opts->symmetry == 2 && (opts->w_lo != 0 || opts->w_hi != 0)) return DF_ERR_ARG;   // needs both +-W
  {
    const int nbos = 2 * opts->m_max + 1;
    const bool full = opts->w_lo == 0 && opts->w_hi == 0;
    if (!full && !(opts->w_lo >= 0 && opts->w_lo < opts->w_hi && opts->w_hi <= nbos)) return DF_ERR_ARG;
  }
  if (opts->precision == DF_FP32_IR && !mixed_supported(opts->n_w)) {
    fprintf(stderr, "libdf: DF_FP32_IR supports n_w <= 128\n");
    return DF_ERR_ARG;
  }

  df_ctx* c = new (std::nothrow) df_ctx();
  if (!c) return DF_ERR_OOM;
  c->opts = *opts;
  c->stream = (cudaStream_t)stream;
  Dims& dm = c->dm;
  dm.D = lat->dim;
  dm.nk = lat->nk;
  dm.p = 0;
  while ((1 << dm.p) < lat->nk) ++dm.p;
  dm.N = N;
  dm.n_w = opts->n_w;
  dm.m_max = opts->m_max;
  dm.nb = 2 * opts->m_max + 1;
  dm.a0 = opts->w_lo;
  dm.na = (opts->w_hi > 0 ? opts->w_hi : dm.nb) - opts->w_lo;
  dm.ne = opts->n_w + 2 * opts->m_max;
  dm.beta = beta;
  dm.T = 1.0 / beta;
  dm.mu = mu;
  dm.t = t;
  dm.tp = lat->tp;

  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    df_status s = fail(c, DF_ERR_CUDA, "no CUDA device", e);
    fprintf(stderr, "libdf: %s\n", c->err.c_str());
    delete c;
    return s;
  }
  cudaGetDevice(&c->device);

  const size_t nplane = (size_t)dm.ne * dm.N;
  const size_t nv = (size_t)dm.nb * dm.n_w * dm.n_w;
  const size_t nchi = (size_t)dm.nb * dm.n_w * dm.N;
  df_status st = DF_OK;
#define ALLOC(ptr, count)                                                   \
  do {                                                                      \
    cudaError_t ea = dalloc(&(ptr), (count));                               \
    if (ea != cudaSuccess) { st = fail(c, DF_ERR_OOM, "cudaMalloc " #ptr, ea); goto bad; } \
  } while (0)
  ALLOC(c->g, dm.ne);
  ALLOC(c->delta, dm.ne);
  ALLOC(c->gam, 2 * nv);
  ALLOC(c->g0, nplane);
  ALLOC(c->gk, nplane);
  ALLOC(c->gr, nplane);
  ALLOC(c->chi, nchi);
  ALLOC(c->kc, 2 * nchi);
  ALLOC(c->prod, nchi);
  ALLOC(c->sigma, (size_t)dm.n_w * dm.N);
  ALLOC(c->lat, (size_t)2 * dm.n_w * dm.N);
  ALLOC(c->lam, (size_t)2 * dm.nb * dm.N);
  ALLOC(c->lam_ok, (size_t)2 * dm.nb * dm.N);
  ALLOC(c->red, (size_t)2 * dm.n_w + 4);
  if (opts->symmetry) {
    std::vector<int> qmap, qrep;
    c->n_orb = build_wedge(dm.D, dm.nk, qmap, qrep);
    const size_t nw = (size_t)c->n_orb;
    ALLOC(c->qmap, (size_t)dm.N);
    ALLOC(c->qrep, nw);
    ALLOC(c->chi_w, (size_t)dm.nb * dm.n_w * nw);
    ALLOC(c->kc_w, (size_t)2 * dm.nb * dm.n_w * nw);
    ALLOC(c->lam_w, (size_t)2 * dm.nb * nw);
    ALLOC(c->lam_ok_w, (size_t)2 * dm.nb * nw);
    ALLOC(c->sym_chk, 2);
    cudaError_t ea;
    if ((ea = cudaMemcpy(c->qmap, qmap.data(), sizeof(int) * dm.N, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ea = cudaMemcpy(c->qrep, qrep.data(), sizeof(int) * nw, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ea = cudaMemsetAsync(c->chi_w, 0, sizeof(double2) * dm.nb * dm.n_w * nw, c->stream)) != cudaSuccess ||
        (ea = cudaMemsetAsync(c->kc_w, 0, sizeof(double2) * 2 * dm.nb * dm.n_w * nw, c->stream)) != cudaSuccess ||
        (ea = cudaMemsetAsync(c->lam_w, 0, sizeof(double2) * 2 * dm.nb * nw, c->stream)) != cudaSuccess ||
        (ea = cudaMemsetAsync(c->lam_ok_w, 0xff, sizeof(int) * 2 * dm.nb * nw, c->stream)) != cudaSuccess) {
      st = fail(c, DF_ERR_CUDA, "point-group tables", ea);
      goto bad;
    }
  }
  c->bse_grid = bse_default_grid(dm, c->device);
  c->bse_ws_bytes = bse_workspace_bytes(dm, c->bse_grid);
  {
    cudaError_t ea = cudaMalloc(&c->bse_ws, c->bse_ws_bytes);
    if (ea != cudaSuccess) { st = fail(c, DF_ERR_OOM, "cudaMalloc bse workspace", ea); goto bad; }
    if (opts->precision == DF_FP32_IR) {
      c->tcr_off = mixed_tcr_offset(dm);
      ea = cudaMalloc(&c->mixed_ws, mixed_workspace_bytes(dm));
      if (ea != cudaSuccess) { st = fail(c, DF_ERR_OOM, "cudaMalloc mixed workspace", ea); goto bad; }
    }
    ea = cudaMallocHost((void**)&c->h_red, 4 * sizeof(double));
    if (ea != cudaSuccess) { st = fail(c, DF_ERR_OOM, "cudaMallocHost", ea); goto bad; }
  }
#undef ALLOC
  {
    cudaError_t ea;
    if ((ea = cudaMemsetAsync(c->sigma, 0, sizeof(double2) * dm.n_w * dm.N, c->stream)) != cudaSuccess ||
        (ea = cudaMemsetAsync(c->lam, 0, sizeof(double2) * 2 * dm.nb * dm.N, c->stream)) != cudaSuccess ||
        (ea = cudaMemsetAsync(c->lam_ok, 0xff, sizeof(int) * 2 * dm.nb * dm.N, c->stream)) != cudaSuccess ||
        (ea = cudaMemsetAsync(c->red, 0, sizeof(double) * (2 * dm.n_w + 4), c->stream)) != cudaSuccess ||
        (ea = cudaMemsetAsync(c->chi, 0, sizeof(double2) * nchi, c->stream)) != cudaSuccess ||
        (ea = cudaMemsetAsync(c->kc, 0, sizeof(double2) * 2 * nchi, c->stream)) != cudaSuccess) {
      st = fail(c, DF_ERR_CUDA, "cudaMemsetAsync", ea);
      goto bad;
    }
  }
  if (opts->symmetry == 2 && (st = check_reflection(c, g, delta, gamma_d, gamma_m, 0)) != DF_OK) goto bad;
  st = upload_inputs(c, g, delta, gamma_d, gamma_m, 0);
  if (st != DF_OK) goto bad;
  {
    cudaError_t ea = cudaStreamSynchronize(c->stream);
    if (ea != cudaSuccess) { st = fail(c, DF_ERR_CUDA, "df_init", ea); goto bad; }
  }
  *out = c;
  return DF_OK;
bad:
  fprintf(stderr, "libdf: df_init failed: %s\n", c->err.c_str());
  df_destroy(c);
  return st;
}

df_status df_set_inputs(df_ctx* c, const double* g, const double* delta, const double* gd, const double* gm,
                        int is_device) {
  if (!c) return DF_ERR_ARG;
  if (!g || !delta || !gd || !gm) return fail(c, DF_ERR_ARG, "NULL input");
  df_status s;
  if (c->opts.symmetry == 2 && (s = check_reflection(c, g, delta, gd, gm, is_device)) != DF_OK) return s;
  s = upload_inputs(c, g, delta, gd, gm, is_device);
  if (s != DF_OK) return s;
  if (!is_device) DF_CUDA(c, cudaStreamSynchronize(c->stream), "df_set_inputs");
  return DF_OK;
}

df_status df_bubble(df_ctx* c) {
  if (!c) return DF_ERR_ARG;
  DF_CUDA(c, run_bubble(c), "dual bubble (Eq. dual_bubble)");
  return DF_OK;
}

df_status df_bse(df_ctx* c, int channel_mask) {
  if (!c) return DF_ERR_ARG;
  if (channel_mask < 1 || channel_mask > 3) return fail(c, DF_ERR_ARG, "channel_mask must be 1, 2 or 3");
  DF_CUDA(c, run_ladders(c, channel_mask), "ladder solve (Eq. lin_alg_inv) and leading eigenvalue");
  return DF_OK;
}

// errors carried in the ladder kernels' flags word
static df_status flag_error(df_ctx* c, int flags) {
  if (flags & kFlagSingular) return fail(c, DF_ERR_SINGULAR, "exactly zero pivot in a ladder solve");
  if (flags & kFlagRefine)
    return fail(c, DF_ERR_REFINE_STALL,
                "a mixed-precision ladder's predicted error exceeded ladder_tol (ladder_fallback = 0)");
  if (flags & kFlagTcTimeout)
    return fail(c, DF_ERR_TIMEOUT, "a tensor-core completion wait in the mixed ladder kernel gave up");
  if (flags & kFlagTcLayout)
    return fail(c, DF_ERR_CUDA, "mixed ladder kernel: shared-memory operands not 1024-byte aligned");
  return DF_OK;
}

df_status df_selftest_wait(int arrive, int spins) {
  if (spins < 1) return DF_ERR_ARG;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return DF_ERR_CUDA;
  int h = 0;
  cudaError_t e = cudaMemset(d, 0, sizeof(int));
  if (e == cudaSuccess) e = df::launch_wait_selftest(arrive ? 1 : 0, (unsigned)spins, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return DF_ERR_CUDA;
  return (h & kFlagTcTimeout) ? DF_ERR_TIMEOUT : DF_OK;
}

static bool full_range(const df_ctx* c) { return c->dm.a0 == 0 && c->dm.na == c->dm.nb; }

// the end of a pass: the residual and the ladder flags of the pass, if asked for
static df_status finish_pass(df_ctx* c, double* resid) {
  ++c->iter_done;
  if (resid) {
    int flags = 0;
    df_status s = read_scalars(c, resid, &flags);
    if (s != DF_OK) return s;
    c->last_resid = *resid;
    if ((s = flag_error(c, flags)) != DF_OK) return s;
    if (flags & kFlagRadius) return DF_WARN_LADDER_RADIUS;
  }
  return DF_OK;
}

df_status df_sigma_partial(df_ctx* c, double* out, int is_device) {
  if (!c) return DF_ERR_ARG;
  if (!out) return fail(c, DF_ERR_ARG, "output pointer is NULL");
  const size_t bytes = sizeof(double2) * c->dm.n_w * c->dm.N;
  // host output: staged in the lattice-observables buffer
  double2* dst = is_device ? (double2*)out : c->lat;
  DF_CUDA(c, launch_sigma_partial(c, dst), "partial dual self-energy (Eq. sd over the handle's planes)");
  if (!is_device) return copy_out(c, out, c->lat, bytes, 0, "df_sigma_partial");
  return DF_OK;
}

df_status df_sigma_finish(df_ctx* c, const double* total, int is_device, double* resid) {
  if (!c) return DF_ERR_ARG;
  if (!total) return fail(c, DF_ERR_ARG, "input pointer is NULL");
  const size_t bytes = sizeof(double2) * c->dm.n_w * c->dm.N;
  const double2* src = (const double2*)total;
  if (!is_device) {
    DF_CUDA(c, cudaMemcpyAsync(c->lat, total, bytes, cudaMemcpyHostToDevice, c->stream), "df_sigma_finish");
    src = c->lat;
  }
  {
    Timed t(c, DF_T_SIGMA, 2);
    DF_CUDA(c, launch_sigma_finish(c, src, c->opts.mix), "mixing + Dyson (Eq. dyson) of the summed Eq. sd");
  }
  df_status s = finish_pass(c, resid);
  if (s == DF_OK && !is_device && !resid) DF_CUDA(c, cudaStreamSynchronize(c->stream), "df_sigma_finish");
  return s;
}

df_status df_get_ladder_stats(df_ctx* c, double* worst_rho2, int* handed_back) {
  if (!c) return DF_ERR_ARG;
  if (!c->mixed_ws) return fail(c, DF_ERR_ARG, "df_get_ladder_stats: the handle is not DF_FP32_IR");
  unsigned h[4] = {0, 0, 0, 0};
  DF_CUDA(c, cudaMemcpyAsync(h, mixed_check_words(c), sizeof h, cudaMemcpyDeviceToHost, c->stream), "ladder stats");
  DF_CUDA(c, cudaStreamSynchronize(c->stream), "ladder stats");
  float w;
  memcpy(&w, &h[0], sizeof w);
  if (worst_rho2) *worst_rho2 = (double)w;
  if (handed_back) *handed_back = c->opts.ladder_fallback ? (int)h[2] : 0;
  return DF_OK;
}

df_status df_sigma(df_ctx* c, double* resid) {
  if (!c) return DF_ERR_ARG;
  if (!full_range(c)) return fail(c, DF_ERR_ARG, "df_sigma needs the full bosonic range (use df_sigma_partial)");
  DF_CUDA(c, run_sigma(c), "dual self-energy (Eq. sd) + Dyson");
  return finish_pass(c, resid);
}

df_status df_iterate(df_ctx* c, int max_iter, double tol, int* iters_done, double* resid) {
  if (!c) return DF_ERR_ARG;
  if (max_iter < 0) return fail(c, DF_ERR_ARG, "max_iter < 0");
  if (!full_range(c)) return fail(c, DF_ERR_ARG, "df_iterate needs the full bosonic range");
  double r = -1.0;
  int it = 0, flags = 0;
  for (; it < max_iter; ++it) {
    DF_CUDA(c, run_bubble(c), "dual bubble (Eq. dual_bubble)");
    DF_CUDA(c, run_ladders(c, 3), "ladder solve (Eq. lin_alg_inv) and leading eigenvalue");
    DF_CUDA(c, run_sigma(c), "dual self-energy (Eq. sd) + Dyson");
    ++c->iter_done;
    if (tol > 0.0 || it == max_iter - 1) {
      df_status s = read_scalars(c, &r, &flags);
      if (s != DF_OK) return s;
      if ((s = flag_error(c, flags)) != DF_OK) {
        if (iters_done) *iters_done = it + 1;
        return s;
      }
      if (tol > 0.0 && r <= tol) {
        ++it;
        break;
      }
    }
  }
  if (iters_done) *iters_done = it;
  if (resid) *resid = r;
  c->last_resid = r;
  if (tol > 0.0 && !(r <= tol)) return DF_ERR_NOT_CONVERGED;
  if (flags & kFlagRadius) return DF_WARN_LADDER_RADIUS;
  return DF_OK;
}

df_status df_get_sigma(df_ctx* c, double* out, int is_device) {
  if (!c) return DF_ERR_ARG;
  return copy_out(c, out, c->sigma, sizeof(double2) * c->dm.n_w * c->dm.N, is_device, "df_get_sigma");
}

df_status df_set_sigma(df_ctx* c, const double* in, int is_device) {
  if (!c) return DF_ERR_ARG;
  if (!in) return fail(c, DF_ERR_ARG, "input pointer is NULL");
  DF_CUDA(c, cudaMemcpyAsync(c->sigma, in, sizeof(double2) * c->dm.n_w * c->dm.N, kind_to_dev(is_device), c->stream),
          "df_set_sigma");
  if (c->opts.symmetry) {
    // the reduction needs an invariant Sigma~: max deviation from the orbit representative
    unsigned long long h[2];
    DF_CUDA(c, launch_sigma_invariance(c, c->sym_chk), "point-group invariance of Sigma~");
    DF_CUDA(c, cudaMemcpyAsync(h, c->sym_chk, sizeof h, cudaMemcpyDeviceToHost, c->stream), "invariance check");
    DF_CUDA(c, cudaStreamSynchronize(c->stream), "invariance check");
    double dev, mag;
    memcpy(&dev, &h[0], sizeof dev);
    memcpy(&mag, &h[1], sizeof mag);
    if (!(dev <= 1e-12 * mag)) {
      DF_CUDA(c, cudaMemsetAsync(c->sigma, 0, sizeof(double2) * c->dm.n_w * c->dm.N, c->stream), "reset Sigma~");
      DF_CUDA(c, launch_dyson_ifft(c, c->dm.m_max, c->dm.n_w), "Dyson + FFT to real space");
      DF_CUDA(c, cudaStreamSynchronize(c->stream), "df_set_sigma");
      return fail(c, DF_ERR_ARG,
                  c->opts.symmetry == 2 ? "Sigma~ breaks the point group or Sigma~(-w) = Sigma~(w)* (df_opts.symmetry = 2)"
                                        : "Sigma~ is not invariant under the lattice's point group (df_opts.symmetry = 1)");
    }
  }
  DF_CUDA(c, launch_dyson_ifft(c, c->dm.m_max, c->dm.n_w), "Dyson + FFT to real space");
  if (!is_device) DF_CUDA(c, cudaStreamSynchronize(c->stream), "df_set_sigma");
  return DF_OK;
}

df_status df_lattice_observables(df_ctx* c, double* sigma_lat, double* g_lat, int is_device) {
  if (!c) return DF_ERR_ARG;
  const size_t cnt = (size_t)c->dm.n_w * c->dm.N;
  double2* so = is_device ? (double2*)sigma_lat : (sigma_lat ? c->lat : nullptr);
  double2* go = is_device ? (double2*)g_lat : (g_lat ? c->lat + cnt : nullptr);
  DF_CUDA(c, launch_lattice(c, so, go), "lattice observables (Eqs. sigma_lat, glat)");
  if (!is_device) {
    df_status s = DF_OK;
    if (sigma_lat) s = copy_out(c, sigma_lat, c->lat, sizeof(double2) * cnt, 0, "df_lattice_observables");
    if (s == DF_OK && g_lat) s = copy_out(c, g_lat, c->lat + cnt, sizeof(double2) * cnt, 0, "df_lattice_observables");
    return s;
  }
  return DF_OK;
}

df_status df_susceptibility(df_ctx* c, double* out, int is_device) {
  if (!c) return DF_ERR_ARG;
  if (!out) return fail(c, DF_ERR_ARG, "output pointer is NULL");
  if (!full_range(c)) return fail(c, DF_ERR_ARG, "df_susceptibility needs the full bosonic range");
  const Dims& dm = c->dm;
  const size_t plane = (size_t)dm.ne * dm.N, pw = (size_t)dm.nb * dm.n_w * dm.N, pq = (size_t)dm.nb * dm.N;
  if (!c->sus) {
    // the planes, P, L, chi0, the result, then the refinement's hand-back list
    const cudaError_t e =
        cudaMalloc((void**)&c->sus, sizeof(double2) * (4 * plane + 2 * pw + 3 * pq) + sizeof(int) * (2 * pq + 4));
    if (e != cudaSuccess) {
      c->sus = nullptr;
      return fail(c, DF_ERR_OOM, "susceptibility buffers", e);
    }
  }
  double2* planes = c->sus;
  double2* P = planes + 4 * plane;
  double2* L = P + pw;
  double2* chi0 = L + pw;
  double2* res = chi0 + pq;
  int* redo = (int*)(res + 2 * pq);
  DF_CUDA(c, launch_bubble(c, 1), "dual bubble (Eq. dual_bubble)");
  DF_CUDA(c, launch_obs_bubbles(c, planes, P, L, chi0), "susceptibility bubbles");
  DF_CUDA(c, cudaMemsetAsync(bse_flags(c), 0, sizeof(int) * 4, c->stream), "flags");
  DF_CUDA(c, launch_chi_ladder(c, L, chi0, is_device ? (double2*)out : res, redo), "susceptibility ladders");
  int fl[4] = {0, 0, 0, 0};
  DF_CUDA(c, cudaMemcpyAsync(fl, bse_flags(c), sizeof fl, cudaMemcpyDeviceToHost, c->stream), "flags");
  if (!is_device)
    DF_CUDA(c, cudaMemcpyAsync(out, res, sizeof(double2) * 2 * pq, cudaMemcpyDeviceToHost, c->stream), "copy out");
  DF_CUDA(c, cudaStreamSynchronize(c->stream), "df_susceptibility");
  if (fl[0] & kFlagSingular) return fail(c, DF_ERR_SINGULAR, "exactly zero pivot in a susceptibility ladder");
  return DF_OK;
}

df_status df_get_gtilde(df_ctx* c, double* out, int is_device) {
  if (!c) return DF_ERR_ARG;
  return copy_out(c, out, c->gk, sizeof(double2) * c->dm.ne * c->dm.N, is_device, "df_get_gtilde");
}

df_status df_get_chi(df_ctx* c, double* out, int is_device) {
  if (!c) return DF_ERR_ARG;
  if (c->opts.symmetry == 2) DF_CUDA(c, launch_chi_reflect(c), "chi~ of W < 0 by the frequency reflection");
  return copy_out(c, out, c->chi, sizeof(double2) * c->dm.nb * c->dm.n_w * c->dm.N, is_device, "df_get_chi");
}

df_status df_get_kernel(df_ctx* c, double* out, int is_device) {
  if (!c) return DF_ERR_ARG;
  return copy_out(c, out, c->kc, sizeof(double2) * 2 * c->dm.nb * c->dm.n_w * c->dm.N, is_device,
                  "df_get_kernel");
}

df_status df_get_lambda(df_ctx* c, double* lam, int* ok, int is_device) {
  if (!c) return DF_ERR_ARG;
  const size_t cnt = (size_t)2 * c->dm.nb * c->dm.N;
  df_status s = copy_out(c, lam, c->lam, sizeof(double2) * cnt, is_device, "df_get_lambda");
  if (s != DF_OK || !ok) return s;
  return copy_out(c, ok, c->lam_ok, sizeof(int) * cnt, is_device, "df_get_lambda");
}

df_status df_get_sizes(const df_ctx* c, int* n_ext, int* n_bos, int* n_k_total) {
  if (!c) return DF_ERR_ARG;
  if (n_ext) *n_ext = c->dm.ne;
  if (n_bos) *n_bos = c->dm.nb;
  if (n_k_total) *n_k_total = c->dm.N;
  return DF_OK;
}

df_status df_set_timing(df_ctx* c, int on) {
  if (!c) return DF_ERR_ARG;
  if (on) {
    for (auto& m : c->marks) {
      c->event_pool.push_back(m.a);
      c->event_pool.push_back(m.b);
    }
    c->marks.clear();
    for (int i = 0; i < DF_T_COUNT; ++i) {
      c->t_ms[i] = 0.0;
      c->t_launches[i] = 0;
    }
  }
  c->timing = on ? 1 : 0;
  return DF_OK;
}

df_status df_get_timing(df_ctx* c, double* ms, int* launches, int count) {
  if (!c) return DF_ERR_ARG;
  if (count < 0 || count > DF_T_COUNT) return fail(c, DF_ERR_ARG, "count out of range");
  DF_CUDA(c, cudaStreamSynchronize(c->stream), "df_get_timing");
  for (auto& m : c->marks) {
    float t = 0.f;
    DF_CUDA(c, cudaEventElapsedTime(&t, m.a, m.b), "cudaEventElapsedTime");
    c->t_ms[m.slot] += t;
    c->t_launches[m.slot] += m.launches;
    c->event_pool.push_back(m.a);
    c->event_pool.push_back(m.b);
  }
  c->marks.clear();
  for (int i = 0; i < count; ++i) {
    if (ms) ms[i] = c->t_ms[i];
    if (launches) launches[i] = c->t_launches[i];
  }
  return DF_OK;
}

df_status df_synchronize(df_ctx* c) {
  if (!c) return DF_ERR_ARG;
  DF_CUDA(c, cudaStreamSynchronize(c->stream), "df_synchronize");
  return DF_OK;
}

}  // extern "C"
