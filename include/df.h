/*
 * libdf: the ladder dual-fermion diagram summation of opendf
 * (Antipov, LeBlanc, Gull, arXiv:1507.00895), GB300 (sm_103a) CUDA.
 *
 * Plain C ABI: opaque handle, plain pointers and sizes, a status code from
 * every call.  All device work runs on the CUDA stream given to df_init
 * (NULL = the legacy default stream).  There is no CPU fallback: on a
 * machine without a usable sm_103a GPU, df_init returns DF_ERR_CUDA.
 *
 * Conventions shared by every call
 * --------------------------------
 * Complex numbers are two doubles (re, im), i.e. the layout of C99
 * `double _Complex` / `std::complex<double>`.
 *
 * Grids (Section "Ladder dual fermion self-consistency loop"):
 *   fermionic frequencies  w_n = (2n+1) pi/beta,  box n in [-n_w/2, n_w/2)
 *                          (box index i = n + n_w/2);
 *   bosonic frequencies    W_m = 2 m pi/beta,     m in [-m_max, m_max]
 *                          (index a = m + m_max, N_W = 2 m_max + 1);
 *   extended grid          n in [-n_w/2 - m_max, n_w/2 + m_max)
 *                          (index e = n + n_w/2 + m_max, n_e = n_w + 2 m_max),
 *                          so that w + W always lies on it;
 *   momenta                k_j = 2 pi x_j / N_k, x_j = 0..N_k-1, j = 1..D,
 *                          flattened with the last axis fastest, N = N_k^D.
 *
 * Array layouts (row-major, complex elements):
 *   g, delta       [n_e]               impurity g_w and hybridisation Delta_w
 *   gamma_d/_m     [N_W][n_w][n_w]     density / magnetic impurity vertex
 *                                      gamma_{W,w,w'} (Eq. spin_symm)
 *   sigma          [n_w][N]            dual self-energy Sigma~_{w,k}
 *   gtilde         [n_e][N]            dual Green's function G~_{w,k}
 *   chi            [N_W][n_w][N]       dual bubble chi~_{W,w}(q)
 *   kernel         [2][N_W][n_w][N]    per channel (0 = d, 1 = m) the bracket
 *                                      term of Eq. sd: c (Gamma_{W,w,w}(q)
 *                                      - Gamma^(2)_{W,w,w}(q)/2), c = 1 (d), 3 (m)
 *   lambda         [2][N_W][N]         leading eigenvalue of gamma chi~
 *
 * Ownership: inputs are copied at the call; the caller keeps its buffers.
 * Device buffers behind the handle are owned by it and freed by df_destroy.
 * A "_is_device" flag says whether a caller pointer is device memory
 * (written/read on the handle's stream, no host synchronisation) or host
 * memory (the call synchronises the stream before returning).
 *
 * Errors: DF_ERR_ARG for a NULL handle/pointer or an unsupported size (the
 * handle is unchanged); DF_ERR_CUDA / DF_ERR_OOM when a CUDA call fails
 * (the handle stays valid but its results are undefined until the next
 * successful df_set_sigma / df_init); df_last_error() returns the message.
 */
#ifndef LIBDF_DF_H
#define LIBDF_DF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct df_ctx df_ctx;

typedef enum df_status {
  DF_OK = 0,
  DF_ERR_ARG = 1,             /* bad argument or unsupported size */
  DF_ERR_CUDA = 2,            /* a CUDA call failed (no GPU, launch error, ...) */
  DF_ERR_OOM = 3,             /* device allocation failed */
  DF_ERR_SINGULAR = 4,        /* an exactly zero pivot in a ladder solve */
  DF_ERR_REFINE_STALL = 5,    /* mixed-precision refinement did not reach its tolerance */
  DF_ERR_NOT_CONVERGED = 6,   /* df_iterate stopped at max_iter above tol */
  DF_ERR_TIMEOUT = 7,         /* a bounded device-side wait gave up */
  DF_WARN_LADDER_RADIUS = 8   /* |leading eigenvalue of gamma chi~| >= 1 was seen: the
                                 ladder is outside its convergence radius (the paper's
                                 condition after Eq. lin_alg_inv); results are still
                                 produced by the direct solve */
} df_status;

typedef enum df_precision {
  DF_FP64 = 0,       /* every step in FP64 (complex128) */
  DF_FP32_IR = 1     /* ladder solves factorised in FP32 (complex64) and refined by
                        one correction with an extended-precision residual (n_w <= 64:
                        exact digit products on the tensor cores; 64 < n_w <= 128:
                        double-float).  Per ladder, rho = max|correction| / max|diag Gamma|
                        predicts the error left (~rho^2 of diag Gamma's largest entry);
                        a ladder with rho^2 > ladder_tol is solved again by the FP64 LU
                        (ladder_fallback = 1) or reported (DF_ERR_REFINE_STALL).  Bubble,
                        Sigma~, Dyson stay FP64.  The susceptibilities' ladders
                        (n_w <= 64) refine to ir_tol */
} df_precision;

/* Hypercubic lattice eps_k = -2t sum_j cos k_j (the paper's dispersion),
 * plus -4 tp cos k_1 cos k_2 for dim == 2.  nk must be a power of two in
 * [2, 64], dim in [1, 4], nk^dim <= 4096. */
typedef struct df_lattice {
  int dim;
  int nk;
  double tp;
} df_lattice;

typedef struct df_opts {
  int n_w;            /* fermionic box size (even, 2..128) */
  int m_max;          /* bosonic cutoff (0..31) */
  double mix;         /* Sigma~ <- mix * new + (1 - mix) * old, in (0, 1]; default 1 */
  int precision;      /* df_precision; default DF_FP64 */
  int eig_mode;       /* leading eigenvalue of gamma chi~: 0 off, 1 at W = 0 (default), 2 all W */
  int ir_max_steps;   /* DF_FP32_IR, susceptibility ladders: most FP32 solves per system before it is
                       * handed to the FP64 LU (default 8; 1..64) */
  double ir_tol;      /* DF_FP32_IR, susceptibility ladders: the refinement stops when the predicted
                       * error left, relative to max |re| + |im| of the solution, is below it
                       * (default 1e-13; in (0, 1)) */
  int radius_order;   /* the convergence-radius extension (the remark after Eq. lin_alg_inv): 0 off
                       * (default: Eq. lin_alg_inv is solved regardless and |lambda| >= 1 raises
                       * DF_WARN_LADDER_RADIUS); K >= 1: every (q, W, channel) whose leading
                       * eigenvalue of gamma chi~ has |lambda| >= 1 takes the low-order iterative
                       * evaluation Gamma <- gamma + gamma chi~ Gamma, K times from Gamma = gamma
                       * (the Neumann series to order K), the others the inversion; decided anew
                       * every pass.  K in [0, 16]; K >= 1 needs DF_FP64 and eig_mode 2. */
  double ladder_tol;  /* DF_FP32_IR: the per-ladder bound on the predicted error rho^2 (see
                       * DF_FP32_IR); default 1e-9, a tenth of the stated 1e-8; in (0, 1) */
  int ladder_fallback;/* DF_FP32_IR: 1 (default) a ladder above ladder_tol is solved again by
                       * the FP64 LU in the same df_bse; 0 its mixed result is kept and the
                       * next df_sigma / df_iterate returns DF_ERR_REFINE_STALL */
  int mixed_sweep;    /* DF_FP32_IR, orders 64 < n_w <= 128: the FP32 Gauss-Jordan inversion on the
                       * tensor cores (0, default: tcgen05 panel updates with three-piece BF16
                       * operands, FP32 accumulation in tensor memory) or on the CUDA cores (1) */
  int w_lo, w_hi;     /* the Omega split (several GPUs, one problem): this handle owns the
                       * bosonic planes a in [w_lo, w_hi) (index a = m + m_max); default 0, 0
                       * = all.  df_bubble and df_bse then cover only those planes and the
                       * pass ends with df_sigma_partial + (caller's sum over handles) +
                       * df_sigma_finish; df_sigma, df_iterate and df_susceptibility need
                       * the full range.  0 <= w_lo < w_hi <= N_W, or both 0. */
  int symmetry;       /* reductions of the ladder stage, exact for inputs with the stated
                       * symmetries.  0 (default): every (q, W, channel) is solved.
                       * 1: the point group -- one momentum per orbit of the lattice's
                       * point group (axis permutations and sign flips k_j -> -k_j: D4 on
                       * the square lattice, O_h on the cubic one; df_wedge lists the
                       * orbits) is solved and its diag Gamma, Eq. sd bracket and leading
                       * eigenvalue are copied to the orbit's other momenta.  Exact when
                       * G~(k) is invariant under the group, which holds for the input
                       * contract (local g, Delta and gamma; eps_k of df_lattice is
                       * invariant) whenever Sigma~ is: Sigma~ = 0 at df_init, and Eq. sd
                       * keeps it invariant.
                       * 2: the point group and the frequency reflection -- only the planes
                       * W >= 0 are solved; those of -W are their frequency-reversed complex
                       * conjugates (bracket_{-W}(w) = bracket_W(-w)*, lambda_{-W} =
                       * lambda_W*; of a dominant pair of equal moduli this may be the
                       * other member than a solve of -W reports).  Needs g(-w) = g(w)*, Delta(-w) = Delta(w)* and
                       * gamma(-W; w, w') = gamma(W; -w, -w')* (checked by df_init and
                       * df_set_inputs to 1e-12 of each array's largest entry: DF_ERR_ARG
                       * and nothing changed otherwise), Sigma~(-w) = Sigma~(w)* (kept by
                       * Eq. sd), and the full bosonic range (w_lo = w_hi = 0).
                       * With 1 or 2 df_set_sigma checks what it is given against the same
                       * symmetries (relative 1e-12 of max |Sigma~|) and rejects it with
                       * DF_ERR_ARG, Sigma~ reset to 0, otherwise.  The susceptibilities'
                       * ladders are not reduced. */
} df_opts;

/* Fill *o with the defaults above (n_w, m_max set to 0: the caller sets them). */
df_status df_default_opts(df_opts* o);

/* Create a handle and copy the inputs of the paper's input list (g_w,
 * Delta_w, mu and the two vertex channels).  Builds eps_k and the bare
 * dual propagator of Eq. gd0,
 *     G0~_{w,k} = [g_w^-1 + Delta_w - eps_k]^-1 - g_w,
 * on the extended grid, sets Sigma~ = 0 and G~ = G0~.
 * beta > 0; mu is kept for observables (the loop itself does not use it);
 * t is the hopping of eps_k.  g, delta, gamma_d, gamma_m are HOST pointers
 * with the layouts above.  stream is a cudaStream_t (may be NULL). */
df_status df_init(df_ctx** out, const df_lattice* lat, double beta, double mu, double t,
                  const double* g, const double* delta,
                  const double* gamma_d, const double* gamma_m,
                  const df_opts* opts, void* stream);

/* Replace g, delta and both vertex channels (same sizes as at df_init),
 * rebuild G0~ (Eq. gd0), keep Sigma~ and rebuild G~ from it (Eq. dyson).
 * Pointers are host memory unless is_device != 0. */
df_status df_set_inputs(df_ctx* c, const double* g, const double* delta,
                        const double* gamma_d, const double* gamma_m, int is_device);

/* Eq. spin_symm on the host: d = uu + ud, m = uu - ud, over `count` complex
 * elements.  Any of the output pointers may alias an input. */
df_status df_vertex_from_spin(const double* gamma_uu, const double* gamma_ud,
                              double* gamma_d, double* gamma_m, size_t count);

/* Eq. dual_bubble from the current G~:
 *     chi~_{W,w}(q) = -(T/N) sum_k G~_{w,k} G~_{w+W,k+q},
 * evaluated as -T sum_r G~_w(-r) G~_{w+W}(r) exp(-i q.r) with shared-memory
 * lattice FFTs; result kept on the device (df_get_chi). */
df_status df_bubble(df_ctx* c);

/* Eq. lin_alg_inv for every (q, W) and each channel in channel_mask
 * (bit 0 = d, bit 1 = m): (1 - gamma chi~) Gamma = gamma, solved by LU with
 * partial pivoting (in FP64, or FP32 + iterative refinement per
 * opts.precision); keeps c (Gamma_{W,w,w} - Gamma^(2)_{W,w,w}/2) with
 * Gamma^(2) = gamma chi~ gamma (the double-counting term of Eq. sd).  With
 * eig_mode != 0 also estimates the leading eigenvalue of gamma chi~ (FP64
 * power iteration).  Asynchronous: a zero pivot or |lambda| >= 1 is
 * recorded on the device and reported by the next df_sigma with a residual
 * pointer (DF_ERR_SINGULAR / DF_WARN_LADDER_RADIUS) or by df_iterate.
 * Needs df_bubble first. */
df_status df_bse(df_ctx* c, int channel_mask);

/* Eq. sd and Eq. dyson: from the ladder kernel and G~,
 *     Sigma~_{w,k} = T/(2N) sum_{W,q} [3(Gm - Gm2/2) + Gd - Gd2/2]_{W,w,w}(q) G~_{w+W,k+q},
 * mixed with the previous Sigma~, then G~ = 1/(1/G0~ - Sigma~) in the box.
 * If resid != NULL, synchronises and stores
 *     r = max|Sigma~_new - Sigma~_old| / max|Sigma~_new|. */
df_status df_sigma(df_ctx* c, double* resid);

/* The Omega split of Eq. sd.  Eq. sd's sum over (W, q) is a sum of independent
 * per-plane terms, so handles that own disjoint bosonic ranges (opts.w_lo,
 * w_hi; same inputs and Sigma~) can each run df_bubble and df_bse on their
 * planes and then:
 *   df_sigma_partial: out [n_w][N] complex = T/(2N) sum over this handle's W
 *                     and all q of [...] G~ (the bracket of Eq. sd), before
 *                     mixing and Dyson;
 *   (the caller sums the partials of all handles, e.g. an all-reduce)
 *   df_sigma_finish:  from the sum `total` [n_w][N]: mixing with the handle's
 *                     Sigma~, the residual, Eq. dyson and G~(r) for the next
 *                     pass, as the second half of df_sigma (resid as there).
 * Pointers are device memory when *_is_device != 0 (asynchronous on the
 * handle's stream), else host memory (the call synchronises).  On a
 * full-range handle df_sigma_partial + df_sigma_finish equals df_sigma up to
 * the rounding of the host round trip (none when the buffers are device
 * memory).  Errors: DF_ERR_ARG, DF_ERR_CUDA; df_sigma_finish with resid !=
 * NULL reports the ladder flags like df_sigma. */
df_status df_sigma_partial(df_ctx* c, double* out, int out_is_device);
df_status df_sigma_finish(df_ctx* c, const double* total, int in_is_device, double* resid);

/* Error control of the last df_bse under DF_FP32_IR: worst_rho2 = the
 * largest predicted error rho^2 over its ladders, handed_back = how many
 * were solved again by the FP64 LU (ladder_fallback = 1).  Synchronises.
 * DF_ERR_ARG under DF_FP64 (no mixed-precision ladders). */
df_status df_get_ladder_stats(df_ctx* c, double* worst_rho2, int* handed_back);

/* The self-consistency loop (the paper: repeat until G~ converges):
 * df_bubble, df_bse(both), df_sigma, up to max_iter times or until
 * r <= tol.  Returns DF_ERR_NOT_CONVERGED if tol > 0 was not reached,
 * DF_WARN_LADDER_RADIUS if the last pass saw |lambda| >= 1, else DF_OK.
 * iters_done and resid may be NULL. */
df_status df_iterate(df_ctx* c, int max_iter, double tol, int* iters_done, double* resid);

df_status df_get_sigma(df_ctx* c, double* out, int out_is_device);
df_status df_set_sigma(df_ctx* c, const double* in, int in_is_device);
df_status df_get_gtilde(df_ctx* c, double* out, int out_is_device);

/* Lattice observables of the current Sigma~ (section "Resulting observables"),
 * each [n_w][N] complex (the box frequencies, k flattened like Sigma~):
 *   Eq. sigma_lat: Sigma_lat = Sigma~ / (1 + g Sigma~) + Sigma^DMFT,
 *                  Sigma^DMFT = i w + mu - Delta - 1/g;
 *   Eq. glat:      G_lat = A + A g^-1 G~ g^-1 A,  A = (Delta - eps_k)^-1,
 *                  G~ = 1 / (1/G0~ - Sigma~) (Eq. gd0, Eq. dyson).
 * The printed Eq. sigma_lat has "1 - g Sigma" in the denominator; the sign
 * used is the one for which the two observables obey the Dyson relation
 * G_lat^-1 = i w + mu - eps_k - Sigma_lat that the paper states.  Either
 * output may be NULL.  Device outputs are written asynchronously on the
 * handle's stream; host outputs are complete on return.
 * Errors: DF_ERR_ARG (no handle), DF_ERR_CUDA. */
df_status df_lattice_observables(df_ctx* c, double* sigma_lat, double* g_lat, int out_is_device);

/* Charge and spin susceptibilities of the current Sigma~ (section "Resulting
 * observables"), out [2][N_W][N] complex (0: chi^ch with Gamma^d, 1: chi^sp
 * with Gamma^m):
 *   chi(W, q) = -(T/N) sum_{w,k} G_{w,k} G_{w+W,k+q}
 *             + sum_{w,w'} L_{W,w}(q) Gamma_{W,w,w'}(q) L_{W,w'}(q),
 *   L_{W,w}(q) = -(T/N) sum_k frakG_{w,k} frakG_{w+W,k+q},
 *   frakG = G~ (G0~ + g) / G0~,
 * G from Eq. glat, Gamma = (1 - gamma chi~)^-1 gamma (Eq. lin_alg_inv, FP64
 * LU with partial pivoting; under DF_FP32_IR an FP32 LU refined in FP64
 * until ir_tol, each system that does not get there within ir_max_steps
 * solves taken again by the FP64 LU) with chi~ the dual bubble of the current G~
 * (recomputed here; df_get_chi returns it afterwards), w over the box.  The
 * printed k sums lack 1/N; both carry it here (per-site normalisation).
 * Synchronous.  Errors: DF_ERR_ARG (no handle or NULL out), DF_ERR_OOM (the
 * first call allocates its buffers), DF_ERR_SINGULAR (an exactly zero pivot),
 * DF_ERR_CUDA. */
df_status df_susceptibility(df_ctx* c, double* out, int out_is_device);
df_status df_get_chi(df_ctx* c, double* out, int out_is_device);
df_status df_get_kernel(df_ctx* c, double* out, int out_is_device);
/* lambda [2][N_W][N] complex; ok [2][N_W][N] ints: 1 converged (to 1e-12),
 * 2 (n_w <= 64) the two largest moduli are equal (a complex-conjugate pair:
 * one power-iteration vector cannot settle) and lambda is the pair's member
 * of larger imaginary part, to FP32 accuracy (~1e-5 relative), 0 not
 * converged, -1 not computed (eig_mode).  ok may be NULL. */
df_status df_get_lambda(df_ctx* c, double* lambda, int* ok, int out_is_device);

/* Sizes of the handle: n_e, N_W, N (any pointer may be NULL). */
df_status df_get_sizes(const df_ctx* c, int* n_ext, int* n_bos, int* n_k_total);

/* Per-kernel device time (CUDA events recorded on the handle's stream
 * around each kernel group).  df_set_timing(c, 1) clears the totals and
 * starts recording, df_set_timing(c, 0) stops.  df_get_timing
 * synchronises and fills, for the first `count` groups, ms[i] = summed
 * device milliseconds and launches[i] = kernels launched (either pointer
 * may be NULL).  Groups: */
enum {
  DF_T_BUBBLE = 0,   /* Eq. dual_bubble: 1 kernel per df_bubble */
  DF_T_BSE = 1,      /* Eq. lin_alg_inv: counted as 1 kernel per channel (both channels may
                        * share one launch; the reductions' gather and scatter add 1 each) */
  DF_T_LAMBDA = 2,   /* leading eigenvalue: 1 kernel per channel (eig_mode != 0) */
  DF_T_SIGMA = 3,    /* Eq. sd + Eq. dyson + residual: 3 kernels per df_sigma */
  DF_T_COUNT = 4
};
df_status df_set_timing(df_ctx* c, int on);
df_status df_get_timing(df_ctx* c, double* ms, int* launches, int count);

/* Wait for all work queued on the handle's stream. */
df_status df_synchronize(df_ctx* c);

/* ---- batches of uneven parameter points ------------------------------------
 * The same loop for many independent points (lattice, beta, n_w, m_max may all
 * differ), run together: each stage of a pass is one launch over all points
 * (the FFT stages over every (point, plane), the FP64 ladders in one
 * persistent kernel with a cost-sorted atomic work queue, the mixed ladders
 * in one persistent launch per padded-order class), the pass is captured in
 * one CUDA graph and replayed, and points that reach tol stop being
 * updated.  Inputs per point as in df_init (host pointers). */
typedef struct df_point {
  int dim;
  int nk;
  double tp;
  double t;
  double beta;
  double mu;
  int n_w;
  int m_max;
  const double* g;        /* [n_w + 2 m_max] */
  const double* delta;    /* [n_w + 2 m_max] */
  const double* gamma_d;  /* [2 m_max + 1][n_w][n_w] */
  const double* gamma_m;
  int symmetry;           /* the reductions of df_opts.symmetry for this point (exact here:
                           * a batch always starts from Sigma~ = 0): 0 every ladder solved,
                           * 1 the point group, 2 also the frequency reflection (inputs
                           * checked as by df_init: DF_ERR_ARG if they lack it) */
} df_point;

typedef struct df_batch df_batch;

/* precision: DF_FP64 for every point, or DF_FP32_IR for every point (n_w <= 64
 * by the register-tile kernel, larger orders by the shared-memory Gauss-Jordan
 * one), with the per-ladder error control of DF_FP32_IR at ladder_tol = 1e-9:
 * ladders above it are solved again by the FP64 LU in the same pass.
 * npts in [1, 4096] (DF_FP32_IR: [1, 127]).  tol > 0: a point stops once its
 * residual r <= tol.  stream may be NULL (the batch then creates its own). */
df_status df_batch_init(df_batch** out, int npts, const df_point* pts, int precision, double mix, double tol,
                        void* stream);
/* Up to max_iter passes (graph replays); stops early when every point has
 * converged.  Per point: resid[i] (last residual), active[i] (1 = not yet
 * converged); either may be NULL.  DF_ERR_NOT_CONVERGED if a point is
 * still active at the end. */
df_status df_batch_iterate(df_batch* b, int max_iter, int* passes_done, double* resid, int* active);
df_status df_batch_get_sigma(df_batch* b, int point, double* out, int out_is_device);
/* Sigma~ = 0 and every point active again (G~ = G0~). */
df_status df_batch_reset(df_batch* b);
/* Times one pass for each candidate (FP64 right-hand-side chunk 8/16/32 or
 * the per-order default, scheduler chunk 1/4 systems), keeps the fastest,
 * appends it to cache_path (if not NULL) under the batch's size signature
 * and reads it from there next time.  Resets the batch (df_batch_reset).
 * chosen (may be NULL): [nc, chunk, 1 if read from the cache]. */
df_status df_batch_autotune(df_batch* b, const char* cache_path, int* chosen);
const char* df_batch_last_error(const df_batch* b);
void df_batch_destroy(df_batch* b);

/* ---- learned warm start -------------------------------------------------------
 * A dense network of 4 layers (n_in -> width -> width -> width -> n_out, tanh
 * between, linear output) that maps parameters and local inputs of a point
 * to its dual self-energy, evaluated and trained by libdf's own kernels:
 * every matrix product rounds its operands to BF16 and accumulates in FP32
 * on the tensor cores; weights, biases, Adam moments and activations are
 * FP32.  Weights are Glorot-uniform from `seed`, biases zero.  All data
 * pointers are device memory (row-major [batch][features]); batch <=
 * max_batch.  The paper has no counterpart (it starts from Sigma~ = 0). */
typedef struct df_mlp df_mlp;
df_status df_mlp_create(df_mlp** out, int n_in, int width, int n_out, int max_batch, unsigned long long seed,
                        void* stream);
df_status df_mlp_param_count(const df_mlp* m, long* count);
/* y[batch][n_out] = net(x[batch][n_in]) */
df_status df_mlp_forward(df_mlp* m, const float* x, int batch, float* y);
/* gradients of the mean squared error mean((net(x) - target)^2) with
 * respect to every parameter, kept inside the handle (df_mlp_grads);
 * loss_host (may be NULL) receives the loss (synchronises). */
df_status df_mlp_gradients(df_mlp* m, const float* x, const float* target, int batch, float* loss_host);
/* one Adam update from the stored gradients (bias-corrected). */
df_status df_mlp_adam_step(df_mlp* m, float lr, float beta1, float beta2, float eps);
/* df_mlp_gradients + df_mlp_adam_step(lr, 0.9, 0.999, 1e-8). */
df_status df_mlp_train_step(df_mlp* m, const float* x, const float* target, int batch, float lr, float* loss_host);
/* flat parameters [W1 (n_in x width, row-major) b1 W2 b2 W3 b3 W4 b4]: set != 0
 * copies buf into the network, else the network into buf. */
df_status df_mlp_params(df_mlp* m, float* buf, int set, int is_device);
df_status df_mlp_grads(df_mlp* m, float* buf, int is_device);
const char* df_mlp_last_error(const df_mlp* m);
void df_mlp_destroy(df_mlp* m);
/* Set the handle's Sigma~ from one network output y (device, [n_wedge][n_w/2][2]
 * floats: re, im at w_n >= 0 on the irreducible wedge), de-normalised as
 * y * sd + mean (same layout, device): Sigma~[i][r] = Y[kmap[r]][n] for
 * n = i - n_w/2 >= 0 and conj Y[kmap[r]][-n-1] for n < 0; kmap (device int
 * [N]) maps every momentum to its wedge representative.  Rebuilds G~
 * (Eq. dyson) like df_set_sigma; asynchronous. */
df_status df_warmstart_sigma(df_ctx* c, const float* y, const float* mean, const float* sd, const int* kmap);

/* Allocation-free variant of the FP64 ladder solves of df_bse (the paper
 * has no counterpart: this is a deployment form).  For callers that cannot
 * allocate device memory at the call, e.g. code inside a host application
 * that owns the whole device-memory budget, or a latency-critical loop that
 * cannot afford cudaMalloc's implicit synchronisation.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   gamma   device [2][n_bos][n_w][n_w] complex: gamma^d then gamma^m
 *   chi     device [n_bos][n_w][n_k_total] complex (df_get_chi's layout)
 *   kernel  device [2][n_bos][n_w][n_k_total] complex, written with
 *           df_get_kernel's content: c (Gamma_ww - Gamma^(2)_ww / 2)
 *   stream  cudaStream_t (may be NULL); the call is asynchronous on it.
 * Limits: n_w even in [2, 96], n_bos odd in [1, 63], n_k_total <= 4096 and
 * 2 n_bos n_w^2 <= 2^19; larger sizes return DF_ERR_ARG (message on stderr).
 * Its scratch is one fixed 8 MiB device array inside libdf, held by every
 * GPU that loads the library until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress), so it
 * should come before any stream capture.  All calls share the array and
 * the last call's contents stay in it: calls that overlap on the GPU (two
 * streams, or two host threads) race and must be serialised by the caller.
 * An exactly singular ladder matrix gives undefined values for that system
 * and is not reported (df_bse reports it).  It always solves Eq. lin_alg_inv
 * by the plain inverse: the convergence-radius extension (opts.radius_order
 * of a handle) is not applied, so ladders with |lambda| >= 1 differ from a
 * df_bse with radius_order > 0. */
df_status df_bse_noalloc(const double* gamma, const double* chi, int n_w, int n_bos, int n_k_total,
                         double* kernel, void* stream);

/* Self-test of the bounded device-side wait used by the tensor-core
 * residual of the mixed path (n_w 33-64): a one-warp kernel on the current
 * device initialises a shared-memory barrier, completes it only when
 * arrive != 0, and waits for it with a limit of `spins` polls.  Returns
 * DF_ERR_TIMEOUT when the wait gave up (arrive = 0), DF_OK when it saw the
 * barrier complete; the device stays usable either way.  Needs no handle.
 * Synchronous.  Errors: DF_ERR_ARG (spins < 1; no CUDA call is made),
 * DF_ERR_CUDA. */
df_status df_selftest_wait(int arrive, int spins);

/* Measured arithmetic peak of the current device, the denominator of the
 * ladder kernels' roofline fractions (the paper has no counterpart: this is
 * measurement support).  kind 0: FP32 fma.rn.f32, 1: FP32 packed
 * fma.rn.f32x2 (two multiply-adds per instruction), 2: FP64 fma.rn.f64.
 * Runs an FMA loop with 8 independent chains per thread over 8 blocks of
 * 256 threads per SM, best of 5 timed launches after one warm-up launch;
 * *gflops = 2 x multiply-adds / second / 1e9.  Synchronous, on the legacy
 * default stream.  Errors: DF_ERR_ARG (NULL gflops or kind out of range),
 * DF_ERR_OOM, DF_ERR_CUDA. */
df_status df_peak_probe(int kind, double* gflops);

/* The momentum orbits of the point group used by df_opts.symmetry (host only,
 * no device work).  For the grid nk^dim (flat index, last axis fastest;
 * dim, nk as in df_lattice) two momenta share an orbit when one maps to the
 * other by permuting axes and flipping signs k_j -> -k_j (mod nk): the
 * canonical form folds every coordinate to min(j, nk - j) and sorts them.
 * qmap [nk^dim] (caller-owned, may be NULL) receives each momentum's orbit
 * index; qrep [*n_orbits] (may be NULL; room for nk^dim entries) the
 * smallest flat index in each orbit; orbits are numbered in the order of
 * their qrep.  *n_orbits = C(nk/2 + dim, dim).  DF_ERR_ARG for sizes
 * df_lattice does not allow. */
df_status df_wedge(int dim, int nk, int* qmap, int* qrep, int* n_orbits);

const char* df_last_error(const df_ctx* c);
const char* df_status_string(df_status s);
void df_destroy(df_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* LIBDF_DF_H */
