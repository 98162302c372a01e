"""ctypes binding of libdf (include/df.h): argument marshalling only.

Every step of the ladder dual-fermion loop runs in the CUDA kernels of
``libdf.so``; this module converts numpy / torch arrays to pointers and
status codes to exceptions.  There is no fallback: if the library is
missing or no GPU is usable, loading or ``DualFermion(...)`` raises.

Complex arrays cross the boundary as complex128 (interleaved re, im).
Device arrays (torch CUDA tensors, complex128, contiguous) are passed
with ``is_device=1`` and never leave the GPU.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdf.so")

DF_OK = 0
DF_ERR_ARG = 1
DF_ERR_CUDA = 2
DF_ERR_OOM = 3
DF_ERR_SINGULAR = 4
DF_ERR_REFINE_STALL = 5
DF_ERR_NOT_CONVERGED = 6
DF_ERR_TIMEOUT = 7
DF_WARN_LADDER_RADIUS = 8

DF_FP64 = 0
DF_FP32_IR = 1

# every symbol include/df.h declares (checked by the CPU tests)
EXPORTS = (
    "df_default_opts", "df_init", "df_set_inputs", "df_vertex_from_spin", "df_bubble", "df_bse",
    "df_sigma", "df_sigma_partial", "df_sigma_finish", "df_get_ladder_stats", "df_iterate", "df_get_sigma", "df_set_sigma", "df_get_gtilde", "df_lattice_observables", "df_susceptibility", "df_get_chi",
    "df_get_kernel", "df_get_lambda", "df_get_sizes", "df_set_timing", "df_get_timing",
    "df_synchronize", "df_bse_noalloc", "df_batch_init", "df_batch_iterate", "df_batch_get_sigma",
    "df_batch_reset", "df_batch_autotune", "df_batch_last_error", "df_batch_destroy", "df_mlp_create",
    "df_mlp_param_count", "df_mlp_forward", "df_mlp_gradients", "df_mlp_adam_step", "df_mlp_train_step",
    "df_mlp_params", "df_mlp_grads", "df_mlp_last_error", "df_mlp_destroy", "df_warmstart_sigma", "df_last_error",
    "df_status_string", "df_destroy", "df_selftest_wait", "df_peak_probe", "df_wedge",
)


class DFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class df_lattice(C.Structure):
    _fields_ = [("dim", C.c_int), ("nk", C.c_int), ("tp", C.c_double)]


class df_point(C.Structure):
    _fields_ = [("dim", C.c_int), ("nk", C.c_int), ("tp", C.c_double), ("t", C.c_double),
                ("beta", C.c_double), ("mu", C.c_double), ("n_w", C.c_int), ("m_max", C.c_int),
                ("g", C.c_void_p), ("delta", C.c_void_p), ("gamma_d", C.c_void_p), ("gamma_m", C.c_void_p),
                ("symmetry", C.c_int)]


class df_opts(C.Structure):
    _fields_ = [("n_w", C.c_int), ("m_max", C.c_int), ("mix", C.c_double), ("precision", C.c_int),
                ("eig_mode", C.c_int), ("ir_max_steps", C.c_int), ("ir_tol", C.c_double),
                ("radius_order", C.c_int), ("ladder_tol", C.c_double), ("ladder_fallback", C.c_int),
                ("mixed_sweep", C.c_int), ("w_lo", C.c_int), ("w_hi", C.c_int), ("symmetry", C.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libdf.so (built by paper_1507_00895_gb300.build.build_lib)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdf.so not found at {path}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    P = C.c_void_p
    D = C.POINTER(C.c_double)
    I = C.POINTER(C.c_int)
    sig = {
        "df_default_opts": [C.POINTER(df_opts)],
        "df_init": [C.POINTER(P), C.POINTER(df_lattice), C.c_double, C.c_double, C.c_double,
                    P, P, P, P, C.POINTER(df_opts), P],
        "df_set_inputs": [P, P, P, P, P, C.c_int],
        "df_vertex_from_spin": [P, P, P, P, C.c_size_t],
        "df_bubble": [P],
        "df_bse": [P, C.c_int],
        "df_sigma": [P, D],
        "df_sigma_partial": [P, P, C.c_int],
        "df_sigma_finish": [P, P, C.c_int, D],
        "df_get_ladder_stats": [P, D, I],
        "df_iterate": [P, C.c_int, C.c_double, I, D],
        "df_get_sigma": [P, P, C.c_int],
        "df_set_sigma": [P, P, C.c_int],
        "df_get_gtilde": [P, P, C.c_int],
        "df_lattice_observables": [P, P, P, C.c_int],
        "df_susceptibility": [P, P, C.c_int],
        "df_get_chi": [P, P, C.c_int],
        "df_get_kernel": [P, P, C.c_int],
        "df_get_lambda": [P, P, P, C.c_int],
        "df_get_sizes": [P, I, I, I],
        "df_set_timing": [P, C.c_int],
        "df_get_timing": [P, D, I, C.c_int],
        "df_synchronize": [P],
        "df_bse_noalloc": [P, P, C.c_int, C.c_int, C.c_int, P, P],
        "df_selftest_wait": [C.c_int, C.c_int],
        "df_peak_probe": [C.c_int, D],
        "df_wedge": [C.c_int, C.c_int, P, P, I],
        "df_batch_init": [C.POINTER(P), C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_double, P],
        "df_batch_iterate": [P, C.c_int, I, D, I],
        "df_batch_get_sigma": [P, C.c_int, P, C.c_int],
        "df_batch_reset": [P],
        "df_batch_autotune": [P, C.c_char_p, I],
        "df_mlp_create": [C.POINTER(P), C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong, P],
        "df_mlp_param_count": [P, C.POINTER(C.c_long)],
        "df_mlp_forward": [P, P, C.c_int, P],
        "df_mlp_gradients": [P, P, P, C.c_int, C.POINTER(C.c_float)],
        "df_mlp_adam_step": [P, C.c_float, C.c_float, C.c_float, C.c_float],
        "df_mlp_train_step": [P, P, P, C.c_int, C.c_float, C.POINTER(C.c_float)],
        "df_mlp_params": [P, P, C.c_int, C.c_int],
        "df_mlp_grads": [P, P, C.c_int],
        "df_warmstart_sigma": [P, P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.df_last_error.argtypes = [P]
    lib.df_last_error.restype = C.c_char_p
    lib.df_status_string.argtypes = [C.c_int]
    lib.df_status_string.restype = C.c_char_p
    lib.df_destroy.argtypes = [P]
    lib.df_destroy.restype = None
    lib.df_batch_last_error.argtypes = [P]
    lib.df_batch_last_error.restype = C.c_char_p
    lib.df_batch_destroy.argtypes = [P]
    lib.df_batch_destroy.restype = None
    lib.df_mlp_last_error.argtypes = [P]
    lib.df_mlp_last_error.restype = C.c_char_p
    lib.df_mlp_destroy.argtypes = [P]
    lib.df_mlp_destroy.restype = None
    _lib = lib
    return lib


def _status_name(s: int) -> str:
    names = {0: "DF_OK", 1: "DF_ERR_ARG", 2: "DF_ERR_CUDA", 3: "DF_ERR_OOM", 4: "DF_ERR_SINGULAR",
             5: "DF_ERR_REFINE_STALL", 6: "DF_ERR_NOT_CONVERGED", 7: "DF_ERR_TIMEOUT",
             8: "DF_WARN_LADDER_RADIUS"}
    return names.get(s, f"status {s}")


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a):
    """(pointer, is_device) of a numpy array or a CUDA torch tensor."""
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data), 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return C.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0)
    raise TypeError(f"unsupported array type {type(a)}")


def current_stream_handle() -> Optional[int]:
    """cudaStream_t of torch's current stream (None when torch/CUDA absent)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class DualFermion:
    """One ladder dual-fermion problem resident on the GPU (a df_ctx handle)."""

    def __init__(self, *, dim: int, nk: int, t: float, tp: float, beta: float, mu: float,
                 n_w: int, m_max: int, g, delta, gamma_d, gamma_m, mix: float = 1.0,
                 precision: int = DF_FP64, eig_mode: int = 1, ir_max_steps: int = 8,
                 ir_tol: float = 1e-13, radius_order: int = 0, ladder_tol: float = 1e-9,
                 ladder_fallback: int = 1, mixed_sweep: int = 0, w_range: Optional[tuple] = None,
                 symmetry: int = 0, stream: Optional[int] = None):
        self.lib = load()
        self.dim, self.nk, self.n_w, self.m_max = dim, nk, n_w, m_max
        self.N = nk ** dim
        self.nb = 2 * m_max + 1
        self.ne = n_w + 2 * m_max
        lat = df_lattice(dim, nk, tp)
        opts = df_opts()
        self.lib.df_default_opts(C.byref(opts))
        opts.n_w, opts.m_max, opts.mix, opts.precision = n_w, m_max, mix, precision
        opts.eig_mode, opts.ir_max_steps, opts.ir_tol = eig_mode, ir_max_steps, ir_tol
        opts.radius_order = radius_order
        opts.ladder_tol, opts.ladder_fallback, opts.mixed_sweep = ladder_tol, ladder_fallback, mixed_sweep
        if w_range is not None:
            opts.w_lo, opts.w_hi = int(w_range[0]), int(w_range[1])
        self.w_range = (opts.w_lo, opts.w_hi if opts.w_hi > 0 else self.nb)
        opts.symmetry = int(symmetry)          # 0 off, 1 point group, 2 + frequency reflection
        g, delta = _c128(g), _c128(delta)
        gd, gm = _c128(gamma_d), _c128(gamma_m)
        if g.shape != (self.ne,) or delta.shape != (self.ne,):
            raise ValueError(f"g, delta must have shape ({self.ne},)")
        if gd.shape != (self.nb, n_w, n_w) or gm.shape != gd.shape:
            raise ValueError(f"gamma_d, gamma_m must have shape {(self.nb, n_w, n_w)}")
        if stream is None:
            stream = current_stream_handle()
        self._stream = stream
        h = C.c_void_p()
        s = self.lib.df_init(C.byref(h), C.byref(lat), beta, mu, t,
                             g.ctypes.data, delta.ctypes.data, gd.ctypes.data, gm.ctypes.data,
                             C.byref(opts), C.c_void_p(stream) if stream else None)
        if s != DF_OK:
            raise DFError(s, "df_init failed (see stderr)")
        self.h = h

    @classmethod
    def from_workload(cls, w, **kw):
        """Build from an ``inputs.Workload`` (channels combined by df_vertex_from_spin)."""
        gd, gm = vertex_from_spin(w.gamma_uu, w.gamma_ud)
        return cls(dim=w.dim, nk=w.nk, t=w.t, tp=w.tp, beta=w.beta, mu=w.mu, n_w=w.n_w,
                   m_max=w.m_max, g=w.g, delta=w.delta, gamma_d=gd, gamma_m=gm, **kw)

    # -- status ---------------------------------------------------------------
    def _check(self, s: int, allow=(DF_OK,)):
        if s in allow:
            return s
        msg = self.lib.df_last_error(self.h).decode()
        raise DFError(s, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.df_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- loop steps -----------------------------------------------------------
    def bubble(self):
        self._check(self.lib.df_bubble(self.h))

    def bse(self, channel_mask: int = 3):
        self._check(self.lib.df_bse(self.h, channel_mask))

    def sigma(self, want_residual: bool = True):
        r = C.c_double(-1.0)
        s = self.lib.df_sigma(self.h, C.byref(r) if want_residual else None)
        self._check(s, (DF_OK, DF_WARN_LADDER_RADIUS))
        return r.value if want_residual else None

    def sigma_partial(self, out=None):
        """This handle's share of Eq. sd (its bosonic planes), [n_w][N], before mixing and Dyson."""
        return self._get(self.lib.df_sigma_partial, (self.n_w, self.N), out)

    def sigma_finish(self, total, want_residual: bool = True):
        """Mixing, residual and Dyson from the sum of every handle's sigma_partial."""
        if isinstance(total, np.ndarray):
            total = _c128(total)
        p, dev = _ptr(total)
        r = C.c_double(-1.0)
        s = self.lib.df_sigma_finish(self.h, p, dev, C.byref(r) if want_residual else None)
        self._check(s, (DF_OK, DF_WARN_LADDER_RADIUS))
        return r.value if want_residual else None

    def ladder_stats(self):
        """(largest predicted error rho^2, ladders handed back to FP64) of the last bse() under DF_FP32_IR."""
        w = C.c_double(0.0)
        n = C.c_int(0)
        self._check(self.lib.df_get_ladder_stats(self.h, C.byref(w), C.byref(n)))
        return w.value, n.value

    def iterate(self, max_iter: int, tol: float = 0.0):
        """Returns (iterations done, residual, status)."""
        it = C.c_int(0)
        r = C.c_double(-1.0)
        s = self.lib.df_iterate(self.h, max_iter, tol, C.byref(it), C.byref(r))
        self._check(s, (DF_OK, DF_WARN_LADDER_RADIUS, DF_ERR_NOT_CONVERGED))
        return it.value, r.value, s

    TIMING_GROUPS = ("bubble", "bse", "lambda", "sigma")

    def set_timing(self, on: bool):
        self._check(self.lib.df_set_timing(self.h, 1 if on else 0))

    def get_timing(self):
        """{group: (device ms, kernel launches)} since set_timing(True)."""
        n = len(self.TIMING_GROUPS)
        ms = (C.c_double * n)()
        la = (C.c_int * n)()
        self._check(self.lib.df_get_timing(self.h, ms, la, n))
        return {g: (ms[i], la[i]) for i, g in enumerate(self.TIMING_GROUPS)}

    def synchronize(self):
        self._check(self.lib.df_synchronize(self.h))

    # -- data -----------------------------------------------------------------
    def _get(self, fn, shape, out=None):
        if out is None:
            out = np.empty(shape, np.complex128)
        p, dev = _ptr(out)
        self._check(fn(self.h, p, dev))
        return out

    def get_sigma(self, out=None):
        return self._get(self.lib.df_get_sigma, (self.n_w, self.N), out)

    def get_gtilde(self, out=None):
        return self._get(self.lib.df_get_gtilde, (self.ne, self.N), out)

    def susceptibility(self, out=None):
        """chi^{ch/sp}(W, q) of the current Sigma~, [2][N_W][N] (0: charge, 1: spin)."""
        return self._get(self.lib.df_susceptibility, (2, 2 * self.m_max + 1, self.N), out)

    def lattice_observables(self, sigma_out=None, g_out=None):
        """(Sigma_lat, G_lat) of the current Sigma~, each [n_w][N] (Eq. sigma_lat, Eq. glat)."""
        shape = (self.n_w, self.N)
        if sigma_out is None:
            sigma_out = np.empty(shape, np.complex128)
        if g_out is None:
            g_out = np.empty(shape, np.complex128)
        ps, ds = _ptr(sigma_out)
        pg, dg = _ptr(g_out)
        if ds != dg:
            raise ValueError("both outputs on the host or both on the device")
        self._check(self.lib.df_lattice_observables(self.h, ps, pg, ds))
        return sigma_out, g_out

    def get_chi(self, out=None):
        return self._get(self.lib.df_get_chi, (self.nb, self.n_w, self.N), out)

    def get_kernel(self, out=None):
        return self._get(self.lib.df_get_kernel, (2, self.nb, self.n_w, self.N), out)

    def get_lambda(self):
        lam = np.empty((2, self.nb, self.N), np.complex128)
        ok = np.empty((2, self.nb, self.N), np.int32)
        self._check(self.lib.df_get_lambda(self.h, lam.ctypes.data, ok.ctypes.data, 0))
        return lam, ok

    def set_sigma(self, sig):
        if isinstance(sig, np.ndarray):
            sig = _c128(sig)
        p, dev = _ptr(sig)
        self._check(self.lib.df_set_sigma(self.h, p, dev))

    def set_inputs(self, g, delta, gamma_d, gamma_m):
        arrs = [a if not isinstance(a, np.ndarray) else _c128(a) for a in (g, delta, gamma_d, gamma_m)]
        ptrs = [_ptr(a) for a in arrs]
        dev = {d for _, d in ptrs}
        if len(dev) != 1:
            raise ValueError("all inputs must be on the same side (host or device)")
        self._check(self.lib.df_set_inputs(self.h, *[p for p, _ in ptrs], dev.pop()))


class DualFermionBatch:
    """Many independent parameter points iterated together (a df_batch handle):
    one launch per stage over all points, one CUDA graph per pass."""

    def __init__(self, workloads, precision: int = DF_FP64, mix: float = 1.0, tol: float = 0.0,
                 symmetry: int = 0, stream: Optional[int] = None):
        self.lib = load()
        self.workloads = list(workloads)
        n = len(self.workloads)
        self._keep = []
        arr = (df_point * n)()
        for i, w in enumerate(self.workloads):
            gd, gm = vertex_from_spin(w.gamma_uu, w.gamma_ud)
            g, dl = _c128(w.g), _c128(w.delta)
            self._keep += [g, dl, gd, gm]
            arr[i] = df_point(w.dim, w.nk, w.tp, w.t, w.beta, w.mu, w.n_w, w.m_max,
                              g.ctypes.data, dl.ctypes.data, gd.ctypes.data, gm.ctypes.data,
                              int(symmetry))
        if stream is None:
            stream = current_stream_handle()
        h = C.c_void_p()
        s = self.lib.df_batch_init(C.byref(h), n, C.cast(arr, C.c_void_p), precision, mix, tol,
                                   C.c_void_p(stream) if stream else None)
        if s != DF_OK:
            raise DFError(s, "df_batch_init failed (see stderr)")
        self.h = h
        self.npts = n

    def _check(self, s, allow=(DF_OK,)):
        if s in allow:
            return s
        raise DFError(s, self.lib.df_batch_last_error(self.h).decode())

    def iterate(self, max_iter: int):
        """Returns (passes, residuals [npts], active [npts], status)."""
        it = C.c_int(0)
        r = (C.c_double * self.npts)()
        a = (C.c_int * self.npts)()
        s = self._check(self.lib.df_batch_iterate(self.h, max_iter, C.byref(it), r, a),
                        (DF_OK, DF_ERR_NOT_CONVERGED))
        return it.value, np.array(r[:]), np.array(a[:]), s

    def get_sigma(self, i: int, out=None):
        w = self.workloads[i]
        if out is None:
            out = np.empty((w.n_w, w.N), np.complex128)
        p, dev = _ptr(out)
        self._check(self.lib.df_batch_get_sigma(self.h, i, p, dev))
        return out

    def reset(self):
        self._check(self.lib.df_batch_reset(self.h))

    def autotune(self, cache_path: Optional[str] = None):
        """Returns (rhs chunk, scheduler chunk, from_cache)."""
        ch = (C.c_int * 3)()
        self._check(self.lib.df_batch_autotune(self.h, cache_path.encode() if cache_path else None, ch))
        return ch[0], ch[1], bool(ch[2])

    def close(self):
        if getattr(self, "h", None):
            self.lib.df_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class MLP:
    """The warm-start network (a df_mlp handle): 4 dense layers
    n_in -> width -> width -> width -> n_out, BF16 tensor-core products with
    FP32 accumulation, FP32 parameters.  Data arguments are CUDA float32
    tensors (row-major [batch][features])."""

    def __init__(self, n_in: int, n_out: int, width: int = 512, max_batch: int = 256, seed: int = 0,
                 stream: Optional[int] = None):
        self.lib = load()
        self.dims = (n_in, width, width, width, n_out)
        self.max_batch = max_batch
        if stream is None:
            stream = current_stream_handle()
        h = C.c_void_p()
        s = self.lib.df_mlp_create(C.byref(h), n_in, width, n_out, max_batch, seed,
                                   C.c_void_p(stream) if stream else None)
        if s != DF_OK:
            raise DFError(s, "df_mlp_create failed (see stderr)")
        self.h = h
        cnt = C.c_long(0)
        self.lib.df_mlp_param_count(self.h, C.byref(cnt))
        self.nparam = cnt.value

    def _check(self, s):
        if s != DF_OK:
            raise DFError(s, self.lib.df_mlp_last_error(self.h).decode())

    def forward(self, x, y):
        self._check(self.lib.df_mlp_forward(self.h, C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(y.data_ptr())))

    def gradients(self, x, t):
        loss = C.c_float(0.0)
        self._check(self.lib.df_mlp_gradients(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()),
                                              x.shape[0], C.byref(loss)))
        return loss.value

    def adam_step(self, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self._check(self.lib.df_mlp_adam_step(self.h, lr, b1, b2, eps))

    def train_step(self, x, t, lr: float, want_loss: bool = False):
        loss = C.c_float(0.0)
        self._check(self.lib.df_mlp_train_step(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()),
                                               x.shape[0], lr, C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def params(self) -> np.ndarray:
        out = np.empty(self.nparam, np.float32)
        self._check(self.lib.df_mlp_params(self.h, out.ctypes.data, 0, 0))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(self.lib.df_mlp_params(self.h, flat.ctypes.data, 1, 0))

    def grads(self) -> np.ndarray:
        out = np.empty(self.nparam, np.float32)
        self._check(self.lib.df_mlp_grads(self.h, out.ctypes.data, 0))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.df_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def warmstart_sigma(d: "DualFermion", y, mean, sd, kmap):
    """Set d's Sigma~ from one network output (device float32 tensors y, mean,
    sd of layout [n_wedge][n_w/2][2], kmap int32 [N])."""
    s = d.lib.df_warmstart_sigma(d.h, C.c_void_p(y.data_ptr()), C.c_void_p(mean.data_ptr()),
                                 C.c_void_p(sd.data_ptr()), C.c_void_p(kmap.data_ptr()))
    d._check(s)


def mixed_supported(n_w: int) -> bool:
    """DF_FP32_IR covers every ladder order a handle or a batch takes: n_w <= 64 with
    [D | RHS] in registers, up to 128 by the shared-memory Gauss-Jordan kernel."""
    return 2 <= n_w <= 128


def vertex_from_spin(gamma_uu, gamma_ud):
    """Eq. spin_symm through libdf's host helper: (d, m) = (uu + ud, uu - ud)."""
    lib = load()
    uu, ud = _c128(gamma_uu), _c128(gamma_ud)
    d = np.empty_like(uu)
    m = np.empty_like(uu)
    s = lib.df_vertex_from_spin(uu.ctypes.data, ud.ctypes.data, d.ctypes.data, m.ctypes.data, uu.size)
    if s != DF_OK:
        raise DFError(s, "df_vertex_from_spin")
    return d, m


def wedge(dim: int, nk: int):
    """(qmap [nk^dim] int32: orbit index of every momentum, qrep [n_orb] int32:
    smallest momentum of each orbit) for the point group of the hypercubic grid
    (df_wedge: axis permutations and sign flips)."""
    lib = load()
    n = C.c_int(0)
    N = nk ** dim
    qmap = np.empty(N, np.int32)
    qrep = np.empty(N, np.int32)
    s = lib.df_wedge(dim, nk, qmap.ctypes.data, qrep.ctypes.data, C.byref(n))
    if s != DF_OK:
        raise DFError(s, "df_wedge")
    return qmap, qrep[:n.value].copy()


def peak_probe(kind: int) -> float:
    """Measured GFLOP/s of the current device by an FMA loop (df_peak_probe):
    kind 0 FP32 fma, 1 FP32 packed f32x2 fma, 2 FP64 fma."""
    lib = load()
    v = C.c_double(0.0)
    s = lib.df_peak_probe(kind, C.byref(v))
    if s != DF_OK:
        raise DFError(s, "df_peak_probe")
    return v.value
