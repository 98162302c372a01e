"""The C ABI library builds, loads and exports every symbol include/df.h
declares; host-only helpers work; device entry points fail loudly (no CPU
fallback) when no GPU is present.  No GPU compute here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_00895_gb300 import build, df
    build.build_lib()
    return df.load()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "df.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(df_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1507_00895_gb300 import df
    syms = header_symbols()
    assert len(syms) >= 19
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(df.EXPORTS)


def test_vertex_from_spin_host_helper(lib):
    from paper_1507_00895_gb300 import df
    rng = np.random.default_rng(0)
    uu = rng.normal(size=(3, 4, 4)) + 1j * rng.normal(size=(3, 4, 4))
    ud = rng.normal(size=(3, 4, 4)) + 1j * rng.normal(size=(3, 4, 4))
    d, m = df.vertex_from_spin(uu, ud)
    assert np.array_equal(d, uu + ud) and np.array_equal(m, uu - ud)


def test_status_strings_and_null_handles(lib):
    assert lib.df_status_string(8) == b"DF_WARN_LADDER_RADIUS"
    assert lib.df_bubble(None) == 1            # DF_ERR_ARG
    assert lib.df_sigma(None, None) == 1
    assert lib.df_last_error(None) == b"NULL handle"


def test_bad_sizes_are_rejected_before_any_device_call(lib):
    from paper_1507_00895_gb300 import df
    h = C.c_void_p()
    opts = df.df_opts()
    lib.df_default_opts(C.byref(opts))
    opts.n_w, opts.m_max = 3, 0                  # odd n_w
    lat = df.df_lattice(2, 4, 0.0)
    buf = np.zeros(64, np.complex128)
    p = buf.ctypes.data
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == 1
    opts.n_w = 4
    lat = df.df_lattice(2, 6, 0.0)               # not a power of two
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == 1
    lat = df.df_lattice(3, 4, -0.2)              # t' only in 2D
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == 1
    lat = df.df_lattice(2, 4, 0.0)
    opts.radius_order = 1                        # the radius extension needs eig_mode 2 ...
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == 1
    opts.eig_mode, opts.precision = 2, df.DF_FP32_IR   # ... and the FP64 path
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == 1
    opts.precision, opts.radius_order = df.DF_FP64, 17
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == 1
    opts.radius_order, opts.ir_max_steps = 0, 0   # refinement steps in [1, 64] ...
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == 1
    opts.ir_max_steps, opts.ir_tol = 8, 0.0       # ... and a tolerance in (0, 1)
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == 1
    assert lib.df_selftest_wait(0, 0) == df.DF_ERR_ARG   # the bounded-wait self-test needs a limit >= 1


def test_no_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1507_00895_gb300 import df, inputs
    w = inputs.workload("square16_b5", nk=4, n_w=4)
    with pytest.raises(df.DFError) as ei:
        df.DualFermion.from_workload(w)
    assert ei.value.status == df.DF_ERR_CUDA


def test_reduction_options_are_checked_before_any_device_call(lib):
    from paper_1507_00895_gb300 import df, inputs
    h = C.c_void_p()
    opts = df.df_opts()
    lib.df_default_opts(C.byref(opts))
    assert opts.symmetry == 0                    # default: every ladder solved
    opts.n_w, opts.m_max = 4, 1
    lat = df.df_lattice(2, 4, 0.0)
    buf = np.zeros(256, np.complex128)
    p = buf.ctypes.data
    opts.symmetry = 3                            # 0, 1 or 2
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == df.DF_ERR_ARG
    opts.symmetry, opts.w_lo, opts.w_hi = 2, 0, 2   # the reflection needs the full bosonic range
    assert lib.df_init(C.byref(h), C.byref(lat), 1.0, 0.0, 1.0, p, p, p, p, C.byref(opts), None) == df.DF_ERR_ARG
    # a batch point: the symmetry field's range, and inputs without the reflection under symmetry 2
    # (checked on the host before the batch touches the device)
    bad = inputs.random_nonsymmetric(8, 1, 2, 4, seed=6)
    gd, gm = df.vertex_from_spin(bad.gamma_uu, bad.gamma_ud)
    g, dl = np.ascontiguousarray(bad.g), np.ascontiguousarray(bad.delta)
    keep = [g, dl, gd, gm]
    for sym in (3, 2):
        pt = df.df_point(bad.dim, bad.nk, bad.tp, bad.t, bad.beta, bad.mu, bad.n_w, bad.m_max,
                         g.ctypes.data, dl.ctypes.data, gd.ctypes.data, gm.ctypes.data, sym)
        b = C.c_void_p()
        assert lib.df_batch_init(C.byref(b), 1, C.cast(C.pointer(pt), C.c_void_p), df.DF_FP64, 1.0, 0.0,
                                 None) == df.DF_ERR_ARG, sym
    del keep
