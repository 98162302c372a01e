"""Mixed-precision ladder solves (DF_FP32_IR) against the CPU oracle.

FP32 LU + one correction with a double-float (~48-bit) residual.  Stated
tolerance of the refined mixed path: Sigma~ within 1e-8 of the oracle
normwise; the ladder kernel within 5e-8 normwise per (channel, W) plane.
The residual's double-float accumulation keeps ~2^-48 relative to the
partial sums of gamma chi~ X0, whose terms exceed the sum by |gamma chi~|
(~3e4 on the 32^2 workload), against 2^-53 for an FP64 residual.
"""
import numpy as np
import pytest

from oracle import df_oracle as O
from paper_1507_00895_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_KERNEL = 5e-8
TOL_SIGMA = 1e-8


@pytest.fixture(scope="module")
def df():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_00895_gb300 import build
    build.build_lib()
    from paper_1507_00895_gb300 import df as dfm
    return dfm


def nrel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def oracle_first_pass(w):
    eps = O.dispersion(w.dim, w.nk, w.t, w.tp)
    g0 = O.bare_dual_g(w.g, w.delta, eps)
    gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    st = O.LoopState(g0_ext=g0, sigma=np.zeros((w.n_w, w.N), complex))
    O.one_iteration(st, gd, gm, w.n_w, w.m_max, w.beta, w.dim, w.nk)
    kd = st.gd_diag - 0.5 * O.second_order_diag(gd, st.chi)
    km = 3.0 * (st.gm_diag - 0.5 * O.second_order_diag(gm, st.chi))
    return st, np.stack([kd, km])


CASES = [
    ("square16_b5", dict(nk=4, n_w=2, m_max=0)),          # n_w=2 padded to 4
    ("square16_b5", dict(nk=8, n_w=6, m_max=1)),          # ragged pad
    ("paper_u20", dict(nk=8, n_w=16, m_max=1)),
    ("square32_tp", dict(nk=8, n_w=30, m_max=2)),
    ("square16_b5", dict()),                              # 16^2, n_w=32
]


@pytest.mark.parametrize("name,kw", CASES)
def test_mixed_first_pass(df, name, kw):
    w = I.workload(name, **kw)
    st, kref = oracle_first_pass(w)
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR) as d:
        d.bubble()
        d.bse(3)
        kern = d.get_kernel()
        for c in range(2):
            for a in range(w.n_bos):
                assert nrel(kern[c, a], kref[c, a]) < TOL_KERNEL, (c, a)
        d.sigma()
        assert nrel(d.get_sigma(), st.sigma) < TOL_SIGMA


def test_mixed_square32_tp_full_size(df):
    # the benchmark workload: 30,720 ladders of order 64, cond up to ~1e6
    w = I.workload("square32_tp")
    st, kref = oracle_first_pass(w)
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR) as d:
        d.bubble()
        d.bse(3)
        kern = d.get_kernel()
        worst = max(nrel(kern[c, a], kref[c, a]) for c in range(2) for a in range(w.n_bos))
        assert worst < TOL_KERNEL, worst
        d.sigma()
        err = nrel(d.get_sigma(), st.sigma)
        print(f"square32_tp mixed: worst kernel plane {worst:.2e}, Sigma~ {err:.2e}")
        assert err < TOL_SIGMA


def test_mixed_matches_fp64_gpu_over_iterations(df):
    # teacher-free comparison of the two GPU paths on the convergent paper workload
    w = I.workload("paper_u20", nk=16, n_w=48, m_max=1)
    with df.DualFermion.from_workload(w) as d64, \
            df.DualFermion.from_workload(w, precision=df.DF_FP32_IR) as d32:
        i64, r64, _ = d64.iterate(25, tol=1e-12)
        i32, r32, _ = d32.iterate(25, tol=1e-12)
        assert r64 <= 1e-12 and r32 <= 1e-12
        assert nrel(d32.get_sigma(), d64.get_sigma()) < TOL_SIGMA


LARGE = [
    ("cubic16_crit", dict(nk=4, n_w=96, m_max=1)),         # the 3D workload's order
    ("square16_b5", dict(nk=4, n_w=66, m_max=1)),          # 2n threads not a warp multiple
    ("paper_u20", dict(nk=4, n_w=128, m_max=0)),           # the largest order
]


@pytest.mark.parametrize("name,kw", LARGE)
def test_mixed_large_orders_first_pass(df, name, kw):
    # 64 < n_w <= 128: FP32 Gauss-Jordan inverse + one double-float-residual correction
    w = I.workload(name, **kw)
    st, kref = oracle_first_pass(w)
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR) as d:
        d.bubble()
        d.bse(3)
        kern = d.get_kernel()
        for c in range(2):
            for a in range(w.n_bos):
                assert nrel(kern[c, a], kref[c, a]) < TOL_KERNEL, (c, a)
        d.sigma()
        assert nrel(d.get_sigma(), st.sigma) < TOL_SIGMA


def test_mixed_large_order_over_iterations(df):
    # the 3D critical workload's order, three passes, against the GPU FP64 path
    w = I.workload("cubic16_crit", nk=4, n_w=96, m_max=2)
    with df.DualFermion.from_workload(w) as d64, \
            df.DualFermion.from_workload(w, precision=df.DF_FP32_IR) as d32:
        d64.iterate(3)
        d32.iterate(3)
        assert nrel(d32.get_sigma(), d64.get_sigma()) < TOL_SIGMA
