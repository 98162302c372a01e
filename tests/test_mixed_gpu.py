"""Mixed-precision ladder solves (DF_FP32_IR) against the CPU oracle.

FP32 factorisation + one correction with an extended-precision residual, and
per-ladder error control: a ladder whose predicted error rho^2 exceeds
ladder_tol (1e-9) is solved again by the FP64 LU.  Stated tolerance of the
refined mixed path (the bound for refined mixed-precision results): Sigma~
and every ladder-kernel (channel, W) plane within 1e-8 of the oracle,
normwise.
"""
import numpy as np
import pytest

from oracle import df_oracle as O
from paper_1507_00895_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_KERNEL = 1e-8
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


def erel(a, b, floor=1e-6):
    """Largest elementwise relative difference over the elements of b above floor * max |b|."""
    m = np.abs(b) > floor * np.max(np.abs(b))
    return float(np.max(np.abs(a - b)[m] / np.abs(b)[m]))


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
        worst_rho2, back = d.ladder_stats()
        d.sigma()
        err = nrel(d.get_sigma(), st.sigma)
        print(f"square32_tp mixed: worst kernel plane {worst:.2e}, Sigma~ {err:.2e}, "
              f"handed back {back} of {2 * w.n_bos * w.N}, worst rho^2 {worst_rho2:.1e}")
        assert err < TOL_SIGMA
        assert erel(d.get_sigma(), st.sigma) < TOL_SIGMA
        assert back < 0.05 * 2 * w.n_bos * w.N


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


@pytest.mark.parametrize("sweep", [0, 1])
@pytest.mark.parametrize("name,kw", LARGE)
def test_mixed_large_orders_first_pass(df, name, kw, sweep):
    # 64 < n_w <= 128: FP32 Gauss-Jordan inverse (on the tensor cores, sweep 0, or the
    # CUDA cores, sweep 1) + one double-float-residual correction
    w = I.workload(name, **kw)
    st, kref = oracle_first_pass(w)
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR, mixed_sweep=sweep) as d:
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


def test_mixed_error_control_hands_back(df):
    # ladder_tol below any attainable rho^2: every ladder is solved again by the
    # FP64 LU, and the kernel equals the FP64 path's bit for bit
    w = I.workload("square32_tp", nk=8, n_w=40, m_max=1)
    with df.DualFermion.from_workload(w) as d64:
        d64.bubble()
        d64.bse(3)
        k64 = d64.get_kernel()
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR, ladder_tol=1e-300) as d:
        d.bubble()
        d.bse(3)
        worst, back = d.ladder_stats()
        assert back == 2 * w.n_bos * w.N and worst > 0.0
        assert np.array_equal(d.get_kernel(), k64)
    # the default bound: a few ill-conditioned ladders are handed back, the rest
    # keep their mixed results, within the stated bound of the FP64 path
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR) as d:
        d.bubble()
        d.bse(3)
        worst, back = d.ladder_stats()
        assert 0.0 < worst and back < 0.05 * 2 * w.n_bos * w.N
        kmix = d.get_kernel()
        for c in range(2):
            for a in range(w.n_bos):
                assert nrel(kmix[c, a], k64[c, a]) < TOL_KERNEL, (c, a)


def test_mixed_error_control_reports_without_fallback(df):
    # ladder_fallback = 0: a ladder above ladder_tol keeps its mixed result and the
    # pass reports DF_ERR_REFINE_STALL
    w = I.workload("square32_tp", nk=4, n_w=16, m_max=1)
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR, ladder_tol=1e-300, ladder_fallback=0) as d:
        with pytest.raises(df.DFError) as e:
            d.iterate(1)
        assert e.value.status == df.DF_ERR_REFINE_STALL
    w = I.workload("cubic16_crit", nk=4, n_w=96, m_max=0)   # the large-order kernel
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR, ladder_tol=1e-300, ladder_fallback=0) as d:
        with pytest.raises(df.DFError) as e:
            d.iterate(1)
        assert e.value.status == df.DF_ERR_REFINE_STALL


@pytest.mark.parametrize("n_w", [12, 80])
def test_mixed_ill_conditioned_ladder_is_handed_back(df, n_w):
    # one ladder made nearly singular: the magnetic vertex of W = 0 is rescaled so
    # that gamma chi~ of one q has an eigenvalue 1 - 1e-9 (cond(D) ~ 1e9 there).  Its
    # FP32 factorisation cannot deliver, the error control hands it to the FP64 LU,
    # and the mixed kernel then matches the FP64 path on every plane
    w = I.workload("paper_u20", nk=4, n_w=n_w, m_max=0)
    st, _ = oracle_first_pass(w)
    gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    q = 5
    ev = np.linalg.eigvals(gm[0] * st.chi[0, :, q][None, :])
    lead = ev[np.argmax(np.abs(ev))]
    gm = gm * ((1.0 - 1e-9) / lead)
    D = np.eye(n_w) - gm[0] * st.chi[0, :, q][None, :]
    assert np.linalg.cond(D) > 1e8
    kw = dict(dim=w.dim, nk=w.nk, t=w.t, tp=w.tp, beta=w.beta, mu=w.mu, n_w=w.n_w, m_max=w.m_max, g=w.g,
              delta=w.delta, gamma_d=gd, gamma_m=gm)
    with df.DualFermion(**kw) as d64:
        d64.bubble()
        d64.bse(3)
        k64 = d64.get_kernel()
    with df.DualFermion(precision=df.DF_FP32_IR, **kw) as d:
        d.bubble()
        d.bse(3)
        worst, back = d.ladder_stats()
        kmix = d.get_kernel()
    assert back >= 1 and worst > 1e-9
    # the handed-back ladder is the FP64 path's, bit for bit
    assert np.array_equal(kmix[1, 0, :, q], k64[1, 0, :, q])
    for c in range(2):
        assert nrel(kmix[c, 0], k64[c, 0]) < TOL_KERNEL, c


def test_mixed_cubic16_full_size_against_the_oracle(df):
    # the 3D workload at its stated size (16^3, n_w = 96, 21 bosonic frequencies,
    # 172,032 ladders of order 96): one mixed pass, the whole Sigma~ and every
    # ladder-kernel plane against the oracle (its ladders over a spawned pool)
    import oracle_pool
    w = I.workload("cubic16_crit")
    sig_ref, kref = oracle_pool.first_pass(w)
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR) as d:
        d.bubble()
        d.bse(3)
        kern = d.get_kernel()
        worst_rho2, back = d.ladder_stats()
        d.sigma()
        sig = d.get_sigma()
    worst = max(nrel(kern[c, a], kref[c, a]) for c in range(2) for a in range(w.n_bos))
    err = nrel(sig, sig_ref)
    print(f"cubic16_crit mixed: worst kernel plane {worst:.2e}, Sigma~ {err:.2e} (elementwise "
          f"{erel(sig, sig_ref):.2e}), handed back {back}, worst rho^2 {worst_rho2:.1e}")
    assert worst < TOL_KERNEL
    assert err < TOL_SIGMA and erel(sig, sig_ref) < TOL_SIGMA


def test_tensor_core_sweep_matches_the_cuda_core_sweep(df):
    # the two FP32 Gauss-Jordan inversions of the large-order kernel (tcgen05 panel
    # updates with three-piece BF16 operands vs FP32 FMAs) give the same corrected
    # ladders within the mixed bound, and both within it of the FP64 path
    w = I.workload("cubic16_crit", nk=4, n_w=96, m_max=2)
    out = {}
    for sweep in (0, 1):
        with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR, mixed_sweep=sweep) as d:
            d.bubble()
            d.bse(3)
            out[sweep] = d.get_kernel()
    with df.DualFermion.from_workload(w) as d:
        d.bubble()
        d.bse(3)
        k64 = d.get_kernel()
    for c in range(2):
        for a in range(w.n_bos):
            assert nrel(out[0][c, a], out[1][c, a]) < TOL_KERNEL
            assert nrel(out[0][c, a], k64[c, a]) < TOL_KERNEL
