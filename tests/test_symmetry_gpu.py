"""The reductions of the ladder stage against the full solve and against the
oracle: the point group (df_opts.symmetry = 1) and, with it, the frequency
reflection (df_opts.symmetry = 2).

With the point group one ladder per momentum orbit is solved and copied to
the orbit (df_wedge); with the reflection only the planes W >= 0 are formed
(ladders, bubble and Eq. sd's products), those of -W entering as their
frequency-reversed conjugates.  The results equal the full solve's up to
rounding: FP64 within 1e-10 of the oracle (the parity bound), the mixed path
within 1e-8 of the full mixed solve (its stated bound).  The handle checks
its inputs and any Sigma~ it is given for the symmetries it relies on and
refuses what breaks them.
"""
import numpy as np
import pytest

from oracle import df_oracle as O
from paper_1507_00895_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL_MIXED = 1e-8


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


CASES = [
    ("square32_tp", dict(nk=8, n_w=10, m_max=3)),
    ("square32_tp", dict(nk=16, n_w=34, m_max=1)),
    ("cubic16_crit", dict(nk=4, n_w=8, m_max=1)),
    ("paper_u20", dict(nk=8, n_w=6, m_max=2)),
]


@pytest.mark.parametrize("name,kw", CASES)
def test_reduced_fp64_matches_the_oracle(df, name, kw):
    w = I.workload(name, **kw)
    st = O.run_workload(w, n_iter=3)
    with df.DualFermion.from_workload(w, eig_mode=2, symmetry=True) as d:
        for it in range(3):
            d.bubble()
            d.bse(3)
            r = d.sigma()
            assert abs(r - st.residuals[it]) < 1e-9 * max(1.0, st.residuals[it])
            assert nrel(d.get_sigma(), st.sigmas[it]) < TOL64, it


@pytest.mark.parametrize("name,kw", [("square32_tp", dict(nk=16, n_w=32, m_max=3)),
                                     ("cubic16_crit", dict(nk=8, n_w=48, m_max=1)),
                                     ("cubic16_crit", dict(nk=4, n_w=96, m_max=1)),
                                     ("square32_tp", dict(nk=8, n_w=128, m_max=1))])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reduced_equals_full(df, name, kw, prec):
    w = I.workload(name, **kw)
    p = df.DF_FP64 if prec == "fp64" else df.DF_FP32_IR
    tol = TOL64 if prec == "fp64" else TOL_MIXED
    with df.DualFermion.from_workload(w, precision=p, eig_mode=2) as full, \
            df.DualFermion.from_workload(w, precision=p, eig_mode=2, symmetry=True) as red:
        for it in range(2):
            for d in (full, red):
                d.bubble()
                d.bse(3)
            assert nrel(red.get_kernel(), full.get_kernel()) < tol, it
            if prec == "mixed":
                # the reduced grid is solved by the same mixed kernels: no more hand-backs
                # to the FP64 LU than on the full grid, proportionally
                _, qrep = df.wedge(w.dim, w.nk)
                back_f = full.ladder_stats()[1] / (2 * w.n_bos * w.N)
                back_r = red.ladder_stats()[1] / (2 * w.n_bos * len(qrep))
                assert back_r <= max(0.05, 3 * back_f), (back_r, back_f)
            lf, okf = full.get_lambda()
            lr, okr = red.get_lambda()
            # the leading eigenvalue is a diagnostic of its own accuracy: the power
            # iteration runs on tiles of 8 momenta, which differ between the full and the
            # reduced grid, and its stopping step can differ with them; where both report a converged
            # single vector (ok 1) they agree to 1e-5, a fitted dominant pair (ok 2) to 1e-4
            scale = max(1.0, float(np.max(np.abs(lf))))
            for flag, bound in ((1, 1e-5), (2, 1e-4)):
                m = (okf == flag) & (okr == flag)
                if np.any(m):
                    assert np.max(np.abs(lr[m] - lf[m])) < bound * scale, flag
            assert np.mean(okf == okr) > 0.95
            full.sigma()
            red.sigma()
            assert nrel(red.get_sigma(), full.get_sigma()) < tol, it


def test_reduced_omega_split(df):
    # the reduction inside the Omega split: each range handle gathers, solves and
    # copies back only its own planes
    w = I.workload("square32_tp", nk=8, n_w=10, m_max=3)
    st = O.run_workload(w, n_iter=2)
    cut = 4
    with df.DualFermion.from_workload(w, w_range=(0, cut), symmetry=True) as d0, \
            df.DualFermion.from_workload(w, w_range=(cut, w.n_bos), symmetry=True) as d1:
        for it in range(2):
            parts = []
            for d in (d0, d1):
                d.bubble()
                d.bse(3)
                parts.append(d.sigma_partial())
            total = parts[0] + parts[1]
            d0.sigma_finish(total)
            d1.sigma_finish(total)
            assert nrel(d0.get_sigma(), st.sigmas[it]) < TOL64, it


def test_set_sigma_checks_the_invariance(df):
    w = I.workload("square32_tp", nk=8, n_w=10, m_max=1)
    st = O.run_workload(w, n_iter=2)
    with df.DualFermion.from_workload(w, symmetry=True) as d:
        d.set_sigma(st.sigmas[0])                 # invariant: accepted
        assert nrel(d.get_sigma(), st.sigmas[0]) == 0.0
        kx = 2 * np.pi * np.repeat(np.arange(w.nk), w.nk) / w.nk
        bad = st.sigmas[0] + 0.01 * np.cos(kx)[None, :]
        with pytest.raises(df.DFError) as e:
            d.set_sigma(bad)
        assert e.value.status == df.DF_ERR_ARG
        assert np.all(d.get_sigma() == 0)         # refused: Sigma~ reset to zero
        # the handle still runs the loop from zero, like a fresh one
        d.bubble()
        d.bse(3)
        d.sigma()
        assert nrel(d.get_sigma(), st.sigmas[0]) < TOL64
    # without the reduction any Sigma~ is taken
    with df.DualFermion.from_workload(w) as d:
        d.set_sigma(bad)
        assert nrel(d.get_sigma(), bad) == 0.0


def test_reduced_iterate_converges_like_the_full_loop(df):
    w = I.workload("paper_u20", nk=8, n_w=12, m_max=2)
    with df.DualFermion.from_workload(w) as full, df.DualFermion.from_workload(w, symmetry=True) as red:
        nf, rf, sf = full.iterate(40, 1e-10)
        nr, rr, sr = red.iterate(40, 1e-10)
        assert sf == sr == df.DF_OK
        assert abs(nf - nr) <= 1
        assert nrel(red.get_sigma(), full.get_sigma()) < TOL64


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reduced_without_eigenvalues(df, prec):
    # eig_mode 0: no leading eigenvalues are computed, only the brackets are copied to the
    # orbits, and the handle's eigenvalue arrays keep their initial state
    w = I.workload("square32_tp", nk=8, n_w=128, m_max=1)
    p = df.DF_FP64 if prec == "fp64" else df.DF_FP32_IR
    tol = TOL64 if prec == "fp64" else TOL_MIXED
    with df.DualFermion.from_workload(w, precision=p, eig_mode=0) as full, \
            df.DualFermion.from_workload(w, precision=p, eig_mode=0, symmetry=True) as red:
        for it in range(2):
            for d in (full, red):
                d.bubble()
                d.bse(3)
                d.sigma()
            assert nrel(red.get_sigma(), full.get_sigma()) < tol, it
        lam, ok = red.get_lambda()
        assert np.all(lam == 0) and np.all(ok == -1)


@pytest.mark.parametrize("name,kw", [("square32_tp", dict(nk=16, n_w=32, m_max=3)),
                                     ("cubic16_crit", dict(nk=4, n_w=96, m_max=2)),
                                     ("square32_tp", dict(nk=8, n_w=128, m_max=2)),
                                     ("paper_u20", dict(nk=8, n_w=12, m_max=0))])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reflection_equals_full(df, name, kw, prec):
    # symmetry = 2: the planes W >= 0 solved on the orbit representatives, W < 0 by
    # the frequency reflection; brackets, eigenvalues (all W) and Sigma~ against the
    # full solve over two passes
    w = I.workload(name, **kw)
    p = df.DF_FP64 if prec == "fp64" else df.DF_FP32_IR
    tol = TOL64 if prec == "fp64" else TOL_MIXED
    with df.DualFermion.from_workload(w, precision=p, eig_mode=2) as full, \
            df.DualFermion.from_workload(w, precision=p, eig_mode=2, symmetry=2) as red:
        for it in range(2):
            for d in (full, red):
                d.bubble()
                d.bse(3)
            # chi~ of W < 0 is not formed by the pass; df_get_chi fills it by the reflection
            # (equal to rounding on the first pass; later passes carry Sigma~'s difference)
            assert nrel(red.get_chi(), full.get_chi()) < (1e-13 if it == 0 else tol), it
            assert nrel(red.get_kernel(), full.get_kernel()) < tol, it
            lf, okf = full.get_lambda()
            lr, okr = red.get_lambda()
            scale = max(1.0, float(np.max(np.abs(lf))))
            m = (okf == 1) & (okr == 1)
            if np.any(m):
                assert np.max(np.abs(lr[m] - lf[m])) < 1e-5 * scale
            # a dominant pair of equal moduli (flag 2): the reflection carries the conjugate
            # of the W plane's member, the -W plane's own solve may pick the other one
            m = (okf == 2) & (okr == 2)
            if np.any(m):
                d = np.minimum(np.abs(lr[m] - lf[m]), np.abs(lr[m] - np.conj(lf[m])))
                assert np.max(d) < 1e-4 * scale
            full.sigma()
            red.sigma()
            assert nrel(red.get_sigma(), full.get_sigma()) < tol, it


def test_reflection_matches_the_oracle(df):
    # Eq. sd from the planes W >= 0 (the -W terms by the reflection), through
    # df_sigma and, on the third pass, through df_sigma_partial + df_sigma_finish
    w = I.workload("square32_tp", nk=8, n_w=10, m_max=3)
    st = O.run_workload(w, n_iter=3)
    with df.DualFermion.from_workload(w, symmetry=2) as d:
        for it in range(3):
            d.bubble()
            d.bse(3)
            if it < 2:
                d.sigma()
            else:
                d.sigma_finish(d.sigma_partial())
            assert nrel(d.get_sigma(), st.sigmas[it]) < TOL64, it


def test_reflection_refuses_inputs_and_sigma_without_it(df):
    # inputs without the reflection: refused at df_init and by df_set_inputs (the
    # handle keeps its inputs); a Sigma~ without it: refused, Sigma~ reset to 0
    bad = I.random_nonsymmetric(8, 1, 2, 4, seed=5)
    with pytest.raises(df.DFError) as e:
        df.DualFermion.from_workload(bad, symmetry=2)
    assert e.value.status == df.DF_ERR_ARG
    w = I.workload("square32_tp", nk=8, n_w=8, m_max=1)
    st = O.run_workload(w, n_iter=1)
    with df.DualFermion.from_workload(w, symmetry=2) as d:
        gd, gm = df.vertex_from_spin(bad.gamma_uu, bad.gamma_ud)
        with pytest.raises(df.DFError) as e:
            d.set_inputs(bad.g, bad.delta, gd, gm)
        assert e.value.status == df.DF_ERR_ARG
        d.set_sigma(st.sigmas[0])                              # has the reflection
        sig = st.sigmas[0] + 0.01j * np.arange(w.n_w)[:, None]   # an imaginary ramp in w: breaks it
        with pytest.raises(df.DFError):
            d.set_sigma(sig)
        assert np.all(d.get_sigma() == 0)
        d.bubble()
        d.bse(3)
        d.sigma()
        assert nrel(d.get_sigma(), st.sigmas[0]) < TOL64      # the handle's inputs are unchanged
    with pytest.raises(df.DFError):                            # needs the full bosonic range
        df.DualFermion.from_workload(w, symmetry=2, w_range=(0, 2))


@pytest.mark.parametrize("dim,nk", [(1, 16), (2, 2), (4, 4)])
@pytest.mark.parametrize("sym", [1, 2])
def test_reductions_in_other_dimensions(df, dim, nk, sym):
    # 1D (sign flip only), the 2 x 2 grid (3 orbits of 4) and the 4D hypercube
    # (hyperoctahedral group: 15 orbits of 256), FP64, against the oracle over two passes
    w = I.half_filled_atom("h", dim, nk, U=6.0, beta=1.5, n_w=8, m_max=2)
    st = O.run_workload(w, n_iter=2)
    with df.DualFermion.from_workload(w, symmetry=sym) as d:
        for it in range(2):
            d.bubble()
            d.bse(3)
            d.sigma()
            assert nrel(d.get_sigma(), st.sigmas[it]) < TOL64, it
