"""Batched loop over uneven parameter points (df_batch_*) against the oracle
and against the single-problem handle."""
import os
import tempfile

import numpy as np
import pytest

from oracle import df_oracle as O
from paper_1507_00895_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


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


def small_batch():
    # uneven: 1D/2D/3D/4D lattices, ladder orders 4..104 (LU in shared and in
    # global memory), 1..7 bosonic frequencies
    ws = [
        I.half_filled_atom("a", 2, 8, U=3.0, beta=2.0, n_w=16, m_max=2),
        I.half_filled_atom("b", 4, 4, U=5.0, beta=3.0, n_w=8, m_max=1),
        I.half_filled_atom("c", 3, 4, U=2.0, beta=4.0, n_w=24, m_max=0),
        I.half_filled_atom("d", 1, 16, U=6.0, beta=1.5, n_w=4, m_max=3),
        I.workload("square32_tp", nk=8, n_w=40, m_max=1),
        I.half_filled_atom("f", 2, 4, U=4.0, beta=2.5, n_w=104, m_max=1),
    ]
    return ws


def test_batch_fp64_matches_oracle_per_point(df):
    ws = small_batch()
    with df.DualFermionBatch(ws) as b:
        it, r, act, _ = b.iterate(2)
        assert it == 2
        for i, w in enumerate(ws):
            st = O.run_workload(w, n_iter=2)
            assert nrel(b.get_sigma(i), st.sigma) < TOL64, (i, w.name)
            assert abs(r[i] - st.residuals[-1]) < 1e-10 * max(1.0, st.residuals[-1])


def test_batch_equals_single_handles(df):
    # the same device functions inlined into two kernels may contract
    # multiply-adds differently: equal to rounding, not bit for bit
    ws = small_batch()
    with df.DualFermionBatch(ws) as b:
        b.iterate(2)
        for i, w in enumerate(ws):
            with df.DualFermion.from_workload(w, eig_mode=0) as d:
                d.iterate(2)
                assert nrel(b.get_sigma(i), d.get_sigma()) < 1e-13, i


def test_batch_mixed_matches_oracle(df):
    ws = small_batch()
    with df.DualFermionBatch(ws, precision=df.DF_FP32_IR) as b:
        b.iterate(1)
        for i, w in enumerate(ws):
            st = O.run_workload(w, n_iter=1)
            assert nrel(b.get_sigma(i), st.sigma) < 1e-8, (i, w.name)


def test_batch_mixed_large_orders(df):
    # DF_FP32_IR points above n_w = 64 (the Gauss-Jordan class) beside a register-tile one
    ws = [I.workload("cubic16_crit", nk=4, n_w=96, m_max=1),
          I.workload("square16_b5", nk=4, n_w=66, m_max=0),
          I.workload("paper_u20", nk=4, n_w=128, m_max=0),
          I.workload("paper_u20", nk=8, n_w=16, m_max=1)]
    with df.DualFermionBatch(ws, precision=df.DF_FP32_IR) as b:
        b.iterate(1)
        for i, w in enumerate(ws):
            st = O.run_workload(w, n_iter=1)
            assert nrel(b.get_sigma(i), st.sigma) < 1e-8, (i, w.name)


def test_batch_convergence_flags_freeze_points(df):
    # the paper's Example I inputs converge; the 32^2-like point does not
    conv = I.workload("paper_u20", nk=8, n_w=16, m_max=1)
    stuck = I.workload("square32_tp", nk=8, n_w=16, m_max=1)
    with df.DualFermionBatch([conv, stuck], tol=1e-12) as b:
        it, r, act, s = b.iterate(40)
        assert s == df.DF_ERR_NOT_CONVERGED and it == 40
        assert act[0] == 0 and act[1] == 1
        assert r[0] <= 1e-12
        ref = O.run_workload(conv, n_iter=40, tol=1e-12)
        assert nrel(b.get_sigma(0), ref.sigma) < TOL64
        frozen = b.get_sigma(0).copy()
        b.iterate(3)
        assert np.array_equal(b.get_sigma(0), frozen)


def test_batch_autotune_and_cache(df):
    ws = small_batch()
    path = os.path.join(tempfile.mkdtemp(), "tune.txt")
    with df.DualFermionBatch(ws) as b:
        nc, ch, cached = b.autotune(path)
        assert not cached and nc in (0, 8, 16, 32) and ch in (1, 4)
        b.iterate(2)
        for i, w in enumerate(ws):
            st = O.run_workload(w, n_iter=2)
            assert nrel(b.get_sigma(i), st.sigma) < TOL64
    with df.DualFermionBatch(ws) as b:
        nc2, ch2, cached2 = b.autotune(path)
        assert cached2 and (nc2, ch2) == (nc, ch)


def test_uneven_batch_recipe_first_pass_sampled(df):
    # the 64-point recipe at capped sizes (n_w <= 48, m <= 3, 2D 8^2/16^2 and 4D 4^4)
    ws = I.uneven_batch(npts=64, seed=4, max_n_w=48, max_m=3, grids=((2, 8), (2, 16), (4, 4)))
    with df.DualFermionBatch(ws, precision=df.DF_FP32_IR) as b:
        b.iterate(1)
        for i in (0, 7, 21, 42, 63):
            st = O.run_workload(ws[i], n_iter=1)
            assert nrel(b.get_sigma(i), st.sigma) < 1e-8, i


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_point_group_reduction_equals_full(df, prec):
    # the reduction per point (df_point.symmetry): one ladder per momentum orbit on
    # 2D, 3D and 4D grids with orders across the mixed classes (16 .. 128), two passes,
    # every point's Sigma~ within 1e-10 (FP64) / 1e-8 (mixed) of the full batch's
    ws = I.uneven_batch(npts=10, seed=11, max_n_w=128, max_m=2, grids=((2, 8), (2, 16), (3, 4), (4, 4)))
    p = df.DF_FP64 if prec == "fp64" else df.DF_FP32_IR
    tol = 1e-10 if prec == "fp64" else 1e-8
    with df.DualFermionBatch(ws, precision=p) as full, df.DualFermionBatch(ws, precision=p, symmetry=True) as red:
        full.iterate(2)
        red.iterate(2)
        for i in range(len(ws)):
            assert nrel(red.get_sigma(i), full.get_sigma(i)) < tol, (i, ws[i].dim, ws[i].nk, ws[i].n_w)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_frequency_reflection_equals_full(df, prec):
    # df_point.symmetry = 2: the point group and only W >= 0 solved per point
    ws = I.uneven_batch(npts=8, seed=12, max_n_w=128, max_m=3, grids=((2, 8), (3, 4), (4, 4)))
    p = df.DF_FP64 if prec == "fp64" else df.DF_FP32_IR
    tol = 1e-10 if prec == "fp64" else 1e-8
    with df.DualFermionBatch(ws, precision=p) as full, df.DualFermionBatch(ws, precision=p, symmetry=2) as red:
        full.iterate(2)
        red.iterate(2)
        for i in range(len(ws)):
            assert nrel(red.get_sigma(i), full.get_sigma(i)) < tol, (i, ws[i].dim, ws[i].nk, ws[i].n_w)


def test_batch_refuses_inputs_without_the_reflection(df):
    bad = I.random_nonsymmetric(8, 1, 2, 4, seed=6)
    with pytest.raises(df.DFError) as e:
        df.DualFermionBatch([bad], symmetry=2)
    assert e.value.status == df.DF_ERR_ARG
