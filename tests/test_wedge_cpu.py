"""The momentum orbits of df_wedge (host only) against a brute-force action
of the hypercubic point group, and the invariance that makes the ladder
reduction of df_opts.symmetry exact, shown on the oracle: eps_k, the bubble
chi~ (Eq. dual_bubble) and the Eq. sd kernel are constant on every orbit
when Sigma~ is, and stop being so for a Sigma~ that is not."""
import itertools
import math

import numpy as np
import pytest

from oracle import df_oracle as O
from paper_1507_00895_gb300 import inputs as I


@pytest.fixture(scope="module")
def df():
    from paper_1507_00895_gb300 import build, df as dfm
    build.build_lib()
    return dfm


def brute_orbits(dim, nk):
    """Orbit label of every flat momentum under all 2^dim dim! signed axis
    permutations, applied to the coordinate tuples."""
    N = nk ** dim
    coords = np.array(list(itertools.product(range(nk), repeat=dim)))   # C order = flat index
    label = -np.ones(N, int)
    ops = [(perm, signs) for perm in itertools.permutations(range(dim))
           for signs in itertools.product((1, -1), repeat=dim)]
    nxt = 0
    for q in range(N):
        if label[q] >= 0:
            continue
        for perm, signs in ops:
            img = [(signs[d] * coords[q][perm[d]]) % nk for d in range(dim)]
            flat = 0
            for x in img:
                flat = flat * nk + x
            label[flat] = nxt
        nxt += 1
    return label, nxt


@pytest.mark.parametrize("dim,nk", [(1, 8), (2, 4), (2, 16), (3, 8), (4, 4)])
def test_orbits_match_the_group_action(df, dim, nk):
    qmap, qrep = df.wedge(dim, nk)
    label, n = brute_orbits(dim, nk)
    assert len(qrep) == n == math.comb(nk // 2 + dim, dim)
    # same partition: the maps are one relabelling of each other
    pairs = set(zip(label.tolist(), qmap.tolist()))
    assert len(pairs) == n
    # representatives: the smallest member, orbits numbered in their order
    for o, r in enumerate(qrep):
        assert r == np.flatnonzero(qmap == o).min()
    assert np.all(np.diff(qrep) > 0)


def test_wedge_rejects_sizes_the_lattice_does_not_allow(df):
    import ctypes as C
    lib = df.load()
    n = C.c_int(0)
    assert lib.df_wedge(2, 6, None, None, C.byref(n)) == df.DF_ERR_ARG      # not a power of two
    assert lib.df_wedge(3, 32, None, None, C.byref(n)) == df.DF_ERR_ARG     # 32^3 > 4096
    assert lib.df_wedge(5, 2, None, None, C.byref(n)) == df.DF_ERR_ARG
    assert lib.df_wedge(2, 8, None, None, C.byref(n)) == df.DF_OK and n.value == 15


def spread(x, qmap):
    """max over orbits of the spread of x[..., q] within the orbit, relative to max |x|."""
    worst = 0.0
    for o in range(qmap.max() + 1):
        cols = x[..., qmap == o]
        worst = max(worst, float(np.max(np.abs(cols - cols[..., :1]))))
    return worst / max(float(np.max(np.abs(x))), 1e-300)


@pytest.mark.parametrize("dim,nk,tp", [(2, 8, -0.2), (3, 4, 0.0)])
def test_eps_is_invariant(df, dim, nk, tp):
    qmap, _ = df.wedge(dim, nk)
    eps = O.dispersion(dim, nk, 1.0, tp)
    assert spread(eps[None, :], qmap) < 1e-14


def one_pass_pieces(w, sigma):
    eps = O.dispersion(w.dim, w.nk, w.t, w.tp)
    g0 = O.bare_dual_g(w.g, w.delta, eps)
    gt = O.dual_g(g0, sigma, w.n_w, w.m_max)
    chi = O.dual_bubble_fft(gt, w.n_w, w.m_max, w.beta, w.dim, w.nk)
    gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    kern = O.sd_kernel(O.ladder_gamma_diag(gd, chi), O.second_order_diag(gd, chi),
                       O.ladder_gamma_diag(gm, chi), O.second_order_diag(gm, chi))
    return chi, kern


def test_bubble_and_kernel_are_invariant_for_an_invariant_sigma(df):
    w = I.workload("square32_tp", nk=8, n_w=8, m_max=1)
    qmap, _ = df.wedge(w.dim, w.nk)
    # an invariant Sigma~: the oracle's after three passes from zero
    st = O.run_workload(w, n_iter=3)
    assert spread(st.sigma, qmap) < 1e-12
    chi, kern = one_pass_pieces(w, st.sigma)
    assert spread(chi, qmap) < 1e-12
    assert spread(kern, qmap) < 1e-10


def test_a_sigma_that_breaks_the_symmetry_breaks_the_reduction(df):
    # planted on the oracle side: Sigma~ with a k_x-only ripple is not D4-invariant,
    # and the bubble then differs within orbits, so the reduction would not be exact
    w = I.workload("square32_tp", nk=8, n_w=8, m_max=1)
    qmap, _ = df.wedge(w.dim, w.nk)
    kx = 2 * np.pi * np.repeat(np.arange(w.nk), w.nk) / w.nk
    sigma = 0.05 * np.cos(kx)[None, :] * np.ones((w.n_w, 1))
    assert spread(sigma, qmap) > 0.1
    chi, _ = one_pass_pieces(w, sigma.astype(np.complex128))
    assert spread(chi, qmap) > 1e-6


def reflect(x, axis_w, axis_a=None):
    """x with the fermionic axis reversed (w -> -w) and, if given, the bosonic
    axis reversed (W -> -W), complex-conjugated."""
    y = np.flip(x, axis=axis_w)
    if axis_a is not None:
        y = np.flip(y, axis=axis_a)
    return np.conj(y)


def test_frequency_reflection_of_the_inputs_bubble_and_kernel():
    # df_opts.symmetry = 2: with g(-w) = g(w)*, Delta likewise and gamma(-W;w,w') =
    # gamma(W;-w,-w')*, the oracle's chi~ and Eq. sd bracket of -W are the
    # frequency-reversed conjugates of those of W, at Sigma~ = 0 and after passes
    w = I.workload("square32_tp", nk=8, n_w=8, m_max=2)
    gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    for x in (w.g, w.delta):
        assert np.max(np.abs(x - reflect(x, 0))) < 1e-14 * np.max(np.abs(x))
    for gx in (gd, gm):
        assert np.max(np.abs(gx - np.flip(reflect(gx, 1, 0), axis=2))) < 1e-13 * np.max(np.abs(gx))
    for sigma in (np.zeros((w.n_w, w.N), complex), O.run_workload(w, n_iter=2).sigma):
        assert np.max(np.abs(sigma - reflect(sigma, 0))) <= 1e-13 * max(np.max(np.abs(sigma)), 1e-300)
        chi, kern = one_pass_pieces(w, sigma)
        assert np.max(np.abs(chi - reflect(chi, 1, 0))) < 1e-13 * np.max(np.abs(chi))
        assert np.max(np.abs(kern - reflect(kern, 1, 0)) / np.abs(kern)) < 1e-11      # elementwise


def test_a_vertex_without_the_reflection_breaks_it():
    # planted on the oracle side: a complex perturbation of gamma that does not map
    # onto its reflection leaves chi~ symmetric (it does not depend on gamma) but
    # breaks the bracket's reflection, so df_init must refuse such a vertex
    w = I.workload("square32_tp", nk=8, n_w=8, m_max=2)
    rng = np.random.default_rng(3)
    w.gamma_ud = w.gamma_ud + 0.5j * rng.normal(size=w.gamma_ud.shape)
    chi, kern = one_pass_pieces(w, np.zeros((w.n_w, w.N), complex))
    assert np.max(np.abs(chi - reflect(chi, 1, 0))) < 1e-13 * np.max(np.abs(chi))
    # (relative to the typical entry: this workload has a few near-singular ladders)
    assert np.max(np.abs(kern - reflect(kern, 1, 0))) > 1e-2 * np.median(np.abs(kern))


def test_reflection_of_the_eq_sd_products():
    # the frequency reflection in Eq. sd's real-space products, which lets the
    # kernels form only the planes W >= 0: with prod_{W,w}(r) = K_{W,w}(-r) G~_{w+W}(r)
    # (K the bracket, to real space), prod_{-W,w}(r) = prod_{W,-w}(-r)*, and the sum
    # over all W equals the sum over W >= 0 plus the conjugated, reversed W > 0 terms
    w = I.workload("square32_tp", nk=8, n_w=8, m_max=2)
    st = O.run_workload(w, n_iter=2)
    eps = O.dispersion(w.dim, w.nk, w.t, w.tp)
    gt = O.dual_g(O.bare_dual_g(w.g, w.delta, eps), st.sigma, w.n_w, w.m_max)
    _, kern = one_pass_pieces(w, st.sigma)
    gr = np.array([O.to_real_space(x, w.dim, w.nk) for x in gt])
    nb, nw, m = w.n_bos, w.n_w, w.m_max
    refl_r = lambda x: O.reflect(x, w.dim, w.nk)
    prod = np.array([[refl_r(O.to_real_space(kern[a, i], w.dim, w.nk)) * gr[i + a] for i in range(nw)]
                     for a in range(nb)])
    scale = np.max(np.abs(prod))
    for a in range(m):
        for i in range(nw):
            assert np.max(np.abs(prod[a, i] - np.conj(refl_r(prod[2 * m - a, nw - 1 - i])))) < 1e-13 * scale
    total = prod.sum(axis=0)
    folded = np.array([prod[m:, i].sum(axis=0)
                       + sum(np.conj(refl_r(prod[a, nw - 1 - i])) for a in range(m + 1, nb))
                       for i in range(nw)])
    assert np.max(np.abs(folded - total)) < 1e-13 * np.max(np.abs(total))
    # planted: pairing -W with +w (no frequency reversal) breaks it
    wrong = np.array([prod[m:, i].sum(axis=0) + sum(np.conj(refl_r(prod[a, i])) for a in range(m + 1, nb))
                      for i in range(nw)])
    assert np.max(np.abs(wrong - total)) > 1e-6 * np.max(np.abs(total))
