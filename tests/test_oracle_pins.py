"""Pins of the CPU oracle to things other than itself (no GPU).

Each test cites the passage of the paper it fixes.  Closed forms are derived
by hand for inputs with a known Fourier content; the brute-force sums are
the definitions written out; invariants follow from the symmetries of the
inputs.  A few tests plant a plausible mistake in the oracle (monkeypatch,
CPU only) and check that a pin catches it.
"""

import math

import numpy as np
import pytest

from oracle import df_oracle as O
from paper_1507_00895_gb300 import inputs as I


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---------------------------------------------------------------------------
# input generator (Eqs. atomic_limit1-4)
# ---------------------------------------------------------------------------

def test_atom_g_half_filling_closed_form():
    # Eq. atomic_limit1: (1/2)[1/(iw-U/2) + 1/(iw+U/2)] = -iw / (w^2 + U^2/4)
    U, beta, nw, mm = 3.0, 4.0, 16, 2
    g = I.atom_g(U, beta, U / 2, nw, mm)
    w = I.fermionic_w(beta, I.fermionic_n(nw, mm))
    assert _rel(g, -1j * w / (w * w + U * U / 4)) < 1e-14


def test_atom_density_and_mu():
    assert abs(I.atom_density(4.0, 10.0, 2.0) - 1.0) < 1e-12          # half filling
    mu = I.atom_mu_for_density(4.0, 10.0, 0.9)
    assert abs(I.atom_density(4.0, 10.0, mu) - 0.9) < 1e-12
    assert abs(mu - math.log(4.5) / 10.0) < 1e-3                      # 2e^{bmu}/(1+2e^{bmu}) = .9


def test_atom_vertex_symmetries():
    # real, symmetric in w<->w', invariant under (W,w,w') -> -(W,w,w')
    guu, gud = I.atom_vertices(2.5, 3.0, 12, 3)
    for gm in (guu, gud):
        assert np.all(np.isfinite(gm))
        assert np.max(np.abs(gm - gm.transpose(0, 2, 1))) < 1e-12 * np.max(np.abs(gm))
        assert np.max(np.abs(gm - gm[::-1, ::-1, ::-1])) < 1e-12 * np.max(np.abs(gm))


def test_atom_vertex_large_frequency_limit():
    # at W != 0, w != w', w+w'+2W != 0 and large |w|, |w'| every delta vanishes:
    # gamma^{ud} -> -U + O(U^3/w^2) and gamma^{uu} = 0 exactly
    U, beta = 1.0, 200.0
    guu, gud = I.atom_vertices(U, beta, 400, 1)
    a, i, j = 0, 5, 390      # W = -2pi/beta, n = -195, n' = 190
    assert abs(gud[a, i, j] + U) < 1e-2
    assert guu[a, i, j] == 0.0


# ---------------------------------------------------------------------------
# lattice
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,nk,tp", [(1, 8, 0.0), (2, 8, 0.0), (2, 16, -0.3), (3, 4, 0.0), (4, 4, 0.0)])
def test_dispersion_moments(dim, nk, tp):
    e = O.dispersion(dim, nk, 1.0, tp)
    assert abs(e[0] - (-2 * dim - 4 * tp)) < 1e-13            # k = 0
    assert abs(e.mean()) < 1e-13
    assert abs((e ** 2).mean() - I.second_moment(dim, 1.0, tp)) < 1e-12


def test_dispersion_bipartite():
    e = O.dispersion(2, 8, 1.0).reshape(8, 8)
    assert np.max(np.abs(np.roll(e, (4, 4), (0, 1)) + e)) < 1e-13   # eps(k+Q) = -eps(k)


def test_bare_dual_g_is_dmft_lattice_g_minus_g():
    # Sigma_DMFT = iw + mu - Delta - 1/g (the paper's lattice-observables section);
    # G_DMFT = 1/(iw + mu - eps - Sigma_DMFT); Eq. gd0 says G0~ = G_DMFT - g.
    w = I.workload("square32_tp", nk=8, n_w=8, m_max=2)
    eps = O.dispersion(2, 8, 1.0, w.tp)
    iw = 1j * I.fermionic_w(w.beta, I.fermionic_n(w.n_w, w.m_max))
    sig_dmft = iw + w.mu - w.delta - 1.0 / w.g
    g_dmft = 1.0 / (iw[:, None] + w.mu - eps[None, :] - sig_dmft[:, None])
    assert _rel(O.bare_dual_g(w.g, w.delta, eps), g_dmft - w.g[:, None]) < 1e-12


# ---------------------------------------------------------------------------
# Eq. dual_bubble
# ---------------------------------------------------------------------------

def _harmonic_g(rng, ne, dim, nk, r0):
    """G~_e(k) = a_e + b_e exp(i k.r0) + c_e exp(-i k.r0)."""
    a, b, c = [rng.normal(size=ne) + 1j * rng.normal(size=ne) for _ in range(3)]
    k = O.kgrid(dim, nk)
    ph = np.exp(1j * (k @ np.asarray(r0, float)))
    return a[:, None] + b[:, None] * ph[None] + c[:, None] * np.conj(ph)[None], (a, b, c), k


@pytest.mark.parametrize("dim,nk,r0", [(1, 8, [1]), (2, 4, [1, 0]), (2, 8, [1, 2]), (3, 4, [0, 1, 1])])
def test_bubble_closed_form_single_harmonic(dim, nk, r0):
    # sum_k G(k) G'(k+q) = N [a a' + b c' e^{-iq.r0} + c b' e^{iq.r0}] when 2 r0 != 0 (mod grid)
    rng = np.random.default_rng(11)
    nw, mm, beta = 4, 1, 2.0
    ne = nw + 2 * mm
    G, (a, b, c), k = _harmonic_g(rng, ne, dim, nk, r0)
    ph = np.exp(1j * (k @ np.asarray(r0, float)))
    T = 1.0 / beta
    expect = np.empty((2 * mm + 1, nw, nk ** dim), complex)
    for A in range(2 * mm + 1):
        for i in range(nw):
            e1, e2 = i + mm, i + A
            expect[A, i] = -T * (a[e1] * a[e2] + b[e1] * c[e2] * np.conj(ph) + c[e1] * b[e2] * ph)
    for fn in (O.dual_bubble_direct, O.dual_bubble_fft):
        assert _rel(fn(G, nw, mm, beta, dim, nk), expect) < 1e-13


@pytest.mark.parametrize("dim,nk", [(1, 8), (2, 4), (2, 8), (3, 4), (4, 4)])
def test_bubble_direct_vs_fft(dim, nk):
    rng = np.random.default_rng(dim * 10 + nk)
    nw, mm = 4, 1
    G = rng.normal(size=(nw + 2 * mm, nk ** dim)) + 1j * rng.normal(size=(nw + 2 * mm, nk ** dim))
    a = O.dual_bubble_direct(G, nw, mm, 3.0, dim, nk)
    b = O.dual_bubble_fft(G, nw, mm, 3.0, dim, nk)
    assert _rel(b, a) < 1e-13


def test_bubble_conjugation_and_particle_hole():
    # g(-w) = g(w)*, real vertices: chi_{-W,-w}(q) = chi_{W,w}(q)*;
    # half filling, t' = 0: Im chi_{W=0}(q) = 0
    w = I.workload("paper_u20", nk=8, n_w=8, m_max=2)
    g0 = O.bare_dual_g(w.g, w.delta, O.dispersion(2, 8, 1.0))
    chi = O.dual_bubble_fft(g0, 8, 2, w.beta, 2, 8)
    assert _rel(chi[::-1, ::-1, :], np.conj(chi)) < 1e-13
    assert np.max(np.abs(chi[2].imag)) < 1e-14 * np.max(np.abs(chi[2]))


def test_planted_bubble_mistake_is_caught(monkeypatch):
    # k - q instead of k + q in the explicit sum: the closed form must fail
    orig = O._shift_index

    def wrong(dim, nk):
        grid = np.indices([nk] * dim).reshape(dim, -1).T
        s = (grid[:, None, :] - grid[None, :, :]) % nk
        flat = np.zeros(s.shape[:2], dtype=np.int64)
        for d in range(dim):
            flat = flat * nk + s[:, :, d]
        return flat

    monkeypatch.setattr(O, "_shift_index", wrong)
    with pytest.raises(AssertionError):
        test_bubble_closed_form_single_harmonic(2, 8, [1, 2])
    monkeypatch.setattr(O, "_shift_index", orig)


# ---------------------------------------------------------------------------
# Eq. lin_alg_inv and Gamma^(2)
# ---------------------------------------------------------------------------

def _random_system(seed, n, rho):
    rng = np.random.default_rng(seed)
    gam = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    chi = rng.normal(size=n) + 1j * rng.normal(size=n)
    r = np.max(np.abs(np.linalg.eigvals(gam * chi[None, :])))
    return gam * (rho / r), chi


def test_ladder_equals_geometric_series():
    # Eq. dual_ladder iterated: Gamma = sum_j (gamma chi)^j gamma, for rho(gamma chi) < 1
    gam, chi = _random_system(3, 12, 0.5)
    series = np.zeros_like(gam)
    term = gam.copy()
    for _ in range(200):
        series += term
        term = (gam * chi[None, :]) @ term
    full = O.ladder_gamma_full(gam, chi)
    assert _rel(full, series) < 1e-13
    # and the batched diagonal path agrees with it
    d = O.ladder_gamma_diag(gam[None], chi[None, :, None])[0, :, 0]
    assert _rel(d, np.diag(series)) < 1e-13


def test_ladder_satisfies_eq_dual_ladder():
    # Gamma = gamma + gamma chi Gamma outside the radius too (any rho)
    gam, chi = _random_system(4, 16, 7.0)
    G = O.ladder_gamma_full(gam, chi)
    assert _rel(gam + (gam * chi[None, :]) @ G, G) < 1e-12


def test_hand_lu_matches_lapack():
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 33):
        a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        b = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        lu, perm = O.lu_partial_pivot(a)
        x = O.lu_solve(lu, perm, b)
        assert _rel(x, np.linalg.solve(a, b)) < 1e-11
        # P A = L U
        L = np.tril(lu, -1) + np.eye(n)
        U = np.triu(lu)
        assert _rel(L @ U, a[perm]) < 1e-13


def test_second_order_diag_direct_sum():
    rng = np.random.default_rng(6)
    nb, n, N = 2, 5, 3
    gam = rng.normal(size=(nb, n, n)) + 1j * rng.normal(size=(nb, n, n))
    chi = rng.normal(size=(nb, n, N)) + 1j * rng.normal(size=(nb, n, N))
    got = O.second_order_diag(gam, chi)
    for a in range(nb):
        for q in range(N):
            for w in range(n):
                s = 0
                for x in range(n):
                    s += gam[a, w, x] * chi[a, x, q] * gam[a, x, w]
                assert abs(got[a, w, q] - s) < 1e-13 * (1 + abs(s))


def test_planted_ladder_order_mistake_is_caught(monkeypatch):
    # (1 - chi gamma) instead of (1 - gamma chi): the series pin must fail
    monkeypatch.setattr(O, "ladder_matrix",
                        lambda g, c: np.eye(g.shape[0]) - c[:, None] * g)
    with pytest.raises(AssertionError):
        test_ladder_equals_geometric_series()


def test_leading_eigenvalue_rank_one():
    # gamma = u v^T: gamma chi has the single nonzero eigenvalue sum_j v_j chi_j u_j
    rng = np.random.default_rng(7)
    n = 9
    u = rng.normal(size=n) + 1j * rng.normal(size=n)
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    chi = rng.normal(size=n) + 1j * rng.normal(size=n)
    lam = O.leading_eigenvalue(np.outer(u, v), chi)
    assert abs(lam - np.sum(v * chi * u)) < 1e-12 * abs(lam)


# ---------------------------------------------------------------------------
# Eq. sd
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,nk,r0", [(1, 8, [3]), (2, 4, [1, 0]), (2, 8, [2, 1]), (3, 4, [1, 0, 1])])
def test_sigma_closed_form_single_harmonic(dim, nk, r0):
    # K(q) = al + be e^{iq.r0}, G~(k) = a + b e^{ik.r0} + c e^{-ik.r0}:
    # sum_q K(q) G~(k+q) = N [al a + be c e^{-ik.r0}]  (2 r0 != 0 mod grid)
    rng = np.random.default_rng(12)
    nw, mm, beta = 4, 1, 1.5
    nb, ne = 2 * mm + 1, nw + 2 * mm
    G, (a, b, c), k = _harmonic_g(rng, ne, dim, nk, r0)
    ph = np.exp(1j * (k @ np.asarray(r0, float)))
    al = rng.normal(size=(nb, nw)) + 1j * rng.normal(size=(nb, nw))
    be = rng.normal(size=(nb, nw)) + 1j * rng.normal(size=(nb, nw))
    kern = al[:, :, None] + be[:, :, None] * ph[None, None, :]
    T = 1.0 / beta
    expect = np.zeros((nw, nk ** dim), complex)
    for i in range(nw):
        for A in range(nb):
            expect[i] += (T / 2) * (al[A, i] * a[i + A] + be[A, i] * c[i + A] * np.conj(ph))
    for fn in (O.dual_sigma_direct, O.dual_sigma_fft):
        assert _rel(fn(kern, G, nw, mm, beta, dim, nk), expect) < 1e-13


@pytest.mark.parametrize("dim,nk", [(1, 8), (2, 4), (3, 4), (4, 2)])
def test_sigma_direct_vs_fft(dim, nk):
    rng = np.random.default_rng(dim + 40)
    nw, mm = 4, 1
    N = nk ** dim
    G = rng.normal(size=(nw + 2 * mm, N)) + 1j * rng.normal(size=(nw + 2 * mm, N))
    K = rng.normal(size=(2 * mm + 1, nw, N)) + 1j * rng.normal(size=(2 * mm + 1, nw, N))
    assert _rel(O.dual_sigma_fft(K, G, nw, mm, 2.0, dim, nk),
                O.dual_sigma_direct(K, G, nw, mm, 2.0, dim, nk)) < 1e-13


def test_zero_vertex_gives_zero_sigma():
    # gamma = 0: Sigma~ == 0 and G~ = G_DMFT - g for every iteration
    w = I.workload("square32_tp", nk=8, n_w=8, m_max=2).scaled(0.0)
    st = O.run_workload(w, n_iter=3)
    assert np.all(st.sigma == 0)
    eps = O.dispersion(2, 8, 1.0, w.tp)
    assert _rel(st.gt_ext, O.bare_dual_g(w.g, w.delta, eps)) < 1e-14


def _one_shot_sigma(w, s):
    eps = O.dispersion(w.dim, w.nk, w.t, w.tp)
    g0 = O.bare_dual_g(w.g, w.delta, eps)
    gd, gm = O.channel_vertices(s * w.gamma_uu, s * w.gamma_ud)
    st = O.LoopState(g0_ext=g0, sigma=np.zeros((w.n_w, w.N), complex))
    sig, _ = O.one_iteration(st, gd, gm, w.n_w, w.m_max, w.beta, w.dim, w.nk)
    return sig, g0


def test_sigma_first_and_second_order_in_vertex():
    """Richardson extrapolation in the vertex scale s.

    O(s):   (T/2) sum_W (3 gm + gd)_{W,w,w} G~loc_{w+W}     (local)
    O(s^2): T/(2N) sum_{W,q} (1/2)(3 gm chi gm + gd chi gd)_{ww}(q) G~_{w+W,k+q}
            (the second-order diagram, explicit sums)."""
    w = I.random_nonsymmetric(n_w=4, m_max=1, dim=2, nk=4, seed=21)
    nb, nw, N, beta = w.n_bos, w.n_w, w.N, w.beta
    T = 1.0 / beta
    g0 = O.bare_dual_g(w.g, w.delta, O.dispersion(2, 4, 1.0))
    chi = O.dual_bubble_direct(g0, nw, w.m_max, beta, 2, 4)
    gd, gm = w.gamma_uu + w.gamma_ud, w.gamma_uu - w.gamma_ud
    rho = max(np.max(np.abs(np.linalg.eigvals(gx[a] * chi[a, :, q][None, :])))
              for gx in (gd, gm) for a in range(nb) for q in range(N))
    h = 0.02 / rho
    pts = h * np.array([-3, -2, -1, 1, 2, 3], float)
    vals = np.stack([_one_shot_sigma(w, s)[0] for s in pts])          # [6][nw][N]
    V = np.stack([pts ** p for p in range(1, 7)], axis=1)              # f(0) = 0 exactly
    coef = np.linalg.solve(V, vals.reshape(6, -1)).reshape(6, nw, N)
    s1, s2 = coef[0], coef[1]

    gloc = g0.mean(axis=1)
    e1 = np.zeros((nw, N), complex)
    for i in range(nw):
        for A in range(nb):
            e1[i] += 0.5 * T * (3 * gm[A, i, i] + gd[A, i, i]) * gloc[i + A]
    assert _rel(s1, e1) < 1e-9

    kq = O._shift_index(2, 4)
    e2 = np.zeros((nw, N), complex)
    for i in range(nw):
        for k in range(N):
            tot = 0
            for A in range(nb):
                for q in range(N):
                    d2 = 0
                    for x in range(nw):
                        d2 += 3 * gm[A, i, x] * chi[A, x, q] * gm[A, x, i]
                        d2 += gd[A, i, x] * chi[A, x, q] * gd[A, x, i]
                    tot += 0.5 * d2 * g0[i + A, kq[k, q]]
            e2[i, k] = T / (2 * N) * tot
    assert _rel(s2, e2) < 1e-7


def test_planted_double_counting_mistake_is_caught(monkeypatch):
    # dropping the -Gamma^(2)/2 of Eq. sd changes the O(s^2) term
    monkeypatch.setattr(O, "sd_kernel", lambda gd, gd2, gm, gm2: 3.0 * gm + gd)
    with pytest.raises(AssertionError):
        test_sigma_first_and_second_order_in_vertex()


def _loop(name, n_iter, **kw):
    w = I.workload(name, **kw)
    return w, O.run_workload(w, n_iter=n_iter)


def test_sigma_conjugation_symmetry():
    # g(-w) = g(w)*, Delta likewise, real vertices: Sigma~(k,-w) = Sigma~(k,w)*
    w, st = _loop("square32_tp", 3, nk=8, n_w=8, m_max=2)
    s = st.sigma
    assert _rel(s[::-1], np.conj(s)) < 1e-12


def test_sigma_point_group():
    # D4 of the square lattice (t' included): transpose and k -> -k
    w, st = _loop("square32_tp", 2, nk=8, n_w=8, m_max=2)
    s = st.sigma.reshape(8, 8, 8)
    assert _rel(s.transpose(0, 2, 1), s) < 1e-12
    flip = s[:, (-np.arange(8)) % 8, :]
    assert _rel(flip, s) < 1e-12
    # O_h of the cubic lattice: axis permutations
    w3 = I.half_filled_atom("c", 3, 4, U=2.0, beta=2.0, n_w=4, m_max=1)
    s3 = O.run_workload(w3, n_iter=2).sigma.reshape(4, 4, 4, 4)
    assert _rel(s3.transpose(0, 2, 3, 1), s3) < 1e-12
    assert _rel(s3.transpose(0, 1, 3, 2), s3) < 1e-12


def test_sigma_particle_hole():
    # half filling, t' = 0: Sigma~(k+Q, w) = -Sigma~(k, w)*
    w, st = _loop("paper_u20", 3, nk=8, n_w=8, m_max=1)
    s = st.sigma.reshape(8, 8, 8)
    shifted = np.roll(s, (4, 4), axis=(1, 2))
    assert _rel(shifted, -np.conj(s)) < 1e-12


def test_paper_workload_converges():
    # the paper's Example I input (U=20, beta=1) is inside the ladder radius and
    # the loop contracts; the residual falls geometrically
    w, st = _loop("paper_u20", 12, nk=8, n_w=16, m_max=1)
    r = st.residuals
    assert r[-1] < 1e-10
    assert all(r[i + 1] < r[i] for i in range(len(r) - 1) if r[i] > 1e-13)


def test_cubic_workload_sits_at_lambda_098():
    # the 3D 16^3 workload's beta puts the leading magnetic eigenvalue of
    # gamma chi~ at (pi,pi,pi), W=0 at 0.98, just inside the ladder radius
    import json
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    gold = json.load(open(os.path.join(here, "golden", "cubic16_beta.json")))
    assert gold["beta"] == I.CUBIC16_BETA_LAMBDA098
    w = I.workload("cubic16_crit", m_max=0)
    g0 = O.bare_dual_g(w.g, w.delta, O.dispersion(3, 16, 1.0))
    chi = O.dual_bubble_fft(g0, w.n_w, 0, w.beta, 3, 16)
    _, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    q = 8 * 256 + 8 * 16 + 8
    lam = O.ladder_lambda(gm, chi, 0, q)
    assert abs(lam - 0.98) < 1e-9


# ---------------------------------------------------------------------------
# section "Resulting observables": Eq. sigma_lat, Eq. glat
# ---------------------------------------------------------------------------

def _obs_inputs(seed=7, dim=2, nk=4, n_w=6, m_max=1):
    w = I.random_nonsymmetric(n_w, m_max, dim, nk, seed=seed, beta=1.7)
    eps = O.dispersion(dim, nk, 1.0, 0.0)
    return w, eps


def test_lattice_observables_dmft_limit():
    # Sigma~ = 0: G_lat is the DMFT lattice Green's function 1/(1/g + Delta - eps)
    # (a different formula from Eq. glat) and Sigma_lat = Sigma^DMFT
    w, eps = _obs_inputs()
    zero = np.zeros((w.n_w, w.N), complex)
    s_lat, g_lat = O.lattice_observables(w.g, w.delta, eps, zero, w.n_w, w.m_max, w.beta, w.mu)
    box = slice(w.m_max, w.m_max + w.n_w)
    g, d = w.g[box][:, None], w.delta[box][:, None]
    g_dmft = 1.0 / (1.0 / g + d - eps[None, :])
    assert np.max(np.abs(g_lat - g_dmft)) / np.max(np.abs(g_dmft)) < 1e-13
    iw = 1j * O.matsubara_box(w.n_w, w.beta)[:, None]
    assert np.max(np.abs(s_lat - (iw + w.mu - d - 1.0 / g))) < 1e-12


def test_lattice_observables_obey_dyson():
    # the paper: Eqs. sigma_lat and glat are related by a Dyson equation for G and
    # Sigma, G^-1 = i w + mu - eps_k - Sigma, for any Sigma~
    w, eps = _obs_inputs(seed=11)
    rng = np.random.default_rng(3)
    sig = 0.3 * (rng.normal(size=(w.n_w, w.N)) + 1j * rng.normal(size=(w.n_w, w.N)))
    s_lat, g_lat = O.lattice_observables(w.g, w.delta, eps, sig, w.n_w, w.m_max, w.beta, w.mu)
    iw = 1j * O.matsubara_box(w.n_w, w.beta)[:, None]
    lhs = 1.0 / g_lat
    rhs = iw + w.mu - eps[None, :] - s_lat
    assert np.max(np.abs(lhs - rhs)) / np.max(np.abs(rhs)) < 1e-12


def test_printed_sigma_lat_sign_breaks_dyson(monkeypatch):
    # the printed denominator 1 - g Sigma~ (planted in the oracle) violates the
    # Dyson relation: the reading 1 + g Sigma~ is forced
    w, eps = _obs_inputs(seed=13)
    rng = np.random.default_rng(5)
    sig = 0.3 * (rng.normal(size=(w.n_w, w.N)) + 1j * rng.normal(size=(w.n_w, w.N)))
    orig = O.lattice_observables

    def planted(g_ext, delta_ext, eps_, sigma_box, n_w, m_max, beta, mu):
        s_lat, g_lat = orig(g_ext, delta_ext, eps_, sigma_box, n_w, m_max, beta, mu)
        g = g_ext[m_max:m_max + n_w][:, None]
        s_lat = s_lat - sigma_box / (1.0 + g * sigma_box) + sigma_box / (1.0 - g * sigma_box)
        return s_lat, g_lat

    monkeypatch.setattr(O, "lattice_observables", planted)
    s_lat, g_lat = O.lattice_observables(w.g, w.delta, eps, sig, w.n_w, w.m_max, w.beta, w.mu)
    iw = 1j * O.matsubara_box(w.n_w, w.beta)[:, None]
    rhs = iw + w.mu - eps[None, :] - s_lat
    assert np.max(np.abs(1.0 / g_lat - rhs)) / np.max(np.abs(rhs)) > 1e-3


def test_example_i_extrapolation_recovers_the_limit():
    # the N_x -> infinity extrapolation of the Example I sweeps: exact for
    # g(N) = g_inf + b / N, and delta_g follows Eq. deltag
    from paper_1507_00895_gb300 import sweeps as S
    ns = [8, 16, 24, 32, 48]
    g_inf = 0.3 - 0.7j
    gs = [g_inf + (0.2 + 0.1j) / n for n in ns]
    assert abs(S.extrapolate(ns, gs) - g_inf) < 1e-14
    d = S.delta_g(gs, g_inf)
    assert all(abs(d[i] - abs(0.2 + 0.1j) / ns[i] / abs(g_inf)) < 1e-14 for i in range(len(ns)))
    gt = np.zeros((10, 4), complex)
    gt[1 + 4, 0] = 2 + 3j      # m_max = 1, n_w = 8: box index n_w/2 is the first w > 0
    assert S.control_value(gt, 8, 1) == 2 + 3j
    assert abs(O.matsubara_box(8, 1.0)[4] - np.pi) < 1e-15


# ---------------------------------------------------------------------------
# section "Resulting observables": charge and spin susceptibilities
# ---------------------------------------------------------------------------

def _sus(w, eps, sigma, gd, gm):
    return O.susceptibilities(w.g, w.delta, eps, sigma, gd, gm, w.n_w, w.m_max, w.beta, w.dim, w.nk)


# Each pin of the susceptibilities is a function returning its error measure, so
# that the planted-mistake tests below can show which pin a mistake breaks.

def pin_flat_band(nk=4):
    """t = 0: G_lat = 1/(1/g + Delta) for every k, so the bare term is the atom's
    -T sum_w G_w G_{w+W}, independent of q and of N (an extensive sum would not be).
    Returns max over W of max |chi - ref| / |ref| (vertex = 0)."""
    w = I.workload("paper_u20", nk=nk, n_w=8, m_max=2)
    eps = np.zeros(w.N)
    zero_g = np.zeros_like(O.channel_vertices(w.gamma_uu, w.gamma_ud)[0])
    chi = _sus(w, eps, np.zeros((w.n_w, w.N), complex), zero_g, zero_g)
    gl = 1.0 / (1.0 / w.g + w.delta)
    T = 1.0 / w.beta
    err = 0.0
    for a in range(w.n_bos):
        ref = -T * sum(gl[i + w.m_max] * gl[i + a] for i in range(w.n_w))
        err = max(err, float(np.max(np.abs(chi[:, a, :] - ref)) / abs(ref)))
    return err


def pin_frak_closed_form(seed=21):
    """frakG at Sigma~ != 0 against a closed form that follows from Eqs. gd0, dyson
    and glat: with A = (Delta - eps)^-1, G0~ + g = (1/g + Delta - eps)^-1 gives
    (G0~ + g)/G0~ = -A/g, so frakG = -A g^-1 G~ = g (1 - (Delta - eps) G), G from
    Eq. glat.  Non-symmetric random inputs; returns max |frakG - ref| / max |ref|."""
    w = I.random_nonsymmetric(6, 1, 2, 4, seed=seed)
    eps = O.dispersion(2, 4, 1.0, 0.0)
    rng = np.random.default_rng(seed + 1)
    sig = 0.3 * (rng.normal(size=(6, 16)) + 1j * rng.normal(size=(6, 16)))
    g_lat, frak = O.lattice_planes_ext(w.g, w.delta, eps, sig, 6, 1)
    # G (Eq. glat) written out with G~ from Eq. gd0 and Eq. dyson, independently of the oracle
    g = w.g[:, None]
    a = 1.0 / (w.delta[:, None] - eps[None, :])
    g0 = 1.0 / (1.0 / g + w.delta[:, None] - eps[None, :]) - g
    gt = g0.copy()
    gt[1:7] = 1.0 / (1.0 / g0[1:7] - sig)
    g_ref = a + a * gt * a / (g * g)
    ref = g * (1.0 - (w.delta[:, None] - eps[None, :]) * g_ref)
    return max(float(np.max(np.abs(frak - ref)) / np.max(np.abs(ref))),
               float(np.max(np.abs(g_lat - g_ref)) / np.max(np.abs(g_ref))))


def pin_brute_force():
    """Non-symmetric inputs, tiny grid: L and the bare term by explicit k sums of
    G (Eq. glat) and frakG from their closed forms, Gamma by an explicit inverse,
    L Gamma L by a double loop.  Returns the largest relative deviation."""
    w = I.random_nonsymmetric(4, 1, 2, 2, seed=23, scale=0.2)
    eps = O.dispersion(2, 2, 1.0, 0.0)
    rng = np.random.default_rng(9)
    sig = 0.2 * (rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)))
    gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    chi = _sus(w, eps, sig, gd, gm)
    g = w.g[:, None]
    a = 1.0 / (w.delta[:, None] - eps[None, :])
    g0 = 1.0 / (1.0 / g + w.delta[:, None] - eps[None, :]) - g
    gt = g0.copy()
    gt[1:5] = 1.0 / (1.0 / g0[1:5] - sig)
    g_lat = a + a * gt * a / (g * g)
    frak = -a * gt / g
    chi0 = O.dual_bubble_direct(g_lat, 4, 1, w.beta, 2, 2).sum(axis=1)
    L = O.dual_bubble_direct(frak, 4, 1, w.beta, 2, 2)
    ct = O.dual_bubble_direct(gt, 4, 1, w.beta, 2, 2)
    err = 0.0
    for c, gam in enumerate((gd, gm)):
        for aa in range(3):
            for q in range(4):
                Gam = np.linalg.inv(np.eye(4) - gam[aa] * ct[aa, :, q][None, :]) @ gam[aa]
                s = sum(L[aa, i, q] * Gam[i, j] * L[aa, j, q] for i in range(4) for j in range(4))
                err = max(err, abs(chi[c, aa, q] - (chi0[aa, q] + s)) / max(1.0, abs(chi[c, aa, q])))
    zero = np.zeros_like(gd)
    chi_z = _sus(w, eps, sig, zero, zero)
    err = max(err, float(np.max(np.abs(chi_z - chi0[None]))))
    return err


def pin_first_order():
    """chi(e gamma) = chi0 + e L^T gamma L + O(e^2): the ladder enters as gamma at
    first order; L from the closed form of frakG.  Returns the relative deviation
    of the Richardson-extrapolated first-order coefficient."""
    w = I.workload("paper_u20", nk=4, n_w=4, m_max=1)
    eps = O.dispersion(2, 4, 1.0, 0.0)
    sig = np.zeros((4, 16), complex)
    gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    base = _sus(w, eps, sig, 0 * gd, 0 * gm)
    e1, e2 = 1e-4, 2e-4
    d1 = (_sus(w, eps, sig, e1 * gd, e1 * gm) - base) / e1
    d2 = (_sus(w, eps, sig, e2 * gd, e2 * gm) - base) / e2
    first = 2 * d1 - d2                                   # Richardson: O(e^2) removed
    g = w.g[:, None]
    gt = 1.0 / (1.0 / g + w.delta[:, None] - eps[None, :]) - g     # Sigma~ = 0: G~ = G0~
    frak = -gt / (g * (w.delta[:, None] - eps[None, :]))
    L = O.dual_bubble_direct(frak, 4, 1, w.beta, 2, 4)
    err = 0.0
    for c, gam in enumerate((gd, gm)):
        ref = np.einsum("aiq,aij,ajq->aq", L, gam, L)
        err = max(err, float(np.max(np.abs(first[c] - ref)) / np.max(np.abs(ref))))
    return err


@pytest.mark.parametrize("nk", [2, 4])
def test_susceptibility_flat_band_closed_form(nk):
    assert pin_flat_band(nk) < 1e-11


def test_frak_g_is_lattice_g_at_zero_dual_self_energy():
    w = I.random_nonsymmetric(6, 1, 2, 4, seed=21)
    eps = O.dispersion(2, 4, 1.0, 0.0)
    g_lat, frak = O.lattice_planes_ext(w.g, w.delta, eps, np.zeros((6, 16), complex), 6, 1)
    g_dmft = 1.0 / (1.0 / w.g[:, None] + w.delta[:, None] - eps[None, :])
    assert np.max(np.abs(frak - g_dmft)) < 1e-12 * np.max(np.abs(g_dmft))
    assert np.max(np.abs(g_lat - g_dmft)) < 1e-12 * np.max(np.abs(g_dmft))


def test_frak_g_closed_form_at_nonzero_dual_self_energy():
    assert pin_frak_closed_form() < 1e-13


def test_susceptibility_brute_force_and_zero_vertex():
    assert pin_brute_force() < 1e-12


def test_susceptibility_first_order_in_the_vertex():
    assert pin_first_order() < 1e-6


# planted mistakes (in the oracle, on the CPU): each breaks the pin named

def test_planted_frak_without_its_factor_fails(monkeypatch):
    orig = O.lattice_planes_ext

    def planted(g_ext, delta_ext, eps, sigma_box, n_w, m_max):
        g_lat, _ = orig(g_ext, delta_ext, eps, sigma_box, n_w, m_max)
        gt = O.dual_g(O.bare_dual_g(g_ext, delta_ext, eps), sigma_box, n_w, m_max)
        return g_lat, gt                                   # frakG = G~, factor dropped

    monkeypatch.setattr(O, "lattice_planes_ext", planted)
    assert pin_frak_closed_form() > 1e-3
    assert pin_brute_force() > 1e-3
    assert pin_first_order() > 1e-3


def test_planted_frak_as_gtilde_plus_g_fails(monkeypatch):
    orig = O.lattice_planes_ext

    def planted(g_ext, delta_ext, eps, sigma_box, n_w, m_max):
        g_lat, _ = orig(g_ext, delta_ext, eps, sigma_box, n_w, m_max)
        gt = O.dual_g(O.bare_dual_g(g_ext, delta_ext, eps), sigma_box, n_w, m_max)
        return g_lat, gt + g_ext[:, None]                  # equal to frakG only at Sigma~ = 0

    monkeypatch.setattr(O, "lattice_planes_ext", planted)
    assert pin_frak_closed_form() > 1e-3
    assert pin_brute_force() > 1e-3


def test_planted_conjugated_l_fails(monkeypatch):
    monkeypatch.setattr(O, "susceptibility_ladder_term", lambda lv, Gam: np.conj(lv) @ Gam @ np.conj(lv))
    assert pin_brute_force() > 1e-3


def test_planted_no_ladder_fails(monkeypatch):
    monkeypatch.setattr(O, "ladder_gamma_full", lambda gamma_W, chi_Wq: np.array(gamma_W))
    # the vertex is scaled down in this pin, so Gamma - gamma is second order: 3e-4
    assert pin_brute_force() > 1e-6


def test_planted_bare_term_from_gtilde_fails(monkeypatch):
    orig = O.lattice_planes_ext

    def planted(g_ext, delta_ext, eps, sigma_box, n_w, m_max):
        _, frak = orig(g_ext, delta_ext, eps, sigma_box, n_w, m_max)
        gt = O.dual_g(O.bare_dual_g(g_ext, delta_ext, eps), sigma_box, n_w, m_max)
        return gt, frak                                    # bare term summed over G~, not G

    monkeypatch.setattr(O, "lattice_planes_ext", planted)
    assert pin_flat_band() > 1e-3
    assert pin_brute_force() > 1e-3


def test_susceptibility_conjugation_symmetry():
    # symmetric atom inputs: chi(-W, q) = chi(W, q)*
    w = I.workload("paper_u20", nk=4, n_w=6, m_max=2)
    eps = O.dispersion(2, 4, 1.0, 0.0)
    gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    st = O.run_workload(w, n_iter=3)
    chi = _sus(w, eps, st.sigma, gd, gm)
    assert np.max(np.abs(chi[:, ::-1, :] - np.conj(chi))) < 1e-11 * np.max(np.abs(chi))


# ---------------------------------------------------------------------------
# mixing (the loop's closing step: Sigma~ <- mix new + (1 - mix) old)
# ---------------------------------------------------------------------------

def test_mixing_first_pass_scales_the_new_self_energy():
    # from Sigma~ = 0 one pass with mix = a gives a * (the unmixed pass): a swapped
    # a <-> 1 - a, or mixing in the wrong order, gives 0.7 instead of 0.3 of it
    w = I.workload("paper_u20", nk=4, n_w=6, m_max=1)
    one = O.run_workload(w, n_iter=1)
    mixed = O.run_workload(w, n_iter=1, mix=0.3)
    assert np.max(np.abs(mixed.sigma - 0.3 * one.sigma)) <= 1e-15 * np.max(np.abs(one.sigma))


def test_mixing_keeps_the_fixed_point():
    # a fixed point of the unmixed map is one of the mixed map: both loops reach the
    # same converged Sigma~, the mixed one more slowly (its contraction is weaker)
    w = I.workload("paper_u20", nk=4, n_w=6, m_max=1)
    a = O.run_workload(w, n_iter=60, tol=1e-14)
    b = O.run_workload(w, n_iter=200, mix=0.3, tol=1e-14)
    assert a.residuals[-1] <= 1e-14 and b.residuals[-1] <= 1e-14
    assert len(b.residuals) > len(a.residuals)
    assert np.max(np.abs(a.sigma - b.sigma)) < 1e-12 * np.max(np.abs(a.sigma))
    # mixed residual: r_k = a max|F(S) - S| / max|S_k|, so a step of the mixed loop
    # moves Sigma~ by exactly 0.3 of the unmixed step from the same state
    st = O.LoopState(g0_ext=O.bare_dual_g(w.g, w.delta, O.dispersion(2, 4, w.t, w.tp)), sigma=b.sigmas[2].copy())
    gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    full, _ = O.one_iteration(O.LoopState(g0_ext=st.g0_ext, sigma=b.sigmas[2].copy()), gd, gm, 6, 1, w.beta, 2, 4)
    part, _ = O.one_iteration(st, gd, gm, 6, 1, w.beta, 2, 4, mix=0.3)
    step_full = full - b.sigmas[2]
    assert np.max(np.abs((part - b.sigmas[2]) - 0.3 * step_full)) < 1e-14 * np.max(np.abs(step_full)) + 1e-17


# ---------------------------------------------------------------------------
# the convergence-radius extension (the remark after Eq. lin_alg_inv)
# ---------------------------------------------------------------------------

def test_radius_extension_is_the_truncated_series_outside_the_radius():
    # config-1-like inputs far outside the radius: every flagged system takes
    # sum_{j <= K} (gamma chi~)^j gamma (explicit matrix powers), the rest the solve
    w = I.workload("square16_b5", nk=4, n_w=8, m_max=2)
    st = O.run_workload(w, n_iter=1)
    gd, _ = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    chi = st.chi
    plain = O.ladder_gamma_diag(gd, chi)
    for K in (1, 3):
        ext = O.ladder_gamma_diag(gd, chi, radius_order=K)
        n_out = 0
        for a in range(w.n_bos):
            for q in range(w.N):
                A = gd[a] * chi[a, :, q][None, :]
                if np.max(np.abs(np.linalg.eigvals(A))) >= 1.0:
                    ref = sum(np.linalg.matrix_power(A, j) @ gd[a] for j in range(K + 1))
                    assert np.max(np.abs(ext[a, :, q] - np.diagonal(ref))) < 1e-10 * np.max(np.abs(ref))
                    n_out += 1
                else:
                    assert np.max(np.abs(ext[a, :, q] - plain[a, :, q])) == 0.0
        assert 0 < n_out < w.n_bos * w.N        # both kinds present


def test_radius_extension_changes_nothing_inside_the_radius():
    w = I.workload("paper_u20", nk=4, n_w=6, m_max=1)
    a = O.run_workload(w, n_iter=3)
    b = O.run_workload(w, n_iter=3, radius_order=2)
    assert np.array_equal(a.sigma, b.sigma)


def test_warm_start_stated_box_lies_beyond_the_ladder_radius():
    # the learned warm start's stated parameter box with the Hubbard-atom inputs
    # (U in [2, 6], beta in [5, 25], mu = U/2 +- 0.5): on the first pass from
    # Sigma~ = 0 the largest |lambda| of gamma chi~ at W = 0 exceeds 1 at every
    # sampled point (the radius remark after Eq. lin_alg_inv), already on an 8^2
    # grid with 16 frequencies; the GPU finds the same at the stated grid
    for w in I.config5_points(8, nk=8, n_w=16, m_max=1):
        st = O.run_workload(w, n_iter=1)
        gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
        lam = max(abs(O.ladder_lambda(g, st.chi, w.m_max, q)) for g in (gd, gm) for q in range(w.N))
        assert lam > 1.0, (w.U, w.beta, lam)
