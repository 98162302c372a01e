"""Seeded synthetic inputs for the ladder dual-fermion loop.

This module only *generates inputs*: the impurity Green's function g(iw),
the hybridisation Delta(iw) and the two spin components of the impurity
vertex, gamma^{uu} and gamma^{ud}, on the frequency grids the loop needs.
It holds none of the dual-fermion arithmetic (no dual propagator, bubble,
ladder, self-energy or Dyson step) and is shared, as plain input, by the
CPU oracle, the tests and the benchmark.

Frequency conventions (used by every array below):

* fermionic Matsubara index n, value w_n = (2n+1) pi / beta;
* the vertex box holds n in [-n_w/2, n_w/2) (box index i = n + n_w/2);
* bosonic index m in [-m_max, m_max], value W_m = 2 m pi / beta
  (bosonic index a = m + m_max, N_W = 2 m_max + 1);
* g and Delta are given on the *extended* fermionic grid
  n in [-n_w/2 - m_max, n_w/2 + m_max) (extended index e = n + n_w/2 + m_max),
  so that w + W is always on the grid;
* vertices are arrays [N_W][n_w][n_w] indexed (a, i, j) <-> (W, w, w').

The closed forms are the Hubbard-atom ("atomic limit") inputs of the
paper's Section "Example I", Eqs. atomic_limit1-atomic_limit4, with
Lambda_w = 1 + U^2 / (4 w^2) and w1 = w, w2 = w + W, w3 = w' + W, w4 = w'.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------

def fermionic_n(n_w: int, m_max: int = 0) -> np.ndarray:
    """Matsubara indices n of the extended fermionic grid (box when m_max=0)."""
    if n_w % 2 or n_w < 2:
        raise ValueError("n_w must be even and >= 2")
    return np.arange(-n_w // 2 - m_max, n_w // 2 + m_max, dtype=np.int64)


def fermionic_w(beta: float, n: np.ndarray) -> np.ndarray:
    """w_n = (2n+1) pi / beta."""
    return (2.0 * np.asarray(n, dtype=np.float64) + 1.0) * math.pi / beta


def bosonic_m(m_max: int) -> np.ndarray:
    return np.arange(-m_max, m_max + 1, dtype=np.int64)


def _logistic_neg(x: float) -> float:
    """1 / (1 + exp(x)) evaluated without overflow."""
    if x >= 0:
        e = math.exp(-x)
        return e / (1.0 + e)
    return 1.0 / (1.0 + math.exp(x))


# --------------------------------------------------------------------------
# Hubbard atom (Eqs. atomic_limit1-4)
# --------------------------------------------------------------------------

def atom_density(U: float, beta: float, mu: float) -> float:
    """Total density of the Hubbard atom H = -mu n + U n_up n_dn."""
    # weights of |0>, |up>/|dn>, |updn>, shifted by the largest exponent
    ex = np.array([0.0, beta * mu, beta * mu, beta * (2 * mu - U)])
    w = np.exp(ex - ex.max())
    return float((w[1] + w[2] + 2.0 * w[3]) / w.sum())


def atom_mu_for_density(U: float, beta: float, n_target: float) -> float:
    """Chemical potential of the Hubbard atom with total density n_target (bisection)."""
    lo, hi = -10.0 * (U + 1.0), 10.0 * (U + 1.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if atom_density(U, beta, mid) < n_target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def atom_g(U: float, beta: float, mu: float, n_w: int, m_max: int) -> np.ndarray:
    """Hubbard-atom g(iw) on the extended grid.

    At half filling (mu = U/2) this is Eq. atomic_limit1,
    g = (1/2)[1/(iw - U/2) + 1/(iw + U/2)].  Away from it the atom's
    occupation <n_sigma> weights the two poles:
    g = (1 - <n_s>)/(iw + mu) + <n_s>/(iw + mu - U).
    """
    iw = 1j * fermionic_w(beta, fermionic_n(n_w, m_max))
    ns = 0.5 * atom_density(U, beta, mu)
    return (1.0 - ns) / (iw + mu) + ns / (iw + mu - U)


def atom_vertices(U: float, beta: float, n_w: int, m_max: int):
    """gamma^{uu}, gamma^{ud} of Eqs. atomic_limit3-4, shape [N_W][n_w][n_w], real.

    Index meaning: (a, i, j) <-> (W_m, w_n, w_n'), m = a - m_max,
    n = i - n_w/2, n' = j - n_w/2.  The Kronecker deltas compare Matsubara
    indices: delta_{w1,w2} <=> m = 0, delta_{w1,w4} <=> n = n',
    delta_{w2,-w3} <=> (n+m) + (n'+m) + 1 = 0.
    """
    nb = fermionic_n(n_w, 0)
    mb = bosonic_m(m_max)
    n = nb[None, :, None]
    npr = nb[None, None, :]
    m = mb[:, None, None]
    w1 = fermionic_w(beta, n + 0 * npr + 0 * m)
    w2 = fermionic_w(beta, n + m + 0 * npr)
    w3 = fermionic_w(beta, npr + m + 0 * n)
    w4 = fermionic_w(beta, npr + 0 * n + 0 * m)

    def lam(w):
        return 1.0 + U * U / (4.0 * w * w)

    d12 = (m == 0) & np.ones_like(w1, dtype=bool)
    d14 = (n == npr) & np.ones_like(w1, dtype=bool)
    d2m3 = ((n + m) + (npr + m) + 1 == 0) & np.ones_like(w1, dtype=bool)
    d12 = d12.astype(np.float64)
    d14 = d14.astype(np.float64)
    d2m3 = d2m3.astype(np.float64)

    pref = beta * U * U / 4.0
    g_uu = pref * (d12 - d14) * lam(w1) * lam(w3)

    f_plus = _logistic_neg(beta * U / 2.0)    # 1/(1+exp(+beta U/2))
    f_minus = _logistic_neg(-beta * U / 2.0)  # 1/(1+exp(-beta U/2))
    s2 = w1 ** 2 + w2 ** 2 + w3 ** 2 + w4 ** 2
    p2 = (w1 ** 2) * (w2 ** 2) * (w3 ** 2) * (w4 ** 2)
    g_ud = (-U
            + (U ** 3 / 8.0) * s2 / p2
            + (3.0 * U ** 5 / 16.0) / (w1 * w2 * w3 * w4)
            + pref * f_plus * (2.0 * d2m3 + d12) * lam(w2) * lam(w3)
            - pref * f_minus * (2.0 * d14 + d12) * lam(w1) * lam(w3))
    return np.ascontiguousarray(g_uu), np.ascontiguousarray(g_ud)


def symmetric_gaussian(rng: np.random.Generator, sigma: float, n_w: int, m_max: int) -> np.ndarray:
    """Real Gaussian vertex perturbation, symmetric in w<->w' and under the
    total sign flip (W, w, w') -> (-W, -w, -w'), shape [N_W][n_w][n_w]."""
    p = rng.normal(0.0, sigma, size=(2 * m_max + 1, n_w, n_w))
    p = 0.5 * (p + p.transpose(0, 2, 1))
    p = 0.5 * (p + p[::-1, ::-1, ::-1])
    return np.ascontiguousarray(p)


def second_moment(dim: int, t: float, tp: float) -> float:
    """<eps_k^2> of eps = -2t sum cos k_i - 4 tp cos kx cos ky (tp only in 2D)."""
    return 2.0 * dim * t * t + (4.0 * tp * tp if dim == 2 else 0.0)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    """One complete input set of the dual-fermion loop (all host numpy)."""
    name: str
    dim: int
    nk: int
    t: float
    tp: float
    U: float
    beta: float
    mu: float
    n_w: int
    m_max: int
    g: np.ndarray          # [n_w + 2 m_max] complex128, extended grid
    delta: np.ndarray      # [n_w + 2 m_max] complex128, extended grid
    gamma_uu: np.ndarray   # [N_W][n_w][n_w] complex128
    gamma_ud: np.ndarray   # [N_W][n_w][n_w] complex128
    n_iter: int = 10

    @property
    def N(self) -> int:
        return self.nk ** self.dim

    @property
    def n_bos(self) -> int:
        return 2 * self.m_max + 1

    @property
    def n_ext(self) -> int:
        return self.n_w + 2 * self.m_max

    def scaled(self, s: float) -> "Workload":
        """Same workload with both vertex components multiplied by s."""
        return dataclasses.replace(self, gamma_uu=self.gamma_uu * s,
                                   gamma_ud=self.gamma_ud * s)


def half_filled_atom(name: str, dim: int, nk: int, U: float, beta: float,
                     n_w: int, m_max: int, t: float = 1.0, tp: float = 0.0,
                     delta_kind: str = "moment", V: float = 1.0,
                     n_iter: int = 10) -> Workload:
    """Half-filled Hubbard-atom input on a hypercubic lattice.

    delta_kind "moment": Delta = <eps^2> g (Eq. atomic_limit2's 2D g for t=1,
    t'=0, generalised); "bath": Delta = V^2 / (iw).
    """
    mu = U / 2.0
    g = atom_g(U, beta, mu, n_w, m_max)
    if delta_kind == "moment":
        delta = second_moment(dim, t, tp) * g
    elif delta_kind == "bath":
        delta = V * V / (1j * fermionic_w(beta, fermionic_n(n_w, m_max)))
    else:
        raise ValueError(delta_kind)
    guu, gud = atom_vertices(U, beta, n_w, m_max)
    return Workload(name, dim, nk, t, tp, U, beta, mu, n_w, m_max, g, delta,
                    guu.astype(np.complex128), gud.astype(np.complex128), n_iter)


# Inverse temperature at which the leading magnetic eigenvalue of gamma chi at
# q = (pi,pi,pi), W = 0 equals 0.98 on the first iteration for the 3D 16^3,
# U = 6, n_w = 96 workload; written by tests/golden/make_golden.py (bisection
# with the CPU oracle) and checked by the oracle pin tests.
CUBIC16_BETA_LAMBDA098 = 1.1678889792226528


def workload(name: str, *, nk: Optional[int] = None, n_w: Optional[int] = None,
             m_max: Optional[int] = None, seed: Optional[int] = None) -> Workload:
    """Named workloads; nk / n_w / m_max override the size for small parity cases.

    * ``square16_b5`` : 2D 16^2, t=1, t'=0, U=2, beta=5, half filling, n_w=32,
      W=0 only, Delta = 1/(iw) (V=1), 10 outer iterations.
    * ``square32_tp`` : 2D 32^2, t=1, t'=-0.2, U=4, beta=10, mu of the atom at
      n=0.9, n_w=64, W=-7..7, Delta = <eps^2> g, vertex = atomic closed form +
      symmetric Gaussian of width 0.05U (seed 2).
    * ``cubic16_crit``: 3D 16^3, t=1, U=6, half filling, beta tuned to
      lambda_m(Q,0) = 0.98, n_w=96, W=-10..10, Delta = 6g.
    * ``paper_u20``   : the paper's Example I workload, 2D 16^2, U=20, beta=1,
      mu=U/2, Delta = 4g, n_w=48, N_W=3.
    """
    if name == "square16_b5":
        w = half_filled_atom(name, 2, nk or 16, U=2.0, beta=5.0, n_w=n_w or 32,
                             m_max=0 if m_max is None else m_max, delta_kind="bath")
        return w
    if name == "square32_tp":
        U, beta, tp = 4.0, 10.0, -0.2
        nw = n_w or 64
        mm = 7 if m_max is None else m_max
        mu = atom_mu_for_density(U, beta, 0.9)
        g = atom_g(U, beta, mu, nw, mm)
        delta = second_moment(2, 1.0, tp) * g
        guu, gud = atom_vertices(U, beta, nw, mm)
        rng = np.random.default_rng(2 if seed is None else seed)
        guu = guu + symmetric_gaussian(rng, 0.05 * U, nw, mm)
        gud = gud + symmetric_gaussian(rng, 0.05 * U, nw, mm)
        return Workload(name, 2, nk or 32, 1.0, tp, U, beta, mu, nw, mm, g, delta,
                        guu.astype(np.complex128), gud.astype(np.complex128))
    if name == "cubic16_crit":
        return half_filled_atom(name, 3, nk or 16, U=6.0, beta=CUBIC16_BETA_LAMBDA098,
                                n_w=n_w or 96, m_max=10 if m_max is None else m_max)
    if name == "paper_u20":
        return half_filled_atom(name, 2, nk or 16, U=20.0, beta=1.0, n_w=n_w or 48,
                                m_max=1 if m_max is None else m_max)
    raise KeyError(name)


def random_nonsymmetric(n_w: int, m_max: int, dim: int, nk: int, seed: int,
                        beta: float = 2.0, scale: float = 1.0) -> Workload:
    """Generic complex inputs with no symmetry, for pins that must see a
    transposed operand or a swapped index: g, Delta with g(-w) = conj g(w)
    not imposed, vertices complex and non-symmetric."""
    rng = np.random.default_rng(seed)
    ne = n_w + 2 * m_max
    w = fermionic_w(beta, fermionic_n(n_w, m_max))
    g = 1.0 / (1j * w + rng.normal(0, 0.5, ne) + 1j * rng.normal(0, 0.2, ne))
    delta = rng.normal(0, 0.5, ne) + 1j * rng.normal(0, 0.5, ne)
    shape = (2 * m_max + 1, n_w, n_w)
    guu = scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))
    gud = scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))
    return Workload("random", dim, nk, 1.0, 0.0, 1.0, beta, 0.5, n_w, m_max,
                    g, delta, guu, gud)


def uneven_batch(npts: int = 64, seed: int = 4, max_n_w: int = 128, max_m: int = 15,
                 grids=((2, 8), (2, 16), (2, 32), (2, 64), (4, 8))):
    """The uneven batch of parameter points: U ~ U[1, 8], beta ~ U[2, 20],
    lattice drawn from `grids` ((dim, N_k) pairs; default 8^2, 16^2, 32^2,
    64^2 and 8^4), n_w in {16, 24, ..., max_n_w}, N_W = 2m + 1 with
    m in {0..max_m}; half-filled Hubbard-atom inputs with Delta = <eps^2> g.
    Smaller max_n_w / max_m / grids give the same recipe at test sizes."""
    rng = np.random.default_rng(seed)
    out = []
    nws = list(range(16, max_n_w + 1, 8))
    for i in range(npts):
        U = float(rng.uniform(1.0, 8.0))
        beta = float(rng.uniform(2.0, 20.0))
        dim, nk = grids[int(rng.integers(0, len(grids)))]
        n_w = int(nws[int(rng.integers(0, len(nws)))])
        m = int(rng.integers(0, max_m + 1))
        out.append(half_filled_atom(f"batch{i}", dim, nk, U=U, beta=beta, n_w=n_w, m_max=m))
    return out


def config5_points(npts: int, seed0: int = 5000, nk: int = 64, n_w: int = 128, m_max: int = 15):
    """Parameter points of the learned-warm-start workload at its stated size:
    2D 64^2, n_w = 128, N_W = 31, U ~ U[2, 6], beta ~ U[5, 25], t' ~ U[-0.3, 0],
    mu = U/2 + U[-0.5, 0.5]; point i from numpy's default_rng(seed0 + i); g of
    the atom at mu, the half-filled closed-form vertex, Delta = <eps^2> g."""
    out = []
    for i in range(npts):
        rng = np.random.default_rng(seed0 + i)
        u = float(rng.uniform(2.0, 6.0))
        b = float(rng.uniform(5.0, 25.0))
        t2 = float(rng.uniform(-0.3, 0.0))
        mu = u / 2.0 + float(rng.uniform(-0.5, 0.5))
        g = atom_g(u, b, mu, n_w, m_max)
        delta = second_moment(2, 1.0, t2) * g
        guu, gud = atom_vertices(u, b, n_w, m_max)
        out.append(Workload(f"c5_{seed0 + i}", 2, nk, 1.0, t2, u, b, mu, n_w, m_max, g, delta,
                            guu.astype(np.complex128), gud.astype(np.complex128)))
    return out


def warmstart_family(npts: int, seed: int, nk: int = 16, n_w: int = 16, m_max: int = 1,
                     U=(12.0, 28.0), beta=(0.6, 1.4), tp=(-0.3, 0.0), dmu=(-1.0, 1.0)):
    """Parameter points of the learned warm start: Hubbard-atom inputs around
    the paper's Example I (U ~ U[12, 28], beta ~ U[0.6, 1.4], t' ~ U[-0.3, 0],
    mu = U/2 + U[-1, 1]) on a 2D N_k^2 lattice; g of the atom at mu, the
    half-filled closed-form vertex, Delta = <eps^2> g.  The loop converges
    for this family (8-17 passes to r <= 1e-10 on 8^2)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(npts):
        u = float(rng.uniform(*U))
        b = float(rng.uniform(*beta))
        t2 = float(rng.uniform(*tp))
        mu = u / 2.0 + float(rng.uniform(*dmu))
        g = atom_g(u, b, mu, n_w, m_max)
        delta = second_moment(2, 1.0, t2) * g
        guu, gud = atom_vertices(u, b, n_w, m_max)
        out.append(Workload(f"ws{seed}_{i}", 2, nk, 1.0, t2, u, b, mu, n_w, m_max, g, delta,
                            guu.astype(np.complex128), gud.astype(np.complex128)))
    return out
