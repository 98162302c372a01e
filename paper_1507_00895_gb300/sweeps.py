"""The paper's Example I sweeps (section "Example I and performance analysis").

The loop on the atomic-limit inputs (Eqs. atomic_limit1-4, D = 2, U = 20,
mu = U/2, beta = 1, Delta = 2D g) is converged for a range of one control
parameter N_x, x in {W, w, k}, the others fixed as in the paper's three
figures:

  * N_W (bosonic frequencies, 2 m_max + 1) at N_w = 48, N_k = 16;
  * N_w (fermionic frequencies)              at N_W = 3,  N_k = 8;
  * N_k^D (lattice volume)                   at N_W = 3,  N_w = 48.

For each point it records the passes and the wall time to r <= tol from
Sigma~ = 0 and the control value g = G~(i pi / beta, k = (0, 0)), and reports
Eq. deltag, delta_g = |g(N_x) - g(inf)| / |g(inf)|, with g(inf) extrapolated
from the three largest N_x by a straight-line fit in 1 / N_x (the paper
extrapolates without saying how; this is the reading used here).

Everything runs through the public API (DualFermion); the loop is the
library's, on the GPU.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I

# the paper's three sweeps: (name, varied parameter, values, fixed n_w, m_max, nk)
SWEEPS = {
    "bosonic": dict(vary="m_max", values=(0, 1, 2, 3, 4, 5, 6, 8, 10), n_w=48, m_max=None, nk=16),
    "fermionic": dict(vary="n_w", values=(8, 12, 16, 24, 32, 48, 64, 96, 128), n_w=None, m_max=1, nk=8),
    "volume": dict(vary="nk", values=(4, 8, 16, 32, 64), n_w=48, m_max=1, nk=None),
}


def control_value(gt_ext: np.ndarray, n_w: int, m_max: int) -> complex:
    """g = G~ at the first positive Matsubara frequency (box index n_w / 2) and k = 0."""
    return complex(gt_ext[m_max + n_w // 2, 0])


def extrapolate(ns, gs, npts: int = 3) -> complex:
    """g(inf) from a least-squares straight line g = a + b / N over the npts largest N."""
    order = np.argsort(ns)[-npts:]
    x = 1.0 / np.asarray(ns, float)[order]
    y = np.asarray(gs, complex)[order]
    A = np.stack([np.ones_like(x), x], axis=1)
    coef_r = np.linalg.lstsq(A, y.real, rcond=None)[0]
    coef_i = np.linalg.lstsq(A, y.imag, rcond=None)[0]
    return complex(coef_r[0], coef_i[0])


def delta_g(gs, g_inf: complex):
    """Eq. deltag for every point."""
    return [abs(g - g_inf) / abs(g_inf) for g in gs]


def run_point(df, n_w: int, m_max: int, nk: int, precision: int, tol: float = 1e-12, max_iter: int = 80):
    """Converge one point from Sigma~ = 0; the second of two identical runs is timed."""
    w = I.workload("paper_u20", nk=nk, n_w=n_w, m_max=m_max)
    if precision == df.DF_FP32_IR and not df.mixed_supported(n_w):
        precision = df.DF_FP64
    zero = np.zeros((w.n_w, w.N), np.complex128)
    with df.DualFermion.from_workload(w, precision=precision) as d:
        d.iterate(max_iter, tol=tol)
        d.set_sigma(zero)
        d.synchronize()
        t0 = time.perf_counter()
        it, r, status = d.iterate(max_iter, tol=tol)
        d.synchronize()
        dt = time.perf_counter() - t0
        g = control_value(d.get_gtilde(), w.n_w, w.m_max)
    return {"n_w": n_w, "N_W": 2 * m_max + 1, "N_k": nk, "volume": nk ** 2, "passes": it, "resid": r,
            "converged": r <= tol, "seconds": dt, "g": [g.real, g.imag],
            "precision": "fp64" if precision == df.DF_FP64 else "fp32ir"}


def sweep(df, name: str, precision: int, values=None, tol: float = 1e-12):
    """One of the paper's three sweeps; returns the points, g(inf) and delta_g."""
    spec = SWEEPS[name]
    pts = []
    for v in (values or spec["values"]):
        kw = {k: spec[k] for k in ("n_w", "m_max", "nk")}
        kw[spec["vary"]] = v
        pts.append(run_point(df, kw["n_w"], kw["m_max"], kw["nk"], precision, tol))
    key = {"m_max": "N_W", "n_w": "n_w", "nk": "volume"}[spec["vary"]]
    ns = [p[key] for p in pts]
    gs = [complex(*p["g"]) for p in pts]
    g_inf = extrapolate(ns, gs)
    for p, d in zip(pts, delta_g(gs, g_inf)):
        p["delta_g"] = d
    return {"varied": key, "g_inf": [g_inf.real, g_inf.imag], "points": pts}


def example_i(df, precision: int, tol: float = 1e-12):
    """All three sweeps."""
    return {name: sweep(df, name, precision, tol=tol) for name in SWEEPS}
