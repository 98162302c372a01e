"""The CPU oracle's pass over a large workload with its bosonic planes spread
over a pool of spawned worker processes (test infrastructure; the oracle's
arithmetic is unchanged: each worker runs oracle.df_oracle on one plane)."""
import multiprocessing as mp
import os

import numpy as np


def _plane(args):
    gd_a, gm_a, chi_a = args
    from oracle import df_oracle as O
    dd = O.ladder_gamma_diag(gd_a, chi_a)
    mm = O.ladder_gamma_diag(gm_a, chi_a)
    kd = dd - 0.5 * O.second_order_diag(gd_a, chi_a)
    km = 3.0 * (mm - 0.5 * O.second_order_diag(gm_a, chi_a))
    return kd, km


def first_pass(w):
    """One oracle pass from Sigma~ = 0: returns (sigma [n_w][N], kernel [2][N_W][n_w][N])."""
    from oracle import df_oracle as O
    eps = O.dispersion(w.dim, w.nk, w.t, w.tp)
    g0 = O.bare_dual_g(w.g, w.delta, eps)
    gd, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    gt = O.dual_g(g0, np.zeros((w.n_w, w.N), complex), w.n_w, w.m_max)
    chi = O.dual_bubble_fft(gt, w.n_w, w.m_max, w.beta, w.dim, w.nk)
    workers = max(1, min(os.cpu_count() or 1, w.n_bos))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_plane, [(gd[a:a + 1], gm[a:a + 1], chi[a:a + 1]) for a in range(w.n_bos)])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    kd = np.concatenate([p[0] for p in parts], axis=0)
    km = np.concatenate([p[1] for p in parts], axis=0)
    kern = np.stack([kd, km])
    sig = O.dual_sigma_fft(kd + km, gt, w.n_w, w.m_max, w.beta, w.dim, w.nk)
    return sig, kern
