"""Write the stored values under tests/golden/ from the CPU oracle only.

cubic16_beta.json: the inverse temperature beta* at which the leading
magnetic eigenvalue of gamma^m chi~ at q = (pi,pi,pi), W = 0, on the first
pass of the loop (G~ = G0~), equals 0.98 for the 3D 16^3 lattice, t = 1,
U = 6, half filling, Delta = 6 g, n_w = 96 (bisection on beta).  The ladder
approaches its convergence radius (the paper's condition that the leading
eigenvalue of gamma chi~ stay below one) at this point.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import df_oracle as O                      # noqa: E402
from paper_1507_00895_gb300 import inputs as I         # noqa: E402


def lambda_m_Q(beta, dim=3, nk=16, U=6.0, n_w=96):
    w = I.half_filled_atom("c3", dim, nk, U=U, beta=beta, n_w=n_w, m_max=0)
    g0 = O.bare_dual_g(w.g, w.delta, O.dispersion(dim, nk, 1.0))
    chi = O.dual_bubble_fft(g0, n_w, 0, beta, dim, nk)
    _, gm = O.channel_vertices(w.gamma_uu, w.gamma_ud)
    q = sum((nk // 2) * nk ** d for d in range(dim))      # (pi, pi, pi)
    return O.ladder_lambda(gm, chi, 0, q)


def bisect_beta(target=0.98, lo=0.5, hi=3.0, steps=40):
    flo = abs(lambda_m_Q(lo)) - target
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        f = abs(lambda_m_Q(mid)) - target
        if (f < 0) == (flo < 0):
            lo, flo = mid, f
        else:
            hi = mid
    return 0.5 * (lo + hi)


if __name__ == "__main__":
    b = bisect_beta()
    lam = lambda_m_Q(b)
    out = {"beta": b, "lambda_m_Q": [lam.real, lam.imag], "target": 0.98,
           "lattice": "3D 16^3, t=1, U=6, half filling, Delta=6g, n_w=96, first pass"}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "cubic16_beta.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)
