"""Learned warm start of the dual self-energy.

Pipeline (every numerical step on the GPU through libdf):
  1. generate: converged Sigma~ of many parameter points with the batched
     loop (df_batch_*), or one handle at a time with the point-group
     reduction where a point's grid is too large to batch (generate_each);
     points that do not converge are dropped;
  2. train: the 4-layer network (df_mlp_*) on (features -> Sigma~ on the
     irreducible wedge of the square lattice, positive frequencies),
     inputs and targets standardised per component;
  3. use: predict, expand to the whole grid (df_warmstart_sigma), iterate
     from there; the plain iteration from Sigma~ = 0 is the fallback and the
     yardstick for the prediction's error.
Host code here only builds feature vectors and index maps.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import df


def features(w) -> np.ndarray:
    """[U/20, beta, mu - U/2, t', Re/Im g(iw_n), Re/Im Delta(iw_n) for w_n > 0]."""
    half = w.n_w // 2
    pos = slice(w.m_max + half, w.m_max + w.n_w)
    g, dl = w.g[pos], w.delta[pos]
    return np.concatenate([[w.U / 20.0, w.beta, w.mu - w.U / 2.0, w.tp],
                           g.real, g.imag, dl.real, dl.imag]).astype(np.float32)


def wedge(nk: int):
    """(kmap [N] int32: wedge index of every momentum, rep [n_wedge]: a
    momentum of each wedge class) for the D4 group of the nk x nk grid."""
    h = nk // 2
    kmap = np.empty(nk * nk, np.int32)
    rep = {}
    for jx in range(nk):
        for jy in range(nk):
            a, b = min(jx, nk - jx), min(jy, nk - jy)
            a, b = max(a, b), min(a, b)
            idx = a * (a + 1) // 2 + b
            kmap[jx * nk + jy] = idx
            rep.setdefault(idx, jx * nk + jy)
    n_wedge = (h + 1) * (h + 2) // 2
    return kmap, np.array([rep[i] for i in range(n_wedge)], np.int64)


def targets(sigma: np.ndarray, n_w: int, rep: np.ndarray) -> np.ndarray:
    """Sigma~ [n_w][N] -> [n_wedge][n_w/2][2] float32 (w_n > 0)."""
    half = n_w // 2
    s = sigma[half:, :][:, rep].T             # [n_wedge][half]
    return np.stack([s.real, s.imag], axis=-1).astype(np.float32)


def generate(workloads, precision=df.DF_FP64, tol: float = 1e-10, max_iter: int = 60, chunk: int = 256):
    """Converged Sigma~ of every workload by the batched loop.
    Returns (X [n][n_in], Y [n][n_out], passes [n], converged mask [n])."""
    kmap, rep = wedge(workloads[0].nk)
    X, Y, passes, ok = [], [], [], []
    for i0 in range(0, len(workloads), chunk):
        ws = workloads[i0:i0 + chunk]
        with df.DualFermionBatch(ws, precision=precision, tol=tol) as b:
            it, r, act, _ = b.iterate(max_iter)
            for j, w in enumerate(ws):
                conv = bool(act[j] == 0)
                ok.append(conv)
                X.append(features(w))
                Y.append(targets(b.get_sigma(j), w.n_w, rep).reshape(-1) if conv else None)
        passes.extend([it] * len(ws))
    mask = np.array(ok)
    Xa = np.stack([x for x, m in zip(X, mask) if m])
    Ya = np.stack([y for y, m in zip(Y, mask) if m])
    return Xa, Ya, np.array(passes), mask


def generate_each(workloads, precision=df.DF_FP32_IR, symmetry: int = 2, tol: float = 1e-8,
                  max_iter: int = 60):
    """Converged Sigma~ of every workload, one handle at a time: the stated
    warm-start grid (64^2, n_w = 128, N_W = 31) holds about 1 GB of device
    arrays per point, too much to batch.  With symmetry = 2 the reductions
    solve 561 of the 4096 momenta on 16 of the 31 planes.  Returns (X, Y,
    passes [n], converged
    mask [n]); a point whose loop does not reach r <= tol in max_iter passes,
    or fails, is dropped."""
    _, rep = wedge(workloads[0].nk)
    X, Y, passes, ok = [], [], [], []
    for w in workloads:
        conv, it, y, r = False, 0, None, float("inf")
        try:
            with df.DualFermion.from_workload(w, precision=precision, eig_mode=0, symmetry=symmetry) as d:
                for it in range(1, max_iter + 1):   # pass by pass: a diverging point stops early
                    d.bubble()
                    d.bse(3)
                    r = d.sigma()
                    if r <= tol or not (r < 1e3):
                        break
                conv = bool(r <= tol)
                if conv:
                    y = targets(d.get_sigma(), w.n_w, rep).reshape(-1)
        except df.DFError:
            conv = False
        ok.append(conv)
        passes.append(it)
        if conv:
            X.append(features(w))
            Y.append(y)
    Xa = np.stack(X) if X else np.zeros((0, 0), np.float32)
    Ya = np.stack(Y) if Y else np.zeros((0, 0), np.float32)
    return Xa, Ya, np.array(passes), np.array(ok)


@dataclass
class Standardiser:
    mean: np.ndarray
    sd: np.ndarray

    @classmethod
    def fit(cls, a):
        m = a.mean(axis=0)
        s = a.std(axis=0)
        return cls(m.astype(np.float32), np.where(s > 1e-12, s, 1.0).astype(np.float32))

    def __call__(self, a):
        return ((a - self.mean) / self.sd).astype(np.float32)


class WarmStart:
    """A trained network plus its standardisers and the wedge map."""

    def __init__(self, n_in: int, n_out: int, nk: int, width: int = 512, max_batch: int = 256, seed: int = 0):
        import torch
        self.torch = torch
        self.net = df.MLP(n_in, n_out, width=width, max_batch=max_batch, seed=seed)
        self.max_batch = max_batch
        kmap, _ = wedge(nk)
        self.kmap = torch.from_numpy(kmap).cuda()
        self.xs = self.ys = None

    def train(self, X, Y, steps: int = 2000, batch: int = 256, lr: float = 1e-3, seed: int = 0, log_every: int = 0):
        torch = self.torch
        self.xs, self.ys = Standardiser.fit(X), Standardiser.fit(Y)
        xd = torch.from_numpy(self.xs(X)).cuda()
        yd = torch.from_numpy(self.ys(Y)).cuda()
        rng = np.random.default_rng(seed)
        n = xd.shape[0]
        b = min(batch, n, self.max_batch)
        hist = []
        for s in range(steps):
            idx = torch.from_numpy(rng.choice(n, size=b, replace=False)).cuda()
            want = log_every and (s % log_every == 0 or s == steps - 1)
            loss = self.net.train_step(xd[idx].contiguous(), yd[idx].contiguous(), lr, want_loss=bool(want))
            if want:
                hist.append((s, loss))
        return hist

    def predict(self, X) -> np.ndarray:
        torch = self.torch
        xd = torch.from_numpy(self.xs(np.atleast_2d(X))).cuda()
        y = torch.empty((xd.shape[0], self.ys.mean.size), dtype=torch.float32, device="cuda")
        self.net.forward(xd, y)
        torch.cuda.synchronize()
        return y.cpu().numpy() * self.ys.sd + self.ys.mean

    def apply(self, d: "df.DualFermion", w):
        """Predict Sigma~ for workload w and set it on handle d."""
        torch = self.torch
        xd = torch.from_numpy(self.xs(features(w)[None, :])).cuda()
        y = torch.empty((1, self.ys.mean.size), dtype=torch.float32, device="cuda")
        self.net.forward(xd, y)
        mean = torch.from_numpy(self.ys.mean).cuda()
        sd = torch.from_numpy(self.ys.sd).cuda()
        df.warmstart_sigma(d, y, mean, sd, self.kmap)


def passes_to(d, sigma_ref, tol: float, max_iter: int):
    """Passes of the loop on handle d until max|Sigma~ - ref| <= tol max|ref|,
    and the device time they took (CUDA events)."""
    import torch
    den = float(np.max(np.abs(sigma_ref)))
    ms = 0.0
    stream = torch.cuda.current_stream()
    for p in range(1, max_iter + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.bubble()
        d.bse(3)
        d.sigma(want_residual=False)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        err = float(np.max(np.abs(d.get_sigma() - sigma_ref)))
        if err <= tol * den:
            return p, ms
        if not (err < 1e3 * den):             # diverged: no point in more passes
            break
    return None, ms


def evaluate(model: WarmStart, workloads, tol: float = 1e-8, max_iter: int = 60,
             precision=df.DF_FP64, symmetry: int = 0):
    """Passes and device time to max|Sigma~ - Sigma~*| <= tol max|Sigma~*| from
    Sigma~ = 0 and from the prediction, on the given path (precision, point-group
    reduction), Sigma~* the FP64 loop at r <= 1e-12 (reduced when the path is);
    a prediction whose loop does not get there falls back to Sigma~ = 0."""
    rows = []
    for w in workloads:
        with df.DualFermion.from_workload(w, eig_mode=0, symmetry=symmetry) as d:
            it, r, _ = d.iterate(max_iter, tol=1e-12)
            ref = d.get_sigma()
        with df.DualFermion.from_workload(w, eig_mode=0, precision=precision, symmetry=symmetry) as d:
            p0, t0 = passes_to(d, ref, tol, max_iter)
        with df.DualFermion.from_workload(w, eig_mode=0, precision=precision, symmetry=symmetry) as d:
            model.apply(d, w)
            pred_err = float(np.max(np.abs(d.get_sigma() - ref)) / np.max(np.abs(ref)))
            p1, t1 = passes_to(d, ref, tol, max_iter)
            fallback = p1 is None
        rows.append({"cold_passes": p0, "cold_ms": t0, "warm_passes": p1 if not fallback else p0,
                     "warm_ms": t1 if not fallback else t1 + t0, "prediction_err": pred_err,
                     "fallback": fallback})
    return rows
