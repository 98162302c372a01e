"""Pins of the warm-start network's CPU oracle (no GPU)."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_bf16_rounding():
    # values exactly representable stay, halfway cases go to even, relative error <= 2^-9
    assert M.bf16_round(np.float32(1.0)) == 1.0
    x = np.float32(1.0) + np.float32(2.0 ** -8)          # halfway between 1 and 1 + 2^-7: to even (1.0)
    assert M.bf16_round(x) == 1.0
    y = np.float32(1.0) + np.float32(3 * 2.0 ** -8)      # halfway between 1+2^-7 and 1+2^-6: to even
    assert M.bf16_round(y) == np.float32(1.0 + 2.0 ** -6)
    r = np.random.default_rng(0).normal(size=1000).astype(np.float32)
    assert np.max(np.abs(M.bf16_round(r) - r) / np.abs(r)) <= 2.0 ** -8


def _net(seed=0, dims=(5, 7, 7, 7, 3)):
    rng = np.random.default_rng(seed)
    n = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(4))
    return rng.normal(scale=0.4, size=n), dims, rng.normal(size=(6, dims[0])), rng.normal(size=(6, dims[-1]))


def test_gradient_matches_central_differences():
    flat, dims, x, t = _net()
    _, g = M.loss_and_grads(flat, dims, x, t, rounding=False)
    h = 1e-6
    fd = np.empty_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = h
        lp, _ = M.loss_and_grads(flat + e, dims, x, t, rounding=False)
        lm, _ = M.loss_and_grads(flat - e, dims, x, t, rounding=False)
        fd[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_planted_backprop_mistake_is_caught(monkeypatch):
    # dropping the tanh derivative (1 - a^2) must break the finite-difference pin
    orig = M.loss_and_grads

    def wrong(flat, dims, x, target, rounding=True):
        acts = M.forward(flat, dims, x, rounding)
        d = acts[-1] - target
        dz = 2.0 * d / d.size
        params = M.split_params(flat, dims)
        grads = [None] * 4
        for l in range(3, -1, -1):
            grads[l] = (acts[l].T @ dz, dz.sum(axis=0))
            if l == 0:
                break
            dz = dz @ params[l][0].T
        return float(np.mean(d * d)), np.concatenate([np.concatenate([a.reshape(-1), b]) for a, b in grads])

    monkeypatch.setattr(M, "loss_and_grads", wrong)
    with pytest.raises(AssertionError):
        test_gradient_matches_central_differences()
    monkeypatch.setattr(M, "loss_and_grads", orig)


def test_adam_first_step_is_signed_lr():
    # bias correction makes the first Adam step -lr * sign(g) (up to eps)
    g = np.array([3.0, -0.5, 1e-3])
    p, _, _ = M.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-4)


def test_wedge_map_covers_d4_classes():
    # every momentum and its 8 images under the square lattice's point group
    # share one wedge index; (nk/2+1)(nk/2+2)/2 classes
    from paper_1507_00895_gb300 import warmstart as W
    for nk in (4, 8, 16):
        kmap, rep = W.wedge(nk)
        assert kmap.max() + 1 == (nk // 2 + 1) * (nk // 2 + 2) // 2 == len(rep)
        for jx in range(nk):
            for jy in range(nk):
                imgs = {(jx, jy), (jy, jx), (-jx % nk, jy), (jx, -jy % nk), (-jx % nk, -jy % nk),
                        (jy, -jx % nk), (-jy % nk, jx), (-jy % nk, -jx % nk)}
                assert len({kmap[a * nk + b] for a, b in imgs}) == 1
        assert all(kmap[r] == i for i, r in enumerate(rep))
