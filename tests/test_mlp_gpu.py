"""Warm-start network kernels (df_mlp_*) against the CPU oracle, and the
warm start itself against the plain loop."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1507_00895_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_00895_gb300 import build
    build.build_lib()
    from paper_1507_00895_gb300 import df as dfm
    return dfm, torch


def nrel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


DIMS = (36, 96, 96, 96, 70)        # ragged against the 64 x 64 x 32 tiles


def _setup(env, batch=37, seed=1):
    df, torch = env
    net = df.MLP(DIMS[0], DIMS[-1], width=DIMS[1], max_batch=64, seed=seed)
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(batch, DIMS[0])).astype(np.float32)
    t = rng.normal(size=(batch, DIMS[-1])).astype(np.float32)
    return net, x, t, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()


def test_forward_matches_oracle(env):
    df, torch = env
    net, x, t, xd, td = _setup(env)
    y = torch.empty((x.shape[0], DIMS[-1]), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    torch.cuda.synchronize()
    ref = M.forward(net.params().astype(np.float64), DIMS, x, rounding=True)[-1]
    err = nrel(y.cpu().numpy(), ref)
    print(f"forward err {err:.2e}")
    # same BF16 operands; FP32 vs FP64 accumulation (a rare BF16 rounding flip
    # of a later layer's input would show as ~1e-3)
    assert err < 1e-4


def test_gradients_match_oracle(env):
    df, torch = env
    net, x, t, xd, td = _setup(env, seed=2)
    loss = net.gradients(xd, td)
    g = net.grads()
    ref_loss, ref_g = M.loss_and_grads(net.params().astype(np.float64), DIMS, x, t, rounding=True)
    assert abs(loss - ref_loss) < 1e-4 * ref_loss
    o = 0
    worst = 0.0
    for l in range(4):
        nW = DIMS[l] * DIMS[l + 1]
        for part in (slice(o, o + nW), slice(o + nW, o + nW + DIMS[l + 1])):
            worst = max(worst, nrel(g[part], ref_g[part]))
        o += nW + DIMS[l + 1]
    print(f"gradient worst layer err {worst:.2e}")
    assert worst < 5e-3
    # and against the exact FP64 chain rule, to BF16 accuracy
    _, g64 = M.loss_and_grads(net.params().astype(np.float64), DIMS, x, t, rounding=False)
    assert nrel(g, g64) < 5e-2


def test_adam_matches_oracle(env):
    df, torch = env
    net, x, t, xd, td = _setup(env, seed=3)
    p0 = net.params().astype(np.float64)
    net.gradients(xd, td)
    g = net.grads().astype(np.float64)
    net.adam_step(1e-3)
    p1 = net.params()
    ref, _, _ = M.adam(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    assert np.max(np.abs(p1 - ref)) < 1e-6


def test_training_reduces_loss(env):
    df, torch = env
    net, x, t, xd, td = _setup(env, seed=4)
    rng = np.random.default_rng(5)
    A = rng.normal(size=(DIMS[0], DIMS[-1])).astype(np.float32) / 6
    X = rng.normal(size=(64, DIMS[0])).astype(np.float32)
    Y = np.sin(X @ A)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    first = net.train_step(Xd, Yd, 2e-3, want_loss=True)
    for _ in range(300):
        last = net.train_step(Xd, Yd, 2e-3, want_loss=True)
    assert last < 0.2 * first, (first, last)


def test_warm_start_cuts_passes(env):
    df, torch = env
    from paper_1507_00895_gb300 import warmstart as W
    train = I.warmstart_family(256, seed=11, nk=8, n_w=8, m_max=1)
    test = I.warmstart_family(8, seed=12, nk=8, n_w=8, m_max=1)
    X, Y, _, mask = W.generate(train, tol=1e-10)
    assert mask.mean() > 0.9
    model = W.WarmStart(X.shape[1], Y.shape[1], nk=8, width=128, max_batch=128, seed=0)
    model.train(X, Y, steps=800, batch=128, lr=2e-3)
    rows = W.evaluate(model, test, tol=1e-8)
    cold = np.mean([r["cold_passes"] for r in rows])
    warm = np.mean([r["warm_passes"] for r in rows])
    err = np.mean([r["prediction_err"] for r in rows])
    print(f"passes cold {cold:.2f} warm {warm:.2f}, prediction err {err:.3f}")
    assert not any(r["fallback"] for r in rows)
    assert warm < cold
    assert err < 0.5
