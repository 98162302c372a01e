"""CPU oracle of the warm-start network: TEST INFRASTRUCTURE ONLY.

A plain numpy implementation of the dense network (n_in -> W -> W -> W ->
n_out, tanh between the layers, linear output), its mean-squared-error
gradient by the chain rule, and one Adam step.  It shares nothing with the
CUDA kernels.  `rounding=True` reproduces the kernels' rounding points:
both operands of every matrix product are rounded to BF16 (round to nearest
even), products are summed exactly in FP64 (the kernels' FP32 accumulation
differs from it by FP32 rounding only), activations and gradients are
stored in FP32.  With `rounding=False` everything is FP64; that version is
pinned to central finite differences in tests/test_mlp_oracle.py.

Parameters use the layout of df_mlp_params: [W1 (n_in x W, row-major), b1,
W2, b2, W3, b3, W4, b4].
"""
import numpy as np


def bf16_round(x):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    x = np.asarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def split_params(flat, dims):
    out, o = [], 0
    for l in range(4):
        W = flat[o:o + dims[l] * dims[l + 1]].reshape(dims[l], dims[l + 1])
        o += dims[l] * dims[l + 1]
        b = flat[o:o + dims[l + 1]]
        o += dims[l + 1]
        out.append((W, b))
    return out


def _mm(a, b, rounding):
    if rounding:
        return bf16_round(a).astype(np.float64) @ bf16_round(b).astype(np.float64)
    return np.asarray(a, np.float64) @ np.asarray(b, np.float64)


def _store(x, rounding):
    return np.asarray(x, np.float32) if rounding else np.asarray(x, np.float64)


def forward(flat, dims, x, rounding=True):
    """Returns the activations [A0 = x, A1, A2, A3, Y]."""
    acts = [_store(x, rounding)]
    for l, (W, b) in enumerate(split_params(flat, dims)):
        z = _mm(acts[-1], W, rounding) + np.asarray(b, np.float64)
        acts.append(_store(np.tanh(z) if l < 3 else z, rounding))
    return acts


def loss_and_grads(flat, dims, x, target, rounding=True):
    """mean((net(x) - target)^2) and its gradient (flat, same layout)."""
    acts = forward(flat, dims, x, rounding)
    y = np.asarray(acts[-1], np.float64)
    d = y - np.asarray(target, np.float64)
    loss = float(np.mean(d * d))
    dz = _store(2.0 * d / d.size, rounding)
    params = split_params(flat, dims)
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, _ = params[l]
        gW = _mm(acts[l].T, dz, rounding)
        gb = np.asarray(dz, np.float64).sum(axis=0)
        grads[l] = (gW, gb)
        if l == 0:
            break
        da = _mm(dz, np.asarray(W).T, rounding)
        a = np.asarray(acts[l], np.float64)
        dz = _store(da * (1.0 - a * a), rounding)
    flat_g = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, flat_g


def adam(flat, grad, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update (returns new params, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * grad
    m2 = b2 * m2 + (1 - b2) * grad * grad
    c1 = 1 - b1 ** step
    c2 = 1 - b2 ** step
    return flat - lr * (m1 / c1) / (np.sqrt(m2 / c2) + eps), m1, m2
