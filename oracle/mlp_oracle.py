"""Plain CPU restatement of the self-energy warm-start network.

TEST INFRASTRUCTURE ONLY (imported by tests/ alone).  The network is not part
of the paper's method: it only supplies a starting self-energy, and the DMFT
loop's converged result does not depend on it.  This module restates, in
NumPy, the layer layout, features, targets, forward pass, mean-squared-error
gradient and the bf16 rounding of GEMM operands that the CUDA kernels use, so
their gradients can be checked; its FP64 unrounded gradient is pinned by
finite differences in tests/test_mlp_pins.py.
"""

from __future__ import annotations

import numpy as np

DIMS = [14, 256, 256, 256, 256, 2]


def param_count() -> int:
    return sum(DIMS[i] * DIMS[i + 1] + DIMS[i + 1] for i in range(len(DIMS) - 1))


def unpack(params: np.ndarray):
    layers, o = [], 0
    for i in range(len(DIMS) - 1):
        n_w = DIMS[i] * DIMS[i + 1]
        w = params[o:o + n_w].reshape(DIMS[i], DIMS[i + 1])
        o += n_w
        b = params[o:o + DIMS[i + 1]]
        o += DIMS[i + 1]
        layers.append((w, b))
    return layers


def bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest bf16 value (ties to even), returned as FP32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _mm(a, b, rounded):
    if rounded:
        return bf16(a).astype(np.float32) @ bf16(b).astype(np.float32)
    return a @ b


def forward(params, x, rounded=True):
    """Returns (y, hidden activations); tanh after each hidden layer."""
    dt = np.float32 if rounded else np.float64
    h = np.asarray(x, dtype=dt)
    acts = []
    layers = unpack(np.asarray(params, dtype=dt))
    for i, (w, b) in enumerate(layers):
        z = _mm(h, w, rounded) + b
        h = np.tanh(z) if i < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grad(params, x, t, rounded=True):
    """Mean-squared error over all outputs and its gradient (same layout as params)."""
    dt = np.float32 if rounded else np.float64
    x = np.asarray(x, dtype=dt)
    t = np.asarray(t, dtype=dt)
    layers = unpack(np.asarray(params, dtype=dt))
    y, acts = forward(params, x, rounded)
    r = y - t
    loss = float(np.mean(r.astype(np.float64) ** 2))
    d = (2.0 / r.size) * r
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        w, _ = layers[i]
        xin = x if i == 0 else acts[i - 1]
        gw = _mm(xin.T, d, rounded)
        gb = d.sum(axis=0)
        grads.append((gw, gb))
        if i > 0:
            d = _mm(d, w.T, rounded) * (1 - acts[i - 1] ** 2)
    grads.reverse()
    return loss, np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])


def features(c, U: float, E: float) -> np.ndarray:
    """Per pair (t_i, t_j): U/2.5, E/4, Re(t_i - t_j)/20, (tau_i - tau_j)/beta, then for
    each time Re t / 20, tau / beta, branch one-hot."""
    n = c.n_c
    per = np.zeros((n, 5))
    for k in range(n):
        per[k, 0] = c.t[k].real / 20.0
        per[k, 1] = -c.t[k].imag / c.beta
        per[k, 2 + (0 if k < c.n_t else (1 if k < 2 * c.n_t else 2))] = 1.0
    f = np.zeros((n, n, 14))
    f[:, :, 0] = U / 2.5
    f[:, :, 1] = E / 4.0
    f[:, :, 2] = per[:, None, 0] - per[None, :, 0]
    f[:, :, 3] = per[:, None, 1] - per[None, :, 1]
    f[:, :, 4:9] = per[:, None, :]
    f[:, :, 9:14] = per[None, :, :]
    return f.reshape(n * n, 14)


def band(c, U: float, w1: float) -> np.ndarray:
    """U w1 delta_c with the point-split contour delta (Eqs. delta_cont_defa/b)."""
    n = c.n_c
    s = np.zeros((n, n), complex)
    for j in range(1, n):
        s[j, j - 1] = U * w1 / c.w[j - 1]
    s[0, n - 1] = -U * w1 / c.w[n - 1]
    return s


def scale(U: float) -> float:
    return max(U, 0.05) ** 2 / 8.0
