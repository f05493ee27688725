"""Plain CPU restatement of the self-energy warm-start network.

TEST INFRASTRUCTURE ONLY (imported by tests/ alone).  The network is not part
of the paper's method: it only supplies a starting self-energy, and the DMFT
loop's converged result does not depend on it.  This module restates, in
NumPy, the layer layout, features, the map between the self-energy and the
impurity Green's function X the network learns (W Sigma W = -w1 D +
w1 (1 - w1) D X D, the impurity step's identity), forward pass,
mean-squared-error gradient and the bf16 rounding of GEMM operands that the
CUDA kernels use, so their gradients can be checked; its FP64 unrounded
gradient is pinned by finite differences in tests/test_mlp_pins.py.
"""

from __future__ import annotations

import numpy as np

DIMS = [17, 256, 256, 256, 256, 2]


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


def features(c, U: float, E: float, dt_feature: float | None = None) -> np.ndarray:
    """Per pair (t_a, t_b): U/2.5, E/4, tanh(Re(t_a - t_b)/3), then for each time
    (real part r, imaginary depth tau) tanh(max(r, 0)/3), min(r, 0)/5, tau/beta and
    the branch one-hot, then the contour order (1 for a >= b) and dt/0.1 (the
    contour's own step unless dt_feature is given)."""
    n = c.n_c
    r = c.t.real
    per = np.zeros((n, 6))
    for k in range(n):
        per[k, 0] = np.tanh(max(r[k], 0.0) / 3.0)
        per[k, 1] = min(r[k], 0.0) / 5.0
        per[k, 2] = -c.t[k].imag / c.beta
        per[k, 3 + (0 if k < c.n_t else (1 if k < 2 * c.n_t else 2))] = 1.0
    f = np.zeros((n, n, 17))
    f[:, :, 0] = U / 2.5
    f[:, :, 1] = E / 4.0
    f[:, :, 2] = np.tanh((r[:, None] - r[None, :]) / 3.0)
    f[:, :, 3:9] = per[:, None, :]
    f[:, :, 9:15] = per[None, :, :]
    f[:, :, 15] = np.tril(np.ones((n, n)))
    f[:, :, 16] = (c.dt if dt_feature is None else dt_feature) / 0.1
    return f.reshape(n * n, 17)


def d_matrix(c, U: float) -> np.ndarray:
    """D = i [M(mu - U) - M(mu)]: -U W_i at (i, i-1) for i >= 1, +U W_0 at (0, N-1)."""
    n = c.n_c
    D = np.zeros((n, n), complex)
    for i in range(1, n):
        D[i, i - 1] = -U * c.w[i]
    D[0, n - 1] = U * c.w[0]
    return D


def sigma_from_xh(c, X: np.ndarray, U: float, w1: float) -> np.ndarray:
    """Sigma from X by W Sigma W = -w1 D + w1 (1 - w1) D X D."""
    D = d_matrix(c, U)
    return (-w1 * D + w1 * (1 - w1) * D @ X @ D) / (c.w[:, None] * c.w[None, :])


def xh_from_sigma(c, sigma: np.ndarray, U: float, w1: float) -> np.ndarray:
    """X from Sigma, the inverse of sigma_from_xh (D is invertible for U != 0)."""
    D = d_matrix(c, U)
    Di = np.linalg.inv(D)
    S = c.w[:, None] * sigma * c.w[None, :]
    return Di @ (S + w1 * D) @ Di / (w1 * (1 - w1))


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
