"""Learned warm start of the DMFT self-energy: training-data collection,
training and prediction, driven through the C ABI.

Every arithmetic step runs in libnedmft.so (features, targets, minibatch
sampling, forward, backward, Adam, the prediction).  This module only
sequences the calls and holds the tensors.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from . import api

N_IN, N_OUT = 14, 2
DIMS = [14, 256, 256, 256, 256, 2]


def scale(U: float) -> float:
    """Target scale: the smooth self-energy grows like U^2."""
    return max(U, 0.05) ** 2 / 8.0


def init_params(seed: int = 20071101) -> np.ndarray:
    """Glorot-uniform weights, small uniform biases (FP32), layer by layer."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(len(DIMS) - 1):
        lim = np.sqrt(6.0 / (DIMS[i] + DIMS[i + 1]))
        out.append(rng.uniform(-lim, lim, DIMS[i] * DIMS[i + 1]))
        out.append(rng.uniform(-0.01, 0.01, DIMS[i + 1]))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == N.lib().nedmft_mlp_param_count()
    return p


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def features(grid: api.Grid, model, device="cuda") -> torch.Tensor:
    x = torch.empty((grid.n_c * grid.n_c, N_IN), dtype=torch.float32, device=device)
    N.check(N.lib().nedmft_mlp_features(ctypes.byref(grid.contour), ctypes.byref(model), _p(x), _s()))
    return x


def targets(grid: api.Grid, model, sigma: torch.Tensor) -> torch.Tensor:
    t = torch.empty((grid.n_c * grid.n_c, N_OUT), dtype=torch.float32, device=sigma.device)
    N.check(N.lib().nedmft_mlp_target(ctypes.byref(grid.contour), ctypes.byref(model), _p(sigma), scale(model.U),
                                      _p(t), _s()))
    return t


def collect(runs, contour_args, n_quad: int, precision="mixed_bf16", tol=1e-8, max_iter=80, device="cuda"):
    """Converged plain (zero-start) solves of each (U, E): features and targets stacked.

    Returns (x, t, iterations per run)."""
    grid = api.contour_grid(*contour_args)
    xs, ts, its = [], [], []
    for U, E in runs:
        model = api.make_model(U, E)
        sol = api.dmft_solve(grid, model, n_quad, precision, tol=tol, max_iter=max_iter, device=device)
        xs.append(features(grid, model, device))
        ts.append(targets(grid, model, sol.sigma))
        its.append(sol.iterations)
    return torch.cat(xs), torch.cat(ts), its


def loss_and_grad(params: torch.Tensor, x: torch.Tensor, t: torch.Tensor):
    n = x.shape[0]
    ws = api.workspace(N.lib().nedmft_mlp_workspace_size(n), params.device)
    g = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    N.check(N.lib().nedmft_mlp_grad(_p(params), _p(x), _p(t), n, _p(g), _p(loss), _p(ws), ws.numel(), _s()))
    return loss, g


def forward(params: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    n = x.shape[0]
    ws = api.workspace(N.lib().nedmft_mlp_workspace_size(n), params.device)
    y = torch.empty((n, N_OUT), dtype=torch.float32, device=params.device)
    N.check(N.lib().nedmft_mlp_forward(_p(params), _p(x), n, _p(y), _p(ws), ws.numel(), _s()))
    return y


def train(x: torch.Tensor, t: torch.Tensor, steps=2000, batch=2048, lr=1e-3, seed=20071101, params=None):
    """Adam on random minibatches; returns (params, per-step losses as a tensor)."""
    dev = x.device
    p = torch.as_tensor(init_params(seed) if params is None else params, device=dev).clone()
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    g = torch.empty_like(p)
    xb = torch.empty((batch, N_IN), dtype=torch.float32, device=dev)
    tb = torch.empty((batch, N_OUT), dtype=torch.float32, device=dev)
    losses = torch.empty(steps, dtype=torch.float32, device=dev)
    ws = api.workspace(N.lib().nedmft_mlp_workspace_size(batch), dev)
    lib = N.lib()
    for s in range(steps):
        N.check(lib.nedmft_mlp_sample(_p(x), _p(t), x.shape[0], batch, seed, s, _p(xb), _p(tb), _s()))
        lr_s = lr * 0.5 * (1 + np.cos(np.pi * s / steps))  # cosine schedule
        N.check(lib.nedmft_mlp_grad(_p(p), _p(xb), _p(tb), batch, _p(g), _p(losses[s:]), _p(ws), ws.numel(), _s()))
        N.check(lib.nedmft_mlp_adam(_p(p), _p(g), _p(m1), _p(m2), s + 1, float(lr_s), _s()))
    return p, losses


def warm_start(grid: api.Grid, model, params: torch.Tensor) -> torch.Tensor:
    """Sigma_0 = U w1 delta_c + scale(U) * network(features), complex128 on the device."""
    dev = params.device
    sigma = torch.empty((grid.n_c, grid.n_c), dtype=torch.complex128, device=dev)
    ws = api.workspace(N.lib().nedmft_sigma_warm_start_workspace_size(ctypes.byref(grid.contour)), dev)
    N.check(N.lib().nedmft_sigma_warm_start(ctypes.byref(grid.contour), ctypes.byref(model), _p(params),
                                            scale(model.U), _p(sigma), _p(ws), ws.numel(), _s()))
    return sigma


def band_only(grid: api.Grid, model, device="cuda") -> torch.Tensor:
    """The closed-form band alone (the network's output set to zero)."""
    zero = torch.zeros(N.lib().nedmft_mlp_param_count(), dtype=torch.float32, device=device)
    return warm_start(grid, model, zero)
