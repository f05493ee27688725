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

N_IN, N_OUT = 17, 2
DIMS = [17, 256, 256, 256, 256, 2]


# Training steps of the network: it learns the discrete X at both, and the
# warm start extrapolates in dt to the contour it starts (see nedmft.h).
TRAIN_DTS = (0.1, 0.2)
# The half-filled model's Mott transition (Sec. III: U > sqrt(2) t* is the
# insulator).  The features assume that the Green's function settles to a
# function of t - t' a few units of time after the field is switched on, as a
# metal's does; plain substitution, the paper's loop, rarely converges on the
# insulating side within the training runs' iteration budget, so the network
# has few of its solutions to learn from.
U_MOTT = 2.0 ** 0.5


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
    """X, the impurity Green's function the network learns, from a converged self-energy."""
    t = torch.empty((grid.n_c * grid.n_c, N_OUT), dtype=torch.float32, device=sigma.device)
    N.check(N.lib().nedmft_mlp_target(ctypes.byref(grid.contour), ctypes.byref(model), _p(sigma), 1.0, _p(t), _s()))
    return t


def collect(runs, contours, n_quad: int, precision="mixed_bf16", tol=1e-8, max_iter=80, device="cuda"):
    """Plain (zero-start) solves of each (U, E) on each contour (one per training
    step); the features and targets of the runs that converged, stacked (a run
    stopped at max_iter has no fixed point to learn).  Returns (x, t, iterations
    per run, converged flag per run), runs in the order (U, E) outer, contour inner."""
    grids = [api.contour_grid(*args) for args in contours]
    xs, ts, its, conv = [], [], [], []
    for U, E in runs:
        model = api.make_model(U, E)
        for grid in grids:
            sol = api.dmft_solve(grid, model, n_quad, precision, tol=tol, max_iter=max_iter, device=device)
            its.append(sol.iterations)
            conv.append(bool(sol.converged))
            if sol.converged:
                xs.append(features(grid, model, device))
                ts.append(targets(grid, model, sol.sigma))
    if not xs:
        raise RuntimeError("collect: no training run converged")
    return torch.cat(xs), torch.cat(ts), its, conv


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


def warm_start(grid: api.Grid, model, params: torch.Tensor, dts=TRAIN_DTS) -> torch.Tensor:
    """Sigma_0 from the network's X, extrapolated in dt from the training steps
    to the grid's own, complex128 on the device."""
    dev = params.device
    sigma = torch.empty((grid.n_c, grid.n_c), dtype=torch.complex128, device=dev)
    ws = api.workspace(N.lib().nedmft_sigma_warm_start_workspace_size(ctypes.byref(grid.contour)), dev)
    d = np.ascontiguousarray(dts, dtype=np.float64)
    N.check(N.lib().nedmft_sigma_warm_start(ctypes.byref(grid.contour), ctypes.byref(model), _p(params), len(d),
                                            d.ctypes.data_as(N.PD), _p(sigma), _p(ws), ws.numel(), _s()))
    return sigma


def band_only(grid: api.Grid, model, device="cuda") -> torch.Tensor:
    """The closed-form part alone, -w1 D (X set to zero): the self-energy of
    the static U w1 term, the band of the point-split contour delta."""
    zero = torch.zeros(N.lib().nedmft_mlp_param_count(), dtype=torch.float32, device=device)
    return warm_start(grid, model, zero, dts=(grid.contour.dt,))


def initial_sigma(grid: api.Grid, model, params: torch.Tensor):
    """The start the DMFT loop should take: the network's on the metallic side
    (U < sqrt 2), None (the plain zero start) on the insulating side."""
    if model.U < U_MOTT:
        return warm_start(grid, model, params)
    return None
