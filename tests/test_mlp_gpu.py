"""The warm-start network on the GPU: gradients against the CPU restatement,
the feature/target round trip, and what the trained network saves."""

import numpy as np
import pytest
import torch

from oracle import mlp_oracle as M
from oracle import nedmft_oracle as O
from paper_0711_0999_gb300 import api, warmstart
from paper_0711_0999_gb300.build import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    build_library()


@pytest.mark.parametrize("n", [300, 5000])  # 3 and 40 row tiles of 128 with a ragged tail; 5 and 79 K chunks of 64
def test_gradient_matches_cpu_restatement(n):
    p = warmstart.init_params(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(n, 17)).astype(np.float32)
    t = rng.normal(size=(n, 2)).astype(np.float32)
    loss, g = warmstart.loss_and_grad(torch.as_tensor(p, device="cuda"), torch.as_tensor(x, device="cuda"),
                                      torch.as_tensor(t, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    lr, gr = M.loss_and_grad(p, x, t, rounded=True)
    l64, g64 = M.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), rounded=False)
    assert abs(loss.item() - lr) < 1e-4 * abs(lr)
    assert np.linalg.norm(g - gr) < 2e-2 * np.linalg.norm(gr)  # same bf16 operands, FP32 sums in another order
    cos = float(g @ g64 / (np.linalg.norm(g) * np.linalg.norm(g64)))
    assert cos > 0.999  # the bf16 path keeps the direction of the exact gradient
    y = warmstart.forward(torch.as_tensor(p, device="cuda"), torch.as_tensor(x, device="cuda")).cpu().numpy()
    yr, _ = M.forward(p, x, rounded=True)
    assert np.abs(y - yr).max() < 2e-2 * np.abs(yr).max()


def test_features_targets_and_warm_start_round_trip():
    args = (-2, 4, 0.2, 10, 0.5)
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    model = api.make_model(1.3, 0.7)
    x = warmstart.features(g, model).cpu().numpy()
    assert np.abs(x - M.features(c, 1.3, 0.7)).max() < 1e-6
    p = torch.as_tensor(warmstart.init_params(5), device="cuda")
    # extrapolation from the steps 0.1 and 0.3 to this contour's 0.2: the mean of the two predictions
    sigma0 = warmstart.warm_start(g, model, p, dts=(0.1, 0.3)).cpu().numpy()
    y = [warmstart.forward(p, torch.as_tensor(M.features(c, 1.3, 0.7, dt_feature=d), dtype=torch.float32,
                                              device="cuda")).cpu().numpy() for d in (0.1, 0.3)]
    yx = 0.5 * (y[0] + y[1])
    X = (yx[:, 0] + 1j * yx[:, 1]).reshape(c.n_c, c.n_c)
    ref = M.sigma_from_xh(c, X, 1.3, 0.5)
    assert np.abs(sigma0 - ref).max() < 1e-5 * np.abs(ref).max()
    # the targets recover X from the self-energy it gives
    t = warmstart.targets(g, model, torch.as_tensor(sigma0, device="cuda")).cpu().numpy()
    assert np.abs(t - yx).max() < 1e-4 * max(1.0, np.abs(yx).max())


def test_trained_warm_start_saves_iterations():
    # train on converged self-energies of 24 runs (U in [0.25, 2.5], E in
    # [0.25, 4], seed 20071101) at the steps 0.1 and 0.2, then solve 3
    # held-out pairs from zero, from the band alone and from the network
    # (extrapolated to the evaluation contour's step, 0.05): the network needs
    # fewer iterations than either in total and converges to the same fixed point.
    train_contours = [(-2, 4, 0.1, 10, 0.5), (-2, 4, 0.2, 10, 0.5)]
    g = api.contour_grid(-2, 4, 0.05, 10, 0.5)
    rng = np.random.default_rng(20071101)
    train_runs = list(zip(rng.uniform(0.25, 2.5, 24), rng.uniform(0.25, 4.0, 24)))
    rng2 = np.random.default_rng(20071102)
    held = list(zip(rng2.uniform(0.4, 1.2, 3), rng2.uniform(0.5, 3.0, 3)))
    x, t, _, _ = warmstart.collect(train_runs, train_contours, n_quad=8, precision="fp64", tol=1e-10, max_iter=150)
    params, losses = warmstart.train(x, t, steps=6000, batch=4096, lr=2e-3)
    losses = losses.cpu().numpy()
    assert losses[-100:].mean() < 0.2 * losses[:20].mean()
    total = {"zero": 0, "band": 0, "net": 0}
    for U, E in held:
        model = api.make_model(float(U), float(E))
        zero = api.dmft_solve(g, model, 8, "fp64", tol=1e-9, max_iter=120)
        band = api.dmft_solve(g, model, 8, "fp64", sigma_init=warmstart.band_only(g, model), tol=1e-9, max_iter=120)
        warm = api.dmft_solve(g, model, 8, "fp64", sigma_init=warmstart.warm_start(g, model, params), tol=1e-9,
                              max_iter=120)
        print(f"U={U:.3f} E={E:.3f} iterations zero {zero.iterations} band {band.iterations} net {warm.iterations}")
        assert zero.converged and band.converged and warm.converged
        ref = zero.gloc.abs().max()
        assert (warm.gloc - zero.gloc).abs().max() < 1e-7 * ref  # the same fixed point
        total["zero"] += zero.iterations
        total["band"] += band.iterations
        total["net"] += warm.iterations
    print("total iterations", total)
    assert total["net"] < total["zero"] and total["net"] < total["band"]
