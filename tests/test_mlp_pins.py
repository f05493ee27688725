"""Pins of the CPU restatement of the warm-start network."""

import numpy as np

from oracle import mlp_oracle as M
from oracle import nedmft_oracle as O


def _params(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(len(M.DIMS) - 1):
        lim = np.sqrt(6.0 / (M.DIMS[i] + M.DIMS[i + 1]))
        out.append(rng.uniform(-lim, lim, M.DIMS[i] * M.DIMS[i + 1]))
        out.append(rng.uniform(-0.1, 0.1, M.DIMS[i + 1]))
    return np.concatenate(out)


def test_param_count():
    assert M.param_count() == 14 * 256 + 256 + 3 * (256 * 256 + 256) + 256 * 2 + 2


def test_gradient_matches_finite_differences():
    p = _params(1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(17, 14))
    t = rng.normal(size=(17, 2))
    _, g = M.loss_and_grad(p, x, t, rounded=False)
    idx = rng.choice(len(p), 40, replace=False)
    idx = np.concatenate([idx, [len(p) - 1, len(p) - 3, 14 * 256 + 5]])  # output and first biases
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (M.loss_and_grad(pp, x, t, rounded=False)[0] - M.loss_and_grad(pm, x, t, rounded=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-20], dtype=np.float32)
    r = M.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == np.float32(1.0078125)
    assert abs(r[3] + 3.140625) < 1e-7
    # 8 significant bits everywhere
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)


def test_features_and_band():
    c = O.contour_grid(-1, 1, 0.5, 2.0, 0.5)
    f = M.features(c, 1.25, 2.0).reshape(c.n_c, c.n_c, 14)
    i, j = 1, 2 * c.n_t + 1  # upper t = -0.5, imaginary tau = 0.5 (Re t = -1)
    assert np.allclose(f[i, j], [0.5, 0.5, 0.025, -0.25, -0.025, 0.0, 1, 0, 0, -0.05, 0.25, 0, 0, 1])
    b = M.band(c, 1.0, 0.5)
    # the band equals the impurity step's <w1> = 1 self-energy scaled by w1
    gl = O.lattice_gloc(c, O.Model(U=1.0, E=1.0), np.zeros((c.n_c, c.n_c), complex), *O.quadrature_points(4))[0]
    s_full, _ = O.impurity_update(c, O.Model(U=1.0, E=1.0, w1=1.0, mu=0.5), gl, np.zeros((c.n_c, c.n_c), complex))
    assert np.abs(b - 0.5 * s_full).max() < 1e-8 * np.abs(b).max()
