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
    assert M.param_count() == 17 * 256 + 256 + 3 * (256 * 256 + 256) + 256 * 2 + 2


def test_gradient_matches_finite_differences():
    p = _params(1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(17, 17))
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
    f = M.features(c, 1.25, 2.0).reshape(c.n_c, c.n_c, 17)
    i, j = 1, 2 * c.n_t + 1  # upper t = -0.5, imaginary tau = 0.5 (Re t = -1)
    assert np.allclose(f[i, j], [0.5, 0.5, np.tanh(0.5 / 3), 0, -0.1, 0, 1, 0, 0, 0, -0.2, 0.25, 0, 0, 1, 0, 5.0])
    k = c.n_t + 1  # lower branch, t = 0.5: elapsed field time tanh(0.5/3), nothing before the field
    assert np.allclose(f[k, i], [0.5, 0.5, np.tanh(1.0 / 3), np.tanh(0.5 / 3), 0, 0, 0, 1, 0, 0, -0.1, 0, 1, 0, 0, 1, 5.0])
    assert np.allclose(M.features(c, 1.25, 2.0, dt_feature=0.2)[:, 16], 2.0)
    b = M.band(c, 1.0, 0.5)
    # the band equals the impurity step's <w1> = 1 self-energy scaled by w1
    gl = O.lattice_gloc(c, O.Model(U=1.0, E=1.0), np.zeros((c.n_c, c.n_c), complex), *O.quadrature_points(4))[0]
    s_full, _ = O.impurity_update(c, O.Model(U=1.0, E=1.0, w1=1.0, mu=0.5), gl, np.zeros((c.n_c, c.n_c), complex))
    assert np.abs(b - 0.5 * s_full).max() < 1e-8 * np.abs(b).max()


def test_sigma_and_xh_maps_are_the_impurity_step():
    # X = inv(A0 + (1 - w1) D) of the oracle's impurity step maps to the oracle's
    # Sigma_new (the identity the network's output goes through), and back
    c = O.contour_grid(-2, 4, 0.2, 10, 0.5)
    m = O.Model(U=1.3, E=0.7, w1=0.4)
    sig = np.zeros((c.n_c, c.n_c), complex)
    gl = O.lattice_gloc(c, m, sig, *O.quadrature_points(6))[0]
    s_new, _ = O.impurity_update(c, m, gl, sig)
    D = M.d_matrix(c, 1.3)
    assert np.allclose(D, 1j * (O.m_matrix(c, m.chem - m.U) - O.m_matrix(c, m.chem)))
    X = np.linalg.inv(np.linalg.inv(gl) + O.weighted_sigma(c, sig) + (1 - 0.4) * D)
    assert np.abs(M.sigma_from_xh(c, X, 1.3, 0.4) - s_new).max() < 1e-10 * np.abs(s_new).max()
    assert np.abs(M.xh_from_sigma(c, s_new, 1.3, 0.4) - X).max() < 1e-9 * np.abs(X).max()
    # X = 0 leaves the band of the point-split delta alone
    assert np.abs(M.sigma_from_xh(c, 0 * X, 1.0, 0.5) - M.band(c, 1.0, 0.5)).max() < 1e-12
