"""The CUDA diagnostics (equal-time moments, density of states) through the C
ABI against the oracle's, on the same contour Green's functions: a free one
(U = 0, E = 1, closed form known) and an interacting DMFT solution from the
oracle (U = 0.5, E = 1).  FP64 on both sides: 1e-12."""

import numpy as np
import pytest
import torch

from oracle import nedmft_oracle as O
from paper_0711_0999_gb300 import api
from paper_0711_0999_gb300.build import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    build_library()


def cases():
    args = (-2, 4, 0.2, 10, 0.5)
    c = O.contour_grid(*args)
    eps, ebar, wq = O.quadrature_points(12)
    free = sum(wq[q] * O.g0_matrix(c, O.Model(U=0.0, E=1.0), float(eps[q]), float(ebar[q])) for q in range(len(wq)))
    inter = O.dmft_solve(c, O.Model(U=0.5, E=1.0), n_quad=12, tol=1e-8, max_iter=60).gloc
    return args, c, [free, inter]


def test_moments_and_dos_match_oracle():
    args, c, gls = cases()
    g = api.contour_grid(*args)
    omega = np.linspace(-4.0, 4.0, 33)
    m_index = [0, 3, c.n_t // 2, c.n_t - 1, c.n_t + 5, -1]  # window edges and two invalid indices
    for gl in gls:
        t = torch.as_tensor(gl, device="cuda")
        mu0, mu1, mu2, dens = (x.cpu().numpy() for x in api.moments(g, t))
        r0, r1, r2, rn = O.moments(c, gl)
        for a, b in ((mu0, r0), (mu1, r1), (mu2, r2), (dens, rn)):
            assert np.array_equal(np.isnan(a), np.isnan(b))
            ok = ~np.isnan(b)
            assert np.abs(a[ok] - b[ok]).max() < 1e-12 * max(1.0, np.abs(b[ok]).max())
        rho = api.dos(g, t, m_index, omega).cpu().numpy()
        for row, m in enumerate(m_index):
            if 0 <= m < c.n_t:
                ref = O.dos(c, gl, m, omega)
                assert np.abs(rho[row] - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
            else:
                assert np.isnan(rho[row]).all()


def test_diagnostics_errors():
    g = api.contour_grid(-2, 4, 0.2, 10, 0.5)
    bad = api.contour_grid(-2, 4, 0.2, 10, 0.5)
    bad.contour.n_c = 7
    t = torch.zeros((g.n_c, g.n_c), dtype=torch.complex128, device="cuda")
    with pytest.raises(api.NedmftError):
        api.moments(bad, t)
    with pytest.raises(api.NedmftError):
        api.dos(bad, t, [1], [0.0])
    assert api.dos(g, t, [], [0.0]).numel() == 0
