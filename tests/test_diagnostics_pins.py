"""Pins of the oracle's accuracy diagnostics (equal-time moments, reading R11;
the density of states of Eqs. gr_omega and dos_def, reading R12) against
closed forms of the noninteracting problem.

At U = 0 the local retarded function is known exactly: with the Gaussian
density of states, i G^R(T + s/2, T - s/2) = exp(-s^2 / 4) for E = 0, and
exp(-sin^2(E s / 2) / E^2) when both times lie after the field is switched on;
both give mu0 = 1, mu1 = 0, mu2 = 1/2 (the band's second moment), and for
E = 0 the density of states is exp(-omega^2) / sqrt(pi).  The quadratic
stencil of R11 leaves errors O(dt^4) in mu0 and O(dt^2) in mu2.
"""

import numpy as np
import pytest

from oracle import nedmft_oracle as O


def free_gloc(c, E, n):
    """G_loc at U = 0: sum_q w_q G0_q (E = 0 needs only the 1-D quadrature in eps)."""
    m = O.Model(U=0.0, E=E)
    if E == 0.0:
        x, w = O.gauss_hermite(n)
        return sum(w[a] * O.g0_matrix(c, m, float(x[a]), 0.0) for a in range(n))
    eps, ebar, wq = O.quadrature_points(n)
    return sum(wq[q] * O.g0_matrix(c, m, float(eps[q]), float(ebar[q])) for q in range(len(wq)))


def test_retarded_equal_time_and_free_form():
    c = O.contour_grid(-2, 6, 0.2, 10, 0.5)
    g = free_gloc(c, 0.0, 40)
    for m in (0, 5, c.n_t - 1):
        assert abs(O.retarded(c, g, m, m) - (-1j)) < 1e-12  # {c, c^dagger} = 1
    for m, k in ((10, 3), (20, 7)):
        s = c.t[m + k].real - c.t[m - k].real
        assert abs(1j * O.retarded(c, g, m + k, m - k) - np.exp(-s * s / 4)) < 1e-10


@pytest.mark.parametrize("E", [0.0, 1.0])
def test_moments_free_closed_form_and_order(E):
    errs = []
    for dt in (0.2, 0.1):
        c = O.contour_grid(-2, 6, dt, 10, 0.5)
        g = free_gloc(c, E, 40 if E == 0.0 else 20)
        mu0, mu1, mu2, n = O.moments(c, g)
        # E != 0: the closed form holds once both times are after t = 0
        t = c.t[: c.n_t].real
        ok = ~np.isnan(mu0) & ((t - 6 * dt > 0) if E else True)
        assert ok.sum() >= 5
        assert np.abs(mu1[ok]).max() < 1e-12
        assert np.abs(n - 0.5).max() < 1e-12  # half filling at U = 0 (node symmetry)
        errs.append((np.abs(mu0[ok] - 1).max(), np.abs(mu2[ok] - 0.5).max()))
    (e0a, e2a), (e0b, e2b) = errs
    assert e0a < 5e-2 and e0b < 5e-3 and e0a / e0b > 8  # O(dt^4)
    assert e2a < 0.35 and e2b < 0.1 and e2a / e2b > 3  # O(dt^2)


def test_dos_free_gaussian():
    c = O.contour_grid(-2, 12, 0.1, 10, 0.5)
    g = free_gloc(c, 0.0, 60)
    omega = np.linspace(-2.5, 2.5, 21)
    rho = O.dos(c, g, c.n_t // 2, omega)
    assert np.abs(rho - np.exp(-omega ** 2) / np.sqrt(np.pi)).max() < 3e-3
    # the edge of the real-time window has no relative-time interval
    assert np.abs(O.dos(c, g, 0, omega)).max() == 0.0
