"""The oracle against the values the paper states (tests/golden/paper_values.txt):
the contour's imaginary branch, the Bloch periods of the noninteracting current,
and the sum rules of the local retarded function in the interacting, converged
DMFT solution after the Delta t -> 0 Lagrange extrapolation (Sec. II) that the
paper itself checks against them."""

import math
import os

import numpy as np
import pytest

from oracle import nedmft_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.txt")


def paper_values():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, rest = line.split("=", 1)
        value, cite = rest.split(";", 1)
        assert cite.strip(), key  # every value carries its source
        vals[key.strip()] = float(value)
    return vals


P = paper_values()


def test_contour_imaginary_branch():
    c = O.contour_grid(-5, 30, 0.05, P["beta"], P["dtau"])
    assert c.n_tau == P["imag_points"]
    tau = c.t[2 * c.n_t:]
    # from t_min down to t_min - i beta + i dtau, in steps of dtau
    assert abs(tau[0] - c.t[0]) < 1e-12
    assert abs(tau[-1] - (c.t[0] - 1j * P["beta"] + 1j * P["dtau"])) < 1e-12
    assert np.allclose(np.diff(tau), -1j * P["dtau"])


def zero_crossings(t, y):
    out = []
    for k in range(len(y) - 1):
        if y[k] == 0.0 or (y[k] < 0) != (y[k + 1] < 0):
            out.append(t[k] - y[k] * (t[k + 1] - t[k]) / (y[k + 1] - y[k]))
    return np.array(out)


@pytest.mark.parametrize("E,key", [(0.125, "bloch_period_e0.125"), (0.25, "bloch_period_e0.25")])
def test_bloch_period_of_the_free_current(E, key):
    # the oracle's U = 0 current, read off its sign changes after the field is on
    t_max = -1 + 0.25 * math.ceil((3.3 * math.pi / E + 2) / 0.25)  # on the grid, past three sign changes
    c = O.contour_grid(-1, t_max, 0.25, 2.0, 0.5)
    eps, ebar, wq = O.quadrature_points(6)
    _, j = O.lattice_gloc(c, O.Model(U=0.0, E=E), np.zeros((c.n_c, c.n_c), complex), eps, ebar, wq)
    t = c.t[: c.n_t].real
    keep = t > 1.0
    z = zero_crossings(t[keep], j.real[keep])
    assert len(z) >= 3
    period = 2 * float(np.mean(np.diff(z)))
    assert period == pytest.approx(2 * math.pi / E, rel=1e-3)
    assert period == pytest.approx(P[key], rel=1e-2)  # the paper's rounded value


@pytest.mark.parametrize("U", [0.5, 1.0, 2.0])
def test_moment_sum_rules_of_the_interacting_solution(U):
    # converged DMFT on a short contour at dt = dtau = 0.1, 0.05, 0.025; the
    # moments at T = 0.5 (after the field is switched on) extrapolated to dt -> 0
    T = 0.5
    dts = (0.1, 0.05, 0.025)
    mu0, mu2, dens = [], [], []
    for dt in dts:
        c = O.contour_grid(-1.5, 1.5, dt, 2.0, dt)
        r = O.dmft_solve(c, O.Model(U=U, E=1.0), n_quad=6, tol=1e-9, max_iter=100)
        assert r.converged
        m0, _, m2, n = O.moments(c, r.gloc)
        m = int(round((T - c.t[0].real) / dt))
        assert abs(c.t[m].real - T) < 1e-12
        mu0.append(m0[m])
        mu2.append(m2[m])
        dens.append(n[m].real)
    x0 = O.lagrange_extrapolate(list(dts), np.array(mu0))
    x2 = O.lagrange_extrapolate(list(dts), np.array(mu2))
    assert x0 == pytest.approx(P["moment0"], rel=5e-3)
    assert x2 == pytest.approx(P["moment2_band"] + P["moment2_u2"] * U * U, rel=5e-3)
    # the extrapolation is what brings mu2 there: the coarsest grid alone misses it
    assert abs(mu2[0] - (P["moment2_band"] + P["moment2_u2"] * U * U)) > 2 * abs(
        x2 - (P["moment2_band"] + P["moment2_u2"] * U * U))
    # half filling, approached as dt -> 0
    assert abs(O.lagrange_extrapolate(list(dts), np.array(dens)) - P["filling"]) < 5e-3
