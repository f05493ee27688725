"""The GPU path against the values the paper states (tests/golden/paper_values.txt):
the converged DMFT solution's moment sum rules and half filling, from the
library's DMFT loop and moment kernels, after the Delta t -> 0 Lagrange
extrapolation (Sec. II) over three contours."""

import numpy as np
import pytest

from oracle import nedmft_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_golden_paper import P  # noqa: E402  (the parsed fixture)


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
@pytest.mark.parametrize("U", [1.0, 2.0])
def test_gpu_moment_sum_rules(precision, U):
    from paper_0711_0999_gb300 import api

    T = 0.5
    dts = (0.1, 0.05, 0.025)
    mu0, mu2, dens = [], [], []
    for dt in dts:
        g = api.contour_grid(-1.5, 1.5, dt, 2.0, dt)
        sol = api.dmft_solve(g, api.make_model(U, 1.0), 6, precision, tol=1e-9, max_iter=100)
        assert sol.converged
        m0, _, m2, n = (t.cpu().numpy() for t in api.moments(g, sol.gloc))
        m = int(round((T + 1.5) / dt))
        mu0.append(m0[m])
        mu2.append(m2[m])
        dens.append(n[m])
    exact2 = P["moment2_band"] + P["moment2_u2"] * U * U
    assert O.lagrange_extrapolate(list(dts), np.array(mu0)) == pytest.approx(P["moment0"], rel=5e-3)
    assert O.lagrange_extrapolate(list(dts), np.array(mu2)) == pytest.approx(exact2, rel=5e-3)
    assert abs(O.lagrange_extrapolate(list(dts), np.array(dens)) - P["filling"]) < 5e-3
