"""dt -> 0 Lagrange extrapolation of the current on the GPU (Sec. II)."""

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


def test_extrapolation_exact_for_quadratic_dt_dependence():
    # j_k(t) = p(t) + a(t) dt_k + b(t) dt_k^2 on each run's own grid -> p(t) at dt = 0
    dts = [0.1, 1 / 15, 0.05]
    grids = [api.contour_grid(-5, 25, dt, 10.0, 0.1) for dt in dts]
    p = lambda t: np.sin(1.3 * t) * np.exp(-0.05 * t * t)
    a = lambda t: 0.7 * np.cos(t)
    b = lambda t: -2.0 + 0.1 * t
    cur = []
    for g, dt in zip(grids, dts):
        t = g.t[: g.n_t].real
        cur.append(torch.as_tensor(p(t) + a(t) * dt + b(t) * dt * dt, device="cuda"))
    t_out = np.arange(-5, 24.8, 0.2)  # common to all three grids
    out = api.extrapolate_current(grids, cur, t_out).cpu().numpy()
    assert np.abs(out - p(t_out)).max() < 1e-12


def test_extrapolation_matches_oracle_dmft_runs():
    # three FP64 DMFT runs on small contours, extrapolated on the GPU, against
    # the oracle's runs and its Lagrange extrapolation at common times
    dts = [0.2, 0.1, 0.05]
    model_o, model_c = O.Model(U=0.8, E=1.0), api.make_model(0.8, 1.0)
    js_o, grids, cur = [], [], []
    for dt in dts:
        args = (-1.0, 1.4, dt, 2.0, dt)
        c = O.contour_grid(*args)
        r = O.dmft_solve(c, model_o, n_quad=6, tol=1e-10, max_iter=80)
        assert r.converged
        g = api.contour_grid(*args)
        sol = api.dmft_solve(g, model_c, 6, "fp64", tol=1e-10, max_iter=80)
        assert sol.converged
        step = int(round(0.2 / dt))
        js_o.append(r.current.real[::step])  # the common times -1.0, -0.8, ..., 1.2
        grids.append(g)
        cur.append(sol.current)
    t_out = -1.0 + 0.2 * np.arange(len(js_o[0]))
    ref = O.lagrange_extrapolate(dts, np.array(js_o))
    out = api.extrapolate_current(grids, cur, t_out).cpu().numpy()
    assert np.abs(out - ref).max() < 1e-8


def test_extrapolation_rejects_times_outside_grids():
    grids = [api.contour_grid(-1, 1, dt, 1.0, 0.5) for dt in (0.2, 0.1)]
    cur = [torch.zeros(g.n_t, dtype=torch.float64, device="cuda") for g in grids]
    with pytest.raises(api.NedmftError):
        api.extrapolate_current(grids, cur, np.array([0.0, 5.0]))
