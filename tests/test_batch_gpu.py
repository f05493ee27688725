"""Several DMFT runs swept together (nedmft_dmft_solve_batch) against each run
solved alone (nedmft_dmft_solve): the same kernels in the same order per run,
so iterations agree and results agree to rounding; runs of different contour
lengths and a run that stops at max_iter.  And the batch autotuner: it picks
one of its candidates, later lattice steps use it, and the result does not
depend on the batch size beyond rounding."""

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


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16"])
def test_batch_matches_single_runs(prec):
    grids = [api.contour_grid(-2, 4, 0.2, 10, 0.5), api.contour_grid(-2, 4, 0.2, 10, 0.5),
             api.contour_grid(-2, 5, 0.125, 8, 0.5)]
    models = [api.make_model(0.5, 1.0), api.make_model(1.0, 2.0), api.make_model(0.75, 0.5)]
    sols = api.dmft_solve_batch(grids, models, 12, prec, tol=1e-8, max_iter=60)
    for g, m, s in zip(grids, models, sols):
        ref = api.dmft_solve(g, m, 12, prec, tol=1e-8, max_iter=60)
        assert s.converged == ref.converged and s.iterations == ref.iterations
        assert rel(s.gloc, ref.gloc) < 1e-12
        assert rel(s.sigma, ref.sigma) < 1e-12
        assert float((s.current - ref.current).abs().max()) < 1e-12
        assert abs(s.error - ref.error) <= 1e-12 * max(1.0, ref.error)


def test_batch_ragged_stop():
    grids = [api.contour_grid(-2, 4, 0.2, 10, 0.5), api.contour_grid(-2, 3, 0.25, 6, 0.5)]
    models = [api.make_model(0.5, 1.0), api.make_model(1.5, 1.0)]
    sols = api.dmft_solve_batch(grids, models, 8, "fp64", tol=1e-14, max_iter=5)
    for s in sols:
        assert not s.converged and s.iterations == 5
    ref = api.dmft_solve(grids[1], models[1], 8, "fp64", tol=1e-14, max_iter=5)
    assert rel(sols[1].gloc, ref.gloc) < 1e-12


def test_autotune_picks_a_candidate():
    g = api.contour_grid(-2, 3, 0.05, 5.0, 0.25)  # N_c = 220
    m = api.make_model(1.0, 1.0)
    eps, ebar, wq = api.quadrature_grid(8)
    sig = torch.zeros((g.n_c, g.n_c), dtype=torch.complex128, device="cuda")
    before, _, _ = api.lattice_gloc(g, m, sig, eps, ebar, wq, precision="mixed_bf16")
    best, ms = api.lattice_autotune(g, m, sig, eps, ebar, wq, "mixed_bf16", candidates=[16, 32, 64])
    assert best in (16, 32, 64) and ms > 0
    assert api.lattice_batch(g, 64, "mixed_bf16") == best
    after, _, _ = api.lattice_gloc(g, m, sig, eps, ebar, wq, precision="mixed_bf16")
    torch.cuda.synchronize()
    assert rel(after, before) < 1e-12


def test_mixed_run_batch_matches_the_oracle():
    # a batch of runs with two contour lengths and three (U, E) pairs on the
    # mixed path against the oracle's DMFT loop for each run (converged to
    # 1e-8; the mixed path's converged G_loc within 1e-6, j(t) within 1e-5)
    args = [(-2, 4, 0.2, 10, 0.5), (-2, 4, 0.2, 10, 0.5), (-2, 3, 0.1, 6, 0.5)]
    models = [(0.5, 1.0), (1.0, 2.0), (0.75, 0.5)]
    sols = api.dmft_solve_batch([api.contour_grid(*a) for a in args], [api.make_model(*m) for m in models], 10,
                                "mixed_bf16", tol=1e-8, max_iter=80)
    for a, (U, E), s in zip(args, models, sols):
        ref = O.dmft_solve(O.contour_grid(*a), O.Model(U=U, E=E), n_quad=10, tol=1e-8, max_iter=80)
        assert ref.converged and s.converged
        g = s.gloc.cpu().numpy()
        assert np.abs(g - ref.gloc).max() < 1e-6 * np.abs(ref.gloc).max()
        assert np.abs(s.current.cpu().numpy() - ref.current.real).max() < 1e-5


def test_block_width_choice_pads_and_solves_correctly():
    # N_c = 620: 256-column steps pad to 768, 128-column steps to 640 (the
    # default here); both match the oracle, and the autotuner records one of
    # the (batch, width) pairs it tried
    args = (-2, 12.5, 0.05, 4.0, 0.1)
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    assert g.n_c == 620
    m = api.make_model(1.0, 1.5)
    from paper_0711_0999_gb300.synth import workload_sigma
    sig = workload_sigma(c.t, c.w, 1.0, seed=8)
    eps, ebar, wq = O.quadrature_points(3)
    ref, jref = O.lattice_gloc(c, O.Model(U=1.0, E=1.5), sig, eps, ebar, wq)
    s = torch.as_tensor(sig, device="cuda")
    assert api.lattice_block_width(g, 9) == 128  # 640 vs 768 rows: (5/6)^3 < 0.8, the default pads to 128
    for width in (256, 128):
        api.lattice_set_tuning(g, 9, "mixed_bf16", batch=0, width=width)
        assert api.lattice_block_width(g, 9) == width
        gl, j, _ = api.lattice_gloc(g, m, s, eps, ebar, wq, precision="mixed_bf16")
        torch.cuda.synchronize()
        api.check_status()
        assert np.abs(gl.cpu().numpy() - ref).max() < 1e-6 * np.abs(ref).max(), width
        assert np.abs(j.cpu().numpy() - jref.real).max() < 1e-5, width
    best, ms = api.lattice_autotune(g, m, s, eps, ebar, wq, "mixed_bf16", candidates=[5, 9])
    assert best in (5, 9) and ms > 0 and api.lattice_block_width(g, 9) in (128, 256)


def test_default_width_follows_the_padding():
    # N_c = 1300 pads to 1408 with 128-column steps (0.77 of the flops of 1536): the default takes them;
    # N_c = 1500 pads to 1536 either way: 256
    g1300 = api.contour_grid(-5, 25, 0.05, 10.0, 0.1)
    g1500 = api.contour_grid(-5, 30, 0.05, 10.0, 0.1)
    assert g1300.n_c == 1300 and g1500.n_c == 1500
    assert api.lattice_block_width(g1300, 1600) == 128
    assert api.lattice_block_width(g1500, 2809) == 256
