"""The DMFT loop of nedmft_dmft_solve (iteration 1 eager, every later
iteration one CUDA-graph launch on a private stream) against the same loop
driven step by step from Python through the lattice and impurity entry
points: the same kernels on the same inputs, so the results agree to
rounding, on the default stream and on a side stream."""

import contextlib

import numpy as np
import pytest
import torch

from paper_0711_0999_gb300 import api
from paper_0711_0999_gb300.build import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    build_library()


def eager_loop(g, m, n_quad, prec, tol, max_iter):
    eps, ebar, wq = api.quadrature_grid(n_quad)
    sigma = torch.zeros((g.n_c, g.n_c), dtype=torch.complex128, device="cuda")
    gl, j, _ = api.lattice_gloc(g, m, sigma, eps, ebar, wq, precision=prec)
    err = float("inf")
    it = 1
    while it < max_iter:
        it += 1
        sigma, _ = api.impurity_update(g, m, gl, sigma)
        gl_new, j, _ = api.lattice_gloc(g, m, sigma, eps, ebar, wq, precision=prec)
        err = float((gl_new - gl).abs().max() / gl_new.abs().max())
        gl = gl_new
        if err < tol:
            break
    torch.cuda.synchronize()
    return sigma, gl, j, it, err


@pytest.mark.parametrize("prec,side_stream", [("fp64", False), ("mixed_bf16", True)])
def test_graph_loop_matches_eager_loop(prec, side_stream):
    g = api.contour_grid(-2, 4, 0.2, 10, 0.5)
    m = api.make_model(0.5, 1.0)
    ref = eager_loop(g, m, 16, prec, 1e-8, 40)
    stream = torch.cuda.Stream() if side_stream else None
    with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
        sol = api.dmft_solve(g, m, 16, prec, tol=1e-8, max_iter=40, stream=stream)
    torch.cuda.synchronize()
    assert sol.converged
    assert sol.iterations == ref[3]
    scale = float(ref[1].abs().max())
    assert float((sol.gloc - ref[1]).abs().max()) / scale < 1e-12
    assert float((sol.sigma - ref[0]).abs().max()) / float(ref[0].abs().max()) < 1e-12
    assert np.abs(sol.current.cpu().numpy() - ref[2].cpu().numpy()).max() < 1e-12
    assert abs(sol.error - ref[4]) <= 1e-12 * max(1.0, ref[4])


def test_graph_loop_single_iteration():
    # max_iter = 1: no impurity step and no graph; not converged by definition
    g = api.contour_grid(-2, 4, 0.2, 10, 0.5)
    m = api.make_model(0.5, 1.0)
    sol = api.dmft_solve(g, m, 8, "fp64", tol=1e-8, max_iter=1)
    assert sol.iterations == 1 and not sol.converged
    eps, ebar, wq = api.quadrature_grid(8)
    gl, _, _ = api.lattice_gloc(g, m, torch.zeros_like(sol.sigma), eps, ebar, wq, precision="fp64")
    torch.cuda.synchronize()
    assert float((sol.gloc - gl).abs().max()) < 1e-14


def test_graph_loop_from_a_fresh_host_thread():
    # a host thread that has never run an impurity step captures the loop
    # (its look-ahead stream is made before the capture): the same result as
    # on the main thread, bit for bit
    import threading

    g = api.contour_grid(-2, 4, 0.2, 10, 0.5)
    m = api.make_model(0.5, 1.0)
    ref = api.dmft_solve(g, m, 8, "fp64", tol=1e-8, max_iter=40)
    torch.cuda.synchronize()
    out, errors = [], []

    def work():
        try:
            out.append(api.dmft_solve(g, m, 8, "fp64", tol=1e-8, max_iter=40))
            torch.cuda.synchronize()
        except Exception as e:  # reported below, on the main thread
            errors.append(e)

    t = threading.Thread(target=work)
    t.start()
    t.join()
    assert not errors, errors
    sol = out[0]
    assert sol.converged and sol.iterations == ref.iterations
    assert torch.equal(sol.gloc, ref.gloc) and torch.equal(sol.sigma, ref.sigma)
