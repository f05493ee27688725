"""The allocation-free lattice entry point against the workspace entry point.

nedmft_lattice_gloc_static serves callers that cannot allocate device memory
(a host code that owns all device memory and passes only its input and output
buffers, or a plugin under a framework whose allocator owns the device): its
scratch is a fixed array inside the library.  This test calls it through the C
ABI twice in a row, with different inputs, and compares each result with
nedmft_lattice_gloc on the same inputs.  The file name makes pytest collect it
last.
"""

import ctypes

import numpy as np
import pytest
import torch

from oracle import nedmft_oracle as O
from paper_0711_0999_gb300 import _native as N
from paper_0711_0999_gb300 import api
from paper_0711_0999_gb300.build import build_library
from paper_0711_0999_gb300.synth import workload_sigma

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    build_library()


def _static_call(g, model, sigma, eps, ebar, wq):
    dev = sigma.device
    gloc = torch.empty_like(sigma)
    j = torch.empty(g.n_t, dtype=torch.float64, device=dev)
    ji = torch.empty(g.n_t, dtype=torch.float64, device=dev)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = N.lib().nedmft_lattice_gloc_static(ctypes.byref(g.contour), ctypes.byref(model), P(sigma), P(eps), P(ebar),
                                            P(wq), eps.numel(), P(gloc), P(j), P(ji),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(rc)
    torch.cuda.synchronize()
    api.check_status()
    return gloc, j, ji


def test_static_entry_matches_workspace_entry_twice():
    args = (-2, 4, 0.2, 10, 0.5)  # N_c = 80
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    model = api.make_model(0.5, 1.0)
    eps, ebar, wq = (torch.as_tensor(a, device="cuda") for a in O.quadrature_points(9))  # 81 points: 3 passes
    for seed in (1, 2):  # two calls in a row; the second must not see the first one's scratch
        sigma = torch.as_tensor(workload_sigma(c.t, c.w, 0.5, seed=seed), device="cuda")
        gs, js, jis = _static_call(g, model, sigma, eps, ebar, wq)
        gw, jw, jiw = api.lattice_gloc(g, model, sigma, eps, ebar, wq, precision="fp64")
        torch.cuda.synchronize()
        scale = gw.abs().max().item()
        assert (gs - gw).abs().max().item() < 1e-12 * scale
        assert (js - jw).abs().max().item() < 1e-12
        assert (jis - jiw).abs().max().item() < 1e-12


def test_static_entry_rejects_large_contours():
    g = api.contour_grid(-2, 4, 0.05, 10, 0.5)  # N_c = 260 > 112
    model = api.make_model(0.5, 1.0)
    z = torch.zeros((g.n_c, g.n_c), dtype=torch.complex128, device="cuda")
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = N.lib().nedmft_lattice_gloc_static(ctypes.byref(g.contour), ctypes.byref(model), P(z), P(e), P(e), P(e), 4,
                                            P(z), None, None, None)
    assert rc == N.NEDMFT_EINVAL
    assert b"static scratch limit" in N.lib().nedmft_last_error()


def test_static_entry_matches_the_oracle_and_runs_gloc_only_on_a_side_stream():
    # the result itself against the FP64 CPU oracle (1e-10 relative, the FP64
    # contract), then the G_loc-only form (no current outputs) on a
    # non-default stream against the workspace entry point on that stream
    args = (-2, 3, 0.1, 4.0, 0.5)  # N_c = 108, close to the 112 limit
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    assert g.n_c == 108
    mo, model = O.Model(U=1.0, E=2.0), api.make_model(1.0, 2.0)
    sig = workload_sigma(c.t, c.w, 1.0, seed=3)
    eps_h, ebar_h, wq_h = O.quadrature_points(6)
    ref, jref = O.lattice_gloc(c, mo, sig, eps_h, ebar_h, wq_h)
    sigma = torch.as_tensor(sig, device="cuda")
    eps, ebar, wq = (torch.as_tensor(a, device="cuda") for a in (eps_h, ebar_h, wq_h))
    gs, js, jis = _static_call(g, model, sigma, eps, ebar, wq)
    scale = np.abs(ref).max()
    assert np.abs(gs.cpu().numpy() - ref).max() < 1e-10 * scale
    assert np.abs(js.cpu().numpy() - jref.real).max() < 1e-10
    assert np.abs(jis.cpu().numpy() - jref.imag).max() < 1e-10

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    with torch.cuda.stream(side):
        gloc = torch.empty_like(sigma)
        rc = N.lib().nedmft_lattice_gloc_static(ctypes.byref(g.contour), ctypes.byref(model), P(sigma), P(eps),
                                                P(ebar), P(wq), eps.numel(), P(gloc), None, None,
                                                ctypes.c_void_p(side.cuda_stream))
        N.check(rc)
        gw, _, _ = api.lattice_gloc(g, model, sigma, eps, ebar, wq, precision="fp64", current=False, stream=side)
    side.synchronize()
    api.check_status(side)
    assert (gloc - gw).abs().max().item() < 1e-12 * scale
    assert np.abs(gloc.cpu().numpy() - ref).max() < 1e-10 * scale
