"""Failure detection without a GPU fault: bounded waits that run out, pivots
below the threshold, non-finite inputs and a loop that stops at max_iter each
give a defined status, and the device stays usable afterwards.

The waits are made to run out by the library's own wait limit (a limit of 0
gives up on the first wait that is not already satisfied; a barrier that
nothing arrives at for the self-test); nothing here traps, faults or hangs.
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

SMALL = (-2, 4, 0.2, 10, 0.5)      # N_c = 80: the FP64 shared-memory path
BLOCKED = (-2, 3, 0.05, 5.0, 0.25)  # N_c = 220: blocked FP64 and tensor-core paths


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    build_library()
    yield
    api.set_wait_limit(2.0)


def status_code():
    try:
        api.check_status()
        return N.NEDMFT_OK
    except N.NedmftError as e:
        return e.code


def lattice(args, sigma, prec, U=1.0, E=1.0, nquad=4):
    g = api.contour_grid(*args)
    eps, ebar, wq = O.quadrature_points(nquad)
    gl, j, _ = api.lattice_gloc(g, api.make_model(U, E), torch.as_tensor(sigma, device="cuda"), eps, ebar, wq,
                                precision=prec)
    return gl, j


def parity_ok(args, prec, U=1.0, E=1.0):
    c = O.contour_grid(*args)
    sig = workload_sigma(c.t, c.w, U, seed=5)
    eps, ebar, wq = O.quadrature_points(4)
    ref, _ = O.lattice_gloc(c, O.Model(U=U, E=E), sig, eps, ebar, wq)
    gl, _ = lattice(args, sig, prec, U, E)
    torch.cuda.synchronize()
    assert status_code() == N.NEDMFT_OK
    tol = 1e-10 if prec == "fp64" else 1e-6
    return float(np.abs(gl.cpu().numpy() - ref).max() / np.abs(ref).max()) < tol


def test_wait_on_a_barrier_nothing_arrives_at_times_out():
    api.set_wait_limit(0.05)
    try:
        api.wait_selftest()
        assert status_code() == N.NEDMFT_ETIMEOUT
    finally:
        api.set_wait_limit(2.0)
    assert status_code() == N.NEDMFT_OK  # the word was cleared by the read
    assert parity_ok(BLOCKED, "mixed_bf16")


def test_expired_waits_abort_the_tensor_core_step_and_leave_the_device_usable():
    c = O.contour_grid(*BLOCKED)
    sig = workload_sigma(c.t, c.w, 1.0, seed=5)
    api.set_wait_limit(0.0)
    try:
        lattice(BLOCKED, sig, "mixed_bf16")
        assert status_code() == N.NEDMFT_ETIMEOUT
    finally:
        api.set_wait_limit(2.0)
    # the same call with the default limit is correct again
    assert parity_ok(BLOCKED, "mixed_bf16")


def test_wait_limit_rejects_out_of_range_values():
    lib = N.lib()
    assert lib.nedmft_set_wait_limit(-1.0, None) == N.NEDMFT_EINVAL
    assert lib.nedmft_set_wait_limit(61.0, None) == N.NEDMFT_EINVAL
    assert lib.nedmft_set_wait_limit(float("nan"), None) == N.NEDMFT_EINVAL


def singular_sigma(args, U, E):
    """Sigma with W Sigma W = B_q for the single point of a 1-point rule
    (eps = ebar = 0): the matrix B_q - S inverted by the lattice step is 0."""
    c = O.contour_grid(*args)
    b = np.linalg.inv(O.g0_matrix(c, O.Model(U=U, E=E), 0.0, 0.0))
    return b / (c.w[:, None] * c.w[None, :])


@pytest.mark.parametrize("args,prec", [(SMALL, "fp64"), (BLOCKED, "fp64"), (SMALL, "mixed_bf16"),
                                       (BLOCKED, "mixed_bf16")])
def test_singular_solve_reports_esingular(args, prec):
    lattice(args, singular_sigma(args, 1.0, 1.0), prec, nquad=1)
    assert status_code() == N.NEDMFT_ESINGULAR
    assert parity_ok(args, prec)


@pytest.mark.parametrize("args,prec", [(SMALL, "fp64"), (BLOCKED, "fp64"), (BLOCKED, "mixed_bf16")])
def test_non_finite_sigma_reports_esingular(args, prec):
    c = O.contour_grid(*args)
    sig = workload_sigma(c.t, c.w, 1.0, seed=6)
    sig[c.n_c // 3, c.n_c // 2] = np.nan
    lattice(args, sig, prec)
    assert status_code() == N.NEDMFT_ESINGULAR
    assert parity_ok(args, prec)


def test_impurity_step_on_a_singular_gloc_reports_esingular():
    g = api.contour_grid(*SMALL)
    z = torch.zeros((g.n_c, g.n_c), dtype=torch.complex128, device="cuda")
    api.impurity_update(g, api.make_model(1.0, 1.0), z, z)
    assert status_code() == N.NEDMFT_ESINGULAR


def _solve_rc(g, model, sigma_init, max_iter, tol=1e-12):
    need = N.lib().nedmft_dmft_workspace_size(ctypes.byref(g.contour), 8, N.FP64)
    ws = api.workspace(need)
    n = g.n_c
    out = [torch.empty((n, n), dtype=torch.complex128, device="cuda") for _ in range(2)]
    it, err = N.c_int32(0), N.c_double(0.0)
    P = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    rc = N.lib().nedmft_dmft_solve(ctypes.byref(g.contour), ctypes.byref(model), 8, N.FP64, P(sigma_init), tol,
                                   max_iter, P(out[0]), P(out[1]), None, ctypes.byref(it), ctypes.byref(err),
                                   P(ws), ws.numel(), None)
    return rc, it.value


def test_dmft_loop_stopped_by_max_iter_returns_enotconv():
    g = api.contour_grid(*SMALL)
    rc, it = _solve_rc(g, api.make_model(0.5, 1.0), None, max_iter=2)
    assert rc == N.NEDMFT_ENOTCONV and it == 2


def test_dmft_loop_from_a_non_finite_sigma_returns_esingular():
    c = O.contour_grid(*SMALL)
    g = api.contour_grid(*SMALL)
    sig = np.full((c.n_c, c.n_c), np.nan, dtype=np.complex128)
    rc, _ = _solve_rc(g, api.make_model(0.5, 1.0), torch.as_tensor(sig, device="cuda"), max_iter=3)
    assert rc == N.NEDMFT_ESINGULAR
    assert status_code() == N.NEDMFT_OK
