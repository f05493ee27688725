"""Parity of the CUDA lattice step (through the C ABI) with the FP64 CPU oracle.

Tolerances (from the contract of the two paths): FP64 path 1e-10 relative on
G_loc (max-norm), mixed paths 1e-6 relative on G_loc; the current 1e-5
absolute on the mixed paths and 1e-10 on the FP64 path.
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

TOL = {"fp64": (1e-10, 1e-10), "mixed_bf16": (1e-6, 1e-5)}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    build_library()


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def setup(args, U, E, nquad, seed=1, sigma_scale=1.0):
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    model_o = O.Model(U=U, E=E)
    model_c = api.make_model(U, E)
    sig = sigma_scale * workload_sigma(c.t, c.w, U if U > 0 else 0.5, seed=seed)
    eps, ebar, wq = O.quadrature_points(nquad)
    return c, g, model_o, model_c, sig, eps, ebar, wq


def run_gpu(g, model_c, sig, eps, ebar, wq, prec):
    s = torch.as_tensor(sig, device="cuda")
    gl, j, ji = api.lattice_gloc(g, model_c, s, eps, ebar, wq, precision=prec)
    torch.cuda.synchronize()
    api.check_status()
    return gl.cpu().numpy(), j.cpu().numpy(), ji.cpu().numpy()


# ------------------------------------------------------------------ G0


@pytest.mark.parametrize("E", [1.0, 0.0, 2.5])
def test_g0_build_matches_oracle(E):
    args = (-2, 3, 0.2, 4.0, 0.5)
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    m_o, m_c = O.Model(U=0.8, E=E), api.make_model(0.8, E)
    eps = np.array([-4.5, -1.1, 0.0, 0.37, 2.2, 5.0])
    ebar = np.array([1.0, -0.3, 0.9, -2.0, 0.0, 3.1])
    g0 = api.g0_build(g, m_c, eps, ebar).cpu().numpy()
    for q in range(len(eps)):
        ref = O.g0_matrix(c, m_o, eps[q], ebar[q])
        assert np.abs(g0[q] - ref).max() < 1e-12


# ------------------------------------------------------------------ lattice step


@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16"])
def test_lattice_cfg_small_contour(prec):
    # N_c = 80 contour of the CPU-sized configuration, 16 x 16 points
    c, g, mo, mc, sig, eps, ebar, wq = setup((-2, 4, 0.2, 10, 0.5), 0.5, 1.0, 16)
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    gl, j, ji = run_gpu(g, mc, sig, eps, ebar, wq, prec)
    tg, tj = TOL[prec]
    assert rel(gl, ref) < tg
    assert np.abs(j - jref.real).max() < tj
    assert np.abs(ji - jref.imag).max() < tj


@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16"])
def test_lattice_ragged_blocked(prec):
    # N_c = 220: several 64/128 tiles and a ragged tail; E = 2, U = 1.5
    c, g, mo, mc, sig, eps, ebar, wq = setup((-2, 3, 0.05, 5.0, 0.25), 1.5, 2.0, 6, seed=4)
    assert c.n_c == 220
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    gl, j, ji = run_gpu(g, mc, sig, eps, ebar, wq, prec)
    tg, tj = TOL[prec]
    assert rel(gl, ref) < tg
    assert np.abs(j - jref.real).max() < tj


@pytest.mark.parametrize("args,n_c", [((-2, 8, 0.05, 5.0, 0.1), 450), ((-2, 14.5, 0.05, 4.0, 0.1), 700)])
def test_lattice_wide_gauss_jordan_blocks(args, n_c):
    # padded sizes 512 and 768: the tensor-core Gauss-Jordan runs in blocks of
    # 256 columns (2 and 3 steps, each pivot block inverted by the 128 blocks)
    c, g, mo, mc, sig, eps, ebar, wq = setup(args, 1.0, 1.5, 4, seed=11)
    assert c.n_c == n_c
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    gl, j, ji = run_gpu(g, mc, sig, eps, ebar, wq, "mixed_bf16")
    tg, tj = TOL["mixed_bf16"]
    assert rel(gl, ref) < tg
    assert np.abs(j - jref.real).max() < tj
    assert np.abs(ji - jref.imag).max() < tj


@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16"])
@pytest.mark.parametrize("args,n_c", [((-2, 2, 0.25, 3.5, 0.5), 39), ((-2, 3, 0.05, 5.5, 0.5), 211),
                                      ((-2, 4, 0.02, 10.5, 0.5), 621)])
def test_lattice_odd_contour_sizes(prec, args, n_c):
    # an odd number of thermal points makes N_c odd: rows of odd length in the
    # FP64 small and blocked paths, and on the mixed path padded to 128, 256
    # and 640 (128-column steps chosen by the padding rule)
    c, g, mo, mc, sig, eps, ebar, wq = setup(args, 1.0, 1.5, 3, seed=13)
    assert c.n_c == n_c
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    gl, j, ji = run_gpu(g, mc, sig, eps, ebar, wq, prec)
    tg, tj = TOL[prec]
    assert rel(gl, ref) < tg
    assert np.abs(j - jref.real).max() < tj
    assert np.abs(ji - jref.imag).max() < tj


@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16"])
@pytest.mark.parametrize("args,n_c", [((0, 1, 1.0, 1.0, 1.0), 3), ((0, 1, 1.0, 2.0, 1.0), 4),
                                      ((0, 2, 1.0, 4.0, 1.0), 8), ((-1, 2, 0.5, 0.5, 0.5), 13)])
def test_tiny_contours(prec, args, n_c):
    # the smallest contours (one real step, one thermal point, ...): the lattice
    # step on both paths and the impurity step against the oracle
    c, g, mo, mc, sig, eps, ebar, wq = setup(args, 1.0, 1.0, 4, seed=17)
    assert c.n_c == n_c
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    gl, j, ji = run_gpu(g, mc, sig, eps, ebar, wq, prec)
    tg, tj = TOL[prec]
    assert rel(gl, ref) < tg
    assert np.abs(j - jref.real).max() < tj
    assert np.abs(ji - jref.imag).max() < tj
    if prec == "fp64":
        s_ref, gi_ref = O.impurity_update(c, mo, ref, sig)
        s_new, gimp = api.impurity_update(g, mc, torch.as_tensor(ref, device="cuda"),
                                          torch.as_tensor(sig, device="cuda"), want_gimp=True)
        torch.cuda.synchronize()
        api.check_status()
        sw = lambda s: c.w[:, None] * s * c.w[None, :]
        assert rel(sw(s_new.cpu().numpy()), sw(s_ref)) < 1e-10
        assert rel(gimp.cpu().numpy(), gi_ref) < 1e-10


def test_lattice_many_batches_fp64():
    # more points than one batch of the blocked FP64 path (152), N_c = 130
    c, g, mo, mc, sig, eps, ebar, wq = setup((-1, 2, 0.05, 1.0, 0.1), 1.0, 1.0, 13, seed=9)
    assert c.n_c == 130 and len(wq) == 169
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    gl, j, _ = run_gpu(g, mc, sig, eps, ebar, wq, "fp64")
    assert rel(gl, ref) < 1e-10
    assert np.abs(j - jref.real).max() < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16"])
def test_lattice_single_point_and_e0(prec):
    c, g, mo, mc, sig, eps, ebar, wq = setup((-2, 2, 0.25, 3.0, 0.5), 1.0, 0.0, 1)
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    gl, j, ji = run_gpu(g, mc, sig, eps, ebar, wq, prec)
    assert rel(gl, ref) < TOL[prec][0]
    assert np.abs(j).max() < 1e-12  # E = 0, single node at 0


@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16"])
def test_u0_closed_form_current_and_density(prec):
    # Sigma = 0, mu = 0: j(t) = -sin(Et) sum_a w_a x_a f(x_a) for t > 0, n(t) = 1/2
    args = (-3, 9, 0.05, 10.0, 0.1)
    g = api.contour_grid(*args)
    c = O.contour_grid(*args)
    x, w = O.gauss_hermite(20)
    eps, ebar, wq = O.quadrature_points(20)
    gl, j, _ = run_gpu(g, api.make_model(0.0, 1.0), np.zeros((g.n_c, g.n_c), complex), eps, ebar, wq, prec)
    amp = float(np.sum(w * x / (1 + np.exp(10.0 * x))))
    tm = c.t[: c.n_t].real
    expect = np.where(tm > 0, -np.sin(tm) * amp, 0.0)
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert np.abs(j - expect).max() < tol
    assert np.abs(O.density(c, gl) - 0.5).max() < tol


def test_current_entry_point_matches_lattice():
    c, g, mo, mc, sig, eps, ebar, wq = setup((-2, 4, 0.2, 10, 0.5), 0.5, 1.0, 8)
    s = torch.as_tensor(sig, device="cuda")
    _, j1, ji1 = api.lattice_gloc(g, mc, s, eps, ebar, wq)
    j2, ji2 = api.current(g, mc, s, eps, ebar, wq)
    assert torch.equal(j1, j2) and torch.equal(ji1, ji2)


def test_full_size_sampled_points():
    # N_c = 1500 contour (t in [-5, 30], dt = 0.05, dtau = 0.1), U = E = 1,
    # a sample of the 53 x 53 grid: extreme and central eps, any ebar.
    args = (-5, 30, 0.05, 10.0, 0.1)
    c, g, mo, mc, sig, _, _, _ = setup(args, 1.0, 1.0, 2, seed=12)
    eps_all, ebar_all, wq_all = O.quadrature_points(53)
    pick = [0 * 53 + 7, 10 * 53 + 26, 26 * 53 + 3, 27 * 53 + 40, 40 * 53 + 20, 52 * 53 + 52]
    eps, ebar, wq = eps_all[pick], ebar_all[pick], wq_all[pick] / wq_all[pick].sum()
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    for prec in ("fp64", "mixed_bf16"):
        gl, j, _ = run_gpu(g, mc, sig, eps, ebar, wq, prec)
        tg, tj = TOL[prec]
        assert rel(gl, ref) < tg, prec
        assert np.abs(j - jref.real).max() < tj, prec


# ------------------------------------------------------------------ errors


def test_lattice_errors():
    g = api.contour_grid(-2, 4, 0.2, 10, 0.5)
    mc = api.make_model(0.5, 1.0)
    s = torch.zeros((g.n_c, g.n_c), dtype=torch.complex128, device="cuda")
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.empty_like(s)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    lib = N.lib()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.nedmft_lattice_gloc(ctypes.byref(g.contour), ctypes.byref(mc), P(s), P(e), P(e), P(e), 4, 0, P(out),
                                 None, None, P(small), small.numel(), None)
    assert rc == N.NEDMFT_ENOMEM
    rc = lib.nedmft_lattice_gloc(ctypes.byref(g.contour), ctypes.byref(mc), P(s), P(e), P(e), P(e), 0, 0, P(out),
                                 None, None, P(small), small.numel(), None)
    assert rc == N.NEDMFT_EINVAL
    rc = lib.nedmft_lattice_gloc(ctypes.byref(g.contour), ctypes.byref(mc), P(s), P(e), P(e), P(e), 4, 9, P(out),
                                 None, None, P(small), small.numel(), None)
    assert rc == N.NEDMFT_EINVAL
    assert b"precision" in lib.nedmft_last_error()


# ------------------------------------------------------------------ impurity and loop


def test_impurity_update_matches_oracle():
    c, g, mo, mc, sig, eps, ebar, wq = setup((-2, 4, 0.2, 10, 0.5), 0.5, 1.0, 8)
    gl, _ = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    s_ref, gi_ref = O.impurity_update(c, mo, gl, sig)
    s_new, gimp = api.impurity_update(g, mc, torch.as_tensor(gl, device="cuda"), torch.as_tensor(sig, device="cuda"),
                                      want_gimp=True)
    torch.cuda.synchronize()
    api.check_status()
    w = c.w
    sw = lambda s: w[:, None] * s * w[None, :]
    assert rel(sw(s_new.cpu().numpy()), sw(s_ref)) < 1e-10
    assert rel(gimp.cpu().numpy(), gi_ref) < 1e-10


@pytest.mark.parametrize("args", [(-1, 1, 0.25, 2.0, 0.5), (-1, 1, 0.125, 2.0, 0.5), (-2, 4, 0.2, 10, 0.5),
                                  (-2, 2, 0.1, 4.0, 0.25), (-2, 3, 0.05, 5.0, 0.25), (-2, 3, 0.05, 5.5, 0.5),
                                  (-2, 4, 0.02, 10, 0.5)])
def test_impurity_update_needs_pivoting(args):
    # G_loc = (cyclic row shift)(I + 0.3 R) with its diagonal set to zero:
    # every pivot of an elimination without row exchanges is 0 at the first
    # step, so the inversions need them; N_c = 20 (one 32-column step), 36 (a
    # four-column last step), 80, 96 (three full steps), 220, 211 (odd) and
    # 620 (ragged last blocks; 620 rows take two tournament rounds per step)
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    n = c.n_c
    rng = np.random.default_rng(7)
    base = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    gl = np.roll(base, 1, axis=0).astype(np.complex128)
    np.fill_diagonal(gl, 0.0)
    sig = workload_sigma(c.t, c.w, 1.0, seed=3)
    mo, mc = O.Model(U=1.0, E=1.0), api.make_model(1.0, 1.0)
    s_ref, gi_ref = O.impurity_update(c, mo, gl, sig)
    s_new, gimp = api.impurity_update(g, mc, torch.as_tensor(gl, device="cuda"), torch.as_tensor(sig, device="cuda"),
                                      want_gimp=True)
    torch.cuda.synchronize()
    api.check_status()
    w = c.w
    sw = lambda s: w[:, None] * s * w[None, :]
    assert rel(sw(s_new.cpu().numpy()), sw(s_ref)) < 1e-10
    assert rel(gimp.cpu().numpy(), gi_ref) < 1e-10


@pytest.mark.parametrize("scale", [1e-24, 1e20])
def test_impurity_update_at_large_and_small_scales(scale):
    # G_loc scaled by 1e-24 or 1e20: the inversions see entries near 1e-24 and
    # 1e24 (or 1e20), past the range where the tensor-core update applies its
    # powers of two in FP32, and the pivoted inversion normalises the scale;
    # G_imp matches the oracle to 1e-10 relative.  W Sigma W is compared at
    # 1e20 only: at 1e-24 it is the difference of two matrices near 1e24,
    # which leaves the oracle's own FP64 value at the level of its rounding.
    args = (-2, 3, 0.05, 5.0, 0.25)  # N_c = 220
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    n = c.n_c
    rng = np.random.default_rng(5)
    base = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    gl = scale * np.roll(base, 1, axis=0).astype(np.complex128)
    np.fill_diagonal(gl, 0.0)
    sig = workload_sigma(c.t, c.w, 1.0, seed=3)
    mo, mc = O.Model(U=1.0, E=1.0), api.make_model(1.0, 1.0)
    s_ref, gi_ref = O.impurity_update(c, mo, gl, sig)
    s_new, gimp = api.impurity_update(g, mc, torch.as_tensor(gl, device="cuda"), torch.as_tensor(sig, device="cuda"),
                                      want_gimp=True)
    torch.cuda.synchronize()
    api.check_status()
    w = c.w
    sw = lambda s: w[:, None] * s * w[None, :]
    if scale > 1.0:
        assert rel(sw(s_new.cpu().numpy()), sw(s_ref)) < 1e-10
    assert rel(gimp.cpu().numpy(), gi_ref) < 1e-10


def test_impurity_update_from_two_host_threads_matches_sequential_calls():
    # each host thread gets its own look-ahead stream: two threads calling the
    # impurity step at once, each on its own stream, give bit for bit the
    # results of the same calls made one after the other (N_c = 220: 7 steps)
    import threading

    args = (-2, 3, 0.05, 5.0, 0.25)
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    n = c.n_c
    mc = api.make_model(1.0, 1.0)
    inputs = []
    for seed in (11, 12):
        rng = np.random.default_rng(seed)
        base = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
        gl = np.roll(base, 1, axis=0).astype(np.complex128)
        np.fill_diagonal(gl, 0.0)
        inputs.append((torch.as_tensor(gl, device="cuda"),
                       torch.as_tensor(workload_sigma(c.t, c.w, 1.0, seed=seed), device="cuda")))
    ref = [api.impurity_update(g, mc, gl, sig, want_gimp=True) for gl, sig in inputs]
    torch.cuda.synchronize()
    api.check_status()
    out = [None, None]
    errors = []
    start = threading.Barrier(2)

    def work(k):
        try:
            s = torch.cuda.Stream()
            start.wait()
            with torch.cuda.stream(s):
                for _ in range(4):
                    out[k] = api.impurity_update(g, mc, *inputs[k], want_gimp=True, stream=s)
            s.synchronize()
        except Exception as e:  # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    api.check_status()
    for k in range(2):
        assert torch.equal(out[k][0], ref[k][0]) and torch.equal(out[k][1], ref[k][1])


def test_dmft_solve_small_config_matches_oracle():
    args = (-2, 4, 0.2, 10, 0.5)
    c = O.contour_grid(*args)
    g = api.contour_grid(*args)
    ref = O.dmft_solve(c, O.Model(U=0.5, E=1.0), n_quad=16, tol=1e-8, max_iter=50)
    sol = api.dmft_solve(g, api.make_model(0.5, 1.0), 16, "fp64", tol=1e-8, max_iter=50)
    assert ref.converged and sol.converged
    assert sol.iterations == ref.iterations <= 50
    assert rel(sol.gloc.cpu().numpy(), ref.gloc) < 1e-9
    assert np.abs(sol.current.cpu().numpy() - ref.current.real).max() < 1e-9
    w = c.w
    sw = lambda s: w[:, None] * s * w[None, :]
    assert rel(sw(sol.sigma.cpu().numpy()), sw(ref.sigma)) < 1e-8


def test_largest_contour_of_the_paper_sampled_points():
    # N_c = 5700, the paper's largest contour (t in [-5, 51], dt = 0.02, dtau =
    # 0.1): 2 points of the 16 x 16 grid near its centre, weights renormalised;
    # the mixed path pads to 5888 (23 steps of 256 columns)
    args = (-5, 51, 0.02, 10.0, 0.1)
    c, g, mo, mc, sig, _, _, _ = setup(args, 1.0, 1.0, 2, seed=23)
    assert c.n_c == 5700
    eps_all, ebar_all, wq_all = O.quadrature_points(16)
    pick = [7 * 16 + 8, 8 * 16 + 6]
    eps, ebar, wq = eps_all[pick], ebar_all[pick], wq_all[pick] / wq_all[pick].sum()
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    for prec in ("mixed_bf16", "fp64"):
        gl, j, _ = run_gpu(g, mc, sig, eps, ebar, wq, prec)
        tg, tj = TOL[prec]
        assert rel(gl, ref) < tg, prec
        assert np.abs(j - jref.real).max() < tj, prec


def test_long_contour_sampled_points():
    # N_c = 3400 contour (t in [-5, 50], dt = 1/30, dtau = 0.1), U = 2, E = 1:
    # the Mott-insulating long-time shape; 8 points of the 64 x 64 grid near its
    # centre, with their own weights renormalised (an integral-like sample)
    args = (-5, 50, 1 / 30, 10.0, 0.1)
    c, g, mo, mc, sig, _, _, _ = setup(args, 2.0, 1.0, 2, seed=21)
    assert c.n_c == 3400
    eps_all, ebar_all, wq_all = O.quadrature_points(64)
    pick = [a * 64 + b for a in (30, 33) for b in (27, 31, 33, 37)]
    eps, ebar, wq = eps_all[pick], ebar_all[pick], wq_all[pick] / wq_all[pick].sum()
    ref, jref = O.lattice_gloc(c, mo, sig, eps, ebar, wq)
    for prec in ("mixed_bf16", "fp64"):
        gl, j, _ = run_gpu(g, mc, sig, eps, ebar, wq, prec)
        tg, tj = TOL[prec]
        assert rel(gl, ref) < tg, prec
        assert np.abs(j - jref.real).max() < tj, prec
