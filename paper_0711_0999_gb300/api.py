"""Python binding of the lattice-step library: the C ABI with the same names.

Marshalling only: arguments become pointers into torch tensors (device memory,
streams) or numpy arrays (host-only grid calls), every computation runs in
``libnedmft.so``.  Functions mirror ``include/nedmft.h`` without the
``nedmft_`` prefix.
"""

from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N
from ._native import FP64, MIXED_BF16, NedmftError, PRECISIONS  # noqa: F401


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, device):
    if isinstance(t, torch.Tensor):
        assert t.is_cuda and t.dtype == dtype and t.is_contiguous(), "expected a contiguous CUDA tensor"
        return t
    return torch.as_tensor(np.ascontiguousarray(t), dtype=dtype, device=device)


def version() -> str:
    return N.lib().nedmft_version().decode()


def check_status(stream=None) -> None:
    N.check(N.lib().nedmft_check_status(ctypes.c_void_p(_stream(stream))))


def set_wait_limit(seconds: float, stream=None) -> None:
    """Limit of the bounded device waits of the tensor-core kernels on the current device."""
    N.check(N.lib().nedmft_set_wait_limit(float(seconds), ctypes.c_void_p(_stream(stream))))


def wait_selftest(stream=None) -> None:
    """One bounded wait on a barrier that nothing arrives at (then check_status raises ETIMEOUT)."""
    N.check(N.lib().nedmft_wait_selftest(ctypes.c_void_p(_stream(stream))))


def make_model(U: float, E: float, w1: float = 0.5, mu: float | None = None) -> N.Model:
    return N.Model(U, E, w1, math.nan if mu is None else mu)


@dataclass
class Grid:
    contour: N.Contour
    t: np.ndarray  # complex128 contour times
    w: np.ndarray  # complex128 weights

    @property
    def n_c(self) -> int:
        return self.contour.n_c

    @property
    def n_t(self) -> int:
        return self.contour.n_t


def contour_grid(t_min: float, t_max: float, dt: float, beta: float, dtau: float) -> Grid:
    c = N.Contour()
    N.check(N.lib().nedmft_contour_grid(t_min, t_max, dt, beta, dtau, ctypes.byref(c), None, None))
    t = np.zeros(c.n_c, np.complex128)
    w = np.zeros(c.n_c, np.complex128)
    N.check(N.lib().nedmft_contour_grid(t_min, t_max, dt, beta, dtau, ctypes.byref(c),
                                        t.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)))
    return Grid(c, t, w)


def gauss_hermite(n: int):
    x = np.zeros(max(n, 1))
    w = np.zeros(max(n, 1))
    N.check(N.lib().nedmft_gauss_hermite(n, x.ctypes.data_as(N.PD), w.ctypes.data_as(N.PD)))
    return x, w


def quadrature_grid(n: int):
    e, b, w = np.zeros(n * n), np.zeros(n * n), np.zeros(n * n)
    N.check(N.lib().nedmft_quadrature_grid(n, e.ctypes.data_as(N.PD), b.ctypes.data_as(N.PD), w.ctypes.data_as(N.PD)))
    return e, b, w


def quadrature_grid_avg(n: int):
    m = n * n + (n + 1) * (n + 1)
    e, b, w = np.zeros(m), np.zeros(m), np.zeros(m)
    N.check(N.lib().nedmft_quadrature_grid_avg(n, e.ctypes.data_as(N.PD), b.ctypes.data_as(N.PD),
                                               w.ctypes.data_as(N.PD)))
    return e, b, w


def extrapolate_current(grids, currents, t_out, stream=None) -> torch.Tensor:
    """dt -> 0 Lagrange extrapolation of j(t) from runs on several contour grids."""
    k = len(grids)
    dev = currents[0].device
    dts = np.array([g.contour.dt for g in grids], dtype=np.float64)
    tmins = np.array([g.contour.t_min for g in grids], dtype=np.float64)
    nts = np.array([g.contour.n_t for g in grids], dtype=np.int32)
    ptrs = (ctypes.c_void_p * k)(*[c.data_ptr() for c in currents])
    t_d = _dev(t_out, torch.float64, dev)
    out = torch.empty(t_d.numel(), dtype=torch.float64, device=dev)
    bad = torch.zeros(1, dtype=torch.int32, device=dev)
    N.check(N.lib().nedmft_extrapolate_current(k, dts.ctypes.data_as(N.PD), tmins.ctypes.data_as(N.PD),
                                               nts.ctypes.data_as(N.PI), ptrs, _ptr(t_d), t_d.numel(), _ptr(out),
                                               _ptr(bad), ctypes.c_void_p(_stream(stream))))
    if int(bad.item()):
        raise NedmftError(N.NEDMFT_EINVAL, "extrapolate_current: an output time lies outside a run's grid")
    return out


def g0_build(grid: Grid, model: N.Model, eps, ebar, device="cuda", stream=None) -> torch.Tensor:
    eps_t = _dev(eps, torch.float64, device)
    ebar_t = _dev(ebar, torch.float64, device)
    nq = eps_t.numel()
    out = torch.empty((nq, grid.n_c, grid.n_c), dtype=torch.complex128, device=eps_t.device)
    N.check(N.lib().nedmft_g0_build(ctypes.byref(grid.contour), ctypes.byref(model), _ptr(eps_t), _ptr(ebar_t), nq,
                                    _ptr(out), ctypes.c_void_p(_stream(stream))))
    return out


def lattice_workspace_size(grid: Grid, nq: int, precision="fp64", batch: int = 0) -> int:
    n = N.lib().nedmft_lattice_workspace_size(ctypes.byref(grid.contour), nq, _prec(precision), batch)
    if n == 0:
        raise NedmftError(N.NEDMFT_EINVAL, "lattice_workspace_size: invalid arguments")
    return n


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def lattice_gloc(grid: Grid, model: N.Model, sigma, eps, ebar, wq, precision="fp64", current=True,
                 ws: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None):
    """G_loc (complex128, n_c x n_c) and, if ``current``, j(t) and its imaginary diagnostic."""
    dev = sigma.device if isinstance(sigma, torch.Tensor) else torch.device("cuda")
    sigma_t = _dev(sigma, torch.complex128, dev)
    eps_t, ebar_t, wq_t = (_dev(a, torch.float64, dev) for a in (eps, ebar, wq))
    nq = eps_t.numel()
    p = _prec(precision)
    need = lattice_workspace_size(grid, nq, p)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    gloc = out if out is not None else torch.empty((grid.n_c, grid.n_c), dtype=torch.complex128, device=dev)
    j = torch.empty(grid.n_t, dtype=torch.float64, device=dev) if current else None
    ji = torch.empty(grid.n_t, dtype=torch.float64, device=dev) if current else None
    N.check(N.lib().nedmft_lattice_gloc(ctypes.byref(grid.contour), ctypes.byref(model), _ptr(sigma_t), _ptr(eps_t),
                                        _ptr(ebar_t), _ptr(wq_t), nq, p, _ptr(gloc), _ptr(j), _ptr(ji), _ptr(ws),
                                        ws.numel(), ctypes.c_void_p(_stream(stream))))
    return gloc, j, ji


def current(grid: Grid, model: N.Model, sigma, eps, ebar, wq, precision="fp64", ws=None, stream=None):
    dev = sigma.device
    eps_t, ebar_t, wq_t = (_dev(a, torch.float64, dev) for a in (eps, ebar, wq))
    nq = eps_t.numel()
    p = _prec(precision)
    need = lattice_workspace_size(grid, nq, p)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    j = torch.empty(grid.n_t, dtype=torch.float64, device=dev)
    ji = torch.empty(grid.n_t, dtype=torch.float64, device=dev)
    N.check(N.lib().nedmft_current(ctypes.byref(grid.contour), ctypes.byref(model), _ptr(sigma), _ptr(eps_t),
                                   _ptr(ebar_t), _ptr(wq_t), nq, p, _ptr(j), _ptr(ji), _ptr(ws), ws.numel(),
                                   ctypes.c_void_p(_stream(stream))))
    return j, ji


def lattice_autotune(grid: Grid, model: N.Model, sigma, eps, ebar, wq, precision="mixed_bf16", candidates=None,
                     stream=None):
    """Times one lattice step per candidate batch size and makes the fastest the
    default for (n_c, nq, precision) in this process; returns (batch, ms)."""
    dev = sigma.device if isinstance(sigma, torch.Tensor) else torch.device("cuda")
    sigma_t = _dev(sigma, torch.complex128, dev)
    eps_t, ebar_t, wq_t = (_dev(a, torch.float64, dev) for a in (eps, ebar, wq))
    nq = eps_t.numel()
    p = _prec(precision)
    if candidates is None:
        candidates = [76, 114, 152, 228, 304]
    cand = (N.c_int32 * len(candidates))(*candidates)
    need = max(N.lib().nedmft_lattice_workspace_size(ctypes.byref(grid.contour), nq, p, int(b)) for b in candidates)
    if need == 0:
        raise NedmftError(N.NEDMFT_EINVAL, "lattice_workspace_size: invalid arguments")
    ws = workspace(need, dev)
    best = N.c_int32(0)
    ms = N.c_double(0.0)
    N.check(N.lib().nedmft_lattice_autotune(ctypes.byref(grid.contour), ctypes.byref(model), _ptr(sigma_t),
                                            _ptr(eps_t), _ptr(ebar_t), _ptr(wq_t), nq, p, cand, len(candidates),
                                            ctypes.byref(best), ctypes.byref(ms), _ptr(ws), ws.numel(),
                                            ctypes.c_void_p(_stream(stream))))
    return best.value, ms.value


def lattice_batch(grid: Grid, nq: int, precision="mixed_bf16") -> int:
    return int(N.lib().nedmft_lattice_batch(ctypes.byref(grid.contour), nq, _prec(precision)))


def lattice_set_tuning(grid: Grid, nq: int, precision="mixed_bf16", batch: int = 0, width: int = 0) -> None:
    N.check(N.lib().nedmft_lattice_set_tuning(ctypes.byref(grid.contour), nq, _prec(precision), batch, width))


def lattice_block_width(grid: Grid, nq: int, precision="mixed_bf16") -> int:
    return int(N.lib().nedmft_lattice_block_width(ctypes.byref(grid.contour), nq, _prec(precision)))


def moments(grid: Grid, gloc: torch.Tensor, stream=None):
    """(mu0, mu1, mu2, n) on the upper-branch times: the equal-time moments of G^R and the density."""
    dev = gloc.device
    out = [torch.empty(grid.n_t, dtype=torch.float64, device=dev) for _ in range(4)]
    N.check(N.lib().nedmft_moments(ctypes.byref(grid.contour), _ptr(gloc), *[_ptr(o) for o in out],
                                   ctypes.c_void_p(_stream(stream))))
    return tuple(out)


def dos(grid: Grid, gloc: torch.Tensor, m_index, omega, stream=None) -> torch.Tensor:
    """rho(t_m, omega), one row per average-time index m."""
    dev = gloc.device
    m_t = torch.as_tensor(np.asarray(m_index, dtype=np.int32), device=dev)
    om = _dev(omega, torch.float64, dev)
    rho = torch.empty((m_t.numel(), om.numel()), dtype=torch.float64, device=dev)
    N.check(N.lib().nedmft_dos(ctypes.byref(grid.contour), _ptr(gloc), _ptr(m_t), m_t.numel(), _ptr(om), om.numel(),
                               _ptr(rho), ctypes.c_void_p(_stream(stream))))
    return rho


def impurity_update(grid: Grid, model: N.Model, gloc: torch.Tensor, sigma: torch.Tensor, want_gimp=False,
                    ws=None, stream=None):
    dev = gloc.device
    need = N.lib().nedmft_impurity_workspace_size(ctypes.byref(grid.contour))
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    sigma_new = torch.empty_like(sigma)
    gimp = torch.empty_like(gloc) if want_gimp else None
    N.check(N.lib().nedmft_impurity_update(ctypes.byref(grid.contour), ctypes.byref(model), _ptr(gloc), _ptr(sigma),
                                           _ptr(sigma_new), _ptr(gimp), _ptr(ws), ws.numel(),
                                           ctypes.c_void_p(_stream(stream))))
    return sigma_new, gimp


@dataclass
class DmftSolution:
    sigma: torch.Tensor
    gloc: torch.Tensor
    current: torch.Tensor
    iterations: int
    error: float
    converged: bool


def dmft_solve(grid: Grid, model: N.Model, n_quad: int, precision="fp64", sigma_init=None, tol=1e-8,
               max_iter=50, device="cuda", stream=None) -> DmftSolution:
    p = _prec(precision)
    need = N.lib().nedmft_dmft_workspace_size(ctypes.byref(grid.contour), n_quad, p)
    if need == 0:
        raise NedmftError(N.NEDMFT_EINVAL, "dmft_workspace_size: invalid arguments")
    ws = workspace(need, device)
    n = grid.n_c
    sigma = torch.empty((n, n), dtype=torch.complex128, device=device)
    gloc = torch.empty((n, n), dtype=torch.complex128, device=device)
    j = torch.empty(grid.n_t, dtype=torch.float64, device=device)
    it = N.c_int32(0)
    err = N.c_double(0.0)
    rc = N.lib().nedmft_dmft_solve(ctypes.byref(grid.contour), ctypes.byref(model), n_quad, p, _ptr(sigma_init),
                                   tol, max_iter, _ptr(sigma), _ptr(gloc), _ptr(j), ctypes.byref(it),
                                   ctypes.byref(err), _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(stream)))
    N.check(rc, allow_warning=True)
    return DmftSolution(sigma, gloc, j, it.value, err.value, rc == N.NEDMFT_OK)


def dmft_solve_batch(grids, models, n_quad: int, precision="fp64", sigma_init=None, tol=1e-8, max_iter=50,
                     device="cuda", stream=None):
    """Several DMFT runs swept together (nedmft_dmft_solve_batch); one DmftSolution per run."""
    n = len(grids)
    assert len(models) == n and n >= 1
    p = _prec(precision)
    cs = (N.Contour * n)(*[g.contour for g in grids])
    ms = (N.Model * n)(*models)
    need = N.lib().nedmft_dmft_batch_workspace_size(n, cs, n_quad, p)
    if need == 0:
        raise NedmftError(N.NEDMFT_EINVAL, "dmft_batch_workspace_size: invalid arguments")
    ws = workspace(need, device)
    sig = [torch.empty((g.n_c, g.n_c), dtype=torch.complex128, device=device) for g in grids]
    gl = [torch.empty((g.n_c, g.n_c), dtype=torch.complex128, device=device) for g in grids]
    js = [torch.empty(g.n_t, dtype=torch.float64, device=device) for g in grids]
    ptrs = lambda ts: (ctypes.c_void_p * n)(*[None if t is None else t.data_ptr() for t in ts])
    init = None if sigma_init is None else ptrs(sigma_init)
    it = (N.c_int32 * n)()
    err = (N.c_double * n)()
    conv = (N.c_int32 * n)()
    rc = N.lib().nedmft_dmft_solve_batch(n, cs, ms, n_quad, p, init, tol, max_iter, ptrs(sig), ptrs(gl), ptrs(js), it,
                                         err, conv, _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(stream)))
    N.check(rc, allow_warning=True)
    return [DmftSolution(sig[r], gl[r], js[r], it[r], err[r], bool(conv[r])) for r in range(n)]
