"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every symbol of include/nedmft.h, and its host-only grid functions
agree with the oracle and with numpy."""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import nedmft_oracle as O
from paper_0711_0999_gb300 import _native as N
from paper_0711_0999_gb300 import api
from paper_0711_0999_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build_library()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "nedmft.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nedmft_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(N.LIB_PATH)
    syms = header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(N.SIGNATURES), "binding and header disagree"
    assert "sm_103a" in api.version()


@pytest.mark.parametrize("args", [(-2, 4, 0.2, 10, 0.5), (-5, 30, 0.05, 10, 0.1), (-5, 25, 1 / 15, 10, 0.1),
                                  (-5, 50, 1 / 30, 10, 0.1)])
def test_contour_grid_matches_oracle(args):
    g = api.contour_grid(*args)
    c = O.contour_grid(*args)
    assert (g.contour.n_t, g.contour.n_tau, g.n_c) == (c.n_t, c.n_tau, c.n_c)
    assert np.abs(g.t - c.t).max() < 1e-12
    assert np.abs(g.w - c.w).max() < 1e-15


def test_contour_grid_rejects_bad_input():
    with pytest.raises(N.NedmftError) as e:
        api.contour_grid(-2, 4, 0.25001, 10, 0.5)
    assert e.value.code == N.NEDMFT_EINVAL and "not a positive integer" in str(e.value)
    with pytest.raises(N.NedmftError):
        api.contour_grid(-2, 4, 0.2, 10, 0.0)


@pytest.mark.parametrize("n", [1, 2, 3, 16, 40, 53, 64, 101, 256])
def test_gauss_hermite_matches_oracle(n):
    x, w = api.gauss_hermite(n)
    xo, wo = O.gauss_hermite(n)
    assert np.abs(x - xo).max() < 1e-12
    assert np.abs(w - wo).max() < 1e-14 * max(1.0, n / 16)
    assert abs(w.sum() - 1.0) < 1e-13


def test_gauss_hermite_rejects_bad_n():
    for n in (0, -3, 513):
        with pytest.raises(N.NedmftError):
            api.gauss_hermite(n)


def test_quadrature_grid_order():
    e, b, w = api.quadrature_grid(7)
    eo, bo, wo = O.quadrature_points(7)
    assert np.abs(e - eo).max() < 1e-13 and np.abs(b - bo).max() < 1e-13 and np.abs(w - wo).max() < 1e-15


def test_workspace_sizes():
    g = api.contour_grid(-2, 4, 0.2, 10, 0.5)
    for p in (N.FP64, N.MIXED_BF16):
        assert api.lattice_workspace_size(g, 256, p) > 0
    big = api.contour_grid(-5, 30, 0.05, 10, 0.1)
    assert api.lattice_workspace_size(big, 2809, N.FP64) > api.lattice_workspace_size(g, 2809, N.FP64)
    assert N.lib().nedmft_lattice_workspace_size(ctypes.byref(g.contour), 0, 0, 0) == 0
    assert N.lib().nedmft_lattice_workspace_size(ctypes.byref(g.contour), 4, 7, 0) == 0
    assert N.lib().nedmft_lattice_workspace_size(ctypes.byref(g.contour), 4, 2, 0) == 0  # no third precision
    assert N.lib().nedmft_impurity_workspace_size(ctypes.byref(g.contour)) > 0
    assert N.lib().nedmft_dmft_workspace_size(ctypes.byref(g.contour), 16, N.FP64) > 0
    assert N.lib().nedmft_dmft_workspace_size(ctypes.byref(g.contour), 0, N.FP64) == 0


def test_status_strings():
    lib = N.lib()
    for code in (0, -1, -2, -3, -4, -5, 1):
        assert lib.nedmft_status_string(code)
    assert lib.nedmft_status_string(-99) == b"unknown status"


def test_quadrature_grid_avg_matches_oracle():
    e, b, w = api.quadrature_grid_avg(6)
    e6, b6, w6 = O.quadrature_points(6)
    e7, b7, w7 = O.quadrature_points(7)
    assert len(e) == 36 + 49
    assert np.abs(e - np.concatenate([e6, e7])).max() < 1e-13
    assert np.abs(b - np.concatenate([b6, b7])).max() < 1e-13
    assert np.abs(w - 0.5 * np.concatenate([w6, w7])).max() < 1e-15
    assert abs(w.sum() - 1.0) < 1e-14
    with pytest.raises(N.NedmftError):
        api.quadrature_grid_avg(0)
