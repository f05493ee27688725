"""Pins of the CPU oracle against what the paper and the mathematics fix.

No test here reads the oracle's own formula back: each compares it with an
independent fact (a closed form derived by hand, a library routine, numerical
integration, an identity of the method, or brute force on tiny inputs).
"""

import math

import numpy as np
import pytest
from scipy import integrate

from oracle import nedmft_oracle as O
from paper_0711_0999_gb300.synth import workload_sigma

# ---------------------------------------------------------------- grid / weights


@pytest.mark.parametrize("args,n_t,n_tau", [
    ((-2, 4, 0.2, 10, 0.5), 30, 20),          # N_c = 80
    ((-5, 30, 0.05, 10, 0.1), 700, 100),      # N_c = 1500
    ((-5, 25, 0.1, 10, 0.1), 300, 100),       # N_c = 700
    ((-5, 25, 1 / 15, 10, 0.1), 450, 100),    # N_c = 1000
    ((-5, 25, 0.05, 10, 0.1), 600, 100),      # N_c = 1300
    ((-5, 50, 1 / 30, 10, 0.1), 1650, 100),   # N_c = 3400
    ((-5, 10, 0.1, 10, 0.1), 150, 100),       # N_c = 400
])
def test_grid_counts_and_weights(args, n_t, n_tau):
    c = O.contour_grid(*args)
    t_min, t_max, dt, beta, dtau = args
    assert (c.n_t, c.n_tau) == (n_t, n_tau)
    assert c.t.shape == (2 * n_t + n_tau,)
    # leftpoint rule integrates constants exactly: forward and back cancel,
    # the imaginary branch has length -i beta (Eq. integration_rule)
    assert abs(c.w[: 2 * n_t].sum()) < 1e-12
    assert abs(c.w[2 * n_t:].sum() - (-1j * beta)) < 1e-12
    # end points stated in Sec. II
    assert abs(c.t[0] - t_min) < 1e-12 and abs(c.t[n_t - 1] - (t_max - dt)) < 1e-12
    assert abs(c.t[n_t] - t_max) < 1e-12 and abs(c.t[2 * n_t - 1] - (t_min + dt)) < 1e-12
    assert abs(c.t[2 * n_t] - t_min) < 1e-12
    assert abs(c.t[-1] - (t_min - 1j * (beta - dtau))) < 1e-12
    # leftpoint: W_j is the step from t_j to the next contour point
    nxt = np.append(c.t[1:], t_min - 1j * beta)
    assert np.allclose(nxt - c.t, c.w, atol=1e-12)


def test_grid_rejects_non_integer_counts():
    with pytest.raises(ValueError):
        O.contour_grid(-2, 4, 0.25001, 10, 0.5)
    with pytest.raises(ValueError):
        O.contour_grid(-2, 4, 0.2, 10, 0.3)


# ---------------------------------------------------------------- Gauss-Hermite


@pytest.mark.parametrize("n", [1, 2, 5, 16, 40, 53, 64])
def test_gauss_hermite_matches_library_and_moments(n):
    x, w = O.gauss_hermite(n)
    xr, wr = np.polynomial.hermite.hermgauss(n)
    assert np.allclose(x, xr, atol=1e-12, rtol=0)
    assert np.allclose(w, wr / math.sqrt(math.pi), atol=1e-14, rtol=1e-10)
    # exact for polynomials up to degree 2n-1: E[x^(2k)] = (2k-1)!!/2^k
    # (checked up to degree 25, beyond which rounding of x^k dominates)
    for k in range(0, min(n, 13)):
        exact = math.prod(range(1, 2 * k, 2)) / 2.0 ** k
        got = float(np.sum(w * x ** (2 * k)))
        assert abs(got - exact) <= 1e-9 * max(1.0, exact)
        odd = w * x ** (2 * k + 1)
        assert abs(float(np.sum(odd))) < 1e-9 * max(1.0, float(np.sum(np.abs(odd))))


def test_quadrature_product_order_and_weights():
    eps, ebar, wq = O.quadrature_points(5)
    x, w = O.gauss_hermite(5)
    assert abs(wq.sum() - 1.0) < 1e-14
    assert eps[7] == x[1] and ebar[7] == x[2] and wq[7] == w[1] * w[2]


# ---------------------------------------------------------------- M and det M


@pytest.mark.parametrize("mu", [0.3, -0.7, 1.1])
def test_det_m_closed_form(mu):
    # cofactor expansion along the first row of the bidiagonal+corner M:
    # det M = 1 + (1 + dt^2 mu^2)^N_t (1 + dtau mu)^N_tau
    c = O.contour_grid(-2, 4, 0.2, 10, 0.5)
    m = O.m_matrix(c, mu)
    exact = 1 + (1 + c.dt ** 2 * mu ** 2) ** c.n_t * (1 + c.dtau * mu) ** c.n_tau
    assert abs(np.linalg.det(m) - exact) < 1e-10 * abs(exact)


def test_det_m_limit_is_partition_function():
    mu = 0.4
    vals = []
    for dt, dtau in [(0.1, 0.1), (0.05, 0.05), (0.025, 0.025)]:
        c = O.contour_grid(-1, 1, dt, 2.0, dtau)
        vals.append(abs(np.linalg.det(O.m_matrix(c, mu)) - (1 + math.exp(2.0 * mu))))
    assert vals[0] > vals[1] > vals[2] and vals[2] < 0.02


def test_free_electron_diagonal_is_inverse_det():
    c = O.contour_grid(-1, 1, 0.1, 2.0, 0.25)
    mu = 0.35
    m = O.m_matrix(c, mu)
    g = -1j * np.linalg.inv(m)
    assert np.allclose(np.diag(g), -1j / np.linalg.det(m), atol=1e-13)


# ---------------------------------------------------------------- G0


def _band_integral(s, eps, ebar, E):
    """F(s) by numerical quadrature of the integrand of Eq. g_contour_non_final2."""
    if s.imag != 0 or s.real <= 0:
        return eps * s
    f = lambda tb: math.cos(E * tb) * eps - math.sin(E * tb) * ebar
    val, _ = integrate.quad(f, 0.0, s.real, epsabs=1e-13, epsrel=1e-13, limit=200)
    return val


@pytest.mark.parametrize("eps,ebar", [(1.3, 0.4), (-2.0, -0.7), (0.1, 1.9)])
def test_g0_inverse_is_bidiagonal_with_closed_form(eps, ebar):
    # inv(G0) = i (I - Z) phi-conjugated: diagonal i, subdiagonal -i phi_j/phi_{j-1},
    # boundary element i e^{-x dtau} (Sherman-Morrison on the theta structure).
    c = O.contour_grid(-2, 3, 0.2, 4.0, 0.5)
    model = O.Model(U=0.6, E=1.3)
    mu = model.chem
    x = eps - mu
    g0 = O.g0_matrix(c, model, eps, ebar)
    b = np.linalg.inv(g0)
    phi = np.array([np.exp(1j * mu * s - 1j * _band_integral(s, eps, ebar, model.E)) for s in c.t])
    n = c.n_c
    ref = 1j * np.eye(n, dtype=complex)
    for j in range(1, n):
        ref[j, j - 1] = -1j * phi[j] / phi[j - 1]
    ref[0, n - 1] = 1j * math.exp(-x * c.dtau)
    assert np.abs(b - ref).max() < 1e-11


def test_g0_elementwise_matches_matrix():
    c = O.contour_grid(-1, 1, 0.25, 2.0, 0.5)
    model = O.Model(U=1.0, E=2.0)
    g = O.g0_matrix(c, model, 0.7, -0.3)
    for i in range(c.n_c):
        for j in range(c.n_c):
            assert abs(g[i, j] - O.g0_element(c.t[i], c.t[j], i >= j, 0.7, -0.3, model, c.beta)) < 1e-14


@pytest.mark.parametrize("eps,ebar", [(0.8, -1.1), (-1.5, 0.3)])
def test_g0_keldysh_antiperiodic_and_density(eps, ebar):
    c = O.contour_grid(-2, 3, 0.25, 5.0, 0.5)
    model = O.Model(U=1.0, E=1.0)
    g = O.g0_matrix(c, model, eps, ebar)
    nt = c.n_t
    up = lambda m: m                       # upper index of time t_min + m dt
    lo = lambda m: 2 * nt - m if m > 0 else 2 * nt  # lower (or first imaginary) partner
    x = eps - model.chem
    f = 1.0 / (1.0 + math.exp(c.beta * x))
    for m in range(nt):
        for k in range(nt):
            # G^<(t, t')^* = -G^<(t', t)
            assert abs(np.conj(g[up(m), lo(k)]) + g[up(k), lo(m)]) < 1e-13
        # equal-time lesser: -i G^<(t, t) = f(eps - mu)
        assert abs(-1j * g[up(m), lo(m)] - f) < 1e-13
    # boundary condition: G(t_min, t') = -G(t_min - i beta, t') (Sec. II)
    # for every t' after t_min (t_min is the earliest point, t_min - i beta the latest)
    tb = c.t_min - 1j * c.beta
    for j in range(1, c.n_c):
        a = O.g0_element(c.t_min + 0j, c.t[j], False, eps, ebar, model, c.beta)
        b = O.g0_element(tb, c.t[j], True, eps, ebar, model, c.beta)
        assert abs(a + b) < 1e-13


# ---------------------------------------------------------------- lattice step


def test_dyson_solve_residual_and_inverse_form():
    c = O.contour_grid(-2, 2, 0.2, 4.0, 0.5)
    model = O.Model(U=1.0, E=1.0)
    sigma = workload_sigma(c.t, c.w, model.U, seed=3)
    s = O.weighted_sigma(c, sigma)
    for eps, ebar in [(1.2, 0.3), (-1.7, -0.5)]:
        g0 = O.g0_matrix(c, model, eps, ebar)
        gq = O.dyson_solve(g0, s)
        # Eq. dyson discretised: G = G0 + G0 W Sigma W G
        assert np.abs(gq - g0 - g0 @ s @ gq).max() < 1e-12 * np.abs(g0).max() * c.n_c
        # exact equivalent form G = (G0^-1 - S)^-1
        assert np.abs(gq - np.linalg.inv(np.linalg.inv(g0) - s)).max() < 1e-11


def test_u0_current_and_density_closed_form():
    # Sigma = 0: G^<_q(t,t) = i f(eps), so j(t) = -sin(Et) sum_a w_a x_a f(x_a)
    # for t > 0 and 0 for t <= 0 (symmetric nodes), n(t) = 1/2 at mu = 0.
    c = O.contour_grid(-2, 4, 0.2, 10, 0.5)
    model = O.Model(U=0.0, E=1.0)
    eps, ebar, wq = O.quadrature_points(12)
    gloc, jc = O.lattice_gloc(c, model, np.zeros((c.n_c, c.n_c), complex), eps, ebar, wq)
    x, w = O.gauss_hermite(12)
    fermi = 1.0 / (1.0 + np.exp(c.beta * x))
    amp = float(np.sum(w * x * fermi))
    tm = c.t[: c.n_t].real
    expect = np.where(tm > 0, -np.sin(model.E * tm) * amp, 0.0)
    assert np.abs(jc.real - expect).max() < 1e-14
    assert np.abs(jc.imag).max() < 1e-14
    assert np.abs(O.density(c, gloc) - 0.5).max() < 1e-14


def test_u0_retarded_closed_form():
    # G^R_loc(t,t') = -i theta(t-t') e^{i mu (t-t')} exp(-[(da)^2 + (db)^2]/4) with
    # F = eps a(t) + ebar b(t): the Gaussian characteristic function of Eq. joint_dos.
    c = O.contour_grid(-2, 6, 0.25, 2.0, 0.5)
    model = O.Model(U=0.0, E=1.0)
    eps, ebar, wq = O.quadrature_points(40)
    gloc, _ = O.lattice_gloc(c, model, np.zeros((c.n_c, c.n_c), complex), eps, ebar, wq)
    nt = c.n_t
    E = model.E

    def ab(s):
        return (s, 0.0) if s <= 0 else (math.sin(E * s) / E, (math.cos(E * s) - 1) / E)

    worst = 0.0
    for i in range(nt):
        for j in range(i):
            ti, tj = c.t[i].real, c.t[j].real
            lo_j = 2 * nt - j if j > 0 else 2 * nt
            gr = gloc[i, j] - gloc[i, lo_j]  # G^t - G^< on the upper branch, t > t'
            (a1, b1), (a2, b2) = ab(ti), ab(tj)
            ref = -1j * math.exp(-((a1 - a2) ** 2 + (b1 - b2) ** 2) / 4)
            worst = max(worst, abs(gr - ref))
    assert worst < 1e-10


def test_e0_no_current_and_ebar_independent():
    c = O.contour_grid(-2, 2, 0.2, 4.0, 0.5)
    model = O.Model(U=1.0, E=0.0)
    sigma = workload_sigma(c.t, c.w, model.U, seed=5)
    eps, ebar, wq = O.quadrature_points(8)
    gloc, jc = O.lattice_gloc(c, model, sigma, eps, ebar, wq)
    # ebar drops out of G0 at E = 0, so the 2-D sum equals the 1-D eps sum
    x, w = O.gauss_hermite(8)
    g1, _ = O.lattice_gloc(c, model, sigma, x, np.full(8, 9.9), w)
    assert np.abs(gloc - g1).max() < 1e-12
    # by ebar -> -ebar symmetry of the nodes the current vanishes
    assert np.abs(jc).max() < 1e-13


def test_quadrature_brute_force_convergence():
    c = O.contour_grid(-1, 2, 0.25, 2.0, 0.5)
    model = O.Model(U=0.8, E=1.0)
    sigma = workload_sigma(c.t, c.w, model.U, seed=7)
    res = {}
    for n in (6, 7, 12, 13, 24, 25, 48):
        e, eb, w = O.quadrature_points(n)
        res[n], _ = O.lattice_gloc(c, model, sigma, e, eb, w)
    d = lambda a, b: np.abs(res[a] - res[b]).max()
    # successive N/N+1 differences shrink, and the 24-point grid agrees with 48
    assert d(6, 7) > d(12, 13) > d(24, 25)
    assert d(24, 48) < 1e-6


# ---------------------------------------------------------------- impurity / loop


def test_impurity_limits():
    c = O.contour_grid(-1, 1, 0.25, 2.0, 0.5)
    nt = c.n_t
    gl = O.lattice_gloc(c, O.Model(U=1.0, E=1.0), np.zeros((c.n_c, c.n_c), complex),
                        *O.quadrature_points(6))[0]
    sigma = workload_sigma(c.t, c.w, 1.0, seed=11)
    # U = 0: no scattering, Sigma_new = 0 whatever Sigma was
    s0, _ = O.impurity_update(c, O.Model(U=0.0, E=1.0), gl, sigma)
    assert np.abs(s0).max() < 1e-9
    # <w_1> = 0: no localized electrons, Sigma_new = 0
    s1, _ = O.impurity_update(c, O.Model(U=1.0, E=1.0, w1=0.0, mu=0.5), gl, sigma)
    assert np.abs(s1).max() < 1e-9
    # <w_1> = 1: Sigma_new = U delta_c, the point-split contour delta function
    # (delta_c(t_j, t_{j-1}) = 1/W_{j-1}, boundary element -1/W_{N_c}; Eqs. delta_cont_defa/b)
    U = 0.7
    s2, _ = O.impurity_update(c, O.Model(U=U, E=1.0, w1=1.0, mu=0.35), gl, sigma)
    n = c.n_c
    ref = np.zeros((n, n), complex)
    for j in range(1, n):
        ref[j, j - 1] = U / c.w[j - 1]
    ref[0, n - 1] = -U / c.w[n - 1]
    assert np.abs(s2 - ref).max() < 1e-8 * np.abs(ref).max()
    del nt


def test_dmft_small_converges_to_fixed_point():
    c = O.contour_grid(-1, 2, 0.25, 4.0, 0.5)
    model = O.Model(U=0.8, E=1.0)
    res = O.dmft_solve(c, model, n_quad=8, tol=1e-10, max_iter=60)
    assert res.converged and res.iterations < 60
    s_new, gimp = O.impurity_update(c, model, res.gloc, res.sigma)
    # at self-consistency the impurity reproduces the lattice
    assert np.abs(gimp - res.gloc).max() < 1e-8
    assert np.abs(O.weighted_sigma(c, s_new - res.sigma)).max() < 1e-8
    # U = 0 converges in one step (Sigma stays 0)
    r0 = O.dmft_solve(c, O.Model(U=0.0, E=1.0), n_quad=8, tol=1e-12, max_iter=5)
    assert r0.converged and r0.iterations == 2 and np.abs(r0.sigma).max() < 1e-12


def test_interacting_invariants_improve_with_dt():
    # n(t) = 1/2 and j(t < 0) = 0 hold only as dt -> 0 for U > 0: check they
    # improve monotonically with dt (first order) on a tiny contour.
    model = O.Model(U=1.0, E=1.0)
    errs_n, errs_j = [], []
    for dt in (0.4, 0.2, 0.1):
        c = O.contour_grid(-1.2, 1.2, dt, 2.0, dt)
        r = O.dmft_solve(c, model, n_quad=6, tol=1e-9, max_iter=80)
        assert r.converged
        tm = c.t[: c.n_t].real
        errs_n.append(np.abs(O.density(c, r.gloc).real - 0.5).max())
        errs_j.append(np.abs(r.current.real[tm < 0]).max())
    assert errs_n[0] > errs_n[1] > errs_n[2]
    assert errs_j[0] > errs_j[1] > errs_j[2]


def test_lagrange_extrapolation_exact_for_polynomials():
    dts = [0.1, 1 / 15, 0.05]
    f = lambda d: 0.3 - 1.7 * d + 4.2 * d * d
    vals = np.array([[f(d), 2 * f(d)] for d in dts])
    out = O.lagrange_extrapolate(dts, vals)
    assert np.allclose(out, [0.3, 0.6], atol=1e-13)
    dts4 = [0.1, 0.08, 0.05, 0.04]
    g = lambda d: 1.0 + d - 3 * d ** 2 + 11 * d ** 3
    assert abs(O.lagrange_extrapolate(dts4, np.array([g(d) for d in dts4])) - 1.0) < 1e-12
