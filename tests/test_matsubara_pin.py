"""The oracle's interacting DMFT chain against an independent equilibrium solution.

Before the field acts, the contour solution is the equilibrium Falicov-Kimball
state, so the imaginary-imaginary block of G_loc is i G_M(tau - tau'), G_M the
Matsubara Green's function of the same model (Sec. II: the contour starts at
t_min with the thermal branch; Eqs. effective_medium, dynamical_mean_field,
g_imp_solve for the DMFT equations, Eq. joint_dos for the Gaussian density of
states).  Here G_M comes from a Matsubara-axis DMFT that shares no code with
the oracle: the lattice sum is the Hilbert transform of the Gaussian density
of states, -i sqrt(pi) w(z) with w the Faddeeva function, the impurity
solution is the Falicov-Kimball one, G_imp = (1 - w1)/a + w1/(a - U) with a the
inverse effective medium, and G_M(tau) is the Fourier sum with the 1/(i omega)
tail taken out in closed form.

The discrete contour (Eq. time_discrete, left-point weights) is first order in
its steps, so the pins are: the error halves when dt = dtau halves, and the
Richardson combination of the two grids is much closer than either.  A
dropped term, a wrong sign or a wrong chemical potential in the oracle's
lattice or impurity step would leave an O(1) difference instead.

The same first-order structure shows in the field dependence: in the exact
theory the thermal block does not depend on E (causality), on the discrete
contour it does at O(dt E^2), and that difference halves with dt.  Likewise
the Keldysh symmetry G^<(t, t')^* = -G^<(t', t) of the interacting G_loc, and
its time-translation invariance at E = 0, hold to first order in the step.
"""

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import wofz

from oracle import nedmft_oracle as O

BETA, U = 2.0, 1.0


def matsubara_fk(U, beta, w1=0.5, n_freq=20000):
    """Equilibrium Falicov-Kimball DMFT on the positive Matsubara frequencies
    (half filling: mu = U / 2).  Returns omega_n and G(i omega_n)."""
    mu = U / 2
    w = (2 * np.arange(n_freq) + 1) * np.pi / beta
    sig = np.zeros(n_freq, complex)
    for _ in range(2000):
        g = -1j * np.sqrt(np.pi) * wofz(1j * w + mu - sig)  # Hilbert transform of exp(-e^2)/sqrt(pi)
        a = 1 / g + sig                                    # inverse effective medium
        gimp = (1 - w1) / a + w1 / (a - U)                 # f site empty / occupied
        new = a - 1 / gimp
        done = np.abs(new - sig).max() < 1e-10             # rounding floor ~1e-11 at the largest omega
        sig = new
        if done:
            break
    else:
        raise AssertionError("Matsubara iteration did not converge")
    return w, -1j * np.sqrt(np.pi) * wofz(1j * w + mu - sig)


def g_tau(w, g, beta, tau):
    """G_M(tau) for 0 <= tau < beta (tau = 0 read as 0+): the 1/(i omega) part
    sums to -1/2, the rest by the symmetric sum over +-omega_n."""
    r = g - 1 / (1j * w)
    tau = np.asarray(tau, float)
    return -0.5 + (2 / beta) * (np.exp(-1j * np.multiply.outer(tau, w)) * r).real.sum(axis=-1)


def thermal_block_reference(w, g, beta, n_tau, dtau):
    """i G_M(tau_i - tau_j) on the thermal points, with G_M antiperiodic."""
    tau = dtau * np.arange(n_tau)
    d = tau[:, None] - tau[None, :]
    gm = g_tau(w, g, beta, np.mod(d, beta))
    return 1j * np.where(d >= 0, gm, -gm)


def thermal_block(c, gloc):
    k = 2 * c.n_t
    return gloc[k:, k:]


def test_matsubara_reference_is_the_free_gaussian_band_at_u0():
    # pins the Fourier sum and the Hilbert transform: at U = 0 G_M(tau) is the
    # Gaussian-band average of -(1 - f(e)) exp(-e tau), by direct integration
    w, g = matsubara_fk(0.0, BETA)
    for tau in (0.0, 0.3, 1.0, 1.9):
        ref = quad(lambda e: -np.exp(-e * e) / np.sqrt(np.pi) * np.exp(-e * tau) / (1 + np.exp(-BETA * e)),
                   -12, 12, epsabs=1e-14)[0]
        assert abs(g_tau(w, g, BETA, tau) - ref) < 1e-12


def test_thermal_block_converges_to_the_matsubara_solution_at_first_order():
    w, g = matsubara_fk(U, BETA)
    blocks = {}
    for d in (0.1, 0.05):
        c = O.contour_grid(-0.4, 0.4, d, BETA, d)
        r = O.dmft_solve(c, O.Model(U=U, E=0.0), n_quad=12, tol=1e-11, max_iter=80)
        assert r.converged
        blocks[d] = thermal_block(c, r.gloc)
    ref = thermal_block_reference(w, g, BETA, round(BETA / 0.1), 0.1)  # the points common to both grids
    coarse, fine = blocks[0.1], blocks[0.05][::2, ::2]
    e_coarse = np.abs(coarse - ref).max()
    e_fine = np.abs(fine - ref).max()
    e_rich = np.abs(2 * fine - coarse - ref).max()
    assert e_coarse < 0.02 and e_fine < 0.01
    assert 0.4 < e_fine / e_coarse < 0.6            # first order in the step
    assert e_rich < 0.25 * e_fine                   # and the first-order term is the error
    # the equal-time value is G_M(0+) = -(1 - n) = -1/2 at half filling
    assert np.abs(np.diag(ref) + 0.5j).max() < 1e-12


def test_field_dependence_of_the_thermal_block_is_first_order_in_dt():
    diffs = []
    for dt in (0.1, 0.05, 0.025):
        c = O.contour_grid(-0.4, 0.8, dt, BETA, 0.1)
        r0 = O.dmft_solve(c, O.Model(U=U, E=0.0), n_quad=8, tol=1e-12, max_iter=80)
        r1 = O.dmft_solve(c, O.Model(U=U, E=1.0), n_quad=8, tol=1e-12, max_iter=80)
        assert r0.converged and r1.converged
        diffs.append(np.abs(thermal_block(c, r0.gloc) - thermal_block(c, r1.gloc)).max())
    assert diffs[2] < 5e-4
    for a, b in zip(diffs, diffs[1:]):
        assert 0.4 < b / a < 0.7


@pytest.mark.parametrize("E", [0.0, 1.0])
def test_keldysh_symmetry_and_time_translation_are_first_order(E):
    # the interacting G_loc keeps G^<(t, t')^* = -G^<(t', t) (and, at E = 0,
    # depends on t - t' only) in the continuum; on the discrete contour both
    # hold to first order in dt = dtau, so the violation halves with the step
    sym, tti = [], []
    for d in (0.2, 0.1, 0.05):
        c = O.contour_grid(-1.0, 1.0, d, BETA, d)
        r = O.dmft_solve(c, O.Model(U=U, E=E), n_quad=8, tol=1e-11, max_iter=80)
        assert r.converged
        g, nt = r.gloc, c.n_t
        lo = lambda m: 2 * nt - m if m > 0 else 2 * nt  # the lower-branch (or first thermal) partner of t_m
        sym.append(max(abs(np.conj(g[m, lo(k)]) + g[k, lo(m)]) for m in range(nt) for k in range(nt)))
        tti.append(max(abs(g[m, lo(k)] - g[m - 1, lo(k - 1)]) for m in range(1, nt) for k in range(1, nt)))
    for a, b in zip(sym, sym[1:]):
        assert 0.35 < b / a < 0.6
    assert sym[-1] < 0.05
    if E == 0.0:
        for a, b in zip(tti, tti[1:]):
            assert 0.3 < b / a < 0.6
        assert tti[-1] < 0.02
