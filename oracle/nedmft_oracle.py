"""Plain FP64 CPU oracle for the nonequilibrium-DMFT lattice step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product path (the
CUDA library and its Python binding) never imports, calls or links it, and this
module imports nothing from the product.

What it computes (J. K. Freericks, "Quenching Bloch oscillations in a strongly
correlated material", Sec. II):

* the discretised Kadanoff-Baym-Keldysh contour and its leftpoint quadrature
  weights (Eqs. time_discrete, integration_rule, integration_weights);
* Gauss-Hermite nodes/weights for the Gaussian joint density of states
  (Eq. joint_dos and the quadrature paragraph of Sec. II);
* the closed-form noninteracting contour Green's function in the diagonal field
  (Eq. g_contour_non_final2), sampled on the contour;
* the nonequilibrium Hilbert transform, literally
  ``G_loc = sum_q w_q [(I - G0_q S)^-1 G0_q]`` with ``S = W Sigma W``
  (Eqs. g_loc, dyson, matrix_multiply);
* the current (Eq. current_def), the Falicov-Kimball impurity update
  (Eqs. effective_medium, dynamical_mean_field, g_imp_solve, the M matrix of
  the discretised ``(i d/dt + mu) delta_c``, Eq. matrix_inverse_discrete), the
  plain-substitution DMFT loop, Lagrange extrapolation to dt -> 0, and the
  accuracy diagnostics (equal-time moments, Eqs. gr_omega and dos_def).

Everything is complex128 / float64.  Library primitives used as single steps:
``numpy.linalg.solve``, ``numpy.linalg.inv``, ``numpy.linalg.eigh``.

Readings of passages the paper leaves open (each one is listed in the design
notes of the repository as well):

R1  Eq. time_discrete prints the first branch as ``-t_min + (j-1) dt``; the
    stated range (t_min .. t_max - dt) fixes the sign: ``t_min + (j-1) dt``.
R2  The imaginary step is a parameter dtau (the paper fixes 0.1):
    ``t_j = t_min - i dtau (j - 2 N_t - 1)``, ``W_j = -i dtau``, ``N_tau = beta/dtau``.
R3  On the diagonal of the sampled G0 the contour theta function is 1
    (``theta_c(t_i, t_j) = 1`` for ``i >= j`` in contour order).
R4  Half filling: ``mu = U/2`` unless given, ``<w_1> = 1/2``.
R5  ``(i d + mu - U) delta_c`` is the same point-split M matrix with mu -> mu-U.
R6  Eq. dynamical_mean_field's second line carries ``+Sigma``; Eq.
    effective_medium gives ``G_0^-1 = G_loc^-1 + Sigma``, the only reading under
    which a converged Sigma is a fixed point.  The oracle follows
    Eq. effective_medium.
R7  Current: ``j(t) = Re[ i sum_q w_q ebar_q(t) G^<_q(t, t) ]`` with e = t* = 1
    and ``ebar_q(t) = ebar cos(Et) + eps sin(Et)`` for t > 0 (``ebar`` for t <= 0);
    the velocity replaced by ``-ebar`` as the text after Eq. current_def says.
R8  ``G^<(t_m, t_m)`` is the element (upper index m, lower index of the same
    time); for the first time t_min the lower-branch partner is the first
    imaginary point (the lower branch ends at t_min + dt).
R9  E = 0 uses the limit ``F(s) = eps s`` of the band phase.
R10 Convergence: ``max|G_new - G_old| / max|G_new| < tol``, plain substitution
    ``Sigma <- Sigma_new``, Sigma starting at 0.
R11 Equal-time moments (the moments paragraph after Eq. current_def): with
    ``G^R(t, t') = G^>(t, t') - G^<(t, t')`` on the real branches and
    ``f(s) = i G^R(T + s/2, T - s/2) = mu0 - i mu1 s - mu2 s^2 / 2 + O(s^3)``, the
    moments at T = t_m come from the quadratic through the relative times
    s = 2 k dt, k = 1, 2, 3 (pairs t_{m+k}, t_{m-k}); the paper's "first two
    derivatives at equal time".  Exact values at half filling: mu0 = 1,
    mu1 = 0, mu2 = 1/2 + U^2/4 (t* = 1).
R12 Density of states (Eqs. gr_omega, dos_def): the relative-time integral is
    the trapezoid rule over the symmetric pairs t_{m+k}, t_{m-k},
    k = 0 .. min(m, N_t - 1 - m), step 2 dt, no window.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# Contour discretisation (Sec. II, Eqs. time_discrete, integration_weights)
# --------------------------------------------------------------------------


@dataclass(frozen=True)
class Contour:
    t_min: float
    t_max: float
    dt: float
    beta: float
    dtau: float
    n_t: int
    n_tau: int
    t: np.ndarray  # complex contour times, upper -> lower -> imaginary
    w: np.ndarray  # complex leftpoint weights W_j

    @property
    def n_c(self) -> int:
        return 2 * self.n_t + self.n_tau


def _as_count(span: float, step: float, what: str) -> int:
    ratio = span / step
    n = int(round(ratio))
    if n < 1 or abs(ratio - n) > 1e-9 * max(1.0, abs(ratio)):
        raise ValueError(f"{what}: {span}/{step} is not a positive integer")
    return n


def contour_grid(t_min: float, t_max: float, dt: float, beta: float, dtau: float) -> Contour:
    """Contour points and weights, Sec. II Eqs. time_discrete and integration_weights.

    N_t points t_min .. t_max-dt on the upper branch (weight +dt), N_t points
    t_max .. t_min+dt on the lower branch (weight -dt), N_tau points
    t_min - i dtau k, k = 0..N_tau-1, on the imaginary branch (weight -i dtau).
    Readings R1, R2.
    """
    n_t = _as_count(t_max - t_min, dt, "(t_max - t_min)/dt")
    n_tau = _as_count(beta, dtau, "beta/dtau")
    t = np.empty(2 * n_t + n_tau, dtype=np.complex128)
    w = np.empty_like(t)
    for j in range(1, n_t + 1):  # upper branch, 1-based j as in the paper
        t[j - 1] = t_min + (j - 1) * dt
        w[j - 1] = dt
    for j in range(n_t + 1, 2 * n_t + 1):  # lower branch
        t[j - 1] = t_max - (j - n_t - 1) * dt
        w[j - 1] = -dt
    for j in range(2 * n_t + 1, 2 * n_t + n_tau + 1):  # imaginary branch
        t[j - 1] = t_min - 1j * dtau * (j - 2 * n_t - 1)
        w[j - 1] = -1j * dtau
    return Contour(t_min, t_max, dt, beta, dtau, n_t, n_tau, t, w)


# --------------------------------------------------------------------------
# Gauss-Hermite quadrature (Sec. II, quadrature paragraph; Eq. joint_dos)
# --------------------------------------------------------------------------


def gauss_hermite(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Nodes and weights for the weight exp(-x^2)/sqrt(pi) (weights sum to 1).

    Golub-Welsch: the nodes are the eigenvalues of the symmetric Jacobi matrix
    of the Hermite recurrence (off-diagonal sqrt(k/2)); each normalised weight
    is the squared first component of the corresponding eigenvector.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    k = np.arange(1, n, dtype=np.float64)
    jac = np.diag(np.sqrt(k / 2.0), 1) + np.diag(np.sqrt(k / 2.0), -1)
    x, v = np.linalg.eigh(jac)
    w = v[0, :] ** 2
    return x, w


def quadrature_points(n: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Product grid over (eps, ebar) with rho = exp(-eps^2 - ebar^2)/pi (Eq. joint_dos).

    Order: the eps index a is outer, the ebar index b inner; q = a*n + b.
    """
    x, w = gauss_hermite(n)
    eps = np.repeat(x, n)
    ebar = np.tile(x, n)
    wq = np.repeat(w, n) * np.tile(w, n)
    return eps, ebar, wq


# --------------------------------------------------------------------------
# Noninteracting contour Green's function (Eq. g_contour_non_final2)
# --------------------------------------------------------------------------


@dataclass(frozen=True)
class Model:
    U: float
    E: float
    w1: float = 0.5
    mu: float | None = None  # None -> U/2 (reading R4)

    @property
    def chem(self) -> float:
        return self.U / 2.0 if self.mu is None else self.mu


def band_phase(s: complex, eps: float, ebar: float, E: float) -> complex:
    """F(s) = contour antiderivative of the Peierls-shifted band energy.

    Eq. g_contour_non_final2: eps(tbar) = [theta(-tbar) + theta(tbar) cos(E tbar)] eps
    - theta(tbar) ebar sin(E tbar).  For points with Re s <= 0 or on the
    imaginary branch (which sits at t_min < 0, before the field) F = eps s;
    for s > 0, F = [eps sin(Es) + ebar (cos(Es) - 1)]/E (reading R9 at E = 0).
    """
    if s.imag != 0.0 or s.real <= 0.0 or E == 0.0:
        return eps * s
    sr = s.real
    return complex((eps * math.sin(E * sr) + ebar * (math.cos(E * sr) - 1.0)) / E)


def _softplus(y: float) -> float:
    """log(1 + e^y) without overflow."""
    return float(np.logaddexp(0.0, y))


def g0_element(ti: complex, tj: complex, later: bool, eps: float, ebar: float,
               model: Model, beta: float) -> complex:
    """One element of G0_{eps,ebar}(t_i, t_j), Eq. g_contour_non_final2.

    G0 = i [f(x) - theta_c] e^{i mu (t_i - t_j)} exp(-i [F(t_i) - F(t_j)]),
    x = eps - mu, f(x) = 1/(1 + e^{beta x}); ``later`` is theta_c(t_i, t_j).
    The real part of the exponent, -x (tau_i - tau_j) with t = Re t - i tau,
    is combined with log f or log(1-f) so that nothing overflows.
    """
    mu = model.chem
    x = eps - mu
    Fi = band_phase(ti, eps, ebar, model.E)
    Fj = band_phase(tj, eps, ebar, model.E)
    expo = 1j * mu * (ti - tj) - 1j * (Fi - Fj)  # complex exponent
    re = expo.real  # = -x (tau_i - tau_j)
    im = expo.imag
    if later:  # i (f - 1) = -i / (1 + e^{-beta x})
        mag = math.exp(re - _softplus(-beta * x))
        return -1j * mag * complex(math.cos(im), math.sin(im))
    mag = math.exp(re - _softplus(beta * x))  # i f = i / (1 + e^{beta x})
    return 1j * mag * complex(math.cos(im), math.sin(im))


def g0_matrix(c: Contour, model: Model, eps: float, ebar: float) -> np.ndarray:
    """G0 sampled on the contour, theta_c(t_i, t_j) = 1 for i >= j (reading R3)."""
    n = c.n_c
    mu = model.chem
    x = eps - mu
    F = np.array([band_phase(s, eps, ebar, model.E) for s in c.t])
    expo = 1j * mu * (c.t[:, None] - c.t[None, :]) - 1j * (F[:, None] - F[None, :])
    later = np.tril(np.ones((n, n), dtype=bool))
    log_mag = np.where(later, expo.real - _softplus(-c.beta * x),
                       expo.real - _softplus(c.beta * x))
    pref = np.where(later, -1j, 1j)
    return pref * np.exp(log_mag) * np.exp(1j * expo.imag)


# --------------------------------------------------------------------------
# Lattice step: nonequilibrium Hilbert transform and current
# --------------------------------------------------------------------------


def weighted_sigma(c: Contour, sigma: np.ndarray) -> np.ndarray:
    """S = W Sigma W: the discretised operator product (Eq. matrix_multiply)."""
    return c.w[:, None] * sigma * c.w[None, :]


def lesser_columns(c: Contour) -> np.ndarray:
    """Column of G^<(t_m, t_m) for upper-branch row m = 0..N_t-1 (reading R8)."""
    return 2 * c.n_t - np.arange(c.n_t)


def ebar_shifted(c: Contour, eps: float, ebar: float, E: float) -> np.ndarray:
    """ebar_{k + theta(t) E t} at the upper-branch times (reading R7)."""
    tm = c.t[: c.n_t].real
    return np.where(tm > 0.0, ebar * np.cos(E * tm) + eps * np.sin(E * tm), ebar)


def dyson_solve(g0: np.ndarray, s: np.ndarray) -> np.ndarray:
    """[(I - G0 S)^-1 G0], the integrand of Eq. g_loc (two products, one inversion)."""
    n = g0.shape[0]
    return np.linalg.solve(np.eye(n, dtype=np.complex128) - g0 @ s, g0)


def lattice_gloc(c: Contour, model: Model, sigma: np.ndarray, eps: np.ndarray,
                 ebar: np.ndarray, wq: np.ndarray, q_indices=None):
    """G_loc = sum_q w_q [(I - G0_q S)^-1 G0_q] (Eq. g_loc) and the current.

    Returns ``(gloc, j_complex)``: ``j_complex[m] = i sum_q w_q ebar_q(t_m) G^<_q(t_m, t_m)``
    (Eq. current_def, reading R7); its real part is j(t), its imaginary part a
    diagnostic that vanishes for the exact solution.  Points are summed in the
    order given (default: q = 0, 1, ...).
    """
    s = weighted_sigma(c, sigma)
    n = c.n_c
    gloc = np.zeros((n, n), dtype=np.complex128)
    jc = np.zeros(c.n_t, dtype=np.complex128)
    rows = np.arange(c.n_t)
    cols = lesser_columns(c)
    qs = range(len(wq)) if q_indices is None else q_indices
    for q in qs:
        g0 = g0_matrix(c, model, float(eps[q]), float(ebar[q]))
        gq = dyson_solve(g0, s)
        gloc += wq[q] * gq
        jc += wq[q] * ebar_shifted(c, float(eps[q]), float(ebar[q]), model.E) * gq[rows, cols]
    return gloc, 1j * jc


def density(c: Contour, g: np.ndarray) -> np.ndarray:
    """n(t_m) = -i G^<(t_m, t_m) on the upper-branch times."""
    return -1j * g[np.arange(c.n_t), lesser_columns(c)]


# --------------------------------------------------------------------------
# Impurity step (Eqs. effective_medium, dynamical_mean_field, g_imp_solve)
# --------------------------------------------------------------------------


def m_matrix(c: Contour, mu: float) -> np.ndarray:
    """M of (i d_t^c + mu) delta_c = i W^-1 M W^-1 (Sec. II, the printed M matrix).

    M_jj = 1, M_{j,j-1} = -(1 + i W_j mu) for j >= 2 and the boundary element
    M_{1,N_c} = +(1 + i W_1 mu) (1-based).  The row's own weight picks the
    branch type; this is the count the printed det M formula uses.
    """
    n = c.n_c
    m = np.eye(n, dtype=np.complex128)
    for j in range(1, n):
        m[j, j - 1] = -(1.0 + 1j * c.w[j] * mu)
    m[0, n - 1] = 1.0 + 1j * c.w[0] * mu
    return m


def impurity_update(c: Contour, model: Model, gloc: np.ndarray, sigma: np.ndarray):
    """One Falicov-Kimball impurity step; returns (Sigma_new, G_imp).

    With S = W Sigma W and the discrete operator inverse of Eq.
    matrix_inverse_discrete (operator inverse of A = (W A W)^-1):
      A0    = inv(G_loc) + S                        (W G_0^-1 W, Eq. effective_medium, R6)
      A1    = A0 + i [M(mu - U) - M(mu)]            (W [(i d + mu - U) delta - lambda] W, R5)
      G_imp = (1 - w1) inv(A0) + w1 inv(A1)         (Eq. g_imp_solve)
      W Sigma_new W = A0 - inv(G_imp)               (impurity Dyson equation)
    """
    mu = model.chem
    s = weighted_sigma(c, sigma)
    a0 = np.linalg.inv(gloc) + s
    a1 = a0 + 1j * (m_matrix(c, mu - model.U) - m_matrix(c, mu))
    gimp = (1.0 - model.w1) * np.linalg.inv(a0) + model.w1 * np.linalg.inv(a1)
    s_new = a0 - np.linalg.inv(gimp)
    sigma_new = s_new / (c.w[:, None] * c.w[None, :])
    return sigma_new, gimp


def convergence_error(g_new: np.ndarray, g_old: np.ndarray) -> float:
    """max|G_new - G_old| / max|G_new| (reading R10)."""
    return float(np.abs(g_new - g_old).max() / np.abs(g_new).max())


@dataclass
class DmftResult:
    sigma: np.ndarray
    gloc: np.ndarray
    current: np.ndarray  # complex, real part = j(t)
    iterations: int
    error: float
    converged: bool


def dmft_solve(c: Contour, model: Model, n_quad: int, tol: float = 1e-8,
               max_iter: int = 50, sigma0: np.ndarray | None = None) -> DmftResult:
    """The DMFT loop of Sec. II: lattice step, impurity step, until G_loc converges.

    Iteration k computes G_loc from Sigma_k; once two successive G_loc agree to
    ``tol`` the loop stops and returns that G_loc, its current and the Sigma it
    came from.  Otherwise Sigma_{k+1} = impurity(G_loc, Sigma_k).  After
    ``max_iter`` lattice steps without convergence the last G_loc and the Sigma
    that produced it are returned.
    """
    eps, ebar, wq = quadrature_points(n_quad)
    sigma = np.zeros((c.n_c, c.n_c), np.complex128) if sigma0 is None else sigma0.copy()
    g_old = None
    err = float("inf")
    for it in range(1, max_iter + 1):
        gloc, jc = lattice_gloc(c, model, sigma, eps, ebar, wq)
        if g_old is not None:
            err = convergence_error(gloc, g_old)
            if err < tol:
                return DmftResult(sigma, gloc, jc, it, err, True)
        if it == max_iter:
            break
        g_old = gloc
        sigma, _ = impurity_update(c, model, gloc, sigma)
    return DmftResult(sigma, gloc, jc, max_iter, err, False)


# --------------------------------------------------------------------------
# Diagnostics: equal-time moments and the nonequilibrium density of states
# (Sec. II, the moments paragraph; Eqs. gr_omega, dos_def)
# --------------------------------------------------------------------------


def real_time_rows(c: Contour, m: int) -> tuple[int, int]:
    """Contour rows of real time t_m: upper-branch row m and its lower-branch
    partner (reading R8: for t_min the partner is the first imaginary point)."""
    return m, 2 * c.n_t - m


def retarded(c: Contour, g: np.ndarray, i: int, j: int) -> complex:
    """G^R(t_i, t_j) = G^>(t_i, t_j) - G^<(t_i, t_j) for i >= j.

    On the contour, G^> is the element (later branch row, earlier branch
    column) = (lower row of t_i, upper row of t_j); G^< = (upper of t_i, lower of t_j).
    """
    ui, li = real_time_rows(c, i)
    uj, lj = real_time_rows(c, j)
    return g[li, uj] - g[ui, lj]


def moments(c: Contour, g: np.ndarray):
    """(mu0, mu1, mu2, n) on the upper-branch times (reading R11); NaN where
    the three pairs leave the real-time window.  n(t) = -i G^<(t, t)."""
    nt = c.n_t
    mu0 = np.full(nt, np.nan)
    mu1 = np.full(nt, np.nan)
    mu2 = np.full(nt, np.nan)
    s = 2.0 * c.dt * np.arange(1, 4)
    for m in range(3, nt - 3):
        f = np.array([1j * retarded(c, g, m + k, m - k) for k in range(1, 4)])
        c2, c1, c0 = np.polyfit(s, f, 2)  # f(s) = c0 + c1 s + c2 s^2
        mu0[m] = c0.real
        mu1[m] = (1j * c1).real
        mu2[m] = (-2.0 * c2).real
    return mu0, mu1, mu2, density(c, g).real


def dos(c: Contour, g: np.ndarray, m: int, omega) -> np.ndarray:
    """rho(T = t_m, omega) = -Im G^R(T, omega) / pi (Eqs. gr_omega, dos_def),
    G^R(T, omega) = integral over t_rel >= 0 of exp(i omega t_rel) G^R(T + t_rel/2, T - t_rel/2)
    by the trapezoid rule (reading R12)."""
    omega = np.asarray(omega, dtype=np.float64)
    kmax = min(m, c.n_t - 1 - m)
    h = 2.0 * c.dt
    out = np.zeros(omega.shape, dtype=np.complex128)
    if kmax == 0:  # no relative-time interval at the edges of the window
        return out.real
    for k in range(kmax + 1):
        wk = 0.5 if k in (0, kmax) else 1.0
        out += wk * h * np.exp(1j * omega * (k * h)) * retarded(c, g, m + k, m - k)
    return -out.imag / np.pi


# --------------------------------------------------------------------------
# dt -> 0 extrapolation (Sec. II, the Lagrange extrapolation paragraph)
# --------------------------------------------------------------------------


def lagrange_extrapolate(dts, values) -> np.ndarray:
    """Value at dt = 0 of the Lagrange polynomial through (dt_k, values_k).

    ``values`` has the dt index first; any trailing shape is extrapolated
    pointwise.  Quadratic for three dt values, cubic for four, and so on.
    """
    dts = np.asarray(dts, dtype=np.float64)
    vals = np.asarray(values)
    out = np.zeros(vals.shape[1:], dtype=np.result_type(vals, np.float64))
    for k in range(len(dts)):
        lk = 1.0
        for m in range(len(dts)):
            if m != k:
                lk *= (0.0 - dts[m]) / (dts[k] - dts[m])
        out = out + lk * vals[k]
    return out
