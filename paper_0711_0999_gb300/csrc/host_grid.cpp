// Host-side grid construction: the contour of Eqs. time_discrete and
// integration_weights and the Gauss-Hermite rule of the joint Gaussian
// density of states (Eq. joint_dos).
#include <math.h>

#include <vector>

#include "common.cuh"

using namespace nedmft;

namespace {

bool integer_ratio(double span, double step, int32_t* out) {
  if (!(step > 0.0) || !(span > 0.0)) return false;
  double r = span / step;
  double n = nearbyint(r);
  if (n < 1.0 || n > 1e8) return false;
  if (fabs(r - n) > 1e-9 * fmax(1.0, fabs(r))) return false;
  *out = (int32_t)n;
  return true;
}

// Scaled orthonormal Hermite values h_k(x) = p_k(x) exp(-x^2/2), k = 0..n,
// for the weight exp(-x^2): h_0 = pi^-1/4 e^{-x^2/2},
// h_{k+1} = sqrt(2/(k+1)) x h_k - sqrt(k/(k+1)) h_{k-1}.
// Returns h_n, sets *hm1 = h_{n-1} and *sumsq = sum_{k<n} h_k^2.
double hermite_scaled(int n, double x, double* hm1, double* sumsq) {
  double h_prev = 0.0;
  double h = pow(M_PI, -0.25) * exp(-0.5 * x * x);
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    s += h * h;
    double h_next = sqrt(2.0 / (k + 1)) * x * h - sqrt((double)k / (k + 1)) * h_prev;
    h_prev = h;
    h = h_next;
  }
  if (hm1) *hm1 = h_prev;
  if (sumsq) *sumsq = s;
  return h;
}

}  // namespace

extern "C" int nedmft_contour_grid(double t_min, double t_max, double dt, double beta, double dtau,
                                   nedmft_contour* out, nedmft_c128* t_host, nedmft_c128* w_host) {
  if (!out) return set_error(NEDMFT_EINVAL, "contour_grid: out is NULL");
  int32_t n_t = 0, n_tau = 0;
  if (!integer_ratio(t_max - t_min, dt, &n_t))
    return set_error(NEDMFT_EINVAL, "contour_grid: (t_max - t_min)/dt = (%g - %g)/%g is not a positive integer",
                     t_max, t_min, dt);
  if (!integer_ratio(beta, dtau, &n_tau))
    return set_error(NEDMFT_EINVAL, "contour_grid: beta/dtau = %g/%g is not a positive integer", beta, dtau);
  if ((int64_t)2 * n_t + n_tau > 65536)
    return set_error(NEDMFT_EINVAL, "contour_grid: N_c = %d exceeds 65536", 2 * n_t + n_tau);
  out->t_min = t_min; out->t_max = t_max; out->dt = dt; out->beta = beta; out->dtau = dtau;
  out->n_t = n_t; out->n_tau = n_tau; out->n_c = 2 * n_t + n_tau;
  ContourDev c = to_dev(*out);
  for (int j = 0; j < c.n; ++j) {
    if (t_host) { t_host[j].re = t_re(c, j); t_host[j].im = -t_tau(c, j); }
    if (w_host) { double2 w = weight(c, j); w_host[j].re = w.x; w_host[j].im = w.y; }
  }
  return NEDMFT_OK;
}

extern "C" int nedmft_gauss_hermite(int32_t n, double* x_host, double* w_host) {
  if (n < 1 || n > 512) return set_error(NEDMFT_EINVAL, "gauss_hermite: n = %d outside [1, 512]", n);
  if (!x_host || !w_host) return set_error(NEDMFT_EINVAL, "gauss_hermite: NULL output");
  // Bracket the n roots of h_n by sign changes on a fine grid covering
  // |x| <= sqrt(2n+1) + 2 (all roots lie inside sqrt(2n+1)), then polish each
  // with Newton steps on h_n, h_n' = sqrt(2n) h_{n-1} - x h_n.
  const double L = sqrt(2.0 * n + 1.0) + 2.0;
  const int steps = (int)(2.0 * L / 1e-3) + 1;
  std::vector<double> roots;
  roots.reserve(n);
  double xa = -L, fa = hermite_scaled(n, xa, nullptr, nullptr);
  for (int s = 1; s <= steps && (int)roots.size() < n; ++s) {
    double xb = -L + 2.0 * L * s / steps;
    double fb = hermite_scaled(n, xb, nullptr, nullptr);
    if (fa == 0.0) {
      roots.push_back(xa);
    } else if ((fa < 0.0) != (fb < 0.0) && fb != 0.0) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 60; ++it) {  // bisection to a tight bracket
        double mid = 0.5 * (lo + hi);
        double fm = hermite_scaled(n, mid, nullptr, nullptr);
        if (fm == 0.0) { lo = hi = mid; break; }
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
        if (hi - lo < 1e-12) break;
      }
      double x = 0.5 * (lo + hi);
      for (int it = 0; it < 8; ++it) {
        double hm1 = 0.0;
        double h = hermite_scaled(n, x, &hm1, nullptr);
        double d = sqrt(2.0 * n) * hm1 - x * h;
        if (d == 0.0) break;
        double step = h / d;
        x -= step;
        if (fabs(step) < 1e-16 * fmax(1.0, fabs(x))) break;
      }
      roots.push_back(x);
    }
    xa = xb; fa = fb;
  }
  if ((int)roots.size() != n)
    return set_error(NEDMFT_EINVAL, "gauss_hermite: found %d of %d roots", (int)roots.size(), n);
  for (int i = 0; i < n; ++i) {
    double sumsq = 0.0;
    hermite_scaled(n, roots[i], nullptr, &sumsq);
    // Christoffel weight 1/sum p_k^2 = e^{-x^2}/sum h_k^2, normalised by sqrt(pi).
    x_host[i] = roots[i];
    w_host[i] = exp(-roots[i] * roots[i]) / sumsq / sqrt(M_PI);
  }
  return NEDMFT_OK;
}

extern "C" int nedmft_quadrature_grid(int32_t n, double* eps_host, double* ebar_host, double* wq_host) {
  if (!eps_host || !ebar_host || !wq_host) return set_error(NEDMFT_EINVAL, "quadrature_grid: NULL output");
  std::vector<double> x(n > 0 ? n : 1), w(n > 0 ? n : 1);
  int st = nedmft_gauss_hermite(n, x.data(), w.data());
  if (st != NEDMFT_OK) return st;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      eps_host[a * n + b] = x[a];
      ebar_host[a * n + b] = x[b];
      wq_host[a * n + b] = w[a] * w[b];
    }
  return NEDMFT_OK;
}
