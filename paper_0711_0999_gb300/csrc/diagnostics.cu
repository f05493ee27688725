// Accuracy diagnostics of a converged contour Green's function (Sec. II): the
// equal-time moments of the retarded function and the nonequilibrium density
// of states of Eqs. gr_omega and dos_def.  FP64 throughout.
#include <math.h>

#include "lattice.cuh"

namespace nedmft {
namespace {

// G^R(t_i, t_j) = G^>(t_i, t_j) - G^<(t_i, t_j) on the real branches, i >= j:
// G^> is the element (lower-branch row of t_i, upper row of t_j), G^< the
// element (upper row of t_i, lower row of t_j); the lower-branch row of t_m
// is 2 N_t - m (for t_min the first imaginary point).
__device__ __forceinline__ double2 retarded_at(const double2* __restrict__ g, int n, int nt, int i, int j) {
  const double2 gt = g[(size_t)(2 * nt - i) * n + j];
  const double2 lt = g[(size_t)i * n + (2 * nt - j)];
  return make_double2(gt.x - lt.x, gt.y - lt.y);
}

// f(s) = i G^R(t_m + s/2, t_m - s/2) = mu0 - i mu1 s - mu2 s^2 / 2 + ...: the
// quadratic through s = h, 2h, 3h (h = 2 dt) has value 3 f1 - 3 f2 + f3 at 0,
// slope (-5 f1 + 8 f2 - 3 f3) / 2h and curvature (f1 - 2 f2 + f3) / 2h^2.
__global__ void moments_kernel(const double2* __restrict__ g, int n, int nt, double dt, double* __restrict__ mu0,
                               double* __restrict__ mu1, double* __restrict__ mu2, double* __restrict__ dens) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nt) return;
  if (dens) dens[m] = g[(size_t)m * n + (2 * nt - m)].y;  // n = -i G^< with G^< = i n
  double a0 = NAN, a1 = NAN, a2 = NAN;
  if (m >= 3 && m + 3 < nt) {
    double2 f[3];
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
      const double2 r = retarded_at(g, n, nt, m + k, m - k);
      f[k - 1] = make_double2(-r.y, r.x);  // i G^R
    }
    const double h = 2.0 * dt;
    const double2 v0 = make_double2(3.0 * f[0].x - 3.0 * f[1].x + f[2].x, 3.0 * f[0].y - 3.0 * f[1].y + f[2].y);
    const double2 v1 = make_double2((-5.0 * f[0].x + 8.0 * f[1].x - 3.0 * f[2].x) / (2.0 * h),
                                    (-5.0 * f[0].y + 8.0 * f[1].y - 3.0 * f[2].y) / (2.0 * h));
    const double2 v2 = make_double2((f[0].x - 2.0 * f[1].x + f[2].x) / (2.0 * h * h),
                                    (f[0].y - 2.0 * f[1].y + f[2].y) / (2.0 * h * h));
    a0 = v0.x;
    a1 = -v1.y;  // Re(i v1)
    a2 = -2.0 * v2.x;
  }
  if (mu0) mu0[m] = a0;
  if (mu1) mu1[m] = a1;
  if (mu2) mu2[m] = a2;
}

// rho(t_m, omega) = -Im G^R(t_m, omega) / pi with the trapezoid rule over the
// relative times 2 k dt, k = 0 .. min(m, N_t - 1 - m).  Block x: average time
// m_list[x]; one thread per omega.
__global__ void dos_kernel(const double2* __restrict__ g, int n, int nt, double dt, const int* __restrict__ m_list,
                           const double* __restrict__ omega, int n_omega, double* __restrict__ rho) {
  const int a = blockIdx.x;
  const int w = blockIdx.y * blockDim.x + threadIdx.x;
  if (w >= n_omega) return;
  const int m = m_list[a];
  double* out = rho + (size_t)a * n_omega + w;
  if (m < 0 || m >= nt) {
    *out = NAN;
    return;
  }
  const int kmax = min(m, nt - 1 - m);
  if (kmax == 0) {
    *out = 0.0;
    return;
  }
  const double h = 2.0 * dt, om = omega[w];
  double im = 0.0;
  for (int k = 0; k <= kmax; ++k) {
    const double2 r = retarded_at(g, n, nt, m + k, m - k);
    double sn, cs;
    sincos(om * (k * h), &sn, &cs);
    const double wk = (k == 0 || k == kmax) ? 0.5 * h : h;
    im += wk * (cs * r.y + sn * r.x);  // Im(e^{i om s} G^R)
  }
  *out = -im / M_PI;
}

}  // namespace
}  // namespace nedmft

using namespace nedmft;

extern "C" int nedmft_moments(const nedmft_contour* c, const nedmft_c128* gloc_d, double* mu0_d, double* mu1_d,
                              double* mu2_d, double* dens_d, void* stream) {
  if (!c || !gloc_d) return set_error(NEDMFT_EINVAL, "moments: NULL argument");
  if (c->n_t < 1 || c->n_tau < 1 || c->n_c != 2 * c->n_t + c->n_tau || !(c->dt > 0))
    return set_error(NEDMFT_EINVAL, "moments: invalid contour");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  moments_kernel<<<ceil_div(c->n_t, 128), 128, 0, st>>>(reinterpret_cast<const double2*>(gloc_d), c->n_c, c->n_t,
                                                        c->dt, mu0_d, mu1_d, mu2_d, dens_d);
  NED_LAUNCH_CHECK("moments_kernel");
  return NEDMFT_OK;
}

extern "C" int nedmft_dos(const nedmft_contour* c, const nedmft_c128* gloc_d, const int32_t* m_d, int32_t n_avg,
                          const double* omega_d, int32_t n_omega, double* rho_d, void* stream) {
  if (!c || !gloc_d) return set_error(NEDMFT_EINVAL, "dos: NULL argument");
  if (c->n_t < 1 || c->n_tau < 1 || c->n_c != 2 * c->n_t + c->n_tau || !(c->dt > 0))
    return set_error(NEDMFT_EINVAL, "dos: invalid contour");
  if (n_avg < 0 || n_omega < 0 || n_avg > 65535) return set_error(NEDMFT_EINVAL, "dos: bad sizes");
  if (n_avg == 0 || n_omega == 0) return NEDMFT_OK;  // nothing to write; the arrays may be NULL
  if (!m_d || !omega_d || !rho_d) return set_error(NEDMFT_EINVAL, "dos: NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dos_kernel<<<dim3(n_avg, ceil_div(n_omega, 128)), 128, 0, st>>>(reinterpret_cast<const double2*>(gloc_d), c->n_c,
                                                                  c->n_t, c->dt, m_d, omega_d, n_omega, rho_d);
  NED_LAUNCH_CHECK("dos_kernel");
  return NEDMFT_OK;
}
