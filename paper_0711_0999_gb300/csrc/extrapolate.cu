// dt -> 0 extrapolation of the current (Sec. II, the Lagrange extrapolation
// paragraph) and the averaged N / N+1 Gauss-Hermite grid (Sec. II quadrature
// paragraph).
#include <math.h>

#include <vector>

#include "common.cuh"

namespace nedmft {
namespace {

constexpr int kMaxRuns = 16;

struct ExtraArgs {
  int k;
  const double* j[kMaxRuns];  // j_k on its own grid t_min + m dt_k, m < n_t[k]
  double t_min[kMaxRuns], dt[kMaxRuns];
  int n_t[kMaxRuns];
  double coef[kMaxRuns];      // L_k(0)
};

// out[e] = sum_k L_k(0) j_k(t_e), j_k(t) linear between the grid points of run k.
__global__ void extrapolate_kernel(ExtraArgs a, const double* __restrict__ t_out, int n_out, double* __restrict__ out,
                                   int* __restrict__ bad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_out) return;
  const double t = t_out[e];
  double acc = 0.0;
  for (int r = 0; r < a.k; ++r) {
    const double x = (t - a.t_min[r]) / a.dt[r];
    int m = (int)floor(x);
    double f = x - m;
    if (m < 0 || m > a.n_t[r] - 1 || (m == a.n_t[r] - 1 && f > 1e-9)) {
      atomicExch(bad, 1);
      return;
    }
    if (m == a.n_t[r] - 1) f = 0.0;
    const double v0 = a.j[r][m];
    const double v1 = f > 0.0 ? a.j[r][m + 1] : v0;
    acc += a.coef[r] * (v0 + f * (v1 - v0));
  }
  out[e] = acc;
}

}  // namespace
}  // namespace nedmft

using namespace nedmft;

extern "C" int nedmft_extrapolate_current(int32_t k, const double* dts_host, const double* t_min_host,
                                          const int32_t* n_t_host, const double* const* j_d, const double* t_out_d,
                                          int32_t n_out, double* out_d, int32_t* bad_d, void* stream) {
  if (k < 1 || k > kMaxRuns) return set_error(NEDMFT_EINVAL, "extrapolate_current: k = %d outside [1, %d]", k, kMaxRuns);
  if (!dts_host || !t_min_host || !n_t_host || !j_d || !t_out_d || !out_d || !bad_d)
    return set_error(NEDMFT_EINVAL, "extrapolate_current: NULL argument");
  if (n_out < 1) return set_error(NEDMFT_EINVAL, "extrapolate_current: n_out < 1");
  ExtraArgs a{};
  a.k = k;
  for (int r = 0; r < k; ++r) {
    if (!(dts_host[r] > 0.0) || n_t_host[r] < 1 || !j_d[r])
      return set_error(NEDMFT_EINVAL, "extrapolate_current: bad run %d", r);
    for (int s = 0; s < r; ++s)
      if (fabs(dts_host[r] - dts_host[s]) < 1e-14 * dts_host[r])
        return set_error(NEDMFT_EINVAL, "extrapolate_current: repeated dt %g", dts_host[r]);
    a.j[r] = j_d[r];
    a.t_min[r] = t_min_host[r];
    a.dt[r] = dts_host[r];
    a.n_t[r] = n_t_host[r];
    double l = 1.0;  // Lagrange basis polynomial of node r at dt = 0
    for (int s = 0; s < k; ++s)
      if (s != r) l *= (0.0 - dts_host[s]) / (dts_host[r] - dts_host[s]);
    a.coef[r] = l;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NED_CUDA(cudaMemsetAsync(bad_d, 0, sizeof(int32_t), st));
  extrapolate_kernel<<<ceil_div(n_out, 256), 256, 0, st>>>(a, t_out_d, n_out, out_d, bad_d);
  NED_LAUNCH_CHECK("extrapolate_kernel");
  return NEDMFT_OK;
}

extern "C" int nedmft_quadrature_grid_avg(int32_t n, double* eps_host, double* ebar_host, double* wq_host) {
  if (!eps_host || !ebar_host || !wq_host) return set_error(NEDMFT_EINVAL, "quadrature_grid_avg: NULL output");
  if (n < 1 || n > 511) return set_error(NEDMFT_EINVAL, "quadrature_grid_avg: n = %d outside [1, 511]", n);
  const size_t a = (size_t)n * n;
  int rc = nedmft_quadrature_grid(n, eps_host, ebar_host, wq_host);
  if (rc) return rc;
  rc = nedmft_quadrature_grid(n + 1, eps_host + a, ebar_host + a, wq_host + a);
  if (rc) return rc;
  const size_t tot = a + (size_t)(n + 1) * (n + 1);
  for (size_t q = 0; q < tot; ++q) wq_host[q] *= 0.5;
  return NEDMFT_OK;
}
