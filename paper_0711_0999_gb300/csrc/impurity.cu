// FP64 impurity step of the Falicov-Kimball DMFT loop (the dense inversions
// with partial pivoting live with the blocked Gauss-Jordan kernels).
#include "lattice.cuh"

namespace nedmft {

// ------------------------------------------------------------------ impurity step

// A0 = inv(G_loc) + W Sigma W (in place on ginv); A1 = A0 + i [M(mu-U) - M(mu)]:
// the difference of the two point-split M matrices has -W_j U on the
// subdiagonal (row j >= 1) and +W_0 U in the boundary element (0, N-1).
__global__ void imp_build_kernel(ContourDev c, ModelDev m, const double2* __restrict__ sigma,
                                 double2* __restrict__ a0, double2* __restrict__ a1, double2* __restrict__ x0) {
  const size_t total = (size_t)c.n * c.n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / c.n), j = (int)(e % c.n);
    double2 s = cmul(cmul(weight(c, i), sigma[e]), weight(c, j));
    double2 v = cadd(a0[e], s);
    a0[e] = v;
    x0[e] = v;
    double2 d = make_double2(0.0, 0.0);
    if (i >= 1 && j == i - 1) { double2 w = weight(c, i); d = make_double2(-w.x * m.U, -w.y * m.U); }
    if (i == 0 && j == c.n - 1) { double2 w = weight(c, 0); d = cadd(d, make_double2(w.x * m.U, w.y * m.U)); }
    a1[e] = cadd(v, d);
  }
}

// G_imp = (1 - w1) inv(A0) + w1 inv(A1)  (written to g and, if requested, gimp_out).
__global__ void imp_mix_kernel(int n, double w1, const double2* __restrict__ x0, const double2* __restrict__ x1,
                               double2* __restrict__ g, double2* __restrict__ gimp_out) {
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    double2 v = make_double2((1.0 - w1) * x0[e].x + w1 * x1[e].x, (1.0 - w1) * x0[e].y + w1 * x1[e].y);
    g[e] = v;
    if (gimp_out) gimp_out[e] = v;
  }
}

// sigma_new = W^-1 (A0 - inv(G_imp)) W^-1.
__global__ void imp_sigma_kernel(ContourDev c, const double2* __restrict__ a0, const double2* __restrict__ ginv,
                                 double2* __restrict__ sigma_new) {
  const size_t total = (size_t)c.n * c.n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / c.n), j = (int)(e % c.n);
    double2 s = csub(a0[e], ginv[e]);
    double2 wi = weight(c, i), wj = weight(c, j);
    double2 ww = cmul(wi, wj);
    double m2 = ww.x * ww.x + ww.y * ww.y;
    double2 r = make_double2(ww.x / m2, -ww.y / m2);
    sigma_new[e] = cmul(s, r);
  }
}

}  // namespace nedmft

using namespace nedmft;

extern "C" size_t nedmft_impurity_workspace_size(const nedmft_contour* c) {
  if (!c || c->n_c < 1) return 0;
  size_t n = (size_t)c->n_c;
  return 4 * align256(sizeof(double2) * n * n) + pivot_inverse_workspace((int)n);
}

extern "C" int nedmft_impurity_update(const nedmft_contour* c, const nedmft_model* m, const nedmft_c128* gloc_d,
                                      const nedmft_c128* sigma_d, nedmft_c128* sigma_new_d, nedmft_c128* gimp_d,
                                      void* ws_d, size_t ws_bytes, void* stream) {
  if (!c || !m || !gloc_d || !sigma_d || !sigma_new_d || !ws_d)
    return set_error(NEDMFT_EINVAL, "impurity_update: NULL argument");
  if (sigma_new_d == gloc_d || sigma_new_d == sigma_d)
    return set_error(NEDMFT_EINVAL, "impurity_update: sigma_new_d aliases an input");
  if (c->n_c < 2) return set_error(NEDMFT_EINVAL, "impurity_update: n_c < 2");
  if (ws_bytes < nedmft_impurity_workspace_size(c))
    return set_error(NEDMFT_ENOMEM, "impurity_update: workspace %zu < %zu", ws_bytes, nedmft_impurity_workspace_size(c));
  int* status = device_status_ptr();
  if (!status) return set_error(NEDMFT_ECUDA, "impurity_update: no device status word");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ContourDev cd = to_dev(*c);
  ModelDev md{m->U, m->E, m->w1, isnan(m->mu) ? m->U / 2 : m->mu};
  const int n = cd.n;
  const size_t mat = align256(sizeof(double2) * (size_t)n * n);
  char* p = static_cast<char*>(ws_d);
  double2* a0 = reinterpret_cast<double2*>(p); p += mat;
  double2* x0 = reinterpret_cast<double2*>(p); p += mat;
  double2* a1 = reinterpret_cast<double2*>(p); p += mat;
  double2* g = reinterpret_cast<double2*>(p); p += mat;
  void* pws = p;
  const size_t total = (size_t)n * n;
  int bx = (int)((total + 255) / 256);
  if (bx > 152 * 8) bx = 152 * 8;
  NED_CUDA(cudaMemcpyAsync(a0, gloc_d, sizeof(double2) * total, cudaMemcpyDeviceToDevice, st));
  int rc = pivot_inverse(a0, n, pws, st, status);  // a0 = inv(G_loc)
  if (rc) return rc;
  imp_build_kernel<<<bx, 256, 0, st>>>(cd, md, reinterpret_cast<const double2*>(sigma_d), a0, a1, x0);
  NED_LAUNCH_CHECK("imp_build_kernel");
  if ((rc = pivot_inverse(x0, n, pws, st, status))) return rc;  // x0 = inv(A0)
  if ((rc = pivot_inverse(a1, n, pws, st, status))) return rc;  // a1 = inv(A1)
  imp_mix_kernel<<<bx, 256, 0, st>>>(n, md.w1, x0, a1, g, reinterpret_cast<double2*>(gimp_d));
  NED_LAUNCH_CHECK("imp_mix_kernel");
  if ((rc = pivot_inverse(g, n, pws, st, status))) return rc;  // g = inv(G_imp)
  imp_sigma_kernel<<<bx, 256, 0, st>>>(cd, a0, g, reinterpret_cast<double2*>(sigma_new_d));
  NED_LAUNCH_CHECK("imp_sigma_kernel");
  return NEDMFT_OK;
}
