// FP64 impurity step of the Falicov-Kimball DMFT loop (the dense inversions
// with partial pivoting live with the blocked Gauss-Jordan kernels).
#include "lattice.cuh"

namespace nedmft {

// ------------------------------------------------------------------ impurity step
//
// With S = W Sigma W, A0 = inv(G_loc) + S (Eq. effective_medium) and the
// point-split difference D = i [M(mu - U) - M(mu)] (one entry per row:
// D_{j,j-1} = -U W_j for j >= 1, D_{0,N-1} = +U W_0), the impurity Green's
// function of Eq. g_imp_solve is G_imp = (1 - w1) inv(A0) + w1 inv(A0 + D).
// Both terms share A_h = A0 + (1 - w1) D:  G_imp = inv(A0) A_h inv(A0 + D),
// so inv(G_imp) = (A0 + D) inv(A_h) A0 and the impurity Dyson equation gives
//   W Sigma_new W = A0 - inv(G_imp) = -w1 D + w1 (1 - w1) D inv(A_h) D,
// two inversions (G_loc and A_h) instead of four; D inv(A_h) D is a scaled
// gather because D is a scaled cyclic shift:
//   (D X D)_{ij} = d_i X[i-1][j+1] d_{j+1}  (indices mod N),
//   d_i = -U W_i (i >= 1), d_0 = +U W_0.

__device__ __forceinline__ double2 d_entry(const ContourDev& c, double U, int i) {
  const double2 w = weight(c, i);
  return i == 0 ? make_double2(U * w.x, U * w.y) : make_double2(-U * w.x, -U * w.y);
}

// a0 <- a0 + S (a0 holds inv(G_loc)); ah = a0 + (1 - w1) D.
__global__ void imp_build_kernel(ContourDev c, ModelDev m, const double2* __restrict__ sigma,
                                 double2* __restrict__ a0, double2* __restrict__ ah) {
  const size_t total = (size_t)c.n * c.n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / c.n), j = (int)(e % c.n);
    const double2 s = cmul(cmul(weight(c, i), sigma[e]), weight(c, j));
    const double2 v = cadd(a0[e], s);
    a0[e] = v;
    double2 h = v;
    if (j == (i == 0 ? c.n - 1 : i - 1)) {
      const double2 d = d_entry(c, m.U, i);
      h = cadd(h, make_double2((1.0 - m.w1) * d.x, (1.0 - m.w1) * d.y));
    }
    ah[e] = h;
  }
}

// sigma_new = W^-1 [-w1 D + w1 (1 - w1) D X_h D] W^-1 with X_h = inv(A_h); if
// g is given, g = A0 - W sigma_new W (= inv(G_imp)).
__global__ void imp_sigma_kernel(ContourDev c, ModelDev m, const double2* __restrict__ xh,
                                 const double2* __restrict__ a0, double2* __restrict__ sigma_new,
                                 double2* __restrict__ g) {
  const int n = c.n;
  const size_t total = (size_t)n * n;
  const double w1 = m.w1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const int ip = i == 0 ? n - 1 : i - 1;  // the column of row i's entry of D
    const int jn = j + 1 == n ? 0 : j + 1;  // the row of D whose entry lies in column j
    const double2 di = d_entry(c, m.U, i), dj = d_entry(c, m.U, jn);
    double2 v = cmul(cmul(di, xh[(size_t)ip * n + jn]), dj);
    v = make_double2(w1 * (1.0 - w1) * v.x, w1 * (1.0 - w1) * v.y);
    if (j == ip) v = make_double2(v.x - w1 * di.x, v.y - w1 * di.y);
    if (g) g[e] = csub(a0[e], v);
    const double2 ww = cmul(weight(c, i), weight(c, j));
    const double m2 = ww.x * ww.x + ww.y * ww.y;
    sigma_new[e] = cmul(v, make_double2(ww.x / m2, -ww.y / m2));
  }
}

}  // namespace nedmft

using namespace nedmft;

extern "C" size_t nedmft_impurity_workspace_size(const nedmft_contour* c) {
  if (!c || c->n_c < 1) return 0;
  size_t n = (size_t)c->n_c;
  return 3 * align256(sizeof(double2) * n * n) + pivot_inverse_workspace((int)n);
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
  double2* ah = reinterpret_cast<double2*>(p); p += mat;
  double2* g = reinterpret_cast<double2*>(p); p += mat;
  void* pws = p;
  const size_t total = (size_t)n * n;
  int bx = (int)((total + 255) / 256);
  if (bx > 152 * 8) bx = 152 * 8;
  NED_CUDA(cudaMemcpyAsync(a0, gloc_d, sizeof(double2) * total, cudaMemcpyDeviceToDevice, st));
  int rc = pivot_inverse(a0, n, pws, st, status);  // a0 = inv(G_loc)
  if (rc) return rc;
  imp_build_kernel<<<bx, 256, 0, st>>>(cd, md, reinterpret_cast<const double2*>(sigma_d), a0, ah);
  NED_LAUNCH_CHECK("imp_build_kernel");
  if ((rc = pivot_inverse(ah, n, pws, st, status))) return rc;  // ah = X_h = inv(A_h)
  imp_sigma_kernel<<<bx, 256, 0, st>>>(cd, md, ah, a0, reinterpret_cast<double2*>(sigma_new_d), gimp_d ? g : nullptr);
  NED_LAUNCH_CHECK("imp_sigma_kernel");
  if (gimp_d) {
    if ((rc = pivot_inverse(g, n, pws, st, status))) return rc;  // G_imp = inv(A0 - W sigma_new W)
    NED_CUDA(cudaMemcpyAsync(gimp_d, g, sizeof(double2) * total, cudaMemcpyDeviceToDevice, st));
  }
  return NEDMFT_OK;
}
