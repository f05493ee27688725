// FP64 impurity step of the Falicov-Kimball DMFT loop and the dense
// partial-pivoting inversion it uses.
#include "lattice.cuh"

namespace nedmft {

// ------------------------------------------------------------------ Gauss-Jordan with partial pivoting

// Workspace: colbuf (n), tmp matrix (n*n), pivot rows (n ints), inverse column map (n ints), pinv (1).
size_t pivot_inverse_workspace(int n) {
  return align256(sizeof(double2) * n) + align256(sizeof(double2) * (size_t)n * n) + align256(sizeof(int) * n) * 2 +
         align256(sizeof(double2));
}

// Step k, part 1 (one CTA): pick the row p >= k with the largest |a_pk|, swap
// rows k and p, save column k, scale row k by 1/a_kk (a_kk <- 1/a_kk).
__global__ void __launch_bounds__(1024) piv_select_kernel(double2* __restrict__ a, int n, int k,
                                                          double2* __restrict__ col, int* __restrict__ piv,
                                                          double2* __restrict__ pinv_out, int* status) {
  __shared__ double best_v[1024];
  __shared__ int best_i[1024];
  __shared__ double2 pinv_s;
  double bv = -1.0;
  int bi = k;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    double2 v = a[(size_t)i * n + k];
    double m = v.x * v.x + v.y * v.y;
    if (m > bv) { bv = m; bi = i; }
  }
  best_v[threadIdx.x] = bv;
  best_i[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double ov = best_v[threadIdx.x + s];
      int oi = best_i[threadIdx.x + s];
      if (ov > best_v[threadIdx.x] || (ov == best_v[threadIdx.x] && oi < best_i[threadIdx.x])) {
        best_v[threadIdx.x] = ov;
        best_i[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int p = best_i[0];
  if (p != k) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double2 t = a[(size_t)k * n + j];
      a[(size_t)k * n + j] = a[(size_t)p * n + j];
      a[(size_t)p * n + j] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 pv = a[(size_t)k * n + k];
    double m = pv.x * pv.x + pv.y * pv.y;
    if (!(m > 1e-280)) {
      atomicCAS(status, 0, DS_SINGULAR);
      pinv_s = make_double2(1e140, 0.0);
    } else {
      pinv_s = make_double2(pv.x / m, -pv.y / m);
    }
    piv[k] = p;
    *pinv_out = pinv_s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = a[(size_t)i * n + k];
  __syncthreads();
  const double2 pinv = pinv_s;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    a[(size_t)k * n + j] = (j == k) ? pinv : cmul(a[(size_t)k * n + j], pinv);
}

// Step k, part 2: eliminate column k from every other row.
__global__ void piv_eliminate_kernel(double2* __restrict__ a, int n, int k, const double2* __restrict__ col,
                                     const double2* __restrict__ pinv_p) {
  const double2 pinv = *pinv_p;
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    if (i == k) continue;
    double2 f = col[i];
    if (j == k) {
      double2 v = cmul(f, pinv);
      a[e] = make_double2(-v.x, -v.y);
    } else {
      double2 r = a[(size_t)k * n + j];
      double2 v = a[e];
      v.x -= f.x * r.x - f.y * r.y;
      v.y -= f.x * r.y + f.y * r.x;
      a[e] = v;
    }
  }
}

// inv[idx] = j such that column j of A^-1 is column idx of the in-place result.
__global__ void piv_colmap_kernel(int n, const int* __restrict__ piv, int* __restrict__ inv) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int j = 0; j < n; ++j) inv[j] = j;
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    int t = inv[k]; inv[k] = inv[p]; inv[p] = t;
  }
}

__global__ void piv_permute_kernel(const double2* __restrict__ x, int n, const int* __restrict__ inv,
                                   double2* __restrict__ y) {
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), c = (int)(e % n);
    y[(size_t)i * n + inv[c]] = x[e];
  }
}

int pivot_inverse(double2* a, int n, void* ws, cudaStream_t st, int* status) {
  char* p = static_cast<char*>(ws);
  double2* col = reinterpret_cast<double2*>(p); p += align256(sizeof(double2) * n);
  double2* tmp = reinterpret_cast<double2*>(p); p += align256(sizeof(double2) * (size_t)n * n);
  int* piv = reinterpret_cast<int*>(p); p += align256(sizeof(int) * n);
  int* inv = reinterpret_cast<int*>(p); p += align256(sizeof(int) * n);
  double2* pinv = reinterpret_cast<double2*>(p);
  const size_t total = (size_t)n * n;
  int bx = (int)((total + 255) / 256);
  if (bx > 152 * 8) bx = 152 * 8;
  for (int k = 0; k < n; ++k) {
    piv_select_kernel<<<1, 1024, 0, st>>>(a, n, k, col, piv, pinv, status);
    NED_LAUNCH_CHECK("piv_select_kernel");
    piv_eliminate_kernel<<<bx, 256, 0, st>>>(a, n, k, col, pinv);
    NED_LAUNCH_CHECK("piv_eliminate_kernel");
  }
  piv_colmap_kernel<<<1, 1, 0, st>>>(n, piv, inv);
  NED_LAUNCH_CHECK("piv_colmap_kernel");
  piv_permute_kernel<<<bx, 256, 0, st>>>(a, n, inv, tmp);
  NED_LAUNCH_CHECK("piv_permute_kernel");
  NED_CUDA(cudaMemcpyAsync(a, tmp, sizeof(double2) * total, cudaMemcpyDeviceToDevice, st));
  return NEDMFT_OK;
}

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
