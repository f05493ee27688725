// Learned warm start of the self-energy.  The impurity step gives
//   W Sigma W = -w1 D + w1 (1 - w1) D X D,  X = inv(A0 + (1 - w1) D),
// with D the point-split difference of the M matrices (one entry per row:
// d_i at (i, i-1), indices mod N, d_i = -U W_i for i >= 1, d_0 = +U W_0).  X
// is an impurity Green's function -- smooth along the contour, of order one
// for any U, with its jump at equal contour times -- while Sigma itself carries
// factors of the step sizes at the ends of the branches.  A small MLP maps
// (U, E, dt, t, t') to X(t, t'); the self-energy follows from the identity
// above.  Forward, backward (mean-squared error) and Adam are
// hand-written kernels; the GEMMs run on the tensor cores (tcgen05, operands
// rounded to bf16, FP32 sums in TMEM), weights and optimizer state are FP32.
#include <math.h>

#include "common.cuh"
#include "umma.cuh"

namespace nedmft {
namespace {

constexpr int kIn = 17;      // features per (t, t') pair
constexpr int kHid = 256;    // width of the four hidden layers
constexpr int kOut = 2;      // Re, Im of the smooth Sigma part
constexpr int kLayers = 5;   // 4 hidden + output
constexpr int kDims[kLayers + 1] = {kIn, kHid, kHid, kHid, kHid, kOut};

constexpr size_t w_off(int l) {  // host only: offsets are passed to kernels as pointers
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += (size_t)kDims[i] * kDims[i + 1] + kDims[i + 1];
  return o;
}
constexpr size_t kParams = w_off(kLayers);

// Largest K split of a weight-gradient GEMM (K = samples): enough CTAs to
// cover the 152 SMs when C has one or two 128-row tiles.
constexpr int kMaxSplits = 152;
int splits_for(int m, int k) {
  const int tiles = (m + 127) / 128, chunks = (k + 63) / 64;
  const int s = kMaxSplits / tiles;
  return s < chunks ? s : chunks;
}
size_t split_bytes() {  // the largest split buffer over the layers
  size_t b = 0;
  for (int l = 0; l < kLayers; ++l) {
    const size_t x = umma_mlp_split_bytes(kDims[l], kDims[l + 1], kMaxSplits / ((kDims[l] + 127) / 128));
    b = x > b ? x : b;
  }
  return b;
}

// C = op(A) op(B) (+ bias) on the tensor cores (bf16 operands, FP32 sums);
// `part` (split_bytes) lets the weight gradients split their long K.
template <bool TA, bool TB>
int gemm(const float* A, const float* B, const float* bias, float* C, int m, int n, int k, bool acc, cudaStream_t st,
         float* part = nullptr) {
  return umma_mlp_gemm(A, B, bias, C, m, n, k, TA, TB, acc, part, part ? splits_for(m, k) : 1, st);
}

__global__ void tanh_kernel(float* __restrict__ h, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    h[e] = tanhf(h[e]);
}

// dZ = dH * (1 - H^2) in place on dH (H = tanh(Z))
__global__ void tanh_back_kernel(const float* __restrict__ h, float* __restrict__ d, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    d[e] *= 1.f - h[e] * h[e];
}

// dY = 2 (Y - T) / n, loss partial sums per block
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy, size_t n,
                           float inv, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float r = y[e] - t[e];
    dy[e] = 2.f * r * inv;
    s += (double)r * r;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void loss_finish_kernel(const double* __restrict__ part, int nb, double inv, float* __restrict__ loss) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0.0;
  for (int i = 0; i < nb; ++i) s += part[i];
  *loss = (float)(s * inv);
}

// db[j] = sum_i d[i][j]
__global__ void bias_grad_kernel(const float* __restrict__ d, int m, int n, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.f;
  for (int i = 0; i < m; ++i) s += d[(size_t)i * n + j];
  db[j] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float a = b1 * m1[e] + (1.f - b1) * gg;
    const float b = b2 * m2[e] + (1.f - b2) * gg * gg;
    m1[e] = a;
    m2[e] = b;
    p[e] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

// Features of the pair (t_a, t_b) of X, built to carry over to contours
// longer than the training runs' (the field is switched on at t = 0; after a
// few units of time a metal's Green's function depends on t - t' alone):
// U/2.5, E/4, tanh(Re(t_a - t_b)/3), then for each time t (real part r,
// imaginary-branch depth tau) tanh(max(r, 0)/3) (the elapsed field time,
// saturating), min(r, 0)/5 (the time before the field), tau/beta and the
// branch one-hot (upper, lower, imaginary), then the contour order
// theta_c(t_a, t_b) (1 for a >= b), across which X jumps, and dt / 0.1 (the
// discrete X differs from the continuum one at order dt, so the network learns
// it at the training steps and the warm start extrapolates in dt).
__global__ void features_kernel(ContourDev c, ModelDev m, double dt_feature, float* __restrict__ x) {
  const size_t total = (size_t)c.n * c.n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / c.n), j = (int)(e % c.n);
    float* f = x + e * kIn;
    f[0] = (float)(m.U / 2.5);
    f[1] = (float)(m.E / 4.0);
    f[2] = (float)tanh((t_re(c, i) - t_re(c, j)) / 3.0);
    const int ij[2] = {i, j};
    for (int s = 0; s < 2; ++s) {
      const int k = ij[s];
      const double r = t_re(c, k);
      f[3 + 6 * s] = (float)tanh(fmax(r, 0.0) / 3.0);
      f[4 + 6 * s] = (float)(fmin(r, 0.0) / 5.0);
      f[5 + 6 * s] = (float)(t_tau(c, k) / c.beta);
      f[6 + 6 * s] = k < c.nt ? 1.f : 0.f;
      f[7 + 6 * s] = (k >= c.nt && k < 2 * c.nt) ? 1.f : 0.f;
      f[8 + 6 * s] = k >= 2 * c.nt ? 1.f : 0.f;
    }
    f[15] = i >= j ? 1.f : 0.f;
    f[16] = (float)(dt_feature / 0.1);
  }
}

// d_i, the entry of D in row i (column i - 1 mod N).
__device__ __forceinline__ double2 d_entry(const ContourDev& c, double U, int i) {
  const double2 w = weight(c, i);
  return i == 0 ? make_double2(U * w.x, U * w.y) : make_double2(-U * w.x, -U * w.y);
}

// Sigma from X: W Sigma W = -w1 D + w1 (1 - w1) D X D, i.e.
// Sigma_ij = [-w1 D_ij + w1 (1 - w1) d_i X[i-1][j+1] d_{j+1}] / (W_i W_j)
// (indices mod N); X[a][b] is the complex value y[(a N + b)] (Re, Im).
__global__ void assemble_sigma_kernel(ContourDev c, ModelDev m, const float* __restrict__ y,
                                      double2* __restrict__ sigma) {
  const int n = c.n;
  const size_t total = (size_t)n * n;
  const double w1 = m.w1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const int ip = i == 0 ? n - 1 : i - 1, jn = j + 1 == n ? 0 : j + 1;
    const size_t f = (size_t)ip * n + jn;
    const double2 x = make_double2(y[2 * f], y[2 * f + 1]);
    const double2 di = d_entry(c, m.U, i);
    double2 v = cmul(cmul(di, x), d_entry(c, m.U, jn));
    v = make_double2(w1 * (1.0 - w1) * v.x, w1 * (1.0 - w1) * v.y);
    if (j == ip) v = make_double2(v.x - w1 * di.x, v.y - w1 * di.y);
    const double2 ww = cmul(weight(c, i), weight(c, j));
    const double m2 = ww.x * ww.x + ww.y * ww.y;
    sigma[e] = cmul(v, make_double2(ww.x / m2, -ww.y / m2));
  }
}

// The training target X[a][b] = [W Sigma W + w1 D]_{a+1, b-1} / (w1 (1 - w1) d_{a+1} d_b), / scale.
__global__ void target_kernel(ContourDev c, ModelDev m, const double2* __restrict__ sigma, double inv_scale,
                              float* __restrict__ t) {
  const int n = c.n;
  const size_t total = (size_t)n * n;
  const double w1 = m.w1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / n), b = (int)(e % n);
    const int i = a + 1 == n ? 0 : a + 1, j = b == 0 ? n - 1 : b - 1;
    const double2 di = d_entry(c, m.U, i);
    double2 v = cmul(cmul(weight(c, i), sigma[(size_t)i * n + j]), weight(c, j));
    if (j == (i == 0 ? n - 1 : i - 1)) v = make_double2(v.x + w1 * di.x, v.y + w1 * di.y);
    const double2 den = cmul(di, d_entry(c, m.U, b));
    const double dm = w1 * (1.0 - w1) * (den.x * den.x + den.y * den.y);
    v = cmul(v, make_double2(den.x / dm, -den.y / dm));
    t[2 * e] = (float)(v.x * inv_scale);
    t[2 * e + 1] = (float)(v.y * inv_scale);
  }
}

// y <- y + lk * yk (n2 complex pairs of FP32): one term of the dt extrapolation.
__global__ void axpy_kernel(float* __restrict__ y, const float* __restrict__ yk, float lk, size_t n, bool first) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = (first ? 0.f : y[e]) + lk * yk[e];
}

int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

// activations for n samples: 4 hidden layers + output
size_t act_floats(int n) { return (size_t)n * (4 * kHid + kOut); }

}  // namespace
}  // namespace nedmft

using namespace nedmft;

extern "C" int32_t nedmft_mlp_param_count(void) { return (int32_t)kParams; }

extern "C" size_t nedmft_mlp_workspace_size(int32_t n) {
  if (n < 1) return 0;
  // activations + their gradients (2 x act) + loss partials + K-split sums
  return align256(sizeof(float) * act_floats(n)) * 2 + align256(sizeof(double) * 152 * 16) + align256(split_bytes());
}

extern "C" int nedmft_mlp_forward(const float* params_d, const float* x_d, int32_t n, float* y_d, void* ws_d,
                                  size_t ws_bytes, void* stream) {
  if (!params_d || !x_d || !y_d || !ws_d || n < 1) return set_error(NEDMFT_EINVAL, "mlp_forward: bad argument");
  if (ws_bytes < nedmft_mlp_workspace_size(n)) return set_error(NEDMFT_ENOMEM, "mlp_forward: workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* act = static_cast<float*>(ws_d);
  const float* in = x_d;
  for (int l = 0; l < kLayers; ++l) {
    const float* W = params_d + w_off(l);  // kDims[l] x kDims[l+1], row-major
    const float* b = W + (size_t)kDims[l] * kDims[l + 1];
    float* out = (l == kLayers - 1) ? y_d : act + (size_t)n * kHid * l;
    int rc = gemm<false, false>(in, W, b, out, n, kDims[l + 1], kDims[l], false, st);
    if (rc) return rc;
    if (l < kLayers - 1) {
      tanh_kernel<<<grid_for((size_t)n * kHid), 256, 0, st>>>(out, (size_t)n * kHid);
      NED_LAUNCH_CHECK("tanh_kernel");
    }
    in = out;
  }
  return NEDMFT_OK;
}

extern "C" int nedmft_mlp_grad(const float* params_d, const float* x_d, const float* target_d, int32_t n,
                               float* grad_d, float* loss_d, void* ws_d, size_t ws_bytes, void* stream) {
  if (!params_d || !x_d || !target_d || !grad_d || !loss_d || !ws_d || n < 1)
    return set_error(NEDMFT_EINVAL, "mlp_grad: bad argument");
  if (ws_bytes < nedmft_mlp_workspace_size(n)) return set_error(NEDMFT_ENOMEM, "mlp_grad: workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* p = static_cast<char*>(ws_d);
  float* act = reinterpret_cast<float*>(p);
  float* dact = reinterpret_cast<float*>(p + align256(sizeof(float) * act_floats(n)));
  double* part = reinterpret_cast<double*>(p + 2 * align256(sizeof(float) * act_floats(n)));
  float* ksplit = reinterpret_cast<float*>(p + 2 * align256(sizeof(float) * act_floats(n)) +
                                           align256(sizeof(double) * 152 * 16));
  float* H[kLayers];
  float* D[kLayers];
  for (int l = 0; l < kLayers; ++l) {
    H[l] = act + (size_t)n * kHid * l;
    D[l] = dact + (size_t)n * kHid * l;
  }
  // forward, keeping every activation (H[4] = output)
  const float* in = x_d;
  for (int l = 0; l < kLayers; ++l) {
    const float* W = params_d + w_off(l);
    const float* b = W + (size_t)kDims[l] * kDims[l + 1];
    int rc = gemm<false, false>(in, W, b, H[l], n, kDims[l + 1], kDims[l], false, st);
    if (rc) return rc;
    if (l < kLayers - 1) {
      tanh_kernel<<<grid_for((size_t)n * kHid), 256, 0, st>>>(H[l], (size_t)n * kHid);
      NED_LAUNCH_CHECK("tanh_kernel");
    }
    in = H[l];
  }
  const size_t no = (size_t)n * kOut;
  const int nbl = grid_for(no);
  mse_kernel<<<nbl, 256, 0, st>>>(H[kLayers - 1], target_d, D[kLayers - 1], no, 1.f / (float)no, part);
  NED_LAUNCH_CHECK("mse_kernel");
  loss_finish_kernel<<<1, 32, 0, st>>>(part, nbl, 1.0 / (double)no, loss_d);
  NED_LAUNCH_CHECK("loss_finish_kernel");
  for (int l = kLayers - 1; l >= 0; --l) {
    const float* W = params_d + w_off(l);
    float* gW = grad_d + w_off(l);
    float* gb = gW + (size_t)kDims[l] * kDims[l + 1];
    const float* xin = l == 0 ? x_d : H[l - 1];
    // dW = xin^T D[l], db = column sums of D[l]
    int rc = gemm<true, false>(xin, D[l], nullptr, gW, kDims[l], kDims[l + 1], n, false, st, ksplit);
    if (rc) return rc;
    bias_grad_kernel<<<ceil_div(kDims[l + 1], 128), 128, 0, st>>>(D[l], n, kDims[l + 1], gb);
    NED_LAUNCH_CHECK("bias_grad_kernel");
    if (l > 0) {
      // D[l-1] = (D[l] W^T) * tanh'(.)
      rc = gemm<false, true>(D[l], W, nullptr, D[l - 1], n, kDims[l], kDims[l + 1], false, st);
      if (rc) return rc;
      tanh_back_kernel<<<grid_for((size_t)n * kHid), 256, 0, st>>>(H[l - 1], D[l - 1], (size_t)n * kHid);
      NED_LAUNCH_CHECK("tanh_back_kernel");
    }
  }
  return NEDMFT_OK;
}

extern "C" int nedmft_mlp_adam(float* params_d, const float* grad_d, float* m1_d, float* m2_d, int32_t step, float lr,
                               void* stream) {
  if (!params_d || !grad_d || !m1_d || !m2_d || step < 1) return set_error(NEDMFT_EINVAL, "mlp_adam: bad argument");
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<grid_for(kParams), 256, 0, static_cast<cudaStream_t>(stream)>>>(params_d, grad_d, m1_d, m2_d, kParams,
                                                                                 lr, b1, b2, 1e-8f, c1, c2);
  NED_LAUNCH_CHECK("adam_kernel");
  return NEDMFT_OK;
}

extern "C" int nedmft_mlp_features(const nedmft_contour* c, const nedmft_model* m, float* x_d, void* stream) {
  if (!c || !m || !x_d || c->n_c < 1) return set_error(NEDMFT_EINVAL, "mlp_features: bad argument");
  const ContourDev cd = to_dev(*c);
  const ModelDev md{m->U, m->E, m->w1, isnan(m->mu) ? m->U / 2 : m->mu};
  features_kernel<<<grid_for((size_t)cd.n * cd.n), 256, 0, static_cast<cudaStream_t>(stream)>>>(cd, md, cd.dt, x_d);
  NED_LAUNCH_CHECK("features_kernel");
  return NEDMFT_OK;
}

extern "C" int nedmft_mlp_target(const nedmft_contour* c, const nedmft_model* m, const nedmft_c128* sigma_d,
                                 double scale, float* t_d, void* stream) {
  if (!c || !m || !sigma_d || !t_d || !(scale > 0)) return set_error(NEDMFT_EINVAL, "mlp_target: bad argument");
  const ContourDev cd = to_dev(*c);
  const ModelDev md{m->U, m->E, m->w1, isnan(m->mu) ? m->U / 2 : m->mu};
  target_kernel<<<grid_for((size_t)cd.n * cd.n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      cd, md, reinterpret_cast<const double2*>(sigma_d), 1.0 / scale, t_d);
  NED_LAUNCH_CHECK("target_kernel");
  return NEDMFT_OK;
}

extern "C" size_t nedmft_sigma_warm_start_workspace_size(const nedmft_contour* c) {
  if (!c || c->n_c < 1) return 0;
  const size_t n2 = (size_t)c->n_c * c->n_c;
  return align256(sizeof(float) * n2 * kIn) + 2 * align256(sizeof(float) * n2 * kOut) +
         nedmft_mlp_workspace_size((int32_t)(n2 > 65536 ? 65536 : n2));
}

extern "C" int nedmft_sigma_warm_start(const nedmft_contour* c, const nedmft_model* m, const float* params_d,
                                       int32_t n_dt, const double* dts_host, nedmft_c128* sigma_d, void* ws_d,
                                       size_t ws_bytes, void* stream) {
  if (!c || !m || !params_d || !sigma_d || !ws_d || !dts_host || n_dt < 1 || n_dt > 8)
    return set_error(NEDMFT_EINVAL, "sigma_warm_start: bad argument");
  if (!(m->U != 0.0) || !(m->w1 > 0.0 && m->w1 < 1.0))
    return set_error(NEDMFT_EINVAL, "sigma_warm_start: needs U != 0 and 0 < w1 < 1");
  for (int k = 0; k < n_dt; ++k)
    for (int q = 0; q < k; ++q)
      if (!(dts_host[k] > 0.0) || dts_host[k] == dts_host[q])
        return set_error(NEDMFT_EINVAL, "sigma_warm_start: steps must be positive and distinct");
  if (ws_bytes < nedmft_sigma_warm_start_workspace_size(c))
    return set_error(NEDMFT_ENOMEM, "sigma_warm_start: workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n2 = (size_t)c->n_c * c->n_c;
  char* p = static_cast<char*>(ws_d);
  float* x = reinterpret_cast<float*>(p);
  float* y = reinterpret_cast<float*>(p + align256(sizeof(float) * n2 * kIn));
  float* yk = reinterpret_cast<float*>(p + align256(sizeof(float) * n2 * kIn) + align256(sizeof(float) * n2 * kOut));
  char* mws = p + align256(sizeof(float) * n2 * kIn) + 2 * align256(sizeof(float) * n2 * kOut);
  const ContourDev cd = to_dev(*c);
  const ModelDev md{m->U, m->E, m->w1, isnan(m->mu) ? m->U / 2 : m->mu};
  for (int k = 0; k < n_dt; ++k) {
    // X at the step dts[k] on this contour's times, weighted by the Lagrange
    // basis polynomial of dts[k] at this contour's step (extrapolation in dt)
    double lk = 1.0;
    for (int q = 0; q < n_dt; ++q)
      if (q != k) lk *= (cd.dt - dts_host[q]) / (dts_host[k] - dts_host[q]);
    features_kernel<<<grid_for(n2), 256, 0, st>>>(cd, md, dts_host[k], x);
    NED_LAUNCH_CHECK("features_kernel");
    for (size_t s = 0; s < n2; s += 65536) {  // evaluate in chunks of 65536 pairs
      const int cnt = (int)((n2 - s) < 65536 ? (n2 - s) : 65536);
      int rc = nedmft_mlp_forward(params_d, x + s * kIn, cnt, yk + s * kOut, mws, nedmft_mlp_workspace_size(cnt),
                                  stream);
      if (rc) return rc;
    }
    axpy_kernel<<<grid_for(n2 * kOut), 256, 0, st>>>(y, yk, (float)lk, n2 * kOut, k == 0);
    NED_LAUNCH_CHECK("axpy_kernel");
  }
  assemble_sigma_kernel<<<grid_for(n2), 256, 0, st>>>(cd, md, y, reinterpret_cast<double2*>(sigma_d));
  NED_LAUNCH_CHECK("assemble_sigma_kernel");
  return NEDMFT_OK;
}

namespace nedmft {
namespace {
// x_b[r] = x[idx(r)], t_b[r] = t[idx(r)], idx from a counter-based hash of
// (seed, step, r) (splitmix64 finaliser) modulo n_total.
__global__ void sample_kernel(const float* __restrict__ x, const float* __restrict__ t, long long n_total, int batch,
                              unsigned long long seed, long long step, float* __restrict__ xb, float* __restrict__ tb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= batch) return;
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(step * (long long)batch + r + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const long long i = (long long)(z % (unsigned long long)n_total);
  for (int f = 0; f < kIn; ++f) xb[(size_t)r * kIn + f] = x[(size_t)i * kIn + f];
  for (int f = 0; f < kOut; ++f) tb[(size_t)r * kOut + f] = t[(size_t)i * kOut + f];
}
}  // namespace
}  // namespace nedmft

extern "C" int nedmft_mlp_sample(const float* x_d, const float* t_d, int64_t n_total, int32_t batch, uint64_t seed,
                                 int64_t step, float* xb_d, float* tb_d, void* stream) {
  if (!x_d || !t_d || !xb_d || !tb_d || n_total < 1 || batch < 1)
    return set_error(NEDMFT_EINVAL, "mlp_sample: bad argument");
  sample_kernel<<<ceil_div(batch, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x_d, t_d, n_total, batch, seed,
                                                                                      step, xb_d, tb_d);
  NED_LAUNCH_CHECK("sample_kernel");
  return NEDMFT_OK;
}
