// CUDA-core kernels of the lattice step: S = W Sigma W, the fused B_q - S
// generator, the dense G0 builder, Gauss-Jordan inversion (single-CTA for
// small N_c, blocked and batched for large N_c), the refinement residual and
// the FP64 quadrature / current reductions.
#include "lattice.cuh"

namespace nedmft {

// ------------------------------------------------------------------ S = W Sigma W

__global__ void build_s_kernel(ContourDev c, const double2* __restrict__ sigma, double2* __restrict__ S) {
  size_t total = (size_t)c.n * c.n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / c.n), j = (int)(e % c.n);
    S[e] = cmul(cmul(weight(c, i), sigma[e]), weight(c, j));
  }
}

int launch_build_s(const ContourDev& c, const double2* sigma, double2* S, cudaStream_t st) {
  size_t total = (size_t)c.n * c.n;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  build_s_kernel<<<blocks, 256, 0, st>>>(c, sigma, S);
  NED_LAUNCH_CHECK("build_s_kernel");
  return NEDMFT_OK;
}

// ------------------------------------------------------------------ G0 (dense)

// G0(t_i, t_j) of Eq. g_contour_non_final2 in the log-stable form:
//   i >= j: -i exp(-x (tau_i - tau_j) - softplus(-beta x)) e^{i phase},
//   i <  j:  i exp(-x (tau_i - tau_j) - softplus( beta x)) e^{i phase},
// phase = mu Re(t_i - t_j) - [F(t_i) - F(t_j)].
__global__ void g0_build_kernel(ContourDev c, ModelDev m, const double* __restrict__ eps_d,
                                const double* __restrict__ ebar_d, double2* __restrict__ g0) {
  const int q = blockIdx.y;
  const double eps = eps_d[q], ebar = ebar_d[q];
  const double x = eps - m.mu;
  const double sp_neg = x > 0 ? log1p(exp(-c.beta * x)) : -c.beta * x + log1p(exp(c.beta * x));   // softplus(-beta x)
  const double sp_pos = x > 0 ? c.beta * x + log1p(exp(-c.beta * x)) : log1p(exp(c.beta * x));    // softplus(beta x)
  size_t total = (size_t)c.n * c.n;
  double2* out = g0 + (size_t)q * total;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / c.n), j = (int)(e % c.n);
    double si = t_re(c, i), sj = t_re(c, j);
    double ph = m.mu * (si - sj) - band_phase_diff(sj, si, eps, ebar, m.E);
    double re = -x * (t_tau(c, i) - t_tau(c, j));
    double sn, cs;
    sincos(ph, &sn, &cs);
    double mag, pre;
    if (i >= j) { mag = exp(re - sp_neg); pre = -1.0; } else { mag = exp(re - sp_pos); pre = 1.0; }
    // pre * i * mag * (cs + i sn) = pre * mag * (-sn + i cs)
    out[e] = make_double2(-pre * mag * sn, pre * mag * cs);
  }
}

int launch_g0_build(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar, int nq,
                    double2* g0, cudaStream_t st) {
  size_t total = (size_t)c.n * c.n;
  int bx = (int)((total + 255) / 256);
  if (bx > 1024) bx = 1024;
  dim3 grid(bx, nq);
  g0_build_kernel<<<grid, 256, 0, st>>>(c, m, eps, ebar, g0);
  NED_LAUNCH_CHECK("g0_build_kernel");
  return NEDMFT_OK;
}

// ------------------------------------------------------------------ A'_q = P (B_q - S), padded

template <class T>
__global__ void gen_a_kernel(ContourDev c, ModelDev m, const double* __restrict__ eps_d,
                             const double* __restrict__ ebar_d, int q0, const double2* __restrict__ S,
                             cplx_t<T>* __restrict__ A, int np) {
  const int b = blockIdx.y;
  const double eps = eps_d[q0 + b], ebar = ebar_d[q0 + b];
  const bool sh = shifted_point(m, eps);
  const size_t total = (size_t)np * np;
  cplx_t<T>* out = A + (size_t)b * total;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(e / np), col = (int)(e % np);
    double2 v;
    if (r < c.n && col < c.n) {
      int i = sh ? (r + 1 == c.n ? 0 : r + 1) : r;
      v = a_entry(c, m, eps, ebar, S, i, col);
    } else {
      v = make_double2(r == col ? 1.0 : 0.0, 0.0);
    }
    out[e] = cvt<T>(v);
  }
}

template <class T>
int launch_gen_a(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar, int q0, int nb,
                 const double2* S, cplx_t<T>* A, int np, cudaStream_t st) {
  size_t total = (size_t)np * np;
  int bx = (int)((total + 255) / 256);
  if (bx > 4096) bx = 4096;
  dim3 grid(bx, nb);
  gen_a_kernel<T><<<grid, 256, 0, st>>>(c, m, eps, ebar, q0, S, A, np);
  NED_LAUNCH_CHECK("gen_a_kernel");
  return NEDMFT_OK;
}
template int launch_gen_a<double>(const ContourDev&, const ModelDev&, const double*, const double*, int, int,
                                  const double2*, double2*, int, cudaStream_t);

// ------------------------------------------------------------------ record a device failure

__device__ __forceinline__ void record_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ in-shared-memory Gauss-Jordan

// In-place inverse of the n x n matrix `a` (row stride ld) held in shared
// memory, no pivoting (the static row order makes the pivots safe), all
// threads of the block participating.  `col` is n scratch entries.
template <class T>
__device__ void smem_gauss_jordan(cplx_t<T>* a, int n, int ld, cplx_t<T>* col, T tiny, int* status) {
  using C = cplx_t<T>;
  for (int k = 0; k < n; ++k) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) col[t] = a[t * ld + k];
    __syncthreads();
    C pinv;
    bool ok = cinv_guard<T>(col[k], pinv, tiny);
    if (!ok && threadIdx.x == 0) record_status(status, DS_SINGULAR);
    for (int t = threadIdx.x; t < n; t += blockDim.x) a[k * ld + t] = (t == k) ? pinv : cmul(a[k * ld + t], pinv);
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int i = e / n, j = e % n;
      if (i == k) continue;
      C f = col[i];
      if (j == k) {
        C v = cmul(f, pinv);
        a[i * ld + k] = mk<T>(-v.x, -v.y);
      } else {
        C v = a[i * ld + j];
        C r = a[k * ld + j];
        v.x -= f.x * r.x - f.y * r.y;
        v.y -= f.x * r.y + f.y * r.x;
        a[i * ld + j] = v;
      }
    }
    __syncthreads();
  }
}

// Small N_c: one CTA per point generates A'_q in shared memory, inverts it
// and writes G_q (columns un-cycled) in FP64 to out[b].
__global__ void __launch_bounds__(512) gj_small_fp64_kernel(ContourDev c, ModelDev m, const double* __restrict__ eps_d,
                                                            const double* __restrict__ ebar_d, int q0,
                                                            const double2* __restrict__ S, double2* __restrict__ out,
                                                            int* status) {
  extern __shared__ double2 sm[];
  const int n = c.n, b = blockIdx.x;
  double2* a = sm;
  double2* col = sm + n * n;
  const double eps = eps_d[q0 + b], ebar = ebar_d[q0 + b];
  const bool sh = shifted_point(m, eps);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int r = e / n, j = e % n;
    int i = sh ? (r + 1 == n ? 0 : r + 1) : r;
    a[e] = a_entry(c, m, eps, ebar, S, i, j);
  }
  __syncthreads();
  smem_gauss_jordan<double>(a, n, n, col, 1e-12, status);
  double2* o = out + (size_t)b * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e % n;
    o[e] = a[i * n + unshift_col(j, n, sh)];
  }
}

int small_path_max_n() { return kSmallPathMaxN; }

int launch_gj_small_fp64(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar, int q0,
                         int nb, const double2* S, double2* out, int* status, cudaStream_t st) {
  size_t smem = (size_t)(c.n * c.n + c.n) * sizeof(double2);
  int rc = ensure_dyn_smem(reinterpret_cast<const void*>(gj_small_fp64_kernel), 227 * 1024);
  if (rc) return rc;
  gj_small_fp64_kernel<<<nb, 512, smem, st>>>(c, m, eps, ebar, q0, S, out, status);
  NED_LAUNCH_CHECK("gj_small_fp64_kernel");
  return NEDMFT_OK;
}

// ------------------------------------------------------------------ blocked Gauss-Jordan, CUDA cores

// Step k of blocked Gauss-Jordan on A (np x np, batch stride np*np):
//   P = inv(A_KK)                                        gj_pivot32_fp64_kernel
//   R = P A_{K,:} with R_{:,K} = P;  C = A_{:,K} with C_K = -I   gj_panels_kernel
//   A <- A(with rows K and columns K zeroed) - C R       gj_update_kernel
// P = inv(A_KK) for the 32 x 32 FP64 block at (k0, k0) of every matrix, on a
// cluster of kPivCtas CTAs per matrix: CTA q holds rows 4q .. 4q+3, one warp
// per row, lane j its column j in registers, so the FP64 work of a step
// spreads over eight SMs (GB300 has two FP64 FMA units per SM).  Each step
// the warp of the next pivot row writes that row, and its lane on the
// diagonal the pivot's inverse, into every CTA's double-buffered shared
// arrays (written for step k + 1 while step k's are still being read), then
// one cluster barrier per step.  A row's entry in the pivot column is its own
// lane's value (a shuffle).  No pivoting: the caller orders the rows.  Row r
// of the block is matrix row rows[r] when `rows` is given and rows[r] >= 0
// (the pivot rows of a step before they are swapped into place), else k0 + r.
constexpr int kPivCtas = 8;
__device__ __forceinline__ void piv_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t piv_cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// store v at shared variable p of CTA `rank` of the cluster
__device__ __forceinline__ void piv_st_remote(const double2* p, uint32_t rank, double2 v) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(a)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}
__global__ void __cluster_dims__(kPivCtas, 1, 1) __launch_bounds__(128)
    gj_pivot32_fp64_kernel(const double2* __restrict__ A, int np, int k0, const int* __restrict__ rows,
                           double2* __restrict__ Pbuf, int* status) {
  __shared__ __align__(16) double2 rowb[2][32];
  __shared__ __align__(16) double2 pinvb[2];
  const int b = blockIdx.x / kPivCtas;  // the matrix; clusters are consecutive CTAs
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = 4 * (int)piv_cluster_rank() + warp;
  const int src = (rows && rows[r] >= 0) ? rows[r] : k0 + r;
  double2 v = A[(size_t)b * np * np + (size_t)src * np + k0 + lane];
  // step k's pivot row (warp-uniform branch) to every CTA
  auto publish = [&](int k, int buf) {
    if (r != k) return;
    double2 pinv = make_double2(0.0, 0.0);
    if (lane == k && !cinv_guard<double>(v, pinv, 1e-12) && status) atomicCAS(status, 0, DS_SINGULAR);
    for (uint32_t d = 0; d < (uint32_t)kPivCtas; ++d) {
      piv_st_remote(&rowb[buf][lane], d, v);
      if (lane == k) piv_st_remote(&pinvb[buf], d, pinv);
    }
  };
  piv_cluster_sync();  // every CTA of the cluster runs before another writes its shared memory
  publish(0, 0);
  piv_cluster_sync();
  for (int k = 0; k < 32; ++k) {
    const int buf = k & 1;
    const double2 pinv = pinvb[buf];
    if (r == k) {
      v = (lane == k) ? pinv : cmul(v, pinv);
    } else {
      const double2 rb = rowb[buf][lane];
      const double2 ck = make_double2(__shfl_sync(0xffffffffu, v.x, k), __shfl_sync(0xffffffffu, v.y, k));
      const double2 g = cmul(ck, pinv);  // a_rk / a_kk
      // v - g rb in four FMAs
      const double2 nv = make_double2(fma(-g.x, rb.x, fma(g.y, rb.y, v.x)), fma(-g.x, rb.y, fma(-g.y, rb.x, v.y)));
      v = (lane == k) ? make_double2(-g.x, -g.y) : nv;
    }
    if (k + 1 < 32) publish(k + 1, buf ^ 1);
    piv_cluster_sync();
  }
  Pbuf[(size_t)b * 32 * 32 + (size_t)r * 32 + lane] = v;
}

// W columns of R and W rows of C per CTA (W = 8 for one matrix: 4 x more
// CTAs than W = 32 on the same work).
template <class T, int NB, int W = 32>
__global__ void __launch_bounds__(256) gj_panels_kernel(const cplx_t<T>* __restrict__ A, int np, int k0,
                                                        const cplx_t<T>* __restrict__ Pbuf,
                                                        cplx_t<T>* __restrict__ Rbuf, cplx_t<T>* __restrict__ Cbuf) {
  using C = cplx_t<T>;
  __shared__ C ps[NB][NB + 1];
  __shared__ C as[NB][W + 1];
  const int b = blockIdx.y;
  const int j0 = blockIdx.x * W;
  const C* a = A + (size_t)b * np * np;
  const C* P = Pbuf + (size_t)b * NB * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) ps[e / NB][e % NB] = P[e];
  for (int e = threadIdx.x; e < NB * W; e += blockDim.x) {
    int r = e / W, cc = e % W;
    as[r][cc] = a[(size_t)(k0 + r) * np + j0 + cc];
  }
  __syncthreads();
  C* R = Rbuf + (size_t)b * NB * np;
  for (int e = threadIdx.x; e < NB * W; e += blockDim.x) {
    int r = e / W, cc = e % W;
    int j = j0 + cc;
    C acc;
    if (j >= k0 && j < k0 + NB) {
      acc = ps[r][j - k0];
    } else {
      acc = mk<T>(0, 0);
      for (int kk = 0; kk < NB; ++kk) cfma(acc, ps[r][kk], as[kk][cc]);
    }
    R[(size_t)r * np + j] = acc;
  }
  // C rows j0 .. j0+W-1
  C* Cb = Cbuf + (size_t)b * np * NB;
  for (int e = threadIdx.x; e < W * NB; e += blockDim.x) {
    int i = j0 + e / NB, kk = e % NB;
    C v;
    if (i >= k0 && i < k0 + NB) v = mk<T>(i - k0 == kk ? T(-1) : T(0), 0);
    else v = a[(size_t)i * np + k0 + kk];
    Cb[(size_t)i * NB + kk] = v;
  }
}

// 64 x 64 output tile per CTA; each thread 4 rows x kUpdRN columns.  The
// complex products use three real products (the 3M form): for a = ax + i ay,
// b = bx + i by,  Re(ab) = ax bx - ay by  and  Im(ab) = (ax + ay)(bx + by) -
// ax bx - ay by.  The three real sums over the 32 k run apart and combine at
// the end: 3 FMAs per complex multiply-add instead of 4.  The sums ax + ay of
// the C panel and bx + by of the R panel are formed once, in shared memory.
// The CTA columns start at tile jt0.  Column j is written iff (wlo <= j <
// whi) == inside: (0, 0, false) writes every column, (lo, hi, false) all but
// a window that another kernel updates.
constexpr int kUpdRN = 4;
constexpr int kUpdThreads = 16 * (64 / kUpdRN);
template <int NB>
constexpr size_t upd_smem_bytes() {  // C panel and R panel tiles with their x + y sums
  return (size_t)64 * (NB + 1) * 24 + (size_t)NB * 64 * 24;
}

template <int NB>
__global__ void __launch_bounds__(kUpdThreads, 1) gj_update_kernel(double2* __restrict__ A, int np, int k0,
                                                                   const double2* __restrict__ Rbuf,
                                                                   const double2* __restrict__ Cbuf, int jt0,
                                                                   int wlo, int whi, bool inside) {
  constexpr int TM = 64, TN = 64, RN = kUpdRN, CX = TN / RN;
  extern __shared__ __align__(16) unsigned char smraw[];
  double2 (*cz)[NB + 1] = reinterpret_cast<double2 (*)[NB + 1]>(smraw);
  double2 (*rz)[TN] = reinterpret_cast<double2 (*)[TN]>(smraw + sizeof(double2) * TM * (NB + 1));
  double (*csum)[NB + 1] =
      reinterpret_cast<double (*)[NB + 1]>(smraw + sizeof(double2) * (TM * (NB + 1) + NB * TN));
  double (*rsum)[TN] = reinterpret_cast<double (*)[TN]>(smraw + sizeof(double2) * (TM * (NB + 1) + NB * TN) +
                                                        sizeof(double) * TM * (NB + 1));
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * TM, j0 = (jt0 + blockIdx.x) * TN;
  const double2* Cb = Cbuf + (size_t)b * np * NB;
  const double2* R = Rbuf + (size_t)b * NB * np;
  for (int e = threadIdx.x; e < TM * NB; e += kUpdThreads) {
    const double2 v = Cb[(size_t)(i0 + e / NB) * NB + e % NB];
    cz[e / NB][e % NB] = v;
    csum[e / NB][e % NB] = v.x + v.y;
  }
  for (int e = threadIdx.x; e < NB * TN; e += kUpdThreads) {
    const double2 v = R[(size_t)(e / TN) * np + j0 + e % TN];
    rz[e / TN][e % TN] = v;
    rsum[e / TN][e % TN] = v.x + v.y;
  }
  __syncthreads();
  const int tx = threadIdx.x % CX, ty = threadIdx.x / CX;
  double pp[4][RN], mm[4][RN], ss[4][RN];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < RN; ++q) pp[r][q] = mm[r][q] = ss[r][q] = 0.0;
#pragma unroll 2
  for (int kk = 0; kk < NB; ++kk) {
    double2 av[4], bv[RN];
    double as[4], bs[RN];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      av[r] = cz[ty + 16 * r][kk];
      as[r] = csum[ty + 16 * r][kk];
    }
#pragma unroll
    for (int q = 0; q < RN; ++q) {
      bv[q] = rz[kk][tx + CX * q];
      bs[q] = rsum[kk][tx + CX * q];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < RN; ++q) {
        pp[r][q] = fma(av[r].x, bv[q].x, pp[r][q]);
        mm[r][q] = fma(av[r].y, bv[q].y, mm[r][q]);
        ss[r][q] = fma(as[r], bs[q], ss[r][q]);
      }
  }
  double2* a = A + (size_t)b * np * np;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    const bool ik = (i >= k0 && i < k0 + NB);
#pragma unroll
    for (int q = 0; q < RN; ++q) {
      const int j = j0 + tx + CX * q;
      if ((j >= wlo && j < whi) != inside) continue;
      const bool jk = (j >= k0 && j < k0 + NB);
      const double2 old = (ik || jk) ? make_double2(0.0, 0.0) : a[(size_t)i * np + j];
      a[(size_t)i * np + j] = make_double2(old.x - (pp[r][q] - mm[r][q]), old.y - (ss[r][q] - pp[r][q] - mm[r][q]));
    }
  }
}

// The update of one 32-column window [w0, w0 + 32) (the next step's panel)
// on every row, in 8-row slices: 8 x 32 outputs per CTA of 64 threads, so
// the window's few flops spread over many SMs.
template <int NB>
__global__ void __launch_bounds__(64) gj_update_window_kernel(double2* __restrict__ A, int np, int k0, int w0,
                                                              const double2* __restrict__ Rbuf,
                                                              const double2* __restrict__ Cbuf) {
  __shared__ double2 cs[8][NB + 1];
  __shared__ double2 rs[NB][32];
  const int i0 = blockIdx.x * 8, t = threadIdx.x;
  for (int e = t; e < 8 * NB; e += 64) cs[e / NB][e % NB] = Cbuf[(size_t)(i0 + e / NB) * NB + e % NB];
  for (int e = t; e < NB * 32; e += 64) rs[e / 32][e % 32] = Rbuf[(size_t)(e / 32) * np + w0 + e % 32];
  __syncthreads();
  const int r = t >> 3, c0 = 4 * (t & 7);
  double2 acc[4] = {};
#pragma unroll 8
  for (int kk = 0; kk < NB; ++kk) {
    const double2 a = cs[r][kk];
#pragma unroll
    for (int u = 0; u < 4; ++u) cfma(acc[u], a, rs[kk][c0 + u]);
  }
  const int i = i0 + r;
  const bool ik = i >= k0 && i < k0 + NB;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = w0 + c0 + u;
    const bool jk = j >= k0 && j < k0 + NB;
    double2* a = A + (size_t)i * np + j;
    *a = csub((ik || jk) ? make_double2(0.0, 0.0) : *a, acc[u]);
  }
}

template <class T>
int gj_blocked_simt(cplx_t<T>* A, int n, int np, int nb_batch, cplx_t<T>* Pbuf, cplx_t<T>* Rbuf, cplx_t<T>* Cbuf,
                    int* status, cudaStream_t st) {
  constexpr int NB = 32;
  if (np % 64 != 0) return set_error(NEDMFT_EINVAL, "gj_blocked_simt: np=%d not a multiple of 64", np);
  const size_t smem = upd_smem_bytes<NB>();
  if (int rc = ensure_dyn_smem(reinterpret_cast<const void*>(gj_update_kernel<NB>), (int)smem)) return rc;
  for (int k0 = 0; k0 < np; k0 += NB) {
    static_assert(NB == 32, "the pivot-block kernel inverts 32 x 32 blocks");
    gj_pivot32_fp64_kernel<<<nb_batch * kPivCtas, 128, 0, st>>>(A, np, k0, nullptr, Pbuf, status);
    NED_LAUNCH_CHECK("gj_pivot32_fp64_kernel");
    gj_panels_kernel<T, NB><<<dim3(np / 32, nb_batch), 256, 0, st>>>(A, np, k0, Pbuf, Rbuf, Cbuf);
    NED_LAUNCH_CHECK("gj_panels_kernel");
    const int slot = instr_begin(st);
    gj_update_kernel<NB><<<dim3(np / 64, np / 64, nb_batch), kUpdThreads, smem, st>>>(A, np, k0, Rbuf, Cbuf, 0, 0, 0,
                                                                                 false);
    NED_LAUNCH_CHECK("gj_update_kernel");
    const int live = n - k0 < NB ? (n - k0 > 0 ? n - k0 : 0) : NB;
    instr_end(slot, st, 8.0 * (double)n * n * live * nb_batch,
              live > 0 ? 2.0 * sizeof(cplx_t<T>) * (double)n * n * nb_batch : 0.0);
  }
  return NEDMFT_OK;
}
template int gj_blocked_simt<double>(double2*, int, int, int, double2*, double2*, double2*, int*, cudaStream_t);

// ------------------------------------------------------------------ FP64 inversion with partial pivoting

// Blocked Gauss-Jordan with partial pivoting for one dense matrix (the
// impurity step).  Before each 32-column step the pivot rows of the block are
// chosen by a tournament (as in communication-avoiding LU): chunks of
// kTourRows candidate rows each run partial-pivoting LU on their part of the
// block's columns and pass the 32 rows they pivot on to the next round, until
// one chunk is left, whose pivot order is the block's.  The choice only
// decides which rows to swap in; it runs in FP32 (a pivot need only be close
// to the largest).  The rows are swapped in the FP64 matrix and the step
// itself is the unpivoted blocked Gauss-Jordan step above.  The column
// permutation of the result is undone at the end.
constexpr int kTourRows = 256;
constexpr int kTourNB = 32;

// One tournament round.  Block c takes candidates c*kTourRows .. +kTourRows-1
// (rows k0 + i of the matrix when `in` is NULL, else in[i]; -1 = no row) and
// writes the <= 32 rows it pivots on (in pivot order, -1 padded) to
// out[c*32 ..].  With final != 0 (one block) it turns the winners into the
// swap sequence piv[k0 .. k0+31] (position k0 + j swaps with piv[k0 + j]),
// and the same swaps as one gather of the <= 64 rows they move: gather[0] =
// count, then pairs (position, row now at that position before the swaps).
//
// Thread t keeps candidate t's 32 panel entries in registers (the step loop
// is unrolled, so every entry index is a constant).  Step j: the largest
// |entry| of column j among the rows not yet chosen (ties: lower candidate
// index) by a shuffle argmax per warp and a scan over the warps; the chosen
// row's thread marks itself and puts its entries j .. 31 in shared memory;
// every other row eliminates column j with it.  Rows do not move, so two
// barriers per step; the winners are recorded in pivot order.
__global__ void __launch_bounds__(kTourRows) tour_kernel(const double2* __restrict__ A, int np, int n, int k0,
                                                         const int* __restrict__ in, int in_count,
                                                         int* __restrict__ out, int final_round,
                                                         int* __restrict__ piv, int* __restrict__ gather,
                                                         int* status) {
  constexpr int kWarps = kTourRows / 32;
  __shared__ float2 prow[2][kTourNB];     // the pivot row of a step (double-buffered by step)
  __shared__ float wv[2][kWarps];         // per-warp maxima (double-buffered by step)
  __shared__ int wi[2][kWarps];
  __shared__ int win[kTourNB];            // the winners' rows, in pivot order (-1: none)
  const int c = blockIdx.x, t = threadIdx.x, lane = t & 31;
  const int i = c * kTourRows + t;
  const int nrows = min(kTourRows, in_count - c * kTourRows);
  int row = -1;
  if (i < in_count) row = in ? in[i] : k0 + i;
  const int ncol = min(kTourNB, n - k0);
  float2 v[kTourNB];
#pragma unroll
  for (int j = 0; j < kTourNB; ++j) {
    v[j] = make_float2(0.f, 0.f);
    if (row >= 0 && j < ncol) {
      const double2 z = A[(size_t)row * np + k0 + j];
      v[j] = make_float2((float)z.x, (float)z.y);
    }
  }
  bool live = row >= 0 && t < nrows;  // a candidate not chosen yet
  const int steps = min(ncol, nrows);
#pragma unroll
  for (int j = 0; j < kTourNB; ++j) {
    if (j < steps) {  // uniform over the block
      const int sb = j & 1;
      float m = live ? v[j].x * v[j].x + v[j].y * v[j].y : -1.f;
      int idx = t;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float om = __shfl_xor_sync(0xffffffffu, m, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (om > m || (om == m && oi < idx)) {
          m = om;
          idx = oi;
        }
      }
      if (lane == 0) {
        wv[sb][t >> 5] = m;
        wi[sb][t >> 5] = idx;
      }
      __syncthreads();
      float bm = wv[sb][0];
      int p = wi[sb][0];
#pragma unroll
      for (int w = 1; w < kWarps; ++w)
        if (wv[sb][w] > bm || (wv[sb][w] == bm && wi[sb][w] < p)) {
          bm = wv[sb][w];
          p = wi[sb][w];
        }
      if (bm < 0.f) p = -1;  // no candidate left (not reached: a round has >= steps rows)
      if (t == p) {
        live = false;
        win[j] = row;
#pragma unroll
        for (int cc = j; cc < kTourNB; ++cc) prow[sb][cc] = v[cc];
      } else if (p < 0 && t == 0) {
        win[j] = -1;
      }
      __syncthreads();
      if (p >= 0 && live) {
        const float2 pv = prow[sb][j];
        const float pm = pv.x * pv.x + pv.y * pv.y;
        if (pm > 0.f) {
          const float2 pinv = make_float2(pv.x / pm, -pv.y / pm);
          const float2 a = v[j];
          const float2 f = make_float2(a.x * pinv.x - a.y * pinv.y, a.x * pinv.y + a.y * pinv.x);
#pragma unroll
          for (int cc = j + 1; cc < kTourNB; ++cc) {
            const float2 r = prow[sb][cc];
            v[cc].x -= f.x * r.x - f.y * r.y;
            v[cc].y -= f.x * r.y + f.y * r.x;
          }
        }
      }
    }
  }
  __syncthreads();
  if (t < kTourNB) out[c * kTourNB + t] = (t < steps) ? win[t] : -1;
  if (final_round) {
    // winners -> swap sequence: position k0 + j takes the row now at the
    // winner's position.  The positions and rows involved (<= 64) get slots:
    // slot j < 32 for position k0 + j, slot 32 + j for winner j when it lies
    // outside the block; row_at[slot] / where[slot] track which row sits at a
    // position and where a row sits, so every swap is O(1)
    __shared__ int row_at[2 * kTourNB], where_at[2 * kTourNB];
    if (t < 2 * kTourNB) row_at[t] = where_at[t] = t;
    __syncthreads();
    if (t == 0) {
      auto value = [&](int sl) { return sl < kTourNB ? k0 + sl : win[sl - kTourNB]; };
      for (int j = 0; j < kTourNB && k0 + j < n; ++j) {
        const int w = j < steps ? win[j] : -1;
        int target = k0 + j, tsl = j;
        if (w >= 0) {
          const int wsl = (w >= k0 && w < k0 + kTourNB) ? w - k0 : kTourNB + j;
          tsl = where_at[wsl];
          target = value(tsl);
        } else if (status) {
          atomicCAS(status, 0, DS_SINGULAR);  // fewer nonzero candidates than columns
        }
        piv[k0 + j] = target;
        if (tsl != j) {
          const int ra = row_at[j], rb = row_at[tsl];
          row_at[j] = rb;
          row_at[tsl] = ra;
          where_at[ra] = tsl;
          where_at[rb] = j;
        }
      }
      if (gather) {
        int cnt = 0;
        for (int sl = 0; sl < 2 * kTourNB; ++sl)
          if (row_at[sl] != sl) {
            gather[1 + 2 * cnt] = value(sl);
            gather[2 + 2 * cnt] = value(row_at[sl]);
            ++cnt;
          }
        gather[0] = cnt;
      }
    }
  }
}

// The swaps of one step as a gather: 32 columns per CTA, the moved rows'
// values staged in shared memory, then written to their new positions.
__global__ void __launch_bounds__(256) apply_gather_kernel(double2* __restrict__ A, int np,
                                                           const int* __restrict__ gather) {
  __shared__ double2 buf[2 * kTourNB][32];
  const int cnt = gather[0];
  const int col0 = blockIdx.x * 32;
  for (int e = threadIdx.x; e < cnt * 32; e += blockDim.x) {
    const int u = e >> 5, c = e & 31;
    buf[u][c] = A[(size_t)gather[2 + 2 * u] * np + col0 + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < cnt * 32; e += blockDim.x) {
    const int u = e >> 5, c = e & 31;
    A[(size_t)gather[1 + 2 * u] * np + col0 + c] = buf[u][c];
  }
}

// The inversion works on A 2^-e, e the exponent of max |Re|, |Im| over A
// (exact scaling): its pivot thresholds are then relative and the FP32 pivot
// choice stays in range.  amax holds the bits of that maximum (non-negative
// doubles order like their bit patterns), set by amax_kernel after a clear.
__device__ __forceinline__ int amax_exponent(const unsigned long long* amax) {
  const double m = __longlong_as_double((long long)*amax);
  int e = 0;
  if (m > 0.0 && m <= 1.7976931348623157e308) frexp(m, &e);
  return e;
}

__global__ void amax_kernel(const double2* __restrict__ a, size_t total, unsigned long long* __restrict__ amax) {
  double m = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double2 z = a[e];
    m = fmax(m, fmax(fabs(z.x), fabs(z.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, (unsigned long long)__double_as_longlong(m));
}

__global__ void pad_identity_kernel(const double2* __restrict__ a, int n, double2* __restrict__ ap, int np,
                                    const unsigned long long* __restrict__ amax) {
  const int sh = -amax_exponent(amax);
  const size_t total = (size_t)np * np;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / np), j = (int)(e % np);
    if (i < n && j < n) {
      const double2 z = a[(size_t)i * n + j];
      ap[e] = make_double2(ldexp(z.x, sh), ldexp(z.y, sh));
    } else {
      ap[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
  }
}

// inv[idx] = j such that column j of A^-1 is column idx of the in-place result
// of the swapped matrix (the swaps applied in order).
__global__ void swap_colmap_kernel(int n, const int* __restrict__ piv, int* __restrict__ inv) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int j = 0; j < n; ++j) inv[j] = j;
  for (int k = 0; k < n; ++k) {
    const int p = piv[k];
    const int t = inv[k];
    inv[k] = inv[p];
    inv[p] = t;
  }
}

// y = the inverse of A: the columns put back in order and the scale undone
// (inv(A 2^-e) = 2^e inv(A))
__global__ void unpermute_kernel(const double2* __restrict__ x, int np, int n, const int* __restrict__ inv,
                                 double2* __restrict__ y, const unsigned long long* __restrict__ amax) {
  const int sh = -amax_exponent(amax);
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), c = (int)(e % n);
    const double2 z = x[(size_t)i * np + c];
    y[(size_t)i * n + inv[c]] = make_double2(ldexp(z.x, sh), ldexp(z.y, sh));
  }
}

size_t pivot_inverse_workspace(int n) {
  const int np = ((n + 127) / 128) * 128;
  const int nchunk = (n + kTourRows - 1) / kTourRows;
  return align256(sizeof(double2) * (size_t)np * np) + align256(sizeof(double2) * kTourNB * kTourNB) +
         2 * align256(sizeof(double2) * (size_t)kTourNB * np) + 2 * align256(sizeof(int) * (size_t)nchunk * kTourNB) +
         2 * align256(sizeof(int) * (size_t)n) + align256(sizeof(int) * (1 + 4 * kTourNB)) + align256(8) +
         oz64_workspace(np);
}

// Second stream (highest priority) and two events per device and host
// thread for the look-ahead below, created on first use and kept.
struct LookAhead {
  cudaStream_t side = nullptr;
  cudaEvent_t panel = nullptr, chain = nullptr;
};

int look_ahead(LookAhead** out) {
  constexpr int kMaxDev = 64;
  thread_local LookAhead la[kMaxDev];
  int dev = 0;
  NED_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return set_error(NEDMFT_ECUDA, "pivot_inverse: device %d out of range", dev);
  LookAhead& l = la[dev];
  if (!l.side) {
    int lo = 0, hi = 0;
    NED_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    NED_CUDA(cudaEventCreateWithFlags(&l.panel, cudaEventDisableTiming));
    NED_CUDA(cudaEventCreateWithFlags(&l.chain, cudaEventDisableTiming));
    NED_CUDA(cudaStreamCreateWithPriority(&l.side, cudaStreamNonBlocking, hi));
  }
  *out = &l;
  return NEDMFT_OK;
}

// Creates this host thread's look-ahead stream and events on the current
// device and sets the kernels' shared-memory limits: for callers that are
// about to capture pivot_inverse into a CUDA graph.
int pivot_inverse_prepare() {
  LookAhead* la = nullptr;
  int rc = look_ahead(&la);
  if (!rc) rc = oz64_prepare();
  return rc;
}

// Every step's pivot choice (the tournament) and pivot-block inverse depend
// only on the step's 32 panel columns, so they run one step ahead, on the
// second stream: there step k updates the next step's panel columns, then
// the tournament and the 32 x 32 inverse of step k + 1 run, while step k
// updates the rest of the matrix on the caller's stream.  The swaps of step
// k + 1 wait for both.
int pivot_inverse(double2* a, int n, void* ws, cudaStream_t st, int* status) {
  constexpr int NB = kTourNB;
  const int np = ((n + 127) / 128) * 128;  // 128-row tiles of the tensor-core update
  const int nchunk = (n + kTourRows - 1) / kTourRows;
  char* p = static_cast<char*>(ws);
  double2* ap = reinterpret_cast<double2*>(p); p += align256(sizeof(double2) * (size_t)np * np);
  double2* pbuf = reinterpret_cast<double2*>(p); p += align256(sizeof(double2) * NB * NB);
  double2* rbuf = reinterpret_cast<double2*>(p); p += align256(sizeof(double2) * (size_t)NB * np);
  double2* cbuf = reinterpret_cast<double2*>(p); p += align256(sizeof(double2) * (size_t)NB * np);
  int* cand[2];
  cand[0] = reinterpret_cast<int*>(p); p += align256(sizeof(int) * (size_t)nchunk * NB);
  cand[1] = reinterpret_cast<int*>(p); p += align256(sizeof(int) * (size_t)nchunk * NB);
  int* piv = reinterpret_cast<int*>(p); p += align256(sizeof(int) * (size_t)n);
  int* inv = reinterpret_cast<int*>(p); p += align256(sizeof(int) * (size_t)n);
  int* gather = reinterpret_cast<int*>(p); p += align256(sizeof(int) * (1 + 4 * kTourNB));
  unsigned long long* amax = reinterpret_cast<unsigned long long*>(p); p += align256(8);
  void* ozws = p;
  LookAhead* la = nullptr;
  int rc = look_ahead(&la);
  if (rc) return rc;
  const size_t total = (size_t)np * np;
  int bx = (int)((total + 255) / 256);
  if (bx > 152 * 8) bx = 152 * 8;
  NED_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned long long), st));
  {
    const size_t nn = (size_t)n * n;
    int ab = (int)((nn + 255) / 256);
    if (ab > 152 * 4) ab = 152 * 4;
    amax_kernel<<<ab, 256, 0, st>>>(a, nn, amax);
    NED_LAUNCH_CHECK("amax_kernel");
  }
  pad_identity_kernel<<<bx, 256, 0, st>>>(a, n, ap, np, amax);
  NED_LAUNCH_CHECK("pad_identity_kernel");
  // tournament over the rows k0 .. n-1 on the panel columns k0 .. k0+31, then
  // the inverse of the winners' 32 x 32 block (read in their rows, before the
  // swaps), on stream s
  auto chain = [&](int k0, cudaStream_t s) -> int {
    const int* in = nullptr;
    int count = n - k0, buf = 0;
    while (true) {
      const int blocks = (count + kTourRows - 1) / kTourRows;
      const int fin = blocks == 1;
      tour_kernel<<<blocks, kTourRows, 0, s>>>(ap, np, n, k0, in, count, cand[buf], fin, piv, gather,
                                                       status);
      NED_LAUNCH_CHECK("tour_kernel");
      if (fin) break;
      in = cand[buf];
      count = blocks * kTourNB;
      buf ^= 1;
    }
    gj_pivot32_fp64_kernel<<<kPivCtas, 128, 0, s>>>(ap, np, k0, cand[buf], pbuf, status);
    NED_LAUNCH_CHECK("gj_pivot32_fp64_kernel");
    return NEDMFT_OK;
  };
  if ((rc = chain(0, st))) return rc;
  for (int k0 = 0; k0 < n; k0 += NB) {
    apply_gather_kernel<<<np / 32, 256, 0, st>>>(ap, np, gather);
    NED_LAUNCH_CHECK("apply_gather_kernel");
    gj_panels_kernel<double, NB, 8><<<dim3(np / 8, 1), 256, 0, st>>>(ap, np, k0, pbuf, rbuf, cbuf);
    NED_LAUNCH_CHECK("gj_panels_kernel");
    const int k1 = k0 + NB;  // the next step
    if (k1 >= n) {
      if ((rc = oz64_update(ap, np, k0, rbuf, cbuf, 0, 0, false, ozws, st, status))) return rc;
      break;
    }
    // side stream: this step's update of the next panel's columns, then the
    // next step's tournament and pivot block; here: the rest of the update
    NED_CUDA(cudaEventRecord(la->panel, st));
    NED_CUDA(cudaStreamWaitEvent(la->side, la->panel, 0));
    gj_update_window_kernel<NB><<<np / 8, 64, 0, la->side>>>(ap, np, k0, k1, rbuf, cbuf);
    NED_LAUNCH_CHECK("gj_update_window_kernel");
    if ((rc = chain(k1, la->side))) return rc;
    NED_CUDA(cudaEventRecord(la->chain, la->side));
    if ((rc = oz64_update(ap, np, k0, rbuf, cbuf, k1, k1 + NB, false, ozws, st, status))) return rc;
    NED_CUDA(cudaStreamWaitEvent(st, la->chain, 0));
  }
  swap_colmap_kernel<<<1, 1, 0, st>>>(n, piv, inv);
  NED_LAUNCH_CHECK("swap_colmap_kernel");
  int by = (int)(((size_t)n * n + 255) / 256);
  if (by > 152 * 8) by = 152 * 8;
  unpermute_kernel<<<by, 256, 0, st>>>(ap, np, n, inv, a, amax);
  NED_LAUNCH_CHECK("unpermute_kernel");
  return NEDMFT_OK;
}

// ------------------------------------------------------------------ FP64 reductions over the points

// gloc[i][j] (= or +=) sum_b wq[q0+b] (X[b] + dX[b])[i][col(j)], b ascending,
// col = unshift_col if `cycled` (the batch holds X' = (P A)^-1).
template <class T>
__global__ void reduce_gloc_kernel(ContourDev c, ModelDev m, const double* __restrict__ eps_d,
                                   const double* __restrict__ wq_d, int q0, int nb, const cplx_t<T>* __restrict__ X,
                                   const cplx_t<T>* __restrict__ dX, int ldx, bool cycled, bool first,
                                   double2* __restrict__ gloc) {
  const size_t total = (size_t)c.n * c.n;
  const size_t bstride = (size_t)ldx * ldx;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / c.n), j = (int)(e % c.n);
    double2 acc = first ? make_double2(0.0, 0.0) : gloc[e];
    for (int b = 0; b < nb; ++b) {
      const int q = q0 + b;
      const bool sh = cycled && shifted_point(m, eps_d[q]);
      const size_t off = (size_t)b * bstride + (size_t)i * ldx + unshift_col(j, c.n, sh);
      double2 v = to_d(X[off]);
      if (dX) v = cadd(v, to_d(dX[off]));
      const double w = wq_d[q];
      acc.x = fma(w, v.x, acc.x);
      acc.y = fma(w, v.y, acc.y);
    }
    gloc[e] = acc;
  }
}

// jacc[m] (= or +=) sum_b wq ebar_q(t_m) G_q[m][2 N_t - m].
template <class T>
__global__ void reduce_current_kernel(ContourDev c, ModelDev mo, const double* __restrict__ eps_d,
                                      const double* __restrict__ ebar_d, const double* __restrict__ wq_d, int q0,
                                      int nb, const cplx_t<T>* __restrict__ X, const cplx_t<T>* __restrict__ dX,
                                      int ldx, bool cycled, bool first, double2* __restrict__ jacc) {
  const int mm = blockIdx.x * blockDim.x + threadIdx.x;
  if (mm >= c.nt) return;
  const double t = t_re(c, mm);
  const int jcol = 2 * c.nt - mm;
  double2 acc = first ? make_double2(0.0, 0.0) : jacc[mm];
  for (int b = 0; b < nb; ++b) {
    const int q = q0 + b;
    const double eps = eps_d[q];
    const bool sh = cycled && shifted_point(mo, eps);
    const size_t off = (size_t)b * ldx * ldx + (size_t)mm * ldx + unshift_col(jcol, c.n, sh);
    double2 v = to_d(X[off]);
    if (dX) v = cadd(v, to_d(dX[off]));
    const double w = wq_d[q] * ebar_at(t, eps, ebar_d[q], mo.E);
    acc.x = fma(w, v.x, acc.x);
    acc.y = fma(w, v.y, acc.y);
  }
  jacc[mm] = acc;
}

// j = Re(i acc) = -acc.y, j_imag = Im(i acc) = acc.x.
__global__ void finish_current_kernel(int nt, const double2* __restrict__ jacc, double* __restrict__ j,
                                      double* __restrict__ ji) {
  const int mm = blockIdx.x * blockDim.x + threadIdx.x;
  if (mm >= nt) return;
  if (j) j[mm] = -jacc[mm].y;
  if (ji) ji[mm] = jacc[mm].x;
}

template <class T>
int launch_reduce(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar, const double* wq,
                  int q0, int nb, const cplx_t<T>* X, const cplx_t<T>* dX, int ldx, bool cycled, bool first,
                  double2* gloc, double2* jacc, cudaStream_t st) {
  size_t total = (size_t)c.n * c.n;
  int bx = (int)((total + 255) / 256);
  if (bx > 152 * 8) bx = 152 * 8;
  reduce_gloc_kernel<T><<<bx, 256, 0, st>>>(c, m, eps, wq, q0, nb, X, dX, ldx, cycled, first, gloc);
  NED_LAUNCH_CHECK("reduce_gloc_kernel");
  if (jacc) {
    reduce_current_kernel<T><<<ceil_div(c.nt, 128), 128, 0, st>>>(c, m, eps, ebar, wq, q0, nb, X, dX, ldx, cycled,
                                                                  first, jacc);
    NED_LAUNCH_CHECK("reduce_current_kernel");
  }
  return NEDMFT_OK;
}
template int launch_reduce<double>(const ContourDev&, const ModelDev&, const double*, const double*, const double*,
                                   int, int, const double2*, const double2*, int, bool, bool, double2*, double2*,
                                   cudaStream_t);

int launch_finish_current(int nt, const double2* jacc, double* j, double* ji, cudaStream_t st) {
  finish_current_kernel<<<ceil_div(nt, 128), 128, 0, st>>>(nt, jacc, j, ji);
  NED_LAUNCH_CHECK("finish_current_kernel");
  return NEDMFT_OK;
}

}  // namespace nedmft
