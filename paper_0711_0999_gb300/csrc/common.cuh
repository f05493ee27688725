// Shared device/host helpers of the lattice-step library.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "nedmft.h"

namespace nedmft {

// ------------------------------------------------------------------ errors

// Set the calling thread's last-error message (printf-style) and return `code`.
int set_error(int code, const char* fmt, ...);
// Map a CUDA error to NEDMFT_ECUDA with a message naming `what`.
int cuda_fail(cudaError_t e, const char* what);

#define NED_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return ::nedmft::cuda_fail(e_, #call); \
  } while (0)

#define NED_LAUNCH_CHECK(what)                           \
  do {                                                   \
    ::nedmft::instr_count();                             \
    cudaError_t e_ = cudaGetLastError();                 \
    if (e_ != cudaSuccess) return ::nedmft::cuda_fail(e_, what); \
  } while (0)

// Instrumentation (off by default): a count of kernel launches and, when
// timing is on, CUDA events around the launches of the dominant kernel
// (the Gauss-Jordan trailing update), recorded on the launch stream.
void instr_count();
bool instr_timing();
int instr_begin(cudaStream_t st);                       // returns a slot, or -1
void instr_end(int slot, cudaStream_t st, double flops, double bytes);  // algorithmic work of the launch

// Device status word (one per device, file-scope in status.cu).  Kernels
// record the first failure with atomicCAS; nedmft_check_status reads it.
enum DeviceStatus : int { DS_OK = 0, DS_SINGULAR = 1, DS_TIMEOUT = 2 };
int* device_status_ptr();  // device address for the current device (cached)

// Per-device launch settings, each applied once per (kernel, device) under a
// lock: cudaFuncSetAttribute and occupancy queries act on the current device
// only, so a process-wide "done" flag would skip them on a second GPU.
int ensure_dyn_smem(const void* kern, int bytes);  // MaxDynamicSharedMemorySize >= bytes
int device_sm_count(int* out);                     // multiprocessors of the current device
// clusters of two CTAs of `kern` (block threads, dynamic shared bytes) that fit at once
int max_active_clusters(const void* kern, int block, int smem_bytes, int* out);

// ------------------------------------------------------------------ complex

template <class T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <class T> using cplx_t = typename cplx<T>::type;

template <class T> __host__ __device__ __forceinline__ cplx_t<T> mk(T re, T im) {
  cplx_t<T> z; z.x = re; z.y = im; return z;
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
// 1/z with a guard: returns false (and a large finite value) if |z| is below `tiny`.
template <class T> __device__ __forceinline__ bool cinv_guard(cplx_t<T> z, cplx_t<T>& out, T tiny) {
  T m = z.x * z.x + z.y * z.y;
  if (!(m > tiny * tiny)) {  // also catches NaN
    out = mk<T>(T(1) / tiny, T(0));
    return false;
  }
  T r = T(1) / m;
  out = mk<T>(z.x * r, -z.y * r);
  return true;
}
template <class T> __device__ __forceinline__ cplx_t<T> cvt(double2 z);
template <> __device__ __forceinline__ double2 cvt<double>(double2 z) { return z; }
template <> __device__ __forceinline__ float2 cvt<float>(double2 z) { return make_float2((float)z.x, (float)z.y); }
__device__ __forceinline__ double2 to_d(double2 z) { return z; }
__device__ __forceinline__ double2 to_d(float2 z) { return make_double2((double)z.x, (double)z.y); }

// ------------------------------------------------------------------ contour

// Contour and model as the kernels see them.
struct ContourDev {
  int nt, ntau, n;  // N_t, N_tau, N_c
  double tmin, tmax, dt, dtau, beta;
};
struct ModelDev {
  double U, E, w1, mu;
};

__host__ __device__ __forceinline__ ContourDev to_dev(const nedmft_contour& c) {
  ContourDev d;
  d.nt = c.n_t; d.ntau = c.n_tau; d.n = c.n_c;
  d.tmin = c.t_min; d.tmax = c.t_max; d.dt = c.dt; d.dtau = c.dtau; d.beta = c.beta;
  return d;
}

// Real part of contour time j (Eq. time_discrete; imaginary points sit at t_min).
__host__ __device__ __forceinline__ double t_re(const ContourDev& c, int j) {
  if (j < c.nt) return c.tmin + j * c.dt;
  if (j < 2 * c.nt) return c.tmax - (j - c.nt) * c.dt;
  return c.tmin;
}
// tau_j = -Im t_j.
__host__ __device__ __forceinline__ double t_tau(const ContourDev& c, int j) {
  return j < 2 * c.nt ? 0.0 : (j - 2 * c.nt) * c.dtau;
}
// Leftpoint weight W_j (Eq. integration_weights).
__host__ __device__ __forceinline__ double2 weight(const ContourDev& c, int j) {
  if (j < c.nt) return make_double2(c.dt, 0.0);
  if (j < 2 * c.nt) return make_double2(-c.dt, 0.0);
  return make_double2(0.0, -c.dtau);
}

// F(s2) - F(s1) for real s1, s2, F the antiderivative of the Peierls-shifted
// band energy of Eq. g_contour_non_final2 (F = eps s for s <= 0,
// [eps sin Es + ebar (cos Es - 1)]/E for s > 0).  Both points on the same
// side of 0 use product-to-sum forms, free of cancellation.
__device__ __forceinline__ double band_phase_diff(double s1, double s2, double eps, double ebar, double E) {
  if (E == 0.0) return eps * (s2 - s1);
  if (s1 <= 0.0 && s2 <= 0.0) return eps * (s2 - s1);
  if (s1 > 0.0 && s2 > 0.0) {
    double sh, ch, sm, cm;
    sincos(0.5 * E * (s2 - s1), &sh, &ch);
    sincos(0.5 * E * (s1 + s2), &sm, &cm);
    return 2.0 * sh * (eps * cm - ebar * sm) / E;
  }
  auto F = [&](double s) {
    if (s <= 0.0) return eps * s;
    double sn, cs;
    sincos(E * s, &sn, &cs);
    return (eps * sn + ebar * (cs - 1.0)) / E;
  };
  return F(s2) - F(s1);
}

// Entries of B_q = G0_q^-1 (bidiagonal plus one boundary element; derived
// from the theta structure of Eq. g_contour_non_final2 by Sherman-Morrison):
//   B_jj = i,
//   B_{j,j-1} = -i exp(i [mu dRe t - dF] - x dtau_j)   (j >= 1),
//   B_{0,N-1} = i exp(-x dtau),
// with x = eps - mu and dtau_j = tau_j - tau_{j-1}.
__device__ __forceinline__ double2 b_sub(const ContourDev& c, const ModelDev& m, double eps, double ebar, int j) {
  double x = eps - m.mu;
  double s1 = t_re(c, j - 1), s2 = t_re(c, j);
  double ph = m.mu * (s2 - s1) - band_phase_diff(s1, s2, eps, ebar, m.E);
  double mag = exp(-x * (t_tau(c, j) - t_tau(c, j - 1)));
  double sn, cs;
  sincos(ph, &sn, &cs);
  // -i * mag * (cs + i sn) = mag * (sn - i cs)
  return make_double2(mag * sn, -mag * cs);
}
__device__ __forceinline__ double2 b_corner(const ContourDev& c, const ModelDev& m, double eps) {
  double x = eps - m.mu;
  return make_double2(0.0, exp(-x * c.dtau));
}
// The dense entry of A_q = B_q - S at (row i, col j) for i, j < N.
__device__ __forceinline__ double2 a_entry(const ContourDev& c, const ModelDev& m, double eps, double ebar,
                                           const double2* __restrict__ S, int i, int j) {
  double2 v = S[(size_t)i * c.n + j];
  v.x = -v.x; v.y = -v.y;
  if (j == i) v.y += 1.0;
  else if (j == i - 1) v = cadd(v, b_sub(c, m, eps, ebar, i));
  if (i == 0 && j == c.n - 1) v = cadd(v, b_corner(c, m, eps));
  return v;
}
// Static row order: for x < 0 the rows of A_q are cycled up by one
// (row r <- row r+1), which makes every elimination multiplier <= 1 on the
// imaginary branch; the inverse is recovered with a column cycle.
__device__ __forceinline__ bool shifted_point(const ModelDev& m, double eps) { return eps - m.mu < 0.0; }
// Column of X' = (P A)^-1 holding column j of A^-1.
__device__ __forceinline__ int unshift_col(int j, int n, bool sh) { return sh ? (j == 0 ? n - 1 : j - 1) : j; }

// ebar_{k + theta(t) E t} at upper-branch time t (Eq. current_def with v -> -ebar).
__device__ __forceinline__ double ebar_at(double t, double eps, double ebar, double E) {
  if (t <= 0.0) return ebar;
  double sn, cs;
  sincos(E * t, &sn, &cs);
  return ebar * cs + eps * sn;
}

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace nedmft
