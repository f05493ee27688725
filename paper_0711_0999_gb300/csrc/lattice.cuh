// Internal launchers of the lattice-step kernels (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace nedmft {

int launch_build_s(const ContourDev& c, const double2* sigma, double2* S, cudaStream_t st);
int launch_g0_build(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar, int nq,
                    double2* g0, cudaStream_t st);
template <class T>
int launch_gen_a(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar, int q0, int nb,
                 const double2* S, cplx_t<T>* A, int np, cudaStream_t st);

// Largest n_c of the single-CTA FP64 Gauss-Jordan path (whole matrix in shared memory).
constexpr int kSmallPathMaxN = 112;
int small_path_max_n();
int launch_gj_small_fp64(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar, int q0,
                         int nb, const double2* S, double2* out, int* status, cudaStream_t st);

template <class T>
int gj_blocked_simt(cplx_t<T>* A, int n, int np, int nb_batch, cplx_t<T>* Pbuf, cplx_t<T>* Rbuf, cplx_t<T>* Cbuf,
                    int* status, cudaStream_t st);

template <class T>
int launch_reduce(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar, const double* wq,
                  int q0, int nb, const cplx_t<T>* X, const cplx_t<T>* dX, int ldx, bool cycled, bool first,
                  double2* gloc, double2* jacc, cudaStream_t st);
int launch_finish_current(int nt, const double2* jacc, double* j, double* ji, cudaStream_t st);

// Dense FP64 inversion with partial pivoting (impurity step).
size_t pivot_inverse_workspace(int n);
int pivot_inverse(double2* a, int n, void* ws, cudaStream_t st, int* status);
int pivot_inverse_prepare();  // before capturing pivot_inverse into a graph
// FP64-accurate trailing update of pivot_inverse on the tensor cores (Ozaki
// split); np a multiple of 128; columns j written iff (wlo <= j < whi) == inside.
size_t oz64_workspace(int np);
int oz64_prepare();  // the update kernel's shared-memory limit and the SM count, cached per device
int oz64_set_wait_ns(uint64_t ns, cudaStream_t st);  // its bounded waits' limit on the current device
int oz64_update(double2* A, int np, int k0, const double2* Rbuf, const double2* Cbuf, int wlo, int whi, bool inside,
                void* ws, cudaStream_t st, int* status);

}  // namespace nedmft
