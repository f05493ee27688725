// Tensor-core (tcgen05) path of the lattice step: bf16x3 Gauss-Jordan with
// TMEM accumulation and an FP64-residual refinement step.
#pragma once

#include "common.cuh"

namespace nedmft {

// padded size for this path: a multiple of 128, of 256 above 512 (wider Gauss-Jordan blocks)
int umma_padded(int n);
size_t umma_batch_bytes_per_matrix(int np);
size_t umma_batch_bytes(int np, int nb);
int umma_default_batch(int np);
size_t umma_shared_bytes(int np, int nq);
int umma_prepare_shared(const ContourDev& c, const double2* S, int np, const double* eps, const double* ebar,
                        const double* wq, int nq, char* shared, cudaStream_t st);
int umma_lattice_batch(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar,
                       const double* wq, int q0, int nb, int nq_total, int np, const double2* S, char* shared,
                       char* batch, bool first, double2* gloc, double2* jacc, int* status, cudaStream_t st);

// Limit of the bounded device waits on the current device (synchronises st).
int umma_set_wait_ns(uint64_t ns, cudaStream_t st);

// A bounded wait on a barrier that nothing arrives at (records DS_TIMEOUT).
int umma_wait_selftest(int* status, cudaStream_t st);

}  // namespace nedmft
