// Tensor-core (tcgen05) path of the lattice step: bf16x3 Gauss-Jordan with
// TMEM accumulation and an FP64-residual refinement step.
#pragma once

#include "common.cuh"

namespace nedmft {

// Gauss-Jordan block width of this path: 128 or 256 columns, or 0 for the
// default (256 where the padded size is a multiple of 256 from 512 up, else
// 128).  Padded size: a multiple of 128 up to 512; above, a multiple of 256
// for width 256, of 128 for width 128, and for the default whichever of the
// two the flop count favours (see umma_padded).
int umma_padded(int n, int width);
int umma_block_width(int np, int width);  // the width the path uses for padded size np
size_t umma_batch_bytes_per_matrix(int np, int width);
size_t umma_batch_bytes(int np, int nb, int width);
int umma_default_batch(int np);
size_t umma_shared_bytes(int np, int nq);
int umma_prepare_shared(const ContourDev& c, const double2* S, int np, const double* eps, const double* ebar,
                        const double* wq, int nq, char* shared, cudaStream_t st);
int umma_lattice_batch(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar,
                       const double* wq, int q0, int nb, int nq_total, int np, const double2* S, char* shared,
                       char* batch, bool first, double2* gloc, double2* jacc, int* status, cudaStream_t st,
                       int width);

// Limit of the bounded device waits on the current device (synchronises st).
int umma_set_wait_ns(uint64_t ns, cudaStream_t st);

// A bounded wait on a barrier that nothing arrives at (records DS_TIMEOUT).
int umma_wait_selftest(int* status, cudaStream_t st);

// C[m x n] = op(A) op(B) (+ bias) (+ C) for the warm-start network, FP32 in
// memory, bf16 tcgen05 products with FP32 sums; n <= 256.  splits > 1 sums K
// in that many parts into `part` (umma_mlp_split_bytes) and adds them in order.
size_t umma_mlp_split_bytes(int m, int n, int splits);
int umma_mlp_gemm(const float* A, const float* B, const float* bias, float* C, int m, int n, int k, bool ta, bool tb,
                  bool accumulate, float* part, int splits, cudaStream_t st);

}  // namespace nedmft
