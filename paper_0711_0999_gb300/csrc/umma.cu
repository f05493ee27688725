#include "umma.cuh"

namespace nedmft {

size_t umma_batch_bytes_per_matrix(int np) { return sizeof(float2) * (size_t)np * np; }
int umma_default_batch(int) { return 1; }
size_t umma_shared_bytes(int) { return 0; }
int umma_prepare_shared(const ContourDev&, const double2*, int, char*, cudaStream_t) { return NEDMFT_OK; }
int umma_lattice_batch(const ContourDev&, const ModelDev&, const double*, const double*, const double*, int, int, int,
                       const double2*, char*, char*, bool, double2*, double2*, int*, cudaStream_t) {
  return set_error(NEDMFT_EINVAL, "lattice: the NEDMFT_MIXED_BF16 tensor-core path is not built in this library");
}

}  // namespace nedmft
