// The lattice step for small contours without any device allocation: its
// scratch is a file-scope device array instead of a caller-provided workspace.
#include <mutex>

#include "lattice.cuh"

namespace nedmft {
namespace {

constexpr int kStaticMaxN = kSmallPathMaxN;  // largest n_c (the single-CTA FP64 Gauss-Jordan path)
static_assert(kStaticMaxN == 112, "the documented limit of nedmft_lattice_gloc_static");
constexpr int kStaticBatch = 32;   // points inverted per pass
constexpr size_t kStaticS = (size_t)kStaticMaxN * kStaticMaxN * sizeof(double2);
constexpr size_t kStaticBatchBytes = (size_t)kStaticBatch * kStaticMaxN * kStaticMaxN * sizeof(double2);
constexpr size_t kStaticJ = (size_t)kStaticMaxN * sizeof(double2);
constexpr size_t kStaticBytes = ((kStaticS + 255) & ~(size_t)255) + ((kStaticBatchBytes + 255) & ~(size_t)255) +
                                ((kStaticJ + 255) & ~(size_t)255);  // about 6.6 MB

// One copy per device that loads the library, kept until the process exits.
// Host code must not use this name as an address: it is only a host-side
// stand-in for the symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the array on the current device, looked up once per device.
int static_scratch(void** out) {
  int dev = 0;
  NED_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(NEDMFT_ECUDA, "lattice_gloc_static: device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NEDMFT_OK;
}

}  // namespace
}  // namespace nedmft

using namespace nedmft;

extern "C" int nedmft_lattice_gloc_static(const nedmft_contour* c, const nedmft_model* m, const nedmft_c128* sigma_d,
                                          const double* eps_d, const double* ebar_d, const double* wq_d, int32_t nq,
                                          nedmft_c128* gloc_d, double* j_d, double* j_imag_d, void* stream) {
  if (!c || !m || !sigma_d || !eps_d || !ebar_d || !wq_d || !gloc_d)
    return set_error(NEDMFT_EINVAL, "lattice_gloc_static: NULL argument");
  if (c->n_t < 1 || c->n_tau < 1 || c->n_c != 2 * c->n_t + c->n_tau)
    return set_error(NEDMFT_EINVAL, "lattice_gloc_static: invalid contour");
  if (c->n_c > kStaticMaxN || c->n_c > small_path_max_n())
    return set_error(NEDMFT_EINVAL, "lattice_gloc_static: n_c = %d exceeds the static scratch limit of %d", c->n_c,
                     kStaticMaxN);
  if (nq < 1) return set_error(NEDMFT_EINVAL, "lattice_gloc_static: nq = %d < 1", nq);
  void* base = nullptr;
  int rc = static_scratch(&base);
  if (rc) return rc;
  int* status = device_status_ptr();
  if (!status) return set_error(NEDMFT_ECUDA, "lattice_gloc_static: no device status word");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ContourDev cd = to_dev(*c);
  const ModelDev md{m->U, m->E, m->w1, isnan(m->mu) ? m->U / 2 : m->mu};
  char* p = static_cast<char*>(base);
  double2* S = reinterpret_cast<double2*>(p);
  double2* out = reinterpret_cast<double2*>(p + ((kStaticS + 255) & ~(size_t)255));
  double2* jacc = reinterpret_cast<double2*>(p + ((kStaticS + 255) & ~(size_t)255) +
                                             ((kStaticBatchBytes + 255) & ~(size_t)255));
  double2* ja = (j_d || j_imag_d) ? jacc : nullptr;
  double2* gl = reinterpret_cast<double2*>(gloc_d);
  // every buffer below is written before it is read: the first pass
  // overwrites gloc and the current accumulator instead of adding to them
  if ((rc = launch_build_s(cd, reinterpret_cast<const double2*>(sigma_d), S, st))) return rc;
  for (int q0 = 0; q0 < nq; q0 += kStaticBatch) {
    const int nb = nq - q0 < kStaticBatch ? nq - q0 : kStaticBatch;
    if ((rc = launch_gj_small_fp64(cd, md, eps_d, ebar_d, q0, nb, S, out, status, st))) return rc;
    if ((rc = launch_reduce<double>(cd, md, eps_d, ebar_d, wq_d, q0, nb, out, nullptr, cd.n, false, q0 == 0, gl, ja,
                                    st)))
      return rc;
  }
  if (ja) {
    if ((rc = launch_finish_current(cd.nt, jacc, j_d, j_imag_d, st))) return rc;
  }
  return NEDMFT_OK;
}
