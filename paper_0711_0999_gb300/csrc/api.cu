// C-ABI entry points of the lattice step, the G0 builder and the DMFT loop.
#include <math.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "lattice.cuh"
#include "umma.cuh"

namespace nedmft {

namespace {

constexpr int kNbSimt = 32;  // Gauss-Jordan block of the CUDA-core path

int padded(int n) { return ((n + 127) / 128) * 128; }

bool valid_contour(const nedmft_contour* c) {
  return c && c->n_t >= 1 && c->n_tau >= 1 && c->n_c == 2 * c->n_t + c->n_tau && c->dt > 0 && c->dtau > 0 &&
         c->beta > 0 && c->n_c <= 65536;
}

ModelDev model_dev(const nedmft_model& m) { return ModelDev{m.U, m.E, m.w1, isnan(m.mu) ? m.U / 2 : m.mu}; }

enum class Path { Small64, Blocked64, MixedUmma };

Path choose_path(const nedmft_contour& c, nedmft_precision p) {
  if (p == NEDMFT_FP64) return c.n_c <= small_path_max_n() ? Path::Small64 : Path::Blocked64;
  return Path::MixedUmma;
}

int padded_for(Path path, int n, int width) { return path == Path::MixedUmma ? umma_padded(n, width) : padded(n); }

// Points per batch and Gauss-Jordan block width chosen by
// nedmft_lattice_autotune, per (n_c, nq, precision); 0 = the default.
struct Tuned {
  int batch, width;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, Tuned> g_tuned;

Tuned tuned_for(const nedmft_contour& c, int nq, nedmft_precision prec) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(std::make_tuple(c.n_c, nq, (int)prec));
  return it == g_tuned.end() ? Tuned{0, 0} : it->second;
}

int default_batch(const nedmft_contour& c, int nq, Path path, int width) {
  const size_t np = padded_for(path, c.n_c, width);
  size_t per = 0, budget = (size_t)96 << 30;  // about 96 GB of batch buffers (a third of HBM)
  int cap = 152;
  switch (path) {
    case Path::Small64: per = sizeof(double2) * c.n_c * c.n_c; cap = 2048; break;
    case Path::Blocked64: per = sizeof(double2) * np * np; cap = 152; break;
    case Path::MixedUmma: per = umma_batch_bytes_per_matrix((int)np, width); cap = umma_default_batch((int)np); break;
  }
  int b = (int)(budget / (per ? per : 1));
  if (b > cap) b = cap;
  if (b > nq) b = nq;
  if (b < 1) b = 1;
  return b;
}

struct LatticeLayout {
  size_t S, gscratch, jacc, batch, pbuf, rbuf, cbuf, extra, total;
  int np, mb, width;
  Path path;
};

// batch <= 0: the tuned batch (else the default); width < 0: the tuned width
// (else the default, 0)
LatticeLayout lattice_layout(const nedmft_contour& c, int nq, nedmft_precision prec, int batch, int width = -1) {
  LatticeLayout L{};
  L.path = choose_path(c, prec);
  const Tuned t = tuned_for(c, nq, prec);
  if (width < 0) width = t.width;
  L.width = width;
  L.np = padded_for(L.path, c.n_c, width);
  if (batch <= 0) batch = t.batch;
  L.mb = batch > 0 ? (batch < nq ? batch : nq) : default_batch(c, nq, L.path, width);
  const size_t n = c.n_c, np = L.np, mb = L.mb;
  L.S = align256(sizeof(double2) * n * n);
  L.gscratch = align256(sizeof(double2) * n * n);
  L.jacc = align256(sizeof(double2) * c.n_t);
  switch (L.path) {
    case Path::Small64:
      L.batch = align256(sizeof(double2) * n * n * mb);
      break;
    case Path::Blocked64:
      L.batch = align256(sizeof(double2) * np * np * mb);
      L.pbuf = align256(sizeof(double2) * kNbSimt * kNbSimt * mb);
      L.rbuf = align256(sizeof(double2) * kNbSimt * np * mb);
      L.cbuf = align256(sizeof(double2) * np * kNbSimt * mb);
      break;
    case Path::MixedUmma:
      L.batch = align256(umma_batch_bytes((int)np, (int)mb, width));
      L.extra = align256(umma_shared_bytes((int)np, nq));
      break;
  }
  L.total = L.S + L.gscratch + L.jacc + L.batch + L.pbuf + L.rbuf + L.cbuf + L.extra + 256;
  return L;
}

}  // namespace

// The lattice step proper (also used by the current and the DMFT loop).
int lattice_run_batch(const nedmft_contour& c, const nedmft_model& m, const double2* sigma, const double* eps,
                      const double* ebar, const double* wq, int nq, nedmft_precision prec, double2* gloc, double* j,
                      double* ji, void* ws, size_t ws_bytes, cudaStream_t st, int batch_pts, int width = -1);

int lattice_run(const nedmft_contour& c, const nedmft_model& m, const double2* sigma, const double* eps,
                const double* ebar, const double* wq, int nq, nedmft_precision prec, double2* gloc, double* j,
                double* ji, void* ws, size_t ws_bytes, cudaStream_t st) {
  return lattice_run_batch(c, m, sigma, eps, ebar, wq, nq, prec, gloc, j, ji, ws, ws_bytes, st, 0);
}

// batch_pts > 0: points per batch (clamped to nq); 0: the tuned or default
// size; width >= 0: the Gauss-Jordan block width (0 = default), < 0: the tuned one
int lattice_run_batch(const nedmft_contour& c, const nedmft_model& m, const double2* sigma, const double* eps,
                      const double* ebar, const double* wq, int nq, nedmft_precision prec, double2* gloc, double* j,
                      double* ji, void* ws, size_t ws_bytes, cudaStream_t st, int batch_pts, int width) {
  LatticeLayout L = lattice_layout(c, nq, prec, batch_pts, width);
  if (ws_bytes < L.total) return set_error(NEDMFT_ENOMEM, "lattice: workspace %zu < %zu bytes", ws_bytes, L.total);
  int* status = device_status_ptr();
  if (!status) return set_error(NEDMFT_ECUDA, "lattice: no device status word");
  const ContourDev cd = to_dev(c);
  const ModelDev md = model_dev(m);
  char* p = static_cast<char*>(ws);
  double2* S = reinterpret_cast<double2*>(p); p += L.S;
  double2* gs = reinterpret_cast<double2*>(p); p += L.gscratch;
  double2* jacc = reinterpret_cast<double2*>(p); p += L.jacc;
  char* batch = p; p += L.batch;
  char* pbuf = p; p += L.pbuf;
  char* rbuf = p; p += L.rbuf;
  char* cbuf = p; p += L.cbuf;
  char* extra = p;
  if (!gloc) gloc = gs;
  double2* ja = (j || ji) ? jacc : nullptr;
  const int np = L.np, mb = L.mb;
  int rc = launch_build_s(cd, sigma, S, st);
  if (rc) return rc;
  if (L.path == Path::MixedUmma) {
    if ((rc = umma_prepare_shared(cd, S, np, eps, ebar, wq, nq, extra, st))) return rc;
  }
  for (int q0 = 0; q0 < nq; q0 += mb) {
    const int nb = (nq - q0) < mb ? (nq - q0) : mb;
    const bool first = (q0 == 0);
    switch (L.path) {
      case Path::Small64: {
        double2* out = reinterpret_cast<double2*>(batch);
        if ((rc = launch_gj_small_fp64(cd, md, eps, ebar, q0, nb, S, out, status, st))) return rc;
        if ((rc = launch_reduce<double>(cd, md, eps, ebar, wq, q0, nb, out, nullptr, cd.n, false, first, gloc, ja, st)))
          return rc;
        break;
      }
      case Path::Blocked64: {
        double2* A = reinterpret_cast<double2*>(batch);
        if ((rc = launch_gen_a<double>(cd, md, eps, ebar, q0, nb, S, A, np, st))) return rc;
        if ((rc = gj_blocked_simt<double>(A, cd.n, np, nb, reinterpret_cast<double2*>(pbuf), reinterpret_cast<double2*>(rbuf),
                                          reinterpret_cast<double2*>(cbuf), status, st)))
          return rc;
        if ((rc = launch_reduce<double>(cd, md, eps, ebar, wq, q0, nb, A, nullptr, np, true, first, gloc, ja, st)))
          return rc;
        break;
      }
      case Path::MixedUmma: {
        if ((rc = umma_lattice_batch(cd, md, eps, ebar, wq, q0, nb, nq, np, S, extra, batch, first, gloc, ja, status, st,
                                     L.width)))
          return rc;
        break;
      }
    }
  }
  if (ja) {
    if ((rc = launch_finish_current(cd.nt, jacc, j, ji, st))) return rc;
  }
  return NEDMFT_OK;
}

}  // namespace nedmft

using namespace nedmft;

extern "C" int nedmft_g0_build(const nedmft_contour* c, const nedmft_model* m, const double* eps_d,
                               const double* ebar_d, int32_t nq, nedmft_c128* g0_d, void* stream) {
  if (!valid_contour(c)) return set_error(NEDMFT_EINVAL, "g0_build: invalid contour");
  if (!m || !eps_d || !ebar_d || !g0_d) return set_error(NEDMFT_EINVAL, "g0_build: NULL argument");
  if (nq < 1 || nq > 65535) return set_error(NEDMFT_EINVAL, "g0_build: nq = %d outside [1, 65535]", nq);
  return launch_g0_build(to_dev(*c), model_dev(*m), eps_d, ebar_d, nq, reinterpret_cast<double2*>(g0_d),
                         static_cast<cudaStream_t>(stream));
}

extern "C" size_t nedmft_lattice_workspace_size(const nedmft_contour* c, int32_t nq, nedmft_precision prec,
                                                int32_t batch) {
  if (!valid_contour(c) || nq < 1) return 0;
  if (prec != NEDMFT_FP64 && prec != NEDMFT_MIXED_BF16) return 0;
  return lattice_layout(*c, nq, prec, batch).total;
}

static int lattice_checks(const nedmft_contour* c, const nedmft_model* m, const void* sigma, const double* eps,
                          const double* ebar, const double* wq, int nq, nedmft_precision prec, void* ws) {
  if (!valid_contour(c)) return set_error(NEDMFT_EINVAL, "lattice: invalid contour");
  if (!m) return set_error(NEDMFT_EINVAL, "lattice: model is NULL");
  if (!sigma || !eps || !ebar || !wq || !ws) return set_error(NEDMFT_EINVAL, "lattice: NULL device pointer");
  if (nq < 1) return set_error(NEDMFT_EINVAL, "lattice: nq = %d < 1", nq);
  if (prec != NEDMFT_FP64 && prec != NEDMFT_MIXED_BF16)
    return set_error(NEDMFT_EINVAL, "lattice: unknown precision %d", (int)prec);
  if (((uintptr_t)ws) & 255) return set_error(NEDMFT_EINVAL, "lattice: workspace not 256-byte aligned");
  if (!(m->w1 >= 0.0 && m->w1 <= 1.0)) return set_error(NEDMFT_EINVAL, "lattice: w1 = %g outside [0, 1]", m->w1);
  return NEDMFT_OK;
}

extern "C" int nedmft_lattice_gloc(const nedmft_contour* c, const nedmft_model* m, const nedmft_c128* sigma_d,
                                   const double* eps_d, const double* ebar_d, const double* wq_d, int32_t nq,
                                   nedmft_precision prec, nedmft_c128* gloc_d, double* j_d, double* j_imag_d,
                                   void* ws_d, size_t ws_bytes, void* stream) {
  int rc = lattice_checks(c, m, sigma_d, eps_d, ebar_d, wq_d, nq, prec, ws_d);
  if (rc) return rc;
  if (!gloc_d) return set_error(NEDMFT_EINVAL, "lattice_gloc: gloc_d is NULL");
  return lattice_run(*c, *m, reinterpret_cast<const double2*>(sigma_d), eps_d, ebar_d, wq_d, nq, prec,
                     reinterpret_cast<double2*>(gloc_d), j_d, j_imag_d, ws_d, ws_bytes,
                     static_cast<cudaStream_t>(stream));
}

extern "C" int nedmft_current(const nedmft_contour* c, const nedmft_model* m, const nedmft_c128* sigma_d,
                              const double* eps_d, const double* ebar_d, const double* wq_d, int32_t nq,
                              nedmft_precision prec, double* j_d, double* j_imag_d, void* ws_d, size_t ws_bytes,
                              void* stream) {
  int rc = lattice_checks(c, m, sigma_d, eps_d, ebar_d, wq_d, nq, prec, ws_d);
  if (rc) return rc;
  if (!j_d && !j_imag_d) return set_error(NEDMFT_EINVAL, "current: both outputs NULL");
  return lattice_run(*c, *m, reinterpret_cast<const double2*>(sigma_d), eps_d, ebar_d, wq_d, nq, prec, nullptr, j_d,
                     j_imag_d, ws_d, ws_bytes, static_cast<cudaStream_t>(stream));
}

extern "C" int nedmft_lattice_autotune(const nedmft_contour* c, const nedmft_model* m, const nedmft_c128* sigma_d,
                                       const double* eps_d, const double* ebar_d, const double* wq_d, int32_t nq,
                                       nedmft_precision prec, const int32_t* candidates, int32_t n_candidates,
                                       int32_t* best_batch, double* best_ms, void* ws_d, size_t ws_bytes,
                                       void* stream) {
  int rc = lattice_checks(c, m, sigma_d, eps_d, ebar_d, wq_d, nq, prec, ws_d);
  if (rc) return rc;
  if (!candidates || n_candidates < 1) return set_error(NEDMFT_EINVAL, "autotune: no candidates");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  NED_CUDA(cudaEventCreate(&e0));
  NED_CUDA(cudaEventCreate(&e1));
  int best = 0, best_w = 0;
  float best_t = 0.f;
  // block widths to try on the tensor-core path above 512 rows: 256 and 128
  // columns (the latter also pads to a multiple of 128 instead of 256)
  int widths[2] = {0, 0};
  int n_widths = 1;
  if (choose_path(*c, prec) == Path::MixedUmma && c->n_c > 512) {
    widths[0] = 256;
    widths[1] = 128;
    n_widths = 2;
  }
  for (int k = 0; k < n_candidates && !rc; ++k) {
    const int b = candidates[k];
    if (b < 1) continue;
    for (int wi = 0; wi < n_widths && !rc; ++wi) {
      const int w = widths[wi];
      if (lattice_layout(*c, nq, prec, b, w).total > ws_bytes) continue;  // does not fit the workspace
      // one untimed pass (first-use setup), one timed pass
      for (int pass = 0; pass < 2 && !rc; ++pass) {
        if (pass == 1) {
          const cudaError_t e = cudaEventRecord(e0, st);
          if (e != cudaSuccess) { rc = cuda_fail(e, "cudaEventRecord"); break; }
        }
        rc = lattice_run_batch(*c, *m, reinterpret_cast<const double2*>(sigma_d), eps_d, ebar_d, wq_d, nq, prec,
                               nullptr, nullptr, nullptr, ws_d, ws_bytes, st, b, w);
      }
      if (rc) break;
      cudaError_t e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) { rc = cuda_fail(e, "autotune timing"); break; }
      if (!best || ms < best_t) { best = b < nq ? b : nq; best_w = w; best_t = ms; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (!best) return set_error(NEDMFT_ENOMEM, "autotune: no candidate batch fits the workspace of %zu bytes", ws_bytes);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::make_tuple(c->n_c, (int)nq, (int)prec)] = Tuned{best, best_w};
  }
  if (best_batch) *best_batch = best;
  if (best_ms) *best_ms = best_t;
  return nedmft_check_status(stream);
}

extern "C" int32_t nedmft_lattice_batch(const nedmft_contour* c, int32_t nq, nedmft_precision prec) {
  if (!valid_contour(c) || nq < 1) return 0;
  if (prec != NEDMFT_FP64 && prec != NEDMFT_MIXED_BF16) return 0;
  return lattice_layout(*c, nq, prec, 0).mb;
}

extern "C" int nedmft_lattice_set_tuning(const nedmft_contour* c, int32_t nq, nedmft_precision prec, int32_t batch,
                                         int32_t width) {
  if (!valid_contour(c) || nq < 1) return set_error(NEDMFT_EINVAL, "set_tuning: invalid contour or nq");
  if (prec != NEDMFT_FP64 && prec != NEDMFT_MIXED_BF16) return set_error(NEDMFT_EINVAL, "set_tuning: precision");
  if (batch < 0 || (width != 0 && width != 128 && width != 256))
    return set_error(NEDMFT_EINVAL, "set_tuning: batch %d < 0 or width %d not 0, 128 or 256", batch, width);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[std::make_tuple(c->n_c, (int)nq, (int)prec)] = Tuned{batch, width};
  return NEDMFT_OK;
}

extern "C" int32_t nedmft_lattice_block_width(const nedmft_contour* c, int32_t nq, nedmft_precision prec) {
  if (!valid_contour(c) || nq < 1) return 0;
  if (prec == NEDMFT_FP64) return 32;
  if (prec != NEDMFT_MIXED_BF16) return 0;
  const LatticeLayout L = lattice_layout(*c, nq, prec, 0);
  return umma_block_width(L.np, L.width);
}
