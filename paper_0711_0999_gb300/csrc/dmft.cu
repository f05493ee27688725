// The DMFT self-consistency loop of Sec. II on the device.
#include <math.h>

#include <vector>

#include "lattice.cuh"

namespace nedmft {

int lattice_run(const nedmft_contour& c, const nedmft_model& m, const double2* sigma, const double* eps,
                const double* ebar, const double* wq, int nq, nedmft_precision prec, double2* gloc, double* j,
                double* ji, void* ws, size_t ws_bytes, cudaStream_t st);

namespace {

constexpr int kNormBlocks = 304;

// Per-block maxima of |a - b| and |a| (pass 1) and their global maxima (pass 2):
// err = max|a - b| / max|a|, deterministic.
__global__ void norm_pass1(const double2* __restrict__ a, const double2* __restrict__ b, size_t total,
                           double* __restrict__ part) {
  __shared__ double sd[256], sa[256];
  double md = 0.0, ma = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    double2 x = a[e], y = b[e];
    double dx = x.x - y.x, dy = x.y - y.y;
    md = fmax(md, sqrt(dx * dx + dy * dy));
    ma = fmax(ma, sqrt(x.x * x.x + x.y * x.y));
  }
  sd[threadIdx.x] = md;
  sa[threadIdx.x] = ma;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + s]);
      sa[threadIdx.x] = fmax(sa[threadIdx.x], sa[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sd[0];
    part[2 * blockIdx.x + 1] = sa[0];
  }
}

__global__ void norm_pass2(const double* __restrict__ part, int nblocks, double* __restrict__ err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double md = 0.0, ma = 0.0;
  for (int i = 0; i < nblocks; ++i) {
    md = fmax(md, part[2 * i]);
    ma = fmax(ma, part[2 * i + 1]);
  }
  *err = ma > 0.0 ? md / ma : (md > 0.0 ? INFINITY : 0.0);
}

struct DmftLayout {
  size_t quad, gbuf, sbuf, part, lat, imp, total;
};

DmftLayout dmft_layout(const nedmft_contour& c, int n_quad, nedmft_precision prec) {
  DmftLayout L{};
  const size_t n = c.n_c, nq = (size_t)n_quad * n_quad;
  L.quad = 3 * align256(sizeof(double) * nq);
  L.gbuf = 2 * align256(sizeof(double2) * n * n);
  L.sbuf = 2 * align256(sizeof(double2) * n * n);
  L.part = align256(sizeof(double) * (2 * kNormBlocks + 1));
  L.lat = align256(nedmft_lattice_workspace_size(&c, (int)nq, prec, 0));
  L.imp = align256(nedmft_impurity_workspace_size(&c));
  L.total = L.quad + L.gbuf + L.sbuf + L.part + L.lat + L.imp + 256;
  return L;
}

// A private non-blocking stream that starts after `user` and that `user`
// waits for when the scope closes.
struct StreamScope {
  cudaStream_t user = nullptr, ws = nullptr;
  cudaEvent_t ev = nullptr;
  int open(cudaStream_t u) {
    user = u;
    NED_CUDA(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
    NED_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    NED_CUDA(cudaEventRecord(ev, user));
    NED_CUDA(cudaStreamWaitEvent(ws, ev, 0));
    return NEDMFT_OK;
  }
  ~StreamScope() {
    if (ws) {
      if (ev) {
        cudaEventRecord(ev, ws);
        cudaStreamWaitEvent(user, ev, 0);
      }
      cudaStreamDestroy(ws);
    }
    if (ev) cudaEventDestroy(ev);
  }
};
struct GraphScope {
  cudaGraph_t* g;
  cudaGraphExec_t* e;
  ~GraphScope() {
    for (int i = 0; i < 2; ++i) {
      if (e[i]) cudaGraphExecDestroy(e[i]);
      if (g[i]) cudaGraphDestroy(g[i]);
    }
  }
};
}  // namespace
}  // namespace nedmft

using namespace nedmft;

extern "C" size_t nedmft_dmft_workspace_size(const nedmft_contour* c, int32_t n_quad, nedmft_precision prec) {
  if (!c || n_quad < 1 || n_quad > 512 || c->n_c < 2) return 0;
  if (nedmft_lattice_workspace_size(c, n_quad * n_quad, prec, 0) == 0) return 0;
  return dmft_layout(*c, n_quad, prec).total;
}

extern "C" int nedmft_dmft_solve(const nedmft_contour* c, const nedmft_model* m, int32_t n_quad,
                                 nedmft_precision prec, const nedmft_c128* sigma_init_d, double tol, int32_t max_iter,
                                 nedmft_c128* sigma_d, nedmft_c128* gloc_d, double* j_d, int32_t* iters, double* err,
                                 void* ws_d, size_t ws_bytes, void* stream) {
  if (!c || !m || !sigma_d || !gloc_d || !ws_d) return set_error(NEDMFT_EINVAL, "dmft_solve: NULL argument");
  if (n_quad < 1 || n_quad > 512) return set_error(NEDMFT_EINVAL, "dmft_solve: n_quad = %d outside [1, 512]", n_quad);
  if (max_iter < 1) return set_error(NEDMFT_EINVAL, "dmft_solve: max_iter < 1");
  if (!(tol > 0.0)) return set_error(NEDMFT_EINVAL, "dmft_solve: tol must be > 0");
  const size_t need = nedmft_dmft_workspace_size(c, n_quad, prec);
  if (need == 0) return set_error(NEDMFT_EINVAL, "dmft_solve: invalid contour or precision");
  if (ws_bytes < need) return set_error(NEDMFT_ENOMEM, "dmft_solve: workspace %zu < %zu", ws_bytes, need);
  if (((uintptr_t)ws_d) & 255) return set_error(NEDMFT_EINVAL, "dmft_solve: workspace not 256-byte aligned");
  // the loop runs on a private stream ordered after the caller's (graph
  // capture is not possible on the legacy default stream); the caller's stream
  // waits for it when the scope closes
  StreamScope scope;
  int src = scope.open(static_cast<cudaStream_t>(stream));
  if (src) return src;
  cudaStream_t st = scope.ws;
  cudaGraph_t graph_of[2] = {nullptr, nullptr};
  cudaGraphExec_t exec_of[2] = {nullptr, nullptr};
  GraphScope gscope{graph_of, exec_of};
  DmftLayout L = dmft_layout(*c, n_quad, prec);
  const int nq = n_quad * n_quad;
  const size_t n = c->n_c, nn = n * n;
  char* p = static_cast<char*>(ws_d);
  double* eps = reinterpret_cast<double*>(p);
  double* ebar = reinterpret_cast<double*>(p + align256(sizeof(double) * nq));
  double* wq = reinterpret_cast<double*>(p + 2 * align256(sizeof(double) * nq));
  p += L.quad;
  double2* g[2] = {reinterpret_cast<double2*>(p), reinterpret_cast<double2*>(p + align256(sizeof(double2) * nn))};
  p += L.gbuf;
  double2* s[2] = {reinterpret_cast<double2*>(p), reinterpret_cast<double2*>(p + align256(sizeof(double2) * nn))};
  p += L.sbuf;
  double* part = reinterpret_cast<double*>(p);
  double* err_d = part + 2 * kNormBlocks;
  p += L.part;
  void* lat_ws = p;
  p += L.lat;
  void* imp_ws = p;

  std::vector<double> he(nq), hb(nq), hw(nq);
  int rc = nedmft_quadrature_grid(n_quad, he.data(), hb.data(), hw.data());
  if (rc) return rc;
  NED_CUDA(cudaMemcpyAsync(eps, he.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, st));
  NED_CUDA(cudaMemcpyAsync(ebar, hb.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, st));
  NED_CUDA(cudaMemcpyAsync(wq, hw.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, st));
  if (sigma_init_d)
    NED_CUDA(cudaMemcpyAsync(s[0], sigma_init_d, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st));
  else
    NED_CUDA(cudaMemsetAsync(s[0], 0, sizeof(double2) * nn, st));

  double e_host = INFINITY;
  int it = 1;
  bool conv = false;
  // Iteration 1 runs eagerly on the private stream; every later iteration --
  // impurity step, lattice step, convergence norm -- is one CUDA-graph launch.
  // graph[par] takes (g[par], s[par]) to s[1 - par], g[1 - par] and the norm of
  // g[1 - par] - g[par]; the iterations alternate par = 0, 1, 0, ...
  rc = lattice_run(*c, *m, s[0], eps, ebar, wq, nq, prec, g[0], j_d, nullptr, lat_ws, L.lat, st);
  if (rc) return rc;
  int cur = 0;  // s[cur], g[cur] hold the latest pair
  if (max_iter > 1) {
    if ((rc = pivot_inverse_prepare())) return rc;  // no stream creation or attribute change inside the capture
    for (int par = 0; par < 2; ++par) {
      NED_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      int crc = nedmft_impurity_update(c, m, reinterpret_cast<const nedmft_c128*>(g[par]),
                                       reinterpret_cast<const nedmft_c128*>(s[par]),
                                       reinterpret_cast<nedmft_c128*>(s[1 - par]), nullptr, imp_ws, L.imp, st);
      if (!crc)
        crc = lattice_run(*c, *m, s[1 - par], eps, ebar, wq, nq, prec, g[1 - par], j_d, nullptr, lat_ws, L.lat, st);
      if (!crc) {
        norm_pass1<<<kNormBlocks, 256, 0, st>>>(g[1 - par], g[par], nn, part);
        norm_pass2<<<1, 32, 0, st>>>(part, kNormBlocks, err_d);
      }
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(st, &graph);
      graph_of[par] = graph;
      if (crc) return crc;
      if (ce != cudaSuccess) return cuda_fail(ce, "dmft_solve: capture of the iteration");
      NED_CUDA(cudaGraphInstantiate(&exec_of[par], graph, 0));
    }
  }
  for (it = 2; it <= max_iter; ++it) {
    const int par = cur;
    NED_CUDA(cudaGraphLaunch(exec_of[par], st));
    NED_CUDA(cudaMemcpyAsync(&e_host, err_d, sizeof(double), cudaMemcpyDeviceToHost, st));
    NED_CUDA(cudaStreamSynchronize(st));
    cur = 1 - par;
    int ds = nedmft_check_status(st);
    if (ds) return ds;
    if (e_host < tol) { conv = true; break; }
  }
  const int gcur = cur;
  if (it > max_iter) it = max_iter;
  NED_CUDA(cudaMemcpyAsync(gloc_d, g[gcur], sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st));
  NED_CUDA(cudaMemcpyAsync(sigma_d, s[cur], sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st));
  NED_CUDA(cudaStreamSynchronize(st));
  int ds = nedmft_check_status(st);
  if (ds) return ds;
  if (iters) *iters = it;
  if (err) *err = e_host;
  return conv ? NEDMFT_OK : NEDMFT_ENOTCONV;
}

// ------------------------------------------------------------------ several runs

namespace {

struct BatchLayout {
  size_t quad, per_run_total, part, errs, lat, imp, total;
  std::vector<size_t> run_off;  // offset of run r's (g[2], s[2]) block
};

BatchLayout batch_layout(int n_runs, const nedmft_contour* cs, int n_quad, nedmft_precision prec) {
  BatchLayout L{};
  const size_t nq = (size_t)n_quad * n_quad;
  L.quad = 3 * align256(sizeof(double) * nq);
  L.run_off.resize(n_runs);
  size_t off = 0;
  for (int r = 0; r < n_runs; ++r) {
    L.run_off[r] = off;
    const size_t nn = (size_t)cs[r].n_c * cs[r].n_c;
    off += 4 * align256(sizeof(double2) * nn);
    const size_t lat = nedmft_lattice_workspace_size(&cs[r], (int)nq, prec, 0);
    const size_t imp = nedmft_impurity_workspace_size(&cs[r]);
    if (lat > L.lat) L.lat = lat;
    if (imp > L.imp) L.imp = imp;
  }
  L.per_run_total = off;
  L.part = align256(sizeof(double) * 2 * kNormBlocks);
  L.errs = align256(sizeof(double) * (size_t)n_runs);
  L.lat = align256(L.lat);
  L.imp = align256(L.imp);
  L.total = L.quad + L.per_run_total + L.part + L.errs + L.lat + L.imp + 256;
  return L;
}

}  // namespace

extern "C" size_t nedmft_dmft_batch_workspace_size(int32_t n_runs, const nedmft_contour* contours, int32_t n_quad,
                                                   nedmft_precision prec) {
  if (n_runs < 1 || !contours || n_quad < 1 || n_quad > 512) return 0;
  for (int r = 0; r < n_runs; ++r)
    if (nedmft_lattice_workspace_size(&contours[r], n_quad * n_quad, prec, 0) == 0) return 0;
  return batch_layout(n_runs, contours, n_quad, prec).total;
}

extern "C" int nedmft_dmft_solve_batch(int32_t n_runs, const nedmft_contour* contours, const nedmft_model* models,
                                       int32_t n_quad, nedmft_precision prec,
                                       const nedmft_c128* const* sigma_init_d, double tol, int32_t max_iter,
                                       nedmft_c128* const* sigma_d, nedmft_c128* const* gloc_d, double* const* j_d,
                                       int32_t* iters, double* errs, int32_t* converged, void* ws_d, size_t ws_bytes,
                                       void* stream) {
  if (n_runs < 1 || !contours || !models || !sigma_d || !gloc_d || !ws_d)
    return set_error(NEDMFT_EINVAL, "dmft_solve_batch: NULL argument or no runs");
  if (max_iter < 1 || !(tol > 0.0)) return set_error(NEDMFT_EINVAL, "dmft_solve_batch: max_iter < 1 or tol <= 0");
  const size_t need = nedmft_dmft_batch_workspace_size(n_runs, contours, n_quad, prec);
  if (need == 0) return set_error(NEDMFT_EINVAL, "dmft_solve_batch: invalid contour, n_quad or precision");
  if (ws_bytes < need) return set_error(NEDMFT_ENOMEM, "dmft_solve_batch: workspace %zu < %zu", ws_bytes, need);
  if (((uintptr_t)ws_d) & 255) return set_error(NEDMFT_EINVAL, "dmft_solve_batch: workspace not 256-byte aligned");
  for (int r = 0; r < n_runs; ++r)
    if (!sigma_d[r] || !gloc_d[r]) return set_error(NEDMFT_EINVAL, "dmft_solve_batch: run %d has a NULL output", r);
  StreamScope scope;
  int rc = scope.open(static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  cudaStream_t st = scope.ws;
  const BatchLayout L = batch_layout(n_runs, contours, n_quad, prec);
  const int nq = n_quad * n_quad;
  char* base = static_cast<char*>(ws_d);
  double* eps = reinterpret_cast<double*>(base);
  double* ebar = reinterpret_cast<double*>(base + align256(sizeof(double) * nq));
  double* wq = reinterpret_cast<double*>(base + 2 * align256(sizeof(double) * nq));
  char* runs = base + L.quad;
  double* part = reinterpret_cast<double*>(runs + L.per_run_total);
  double* err_d = reinterpret_cast<double*>(reinterpret_cast<char*>(part) + L.part);
  void* lat_ws = reinterpret_cast<char*>(err_d) + L.errs;
  void* imp_ws = static_cast<char*>(lat_ws) + L.lat;
  std::vector<double> he(nq), hb(nq), hw(nq);
  if ((rc = nedmft_quadrature_grid(n_quad, he.data(), hb.data(), hw.data()))) return rc;
  NED_CUDA(cudaMemcpyAsync(eps, he.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, st));
  NED_CUDA(cudaMemcpyAsync(ebar, hb.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, st));
  NED_CUDA(cudaMemcpyAsync(wq, hw.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, st));

  struct Run {
    double2* g[2];
    double2* s[2];
    size_t nn;
    int cur, it;
    bool active, conv;
    double err;
  };
  std::vector<Run> R(n_runs);
  for (int r = 0; r < n_runs; ++r) {
    Run& u = R[r];
    u.nn = (size_t)contours[r].n_c * contours[r].n_c;
    const size_t one = align256(sizeof(double2) * u.nn);
    char* p = runs + L.run_off[r];
    u.g[0] = reinterpret_cast<double2*>(p);
    u.g[1] = reinterpret_cast<double2*>(p + one);
    u.s[0] = reinterpret_cast<double2*>(p + 2 * one);
    u.s[1] = reinterpret_cast<double2*>(p + 3 * one);
    u.cur = 0;
    u.it = 1;
    u.active = true;
    u.conv = false;
    u.err = INFINITY;
    if (sigma_init_d && sigma_init_d[r])
      NED_CUDA(cudaMemcpyAsync(u.s[0], sigma_init_d[r], sizeof(double2) * u.nn, cudaMemcpyDeviceToDevice, st));
    else
      NED_CUDA(cudaMemsetAsync(u.s[0], 0, sizeof(double2) * u.nn, st));
    double* jr = j_d ? j_d[r] : nullptr;
    if ((rc = lattice_run(contours[r], models[r], u.s[0], eps, ebar, wq, nq, prec, u.g[0], jr, nullptr, lat_ws, L.lat,
                          st)))
      return rc;
  }
  std::vector<double> eh(n_runs);
  int active = max_iter > 1 ? n_runs : 0;
  // one sweep: every active run takes one iteration; one host sync per sweep
  while (active > 0) {
    for (int r = 0; r < n_runs; ++r) {
      Run& u = R[r];
      if (!u.active) continue;
      const int c = u.cur;
      if ((rc = nedmft_impurity_update(&contours[r], &models[r], reinterpret_cast<const nedmft_c128*>(u.g[c]),
                                       reinterpret_cast<const nedmft_c128*>(u.s[c]),
                                       reinterpret_cast<nedmft_c128*>(u.s[1 - c]), nullptr, imp_ws, L.imp, st)))
        return rc;
      double* jr = j_d ? j_d[r] : nullptr;
      if ((rc = lattice_run(contours[r], models[r], u.s[1 - c], eps, ebar, wq, nq, prec, u.g[1 - c], jr, nullptr,
                            lat_ws, L.lat, st)))
        return rc;
      norm_pass1<<<kNormBlocks, 256, 0, st>>>(u.g[1 - c], u.g[c], u.nn, part);
      NED_LAUNCH_CHECK("norm_pass1");
      norm_pass2<<<1, 32, 0, st>>>(part, kNormBlocks, err_d + r);
      NED_LAUNCH_CHECK("norm_pass2");
    }
    NED_CUDA(cudaMemcpyAsync(eh.data(), err_d, sizeof(double) * n_runs, cudaMemcpyDeviceToHost, st));
    NED_CUDA(cudaStreamSynchronize(st));
    if ((rc = nedmft_check_status(st))) return rc;
    for (int r = 0; r < n_runs; ++r) {
      Run& u = R[r];
      if (!u.active) continue;
      u.cur = 1 - u.cur;
      ++u.it;
      u.err = eh[r];
      if (u.err < tol) u.conv = true;
      if (u.conv || u.it >= max_iter) {
        u.active = false;
        --active;
      }
    }
  }
  bool all = true;
  for (int r = 0; r < n_runs; ++r) {
    const Run& u = R[r];
    NED_CUDA(cudaMemcpyAsync(gloc_d[r], u.g[u.cur], sizeof(double2) * u.nn, cudaMemcpyDeviceToDevice, st));
    NED_CUDA(cudaMemcpyAsync(sigma_d[r], u.s[u.cur], sizeof(double2) * u.nn, cudaMemcpyDeviceToDevice, st));
    if (iters) iters[r] = u.it;
    if (errs) errs[r] = u.err;
    if (converged) converged[r] = u.conv ? 1 : 0;
    all = all && u.conv;
  }
  NED_CUDA(cudaStreamSynchronize(st));
  if ((rc = nedmft_check_status(st))) return rc;
  return all ? NEDMFT_OK : NEDMFT_ENOTCONV;
}
