/*
 * nedmft.h -- C ABI of the GB300 nonequilibrium-DMFT lattice-step library.
 *
 * Physics (J. K. Freericks, "Quenching Bloch oscillations in a strongly
 * correlated material", Sec. II): the spinless Falicov-Kimball model at half
 * filling on the infinite-dimensional hypercubic lattice, in a uniform field
 * along the diagonal switched on at t = 0, solved on the Kadanoff-Baym-Keldysh
 * contour discretised into an N_c x N_c complex matrix.
 *
 * Conventions shared by every entry point
 *   - Contour index order: upper real branch (N_t points), lower real branch
 *     (N_t points), imaginary branch (N_tau points); N_c = 2 N_t + N_tau
 *     (Eq. time_discrete).  All indices below are 0-based.
 *   - Matrices are dense, row-major, N_c x N_c, interleaved complex
 *     (nedmft_c128 == {re, im} == torch.complex128 == C99 double _Complex).
 *   - A "_d" suffix marks a DEVICE pointer (CUDA global memory of the current
 *     device); "_host" marks host memory.  The library never frees caller
 *     memory and never allocates device memory: scratch comes only through an
 *     explicit workspace whose size a *_workspace_size call returns.  Device
 *     pointers and the workspace must be 256-byte aligned.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *     take a stream are stream-ordered and do not synchronise the host unless
 *     stated; their outputs are ready when the stream reaches them.
 *   - Return value: 0 (NEDMFT_OK) on success, < 0 on error, > 0 for a
 *     warning.  No C++ exception crosses this boundary.  On error,
 *     nedmft_last_error() returns a message for the calling thread.
 *   - Device-side failures (a pivot below the safety threshold, a bounded
 *     wait that ran out) are recorded in a device status word that the
 *     synchronising calls (nedmft_dmft_solve, nedmft_check_status) read back;
 *     no kernel traps.
 */
#ifndef NEDMFT_H
#define NEDMFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- types */

typedef struct {
  double re, im;
} nedmft_c128;

/* The discretised contour (Eqs. time_discrete, integration_weights). */
typedef struct {
  double t_min, t_max, dt, beta, dtau;
  int32_t n_t;   /* points per real branch, (t_max - t_min)/dt */
  int32_t n_tau; /* imaginary points, beta/dtau */
  int32_t n_c;   /* 2 n_t + n_tau */
} nedmft_contour;

/* Falicov-Kimball model in the diagonal field (Eq. hamiltonian_fk,
 * Eq. vector_potential).  mu = NaN selects half filling, mu = U/2. */
typedef struct {
  double U;  /* interaction */
  double E;  /* field strength, switched on at t = 0 */
  double w1; /* localized-electron filling <w_1> (1/2 at half filling) */
  double mu; /* chemical potential, NaN -> U/2 */
} nedmft_model;

/* Arithmetic of the per-point Dyson solve of nedmft_lattice_gloc. */
typedef enum {
  /* FP64 Gauss-Jordan inversion of each B_q - S (DFMA). */
  NEDMFT_FP64 = 0,
  /* bf16x3 (hi*hi + hi*lo + lo*hi) tcgen05 tensor-core Gauss-Jordan with
   * FP32 accumulation in TMEM; then, for every point outside the
   * smallest-weight tail (total weight <= 1e-3 of the sum), one refinement
   * step X + X R with R = I - A X, whose entries of S on the pattern of B_q
   * are applied in double-float and whose dense rest S_d X runs as an exact
   * Ozaki split on the bf16 tensor cores (4 slices of 7 bits, exact chunk
   * sums combined in double-float); the sum over q is double-float, then
   * FP64.  (Three bf16 products per FP32-accurate product: no TF32 variant,
   * since one TF32 product keeps only 11 mantissa bits and three of them run
   * slower than three bf16 products.) */
  NEDMFT_MIXED_BF16 = 1
} nedmft_precision;

/* ---------------------------------------------------------------- status */

#define NEDMFT_OK 0
#define NEDMFT_EINVAL (-1)    /* bad argument (message in nedmft_last_error) */
#define NEDMFT_ENOMEM (-2)    /* workspace smaller than *_workspace_size */
#define NEDMFT_ECUDA (-3)     /* a CUDA runtime call failed */
#define NEDMFT_ESINGULAR (-4) /* a Gauss-Jordan pivot fell below the threshold */
#define NEDMFT_ETIMEOUT (-5)  /* a bounded device wait ran out */
#define NEDMFT_ENOTCONV 1     /* dmft_solve stopped at max_iter (warning) */

/* Static string for a status code. */
const char* nedmft_status_string(int status);
/* Last error message of the calling thread ("" if none). */
const char* nedmft_last_error(void);
/* Library version string. */
const char* nedmft_version(void);

/* Synchronise `stream`, read and clear the device status word (set by the
 * kernels on a bad pivot or an expired wait).  Returns NEDMFT_OK,
 * NEDMFT_ESINGULAR or NEDMFT_ETIMEOUT.  A non-finite input (a NaN or an
 * infinity in Sigma or G_loc) reaches a pivot of the Gauss-Jordan
 * elimination, where it counts as a pivot below the threshold:
 * NEDMFT_ESINGULAR. */
int nedmft_check_status(void* stream);

/* Failure detection of the tensor-core kernels.  Every wait of those kernels
 * for work (a filled or a free pipeline stage, an accumulator) is bounded: it
 * gives up after the device's wait limit, the kernel stops issuing work,
 * waits (for at most 2 s) for the copies and products it already issued,
 * releases its tensor memory, records NEDMFT_ETIMEOUT in the status word and
 * returns; the context stays usable and the outputs of that call are
 * undefined.
 * nedmft_set_wait_limit sets the limit on the current device (default 2 s;
 * seconds in [0, 60]; 0 makes every wait that is not satisfied at once give
 * up, which only a test of this path wants).  Synchronises `stream` and
 * applies to kernels launched after it returns.
 * nedmft_wait_selftest launches one kernel that waits, bounded by that
 * limit, on a barrier that nothing arrives at: nedmft_check_status then
 * returns NEDMFT_ETIMEOUT.  Stream-ordered. */
int nedmft_set_wait_limit(double seconds, void* stream);
int nedmft_wait_selftest(void* stream);

/* ---------------------------------------------------------------- instrumentation */

/* Measurement hooks used by the benchmark (off by default; not for use
 * while another thread drives the library).  enable != 0 resets and starts
 * a count of kernel launches; timing != 0 additionally brackets every launch
 * of the dominant kernel -- the Gauss-Jordan trailing update of the lattice
 * step -- with CUDA events recorded on its launch stream.  enable = 0 stops
 * counting. */
int nedmft_instrument(int enable, int timing);

/* Read the counters: kernel launches since nedmft_instrument(1, .), the
 * number of timed (trailing-update) launches, their summed event time in
 * milliseconds, their summed algorithmic work in real flops (8 n_c^2 nb per
 * matrix for a rank-nb Gauss-Jordan step, the complex multiply-add counted
 * as 8 real flops) and their summed algorithmic DRAM bytes (one read and one
 * write of each n_c x n_c working matrix: 2 n_c^2 times its element size).
 * Synchronises on the recorded events.  Any output pointer may be NULL. */
int nedmft_instrument_read(int64_t* launches, int64_t* timed_launches, double* timed_ms, double* timed_flops,
                           double* timed_bytes);

/* ---------------------------------------------------------------- grid */

/* Contour grid, Sec. II Eqs. time_discrete and integration_weights, with
 * the first-branch sign fixed by the stated range (t_j = t_min + j dt) and
 * the imaginary step dtau as a parameter (t = t_min - i dtau k).
 * Host only.  t_host / w_host (length n_c each) may be NULL for a size
 * query.  Fails with NEDMFT_EINVAL unless (t_max - t_min)/dt and beta/dtau
 * are positive integers to within 1e-9 relative. */
int nedmft_contour_grid(double t_min, double t_max, double dt, double beta,
                        double dtau, nedmft_contour* out,
                        nedmft_c128* t_host, nedmft_c128* w_host);

/* Gauss-Hermite rule for the weight exp(-x^2)/sqrt(pi) (Sec. II quadrature
 * paragraph; Eq. joint_dos), weights summing to 1, nodes ascending.
 * Host only.  n in [1, 512]. */
int nedmft_gauss_hermite(int32_t n, double* x_host, double* w_host);

/* Product grid over (eps, ebar), q = a*n + b (eps index outer):
 * eps[q] = x_a, ebar[q] = x_b, wq[q] = w_a w_b.  Host only, arrays of n*n. */
int nedmft_quadrature_grid(int32_t n, double* eps_host, double* ebar_host,
                           double* wq_host);

/* The average of the N- and (N+1)-point product grids (Sec. II: averaging
 * the two Gaussian quadratures works better than one 2N+1 rule): n^2 points
 * of the n-point grid followed by (n+1)^2 points of the (n+1)-point grid,
 * every weight halved.  Host only; arrays of n^2 + (n+1)^2.  n in [1, 511]. */
int nedmft_quadrature_grid_avg(int32_t n, double* eps_host, double* ebar_host,
                               double* wq_host);

/* ---------------------------------------------------------------- diagnostics */

/* Equal-time moments of the retarded Green's function (Sec. II, the
 * paragraph on moments after Eq. current_def), on the upper-branch times t_m,
 * m = 0 .. N_t - 1.  With G^R(t, t') = G^>(t, t') - G^<(t, t') read from the
 * contour matrix (G^> = element (lower-branch row of t, upper row of t'),
 * G^< = (upper row of t, lower row of t'); the lower-branch row of t_m is
 * 2 N_t - m) and f(s) = i G^R(t_m + s/2, t_m - s/2) = mu0 - i mu1 s - mu2 s^2/2
 * + O(s^3), the quadratic through s = 2 dt, 4 dt, 6 dt gives mu0, mu1, mu2
 * (exact values at half filling: 1, 0, 1/2 + U^2/4; the discrete ones carry
 * O(dt) errors that the dt -> 0 extrapolation removes).
 *   gloc_d: N_c x N_c complex128 on the device (any contour Green's function).
 *   mu0_d, mu1_d, mu2_d: N_t doubles each, NaN where t_m +- 3 dt leaves the
 *   real-time window; dens_d: N_t doubles, n(t_m) = -i G^<(t_m, t_m).  Any
 *   output may be NULL.  Stream-ordered; EINVAL for a NULL gloc or a bad contour. */
int nedmft_moments(const nedmft_contour* c, const nedmft_c128* gloc_d,
                   double* mu0_d, double* mu1_d, double* mu2_d, double* dens_d,
                   void* stream);

/* Nonequilibrium density of states (Eqs. gr_omega, dos_def):
 * rho(T, omega) = -Im G^R(T, omega) / pi with G^R(T, omega) the integral over
 * t_rel >= 0 of exp(i omega t_rel) G^R(T + t_rel/2, T - t_rel/2), evaluated by
 * the trapezoid rule over the symmetric pairs (t_{m+k}, t_{m-k}),
 * k = 0 .. min(m, N_t - 1 - m), step 2 dt, with no window.
 *   m_d: n_avg average-time indices T = t_m on the device (an index outside
 *   [0, N_t) yields NaN); omega_d: n_omega frequencies on the device;
 *   rho_d: n_avg x n_omega doubles, row-major.  With n_avg or n_omega zero
 *   nothing is written and the arrays may be NULL.  Stream-ordered. */
int nedmft_dos(const nedmft_contour* c, const nedmft_c128* gloc_d,
               const int32_t* m_d, int32_t n_avg, const double* omega_d,
               int32_t n_omega, double* rho_d, void* stream);

/* ---------------------------------------------------------------- G0 */

/* Noninteracting contour Green's function of Eq. g_contour_non_final2 for
 * nq points: g0_d[q][i][j] = G0_{eps_q, ebar_q}(t_i, t_j), with the contour
 * theta function equal to 1 for i >= j.  eps_d, ebar_d: device, nq doubles.
 * g0_d: device, nq * n_c * n_c nedmft_c128.  Evaluated in a log-stable form
 * (every magnitude <= 1).  Stream-ordered. */
int nedmft_g0_build(const nedmft_contour* c, const nedmft_model* m,
                    const double* eps_d, const double* ebar_d, int32_t nq,
                    nedmft_c128* g0_d, void* stream);

/* ---------------------------------------------------------------- lattice */

/* Workspace bytes nedmft_lattice_gloc / nedmft_current need for this contour,
 * point count and precision.  `batch` = points solved concurrently
 * (0 = library default for n_c).  Returns 0 on a bad argument. */
size_t nedmft_lattice_workspace_size(const nedmft_contour* c, int32_t nq,
                                     nedmft_precision prec, int32_t batch);

/* The lattice step (Eq. g_loc and Eq. current_def):
 *   gloc = sum_q wq[q] G_q,   G_q = [(I - G0_q S)^-1 G0_q] = (B_q - S)^-1,
 *   S = W Sigma W (Eq. matrix_multiply), B_q = G0_q^-1 (bidiagonal + one
 *   boundary element, built in closed form),
 *   j[m]      = Re[ i sum_q wq[q] ebar_q(t_m) G_q[m][2 N_t - m] ],
 *   j_imag[m] = Im[ same ]      (vanishes for the exact solution),
 * for the upper-branch times t_m = t_min + m dt, m = 0..N_t-1, with
 * ebar_q(t) = ebar cos(Et) + eps sin(Et) for t > 0, ebar otherwise.
 * Points are summed in ascending q in FP64, so the result is deterministic.
 *   sigma_d: device, n_c x n_c self-energy Sigma(t_i, t_j).
 *   eps_d, ebar_d, wq_d: device, nq doubles each.
 *   gloc_d: device, n_c x n_c output (overwritten).
 *   j_d, j_imag_d: device, n_t doubles each, or NULL to skip.
 *   ws_d / ws_bytes: workspace of at least
 *     nedmft_lattice_workspace_size(c, nq, prec, batch) bytes, where batch is
 *     the value of the environment-free default (0).
 * Stream-ordered; no host synchronisation. */
int nedmft_lattice_gloc(const nedmft_contour* c, const nedmft_model* m,
                        const nedmft_c128* sigma_d, const double* eps_d,
                        const double* ebar_d, const double* wq_d, int32_t nq,
                        nedmft_precision prec, nedmft_c128* gloc_d,
                        double* j_d, double* j_imag_d, void* ws_d,
                        size_t ws_bytes, void* stream);

/* The current alone (Eq. current_def): one lattice pass whose G_loc stays in
 * the workspace.  Same arguments and workspace as nedmft_lattice_gloc. */
int nedmft_current(const nedmft_contour* c, const nedmft_model* m,
                   const nedmft_c128* sigma_d, const double* eps_d,
                   const double* ebar_d, const double* wq_d, int32_t nq,
                   nedmft_precision prec, double* j_d, double* j_imag_d,
                   void* ws_d, size_t ws_bytes, void* stream);

/* Batch autotuner (choices the paper leaves to the machine: how many
 * quadrature points, its independent solves of Sec. II, run at once, and how
 * the solves are blocked).  Times one lattice step (after an untimed one) for
 * every candidate number of points per batch that fits the workspace and, on
 * the tensor-core path above 512 rows, for both Gauss-Jordan block widths
 * (256 columns with N_c padded to a multiple of 256, 128 with a multiple of
 * 128; by default the library takes 128 only where that padding saves more
 * than a fifth of the flops), and records the fastest pair for this
 * (n_c, nq, prec); later calls of nedmft_lattice_workspace_size(..., batch =
 * 0), nedmft_lattice_gloc, nedmft_current and the DMFT drivers in this
 * process use it.  Tune before sizing workspaces: a workspace sized for the
 * former choice may be too small afterwards (ENOMEM, never an overrun).
 *   Arguments 1-8 as nedmft_lattice_gloc (Sigma and the points are the ones
 *   to time with); candidates: n_candidates batch sizes on the host;
 *   best_batch, best_ms: host outputs (may be NULL).  Synchronises the stream.
 *   ENOMEM if no candidate fits ws_bytes. */
int nedmft_lattice_autotune(const nedmft_contour* c, const nedmft_model* m,
                            const nedmft_c128* sigma_d, const double* eps_d,
                            const double* ebar_d, const double* wq_d,
                            int32_t nq, nedmft_precision prec,
                            const int32_t* candidates, int32_t n_candidates,
                            int32_t* best_batch, double* best_ms,
                            void* ws_d, size_t ws_bytes, void* stream);

/* Points per batch that nedmft_lattice_gloc uses for (c, nq, prec): the tuned
 * size if nedmft_lattice_autotune ran for them, else the default (clamped to
 * nq).  0 for invalid arguments. */
int32_t nedmft_lattice_batch(const nedmft_contour* c, int32_t nq,
                             nedmft_precision prec);

/* Record a choice for (c, nq, prec) as nedmft_lattice_autotune would: batch
 * points per batch (0 = the default) and Gauss-Jordan block width (0 = the
 * default, 128 or 256; 256 applies only where N_c pads to a multiple of 256
 * from 512 up, otherwise 128 is used).  Same effect on later calls as a tuning
 * run.  EINVAL for other values. */
int nedmft_lattice_set_tuning(const nedmft_contour* c, int32_t nq,
                              nedmft_precision prec, int32_t batch,
                              int32_t width);

/* Columns per Gauss-Jordan step that nedmft_lattice_gloc uses for (c, nq,
 * prec): 32 on the FP64 path; 128 or 256 on the tensor-core path (the tuned
 * width if nedmft_lattice_autotune ran for them, else the default).  0 for
 * invalid arguments. */
int32_t nedmft_lattice_block_width(const nedmft_contour* c, int32_t nq,
                                   nedmft_precision prec);

/* The lattice step for small contours (n_c <= 112), FP64 arithmetic, with
 * no workspace argument and no device allocation of any kind.  The paper has
 * no counterpart to this entry point: it exists for callers that cannot
 * allocate device memory -- for example a host physics code that manages all
 * device memory itself and only hands this library its input and output
 * buffers, or a plugin running under a framework whose caching allocator owns
 * the device and exposes no raw workspace to it.
 *   Arguments and results are those of nedmft_lattice_gloc with prec =
 *   NEDMFT_FP64 (points are inverted 32 at a time).
 *   Scratch: a fixed device array of about 6.6 MB inside the library, one
 *   per GPU that loads the library, held until the process exits.  The
 *   first call on a device looks up that array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it.
 *   Calls share the array: two calls whose work overlaps on the GPU (on
 *   different streams, or from different host threads) race and corrupt each
 *   other's results.  Every scratch byte a call reads was written earlier in
 *   the same call, so nothing needs clearing between calls.
 *   Errors: NEDMFT_EINVAL for n_c > 112, nq < 1, a NULL pointer or an invalid
 *   contour (message in nedmft_last_error); NEDMFT_ECUDA if the address
 *   lookup or a launch fails.  Stream-ordered. */
int nedmft_lattice_gloc_static(const nedmft_contour* c, const nedmft_model* m,
                               const nedmft_c128* sigma_d, const double* eps_d,
                               const double* ebar_d, const double* wq_d,
                               int32_t nq, nedmft_c128* gloc_d, double* j_d,
                               double* j_imag_d, void* stream);

/* dt -> 0 extrapolation of the current (Sec. II, Lagrange extrapolation):
 * out[e] = sum_r L_r(0) j_r(t_e), L_r the Lagrange basis polynomials of the
 * k step sizes dts_host[r] (k = 3: quadratic, 4: cubic, ...), each j_r read
 * at t_e by linear interpolation on its own upper-branch grid
 * t_min_host[r] + m dts_host[r], m < n_t_host[r].  j_d: host array of k
 * device pointers; t_out_d, out_d: device, n_out doubles.  Times outside a
 * run's grid set *bad_d (device int) to 1 and leave their output unset.
 * k in [1, 16], distinct dts.  Stream-ordered. */
int nedmft_extrapolate_current(int32_t k, const double* dts_host,
                               const double* t_min_host,
                               const int32_t* n_t_host, const double* const* j_d,
                               const double* t_out_d, int32_t n_out,
                               double* out_d, int32_t* bad_d, void* stream);

/* ---------------------------------------------------------------- impurity */

/* Workspace bytes for nedmft_impurity_update. */
size_t nedmft_impurity_workspace_size(const nedmft_contour* c);

/* One Falicov-Kimball impurity step in FP64 (Eqs. effective_medium,
 * dynamical_mean_field, g_imp_solve; the M matrix of the discretised
 * (i d/dt + mu) delta_c; the operator inverse of Eq.
 * matrix_inverse_discrete):
 *   A0 = inv(G_loc) + S,  A1 = A0 + D with D = i [M(mu - U) - M(mu)],
 *   G_imp = (1 - w1) inv(A0) + w1 inv(A1),
 *   sigma_new = W^-1 (A0 - inv(G_imp)) W^-1.
 * Evaluated with two inversions instead of four: with A_h = A0 + (1 - w1) D,
 * G_imp = inv(A0) A_h inv(A1), so A0 - inv(G_imp) = -w1 D + w1 (1 - w1)
 * D inv(A_h) D, and D (one entry per row, -U W_j at (j, j-1), +U W_0 at
 * (0, N-1)) makes the last product a gather.  Inversions: blocked
 * Gauss-Jordan (32 columns per step) whose pivot rows a tournament of
 * partial-pivoting rounds on 256-row chunks chooses, their trailing updates
 * on the tensor cores with FP64 accuracy (each operand row cut into seven
 * 7-bit integer digits, digit products exact in FP32); each step's tournament
 * and pivot block run one step ahead on a second, library-owned stream of
 * the highest priority (one per device and host thread, made by the thread's
 * first call and kept, with its two events, until the process ends), forked
 * from and joined back into `stream` with events; to
 * capture the call into a CUDA graph, call it once outside the capture first
 * (nedmft_dmft_solve does so for its own graph).  gimp_d may be NULL;
 * if given, G_imp = inv(A0 - W sigma_new W) costs a third inversion.
 * sigma_new_d may not alias gloc_d or sigma_d.  Stream-ordered with respect
 * to `stream`. */
int nedmft_impurity_update(const nedmft_contour* c, const nedmft_model* m,
                           const nedmft_c128* gloc_d,
                           const nedmft_c128* sigma_d,
                           nedmft_c128* sigma_new_d, nedmft_c128* gimp_d,
                           void* ws_d, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- learned warm start */

/* A multilayer perceptron whose prediction starts the DMFT loop in place of
 * the equilibrium self-energy the paper starts from (Sec. II, the summary of
 * the iterative algorithm).  The result of the loop does not depend on the
 * guess; only the number of iterations does.
 * What it predicts: the impurity Green's function X = inv(A0 + (1 - w1) D)
 * of the impurity step (nedmft_impurity_update), from which the self-energy
 * follows exactly: W Sigma W = -w1 D + w1 (1 - w1) D X D.  X is smooth along
 * the contour and of order one for any U; Sigma itself carries ratios of the
 * step sizes in the columns at the ends of the branches, which no network that
 * does not know the grid could predict.
 * Network: 17 features -> 4 tanh layers of 256 -> 2 outputs (Re, Im of X).
 * Parameters: one FP32 array of nedmft_mlp_param_count() values, layer by
 * layer, each layer a row-major (in x out) weight block followed by its
 * out biases.  The GEMMs run on the tensor cores: operands rounded to bf16,
 * sums in FP32; the weight gradients add their K slices in a fixed order, so
 * nedmft_mlp_grad is deterministic.
 * Features of the pair (t_a, t_b), chosen to carry over from short training
 * contours to longer ones: U/2.5, E/4, tanh(Re(t_a - t_b)/3), then for t_a
 * and t_b in turn (real part r, imaginary depth tau) tanh(max(r, 0)/3) (the
 * elapsed field time, saturating), min(r, 0)/5, tau/beta and the one-hot
 * branch (upper, lower, imaginary); then the contour order (1 for a >= b) and
 * dt / 0.1 (the discrete X differs from the continuum one at order dt).
 * Targets: X[a][b] = [W Sigma W + w1 D]_{a+1, b-1} / (w1 (1 - w1) d_{a+1} d_b)
 * / scale (indices mod N; d_i = -U W_i for i >= 1, d_0 = +U W_0). */
int32_t nedmft_mlp_param_count(void);
/* Workspace bytes for n samples of nedmft_mlp_forward / nedmft_mlp_grad. */
size_t nedmft_mlp_workspace_size(int32_t n);
/* y_d (n x 2) = network(x_d (n x 17)).  Device arrays. */
int nedmft_mlp_forward(const float* params_d, const float* x_d, int32_t n,
                       float* y_d, void* ws_d, size_t ws_bytes, void* stream);
/* Mean-squared error over the n x 2 outputs against target_d and its
 * gradient with respect to every parameter (grad_d, same layout as the
 * parameters); *loss_d (device float) receives the loss. */
int nedmft_mlp_grad(const float* params_d, const float* x_d,
                    const float* target_d, int32_t n, float* grad_d,
                    float* loss_d, void* ws_d, size_t ws_bytes, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at step number step >= 1. */
int nedmft_mlp_adam(float* params_d, const float* grad_d, float* m1_d,
                    float* m2_d, int32_t step, float lr, void* stream);
/* Features of every (t_a, t_b) pair of the contour (dt feature c->dt): x_d is n_c^2 x 17. */
int nedmft_mlp_features(const nedmft_contour* c, const nedmft_model* m,
                        float* x_d, void* stream);
/* Targets of every pair from a self-energy: t_d is n_c^2 x 2. */
int nedmft_mlp_target(const nedmft_contour* c, const nedmft_model* m,
                      const nedmft_c128* sigma_d, double scale, float* t_d,
                      void* stream);
/* A random minibatch (a counter-based hash of seed, step and row picks each
 * sample) of batch rows from n_total samples: xb_d batch x 17, tb_d batch x 2. */
int nedmft_mlp_sample(const float* x_d, const float* t_d, int64_t n_total,
                      int32_t batch, uint64_t seed, int64_t step, float* xb_d,
                      float* tb_d, void* stream);
/* Workspace bytes for nedmft_sigma_warm_start on this contour. */
size_t nedmft_sigma_warm_start_workspace_size(const nedmft_contour* c);
/* The warm start for nedmft_dmft_solve's sigma_init_d on contour c: the
 * network's X on this contour's times with the dt feature set to each of the
 * n_dt training steps dts_host[k] (1 <= n_dt <= 8, distinct, > 0), combined
 * by Lagrange extrapolation to c->dt (the paper's dt -> 0 extrapolation, here
 * to the contour's own step), then sigma_d = W^-1 (-w1 D + w1 (1 - w1) D X D)
 * W^-1.  Needs U != 0 and 0 < w1 < 1.  Stream-ordered. */
int nedmft_sigma_warm_start(const nedmft_contour* c, const nedmft_model* m,
                            const float* params_d, int32_t n_dt,
                            const double* dts_host, nedmft_c128* sigma_d,
                            void* ws_d, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- loop */

/* Workspace bytes for nedmft_dmft_solve. */
size_t nedmft_dmft_workspace_size(const nedmft_contour* c, int32_t n_quad,
                                  nedmft_precision prec);

/* The DMFT loop of Sec. II on an n_quad x n_quad Gauss-Hermite grid:
 * lattice step, convergence test max|G_new - G_old| / max|G_new| < tol,
 * impurity step, Sigma <- Sigma_new (no mixing).  Sigma starts at
 * sigma_init_d (device, n_c x n_c) or at 0 if it is NULL.
 * Outputs (device): sigma_d (the Sigma that produced the returned G_loc),
 * gloc_d, j_d (n_t doubles, or NULL).  Host outputs: *iters (lattice steps
 * taken), *err (last convergence error).  Synchronises `stream` once per
 * iteration (one scalar read).  Returns NEDMFT_ENOTCONV if max_iter lattice
 * steps did not converge. */
int nedmft_dmft_solve(const nedmft_contour* c, const nedmft_model* m,
                      int32_t n_quad, nedmft_precision prec,
                      const nedmft_c128* sigma_init_d, double tol,
                      int32_t max_iter, nedmft_c128* sigma_d,
                      nedmft_c128* gloc_d, double* j_d, int32_t* iters,
                      double* err, void* ws_d, size_t ws_bytes, void* stream);

/* Several DMFT runs at once (the paper's workflow: runs at several (U, E)
 * and several dt for the Lagrange extrapolation of Sec. II): run r has its own contour (n_c may differ between runs) and model,
 * all share n_quad and prec.  Every sweep takes one iteration of each run that
 * is still active -- impurity step, lattice step, convergence norm, all on one
 * stream without a host sync in between -- and synchronises once; a run leaves
 * the sweep when it converges (same norm as nedmft_dmft_solve) or reaches
 * max_iter.  The points of different runs are not mixed within a Gauss-Jordan
 * batch: each run's own points fill its batches.
 *   contours, models: host arrays of n_runs; sigma_init_d: NULL (all runs
 *   start at Sigma = 0) or a host array of n_runs device pointers, each NULL
 *   or N_c(r)^2 complex128; sigma_d, gloc_d: host arrays of n_runs device
 *   pointers (N_c(r)^2 complex128 outputs, as nedmft_dmft_solve); j_d: NULL
 *   or a host array of n_runs device pointers (N_t(r) doubles, each may be
 *   NULL); iters, errs, converged: host arrays of n_runs (may be NULL).
 *   Workspace: nedmft_dmft_batch_workspace_size bytes, 256-byte aligned.
 *   Returns ENOTCONV (> 0) if any run did not converge. */
size_t nedmft_dmft_batch_workspace_size(int32_t n_runs,
                                        const nedmft_contour* contours,
                                        int32_t n_quad, nedmft_precision prec);
int nedmft_dmft_solve_batch(int32_t n_runs, const nedmft_contour* contours,
                            const nedmft_model* models, int32_t n_quad,
                            nedmft_precision prec,
                            const nedmft_c128* const* sigma_init_d, double tol,
                            int32_t max_iter, nedmft_c128* const* sigma_d,
                            nedmft_c128* const* gloc_d, double* const* j_d,
                            int32_t* iters, double* errs, int32_t* converged,
                            void* ws_d, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NEDMFT_H */
