"""Write the oracle's full-grid lattice step of the N_c = 1500 production workload.

The production workload: U = E = 1, beta = 10, t in [-5, 30] with dt = 0.05,
dtau = 0.1 (N_c = 1500), every one of the 53 x 53 Gauss-Hermite points with its
own weight (2809 Dyson solves), and the seeded synthetic self-energy of
``synth.workload_sigma`` (seed 20071101).  The sum over points is the oracle's
literal ``sum_q w_q (I - G0_q S)^-1 G0_q`` (Eq. g_loc) and its current
(Eq. current_def); the points are split into contiguous chunks that worker
processes sum in ascending q, and the chunk sums are added in chunk order.

Stored (``cfg1_lattice_oracle.npz``), for a test that compares the CUDA path
element by element without re-running 2809 CPU solves:
  * ``max_abs``: max_ij |G_loc|, the scale of the relative error;
  * ``rows``/``cols``/``vals``: G_loc at the diagonal, at whole rows and columns
    at the branch boundaries and at seeded random entries;
  * ``proj``: u_k^T G_loc v_k for the seeded random sign vectors of
    ``projection_vectors`` (entries +-1/N_c, so |u^T dG v| <= max|dG| and the
    element tolerance bounds them), which see an error anywhere in the matrix;
  * ``j``: the complex current i sum_q w_q ebar_q(t) G^<_q(t, t) at every t_m;
  * ``sigma_sha256``: a hash of the self-energy, so a test can tell whether
    its own seeded input is the one these values came from;
  * ``eps``/``ebar``/``wq``: the points and weights used (the Golub-Welsch
    eigensolver differs in the last bits between LAPACK builds, so a test
    compares its own within a tolerance rather than by hash).

Calls only ``oracle/`` (and the seeded input generator).  Run from the
repository root:  python tests/golden/make_cfg1_golden.py [processes]
"""

from __future__ import annotations

import hashlib
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg1_lattice_oracle.npz")
ARGS = (-5.0, 30.0, 0.05, 10.0, 0.1)
U, E, NQUAD = 1.0, 1.0, 53
N_RANDOM = 8192
N_PROJ = 32
SAMPLE_SEED = 15002809


def inputs():
    from oracle import nedmft_oracle as O
    from paper_0711_0999_gb300.synth import workload_sigma

    c = O.contour_grid(*ARGS)
    sigma = workload_sigma(c.t, c.w, U)
    eps, ebar, wq = O.quadrature_points(NQUAD)
    return c, sigma, eps, ebar, wq


def sigma_hash(sigma) -> str:
    return hashlib.sha256(np.ascontiguousarray(sigma).tobytes()).hexdigest()


def same_inputs(d, sigma, eps, ebar, wq, tol: float = 1e-13) -> bool:
    """Whether stored values `d` came from these inputs: the same self-energy
    bits, points and weights equal to within `tol` (relative)."""
    if str(d["sigma_sha256"]) != sigma_hash(sigma):
        return False
    return all(np.abs(d[k] - a).max() <= tol * max(1.0, np.abs(a).max()) for k, a in
               (("eps", eps), ("ebar", ebar), ("wq", wq)))


def sample_positions(n_c: int, n_t: int):
    """Entries the file stores: the diagonal, whole rows and columns at the
    branch boundaries, and seeded random entries."""
    rows, cols = [], []
    d = np.arange(n_c)
    rows.append(d)
    cols.append(d)
    for r in (0, n_t - 1, n_t, 2 * n_t - 1, 2 * n_t, n_c - 1):
        rows.append(np.full(n_c, r))
        cols.append(d)
    for k in (0, n_t, n_c - 1):
        rows.append(d)
        cols.append(np.full(n_c, k))
    rng = np.random.default_rng(SAMPLE_SEED)
    rows.append(rng.integers(0, n_c, N_RANDOM))
    cols.append(rng.integers(0, n_c, N_RANDOM))
    return np.concatenate(rows).astype(np.int64), np.concatenate(cols).astype(np.int64)


def projection_vectors(n_c: int):
    rng = np.random.default_rng(SAMPLE_SEED + 1)
    u = rng.choice([-1.0, 1.0], size=(N_PROJ, n_c)) / n_c
    v = rng.choice([-1.0, 1.0], size=(N_PROJ, n_c)) / n_c
    return u, v


def _chunk(task):
    lo, hi = task
    from oracle import nedmft_oracle as O

    c, sigma, eps, ebar, wq = inputs()
    g, jc = O.lattice_gloc(c, O.Model(U=U, E=E), sigma, eps, ebar, wq, q_indices=range(lo, hi))
    return lo, g, jc


def compute(procs: int) -> dict:
    """The stored quantities (see the module docstring), from the oracle on
    `procs` spawned processes."""
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    c, sigma, eps, ebar, wq = inputs()
    nq = len(wq)
    n_chunks = 4 * procs
    bounds = np.linspace(0, nq, n_chunks + 1).round().astype(int)
    tasks = [(int(bounds[i]), int(bounds[i + 1])) for i in range(n_chunks) if bounds[i + 1] > bounds[i]]
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = sorted(pool.map(_chunk, tasks), key=lambda p: p[0])
    g = np.zeros((c.n_c, c.n_c), np.complex128)
    jc = np.zeros(c.n_t, np.complex128)
    for _, gp, jp in parts:  # chunk order = ascending q
        g += gp
        jc += jp
    rows, cols = sample_positions(c.n_c, c.n_t)
    u, v = projection_vectors(c.n_c)
    proj = np.einsum("ki,ij,kj->k", u, g, v)
    print(f"oracle: {nq} points, {len(tasks)} chunks on {procs} processes, {time.time() - t0:.0f} s")
    return dict(max_abs=np.abs(g).max(), rows=rows, cols=cols, vals=g[rows, cols], proj=proj, j=jc,
                sigma_sha256=sigma_hash(sigma), eps=eps, ebar=ebar, wq=wq, n_c=c.n_c, n_t=c.n_t, nq=nq)


def main():
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    np.savez_compressed(OUT, **compute(procs))
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
