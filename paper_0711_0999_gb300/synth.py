"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module generates inputs only.  It holds none of the lattice-step
arithmetic: it never builds a Green's function, never solves, never sums a
quadrature.  Both the CUDA path and the CPU oracle receive the arrays it
returns, so neither side's expected values depend on the other.

The self-energy workload is shaped like the converged Falicov-Kimball
self-energy of small runs: a point-split band of height ``h/|W|`` on the first
subdiagonal (the static ``U <w_1>`` part, a contour delta function placed off
the diagonal with the boundary element carrying the opposite sign) plus a
smooth, dense, two-time kernel of magnitude ``a``.
"""

from __future__ import annotations

import numpy as np

SEED_DEFAULT = 20071101


def synthetic_sigma(t: np.ndarray, w: np.ndarray, band: float, amp: float,
                    seed: int = SEED_DEFAULT, rank: int = 6) -> np.ndarray:
    """Return a complex128 N_c x N_c self-energy workload.

    ``t``/``w`` are the contour times and weights (complex, length N_c);
    ``band`` is the height of the subdiagonal band times its weight; ``amp``
    the scale of the smooth part.  Deterministic in ``seed``.
    """
    t = np.asarray(t, dtype=np.complex128)
    w = np.asarray(w, dtype=np.complex128)
    n = t.shape[0]
    rng = np.random.default_rng(seed)
    tr = t.real
    tau = -t.imag
    sig = np.zeros((n, n), dtype=np.complex128)
    # smooth part: a sum of separable damped oscillations in (t, t')
    for _ in range(rank):
        k1, k2 = rng.uniform(-1.5, 1.5, size=2)
        d1, d2 = rng.uniform(0.05, 0.4, size=2)
        c = (rng.normal() + 1j * rng.normal()) / np.sqrt(2 * rank)
        u = np.exp(1j * k1 * tr - d1 * tau)
        v = np.exp(-1j * k2 * tr - d2 * tau)
        sig += amp * c * np.outer(u, v)
    sig += amp * 0.05 * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    # point-split band: Sigma_{j, j-1} = band / W_{j-1}, boundary element -band / W_{N-1}
    idx = np.arange(1, n)
    sig[idx, idx - 1] += band / w[idx - 1]
    sig[0, n - 1] -= band / w[n - 1]
    return sig


def workload_sigma(t, w, U: float, seed: int = SEED_DEFAULT) -> np.ndarray:
    """The default self-energy workload for interaction U (band U/2, smooth part U^2/8)."""
    return synthetic_sigma(t, w, band=U / 2.0, amp=U * U / 8.0, seed=seed)
