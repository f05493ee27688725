"""The multi-rank host path on CPU: gloo ranks split the quadrature points
of a lattice step into contiguous blocks, each computes its partial G_loc and
current (with the CPU oracle standing in for the per-GPU library call), and
the rank-ordered sum must equal the single-process result on both ranks; the
job time is the slowest rank's."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import nedmft_oracle as O
from paper_0711_0999_gb300 import sharding


@pytest.mark.parametrize("n,world", [(0, 1), (7, 1), (7, 2), (16, 3), (2809, 8), (3, 5)])
def test_block_range_partitions(n, world):
    seen = []
    sizes = []
    for r in range(world):
        lo, hi = sharding.block_range(n, world, r)
        seen.extend(range(lo, hi))
        sizes.append(hi - lo)
    assert seen == list(range(n))
    assert max(sizes) - min(sizes) <= 1


def test_block_range_rejects():
    with pytest.raises(ValueError):
        sharding.block_range(5, 0, 0)
    with pytest.raises(ValueError):
        sharding.block_range(5, 2, 2)


ARGS = (-2, 4, 0.2, 10, 0.5)


def _case(n_quad=5):
    c = O.contour_grid(*ARGS)
    from paper_0711_0999_gb300.synth import workload_sigma
    sig = workload_sigma(c.t, c.w, 0.5, seed=5)
    eps, ebar, wq = O.quadrature_points(n_quad)
    return c, O.Model(U=0.5, E=1.0), sig, eps, ebar, wq


def _rank_main(rank, world, port, out_dir, n_quad):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c, m, sig, eps, ebar, wq = _case(n_quad)
        lo, hi = sharding.block_range(len(wq), world, rank)
        if hi > lo:
            gl, jc = O.lattice_gloc(c, m, sig, eps[lo:hi], ebar[lo:hi], wq[lo:hi])
        else:  # a rank without points adds zeros, as lattice_gloc_sharded does
            gl, jc = np.zeros((c.n_c, c.n_c), complex), np.zeros(c.n_t, complex)
        g_sum = sharding.ordered_sum(torch.as_tensor(gl))
        j_sum = sharding.ordered_sum(torch.as_tensor(jc.real.copy()))
        t = sharding.max_over_ranks(1.0 + rank, "cpu")
        np.save(os.path.join(out_dir, f"g{rank}.npy"), g_sum.numpy())
        np.save(os.path.join(out_dir, f"j{rank}.npy"), j_sum.numpy())
        np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


# 25 points on 2 ranks (13 + 12) and on 3 (9 + 8 + 8); 1 point on 2 ranks (rank 1 empty)
@pytest.mark.parametrize("world,n_quad", [(2, 5), (3, 5), (2, 1)])
def test_gloo_ranks_sum_like_one_process(tmp_path, world, n_quad):
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), n_quad), nprocs=world, join=True)
    c, m, sig, eps, ebar, wq = _case(n_quad)
    g_ref, j_ref = O.lattice_gloc(c, m, sig, eps, ebar, wq)
    for r in range(world):
        g = np.load(tmp_path / f"g{r}.npy")
        j = np.load(tmp_path / f"j{r}.npy")
        assert np.abs(g - g_ref).max() <= 1e-13 * np.abs(g_ref).max()
        assert np.abs(j - j_ref.real).max() <= 1e-13 * max(1.0, np.abs(j_ref.real).max())
        assert float(np.load(tmp_path / f"t{r}.npy")[0]) == float(world)  # the slowest rank's time
    # every rank holds the same bits (the sum runs in rank order on each)
    for r in range(1, world):
        assert np.array_equal(np.load(tmp_path / "g0.npy"), np.load(tmp_path / f"g{r}.npy"))
        assert np.array_equal(np.load(tmp_path / "j0.npy"), np.load(tmp_path / f"j{r}.npy"))


@pytest.mark.gpu
def test_sharded_lattice_step_single_rank_gpu():
    # the GPU entry point of the sharded step, in a one-rank group: the same
    # G_loc and current as the plain lattice step
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_0711_0999_gb300 import api
    from paper_0711_0999_gb300.build import build_library
    build_library()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        c, m, sig, eps, ebar, wq = _case()
        g = api.contour_grid(*ARGS)
        mc = api.make_model(0.5, 1.0)
        s = torch.as_tensor(sig, device="cuda")
        gl, j, ji = sharding.lattice_gloc_sharded(g, mc, s, eps, ebar, wq, precision="fp64")
        ref, jr, _ = api.lattice_gloc(g, mc, s, eps, ebar, wq, precision="fp64")
        torch.cuda.synchronize()
        assert float((gl - ref).abs().max()) == 0.0 and float((j - jr).abs().max()) == 0.0
    finally:
        dist.destroy_process_group()
