"""Multi-rank logic on CPU ranks (gloo, world size 2): the shot sharding, the
sharded Hessian apply (per-rank extended images summed in rank order, folded
once) and the max-over-ranks timing that bench.py uses under torchrun.  The
per-rank solve here is the FP64 oracle on the rank's shots (its extended image
and its fold), so the sharding and the sum are the product's own functions."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2507_10804_gb300.parallel import (fixed_order_allreduce, max_over_ranks, shard_problem, shard_shots,
                                             sharded_hessian_apply)


def test_shard_shots_partitions_in_order():
    for ns in (1, 2, 7, 32):
        for world in (1, 2, 3, 8):
            got = [s for r in range(world) for s in shard_shots(ns, r, world)]
            assert got == list(range(ns))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import oracle as O
    from tests._helpers import oracle_problem, ragged_workload
    w = ragged_workload(nt=60, ns=5, nr=6, k=2)

    def oracle_cls(nz, nx, nb, h, nt, dt, f0, t0, vmax, src_iz, src_ix, rec_iz, rec_ix, R, sigma, device):
        return O.Problem(nz=nz, nx=nx, nb=nb, h=h, nt=nt, dt=dt, f0=f0, t0=t0, vmax=vmax, src_iz=src_iz,
                         src_ix=src_ix, rec_iz=rec_iz, rec_ix=rec_ix, R=R, sigma=sigma)

    P_r = shard_problem(oracle_cls, w, rank, world)
    assert P_r.src_iz.size == len(shard_shots(w.ns, rank, world))

    def fold(ext):
        return torch.from_numpy(np.stack([O.fold(P_r, e) for e in ext.numpy()]))

    total = sharded_hessian_apply(lambda: torch.from_numpy(O.hessian_image(P_r, w.m, w.v, nthreads=1)), fold).numpy()
    slowest = max_over_ranks(0.5 + rank)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), total)
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([slowest]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_hessian_fixed_order_sum(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    from oracle import oracle as O
    from tests._helpers import oracle_problem, ragged_workload
    w = ragged_workload(nt=60, ns=5, nr=6, k=2)
    full = O.hessian_apply(oracle_problem(w), w.m, w.v, nthreads=1)
    r0, r1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)                              # identical on every rank
    assert np.allclose(r0, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    part0 = O.hessian_apply(oracle_problem(w), w.m, w.v, nthreads=1)
    assert np.abs(r0 - part0).max() <= 1e-12 * np.abs(full).max()
    assert float(np.load(tmp_path / "t0.npy")[0]) == float(np.load(tmp_path / "t1.npy")[0]) == 1.5
