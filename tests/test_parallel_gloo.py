"""Multi-rank logic on CPU ranks (gloo, world size 2): shot sharding, the
fixed-order sum and the max-over-ranks timing used by bench.py under torchrun.
The per-rank H v here is the FP64 oracle on the rank's shots."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2507_10804_gb300.parallel import fixed_order_allreduce, max_over_ranks, shard_shots


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
    mine = shard_shots(w.ns, rank, world)
    w_r = ragged_workload(nt=60, ns=5, nr=6, k=2)
    idx = list(mine)
    from paper_2507_10804_gb300.synth import Acquisition
    w_r.acq = Acquisition(w.acq.src_iz[idx], w.acq.src_ix[idx], w.acq.rec_iz[idx], w.acq.rec_ix[idx])
    part = O.hessian_apply(oracle_problem(w_r), w.m, w.v, nthreads=1)
    total = fixed_order_allreduce(torch.from_numpy(part)).numpy()
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
    assert float(np.load(tmp_path / "t0.npy")[0]) == float(np.load(tmp_path / "t1.npy")[0]) == 1.5
