"""The Hessian apply split over two processes (section 3: a sum over sources):
each gloo rank owns half of the shots, computes its block's extended image on
the GPU (hv_hessian_apply_partial), the images are gathered on the host and
summed in rank order (parallel.sharded_hessian_apply), and each rank folds the
sum once.  Both ranks share the one GPU here; their kernels never wait on one
another (the only exchange is the host-side gather).  The result must equal the
one-process apply of all shots (the same 8-shot groups: FP64 rounding only) and
be bitwise the same on both ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    from paper_2507_10804_gb300 import synth
    from paper_2507_10804_gb300.hv import Problem
    from paper_2507_10804_gb300.parallel import shard_problem, sharded_hessian_apply
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.workload(3, nt=200, ns=16)
    w.v = w.v[[5, 60]]
    P = shard_problem(Problem, w, rank, world, device="cuda:0")
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda:0")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda:0")
    Hv = sharded_hessian_apply(lambda: P.hessian_apply_partial(m, v, ckpt=10).cpu(),
                               lambda ext: P.fold(ext.to("cuda:0"), torch.float64))
    np.save(os.path.join(out_dir, f"hv{rank}.npy"), Hv.cpu().numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_split_the_shots(tmp_path):
    from paper_2507_10804_gb300 import synth
    from paper_2507_10804_gb300.hv import Problem
    mp.start_processes(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    a, b = np.load(tmp_path / "hv0.npy"), np.load(tmp_path / "hv1.npy")
    assert np.array_equal(a, b)
    w = synth.workload(3, nt=200, ns=16)
    w.v = w.v[[5, 60]]
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    full = Problem.from_workload(w).hessian_apply(m, v, ckpt=10, out_dtype=torch.float64).cpu().numpy()
    for j in range(2):
        assert np.linalg.norm(a[j] - full[j]) < 1e-12 * np.linalg.norm(full[j])
