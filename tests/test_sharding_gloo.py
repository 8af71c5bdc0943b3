"""Multi-process path on CPU (gloo, world size 2): each rank evaluates its
block of the batch (paper partition rule), the blocks cover the batch exactly
once, the gathered results equal the single-process ones, timings reduce by
max and the weight gradient by one sum."""
import os
import socket

import numpy as np
import pytest

from paper_2404_06314_gb300 import shard


def test_partition_rule():
    for B, R in [(48, 12), (50, 12), (7, 3), (3, 8), (1024, 2)]:
        spans = [shard.partition(B, R, r) for r in range(R)]
        assert sum(c for _, c in spans) == B
        assert spans[0][0] == 0
        for r in range(1, R):
            assert spans[r][0] == spans[r - 1][0] + spans[r - 1][1]
        extra = B % R
        assert [c for _, c in spans] == [B // R + (r < extra) for r in range(R)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2404_06314_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = W.workload_4q()
    B = 13
    inp = W.make_inputs(c, B, 1000)
    start, count = shard.partition(B, world, rank)
    x, gE = inp.x[start:start + count], inp.gE[start:start + count]
    E = oracle.forward(c, x, inp.w)
    _, gx, gw = oracle.adjoint(c, gE, x, inp.w)
    parts = [None] * world
    dist.all_gather_object(parts, (start, E, gx))
    gws = torch.tensor(gw.sum(0))
    shard.sum_grad_w(gws)
    tmax = shard.max_over_ranks(float(rank + 1))
    if rank == 0:
        np.savez(os.path.join(out_dir, "res.npz"),
                 E=np.concatenate([p[1] for p in sorted(parts, key=lambda t: t[0])]),
                 gx=np.concatenate([p[2] for p in sorted(parts, key=lambda t: t[0])]),
                 gw=gws.numpy(), tmax=tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_2404_06314_gb300 import workloads as W
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = np.load(tmp_path / "res.npz")
    c = W.workload_4q()
    inp = W.make_inputs(c, 13, 1000)
    E = oracle.forward(c, inp.x, inp.w)
    _, gx, gw = oracle.adjoint(c, inp.gE, inp.x, inp.w)
    assert np.array_equal(r["E"], E)
    assert np.array_equal(r["gx"], gx)
    assert np.allclose(r["gw"], gw.sum(0), rtol=0, atol=1e-13)
    assert float(r["tmax"]) == 2.0
