"""Multi-rank logic on CPU with the gloo backend (world size 2).

* The q-sharded self-energy: each rank sums the contributions of its own q
  (Eq. sigma_gw is a sum over q), the ranks all-reduce the partial Sigma, and
  the result equals the single-rank Sigma. This is the one exchange step of
  a q-sharded multi-GPU run.
* The benchmark's max-over-ranks timing reduction.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        sys.path.insert(0, root)
        from oracle import gw as O
        from paper_2406_18479_gb300 import inputs as I
        import bench
        w = I.Workload("shard", (2, 2, 1), 3, 5, 6, 6, 6.0, 0.0, 4.0, 21, solid=True)
        h, v, g = I.make_inputs(w)
        from oracle import grids
        _, F, B = grids.transform_matrices(w.ntau, w.beta, 0)
        q_mine = [q for q in range(w.nk) if q % world == rank]
        p0 = O.polarization(v, g, w.nk3, 2.0, q_list=q_mine)
        _, _, pt_mine = O.screened_interaction(p0, F, B)
        # every rank needs P~ only for its own q: Sigma partial over those q
        pt_full = np.zeros((w.nk,) + pt_mine.shape[1:], complex)
        pt_full[q_mine] = pt_mine
        part = O.self_energy(v, g, pt_full, w.nk3, q_list=q_mine)
        t = torch.from_numpy(np.ascontiguousarray(part))
        t_ri = torch.view_as_real(t).contiguous()
        dist.all_reduce(t_ri, op=dist.ReduceOp.SUM)
        total = torch.view_as_complex(t_ri).numpy()
        ref = O.sigma_eval(v, g, w.nk3, w.beta, 2.0)["Sig"]
        err = float(np.abs(total - ref).max() / np.abs(ref).max())
        tmax = bench.max_over_ranks(float(rank + 1) * 10.0, dist)
        out[rank] = (err, tmax)
    finally:
        dist.destroy_process_group()


def test_q_sharded_sigma_and_timing_reduction():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        err, tmax = out[r]
        assert err < 1e-12
        assert tmax == 20.0


def _turns_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        import time
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import bench

        def work():
            t0 = time.monotonic()
            time.sleep(0.3)
            return (t0, time.monotonic())

        out[rank] = bench.in_turns(rank, world, work, dist.barrier)
    finally:
        dist.destroy_process_group()


def test_inputs_are_built_in_turns_of_two_ranks():
    """bench.py builds each rank's inputs (the host copy of V is 71 GB on the 4x4x4 solid) two
    ranks at a time: every rank builds exactly once, and a later turn starts only after every
    rank of the earlier turns has finished."""
    world = 5
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_turns_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    spans = {r: out[r] for r in range(world)}
    assert sorted(spans) == list(range(world))
    for a in range(world):
        for b in range(world):
            if a // 2 < b // 2:
                assert spans[a][1] <= spans[b][0], (a, b)
