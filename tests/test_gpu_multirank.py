"""The q-sharded self-energy through the library (world size 2, gloo, both ranks on one GPU).

Eq. sigma_gw is a sum over q and P0^q, P~^q are per q, so a multi-GPU run gives each rank a
range of q: the rank computes its partial Sigma with gw_sigma_eval_q, and one sum over ranks
(here a gloo all-reduce of host copies) gives the full Sigma. The two ranks are processes that
share the one GPU; their kernels never wait on one another (the only exchange is on the host
after each rank has finished). The sum must equal the single-rank gw_sigma_eval: to 1e-13
relative in FP64 (rounding order of the q sum), and within the mixed path's tolerance (1e-7)
in the mixed precision, where a q whose -q sits on the other rank is computed at every tau
node instead of through the mirror relation.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, prec, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        sys.path.insert(0, root)
        from paper_2406_18479_gb300 import gw, inputs as I
        torch.cuda.set_device(0)
        w = I.Workload("shard", (3, 2, 1), 8, 40, 8, 8, 8.0, 0.0, 6.0, 23, solid=True)
        h, v, g = I.make_inputs(w)
        ctx = gw.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=prec)
        V = torch.from_numpy(v).cuda()
        G = torch.from_numpy(g).cuda()
        gw.gw_set_coulomb(ctx, V)
        S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
        # contiguous q ranges: rank r takes [r nk / world, (r + 1) nk / world)
        q0, q1 = rank * w.nk // world, (rank + 1) * w.nk // world
        gw.gw_sigma_eval_q(ctx, G, S, q0, q1)
        gw.gw_synchronize(ctx)
        part = torch.view_as_real(S.cpu()).contiguous()
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        total = torch.view_as_complex(part).numpy()
        # the single-rank evaluation on the same context
        gw.gw_sigma_eval(ctx, G, S)
        gw.gw_synchronize(ctx)
        ref = S.cpu().numpy()
        ctx.destroy()
        out[rank] = float(np.abs(total - ref).max() / np.abs(ref).max())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("bf16x3", 1e-7)])
def test_q_sharded_sigma_through_the_library(prec, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), prec, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        assert out[r] < tol
