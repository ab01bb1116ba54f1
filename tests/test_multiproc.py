"""World-size-2 host path on CPU (gloo): the bench's rendezvous, barrier and
max-over-ranks timing, and the paper's row partition of the pair sum (each rank takes a
block of rows, a sum over ranks gives the whole)."""
import os
import socket
import sys
import types

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2308_07487_gb300 import synth
    got_ws, got_rank, _ = bench.dist_setup(types.SimpleNamespace(impl="reference"))
    assert (got_ws, got_rank) == (ws, rank) and dist.get_backend() == "gloo"
    bench.barrier(ws)
    t = bench.allmax(ws, 1.0 + rank)            # a rank's own time
    lat = synth.hypercubic(6, 2, True)
    tr = synth.traj_precess(lat.n_sites, 12, seed=3)
    geo = oracle.Geometry.of_lattice(lat)
    half = lat.n_sites // 2
    rows = (0, half) if rank == 0 else (half, lat.n_sites)
    part = oracle.pair_corr(tr, 6, [0, 3], geo, 1.0, 6, rows=rows)["C_sum"]
    buf = torch.from_numpy(np.ascontiguousarray(part))
    dist.all_reduce(buf)                        # sum of the row blocks
    out[rank] = (t, buf.numpy().tolist())
    bench.barrier(ws)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0        # max over ranks
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2308_07487_gb300 import synth
    lat = synth.hypercubic(6, 2, True)
    tr = synth.traj_precess(lat.n_sites, 12, seed=3)
    full = oracle.pair_corr(tr, 6, [0, 3], oracle.Geometry.of_lattice(lat), 1.0, 6)["C_sum"]
    for r in (0, 1):
        np.testing.assert_allclose(np.array(res[r][1]), full, rtol=1e-12, atol=1e-12)
