"""The multi-rank path of bench.py on CPU: two gloo ranks.

The workload is 2 x `lattices` independent lattices placed on the ranks by
bytes (weak scaling), so the only cross-rank operations are the timing
barrier and the max over ranks; the reported value is all ranks' units over
that max time.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    class A:
        lattices = 6
        lbm_steps = 10

    specs = bench.rank_specs(A, rank, world)
    nodes = sum(s["nx"] * s["ny"] for s in specs)
    # ranks report different times; everyone must see the slowest
    t = bench.reduce_max(1.0 + rank, device="cpu")
    units = bench.reduce_sum(nodes * A.lbm_steps, device="cpu")
    value = bench.job_mlups(units, t)
    out.put((rank, [(s["nx"], s["ny"]) for s in specs], t, value, nodes))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0, n0), (r1, s1, t1, v1, n1) = res
    assert s0 != s1                      # independent shards
    # together the shards are the 12-lattice workload, each lattice once
    import lbm_inputs as inp

    whole = inp.batch_specs(12, seed=1107 + 4, steps=10)
    assert sorted(s0 + s1) == sorted((s["nx"], s["ny"]) for s in whole)
    assert abs(n0 - n1) <= max(s["nx"] * s["ny"] for s in whole)  # balanced by bytes
    assert t0 == t1 == 2.0               # max over ranks
    assert v0 == v1 == pytest.approx((n0 + n1) * 10 / 2.0 / 1e6)
