"""Host logic of the multi-GPU paths, on CPU: gloo ranks, no CUDA.

* placement of independent lattices by bytes, and the gather of results;
* the slab decomposition of one periodic lattice: rows per rank, the ring of
  neighbours and the halo exchange of multi_gpu.exchange, checked by running
  a lattice split over 2 and 3 gloo ranks with the FP64 oracle stepping each
  rank's slab (plus one halo row on each side) and comparing with the
  unsplit oracle run bit for bit.  The library's own slabs (lbm_slabs_*,
  lbm_slab_pack / unpack) are checked on the GPU in test_gpu_slabs.py.
"""
import os
import socket
import sys

import numpy as np
import pytest

import lbm_inputs as inp
import oracle as orc
from paper_1107_4543_gb300 import multi_gpu as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_by_bytes_is_balanced_and_complete():
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(1e3), np.log(1e6), 200))]
    for parts in (1, 2, 3, 8):
        out = mg.partition_by_bytes(sizes, parts)
        assert len(out) == parts
        flat = sorted(i for p in out for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in out]
        assert max(loads) - sum(sizes) / parts <= max(sizes)
        assert out == mg.partition_by_bytes(sizes, parts)  # deterministic
    with pytest.raises(ValueError):
        mg.partition_by_bytes(sizes, 0)


def test_slab_rows_and_ring():
    for ny, world in ((7, 1), (7, 3), (64, 4), (5, 5), (29, 4)):
        rows = mg.slab_rows(ny, world)
        assert rows[0][0] == 0 and sum(r for _, r in rows) == ny
        for k in range(world - 1):
            assert rows[k][0] + rows[k][1] == rows[k + 1][0]
        assert all(r >= 1 for _, r in rows)
        assert mg.neighbours(0, world) == ((world - 1) % world, 1 % world)
    with pytest.raises(ValueError):
        mg.slab_rows(3, 4)


def _slab_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's parts carry its rank, so the routing is visible
        tb = torch.full((5,), 10.0 * rank + 1)
        ta = torch.full((5,), 10.0 * rank + 2)
        fb, fa = torch.zeros(5), torch.zeros(5)
        mg.exchange(tb, ta, fb, fa, rank, world)
        below, above = mg.neighbours(rank, world)
        routed = bool(torch.all(fb == 10.0 * below + 2) and torch.all(fa == 10.0 * above + 1))

        # one 23 x 13 lattice split over the ranks; each rank steps its rows
        # plus one halo row on each side with the plain oracle (the halo
        # rows carry the neighbours' full boundary populations, so the
        # interior rows come out right), then exchanges its new boundary
        # rows with exchange()
        nx, ny, T = 23, 13, 9
        s = inp.s_paper(inp.rates("OPT"))
        f = inp.random_populations(nx, ny, seed=3, amp=1e-2)
        y0, rows = mg.slab_rows(ny, world)[rank]
        ext = np.take(f, np.arange(y0 - 1, y0 + rows + 1) % ny, axis=1)
        for _ in range(T):
            ext = orc.run(ext, s, 1)
            mine = ext[:, 1:rows + 1]
            tb = torch.from_numpy(np.ascontiguousarray(mine[:, 0]))   # my row 0, downwards
            ta = torch.from_numpy(np.ascontiguousarray(mine[:, -1]))  # my last row, upwards
            fb, fa = torch.empty_like(tb), torch.empty_like(ta)
            mg.exchange(tb, ta, fb, fa, rank, world)
            ext = np.concatenate([fb.numpy()[:, None], mine, fa.numpy()[:, None]], axis=1)
        gathered = mg.gather_by_index({rank: ext[:, 1:rows + 1]}, world, rank)
        if rank == 0:
            whole = np.concatenate(gathered, axis=1)
            out.put(("slabs", routed, bool(np.array_equal(whole, orc.run(f, s, T)))))
        else:
            out.put(("slabs", routed, None))

        # placement: lattices spread by bytes, results gathered in order
        specs = inp.batch_specs(7, seed=41, amin=6 * 6, amax=20 * 20)
        sizes = [mg.lattice_bytes(sp["nx"], sp["ny"], 1) for sp in specs]
        share = mg.partition_by_bytes(sizes, world)[rank]
        local = {}
        for i in share:
            sp = specs[i]
            fr = orc.run(orc.init_eq(*inp.batch_fields(sp)), inp.s_paper(sp["rates"]), 5)
            local[i] = orc.moments(fr)[0]
        got = mg.gather_by_index(local, world, rank)
        if rank == 0:
            ok = all(np.array_equal(g, orc.moments(orc.run(orc.init_eq(*inp.batch_fields(sp)),
                                                            inp.s_paper(sp["rates"]), 5))[0])
                     for g, sp in zip(got, specs))
            out.put(("placement", len(got) == len(specs), ok))
        else:
            out.put(("placement", None, None))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_halos_and_gather(world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2 * world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    slabs = [r for r in res if r[0] == "slabs"]
    assert all(r[1] for r in slabs)                          # every rank routed right
    assert [r[2] for r in slabs if r[2] is not None] == [True]  # split == unsplit
    place = [r for r in res if r[0] == "placement" and r[1] is not None]
    assert place == [("placement", True, True)]
