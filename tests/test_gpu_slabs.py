"""One periodic lattice split into y-slabs, on one GPU.

Slabs run the same node arithmetic on the same inputs as the unsplit
lattice, so every check here is bit for bit: the in-process slab group
(lbm_slabs_*, halo copies overlapped with the interior rows) and the
one-slab-per-process calls (lbm_slab_pack / unpack: with the transport done
by plain device copies between the slabs of one process, through
multi_gpu.SlabRank with one rank, and through SlabRank in two or three
processes on the one GPU exchanging over gloo) against lbm_create on the
whole lattice, for FP64, FP32 and BF16 storage, ragged sizes, one-row slabs
and a single slab; FP64 also against the oracle.
"""
import os

import numpy as np
import pytest

import lbm_inputs as inp
import oracle as orc

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1107_4543_gb300 import build, lbm

    build.build()
    lbm.load()
    orc.set_threads(os.cpu_count() or 1)
    return lbm


def unsplit(L, nx, ny, r, dtype, steps, fields=None, pops=None, u0=(0.0, 0.0)):
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, u0, L.DTYPES[dtype])
    try:
        if fields is not None:
            L.lbm_init_field(h, *fields)
        else:
            L.lbm_set_populations(h, pops)
        d0 = L.lbm_drift(h)
        L.lbm_step(h, steps)
        return L.lbm_get_populations(h), L.lbm_moments(h), d0, L.lbm_drift(h)
    finally:
        L.lbm_destroy(h)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f64dev"])
@pytest.mark.parametrize("nx,ny,nslabs", [(64, 48, 3), (37, 29, 4), (33, 4, 4), (40, 17, 1),
                                          (130, 9, 2)])
def test_slabs_equal_unsplit_lattice(L, dtype, nx, ny, nslabs):
    steps = 23
    r = inp.rates("OPT")
    u0 = (0.05, -0.02)
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 3.0, u0=u0)
    want_f, want_m, want_d0, want_d1 = unsplit(L, nx, ny, r, dtype, steps, fields=fields, u0=u0)
    s = L.lbm_slabs_create(nx, ny, inp.s_ll(r), 1.0, u0, L.DTYPES[dtype], nslabs)
    try:
        rows = [L.lbm_slabs_rows(s, k) for k in range(nslabs)]
        assert sum(rr for _, rr, _ in rows) == ny
        L.lbm_slabs_init_field(s, *fields)
        d0 = L.lbm_slabs_drift(s)
        L.lbm_slabs_step(s, steps)
        f = L.lbm_slabs_get_populations(s, ny, nx)
        m = L.lbm_slabs_moments(s, ny, nx)
        d1 = L.lbm_slabs_drift(s)
    finally:
        L.lbm_slabs_destroy(s)
    assert np.array_equal(f, want_f)
    for a, b in zip(m, want_m):
        assert np.array_equal(a, b)
    # the drift sums every stored slot: the slabs' sums agree with the whole
    # lattice's up to the order of the lattice-wide sum
    scale = np.abs(want_d0[:3]).max()
    assert np.max(np.abs(d0[:3] - want_d0[:3])) <= 1e-13 * scale
    assert np.max(np.abs(d1[:3] - want_d1[:3])) <= 1e-13 * scale
    if dtype == "f64":
        want_o = orc.run(orc.init_eq(*fields), inp.s_paper(r), steps)
        assert np.array_equal(f, want_o)


def test_slabs_from_set_populations(L):
    """Non-equilibrium populations through lbm_slabs_set_populations."""
    nx, ny, steps = 35, 22, 17
    r = inp.rates("LL", nu=2e-3)
    pops = inp.random_populations(nx, ny, seed=8, amp=1e-2)
    want_f = unsplit(L, nx, ny, r, "f64", steps, pops=pops)[0]
    s = L.lbm_slabs_create(nx, ny, inp.s_ll(r), 1.0, (0.0, 0.0), L.LBM_F64, 3)
    try:
        L.lbm_slabs_set_populations(s, pops)
        assert np.array_equal(L.lbm_slabs_get_populations(s, ny, nx), pops)
        L.lbm_slabs_step(s, steps)
        f = L.lbm_slabs_get_populations(s, ny, nx)
    finally:
        L.lbm_slabs_destroy(s)
    assert np.array_equal(f, want_f)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_slab_pack_unpack_between_handles(L, dtype):
    """The one-slab-per-process calls, with the ranks' transport replaced by
    device copies between the slab handles of this process."""
    torch = pytest.importorskip("torch")
    from paper_1107_4543_gb300 import multi_gpu as mg

    nx, ny, world, steps = 48, 31, 3, 19
    r = inp.rates("OPT")
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 3.0)
    want_f = unsplit(L, nx, ny, r, dtype, steps, fields=fields)[0]
    rows = mg.slab_rows(ny, world)
    hs = [L.lbm_slab_create(nx, ny, y0, rr, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
          for y0, rr in rows]
    try:
        nb = L.lbm_slab_halo_bytes(hs[0])
        bufs = [[torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(4)]
                for _ in hs]

        def exchange(reverse):
            for h, b in zip(hs, bufs):
                L.lbm_slab_pack(h, reverse, b[0], b[1])
                L.lbm_sync(h)
            for k in range(world):
                below, above = mg.neighbours(k, world)
                bufs[k][2].copy_(bufs[below][1])  # what the lower slab sent up
                bufs[k][3].copy_(bufs[above][0])  # what the upper slab sent down
            torch.cuda.synchronize()
            for h, b in zip(hs, bufs):
                L.lbm_slab_unpack(h, reverse, b[2], b[3])

        for h, (y0, rr) in zip(hs, rows):
            L.lbm_init_field(h, *(np.ascontiguousarray(a[y0:y0 + rr]) for a in fields))
        exchange(True)
        for _ in range(steps):
            for h in hs:
                L.lbm_step(h, 1)
            exchange(False)
        f = np.concatenate([L.lbm_get_populations(h) for h in hs], axis=1)
        with pytest.raises(L.LbmError):
            L.lbm_step(hs[0], 2)  # a slab steps once between exchanges
        with pytest.raises(L.LbmError):
            L.lbm_init_analytic(hs[0], L.LBM_INIT_GAUSSIAN, (1e-3, 4.0, 1.0, 1.0))
    finally:
        for h in hs:
            L.lbm_destroy(h)
    assert np.array_equal(f, want_f)


def test_slab_rank_single_process(L):
    """multi_gpu.SlabRank with one rank (its exchange then wraps onto
    itself) equals the unsplit lattice."""
    from paper_1107_4543_gb300 import multi_gpu as mg

    nx, ny, steps = 40, 20, 11
    r = inp.rates("OPT")
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 3.0)
    want = unsplit(L, nx, ny, r, "f32", steps, fields=fields)[1][0]
    sr = mg.SlabRank(L, nx, ny, inp.s_ll(r), 0, 1)
    try:
        sr.init_field(*fields)
        sr.step(steps)
        got = sr.moments()[0]
    finally:
        sr.close()
    assert np.array_equal(got, want)


def test_slabs_reject_fp16_and_bad_splits(L):
    S = inp.s_ll(inp.rates("OPT"))
    with pytest.raises(L.LbmError):
        L.lbm_slabs_create(16, 16, S, 1.0, (0.0, 0.0), L.LBM_F16DEV, 2)
    with pytest.raises(L.LbmError):
        L.lbm_slabs_create(16, 3, S, 1.0, (0.0, 0.0), L.LBM_F32DEV, 4)
    with pytest.raises(L.LbmError):
        L.lbm_slab_create(16, 16, 10, 8, S)


def _slab_rank_worker(rank, world, port, out_dir, nx, ny, steps):
    """One rank of a lattice split over `world` processes on the one GPU,
    its halo rows exchanged over gloo (host-staged): no kernel of one rank
    waits on another's."""
    import datetime
    import sys

    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=120))
    try:
        from paper_1107_4543_gb300 import lbm
        from paper_1107_4543_gb300 import multi_gpu as mg

        lbm.load()
        torch.cuda.set_device(0)
        fields = inp.gaussian_pulse(nx, ny, 1e-3, 3.0, u0=(0.05, -0.02))
        sr = mg.SlabRank(lbm, nx, ny, inp.s_ll(inp.rates("OPT")), rank, world, u0=(0.05, -0.02))
        try:
            assert sr.host is not None  # gloo: staged through host memory
            sr.init_field(*fields)
            sr.step(steps)
            rho, ux, uy = sr.moments()
            np.savez(os.path.join(out_dir, "rank%d.npz" % rank), y0=sr.y0, rho=rho, ux=ux, uy=uy)
        finally:
            sr.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_ranks_over_gloo_on_one_gpu(L, tmp_path, world):
    """multi_gpu.SlabRank across `world` processes (one slab each, halo rows
    exchanged through torch.distributed, here gloo with host staging, all on
    the one GPU) equals the unsplit lattice bit for bit; with two ranks both
    neighbours of a rank are the same rank, which the exchange's message
    order has to keep apart."""
    pytest.importorskip("torch")
    import socket

    import torch.multiprocessing as mp

    nx, ny, steps = 48, 21, 13
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_slab_rank_worker,
                         args=(k, world, port, str(tmp_path), nx, ny, steps))
             for k in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
    assert [p.exitcode for p in procs] == [0] * world
    u0 = (0.05, -0.02)
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 3.0, u0=u0)
    want = unsplit(L, nx, ny, inp.rates("OPT"), "f32", steps, fields=fields, u0=u0)[1]
    got = [np.full((ny, nx), np.nan) for _ in range(3)]
    for k in range(world):
        z = np.load(os.path.join(str(tmp_path), "rank%d.npz" % k))
        y0 = int(z["y0"])
        for c, key in enumerate(("rho", "ux", "uy")):
            got[c][y0:y0 + z[key].shape[0]] = z[key]
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
