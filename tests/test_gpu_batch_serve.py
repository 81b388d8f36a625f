"""GPU checks of the batched step and of the continuous-batching server.

A lattice advanced inside a batch, or served among other requests, must
give exactly the result it gives alone (same kernel body, same per-lattice
parameters), and that result must match the FP64 oracle within its storage
type's tolerance.
"""
import os
import time

import numpy as np
import pytest

import lbm_inputs as inp
import oracle as orc

pytestmark = pytest.mark.gpu
TOL = {"f32": 1e-6, "f16": 2e-3, "bf16": 2e-3}


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


def alone(L, spec, dtype, steps):
    h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                     L.DTYPES[dtype])
    try:
        L.lbm_init_field(h, *inp.batch_fields(spec))
        L.lbm_step(h, steps)
        return L.lbm_get_populations(h), L.lbm_moments(h)
    finally:
        L.lbm_destroy(h)


def small_specs(n, seed):
    return inp.batch_specs(n, seed=seed, amin=6 * 6, amax=96 * 96)


@pytest.mark.parametrize("steps", [1, 7, 64, 131])
def test_batch_member_equals_alone(L, steps):
    specs = small_specs(12, seed=11)
    dtypes = ["f32", "f16", "bf16"] * 4
    hs = []
    try:
        for spec, dt in zip(specs, dtypes):
            h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                             L.DTYPES[dt])
            L.lbm_init_field(h, *inp.batch_fields(spec))
            hs.append(h)
        # one member starts on its other buffer
        L.lbm_step(hs[0], 1)
        b = L.lbm_batch_create(hs)
        L.lbm_batch_step(b, steps)
        L.lbm_batch_step(b, 3)
        got = [L.lbm_get_populations(h) for h in hs]
        L.lbm_batch_destroy(b)
    finally:
        for h in hs:
            L.lbm_destroy(h)
    for k, (spec, dt) in enumerate(zip(specs, dtypes)):
        want, _ = alone(L, spec, dt, steps + 3 + (1 if k == 0 else 0))
        # some sweep members are linearly unstable (Lallemand-Luo free rates
        # at small bulk viscosity, section 4.2) and overflow: NaN == NaN here
        assert np.array_equal(got[k], want, equal_nan=True), (k, dt, spec["nx"], spec["ny"])


@pytest.mark.parametrize("variant", range(6))
def test_every_batch_launch_variant_equals_alone(L, variant):
    """All launch variants (register caps; one warp per task or persistent
    contiguous task ranges) give the standalone result bit for bit."""
    specs = small_specs(20, seed=14)
    dtypes = ["f32", "f16", "bf16"] * 7
    hs = []
    try:
        for spec, dt in zip(specs, dtypes):
            h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                             L.DTYPES[dt])
            L.lbm_init_field(h, *inp.batch_fields(spec))
            hs.append(h)
        b = L.lbm_batch_create(hs)
        L.lbm_batch_set_variant(b, variant)
        L.lbm_batch_step(b, 70)
        got = [L.lbm_get_populations(h) for h in hs]
        L.lbm_batch_destroy(b)
    finally:
        for h in hs:
            L.lbm_destroy(h)
    for k, (spec, dt) in enumerate(zip(specs, dtypes)):
        want, _ = alone(L, spec, dt, 70)
        assert np.array_equal(got[k], want, equal_nan=True), (variant, k, dt)


RESIDENT_CASES = [(5, 3, "f32"), (56, 56, "f32"), (58, 56, "f32"), (2, 7, "f32"),
                  (33, 17, "f16"), (80, 80, "f16"), (81, 80, "f16"), (80, 80, "bf16"),
                  (9, 2, "bf16"), (130, 40, "f32"), (200, 90, "bf16")]


@pytest.mark.parametrize("cap", [None, "0"])
def test_resident_members_equal_alone(L, cap, monkeypatch):
    """Members small enough for one block's shared memory (both step buffers
    of 9 compact planes) are stepped there for all the steps of a launch,
    beside the per-step launches of the others (lbm_batch_resident says
    which); every member equals its standalone run bit for bit, with the
    resident path on and off (LBM_RESIDENT_BYTES=0), over calls of odd and
    even length, one of them starting at batch parity 1."""
    torch = pytest.importorskip("torch")
    optin = torch.cuda.get_device_properties(0).shared_memory_per_block_optin
    if cap is not None:
        monkeypatch.setenv("LBM_RESIDENT_BYTES", cap)
    specs = small_specs(len(RESIDENT_CASES), seed=17)
    for sp, (nx, ny, _) in zip(specs, RESIDENT_CASES):
        sp.update(nx=nx, ny=ny, xc=nx / 2, yc=ny / 2, b=2.0)
    dtypes = [dt for _, _, dt in RESIDENT_CASES]
    esize = {"f32": 4, "f16": 2, "bf16": 2}
    want_res = [cap is None and 2 * 9 * nx * ny * esize[dt] <= optin for nx, ny, dt in RESIDENT_CASES]
    # the cases straddle the limit on GB300 (227 KB): 56 x 56 FP32 and
    # 80 x 80 FP16 fit, 58 x 56 and 81 x 80 do not
    assert cap is not None or (any(want_res) and not all(want_res))
    hs = []
    try:
        for spec, dt in zip(specs, dtypes):
            h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                             L.DTYPES[dt])
            L.lbm_init_field(h, *inp.batch_fields(spec))
            hs.append(h)
        b = L.lbm_batch_create(hs)
        assert list(L.lbm_batch_resident(b)) == want_res
        for n in (37, 1, 64, 2):
            L.lbm_batch_step(b, n)
        drift = L.lbm_batch_drift(b, len(hs))
        got = [L.lbm_get_populations(h) for h in hs]
        L.lbm_batch_destroy(b)
    finally:
        for h in hs:
            L.lbm_destroy(h)
    for k, (spec, dt) in enumerate(zip(specs, dtypes)):
        want, _ = alone(L, spec, dt, 104)
        assert np.array_equal(got[k], want), (k, dt, spec["nx"], spec["ny"], want_res[k])
    assert np.all(np.isfinite(drift))


def _scaled(fields, a):
    rho, ux, uy = fields
    return 1.0 + a * (rho - 1.0), a * ux, a * uy


@pytest.mark.parametrize("mode", ["fallback", "reused", "off"])
def test_const_table_slots_equal_alone(L, mode, monkeypatch):
    """The members' collision constants come from a constant-memory table
    per storage type and device (960 slots for FP16 and BF16, 640 for FP32;
    lbm_batch_const_table says whose).  A batch that finds no room (another
    batch holds the FP16 slots) or is made with LBM_CONST_TABLE=0 reads them
    from its entries;
    slots a destroyed batch held are taken again.  Every member equals its
    standalone run bit for bit in each case, across a batch-level re-init
    between calls that changes the FP16 storage scales (the table is
    refreshed before each stepping call)."""
    monkeypatch.setenv("LBM_RESIDENT_BYTES", "0")  # every member on the per-step path
    if mode == "off":
        monkeypatch.setenv("LBM_CONST_TABLE", "0")
    specs = small_specs(12, seed=23)
    dtypes = ["f32", "f16", "bf16"] * 4
    fields = [inp.batch_fields(sp) for sp in specs]
    S = inp.s_ll(inp.rates("OPT"))
    hold, hb, hs, b = [], None, [], None
    try:
        if mode != "off":
            # 958 of the 960 FP16 slots taken by another batch
            hold = [L.lbm_create(8, 8, S, 1.0, (0.0, 0.0), L.LBM_F16DEV) for _ in range(958)]
            hb = L.lbm_batch_create(hold)
            assert L.lbm_batch_const_table(hb).all()
        for spec, dt, f in zip(specs, dtypes, fields):
            h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                             L.DTYPES[dt])
            L.lbm_init_field(h, *f)
            hs.append(h)
        if mode == "reused":
            L.lbm_batch_destroy(hb)
            hb = None
        b = L.lbm_batch_create(hs)
        want_flags = [{"fallback": dt != "f16", "reused": True, "off": False}[mode]
                      for dt in dtypes]
        assert list(L.lbm_batch_const_table(b)) == want_flags
        L.lbm_batch_step(b, 10)
        L.lbm_batch_init_fields(b, [_scaled(f, 20.0) for f in fields])
        L.lbm_batch_step(b, 23)
        L.lbm_batch_step(b, 8)
        got = [L.lbm_get_populations(h) for h in hs]
    finally:
        if b is not None:
            L.lbm_batch_destroy(b)
        if hb is not None:
            L.lbm_batch_destroy(hb)
        for h in hs + hold:
            L.lbm_destroy(h)
    for k, (spec, dt, f) in enumerate(zip(specs, dtypes, fields)):
        h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                         L.DTYPES[dt])
        try:
            L.lbm_init_field(h, *_scaled(f, 20.0))
            L.lbm_step(h, 31)
            want = L.lbm_get_populations(h)
        finally:
            L.lbm_destroy(h)
        assert np.array_equal(got[k], want), (mode, k, dt)


def test_const_table_two_live_batches(L, monkeypatch):
    """Two batches alive at once hold neighbouring ranges of the FP32, FP16
    and BF16 constant tables (the second one's start past slot 0) and step in
    turns, each call refreshing its own range: every member of both equals
    its standalone run bit for bit."""
    monkeypatch.setenv("LBM_RESIDENT_BYTES", "0")
    specs = small_specs(14, seed=29)
    dtypes = ["f16", "bf16", "f32", "f16", "bf16", "f16", "bf16"] * 2
    groups = [(0, 7), (7, 14)]
    steps = [(9, 4, 13), (6, 17, 2)]  # per batch, its calls in turn
    hs, bs = [], []
    try:
        for spec, dt in zip(specs, dtypes):
            h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                             L.DTYPES[dt])
            L.lbm_init_field(h, *inp.batch_fields(spec))
            hs.append(h)
        for lo, hi in groups:
            bs.append(L.lbm_batch_create(hs[lo:hi]))
            assert L.lbm_batch_const_table(bs[-1]).all()
        for c in range(3):
            for b, st in zip(bs, steps):
                L.lbm_batch_step(b, st[c])
        got = [L.lbm_get_populations(h) for h in hs]
    finally:
        for b in bs:
            L.lbm_batch_destroy(b)
        for h in hs:
            L.lbm_destroy(h)
    for k, (spec, dt) in enumerate(zip(specs, dtypes)):
        n = sum(steps[0 if k < 7 else 1])
        want, _ = alone(L, spec, dt, n)
        assert np.array_equal(got[k], want), (k, dt)


def test_batch_host_io_equals_member_calls(L):
    """lbm_batch_init_fields / lbm_batch_moments give exactly what the
    per-member calls give, keep the batch usable across re-inits, and reject
    an invalid field."""
    specs = small_specs(9, seed=15)
    dtypes = ["f32", "f16", "bf16"] * 3
    fields = [inp.batch_fields(sp) for sp in specs]
    hs = []
    try:
        for spec, dt in zip(specs, dtypes):
            hs.append(L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0,
                                   (0.0, 0.0), L.DTYPES[dt]))
        L.lbm_step(hs[2], 3)  # a member on its other buffer
        b = L.lbm_batch_create(hs)
        for rep in range(2):
            L.lbm_batch_init_fields(b, fields)
            L.lbm_batch_step(b, 33 + rep)
            outs = [tuple(np.empty((sp["ny"], sp["nx"])) for _ in range(3)) for sp in specs]
            L.lbm_batch_moments(b, outs)
            for k, h in enumerate(hs):
                assert np.array_equal(outs[k][0], L.lbm_moments(h)[0], equal_nan=True)
        bad = [tuple(a.copy() for a in f) for f in fields]
        bad[4][0][1, 1] = -1.0
        with pytest.raises(L.LbmError) as e:
            L.lbm_batch_init_fields(b, bad)
        assert e.value.code == L.LBM_EINVAL
        L.lbm_batch_destroy(b)
    finally:
        for h in hs:
            L.lbm_destroy(h)
    for k, (spec, dt) in enumerate(zip(specs, dtypes)):
        # the second round: init, 34 steps
        _, (rho, _, _) = alone(L, spec, dt, 34)
        assert np.array_equal(outs[k][0], rho, equal_nan=True), (k, dt)


def test_batch_packed_io_equals_per_member_io(L):
    """lbm_batch_init_packed / lbm_batch_moments_packed give bit for bit what
    the per-member calls give, across several copy groups (over 2^23 nodes)
    with mixed storage types; the packed arrays are checked for size."""
    specs = inp.batch_specs(9, seed=16, amin=700 * 700, amax=1800 * 1800)
    specs[1].update(nx=33, ny=17)  # a ragged small member between large ones
    dtypes = ["f32", "f16", "bf16"] * 3
    fields = [inp.batch_fields(sp) for sp in specs]
    total = sum(sp["nx"] * sp["ny"] for sp in specs)
    assert total > 2 ** 23  # at least two copy groups

    def make():
        return [L.lbm_create(sp["nx"], sp["ny"], inp.s_ll(sp["rates"]), 1.0, (0.0, 0.0),
                             L.DTYPES[dt]) for sp, dt in zip(specs, dtypes)]

    ha, hb = make(), make()
    try:
        ba, bb = L.lbm_batch_create(ha), L.lbm_batch_create(hb)
        assert L.lbm_batch_size(bb) == (9, total)
        packed = [np.concatenate([f[c].ravel() for f in fields]) for c in range(3)]
        for rep in range(2):
            L.lbm_batch_init_fields(ba, fields)
            L.lbm_batch_init_packed(bb, *packed)
            L.lbm_batch_step(ba, 5 + rep)
            L.lbm_batch_step(bb, 5 + rep)
            outs = [tuple(np.empty((sp["ny"], sp["nx"])) for _ in range(3)) for sp in specs]
            L.lbm_batch_moments(ba, outs)
            got = L.lbm_batch_moments_packed(bb)
            for c in range(3):
                want = np.concatenate([o[c].ravel() for o in outs])
                assert np.array_equal(got[c], want), (rep, c)
        with pytest.raises(ValueError):
            L.lbm_batch_init_packed(bb, packed[0][:-1], packed[1], packed[2])
        L.lbm_batch_destroy(ba)
        L.lbm_batch_destroy(bb)
    finally:
        for h in ha + hb:
            L.lbm_destroy(h)


def test_host_array(L):
    """lbm_host_alloc arrays: any size, written and read through numpy, a
    device copy round trip, released with the array; other pointers are
    refused by lbm_host_free."""
    torch = pytest.importorskip("torch")
    for n in (1, 1000, 3 << 20):
        a = L.host_array(n)
        assert a.shape == (n,) and a.dtype == np.float64 and np.all(a == 0)
        a[:] = np.arange(n)
        t = torch.from_numpy(a)
        assert t.is_pinned()
        d = t.to("cuda", non_blocking=True)
        back = L.host_array((n,))
        torch.from_numpy(back).copy_(d, non_blocking=True)
        torch.cuda.synchronize()
        assert np.array_equal(back, a)
        del a, t, back
    with pytest.raises(L.LbmError) as e:
        L.lbm_host_free(12345)
    assert e.value.code == L.LBM_EINVAL


def test_batch_solve_packed_equals_synchronous_calls(L):
    """lbm_batch_solve_packed (upload, init, steps, drift, moments, download
    queued without waiting, successive solves overlapping through two
    staging slots) gives bit for bit what lbm_batch_init_packed +
    lbm_batch_step + lbm_batch_drift + lbm_batch_moments_packed give, for
    three solves queued back to back with different fields (both slots
    reused), FP32, BF16 and FP16 members -- the FP16 members choosing their
    storage scale on the device, a different one per solve, which the host
    copies follow at the wait; invalid fields are reported."""
    torch = pytest.importorskip("torch")
    specs = inp.batch_specs(7, seed=17, amin=300 * 300, amax=1500 * 1500)
    specs[2].update(nx=33, ny=17)
    dtypes = ["f32", "bf16", "f16", "f32", "bf16", "f16", "f32"]
    steps = [40, 7, 65]
    total = sum(sp["nx"] * sp["ny"] for sp in specs)

    def pinned(n):
        return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()

    ins = []
    for rep in range(3):
        sp2 = [dict(sp, amp=sp["amp"] * (1 + rep), xc=sp["xc"] + 3 * rep) for sp in specs]
        fields = [inp.batch_fields(sp) for sp in sp2]
        tri = tuple(pinned(total) for _ in range(3))
        for c in range(3):
            np.concatenate([f[c].ravel() for f in fields], out=tri[c])
        ins.append(tri)

    def make():
        return [L.lbm_create(sp["nx"], sp["ny"], inp.s_ll(sp["rates"]), 1.0, (0.0, 0.0),
                             L.DTYPES[dt]) for sp, dt in zip(specs, dtypes)]

    ha, hb = make(), make()
    try:
        ba, bb = L.lbm_batch_create(ha), L.lbm_batch_create(hb)
        # outputs in page-locked huge-page memory (lbm_host_alloc), inputs
        # in torch's page-locked memory
        outs = [tuple(L.host_array(total) for _ in range(3)) for _ in range(3)]
        drifts = [np.zeros((len(specs), 4)) for _ in range(3)]
        for rep in range(3):
            L.lbm_batch_solve_packed(bb, steps[rep], ins[rep], outs[rep], drifts[rep])
        phases = L.lbm_batch_wait(bb)
        assert set(phases) == set(L.BATCH_PHASES) | {"unstable"} and phases["steps_ms"] > 0
        assert not phases["unstable"]
        scales = [L.lbm_info(h)["qscale"] for h in hb]
        for rep in range(3):
            L.lbm_batch_init_packed(ba, *ins[rep])
            L.lbm_batch_step(ba, steps[rep])
            d = L.lbm_batch_drift(ba, len(specs))
            want = L.lbm_batch_moments_packed(ba)
            for c in range(3):
                assert np.array_equal(outs[rep][c], want[c]), (rep, c)
            assert np.array_equal(drifts[rep], d), rep
        # the host copies of the device-chosen FP16 scales (last solve) equal
        # the host-chosen ones of the synchronous calls on the same fields
        assert scales == [L.lbm_info(h)["qscale"] for h in ha]
        assert any(sc != 1.0 for sc, dt in zip(scales, dtypes) if dt == "f16")
        # invalid fields are reported by the wait, naming the member
        bad = tuple(a.copy() for a in ins[0])
        bad[0][total - 5] = -1.0
        L.lbm_batch_solve_packed(bb, 3, bad, outs[0])
        with pytest.raises(L.LbmError) as e:
            L.lbm_batch_wait(bb)
        assert e.value.code == L.LBM_EINVAL and "member 6" in str(e.value)
        L.lbm_batch_solve_packed(bb, 3, ins[0], outs[0])
        L.lbm_batch_wait(bb)  # the counters were cleared
        with pytest.raises(ValueError):
            L.lbm_batch_solve_packed(bb, 3, (ins[0][0][:-1],) + ins[0][1:], outs[0])
        L.lbm_batch_destroy(ba)
        L.lbm_batch_destroy(bb)
    finally:
        for h in ha + hb:
            L.lbm_destroy(h)


def test_batch_results_match_oracle(L):
    specs = small_specs(6, seed=12)
    hs = []
    steps = 60
    try:
        for spec in specs:
            h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                             L.LBM_F32DEV)
            L.lbm_init_field(h, *inp.batch_fields(spec))
            hs.append(h)
        b = L.lbm_batch_create(hs)
        L.lbm_batch_step(b, steps)
        L.lbm_batch_destroy(b)
        got = [L.lbm_moments(h)[0] for h in hs]
    finally:
        for h in hs:
            L.lbm_destroy(h)
    for spec, rho in zip(specs, got):
        f = orc.run(orc.init_eq(*inp.batch_fields(spec)), inp.s_paper(spec["rates"]), steps)
        rho_o = orc.moments(f)[0]
        assert np.max(np.abs(rho - rho_o)) / spec["amp"] <= TOL["f32"]


def test_batch_drift_equals_member_drift(L):
    specs = small_specs(9, seed=13)
    hs = []
    try:
        for k, spec in enumerate(specs):
            dt = ("f32", "f16", "bf16")[k % 3]
            h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                             L.DTYPES[dt])
            L.lbm_init_field(h, *inp.batch_fields(spec))
            hs.append(h)
        L.lbm_step(hs[1], 1)
        b = L.lbm_batch_create(hs)
        for steps in (0, 5, 64):
            L.lbm_batch_step(b, steps)
            got = L.lbm_batch_drift(b, len(hs))
            for k, h in enumerate(hs):
                want = L.lbm_drift(h)
                scale = max(1e-300, abs(specs[k]["amp"]) * 50.0)
                assert np.all(np.abs(got[k, :3] - want[:3]) <= 1e-12 * scale), (k, steps)
                assert got[k, 3] == want[3]
            assert np.array_equal(got, L.lbm_batch_drift(b, len(hs)))
        L.lbm_batch_destroy(b)
    finally:
        for h in hs:
            L.lbm_destroy(h)


def test_batch_rejects_bad_members(L):
    S = inp.s_ll(inp.rates("OPT"))
    h64 = L.lbm_create(8, 8, S, dtype=L.LBM_F64)
    h = L.lbm_create(8, 8, S, dtype=L.LBM_F32DEV)
    try:
        with pytest.raises(L.LbmError):
            L.lbm_batch_create([h64])
        with pytest.raises(L.LbmError):
            L.lbm_batch_create([h, h])
        b = L.lbm_batch_create([h])
        with pytest.raises(L.LbmError):
            L.lbm_step(h, 1)  # members step through the batch only
        with pytest.raises(L.LbmError):
            L.lbm_batch_create([h])  # already in a batch
        L.lbm_batch_destroy(b)
        L.lbm_step(h, 1)  # released
    finally:
        L.lbm_destroy(h)
        L.lbm_destroy(h64)


def served_requests(n, seed):
    reqs = inp.request_stream(n, rate=1e9, seed=seed, side=(8, 80), steps=(1, 300))
    return reqs


def submit(L, srv, q, fields=False):
    init = q["init"]
    if fields:
        kind, params, fl = L.LBM_INIT_FIELDS, (), inp.request_fields(q)
    elif init["kind"] == "gaussian":
        kind, params, fl = L.LBM_INIT_GAUSSIAN, (init["amp"], init["b"], init["xc"], init["yc"]), None
    else:
        kind, params, fl = L.LBM_INIT_PLANE, (init["amp"], init["m"]), None
    req, keep = L.make_request(q["nx"], q["ny"], inp.s_ll(q["rates"]), q["steps"],
                               dtype=q["dtype"], init_kind=kind, init_params=params, fields=fl)
    return L.lbm_submit(srv, req), kind, params


def alone_request(L, q, kind, params):
    h = L.lbm_create(q["nx"], q["ny"], inp.s_ll(q["rates"]), 1.0, (0.0, 0.0),
                     L.DTYPES[q["dtype"]])
    try:
        if kind == L.LBM_INIT_FIELDS:
            L.lbm_init_field(h, *inp.request_fields(q))
        else:
            L.lbm_init_analytic(h, kind, params)
        L.lbm_step(h, q["steps"])
        return L.lbm_moments(h)
    finally:
        L.lbm_destroy(h)


def wait_all(L, srv, ids, reqs, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        assert time.time() - t0 < timeout, "server did not finish in time"
        for rid, q in zip(ids, reqs):
            if rid in out:
                continue
            rc, rho, ux, uy, lat = L.lbm_poll(srv, rid, q["nx"], q["ny"])
            if rc == L.LBM_OK:
                out[rid] = (rho, ux, uy, lat)
        time.sleep(0.001)
    return out


@pytest.mark.parametrize("budget_mb,policy,cap", [(1000, 0, 0), (2, 0, 0), (1000, 1, 20000)])
def test_served_result_equals_alone(L, budget_mb, policy, cap):
    """Each served result equals the same solve run alone: with a budget
    that admits everything at once, with one so tight that requests queue
    and join generations as others retire, and shortest-work-first with a
    resident-node cap.  Lattices of one generation stop at different step
    counts."""
    reqs = served_requests(16, seed=21)
    srv = L.lbm_server_create(budget_mb * 2**20, 37)
    L.lbm_server_set_policy(srv, policy, cap)
    try:
        ids, kinds = [], []
        for k, q in enumerate(reqs):
            rid, kind, params = submit(L, srv, q, fields=(k % 4 == 0))
            ids.append(rid)
            kinds.append((kind, params))
        out = wait_all(L, srv, ids, reqs)
        st = L.lbm_server_stats(srv)
        done = L.lbm_server_done(srv, cap=5) + L.lbm_server_done(srv)
        assert L.lbm_server_done(srv) == []
    finally:
        L.lbm_server_destroy(srv)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    # every finished request is reported once, whatever the chunking
    assert sorted(done) == sorted(ids)
    if budget_mb == 2:
        assert st["peak_bytes"] <= 2 * 2**20
        assert st["generations"] > 3
    else:
        assert st["peak_resident"] > 1
    for rid, q, (kind, params) in zip(ids, reqs, kinds):
        want = alone_request(L, q, kind, params)
        for a, b in zip(out[rid][:3], want):
            assert np.array_equal(a, b), (q["nx"], q["steps"], q["dtype"])


def test_served_results_match_oracle(L):
    reqs = served_requests(6, seed=22)
    srv = L.lbm_server_create(2**30, 50)
    try:
        ids = [submit(L, srv, q, fields=True)[0] for q in reqs]
        out = wait_all(L, srv, ids, reqs)
    finally:
        L.lbm_server_destroy(srv)
    for rid, q in zip(ids, reqs):
        f = orc.run(orc.init_eq(*inp.request_fields(q)), inp.s_paper(q["rates"]), q["steps"])
        rho_o = orc.moments(f)[0]
        err = np.max(np.abs(out[rid][0] - rho_o)) / q["init"]["amp"]
        assert err <= TOL[q["dtype"]], (q["dtype"], err)
        assert out[rid][3] > 0


def test_server_rejects_and_reports(L):
    srv = L.lbm_server_create(2**20, 10)
    try:
        big, _ = L.make_request(2048, 2048, inp.s_ll(inp.rates("OPT")), 10)
        with pytest.raises(L.LbmError) as e:
            L.lbm_submit(srv, big)
        assert e.value.code == L.LBM_ENOMEM
        bad, _ = L.make_request(1, 8, inp.s_ll(inp.rates("OPT")), 10)
        with pytest.raises(L.LbmError) as e:
            L.lbm_submit(srv, bad)
        assert e.value.code == L.LBM_EINVAL
        with pytest.raises(L.LbmError) as e:
            L.lbm_poll(srv, 12345, 8, 8)
        assert e.value.code == L.LBM_ENOTFOUND
    finally:
        L.lbm_server_destroy(srv)
