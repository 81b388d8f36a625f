"""Parity at the full workload sizes, in the launch configuration the
benchmark times, on sampled outputs.

A node's state after T steps depends only on the initial field within T
nodes, so the oracle computes sampled nodes one by one on a (2T+3)^2 window
(oracle.window_run) -- or whole lattices when they are small enough.
"""
import os

import numpy as np
import pytest

import lbm_inputs as inp
import oracle as orc

pytestmark = pytest.mark.gpu
# max |rho'_gpu - rho'_oracle| / A against the stated bars: FP32 1e-6,
# FP16 and BF16 2e-3.  BF16 keeps an 8-bit significand, so every stored
# population is rounded by up to 2^-9 = 1.95e-3 of itself each step; the
# cases below that miss the 2e-3 bar are marked as expected failures at that
# bar (strict: they fail the run if they start passing) and listed as
# misses in the design notes, not gated at a wider tolerance.
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


@pytest.fixture(scope="module")
def large_fields():
    n = 8192
    return inp.pulse_with_vortices(n, n, seed=1107 + 3)


def samples(n, T):
    # the pulse centre, a point on the outgoing ring, one in the quiet field
    c = n // 2
    r = int(round(inp.CS * T))
    return [(c, c), (c + r, c + 3), (1234, 6543)]


@pytest.mark.parametrize("dtype,T", [("f32", 1000), ("f16", 200), ("bf16", 200)])
def test_large_lattice_sampled(L, large_fields, dtype, T):
    """8192^2 lattice, optimized rates (Table 5 group A), pulse A = 1e-3
    (b = 20) plus vortical velocity (std 1e-4)."""
    n = 8192
    r = inp.rates("OPT")
    rho, ux, uy = large_fields
    h = L.lbm_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
    try:
        L.lbm_init_field(h, rho, ux, uy)
        L.lbm_step(h, T)
        got_rho = L.lbm_moments(h)[0]
        drift = L.lbm_drift(h)
    finally:
        L.lbm_destroy(h)
    assert drift[3] == 0
    errs = []
    for (x, y) in samples(n, T):
        f = orc.window_run(rho, ux, uy, inp.s_paper(r), T, x, y)
        errs.append(abs(got_rho[y, x] - f.sum()) / 1e-3)
    print("\n8192^2 %s T=%d sampled max|drho'|/A = %s" % (dtype, T, ["%.2e" % e for e in errs]))
    assert max(errs) <= TOL[dtype]


_BATCH = {}


def batch_results(L, dtype, T):
    """Run the 512-lattice batch once per storage type (cached): the three
    checked lattices' density fields after T batched steps."""
    if dtype in _BATCH:
        return _BATCH[dtype]
    specs = inp.batch_specs(512, seed=1107 + 4, steps=500)
    hs = []
    try:
        for spec in specs:
            h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                             L.DTYPES[dtype])
            L.lbm_init_field(h, *inp.batch_fields(spec))
            hs.append(h)
        b = L.lbm_batch_create(hs)
        L.lbm_batch_step(b, T)
        L.lbm_batch_destroy(b)
        areas = np.array([s["nx"] * s["ny"] for s in specs])
        order = np.argsort(areas)
        picks = {"small": int(order[5]), "medium": int(order[256]), "large": int(order[-1])}
        results = {name: (specs[k], L.lbm_moments(hs[k])[0]) for name, k in picks.items()}
    finally:
        for h in hs:
            L.lbm_destroy(h)
    _BATCH[dtype] = results
    return results


BF16_SMALL_MISS = pytest.mark.xfail(
    strict=True,
    reason="BF16 storage misses the stated 2e-3 bar on the smallest checked batch lattice "
           "(31 x 35, A = 1.9e-5, 200 steps): measured 2.03e-3 of the amplitude, one BF16 "
           "rounding being up to 1.95e-3 of a stored population")


@pytest.mark.parametrize("dtype,T,which", [
    ("f32", 500, "small"), ("f32", 500, "medium"), ("f32", 500, "large"),
    ("f16", 200, "small"), ("f16", 200, "medium"), ("f16", 200, "large"),
    pytest.param("bf16", 200, "small", marks=BF16_SMALL_MISS),
    ("bf16", 200, "medium"), ("bf16", 200, "large")])
def test_batched_workload_sampled(L, dtype, T, which):
    """The 512-lattice batch in the batched launch (FP32 deviation: the
    benchmark's 500 steps; the 16-bit types, measured with --batch-dtype,
    200 steps as for the large lattice); three lattices (small, medium,
    large) checked against the oracle: whole lattices when small, sampled
    windows otherwise."""
    spec, got = batch_results(L, dtype, T)[which]
    fields = inp.batch_fields(spec)
    s = inp.s_paper(spec["rates"])
    if spec["nx"] * spec["ny"] <= 400 * 400:
        want = orc.moments(orc.run(orc.init_eq(*fields), s, T))[0]
        err = np.max(np.abs(got - want)) / spec["amp"]
    else:
        pts = [(int(spec["xc"]), int(spec["yc"])), (0, 0), (spec["nx"] // 3, spec["ny"] - 1)]
        err = max(abs(got[y, x] - orc.window_run(*fields, s, T, x, y).sum()) / spec["amp"]
                  for (x, y) in pts)
    print("\nbatch %s %s lattice (%dx%d), T=%d: max|drho'|/A = %.2e"
          % (dtype, which, spec["nx"], spec["ny"], T, err))
    assert err <= TOL[dtype]
