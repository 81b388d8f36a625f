"""The debug build's device-side index checks (compiled with
-DLBM_DEBUG_BOUNDS into _build_debug/liblbm.so).

No sanitizer runs on this pool, so the kernels whose indices depend on data
or on loop state carry checks of their own in that build: a failed check
sets a bit of a device word and the access is redirected to the array's
first element (no trap).  A fresh process loads the debug library and runs
small cases of every checked kernel -- the von Neumann sweep, the optimizer
cost (orders 3 - 6, both kinds), batched steps in every launch variant with
mixed storage types (plain and persistent grids, the small members held in
shared memory, ragged step counts through the server), the pipelined
solve's batched FP16 scales, init and moments -- and the
word must stay zero; the self-test (one checked access past its bound) must
set its bit, which shows the checks are live.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import lbm_inputs as inp
from paper_1107_4543_gb300 import build, lbm as L
L.load(build.build(debug=True))
out = {}
L.lbm_debug_bounds(reset=True)
# von Neumann sweep: random wavevectors, flows and rate sets
rng = np.random.default_rng(3)
n = 512
names = ["LL", "OPT", "OPT-Z", "LL*", "OPT-B"]
S = np.array([inp.s_ll(inp.rates(names[i % 5], nu=1e-3)) for i in range(n)])
L.lbm_vn_eigs(rng.uniform(-3.1, 3.1, n), rng.uniform(-3.1, 3.1, n),
              rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n), S)
out["vn"] = L.lbm_debug_bounds()
# optimizer costs: both kinds, orders 3..6, all parts
t3 = inp.TABLE3["A"]
sig = np.array([[t3["sigma_e"], 0.1, 0.2, t3["sigma_nu"]], [0.01, 0.3, 0.05, 0.002]])
for kind in ("F", "G"):
    for order in (3, 4, 5, 6):
        for part in ("all", "odd", "even"):
            L.lbm_opt_cost(L.cost_spec(kind, order, part), sig)
out["opt"] = L.lbm_debug_bounds()
# batched steps, every launch variant, FP32 / FP16 / BF16 members
specs = inp.batch_specs(9, seed=5, amin=6 * 6, amax=300 * 300)
hs = []
for k, sp in enumerate(specs):
    h = L.lbm_create(sp["nx"], sp["ny"], inp.s_ll(sp["rates"]), 1.0, (0.0, 0.0),
                     (L.LBM_F32DEV, L.LBM_F16DEV, L.LBM_BF16DEV)[k % 3])
    L.lbm_init_field(h, *inp.batch_fields(sp))
    hs.append(h)
b = L.lbm_batch_create(hs)
for v in range(L.LBM_BATCH_TUNE_VARIANTS):
    L.lbm_batch_set_variant(b, v)
    L.lbm_batch_step(b, 67)
L.lbm_batch_drift(b, len(hs))
L.lbm_batch_destroy(b)
for h in hs:
    L.lbm_destroy(h)
out["batch"] = L.lbm_debug_bounds()
# ragged generations through the server
srv = L.lbm_server_create(2 ** 30, 23)
ids = []
for q in inp.request_stream(12, rate=1e9, seed=9, side=(8, 60), steps=(1, 90)):
    req, _ = L.make_request(q["nx"], q["ny"], inp.s_ll(q["rates"]), q["steps"], dtype=q["dtype"],
                            init_kind=L.LBM_INIT_GAUSSIAN, init_params=(1e-3, 4.0, 3.0, 3.0))
    ids.append(L.lbm_submit(srv, req))
left = set(ids)
import time
t0 = time.time()
while left and time.time() - t0 < 120:
    for rid in L.lbm_server_done(srv):
        L.lbm_poll(srv, rid)
        left.discard(rid)
    time.sleep(0.01)
L.lbm_server_destroy(srv)
out["serve"] = L.lbm_debug_bounds()
out["served_all"] = not left
# pipelined solves: the batched init and moments kernels
specs = inp.batch_specs(7, seed=6, amin=20 * 20, amax=200 * 200)
hs = [L.lbm_create(sp["nx"], sp["ny"], inp.s_ll(sp["rates"]), 1.0, (0.0, 0.0),
                   (L.LBM_F32DEV, L.LBM_BF16DEV, L.LBM_F16DEV)[k % 3])
      for k, sp in enumerate(specs)]
b = L.lbm_batch_create(hs)
tot = L.lbm_batch_size(b)[1]
fin = [np.concatenate([f[c].ravel() for f in (inp.batch_fields(sp) for sp in specs)])
       for c in range(3)]
fout = tuple(np.empty(tot) for _ in range(3))
for _ in range(3):
    L.lbm_batch_solve_packed(b, 5, fin, fout)
L.lbm_batch_wait(b)
L.lbm_batch_destroy(b)
for h in hs:
    L.lbm_destroy(h)
out["solve"] = L.lbm_debug_bounds()
L.lbm_debug_bounds_selftest()
out["selftest"] = L.lbm_debug_bounds(reset=True)
out["after_reset"] = L.lbm_debug_bounds()
print("BOUNDS " + json.dumps(out))
'''


def test_debug_build_index_checks_stay_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1107_4543_gb300 import build

    build.build(debug=True)
    r = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT), 1)],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("BOUNDS ")][-1]
    res = json.loads(line[len("BOUNDS "):])
    print("\n" + json.dumps(res))
    for k in ("vn", "opt", "batch", "serve", "solve"):
        assert res[k] == 0, (k, res[k])
    assert res["served_all"]
    assert res["selftest"] == 1 << 31   # the checks are compiled in and report
    assert res["after_reset"] == 0
