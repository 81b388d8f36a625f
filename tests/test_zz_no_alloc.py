"""The no-allocation drift entry point against the allocating one.

lbm_drift_pop_noalloc serves callers that cannot allocate device memory
(their own allocator owns the GPU's memory, or they run under a fixed memory
budget): it reduces a caller-owned population array using a fixed scratch
array inside the library.  It must return the sums lbm_drift returns for
the same state, on repeated calls (the shared scratch keeps the previous
call's contents).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import lbm_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1107_4543_gb300 import build, lbm

    build.build()
    lbm.load()
    return torch, lbm


def state(L, nx, ny, steps, u0=(0.0, 0.0)):
    r = inp.rates("LL", nu=1e-3)
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, u0, L.LBM_F64)
    L.lbm_init_field(h, *inp.gaussian_pulse(nx, ny, 1e-3, 4.0, u0=u0))
    L.lbm_step(h, steps)
    return h


@pytest.mark.parametrize("nx,ny,u0", [(64, 64, (0.0, 0.0)), (37, 101, (0.1, 0.0)),
                                      (130, 7, (0.0, -0.05))])
def test_noalloc_drift_equals_lbm_drift(env, nx, ny, u0):
    torch, L = env
    h = state(L, nx, ny, 40, u0)
    try:
        want = L.lbm_drift(h)
        f = torch.from_numpy(L.lbm_get_populations(h)).cuda()
    finally:
        L.lbm_destroy(h)
    j0 = (1.0 * u0[0], 1.0 * u0[1])
    scale = 1e-3 * 16 * np.pi / np.log(2)  # size of the pulse's mass
    for _ in range(2):  # two calls in a row share the scratch array
        got = L.lbm_drift_pop_noalloc(f, nx, ny, 1.0, j0)
        assert np.max(np.abs(got[:3] - want[:3])) <= 1e-12 * scale
        assert got[3] == want[3] == 0


def test_noalloc_rejects_oversize_and_counts_nonfinite(env):
    torch, L = env
    f = torch.zeros((9, 8193, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LbmError) as e:
        L.lbm_drift_pop_noalloc(f, 2, 8193)
    assert e.value.code == L.LBM_EINVAL
    g = torch.full((9, 4, 4), 1.0 / 9.0, dtype=torch.float64, device="cuda")
    g[3, 2, 1] = float("nan")
    out = L.lbm_drift_pop_noalloc(g, 4, 4)
    assert out[3] == 1
