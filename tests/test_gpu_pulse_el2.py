"""The Gaussian pulse of section 5.2 against its linear-acoustics solution,
reported in the paper's manner: the relative L2 error E_L2 of the density
(the fluctuation rho - rho0 here) over all nodes, on the [0,1]^2 domain at
physical time t = 0.4 with b = 0.04, for several resolutions.

With the paper's amplitude eps = 0.01 the simulation is nonlinear and the
reference solution is not: their difference, of order eps x (distance
travelled / width) ~ 7e-3, is reached by N = 512 and the error stops
falling there (reported, not gated).  At eps = 1e-4 the run is linear and
the error falls at second order in dx (gated).

Readings: the paper leaves the resolutions and the sound speed in physical
units unstated; here dx = dt = 1/N (so t = 0.4 is 0.4 N steps, b = 0.04 N
nodes, c_s = 1/sqrt(3)), and the reference solution is the inviscid one of
Eq. exactpules summed over periodic images (oracle.pulse.periodic).
"""
import math
import os

import numpy as np
import pytest

import lbm_inputs as inp
import oracle as orc
from oracle import pulse

pytestmark = pytest.mark.gpu
RES = (128, 256, 512, 1024)


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


def el2(L, N, name, U0, eps, dtype="f32", oracle=False):
    b, T = 0.04 * N, int(round(0.4 * N))
    r = inp.rates(name, nu=1e-3)
    fields = inp.gaussian_pulse(N, N, eps, b, N / 2, N / 2, u0=(U0, 0.0))
    if oracle:
        f = orc.run(orc.init_eq(*fields), inp.s_paper(r), T)
        got = orc.moments(f)[0] - 1.0
    else:
        h = L.lbm_create(N, N, inp.s_ll(r), 1.0, (U0, 0.0), L.DTYPES[dtype])
        try:
            L.lbm_init_field(h, *fields)
            L.lbm_step(h, T)
            got = L.lbm_moments(h)[0] - 1.0
        finally:
            L.lbm_destroy(h)
    th = pulse.periodic(N, N, N / 2, N / 2, T, eps, b, U0=U0)
    return float(np.linalg.norm(got - th) / np.linalg.norm(th))


def report(L, U0, eps):
    table = {}
    print("\nE_L2 of rho' at t = 0.4, U0 = %.1f, eps = %g, N = %s" % (U0, eps, list(RES)))
    for name in ("OPT", "OPT-B", "LL*"):
        row = [el2(L, N, name, U0, eps) for N in RES]
        orders = [math.log(row[i] / row[i + 1], 2) for i in range(len(row) - 1)]
        print("  %-6s %s   orders %s" % (name, " ".join("%.3e" % e for e in row),
                                         " ".join("%.2f" % o for o in orders)))
        table[name] = (row, orders)
    return table


@pytest.mark.parametrize("U0", [0.0, 0.1])
def test_pulse_el2_second_order_in_the_linear_regime(L, U0):
    table = report(L, U0, 1e-4)
    for name in ("OPT", "OPT-B"):  # the original rates at s_nu ~ 2 are reported only
        row, orders = table[name]
        assert all(np.isfinite(row))
        assert all(row[i + 1] < row[i] for i in range(len(row) - 1))
        assert 1.6 < orders[-1] < 2.4
    # the GPU run is the oracle's run up to FP32 storage rounding
    assert el2(L, 128, "OPT", U0, 1e-4) == pytest.approx(
        el2(L, 128, "OPT", U0, 1e-4, oracle=True), rel=1e-4)


def test_pulse_el2_at_the_papers_amplitude(L):
    table = report(L, 0.0, 0.01)
    row, _ = table["OPT"]
    assert all(np.isfinite(row)) and max(row[1:]) < 1e-2
