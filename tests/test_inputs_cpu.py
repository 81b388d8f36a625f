"""The seeded synthetic inputs follow the stated recipes (the 512-lattice
batch, the Poisson request stream, the Gaussian pulse and the plane wave of
sections 5.1-5.2), and the same seed gives the same workload."""
import math

import numpy as np
import pytest

import lbm_inputs as inp


def test_batch_workload_recipe():
    specs = inp.batch_specs(512, seed=1107 + 4, steps=500)
    assert specs == inp.batch_specs(512, seed=1107 + 4, steps=500)  # seeded
    nodes = sum(s["nx"] * s["ny"] for s in specs)
    assert nodes == 67398739  # the node count the benchmark line reports
    area = np.array([s["nx"] * s["ny"] for s in specs], dtype=float)
    aspect = np.array([s["nx"] / s["ny"] for s in specs])
    assert area.min() > 0.8 * 32 ** 2 and area.max() < 1.2 * 1024 ** 2
    assert aspect.min() > 0.2 and aspect.max() < 5.0
    # log-uniform areas: the median area near the geometric mean
    assert 0.7 < np.median(area) / (32 * 1024) < 1.4
    s_e = np.array([s["rates"]["s_e"] for s in specs])
    nu = np.array([s["nu"] for s in specs])
    amp = np.array([s["amp"] for s in specs])
    assert s_e.min() >= 1.0 and s_e.max() <= 1.99
    assert nu.min() >= 1e-4 and nu.max() <= 1e-2
    assert amp.min() >= 1e-5 and amp.max() <= 1e-3
    for s in specs:
        assert s["rates"]["s_nu"] == pytest.approx(1.0 / (3.0 * s["nu"] + 0.5))
        assert 0 <= s["xc"] < s["nx"] and 0 <= s["yc"] < s["ny"] and s["b"] == 4.0
    assert 0.4 < np.mean([s["set"] == "OPT" for s in specs]) < 0.6


def test_request_stream_recipe():
    reqs = inp.request_stream(10000, seed=1107 + 5)
    gaps = np.diff([0.0] + [r["arrival"] for r in reqs])
    assert np.mean(gaps) == pytest.approx(1.0 / 200.0, rel=0.05)  # Poisson at 200/s
    side = np.array([r["nx"] for r in reqs])
    steps = np.array([r["steps"] for r in reqs])
    assert side.min() >= 64 and side.max() <= 2048 and all(r["nx"] == r["ny"] for r in reqs)
    assert steps.min() >= 100 and steps.max() <= 5000
    for key, value in (("dtype", "f16"), ("set", "OPT")):
        assert 0.47 < np.mean([r[key] == value for r in reqs]) < 0.53
    assert 0.47 < np.mean([r["init"]["kind"] == "plane" for r in reqs]) < 0.53


def test_gaussian_pulse_half_width_and_periodic_image():
    """rho' = A exp(-ln2 eta^2 / b^2): A at the centre, A/2 at distance b,
    measured by the minimum-image distance on the periodic lattice."""
    n, A, b = 64, 1e-3, 4.0
    rho, ux, uy = inp.gaussian_pulse(n, n, A, b, 10.0, 20.0, u0=(0.1, 0.0))
    assert rho[20, 10] - 1.0 == pytest.approx(A, rel=1e-14)
    assert rho[20, 14] - 1.0 == pytest.approx(A / 2, rel=1e-14)
    assert rho[24, 10] - 1.0 == pytest.approx(A / 2, rel=1e-14)
    # across the wrap: x = 10 - 4 + 64 = 70 -> column 6 is at distance 4
    assert rho[20, 6] - 1.0 == pytest.approx(A / 2, rel=1e-14)
    rho2, _, _ = inp.gaussian_pulse(n, n, A, b, 62.0, 20.0)
    assert rho2[20, 2] - 1.0 == pytest.approx(A / 2, rel=1e-14)  # 62 + 4 wraps to 2
    assert np.all(ux == 0.1) and np.all(uy == 0.0)


def test_plane_wave_is_a_right_running_acoustic_wave():
    """rho' = A cos(k x), u' = c_s rho' / rho0: the right-running
    characteristic of linear acoustics (u' = c_s rho'/rho0)."""
    n, A, m = 64, 1e-4, 3
    rho, ux, uy = inp.plane_wave(n, 8, A, m, U=0.1)
    k = 2 * math.pi * m / n
    assert np.allclose(rho[3] - 1.0, A * np.cos(k * np.arange(n)), atol=1e-18)
    assert np.allclose(ux - 0.1, inp.CS * (rho - 1.0), atol=1e-18)
    assert np.all(uy == 0.0)
