"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (all on the same seeded inputs):
  * LBM_F64: bit-identical populations (the kernels keep the oracle's
    operation order and are built without multiply-add contraction); the
    stated gate is a relative L2 error of the density fluctuation <= 1e-12;
  * LBM_F32DEV: max |rho'_gpu - rho'_oracle| <= 1e-6 A, A the initial
    fluctuation amplitude;
  * LBM_F16DEV / LBM_BF16DEV: max |rho'_gpu - rho'_oracle| <= 2e-3 A over
    the short runs below (longer runs are measured and reported, not gated).
"""
import math
import os

import numpy as np
import pytest

import lbm_inputs as inp
import oracle as orc

pytestmark = pytest.mark.gpu


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


def run_gpu(L, nx, ny, r, steps, dtype, fields=None, pops=None, u0=(0.0, 0.0), rho0=1.0):
    h = L.lbm_create(nx, ny, inp.s_ll(r), rho0, u0, dtype)
    try:
        if fields is not None:
            L.lbm_init_field(h, *fields)
        if pops is not None:
            L.lbm_set_populations(h, pops)
        L.lbm_step(h, steps)
        mom = L.lbm_moments(h)
        f = L.lbm_get_populations(h)
    finally:
        L.lbm_destroy(h)
    return mom, f


def run_orc(r, steps, fields=None, pops=None):
    f = orc.init_eq(*fields) if fields is not None else pops
    f = orc.run(f, inp.s_paper(r), steps)
    return orc.moments(f), f


def max_rel(a, b, amp):
    return float(np.max(np.abs(a - b)) / amp)


# --------------------------------------------------------------- FP64
def test_f64_config1_pulse_bit_identical(L):
    """64x64, Lallemand-Luo rates with nu = 1e-3, Gaussian pulse A = 1e-3,
    b = 4, 200 steps."""
    nx = ny = 64
    r = inp.rates("LL", nu=1e-3)
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 4.0)
    (rho, ux, uy), f = run_gpu(L, nx, ny, r, 200, L.LBM_F64, fields=fields)
    (rho_o, ux_o, uy_o), f_o = run_orc(r, 200, fields=fields)
    drho, drho_o = rho - 1.0, rho_o - 1.0
    assert np.linalg.norm(drho - drho_o) / np.linalg.norm(drho_o) <= 1e-12
    assert np.array_equal(f, f_o)
    assert np.array_equal(rho, rho_o) and np.array_equal(ux, ux_o) and np.array_equal(uy, uy_o)


@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (7, 2), (33, 17), (65, 9), (130, 7),
                                   (64, 64), (257, 3)])
def test_f64_random_populations_ragged_sizes(L, nx, ny):
    """Non-equilibrium populations on lattices that span several tiles, leave
    ragged row tails and wrap within one vector."""
    r = inp.rates("OPT")
    pops = inp.random_populations(nx, ny, seed=nx * 1000 + ny, amp=1e-2)
    _, f = run_gpu(L, nx, ny, r, 13, L.LBM_F64, pops=pops)
    _, f_o = run_orc(r, 13, pops=pops)
    assert np.array_equal(f, f_o)


def test_f64_mean_flow_plane_wave(L):
    nx, ny, steps = 512, 16, 400
    r = inp.rates("OPT")
    fields = inp.plane_wave(nx, ny, 1e-4, 64, U=0.1)
    _, f = run_gpu(L, nx, ny, r, steps, L.LBM_F64, fields=fields, u0=(0.1, 0.0))
    _, f_o = run_orc(r, steps, fields=fields)
    assert np.array_equal(f, f_o)


def test_f64_scaling_by_two_commutes(L):
    """m^eq is homogeneous of degree 1: step(2 f) = 2 step(f) bit for bit."""
    nx, ny = 37, 21
    r = inp.rates("LL", nu=2e-3)
    pops = inp.random_populations(nx, ny, seed=3, amp=1e-2)
    _, f1 = run_gpu(L, nx, ny, r, 20, L.LBM_F64, pops=pops)
    _, f2 = run_gpu(L, nx, ny, r, 20, L.LBM_F64, pops=2.0 * pops, rho0=2.0)
    assert np.array_equal(2.0 * f1, f2)


# ------------------------------------------------- FP64 deviation storage
# LBM_F64DEV collides FP64 deviations with fused multiply-adds, so it is not
# bit-identical to the oracle; its reference is the oracle's
# extended-precision build (oracle.run_ext, long double).  The stated FP64
# gate is 1e-12 relative L2 of rho'.  The plain FP64 oracle is itself only
# ~6e-12 from the extended build on config 1 (its populations of size ~0.4
# are rounded every step against a 1e-3 fluctuation), which the plain GPU
# path reproduces bit for bit; both figures are printed.
def rel_l2_rho(f, g):
    a, b = f.sum(axis=0) - 1.0, g.sum(axis=0) - 1.0
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["config1", "config1-fields", "mean-flow-plane-wave",
                                  "random-33x17", "random-130x7"])
def test_f64dev_matches_extended_oracle(L, case):
    if case.startswith("config1"):
        nx, ny, steps, r, u0 = 64, 64, 200, inp.rates("LL", nu=1e-3), (0.0, 0.0)
        fields = inp.gaussian_pulse(nx, ny, 1e-3, 4.0)
        f0 = orc.init_eq(*fields)
    elif case == "mean-flow-plane-wave":
        nx, ny, steps, r, u0 = 512, 16, 400, inp.rates("OPT"), (0.1, 0.0)
        fields = inp.plane_wave(nx, ny, 1e-4, 64, U=0.1)
        f0 = orc.init_eq(*fields)
    else:
        nx, ny = (33, 17) if case == "random-33x17" else (130, 7)
        steps, r, u0 = 13, inp.rates("OPT"), (0.0, 0.0)
        fields = None
        f0 = inp.random_populations(nx, ny, seed=nx + ny, amp=1e-3)
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, u0, L.LBM_F64DEV)
    try:
        if case == "config1-fields":
            L.lbm_init_field(h, *fields)
        else:
            L.lbm_set_populations(h, f0)
        L.lbm_step(h, steps)
        f = L.lbm_get_populations(h)
    finally:
        L.lbm_destroy(h)
    s = inp.s_paper(r)
    want = orc.run_ext(f0, s, steps)
    err = rel_l2_rho(f, want)
    err_plain = rel_l2_rho(orc.run(f0, s, steps), want)
    print("\nf64dev %s: rel L2 of rho' vs extended oracle %.2e (plain FP64 oracle: %.2e)"
          % (case, err, err_plain))
    assert err <= 1e-12


def test_f64dev_checkpoint_and_conservation(L):
    nx, ny = 40, 24
    r = inp.rates("OPT")
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 4.0, u0=(0.05, 0.02))
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, (0.05, 0.02), L.LBM_F64DEV)
    try:
        L.lbm_init_field(h, *fields)
        d0 = L.lbm_drift(h)
        L.lbm_step(h, 60)
        mid = L.lbm_get_populations(h)
        L.lbm_set_populations(h, mid)
        assert np.array_equal(L.lbm_get_populations(h), mid)
        L.lbm_step(h, 60)
        d1 = L.lbm_drift(h)
    finally:
        L.lbm_destroy(h)
    # FP64 deviations conserve mass and momentum to their own rounding
    assert np.all(np.abs(d1[:3] - d0[:3]) <= 1e-14 * np.abs(d0[:3]).max())


# ---------------------------------------------------------- deviation
DEV_TOL = {"f32": 1e-6, "f16": 2e-3, "bf16": 2e-3}


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_dev_config1_pulse(L, dtype):
    nx = ny = 64
    amp, steps = 1e-3, 200
    r = inp.rates("LL", nu=1e-3)
    fields = inp.gaussian_pulse(nx, ny, amp, 4.0)
    (rho, _, _), _ = run_gpu(L, nx, ny, r, steps, L.DTYPES[dtype], fields=fields)
    (rho_o, _, _), _ = run_orc(r, steps, fields=fields)
    err = max_rel(rho, rho_o, amp)
    print("\n%s config-1 pulse: max|drho'|/A = %.3e" % (dtype, err))
    assert err <= DEV_TOL[dtype]


# Random populations are a stress case, not a workload: each direction
# carries an independent deviation as large as the density fluctuation A
# itself, and each step rounds every stored deviation once.  The stated
# bars hold for FP32 and FP16; BF16 keeps 9 significant bits (one rounding
# is up to 2^-9 = 1.95e-3 of a stored population) and misses 2e-3 here.
RANDOM_TOL = {"f32": 1e-6, "f16": 2e-3, "bf16": 2e-3}
BF16_RANDOM_MISS = pytest.mark.xfail(
    strict=True,
    reason="BF16 storage misses the stated 2e-3 bar on random non-equilibrium populations "
           "(measured 3.2e-3 - 4.3e-3 of A after 17 steps): every direction carries a "
           "deviation as large as A, and one BF16 rounding is up to 2^-9 of a stored population")


def random_case(L, dtype, nx, ny):
    amp, steps = 1e-3, 17
    r = inp.rates("OPT")
    pops = inp.random_populations(nx, ny, seed=nx + 7 * ny, amp=amp)
    (rho, ux, uy), f = run_gpu(L, nx, ny, r, steps, L.DTYPES[dtype], pops=pops)
    (rho_o, ux_o, uy_o), f_o = run_orc(r, steps, pops=pops)
    A = np.max(np.abs(pops.sum(axis=0) - 1.0))
    errs = (max_rel(rho, rho_o, A), max_rel(f, f_o, A), max_rel(ux, ux_o, A))
    return pops, A, steps, errs


@pytest.mark.parametrize("dtype", [pytest.param("bf16", marks=BF16_RANDOM_MISS), "f16", "f32"])
@pytest.mark.parametrize("nx,ny", [(5, 3), (33, 17), (130, 7), (96, 40)])
def test_dev_random_populations_ragged(L, dtype, nx, ny):
    _, _, _, errs = random_case(L, dtype, nx, ny)
    print("\n%s random populations %dx%d: max|drho'|/A = %.2e, max|df|/A = %.2e"
          % (dtype, nx, ny, errs[0], errs[1]))
    assert max(errs) <= RANDOM_TOL[dtype]


@pytest.mark.parametrize("nx,ny", [(5, 3), (33, 17), (130, 7), (96, 40)])
def test_bf16_random_populations_within_rounding_bound(L, nx, ny):
    """Not the acceptance bar (that is missed, above) but the BF16 rounding
    model: after n steps of one rounding per stored deviation (relative
    2^-9 at most) the error stays below sqrt(n) 2^-9 max_node sum_i |f'_i|,
    the random-walk growth of the per-step roundings (~1e-2 of A here)."""
    pops, A, steps, errs = random_case(L, "bf16", nx, ny)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4).reshape(9, 1, 1)  # f^eq(1, 0)
    dev = np.abs(pops - w).sum(axis=0).max() / A
    bound = math.sqrt(steps) * 2.0 ** -9 * dev
    print("\nbf16 random populations %dx%d: %.2e of A against the rounding bound %.2e"
          % (nx, ny, max(errs), bound))
    assert max(errs) <= bound


# Over the 2000 steps of config 2 the FP32 storage rounding of every step
# feeds the shear-stress moments, which the s_nu = 1.99996 of Table 5 (LL*
# and OPT keep it) leaves almost undamped (|1 - s_nu| = 0.99996): the noise
# then integrates instead of relaxing.  The stated bar is 1e-6 of the
# amplitude for every set.  LL* with the mean flow U = 0.1 misses it: the
# von Neumann matrix of section 4.1 for those rates (optimized s_e, s_nu
# with the original s_eps = 1.54, s_q = 1.9) has a growing mode along the
# flow, |lambda| = 1.00098 at k_x = 3 pi / 4, which amplifies the storage
# rounding it is seeded with about sevenfold over 2000 steps (the FP64
# oracle's own rounding is 2^29 times smaller and stays invisible); measured
# 1.1e-6.  That case is an expected failure at the stated bar (strict), not
# a wider gate; test_llstar_mean_flow_has_growing_mode pins the mode.
PLANE_TOL = 1e-6
LLSTAR_U01_MISS = pytest.mark.xfail(
    strict=True,
    reason="LL* at U = 0.1 misses the stated 1e-6 bar in FP32 (measured 1.1e-6): a growing "
           "von Neumann mode (|lambda| = 1.00098 at k_x = 3 pi/4) amplifies storage rounding")


@pytest.mark.parametrize("dtype", ["f32"])
@pytest.mark.parametrize("U,name", [(0.0, "LL"), (0.1, "LL"), (0.1, "OPT"), (0.0, "OPT"),
                                    (0.0, "LL*"),
                                    pytest.param(0.1, "LL*", marks=LLSTAR_U01_MISS)])
def test_dev_plane_wave_config2(L, dtype, U, name):
    """512 x 16 plane wave (lambda = 8), amplitude 1e-4, 2000 steps, FP32
    deviation about f^eq(1, (U, 0))."""
    nx, ny, amp, steps = 512, 16, 1e-4, 2000
    r = inp.rates(name, nu=1e-3)
    fields = inp.plane_wave(nx, ny, amp, 64, U=U)
    (rho, _, _), _ = run_gpu(L, nx, ny, r, steps, L.DTYPES[dtype], fields=fields, u0=(U, 0.0))
    (rho_o, _, _), _ = run_orc(r, steps, fields=fields)
    err = max_rel(rho, rho_o, amp)
    print("\n%s plane wave U=%.1f %s: max|drho'|/A = %.3e" % (dtype, U, name, err))
    assert err <= PLANE_TOL


# ----------------------------------------------------- whole-path checks
@pytest.mark.parametrize("dtype", ["f64", "f32", "f16"])
def test_checkpoint_restore_is_exact(L, dtype):
    """100 steps straight equal 50 steps, get, set, 50 steps: bit for bit
    for FP64 and FP32; FP16 re-chooses its storage scale from the snapshot's
    largest deviation on restore, so there the two runs agree to the FP16
    bar (2e-3 of the amplitude) and a snapshot restored and read back moves
    by at most one FP16 rounding."""
    nx, ny = 40, 24
    r = inp.rates("OPT")
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 4.0)
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
    g = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
    try:
        L.lbm_init_field(h, *fields)
        L.lbm_step(h, 100)
        a = L.lbm_get_populations(h)
        L.lbm_init_field(g, *fields)
        L.lbm_step(g, 50)
        mid = L.lbm_get_populations(g)
        L.lbm_set_populations(g, mid)
        back = L.lbm_get_populations(g)
        L.lbm_step(g, 50)
        b = L.lbm_get_populations(g)
    finally:
        L.lbm_destroy(h)
        L.lbm_destroy(g)
    if dtype == "f16":
        err = np.max(np.abs(a - b)) / 1e-3
        print("\nf16 restore: max|df| / A = %.2e, read-back exact: %s"
              % (err, np.array_equal(back, mid)))
        assert err <= 2e-3
        assert np.max(np.abs(back - mid)) <= 1e-3 * 2.0 ** -11
    else:
        assert np.array_equal(back, mid)
        assert np.array_equal(a, b)


def test_fp16_reinit_with_a_new_scale_after_graph_runs(L):
    """An FP16 lattice re-initialised (or restored) with a field of another
    amplitude picks a new storage scale; runs long enough to replay the
    captured step graph (and the forced-step graph with a point source)
    must use it: the result equals that of a fresh lattice."""
    n, steps = 48, 130
    r = inp.rates("OPT")
    small = inp.gaussian_pulse(n, n, 1e-5, 4.0)
    large = inp.gaussian_pulse(n, n, 1e-2, 4.0)

    def fresh(fields, source):
        h = L.lbm_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.LBM_F16DEV)
        try:
            if source:
                L.lbm_set_source(h, 20, 21, 1e-3, 20.0)
            L.lbm_init_field(h, *fields)
            L.lbm_step(h, steps)
            return L.lbm_get_populations(h)
        finally:
            L.lbm_destroy(h)

    for source in (False, True):
        h = L.lbm_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.LBM_F16DEV)
        try:
            if source:
                L.lbm_set_source(h, 20, 21, 1e-3, 20.0)
            L.lbm_init_field(h, *small)
            L.lbm_step(h, steps)  # captures the graph at the small field's scale
            L.lbm_init_field(h, *large)
            L.lbm_step(h, steps)
            got = L.lbm_get_populations(h)
            snap = fresh(small, source)
            L.lbm_set_populations(h, snap)  # back to the small scale
            L.lbm_step(h, steps)
            got2 = L.lbm_get_populations(h)
        finally:
            L.lbm_destroy(h)
        assert np.array_equal(got, fresh(large, source)), source
        ref = L.lbm_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.LBM_F16DEV)
        try:
            if source:
                L.lbm_set_source(ref, 20, 21, 1e-3, 20.0)
            L.lbm_set_populations(ref, snap)
            L.lbm_step(ref, steps)
            want2 = L.lbm_get_populations(ref)
        finally:
            L.lbm_destroy(ref)
        assert np.array_equal(got2, want2), source
    # a source far beyond the scale of an FP16 state already stored is refused
    h = L.lbm_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.LBM_F16DEV)
    try:
        L.lbm_init_field(h, *small)
        with pytest.raises(L.LbmError):
            L.lbm_set_source(h, 20, 21, 1.0, 20.0)
    finally:
        L.lbm_destroy(h)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_drift_is_small_and_deterministic(L, dtype):
    nx = ny = 64
    r = inp.rates("LL", nu=1e-3)
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 4.0)
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
    try:
        L.lbm_init_field(h, *fields)
        d0 = L.lbm_drift(h)
        L.lbm_step(h, 200)
        d1 = L.lbm_drift(h)
        d2 = L.lbm_drift(h)
    finally:
        L.lbm_destroy(h)
    mass = 1e-3 * math.pi / (math.log(2) / 16)  # sum of the pulse
    assert abs(d0[0] - mass) / mass < 1e-3
    tol = 1e-11 if dtype == "f64" else 1e-5
    assert abs(d1[0] - d0[0]) <= tol * mass
    assert abs(d1[1]) <= tol * mass and abs(d1[2]) <= tol * mass
    assert d1[3] == 0
    assert np.array_equal(d1, d2)


# Drift (the a7 reduction) against the oracle, with a mean flow so that the
# momentum sums are far from zero: a Gaussian pulse A = 1e-2 (b = 6) carried
# by u0 = (0.1, -0.05) has sum rho' = A pi / alpha and sum j' = u0 sum rho'.
# Collision and streaming conserve both (section 2.1, Eq. eq_conservative),
# so the exact values at any time are those of the initial field.
#   * FP64 storage: the GPU state is the oracle's bit for bit, so lbm_drift
#     must equal the sums of the oracle's state to 1e-12 relative (only the
#     order of the lattice-wide sum differs), and the initial field's exact
#     sums within the rounding of the FP64 initial populations (FP64
#     conservation);
#   * FP32 deviation storage: every stored deviation is rounded once per step
#     (relative error <= 2^-24), which does not conserve mass exactly; over
#     T steps the sums can move by at most T 2^-24 sum|f'| (the storage
#     rounding bound, sum|f'| taken at twice its initial value), against the
#     exact initial sums and against the oracle's state.
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_drift_matches_oracle_with_mean_flow(L, dtype):
    nx, ny, T, amp, b = 80, 64, 150, 1e-2, 6.0
    u0 = (0.1, -0.05)
    r = inp.rates("LL", nu=1e-3)
    s = inp.s_paper(r)
    fields = inp.gaussian_pulse(nx, ny, amp, b, u0=u0)
    rho_in = fields[0]
    exact = np.array([(rho_in - 1.0).sum(), u0[0] * (rho_in - 1.0).sum(),
                      u0[1] * (rho_in - 1.0).sum()])
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, u0, L.DTYPES[dtype])
    try:
        L.lbm_init_field(h, *fields)
        d0 = L.lbm_drift(h)
        L.lbm_step(h, T)
        d1 = L.lbm_drift(h)
    finally:
        L.lbm_destroy(h)
    f0 = orc.init_eq(*fields)
    f_o = orc.run(f0, s, T)
    cx, cy = orc.velocities()
    base = orc.init_eq(np.ones((1, 1)), np.full((1, 1), u0[0]), np.full((1, 1), u0[1]))
    dev = f_o - base
    want = np.array([dev.sum(), (cx[:, None, None] * dev).sum(), (cy[:, None, None] * dev).sum()])
    assert d0[3] == 0 and d1[3] == 0
    print("\n%s drift: GPU %s oracle %s exact %s" % (dtype, d1[:3], want, exact))
    if dtype == "f64":
        assert np.all(np.abs(d1[:3] - want) <= 1e-12 * np.abs(want))
        # conservation: each FP64 population of the initial equilibrium is
        # rounded once (<= 2^-53 of it), and those roundings need not cancel
        # in the sums
        cons = 9 * nx * ny * 2.0 ** -53 * np.max(np.abs(f0))
        assert np.all(np.abs(d1[:3] - exact) <= cons)
        assert np.all(np.abs(d0[:3] - exact) <= cons)
    else:
        # the deviation types hold the reference momentum as the FP32 number
        # nearest rho0 u0, and lbm_drift measures j' against that value
        off = nx * ny * (np.array(u0) - np.array(u0, dtype=np.float32).astype(np.float64))
        exact[1:] += off
        want[1:] += off
        bound = (T + 1) * 2.0 ** -24 * 2.0 * np.abs(f0 - base).sum()
        assert np.all(np.abs(d0[:3] - exact) <= 2.0 ** -24 * np.abs(f0 - base).sum())
        assert np.all(np.abs(d1[:3] - exact) <= bound)
        assert np.all(np.abs(d1[:3] - want) <= bound)
    # the sums are those of a moving pulse: momentum = u0 x mass, no sign or
    # component swapped
    assert d1[1] > 0 > d1[2]


def test_nonfinite_state_is_reported(L):
    """A density of nearly zero makes 1/rho overflow: the drift check must
    report non-finite populations (no fault, only IEEE arithmetic)."""
    nx = ny = 16
    r = inp.rates("LL", nu=1e-3)
    rho = np.full((ny, nx), 1.0)
    ux = np.zeros((ny, nx))
    uy = np.zeros((ny, nx))
    ux[8, 8] = 1e30
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, (0.0, 0.0), L.LBM_F32DEV)
    try:
        L.lbm_init_field(h, rho, ux, uy)
        L.lbm_step(h, 3)
        d = L.lbm_drift(h)
    finally:
        L.lbm_destroy(h)
    assert d[3] > 0


def test_invalid_arguments_are_rejected(L):
    S = inp.s_ll(inp.rates("OPT"))
    bad = S.copy()
    bad[1] = 2.5
    for args in ((1, 8, S), (8, 8, bad)):
        with pytest.raises(L.LbmError) as e:
            L.lbm_create(*args)
        assert e.value.code == L.LBM_EINVAL
    with pytest.raises(L.LbmError):
        L.lbm_create(8, 8, S, rho0=-1.0)
    h = L.lbm_create(8, 8, S)
    try:
        with pytest.raises(L.LbmError):
            L.lbm_step(h, -1)
        with pytest.raises(L.LbmError):
            L.lbm_init_field(h, np.zeros((8, 8)), np.zeros((8, 8)), np.zeros((8, 8)))
    finally:
        L.lbm_destroy(h)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16", "bf16"])
def test_translation_shifts_the_result(L, dtype):
    """Every node runs the same arithmetic: stepping a shifted initial field
    gives the shifted result bit for bit (no oracle needed)."""
    nx, ny, steps = 45, 26, 37
    r = inp.rates("OPT")
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 3.0, 14.3, 9.6)
    shifted = tuple(np.roll(a, (5, 11), axis=(0, 1)) for a in fields)
    (rho_a, _, _), _ = run_gpu(L, nx, ny, r, steps, L.DTYPES[dtype], fields=fields)
    (rho_b, _, _), _ = run_gpu(L, nx, ny, r, steps, L.DTYPES[dtype], fields=shifted)
    assert np.array_equal(np.roll(rho_a, (5, 11), axis=(0, 1)), rho_b)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 1e-6)])
def test_centred_pulse_keeps_d4_symmetry(L, dtype, tol):
    """A pulse centred on a node of a square lattice at rest stays symmetric
    under the 8 symmetries of the square, up to rounding: mirrored nodes
    add their populations in different orders (FP64: ~1e-15 on rho ~ 1)."""
    n, steps, amp = 48, 120, 1e-3
    r = inp.rates("LL", nu=1e-3)
    fields = inp.gaussian_pulse(n, n, amp, 4.0, 24.0, 24.0)
    (rho, _, _), _ = run_gpu(L, n, n, r, steps, L.DTYPES[dtype], fields=fields)
    d = rho - 1.0
    c = np.roll(d, (-24, -24), axis=(0, 1))  # centre at index 0
    # reflections i -> -i (mod n) about the centre, and the diagonal
    images = (np.roll(c[::-1, :], 1, axis=0), np.roll(c[:, ::-1], 1, axis=1), c.T,
              np.roll(c[::-1, ::-1], (1, 1), axis=(0, 1)))
    assert np.max(np.abs(d)) > 1e-2 * amp
    for img in images:
        assert np.max(np.abs(img - c)) <= tol * amp


@pytest.mark.parametrize("dtype,tol", [("f64", 0.0), ("f32", 1e-6)])
def test_bgk_rates_match_oracle(L, dtype, tol):
    """All non-conserved rates equal: the single-relaxation-time scheme of
    section 2.1 (Lambda = s I) as a special case of the MRT path."""
    nx, ny, steps, amp = 40, 36, 150, 1e-3
    sv = 1.0 / (0.5 + 3e-3)
    r = dict(s_e=sv, s_eps=sv, s_q=sv, s_nu=sv)
    fields = inp.gaussian_pulse(nx, ny, amp, 4.0)
    (rho, _, _), f = run_gpu(L, nx, ny, r, steps, L.DTYPES[dtype], fields=fields)
    (rho_o, _, _), f_o = run_orc(r, steps, fields=fields)
    assert np.max(np.abs(rho - rho_o)) <= tol * amp
    if dtype == "f64":
        assert np.array_equal(f, f_o)


def point_source_rates(name):
    """The three schemes of section 5.1 with Table 4's s_e = s_nu: BGK (all
    rates s_nu), the original MRT (Lallemand-Luo s_eps, s_q) and the
    optimized one (Table 4 group A)."""
    t = inp.TABLE4["A"]
    if name == "BGK":
        return dict(s_e=t["s_nu"], s_eps=t["s_nu"], s_q=t["s_nu"], s_nu=t["s_nu"])
    if name == "original":
        return dict(s_e=t["s_e"], s_eps=inp.LL["s_eps"], s_q=inp.LL["s_q"], s_nu=t["s_nu"])
    return inp.rates("OPT-Z")


@pytest.mark.parametrize("name", ["BGK", "original", "optimized"])
@pytest.mark.parametrize("dtype,tol", [("f64", 0.0), ("f32", 1e-6)])
def test_point_source_matches_oracle(L, name, dtype, tol):
    """Section 5.1: 101 x 101 periodic lattice, source at the centre,
    rho_s = 0.01, period T = 20 (the paper leaves T unstated), t = 80."""
    n, rs, T, steps = 101, 0.01, 20.0, 80
    r = point_source_rates(name)
    h = L.lbm_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
    try:
        L.lbm_set_source(h, 50, 50, rs, T)
        L.lbm_step(h, steps)
        rho = L.lbm_moments(h)[0]
        f = L.lbm_get_populations(h)
    finally:
        L.lbm_destroy(h)
    f0 = orc.init_eq(np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
    f_o = orc.run_source(f0, inp.s_paper(r), steps, (50, 50, rs, T))
    rho_o = orc.moments(f_o)[0]
    assert np.max(np.abs(rho_o - 1.0)) > 1e-3 * rs
    assert np.max(np.abs(rho - rho_o)) <= tol * rs
    if dtype == "f64":
        assert np.array_equal(f, f_o)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_point_source_isotropy_claim_on_the_gpu(L, dtype):
    """Section 5.1 through the C ABI: at t = 80 the optimized rates' radiated
    wave is an order of magnitude more isotropic than BGK's and the original
    MRT's, with two orders less energy at the grid's highest wavenumbers."""
    from test_oracle_pins import source_field_metrics

    n = 101
    got = {}
    for name in ("BGK", "original", "optimized"):
        h = L.lbm_create(n, n, inp.s_ll(point_source_rates(name)), 1.0, (0.0, 0.0),
                         L.DTYPES[dtype])
        try:
            L.lbm_set_source(h, 50, 50, 0.01, 20.0)
            L.lbm_step(h, 80)
            got[name] = source_field_metrics(L.lbm_moments(h)[0] - 1.0)
        finally:
            L.lbm_destroy(h)
    aniso, high = got["optimized"]
    print("\n%s point source t=80: anisotropy / high-k energy %s" % (dtype, got))
    assert aniso < 0.05 and aniso < 0.25 * min(got["BGK"][0], got["original"][0])
    assert high < 1e-3 and high < 0.1 * min(got["BGK"][1], got["original"][1])


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_tuning_leaves_state_unchanged(L, dtype):
    """Trial launches of the tuner write only the idle buffer; every launch
    variant then gives the same populations."""
    nx, ny = 300, 70
    r = inp.rates("OPT")
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
    g = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
    try:
        fields = inp.gaussian_pulse(nx, ny, 1e-3, 6.0)
        L.lbm_init_field(h, *fields)
        L.lbm_init_field(g, *fields)
        L.lbm_step(h, 5)
        L.lbm_step(g, 5)
        before = L.lbm_get_populations(h)
        times, chosen = L.lbm_tune(h)
        assert np.all(times > 0) and 0 <= chosen < L.LBM_TUNE_VARIANTS
        assert np.array_equal(before, L.lbm_get_populations(h))
        L.lbm_step(h, 9)
        L.lbm_step(g, 9)
        assert np.array_equal(L.lbm_get_populations(h), L.lbm_get_populations(g))
    finally:
        L.lbm_destroy(h)
        L.lbm_destroy(g)


def test_analytic_init_matches_host_fields(L):
    """The device-side Gaussian initial field equals the host recipe to
    rounding (exp evaluated on different machines)."""
    nx, ny = 50, 30
    r = inp.rates("OPT")
    params = (1e-3, 4.0, 12.3, 20.7)
    h = L.lbm_create(nx, ny, inp.s_ll(r), 1.0, (0.0, 0.0), L.LBM_F64)
    try:
        L.lbm_init_analytic(h, L.LBM_INIT_GAUSSIAN, params)
        rho, _, _ = L.lbm_moments(h)
    finally:
        L.lbm_destroy(h)
    want = inp.gaussian_pulse(nx, ny, *params)[0]
    assert np.max(np.abs(rho - want)) < 1e-15 * 4


def test_torch_caching_allocator_through_lbm_set_allocator(L):
    """The library's device memory can come from torch's caching allocator
    (lbm_set_allocator with ctypes callbacks); results are unchanged."""
    import ctypes

    import torch

    calls = {"alloc": 0, "free": 0}

    @ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    def alloc(nbytes, ctx):
        calls["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(int(nbytes))

    @ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
    def free(ptr, ctx):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    nx, ny = 70, 50
    r = inp.rates("OPT")
    fields = inp.gaussian_pulse(nx, ny, 1e-3, 4.0)
    (want, _, _), _ = run_gpu(L, nx, ny, r, 40, L.LBM_F32DEV, fields=fields)
    L.lbm_set_allocator(alloc, free)
    try:
        (got, _, _), _ = run_gpu(L, nx, ny, r, 40, L.LBM_F32DEV, fields=fields)
    finally:
        L.lbm_set_allocator(None, None)
    assert calls["alloc"] > 0 and calls["free"] == calls["alloc"]
    assert np.array_equal(got, want)


TUNE_SCRIPT = """
import lbm_inputs as inp
from paper_1107_4543_gb300 import lbm as L
L.load()
h = L.lbm_create(1024, 1024, inp.s_ll(inp.rates("OPT")), 1.0, (0.0, 0.0), L.LBM_F32DEV)
assert L.lbm_get_variant(h) == -1
L.lbm_init_analytic(h, L.LBM_INIT_GAUSSIAN, (1e-3, 8.0, 512.0, 512.0))
L.lbm_step(h, 1)
print("VARIANT", L.lbm_get_variant(h))
L.lbm_destroy(h)
"""


def test_tuning_file_is_written_and_read(L, tmp_path):
    """LBM_TUNE_CACHE: the first process tunes a 2^20-node lattice and
    appends its choice; a second process takes the (edited) choice from the
    file instead of timing."""
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = tmp_path / "tune.txt"
    env = dict(os.environ, LBM_TUNE_CACHE=str(path), LBM_AUTOTUNE="1")

    def run():
        r = subprocess.run([sys.executable, "-c", TUNE_SCRIPT], cwd=root, env=env,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        return int(r.stdout.split("VARIANT")[1].split()[0])

    v = run()
    lines = path.read_text().split("\n")
    rec = [ln.split() for ln in lines if " L 1:1024:1024 " in ln]
    assert len(rec) == 1 and int(rec[0][3]) == v and 0 <= v < 3
    w = (v + 1) % 3
    path.write_text("%s L 1:1024:1024 %d\n" % (rec[0][0], w))
    assert run() == w
