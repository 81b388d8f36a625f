"""Pins of the CPU oracle to what the paper and the mathematics fix.

None of these checks re-types the oracle's own formulas: each compares it
with an independent statement (the textbook polynomial equilibrium, the
printed Psi of section 2.3, the printed tables, closed-form limits of
section 4.1, numpy's roll/FFT/eig).  A dropped term, a wrong sign, a swapped
moment row or a transposed operand in the oracle fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest

import lbm_inputs as inp
import oracle as orc
from oracle import vn

HERE = os.path.dirname(os.path.abspath(__file__))
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def feq_poly(rho, ux, uy, cx, cy):
    """Textbook second-order D2Q9 equilibrium, written independently."""
    cu = cx * ux + cy * uy
    return W * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))


@pytest.fixture(scope="module")
def vel():
    return orc.velocities()


def test_velocity_set_is_d2q9(vel):
    cx, cy = vel
    assert cx[0] == 0 and cy[0] == 0
    pairs = {(int(a), int(b)) for a, b in zip(cx, cy)}
    assert pairs == {(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)}
    # the opposite of every velocity is in the set
    for a, b in pairs:
        assert (-a, -b) in pairs


def test_moment_matrix_conditions_and_orthogonality(vel):
    """M_0j = 1, M_aj = v_j^a (section 2.1); rows orthogonal with the
    Lallemand-Luo norms."""
    cx, cy = vel
    M, Mi = orc.matrices()
    assert np.array_equal(M[0], np.ones(9))
    assert np.array_equal(M[1], cx)
    assert np.array_equal(M[2], cy)
    G = M @ M.T
    assert np.array_equal(G, np.diag([9, 6, 6, 36, 36, 12, 12, 4, 4]).astype(float))
    assert np.max(np.abs(M @ Mi - np.eye(9))) < 1e-15
    # same matrix as the polynomial basis built independently in oracle.vn
    assert np.array_equal(M, vn.moment_matrix())


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments_give_polynomial_equilibrium(vel, seed):
    """M^-1 m^eq(rho, j) of section 2.3 equals the textbook f^eq."""
    cx, cy = vel
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.8, 1.2)
    ux, uy = rng.uniform(-0.2, 0.2, 2)
    _, Mi = orc.matrices()
    f = Mi @ orc.meq(rho, rho * ux, rho * uy)
    assert np.max(np.abs(f - feq_poly(rho, ux, uy, cx, cy))) < 2e-16 * 8
    # and the oracle's lattice init agrees
    fl = orc.init_eq(np.full((1, 1), rho), np.full((1, 1), ux), np.full((1, 1), uy))
    assert np.max(np.abs(fl[:, 0, 0] - feq_poly(rho, ux, uy, cx, cy))) < 2e-15


@pytest.mark.parametrize("U,V", [(0.0, 0.0), (0.1, 0.0), (0.07, -0.05)])
def test_meq_jacobian_matches_printed_psi(U, V):
    """Linearizing the oracle's m^eq about (rho=1, U, V) and relaxing with S
    reproduces every entry of the Psi printed in section 2.3."""
    s = inp.s_paper(dict(s_e=1.3, s_eps=1.7, s_q=0.6, s_nu=1.9))
    h = 1e-6
    J = np.zeros((9, 3))
    w0 = np.array([1.0, U, V])
    for c in range(3):
        d = np.zeros(3)
        d[c] = h
        J[:, c] = (orc.meq(*(w0 + d)) - orc.meq(*(w0 - d))) / (2 * h)
    S = np.diag(s)
    Psi = np.eye(9) - S
    Psi[3:, :3] += S[3:, 3:] @ J[3:, :]
    assert np.max(np.abs(Psi - vn.psi(U, V, s))) < 1e-9


@pytest.mark.parametrize("seed", range(4))
def test_collision_conserves_mass_and_momentum(vel, seed):
    cx, cy = vel
    rng = np.random.default_rng(seed)
    s = inp.s_paper(dict(s_e=rng.uniform(0.2, 2), s_eps=rng.uniform(0.2, 2),
                         s_q=rng.uniform(0.2, 2), s_nu=rng.uniform(0.2, 2)))
    f = W * (1 + 0.05 * rng.standard_normal(9))
    g = orc.collide(s, f)
    for row in (np.ones(9), cx, cy):
        assert abs(row @ g - row @ f) < 4e-16
    # the collision really moves the non-conserved moments
    assert np.max(np.abs(g - f)) > 1e-4


def test_equilibrium_is_fixed_point(vel):
    cx, cy = vel
    s = inp.s_paper(inp.rates("OPT"))
    f = feq_poly(1.02, 0.08, -0.03, cx, cy)
    assert np.max(np.abs(orc.collide(s, f) - f)) < 1e-16 * 4
    rho = np.full((6, 7), 1.02)
    f = orc.init_eq(rho, np.full((6, 7), 0.08), np.full((6, 7), -0.03))
    g = orc.run(f, s, 10)
    assert np.max(np.abs(g - f)) < 1e-15


def test_bgk_special_case(vel):
    """All rates equal s: Lambda = s I (section 2.1, Eq. eq_BGK_LBM_R)."""
    cx, cy = vel
    rng = np.random.default_rng(3)
    sv = 1.0 / 0.53
    f = W * (1 + 0.05 * rng.standard_normal(9))
    rho = f.sum()
    ux, uy = (cx @ f) / rho, (cy @ f) / rho
    bgk = f - sv * (f - feq_poly(rho, ux, uy, cx, cy))
    g = orc.collide(np.full(9, sv), f)
    assert np.max(np.abs(g - bgk)) < 1e-15


@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (7, 2), (5, 3)])
def test_streaming_by_brute_force(vel, nx, ny):
    """With S = 0 the step is pure streaming f_i(x + c_i) <- f_i(x) on the
    periodic lattice, compared with numpy.roll."""
    cx, cy = vel
    rng = np.random.default_rng(nx * 10 + ny)
    f = rng.standard_normal((9, ny, nx))
    g = f.copy()
    for t in range(1, 4):
        g = np.stack([np.roll(g[i], (cy[i], cx[i]), axis=(0, 1)) for i in range(9)])
        assert np.array_equal(orc.run(f, np.zeros(9), t), g)


def test_translation_invariance():
    s = inp.s_paper(inp.rates("LL", nu=1e-3))
    f = inp.random_populations(9, 6, 11, amp=1e-2)
    a = orc.run(np.roll(f, (2, 3), axis=(1, 2)), s, 7)
    b = np.roll(orc.run(f, s, 7), (2, 3), axis=(1, 2))
    assert np.array_equal(a, b)


def test_scaling_commutes_with_step():
    """m^eq is homogeneous of degree 1 in (rho, j), so stepping 2f gives
    exactly 2 step(f) (powers of two scale without rounding)."""
    s = inp.s_paper(inp.rates("OPT"))
    f = inp.random_populations(8, 5, 12, amp=1e-2)
    assert np.array_equal(orc.run(2.0 * f, s, 5), 2.0 * orc.run(f, s, 5))


def test_vn_reference_state_is_oracle_equilibrium():
    for U, V in [(0.0, 0.0), (0.1, 0.0), (0.05, 0.02)]:
        a = vn.equilibrium(1.0, U, V)
        b = orc.init_eq(np.ones((1, 1)), np.full((1, 1), U), np.full((1, 1), V))[:, 0, 0]
        assert np.max(np.abs(a - b)) < 1e-15


# ------------------------------------------------------- von Neumann pins
def sig(r, key):
    return 1.0 / r[key] - 0.5


@pytest.mark.parametrize("name", ["LL", "OPT", "LL*"])
def test_vn_small_k_limits(name):
    """As k -> 0 the eigenvalues of G(k) reproduce the L-NSE modes of
    section 4.1 with nu = sigma_nu/3 and bulk eta = sigma_e/3 (the delta-t
    matrix of section 2.3): acoustic phase speed c_s, acoustic damping
    k^2 (sigma_e + sigma_nu)/6, shear damping k^2 sigma_nu/3."""
    r = inp.rates(name, nu=1e-3)
    s = inp.s_paper(r)
    se, sn = sig(r, "s_e"), sig(r, "s_nu")
    for k in (0.02, 0.04):
        for theta in (0.0, math.pi / 6, math.pi / 4):
            lam = vn.eigs(k * math.cos(theta), k * math.sin(theta), 0.0, 0.0, s)
            damp, c = vn.mode_rates(lam, k)
            ac = np.argsort(-np.abs(lam))[:3]  # the three hydrodynamic modes
            speeds = np.sort(c[ac])
            assert abs(speeds[2] - vn.CS) < 5 * k * k
            assert abs(speeds[0] + vn.CS) < 5 * k * k
            assert abs(speeds[1]) < 1e-6
            i_sh = ac[np.argmin(np.abs(c[ac]))]
            i_ac = ac[np.argmax(c[ac])]
            gam_ac = k * k * (se + sn) / 6
            gam_sh = k * k * sn / 3
            assert abs(damp[i_ac] - gam_ac) < 0.05 * gam_ac + 2 * k ** 4
            assert abs(damp[i_sh] - gam_sh) < 0.05 * gam_sh + 2 * k ** 4


@pytest.mark.parametrize("U", [0.1, -0.05])
def test_vn_mean_flow_convection(U):
    """With a uniform flow the acoustic speeds are c_s +- U (the delta-t^0
    matrix of the uniform-flow case, section 2.3)."""
    s = inp.s_paper(inp.rates("OPT"))
    k = 0.02
    lam = vn.acoustic_modes(k, 0.0, U, 0.0, s)
    _, c = vn.mode_rates(lam, k)
    assert abs(c[0] - (U + vn.CS)) < 1e-3
    assert abs(c[1] - (U - vn.CS)) < 1e-3


def test_vn_unstable_band_claim():
    """Section 4.2 (Fig. 4-2 discussion): at sigma_e = sigma_nu = 0.0025 one
    mode grows for 0.75 < k < 1.75 off the axes and none along them.  Read
    here as a statement on the original scheme (Lallemand-Luo s_eps, s_q),
    whose unstable band the optimized Table 1 group A rates remove."""
    t = inp.TABLE1["A"]
    opt = {k_: 1.0 / (t["sigma_" + k_[2:]] + 0.5) for k_ in ("s_e", "s_eps", "s_q", "s_nu")}
    orig = dict(opt, s_eps=inp.LL["s_eps"], s_q=inp.LL["s_q"])
    band = np.linspace(0.8, 1.7, 10)
    for th in (math.pi / 6, math.pi / 4, 2 * math.pi / 3, 3 * math.pi / 4):
        g_orig = [np.max(np.abs(vn.eigs(k * math.cos(th), k * math.sin(th), 0, 0,
                                        inp.s_paper(orig)))) for k in band]
        g_opt = [np.max(np.abs(vn.eigs(k * math.cos(th), k * math.sin(th), 0, 0,
                                       inp.s_paper(opt)))) for k in band]
        assert max(g_orig) > 1.005          # a growing mode inside the band
        assert g_orig[4] > 1.001            # k = 1.2, mid-band
        assert max(g_opt) < 1.0 + 1e-12
        # outside the band the original scheme is stable again
        for k in (0.4, 2.2):
            lam = vn.eigs(k * math.cos(th), k * math.sin(th), 0, 0, inp.s_paper(orig))
            assert np.max(np.abs(lam)) < 1.0 + 1e-12
    for th in (0.0, math.pi / 2):
        for k in np.linspace(0.05, 3.0, 40):
            for r in (opt, orig):
                lam = vn.eigs(k * math.cos(th), k * math.sin(th), 0, 0, inp.s_paper(r))
                assert np.max(np.abs(lam)) < 1.0 + 1e-9


def test_vn_mean_flow_claims():
    """Section 4.2 on Fig. 4-4 (U = V = 0.1, Table 2 group A against the
    original free rates, the same s_e and s_nu): the optimized scheme is the
    more stable one -- off the axes the original rates have a growing mode
    near k = 1.5 (k along the flow and across it) and the optimized rates
    none -- while along the axes (theta = 0, pi/2, pi) the two schemes'
    hydrodynamic modes (the three least damped) nearly coincide."""
    t = inp.TABLE2["A"]
    opt = {k_: 1.0 / (t["sigma_" + k_[2:]] + 0.5) for k_ in ("s_e", "s_eps", "s_q", "s_nu")}
    orig = dict(opt, s_eps=inp.LL["s_eps"], s_q=inp.LL["s_q"])
    U = V = 0.1
    ks = np.linspace(0.02, math.pi, 160)

    def growth(r, th):
        return max(np.max(np.abs(vn.eigs(k * math.cos(th), k * math.sin(th), U, V,
                                          inp.s_paper(r)))) for k in ks)

    for th in (math.pi / 4, 3 * math.pi / 4):
        assert growth(orig, th) > 1.005
        assert growth(opt, th) < 1.0 + 1e-12
    for th in (0.0, math.pi / 2, math.pi):
        assert growth(orig, th) < 1.0 + 1e-12 and growth(opt, th) < 1.0 + 1e-12

    def hydro(r, th, k):
        lam = vn.eigs(k * math.cos(th), k * math.sin(th), U, V, inp.s_paper(r))
        top = lam[np.argsort(-np.abs(lam))[:3]]
        return np.sort(np.abs(top)), np.sort(np.angle(top))

    for th, near in ((0.0, True), (math.pi / 2, True), (math.pi, True), (math.pi / 4, False),
                     (3 * math.pi / 4, False)):
        dmag = dphase = 0.0
        for k in np.linspace(0.1, 1.0, 10):
            (ma, pa), (mb, pb) = hydro(opt, th, k), hydro(orig, th, k)
            dmag = max(dmag, np.max(np.abs(ma - mb)))
            dphase = max(dphase, np.max(np.abs(pa - pb)))
        if near:
            assert dmag < 1e-4 and dphase < 1e-5, (th, dmag, dphase)
        else:
            assert dmag > 1e-3, (th, dmag)


def test_vn_shear_mode_claim_at_very_small_bulk_viscosity():
    """Section 4.2 on Fig. 4-6 (U = 0.1, V = 0, Table 3 group B: sigma_e =
    2.5e-6, sigma_nu = 1e-5): the optimized scheme's shear mode damps at the
    exact rate sigma_nu k^2 / 3 within 10% for k <= 1, the original free
    rates miss it by more than half off the axes (the mode taken as the
    eigenvalue nearest the exact exp(-i k.U - sigma_nu k^2 / 3))."""
    t = inp.TABLE3["B"]
    opt = {k_: 1.0 / (t["sigma_" + k_[2:]] + 0.5) for k_ in ("s_e", "s_eps", "s_q", "s_nu")}
    orig = dict(opt, s_eps=inp.LL["s_eps"], s_q=inp.LL["s_q"])
    U, V, snu = 0.1, 0.0, t["sigma_nu"]

    def shear_error(r, th):
        worst = 0.0
        for k in np.linspace(0.1, 1.0, 10):
            lam = vn.eigs(k * math.cos(th), k * math.sin(th), U, V, inp.s_paper(r))
            exact = np.exp(-1j * k * (U * math.cos(th) + V * math.sin(th)) - snu * k * k / 3)
            got = lam[np.argmin(np.abs(lam - exact))]
            worst = max(worst, abs(-math.log(abs(got)) - snu * k * k / 3) / (snu * k * k / 3))
        return worst

    for th in (0.0, math.pi / 4, math.pi / 3, math.pi / 2):
        assert shear_error(opt, th) < 0.1, th
    for th in (0.0, math.pi / 4, math.pi / 3):
        assert shear_error(orig, th) > 0.5, th


@pytest.mark.parametrize("group", ["A", "B"])
def test_vn_acoustic_damping_claim_at_small_viscosities(group):
    """Section 4.2 on Fig. 4-7 and the conclusion: at very small shear and
    bulk viscosities (Table 3, U = 0.1, V = 0) the optimized acoustic modes
    damp at the exact rate k^2 (sigma_e + sigma_nu) / 6 within 10% for
    k <= 0.6 in every direction, while off the axes the original free rates'
    acoustic modes miss it by more than 100% (modes taken as the eigenvalues
    nearest the exact exp(-i k (U cos(theta) +- c_s) - Gamma))."""
    t = inp.TABLE3[group]
    opt = {k_: 1.0 / (t["sigma_" + k_[2:]] + 0.5) for k_ in ("s_e", "s_eps", "s_q", "s_nu")}
    orig = dict(opt, s_eps=inp.LL["s_eps"], s_q=inp.LL["s_q"])
    U, V = 0.1, 0.0

    def acoustic_error(r, th):
        worst = 0.0
        for k in np.linspace(0.1, 0.6, 6):
            gamma = k * k * (t["sigma_e"] + t["sigma_nu"]) / 6
            lam = vn.eigs(k * math.cos(th), k * math.sin(th), U, V, inp.s_paper(r))
            for sgn in (1.0, -1.0):
                exact = np.exp(-1j * k * (U * math.cos(th) + V * math.sin(th) + sgn * vn.CS) - gamma)
                got = lam[np.argmin(np.abs(lam - exact))]
                worst = max(worst, abs(-math.log(abs(got)) - gamma) / gamma)
        return worst

    for th in (0.0, math.pi / 4, math.pi / 3, math.pi / 2):
        assert acoustic_error(opt, th) < 0.1, th
    for th in (math.pi / 4, math.pi / 3):
        assert acoustic_error(orig, th) > 1.0, th


def test_vn_small_bulk_viscosity_claims():
    """Section 4.2 on Table 3 (sigma_e, sigma_nu ~ 1e-3 .. 1e-6): the
    original free rates (Lallemand-Luo s_eps, s_q) grow for almost every
    wave direction, and grow faster as the bulk viscosity shrinks (group B
    against group A); the optimized rates are stable without a mean flow.
    (With the mean flow U = V = 0.1 of the paper's figures the optimized
    sets keep a weakly growing mode at k ~ 2 near the axes, max |lambda|
    1.008 for group A, far below the original rates' 1.04.)"""
    ks = np.linspace(0.05, math.pi, 48)
    ths = np.linspace(0.0, 2 * math.pi, 36, endpoint=False)
    K, T = np.meshgrid(ks, ths)

    def rates(t, original):
        d = {k_: 1.0 / (t["sigma_" + k_[2:]] + 0.5) for k_ in ("s_e", "s_eps", "s_q", "s_nu")}
        if original:
            d.update(s_eps=inp.LL["s_eps"], s_q=inp.LL["s_q"])
        return inp.s_paper(d)

    def growth(t, original, U, V):
        lam = vn.eigs(K * np.cos(T), K * np.sin(T), U, V, rates(t, original))
        return np.max(np.abs(lam), axis=-1)  # (direction, k)

    for U, V in ((0.0, 0.0), (0.1, 0.0), (0.1, 0.1)):
        gA = growth(inp.TABLE3["A"], True, U, V)
        gB = growth(inp.TABLE3["B"], True, U, V)
        assert np.mean(gA.max(axis=1) > 1.0 + 1e-9) > 0.85  # all but the axes
        assert gB.max() > gA.max() > 1.009
        oA = growth(inp.TABLE3["A"], False, U, V)
        assert oA.max() < 1.0 + 0.25 * (gA.max() - 1.0)
    for g in ("A", "B"):
        assert growth(inp.TABLE3[g], False, 0.0, 0.0).max() < 1.0 + 1e-12


@pytest.mark.parametrize("U,name", [(0.0, "LL"), (0.1, "OPT"), (0.0, "OPT-Z")])
def test_step_matches_linear_propagation(U, name):
    """At amplitude 1e-7 the nonlinear oracle equals the exact linear
    evolution (every Fourier mode times G(k)^T built from the printed Psi)
    up to O(amplitude^2): pins the oracle's streaming and collision against
    section 2.3's Psi and section 4.1's amplification matrix."""
    nx, ny, T = 24, 16, 40
    r = inp.rates(name, nu=1e-3)
    s = inp.s_paper(r)
    rng = np.random.default_rng(5)
    base = orc.init_eq(np.ones((ny, nx)), np.full((ny, nx), U), np.zeros((ny, nx)))
    fp = 1e-7 * rng.standard_normal((9, ny, nx)) * base
    got = orc.run(base + fp, s, T) - base
    want = vn.propagate_linear(fp, T, U, 0.0, s)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-6


def test_plane_wave_eigenmode_rate():
    """A small-amplitude acoustic eigenmode of G(k) put on the lattice by the
    oracle decays and turns by exactly lambda per step."""
    nx, ny, m, T = 32, 4, 3, 25
    s = inp.s_paper(inp.rates("LL", nu=2e-3))
    k = 2 * math.pi * m / nx
    G = vn.amplification(k, 0.0, 0.0, 0.0, s)
    lam, vec = np.linalg.eig(G)
    j = np.argmax(np.abs(lam) - 10 * (np.abs(vn.mode_rates(lam, k)[1] - vn.CS) > 0.1))
    x = np.arange(nx)
    mode = vec[:, j][:, None, None] * np.exp(1j * k * x)[None, None, :] * np.ones((1, ny, 1))
    base = orc.init_eq(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    A = 1e-8
    f = base + A * np.real(mode)
    g = orc.run(f, s, T) - base
    want = A * np.real(lam[j] ** T * mode)
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-6


# ----------------------------------------------------------- pulse pins
def test_pulse_integral_at_t0_is_gaussian():
    """Eq. exactpules at t = 0: the Hankel transform of the Gaussian returns
    the initial pulse eps exp(-alpha eta^2)."""
    from oracle import pulse
    eta = np.linspace(0, 30, 61)
    eps, b = 1e-3, 4.0
    got = pulse.bessel(eta, 0.0, eps, b)
    want = eps * np.exp(-pulse.alpha_of(b) * eta ** 2)
    assert np.max(np.abs(got - want)) < 1e-12 * eps * 1e3


def test_pulse_periodic_equals_free_space_before_images_arrive():
    from oracle import pulse
    n, eps, b, t = 256, 1e-3, 4.0, 40.0
    rho = pulse.periodic(n, n, 128.0, 128.0, t, eps, b)
    x = np.arange(100, 160)
    eta = np.abs(x - 128.0)
    want = pulse.bessel(eta, t, eps, b)
    assert np.max(np.abs(rho[128, 100:160] - want)) < 1e-9 * eps * 1e3
    # a ring: the wave front sits near c_s t
    r_peak = eta[np.argmax(want)]
    assert abs(r_peak - vn.CS * t) < 3 * b


def test_pulse_mass_is_conserved():
    from oracle import pulse
    eps, b = 1e-3, 4.0
    for t in (0.0, 17.0, 200.0):
        rho = pulse.periodic(64, 64, 32.0, 32.0, t, eps, b)
        assert abs(rho.sum() - math.pi * eps / pulse.alpha_of(b)) < 1e-12


def test_oracle_pulse_follows_linear_acoustics():
    """The oracle's Gaussian pulse against the continuum solution with
    viscous damping k^2 (sigma_e + sigma_nu)/6: the two differ only by the
    scheme's dispersion error, which is small for a well-resolved pulse."""
    from oracle import pulse
    n, eps, b, T = 96, 1e-6, 6.0, 60
    r = inp.rates("LL", nu=1e-3)
    s = inp.s_paper(r)
    rho, ux, uy = inp.gaussian_pulse(n, n, eps, b, 48.0, 48.0)
    f = orc.run(orc.init_eq(rho, ux, uy), s, T)
    got = orc.moments(f)[0] - 1.0
    se, sn = sig(r, "s_e"), sig(r, "s_nu")
    want = pulse.periodic(n, n, 48.0, 48.0, T, eps, b,
                          gamma=lambda k: k * k * (se + sn) / 6)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 0.03
    # without the damping the continuum model is clearly worse
    free = pulse.periodic(n, n, 48.0, 48.0, T, eps, b)
    assert np.linalg.norm(got - free) / np.linalg.norm(free) > err


@pytest.mark.parametrize("name", ["BGK", "LL", "OPT-Z"])
def test_point_source_radiates_at_cs_times_period(name):
    """The harmonic point source of section 5.1 (density rho0 + rho_s
    sin(2 pi t / T) forced at one node, u = 0) radiates at the sound speed:
    the dominant wavenumber of the far field along the source row is
    2 pi / (c_s T)."""
    n, T, rs, steps = 161, 20.0, 0.01, 120
    if name == "BGK":
        sv = 1.0 / (0.5 + 3e-3)
        r = dict(s_e=sv, s_eps=sv, s_q=sv, s_nu=sv)
    else:
        r = inp.rates(name, nu=1e-3)
    f = orc.init_eq(np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
    f = orc.run_source(f, inp.s_paper(r), steps, (80, 80, rs, T))
    rho = orc.moments(f)[0] - 1.0
    x = np.arange(100, 145)  # 20 .. 64 nodes from the source, inside the front
    line = rho[80, 100:145]
    ks = np.linspace(0.3, 0.8, 501)
    power = [abs(np.sum((line - line.mean()) * np.exp(-1j * k * x))) for k in ks]
    k_fit = ks[int(np.argmax(power))]
    assert abs(k_fit / (2 * math.pi / (vn.CS * T)) - 1) < 0.02


# ----------------------------------------------------- printed parameters
@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "paper_tables.json")) as fh:
        return json.load(fh)


def source_field_metrics(rho, c=50):
    """Isotropy and spurious-fluctuation measures of a point-source field
    rho' (101 x 101, source at (c, c)): the largest difference between the
    profile along the diagonal and the axis profile at the same radius
    (radius >= 5), and the energy fraction at |k| > 0.8 pi, both relative."""
    ax_r = np.arange(0, 46)
    ax = rho[c, c:c + 46]
    diag_r = np.arange(0, 33) * math.sqrt(2)
    diag = np.array([rho[c + d, c + d] for d in range(33)])
    sel = diag_r >= 5
    aniso = np.max(np.abs(diag[sel] - np.interp(diag_r, ax_r, ax)[sel])) / np.max(np.abs(rho))
    F = np.fft.fft2(rho)
    k = np.fft.fftfreq(rho.shape[0]) * 2 * math.pi
    K = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    high = np.sum(np.abs(F[K > 0.8 * math.pi]) ** 2) / np.sum(np.abs(F) ** 2)
    return aniso, high


def point_source_schemes():
    t4 = inp.TABLE4["A"]
    return {"BGK": dict(s_e=t4["s_nu"], s_eps=t4["s_nu"], s_q=t4["s_nu"], s_nu=t4["s_nu"]),
            "original": dict(s_e=t4["s_e"], s_eps=inp.LL["s_eps"], s_q=inp.LL["s_q"],
                             s_nu=t4["s_nu"]),
            "optimized": inp.rates("OPT-Z")}


def test_point_source_isotropy_claim():
    """Section 5.1: on the 101 x 101 point-source problem (rho_s = 0.01,
    T = 20, t = 80) the optimized rates (Table 4 group A) correct the
    anisotropy of the radiated wave and remove the spurious fluctuations
    that BGK and the original MRT rates (same s_e = s_nu) show."""
    n = 101
    got = {}
    for name, r in point_source_schemes().items():
        f0 = orc.init_eq(np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
        f = orc.run_source(f0, inp.s_paper(r), 80, (50, 50, 0.01, 20.0))
        got[name] = source_field_metrics(orc.moments(f)[0] - 1.0)
    aniso, high = got["optimized"]
    others = [got["BGK"], got["original"]]
    assert aniso < 0.05 and aniso < 0.25 * min(o[0] for o in others)
    assert high < 1e-3 and high < 0.1 * min(o[1] for o in others)


@pytest.mark.parametrize("U0", [0.0, 0.1])
def test_pulse_claim_original_rates_damp_the_crests(U0):
    """Section 5.2: the original MRT-LBM (Lallemand-Luo free rates with its
    s_e = 1.64, i.e. bulk viscosity 0.11, at the same small shear viscosity)
    damps the crests and troughs of the pulse; the optimized rates (Table 5
    group A) keep them and reach a smaller E_L2.  The [0,1]^2 pulse on
    128^2 nodes (b = 0.04 N, t = 0.4 N), in the linear regime (eps = 1e-4),
    against the inviscid solution summed over periodic images."""
    from oracle import pulse

    N = 128
    b, T = 0.04 * N, int(round(0.4 * N))
    fields = inp.gaussian_pulse(N, N, 1e-4, b, N / 2, N / 2, u0=(U0, 0.0))
    exact = pulse.periodic(N, N, N / 2, N / 2, T, 1e-4, b, U0=U0)
    opt = inp.rates("OPT")
    original = dict(s_e=1.64, s_eps=inp.LL["s_eps"], s_q=inp.LL["s_q"], s_nu=opt["s_nu"])
    res = {}
    for name, r in (("optimized", opt), ("original", original)):
        rho = orc.moments(orc.run(orc.init_eq(*fields), inp.s_paper(r), T))[0] - 1.0
        row, ex = rho[N // 2], exact[N // 2]
        res[name] = (np.linalg.norm(rho - exact) / np.linalg.norm(exact),
                     np.max(row) / np.max(ex), np.min(row) / np.min(ex))
    e_opt, crest_opt, trough_opt = res["optimized"]
    e_org, crest_org, trough_org = res["original"]
    assert e_opt < 0.5 * e_org
    assert crest_org < 0.95 and trough_org < 0.98          # damped
    assert abs(crest_opt - 1.0) < 0.02 and abs(trough_opt - 1.0) < 0.04


def test_input_tables_match_the_paper(golden):
    for tab, mine in (("table1", inp.TABLE1), ("table2", inp.TABLE2),
                      ("table3", inp.TABLE3), ("table4", inp.TABLE4),
                      ("table5", inp.TABLE5)):
        for grp, vals in mine.items():
            for key, v in vals.items():
                assert golden[tab][grp][key] == v, (tab, grp, key)
    assert golden["lallemand_luo"]["s_e"] == inp.LL["s_e"]
    assert golden["lallemand_luo"]["s_eps"] == inp.LL["s_eps"]
    assert golden["lallemand_luo"]["s_q"] == inp.LL["s_q"]


def test_table3_and_table5_agree_through_sigma(golden):
    """sigma = 1/s - 1/2 (section 2.3) maps Table 5 onto Table 3."""
    for grp in ("A", "B"):
        t3, t5 = golden["table3"][grp], golden["table5"][grp]
        for key in ("e", "nu", "eps", "q"):
            s_from_sigma = 1.0 / (t3["sigma_" + key] + 0.5)
            assert abs(s_from_sigma - t5["s_" + key]) < 2e-9


def test_table4_viscosity_column(golden):
    """Table 4's nu equals sigma_nu / 3 = (1/s_nu - 1/2)/3 to printed digits."""
    for grp in ("A", "B"):
        t = golden["table4"][grp]
        nu = (1.0 / t["s_nu"] - 0.5) / 3.0
        assert abs(nu - t["nu"]) / t["nu"] < 2e-5


def test_sound_speed(golden):
    assert abs(vn.CS - golden["sound_speed"]["cs"]) < 5e-6


def test_ll_order_is_the_c_abi_vector():
    """The Lallemand-Luo vector s = (0, 1.64, 1.54, 0, 1.9, 0, 1.9, 1/tau,
    1/tau), tau = 1/2 + 3 nu, is the ABI's order; the paper's order puts
    s_e at index 3 (section 2.3)."""
    r = inp.rates("LL", nu=1e-3)
    tau = 0.5 + 3e-3
    assert np.allclose(inp.s_ll(r), [0, 1.64, 1.54, 0, 1.9, 0, 1.9, 1 / tau, 1 / tau],
                       rtol=0, atol=1e-15)
    sp = inp.s_paper(r)
    assert sp[3] == 1.64 and sp[4] == 1.54 and sp[5] == sp[6] == 1.9
    assert sp[7] == sp[8] == 1 / tau and not sp[:3].any()


# ------------------------------------------------------- moments and windows
@pytest.mark.parametrize("seed", range(3))
def test_moments_velocity_round_trip(seed):
    """oracle.moments returns u = j / rho: the textbook equilibrium carries
    exactly the density rho and momentum rho u it was built from (its zeroth
    and first velocity moments, section 2.3), and init_eq is pinned to that
    equilibrium above, so moments(init_eq(rho, u)) must give back (rho, u)
    to rounding.  A u taken as j (no division), swapped components or a
    sign error fail it: rho differs from 1 by up to 20% here."""
    rng = np.random.default_rng(100 + seed)
    ny, nx = 7, 11
    rho = rng.uniform(0.8, 1.2, (ny, nx))
    ux = rng.uniform(-0.2, 0.2, (ny, nx))
    uy = rng.uniform(-0.2, 0.2, (ny, nx))
    r, u, v = orc.moments(orc.init_eq(rho, ux, uy))
    assert np.max(np.abs(r - rho)) <= 1e-15
    assert np.max(np.abs(u - ux)) <= 1e-15
    assert np.max(np.abs(v - uy)) <= 1e-15


@pytest.mark.parametrize("T", [5, 40])
def test_window_run_equals_whole_lattice(T):
    """oracle.window_run (the light-cone sampler behind the full-size parity
    tests) against the plain whole-lattice run: after T steps a node depends
    only on the initial field within T nodes, so the window's centre must
    equal the whole lattice's node bit for bit -- at the wrap corners, in the
    interior, and on a lattice narrower than the window along y (there the
    whole periodic extent is kept)."""
    s = inp.s_paper(inp.rates("OPT"))
    for nx, ny in ((2 * T + 41, 2 * T + 17), (2 * T + 29, 2 * T - 1)):
        rho, ux, uy = inp.pulse_with_vortices(nx, ny, seed=T + nx, amp=1e-3, b=4.0,
                                              vstd=1e-3)
        whole = orc.run(orc.init_eq(rho, ux, uy), s, T)
        for x, y in ((0, 0), (nx - 1, ny - 1), (1, ny - 2), (nx - 2, 0), (nx // 2, ny // 3)):
            got = orc.window_run(rho, ux, uy, s, T, x, y)
            assert np.array_equal(got, whole[:, y, x]), (nx, ny, x, y)


def test_llstar_mean_flow_has_growing_mode():
    """Config 2's sets along the x axis of the 512 x 16 lattice (k_y = 0, the
    modes a y-independent plane wave can seed): the von Neumann matrix of
    section 4.1 is stable for LL, OPT (U = 0) and LL* at U = 0, while LL*
    (optimized s_e, s_nu with the original s_eps, s_q) at U = 0.1 has a
    growing mode near k_x = 3 pi / 4 -- the original free rates' mean-flow
    instability that section 4.2 describes for off-axis waves -- which grows
    about sevenfold over the 2000 steps of config 2."""
    kx = 2 * np.pi * np.fft.fftfreq(512)
    for name, U in (("LL", 0.0), ("LL", 0.1), ("OPT", 0.0), ("LL*", 0.0)):
        lam = vn.eigs(kx, 0 * kx, U, 0.0, inp.s_paper(inp.rates(name, nu=1e-3)))
        assert np.max(np.abs(lam)) < 1.0 + 1e-12, (name, U)
    lam = np.abs(vn.eigs(kx, 0 * kx, 0.1, 0.0, inp.s_paper(inp.rates("LL*", nu=1e-3))))
    g = lam.max(axis=1)
    j = int(np.argmax(g))
    assert 1.0009 < g[j] < 1.0011
    assert abs(abs(kx[j]) - 3 * np.pi / 4) < 0.05
    assert 6.0 < g[j] ** 2000 < 8.5


# ------------------------------------------- the extended-precision build
def test_extended_oracle_is_the_same_scheme():
    """oracle.run_ext is lbm_oracle.c built with long double arithmetic.  It
    must be the same scheme: on config 1 it agrees with the FP64 build to the
    FP64 build's own rounding (6e-12 relative L2 of rho' after 200 steps,
    the populations of size ~0.4 rounded every step against a 1e-3
    fluctuation), it is not bit-identical to it (the wider type is in
    effect), and at amplitude 1e-7 it follows the exact linear evolution of
    section 4.1 as the FP64 build does."""
    r = inp.rates("LL", nu=1e-3)
    s = inp.s_paper(r)
    f0 = orc.init_eq(*inp.gaussian_pulse(64, 64, 1e-3, 4.0))
    fe = orc.run_ext(f0, s, 200)
    fd = orc.run(f0, s, 200)
    re, rd = fe.sum(axis=0) - 1.0, fd.sum(axis=0) - 1.0
    rel = np.linalg.norm(rd - re) / np.linalg.norm(re)
    assert 1e-13 < rel < 2e-11
    nx, ny, T = 24, 16, 40
    s = inp.s_paper(inp.rates("OPT"))
    rng = np.random.default_rng(5)
    base = orc.init_eq(np.ones((ny, nx)), np.full((ny, nx), 0.1), np.zeros((ny, nx)))
    fp = 1e-7 * rng.standard_normal((9, ny, nx)) * base
    got = orc.run_ext(base + fp, s, T) - base
    want = vn.propagate_linear(fp, T, 0.1, 0.0, s)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-6
