"""Seeded synthetic inputs for the D2Q9 MRT lattice Boltzmann workloads.

Shared by the tests, the benchmark and the oracle checks.  This module holds
none of the lattice Boltzmann arithmetic: only relaxation-rate sets copied
from the paper's tables, initial macroscopic fields (rho, u), random
populations, and the recipes of the batched and served workloads.  Every
generator takes an explicit seed and returns float64 numpy arrays.

Relaxation-rate vectors come in two orders:
  * Lallemand-Luo order (rho, e, eps, jx, qx, jy, qy, pxx, pxy): the order of
    the C ABI's S[9] argument and of the Lallemand-Luo vector
    s = (0, 1.64, 1.54, 0, 1.9, 0, 1.9, 1/tau, 1/tau);
  * the paper's order (rho, jx, jy, e, eps, qx, qy, pxx, pxy) of section 2.3,
    which the oracle takes.
"""
import math

import numpy as np

CS = 1.0 / math.sqrt(3.0)  # D2Q9 sound speed (section 5.1)

# ---------------------------------------------------------------- rate sets
# Lallemand-Luo values of the free rates (section 2.3); s_nu is free.
LL = dict(s_e=1.64, s_eps=1.54, s_q=1.9)

# Table 4 (section 5.1): optimized rates for zero mean flow, point source.
TABLE4 = {
    "A": dict(s_e=1.99044751, s_nu=1.99044751, s_eps=2.0, s_q=0.00875438872,
              nu=0.000799861),
    "B": dict(s_e=1.95321, s_nu=1.95321, s_eps=2.0, s_q=0.04126919093,
              nu=0.00399257),
}

# Table 5 (section 5.2): optimized rates for uniform flows (bulk-separated).
TABLE5 = {
    "A": dict(s_e=1.99, s_nu=1.999960001, s_eps=1.962820428, s_q=1.992761413),
    "B": dict(s_e=1.99999, s_nu=1.999960001, s_eps=1.999875273, s_q=1.999969578),
}

# Tables 1-3 (section 4.2) as printed, in sigma = 1/s - 1/2 form.
TABLE1 = {
    "A": dict(sigma_e=0.0025, sigma_nu=0.0025, sigma_eps=0.0, sigma_q=105.468091254867),
    "B": dict(sigma_e=0.0025, sigma_nu=0.0025, sigma_eps=0.0, sigma_q=105.465307838135),
    "C": dict(sigma_e=0.1, sigma_nu=0.1, sigma_eps=0.0, sigma_q=26.3631592758091),
    "D": dict(sigma_e=0.1, sigma_nu=0.1, sigma_eps=0.0, sigma_q=26.3520430827600),
}
# Reading: groups C and D print sigma_e = sigma_nu = 0.1, but their sigma_q
# and cost values are those of sigma_e = sigma_nu = 0.01 (the cost F^o at
# the printed optimum is 17.9107478 with 0.01 and 2.2e5 with 0.1, and
# minimizing with 0.01 reproduces the printed sigma_q to 1e-7); read as 0.01.
TABLE1_READ = {g: (dict(t, sigma_e=0.01, sigma_nu=0.01) if g in "CD" else dict(t))
               for g, t in TABLE1.items()}
TABLE2 = {
    "A": dict(sigma_e=0.001, sigma_nu=0.001, sigma_eps=0.00751873323089156,
              sigma_q=0.00171909400064198),
    "B": dict(sigma_e=0.0025, sigma_nu=0.0025, sigma_eps=0.0187982349323006,
              sigma_q=0.00429903714246050),
}
TABLE3 = {
    "A": dict(sigma_e=0.0025125628, sigma_nu=0.00001, sigma_eps=0.00947095595580122,
              sigma_q=0.00181622011980382),
    "B": dict(sigma_e=0.0000025, sigma_nu=0.00001, sigma_eps=0.0000311837523990053,
              sigma_q=0.00000760552251906507),
}


def s_from_nu(nu):
    """Shear rate for lattice viscosity nu: tau = 1/2 + 3 nu, s = 1/tau."""
    return 1.0 / (0.5 + 3.0 * nu)


def rates(name, nu=None):
    """Named set -> dict(s_e, s_eps, s_q, s_nu).

    'LL'    Lallemand-Luo free rates with s_nu = s_from_nu(nu)
    'OPT'   Table 5 group A (the default optimized set); 'OPT-B' its group B
    'OPT-Z' Table 4 group A; 'OPT-Z-B' its group B
    'LL*'   Table 5 group A's s_e and s_nu with the Lallemand-Luo s_eps, s_q
    """
    if name == "LL":
        if nu is None:
            raise ValueError("LL needs nu")
        return dict(LL, s_nu=s_from_nu(nu))
    if name in ("OPT", "OPT-B"):
        t = TABLE5["A" if name == "OPT" else "B"]
        return dict(s_e=t["s_e"], s_eps=t["s_eps"], s_q=t["s_q"], s_nu=t["s_nu"])
    if name in ("OPT-Z", "OPT-Z-B"):
        t = TABLE4["A" if name == "OPT-Z" else "B"]
        return dict(s_e=t["s_e"], s_eps=t["s_eps"], s_q=t["s_q"], s_nu=t["s_nu"])
    if name == "LL*":
        t = TABLE5["A"]
        return dict(s_e=t["s_e"], s_eps=LL["s_eps"], s_q=LL["s_q"], s_nu=t["s_nu"])
    raise KeyError(name)


def s_ll(r):
    """Rate dict -> 9-vector in Lallemand-Luo order (the C ABI's S[9])."""
    return np.array([0.0, r["s_e"], r["s_eps"], 0.0, r["s_q"], 0.0, r["s_q"],
                     r["s_nu"], r["s_nu"]])


def s_paper(r):
    """Rate dict -> 9-vector in the paper's order (the oracle's S)."""
    return np.array([0.0, 0.0, 0.0, r["s_e"], r["s_eps"], r["s_q"], r["s_q"],
                     r["s_nu"], r["s_nu"]])


# ------------------------------------------------------------ field recipes
def _min_image(d, n):
    return (d + 0.5 * n) % n - 0.5 * n


def gaussian_pulse(nx, ny, amp, b, xc=None, yc=None, rho0=1.0, u0=(0.0, 0.0)):
    """rho = rho0 + amp exp(-alpha eta^2), alpha = ln2/b^2, u = u0 (section 5.2).
    eta is the minimum-image distance to (xc, yc) on the periodic lattice."""
    xc = nx / 2.0 if xc is None else xc
    yc = ny / 2.0 if yc is None else yc
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    dx = _min_image(x - xc, nx)
    dy = _min_image(y - yc, ny)
    alpha = math.log(2.0) / (b * b)
    rho = rho0 + amp * np.exp(-alpha * (dx * dx + dy * dy))
    ux = np.full((ny, nx), float(u0[0]))
    uy = np.full((ny, nx), float(u0[1]))
    return rho, ux, uy


def plane_wave(nx, ny, amp, m, U=0.0, rho0=1.0):
    """Right-running acoustic wave along x with m wavelengths in the period:
    rho = rho0 + amp cos(k x), u = U + c_s amp cos(k x)/rho0, v = 0."""
    k = 2.0 * math.pi * m / nx
    c = np.cos(k * np.arange(nx, dtype=np.float64))[None, :] * np.ones((ny, 1))
    rho = rho0 + amp * c
    ux = U + CS * amp * c / rho0
    uy = np.zeros((ny, nx))
    return rho, ux, uy


def wavelength_modes(nx, wavelengths=(4, 6, 8, 12, 16, 32, 64)):
    """Commensurate mode numbers m = round(nx / lambda) for each wavelength."""
    return [int(round(nx / lam)) for lam in wavelengths]


def vortical(nx, ny, seed, nmodes=32, kmax=64, std=1e-4, period=None):
    """Divergence-free velocity u = (d psi/dy, -d psi/dx) of a seeded stream
    function psi = sum_n a_n cos(k_n.x + phi_n), k_n = 2 pi (p, q)/period with
    integers 1 <= |p|,|q| <= kmax, scaled to the given velocity std.
    The lattice side sets the period, so the field is exactly periodic."""
    rng = np.random.default_rng(seed)
    px = rng.integers(1, kmax + 1, nmodes) * rng.choice([-1, 1], nmodes)
    qy = rng.integers(1, kmax + 1, nmodes) * rng.choice([-1, 1], nmodes)
    a = rng.standard_normal(nmodes)
    phi = rng.uniform(0.0, 2 * math.pi, nmodes)
    Lx = nx if period is None else period[0]
    Ly = ny if period is None else period[1]
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    kx = 2 * math.pi * px / Lx
    ky = 2 * math.pi * qy / Ly
    ax = kx[:, None] * x[None, :] + phi[:, None]  # (nmodes, nx)
    by = ky[:, None] * y[None, :]                 # (nmodes, ny)
    # sin(kx x + ky y + phi) = sin(ax) cos(by) + cos(ax) sin(by): every
    # component is a sum of separable products, i.e. one matrix product
    Y = np.concatenate([np.cos(by), np.sin(by)]).T          # (ny, 2 nmodes)
    Sx = np.concatenate([np.sin(ax), np.cos(ax)])            # (2 nmodes, nx)
    wx = np.concatenate([-a * ky, -a * ky])[:, None]
    wy = np.concatenate([a * kx, a * kx])[:, None]
    ux = Y @ (wx * Sx)
    uy = Y @ (wy * Sx)
    # the rms of each mode is known in closed form: scale without a pass
    var = 0.5 * np.sum(a * a * ((2 * math.pi * qy / Ly) ** 2 + (2 * math.pi * px / Lx) ** 2))
    scale = std / math.sqrt(var / 2.0)
    return ux * scale, uy * scale


def pulse_with_vortices(nx, ny, seed, amp=1e-3, b=20.0, vstd=1e-4, rho0=1.0):
    """Large-lattice workload: centred Gaussian pulse plus seeded vortical
    velocity perturbation."""
    rho, _, _ = gaussian_pulse(nx, ny, amp, b, rho0=rho0)
    ux, uy = vortical(nx, ny, seed, std=vstd)
    return rho, ux, uy


def random_populations(nx, ny, seed, amp=1e-3, base=None):
    """Positive random populations about a rest-state base (9, ny, nx):
    f_i = base_i (1 + amp * N(0,1)).  Exercises every moment of the
    collision, unlike an equilibrium field."""
    rng = np.random.default_rng(seed)
    if base is None:
        base = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    noise = rng.standard_normal((9, ny, nx))
    return base[:, None, None] * (1.0 + amp * noise)


# --------------------------------------------------------- batch workload
def batch_specs(n=512, seed=1107 + 4, amin=32 * 32, amax=1024 * 1024, steps=500):
    """Independent periodic lattices: area log-uniform in [amin, amax], aspect
    ratio r log-uniform in [1/4, 4], nx = max(8, round(sqrt(A r))),
    ny = max(8, round(sqrt(A / r))); s_e ~ U[1.0, 1.99], nu log-uniform in
    [1e-4, 1e-2], (s_eps, s_q) from the optimized or the Lallemand-Luo set;
    Gaussian pulse (b = 4) at a random position, amplitude log-uniform in
    [1e-5, 1e-3]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        A = math.exp(rng.uniform(math.log(amin), math.log(amax)))
        r = math.exp(rng.uniform(math.log(0.25), math.log(4.0)))
        nx = max(8, int(round(math.sqrt(A * r))))
        ny = max(8, int(round(math.sqrt(A / r))))
        s_e = rng.uniform(1.0, 1.99)
        nu = math.exp(rng.uniform(math.log(1e-4), math.log(1e-2)))
        base = "OPT" if rng.random() < 0.5 else "LL"
        free = rates("OPT") if base == "OPT" else dict(LL)
        r_ = dict(s_e=s_e, s_eps=free["s_eps"], s_q=free["s_q"], s_nu=s_from_nu(nu))
        amp = math.exp(rng.uniform(math.log(1e-5), math.log(1e-3)))
        out.append(dict(nx=nx, ny=ny, rates=r_, set=base, nu=nu, amp=amp, b=4.0,
                        xc=float(rng.uniform(0, nx)), yc=float(rng.uniform(0, ny)),
                        steps=steps))
    return out


def batch_fields(spec):
    return gaussian_pulse(spec["nx"], spec["ny"], spec["amp"], spec["b"],
                          spec["xc"], spec["yc"])


# ------------------------------------------------------- serving workload
def request_stream(n=10000, rate=200.0, seed=1107 + 5, side=(64, 2048),
                   steps=(100, 5000)):
    """Poisson arrivals (mean `rate` per second) of MRT-LBM solve requests:
    square side log-uniform in `side`, steps uniform in `steps`, storage FP32
    or FP16 deviation (50/50), optimized or Lallemand-Luo rates (50/50,
    nu = 1e-3 for the latter), Gaussian (amplitude log-uniform in
    [1e-5, 1e-3], b = 4) or plane-wave initial field (50/50)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    out = []
    for i in range(n):
        side_ = int(round(math.exp(rng.uniform(math.log(side[0]), math.log(side[1])))))
        st = int(rng.integers(steps[0], steps[1] + 1))
        dtype = "f32" if rng.random() < 0.5 else "f16"
        set_ = "OPT" if rng.random() < 0.5 else "LL"
        r_ = rates("OPT") if set_ == "OPT" else rates("LL", nu=1e-3)
        amp = math.exp(rng.uniform(math.log(1e-5), math.log(1e-3)))
        if rng.random() < 0.5:
            init = dict(kind="gaussian", amp=amp, b=4.0,
                        xc=float(rng.uniform(0, side_)), yc=float(rng.uniform(0, side_)))
        else:
            init = dict(kind="plane", amp=amp, m=int(rng.integers(1, max(2, side_ // 8))))
        out.append(dict(id=i, arrival=float(t[i]), nx=side_, ny=side_, steps=st,
                        dtype=dtype, set=set_, rates=r_, init=init))
    return out


def request_fields(req):
    init = req["init"]
    if init["kind"] == "gaussian":
        return gaussian_pulse(req["nx"], req["ny"], init["amp"], init["b"],
                              init["xc"], init["yc"])
    return plane_wave(req["nx"], req["ny"], init["amp"], init["m"])
