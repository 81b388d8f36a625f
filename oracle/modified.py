"""Modified-equation analysis of the linearized MRT scheme and the cost
functions of the free-parameter optimization (sections 2.2, 3 and 4.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

In wave-number space the linearized scheme advances the moments by
m(t + dt) = sum_n dt^n A_n m with A_n = (1/n!) M (-i v.k)^n M^-1 Psi (Psi the
printed relaxation-with-equilibrium matrix of section 2.3).  The recursive
algorithm of section 2.2 turns this into an equation for the conserved
quantities W = (rho, jx, jy) alone,

    dW/dt = B_n W + O(dt^n),      B_n = sum_{l=0}^{n-1} dt^l k^(l+1) b^l(theta),

through two recursions, one for the map m = Phi_n W of all moments
(Eqs. R-A, R-B) and one for B_n (Eqs. R-D, R-E), each truncated at
dt^(n-1).  This module runs both recursions numerically, with dt kept as a
formal variable (every matrix is a polynomial in dt stored as its
coefficient array) and |k| = 1, so the coefficient of dt^l is b^l itself.
Matrix powers B^l are taken in the polynomial ring and truncated, as the
recursions prescribe.

Section 3 compares B_n with the exact linearized Navier-Stokes matrix B:
M_eps = B_n - B (Eq. perturbation), or B_n - B + Bbulk when the bulk
viscosity is separated (section 3.2.3), and minimizes integrals of the
squared Frobenius norm of M_eps over the wave number dt k in [0, pi] and its
direction theta in [0, 2 pi) -- and, for mean flows, the flow direction in
[0, 2 pi) and speed in [0, u0].  With dt = 1 and K = dt k,

    M_eps(K) = sum_l K^(l+1) E^l,   E^l = b^l - b_exact^l,

where b_exact^0 is the exact convection (the scheme reproduces it: E^0 = 0)
and b_exact^1 the exact dissipation; the K integral is done in closed form,
sum_{l,m} Re<E^l, E^m>_F pi^(l+m+3) / (l+m+3), the direction integrals by the
trapezoid rule (exact for these trigonometric polynomials) and the speed
integral by Gauss-Legendre quadrature.  The odd (dispersion) and even
(dissipation) parts of M_eps are its terms of odd and even powers of K.
"""
import math

import numpy as np

from .vn import CX, CY, moment_matrix

Q = 9


def sigma_to_s(sig):
    """s = 1 / (sigma + 1/2), the inverse of sigma = 1/s - 1/2 (section 2.3)."""
    return 1.0 / (np.asarray(sig, dtype=np.float64) + 0.5)


def s_paper_from_sigmas(sigma_e, sigma_eps, sigma_q, sigma_nu):
    """Rates in the paper's order (rho, jx, jy, e, eps, qx, qy, pxx, pxy);
    the conserved slots are unused (zero)."""
    se, seps, sq, snu = (float(sigma_to_s(x)) for x in (sigma_e, sigma_eps, sigma_q, sigma_nu))
    return np.array([0.0, 0.0, 0.0, se, seps, sq, sq, snu, snu])


def psi_batch(U, V, s):
    """The printed Psi of section 2.3 for arrays U, V (same shape) ->
    (..., 9, 9)."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    se, seps, sq, snu = s[3], s[4], s[5], s[7]
    P = np.zeros(U.shape + (Q, Q))
    P[..., range(Q), range(Q)] = 1.0
    u2 = U * U + V * V
    P[..., 3, 0] = -2 * se - 3 * u2 * se
    P[..., 3, 1] = 6 * U * se
    P[..., 3, 2] = 6 * V * se
    P[..., 3, 3] = 1 - se
    P[..., 4, 0] = seps + 3 * u2 * seps
    P[..., 4, 1] = -6 * U * seps
    P[..., 4, 2] = -6 * V * seps
    P[..., 4, 4] = 1 - seps
    P[..., 5, 1] = -sq
    P[..., 5, 5] = 1 - sq
    P[..., 6, 2] = -sq
    P[..., 6, 6] = 1 - sq
    P[..., 7, 0] = -(U * U - V * V) * snu
    P[..., 7, 1] = 2 * U * snu
    P[..., 7, 2] = -2 * V * snu
    P[..., 7, 7] = 1 - snu
    P[..., 8, 0] = -U * V * snu
    P[..., 8, 1] = V * snu
    P[..., 8, 2] = U * snu
    P[..., 8, 8] = 1 - snu
    return P


def _pmul(X, Y, maxdeg):
    """Product of two polynomial matrices (coefficient axis -3), truncated
    at degree maxdeg."""
    dx, dy = X.shape[-3], Y.shape[-3]
    out = np.zeros(X.shape[:-3] + (maxdeg + 1, X.shape[-2], Y.shape[-1]), dtype=complex)
    for i in range(min(dx, maxdeg + 1)):
        for j in range(min(dy, maxdeg + 1 - i)):
            out[..., i + j, :, :] += X[..., i, :, :] @ Y[..., j, :, :]
    return out


def _ppow(X, p, maxdeg):
    """X^p for a square polynomial matrix, truncated at degree maxdeg."""
    R = X[..., : maxdeg + 1, :, :].copy() if X.shape[-3] > maxdeg + 1 else X.copy()
    for _ in range(p - 1):
        R = _pmul(R, X, maxdeg)
    return R


def _embed(X, lo, out):
    """out += X shifted up by lo degrees (dt^lo X), within out's degrees."""
    n = min(X.shape[-3], out.shape[-3] - lo)
    if n > 0:
        out[..., lo : lo + n, :, :] += X[..., :n, :, :]


def bn_coeffs(theta, U, V, s, n):
    """b^l(theta), l = 0..n-1: the dt^l coefficients of B_n at |k| = 1 for
    wave direction theta and mean flow (U, V) (arrays of one shape P), rates
    s in the paper's order.  Returns (P..., n, 3, 3) complex."""
    theta = np.asarray(theta, dtype=np.float64)
    shape = np.broadcast(theta, np.asarray(U), np.asarray(V)).shape
    theta = np.broadcast_to(theta, shape)
    U = np.broadcast_to(np.asarray(U, dtype=np.float64), shape)
    V = np.broadcast_to(np.asarray(V, dtype=np.float64), shape)
    M = moment_matrix()
    Minv = np.linalg.inv(M)
    Ps = psi_batch(U, V, s)  # (..., 9, 9)
    vk = np.cos(theta)[..., None] * CX + np.sin(theta)[..., None] * CY  # v_j . k, |k| = 1
    MinvPsi = Minv @ Ps
    # A_l = (1/l!) M diag((-i v.k)^l) M^-1 Psi, l = 1..n (polynomials of degree 0)
    A = [None]
    for l in range(1, n + 1):
        d = (-1j * vk) ** l / math.factorial(l)
        A.append((M @ (d[..., :, None] * MinvPsi))[..., None, :, :])
    si = np.asarray(s, dtype=np.float64)[3:]  # rates of the non-conserved rows
    Psi_c = Ps[..., :, 0:3].astype(complex)

    def finish_phi(acc):
        acc[..., :, 0:3, :] = 0.0
        acc[..., 0, 0:3, :] = np.eye(3)
        acc[..., :, 3:, :] /= si[:, None]
        return acc

    # first order: m = Phi_1 W, B_1 = A_1 Phi_1 (conserved rows)
    phi = {1: finish_phi(Psi_c[..., None, :, :].copy())}
    B = {1: _pmul(A[1][..., 0:3, :], phi[1], 0)}
    for m in range(2, n + 1):
        deg = m - 1
        acc = np.zeros(shape + (m, Q, 3), dtype=complex)
        acc[..., 0, :, :] = Psi_c
        for l in range(1, m):
            Bp = _ppow(B[m - l], l, deg - l)
            _embed(-_pmul(phi[m - l], Bp, deg - l) / math.factorial(l), l, acc)
            _embed(_pmul(A[l], phi[m - l], deg - l), l, acc)
        phi[m] = finish_phi(acc)
        Bacc = np.zeros(shape + (m, 3, 3), dtype=complex)
        for l in range(1, m):
            _embed(-_ppow(B[m - l], l + 1, deg - l) / math.factorial(l + 1), l, Bacc)
        for l in range(1, m + 1):
            _embed(_pmul(A[l][..., 0:3, :], phi[m + 1 - l], deg - (l - 1)), l - 1, Bacc)
        B[m] = Bacc
    return B[n]


# The reference matrix B that M_eps is measured against (readings, each
# pinned by the cost values the paper prints in Tables 1-3):
#   'ns'      convection + the exact dissipation (zero mean flow, section
#             3.2.1: M_eps starts at (dt k)^3);
#   'euler'   convection only (section 3.2.2, Table 2: every dissipation term
#             of B_n, the physical one included, counts as error);
#   'ns-bulk' convection + the shear part of the exact dissipation, i.e.
#             B - Bbulk (section 3.2.3, Table 3).
REFERENCES = ("ns", "euler", "ns-bulk")


def exact_coeffs(theta, U, V, sigma_e, sigma_nu, reference="ns"):
    """b_exact^0 (linearized convection about the mean flow) and b_exact^1
    (dissipation: the exact linearized one of section 3.2.3, independent of
    the mean flow, for 'ns'; its shear part for 'ns-bulk'; none for
    'euler') at |k| = 1.  Returns (..., 2, 3, 3) complex."""
    if reference not in REFERENCES:
        raise ValueError(reference)
    theta = np.asarray(theta, dtype=np.float64)
    shape = np.broadcast(theta, np.asarray(U), np.asarray(V)).shape
    kx = np.broadcast_to(np.cos(theta), shape)
    ky = np.broadcast_to(np.sin(theta), shape)
    U = np.broadcast_to(np.asarray(U, dtype=np.float64), shape)
    V = np.broadcast_to(np.asarray(V, dtype=np.float64), shape)
    out = np.zeros(shape + (2, 3, 3), dtype=complex)
    c = out[..., 0, :, :]
    c[..., 0, 1] = -1j * kx
    c[..., 0, 2] = -1j * ky
    c[..., 1, 0] = 1j * (-kx / 3 + kx * U * U + ky * U * V)
    c[..., 1, 1] = 1j * (-2 * kx * U - ky * V)
    c[..., 1, 2] = 1j * (-ky * U)
    c[..., 2, 0] = 1j * (-ky / 3 + ky * V * V + kx * U * V)
    c[..., 2, 1] = 1j * (-kx * V)
    c[..., 2, 2] = 1j * (-2 * ky * V - kx * U)
    if reference == "euler":
        return out
    d = out[..., 1, :, :]
    se = 0.0 if reference == "ns-bulk" else sigma_e
    d[..., 1, 1] = -(kx * kx * se + (kx * kx + ky * ky) * sigma_nu) / 3
    d[..., 1, 2] = -kx * ky * se / 3
    d[..., 2, 1] = -kx * ky * se / 3
    d[..., 2, 2] = -(ky * ky * se + (kx * kx + ky * ky) * sigma_nu) / 3
    return out


def _k_integral(E, parity):
    """int_0^pi || sum_l K^(l+1) E^l ||_F^2 dK over the terms whose power
    l+1 has the given parity ('odd', 'even' or 'all')."""
    n = E.shape[-3]
    keep = [l for l in range(n) if parity == "all" or ((l + 1) % 2 == 1) == (parity == "odd")]
    tot = 0.0
    for l in keep:
        for m in keep:
            g = np.real(np.sum(np.conj(E[..., l, :, :]) * E[..., m, :, :], axis=(-2, -1)))
            p = l + m + 3
            tot = tot + g * math.pi ** p / p
    return tot


# Quadrature sizes that integrate the trigonometric / polynomial integrands
# exactly for truncation orders n <= 5 (tested against larger grids).
N_THETA, N_DIR, N_SPEED = 16, 24, 9


def cost(sigmas, n, kind="F", parity="all", u0=0.2, reference=None, n_theta=N_THETA,
         n_dir=N_DIR, n_speed=N_SPEED, fixed_speed=False):
    """The cost functions of section 3.2.

    sigmas = (sigma_e, sigma_eps, sigma_q, sigma_nu); n = truncation order.
    kind 'F' (zero mean flow): F^o (parity 'odd'), F^e ('even'), calligraphic
    F ('all'), Eqs. Minimization-A/B/C.  kind 'G' (mean flows): G^o, G^e,
    calligraphic G, Eqs. approximation-D/E, Minimization-F, integrated over
    the flow direction in [0, 2 pi) and the speed in [0, u0] (u0 = 0.2, the
    paper's stated upper bound; or at the fixed speed u0 when fixed_speed).
    reference: see REFERENCES ('ns' for F, 'euler' for G by default)."""
    if reference is None:
        reference = "ns" if kind == "F" else "euler"
    sigma_e, sigma_eps, sigma_q, sigma_nu = (float(x) for x in sigmas)
    s = s_paper_from_sigmas(sigma_e, sigma_eps, sigma_q, sigma_nu)
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    if kind == "F":
        b = bn_coeffs(th, 0.0, 0.0, s, n)
        ex = exact_coeffs(th, 0.0, 0.0, sigma_e, sigma_nu, reference)
        E = b.copy()
        E[..., :2, :, :] -= ex
        return float(np.mean(_k_integral(E, parity)) * 2 * np.pi)
    if kind != "G":
        raise ValueError(kind)
    ph = 2 * np.pi * np.arange(n_dir) / n_dir
    if fixed_speed:
        um = np.array([u0])
        wu = np.array([1.0])
    else:
        x, w = np.polynomial.legendre.leggauss(n_speed)
        um = 0.5 * u0 * (x + 1.0)
        wu = 0.5 * u0 * w
    TH, PH, UM = np.meshgrid(th, ph, um, indexing="ij")
    U = UM * np.cos(PH)
    V = UM * np.sin(PH)
    b = bn_coeffs(TH, U, V, s, n)
    ex = exact_coeffs(TH, U, V, sigma_e, sigma_nu, reference)
    E = b.copy()
    E[..., :2, :, :] -= ex
    vals = _k_integral(E, parity)  # (n_theta, n_dir, n_speed)
    per_speed = vals.mean(axis=(0, 1)) * (2 * np.pi) ** 2
    return float(np.sum(per_speed * wu))


FREE = ("sigma_e", "sigma_eps", "sigma_q", "sigma_nu")


def minimize(fixed, free, start, n, kind="F", parity="all", reference=None, u0=0.2):
    """Minimize a section 3.2 cost over the free sigmas (each >= 0, i.e.
    s in (0, 2]) with the others fixed: fixed maps names of FREE to values,
    free lists the names varied, start their initial values.  A library
    library method does the search: scipy's bounded Nelder-Mead on the
    sigmas scaled by their starting values, restarted from its result until
    the cost stops improving.  Returns (dict of all four sigmas, cost)."""
    from scipy.optimize import minimize as sp_minimize

    scale = np.maximum(np.abs(np.asarray(start, dtype=np.float64)), 1e-6)

    def full(x):
        d = dict(fixed)
        d.update(zip(free, x * scale))
        return tuple(d[k] for k in FREE)

    def f(x):
        return cost(full(x), n, kind, parity, u0, reference)

    x = np.ones(len(free))
    best = f(x)
    for _ in range(8):
        r = sp_minimize(f, x, method="Nelder-Mead", bounds=[(0.0, None)] * len(free),
                        options=dict(xatol=1e-11, fatol=1e-15, maxiter=4000))
        x = r.x
        if best - r.fun <= 1e-14 * abs(best):
            best = min(best, float(r.fun))
            break
        best = float(r.fun)
    return dict(zip(FREE, full(x))), best
