"""Von Neumann analysis of the linearized D2Q9 MRT scheme (section 4.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The linearized scheme of section 2.2 (Eq. l-mrt-lbs) relaxes the moment
perturbations with the matrix Psi printed in section 2.3 for the reference
state rho = 1, mean flow (U, V).  A plane wave f' = A exp(i(k.x - omega t))
then obeys  exp(-i omega) f' = G(k) f'  with

    G(k) = diag(exp(-i k.c_j)) M^-1 Psi M,

which is the paper's M^mrt = A^-1 [I - M^-1 S M N^bgk] of section 4.1 written
through Psi (the garbled derivative in the definition of N^bgk is read as
the Jacobian of f^eq).  Eigenvalues lambda = exp(-i omega): per-step damping
-ln|lambda| and phase speed -arg(lambda)/|k|.

This module builds M itself from the Lallemand-Luo basis polynomials of the
velocities (not from the C oracle's table) and Psi from its printed entries,
so it is an independent check of the step oracle's linearization.
"""
import numpy as np

Q = 9
CS = 1.0 / np.sqrt(3.0)  # D2Q9 sound speed (section 5.1)

# velocity order (reading: the paper prints none)
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def moment_matrix():
    """Rows rho, jx, jy, e, eps, qx, qy, pxx, pxy as polynomials of c."""
    c2 = CX ** 2 + CY ** 2
    rows = [
        np.ones(Q),
        CX,
        CY,
        3 * c2 - 4,
        (9 * c2 ** 2 - 21 * c2 + 8) / 2,
        (3 * c2 - 5) * CX,
        (3 * c2 - 5) * CY,
        CX ** 2 - CY ** 2,
        CX * CY,
    ]
    return np.array(rows, dtype=np.float64)


def psi(U, V, s):
    """The printed Psi of section 2.3; s in paper order (s[3]=s_e, s[4]=s_eps,
    s[5]=s[6]=s_q, s[7]=s[8]=s_nu)."""
    se, seps, sq, snu = s[3], s[4], s[5], s[7]
    P = np.eye(Q)
    u2 = U * U + V * V
    P[3, :4] = [-2 * se - 3 * u2 * se, 6 * U * se, 6 * V * se, 1 - se]
    P[4, :5] = [seps + 3 * u2 * seps, -6 * U * seps, -6 * V * seps, 0, 1 - seps]
    P[5, :6] = [0, -sq, 0, 0, 0, 1 - sq]
    P[6, :7] = [0, 0, -sq, 0, 0, 0, 1 - sq]
    P[7, :8] = [-(U * U - V * V) * snu, 2 * U * snu, -2 * V * snu, 0, 0, 0, 0, 1 - snu]
    P[8, :9] = [-U * V * snu, V * snu, U * snu, 0, 0, 0, 0, 0, 1 - snu]
    return P


def amplification(kx, ky, U, V, s):
    """G(k) for one wavevector, or a stack for arrays kx, ky of equal shape."""
    M = moment_matrix()
    C = np.linalg.inv(M) @ psi(U, V, s) @ M
    kx = np.asarray(kx, dtype=np.float64)
    ky = np.asarray(ky, dtype=np.float64)
    phase = np.exp(-1j * (kx[..., None] * CX + ky[..., None] * CY))
    return phase[..., :, None] * C


def eigs(kx, ky, U, V, s):
    return np.linalg.eigvals(amplification(kx, ky, U, V, s))


def mode_rates(lam, k):
    """(damping per step, phase speed) of eigenvalue(s) lam at |k| = k."""
    lam = np.asarray(lam)
    return -np.log(np.abs(lam)), -np.angle(lam) / k


def acoustic_modes(k, theta, U, V, s):
    """The two acoustic eigenvalues at wavevector k (cos theta, sin theta):
    those whose phase speeds lie nearest +-c_s + u.khat."""
    kx, ky = k * np.cos(theta), k * np.sin(theta)
    lam = eigs(kx, ky, U, V, s)
    _, c = mode_rates(lam, k)
    ukh = U * np.cos(theta) + V * np.sin(theta)
    out = []
    for target in (ukh + CS, ukh - CS):
        out.append(lam[np.argmin(np.abs(c - target))])
    return np.array(out)


def equilibrium(rho, U, V):
    """Populations of the uniform reference state, via M^-1 m^eq (section 2.3)."""
    jx, jy = rho * U, rho * V
    j2 = jx * jx + jy * jy
    m = np.array([rho, jx, jy, -2 * rho + 3 * j2 / rho, rho - 3 * j2 / rho,
                  -jx, -jy, (jx * jx - jy * jy) / rho, jx * jy / rho])
    return np.linalg.solve(moment_matrix(), m)


def propagate_linear(fp, nsteps, U, V, s):
    """Exact evolution of a periodic perturbation fp (9, ny, nx) about the
    uniform state (rho=1, U, V) under the linearized scheme: each Fourier mode
    is multiplied by G(k)^nsteps."""
    _, ny, nx = fp.shape
    fh = np.fft.fft2(fp, axes=(1, 2))  # (9, ny, nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)[:, None] * np.ones((1, nx))
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, :] * np.ones((ny, 1))
    G = amplification(kx, ky, U, V, s)  # (ny, nx, 9, 9)
    Gt = np.linalg.matrix_power(G, int(nsteps))
    v = np.moveaxis(fh, 0, -1)[..., None]  # (ny, nx, 9, 1)
    out = (Gt @ v)[..., 0]
    return np.real(np.fft.ifft2(np.moveaxis(out, -1, 0), axes=(1, 2)))
