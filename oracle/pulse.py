"""Linear-acoustics solution of the Gaussian pressure pulse (section 5.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Initial state rho = rho0 + eps exp(-alpha eta^2), u = (U0, 0), with
alpha = ln 2 / b^2 and eta the distance to the pulse centre.  Section 5.2
gives the inviscid solution as a Hankel integral (Eq. exactpules):

    rho = rho0 + eps/(2 alpha) int_0^inf exp(-xi^2/(4 alpha)) cos(c_s xi t)
                                     J0(xi eta) xi dxi,

with eta = |x - U0 t e_x - x_c| (the paper prints eta without its square
root; the radial coordinate it names is the reading taken here).

``bessel`` evaluates that integral by composite Gauss-Legendre quadrature.
``periodic`` gives the same solution on a periodic nx x ny lattice: by the
2D Fourier/Hankel identity the integral is the inverse Fourier transform of
(pi eps/alpha) exp(-|k|^2/(4 alpha)) cos(c_s |k| t), and summing it over the
periodic images (Poisson summation) leaves the Fourier series over the
lattice wavevectors, evaluated exactly at the nodes by an inverse FFT as long
as the Gaussian spectrum is negligible beyond the Nyquist wavenumber.  An
optional per-mode damping exp(-Gamma(|k|) t) models viscosity.
"""
import numpy as np
from scipy.special import j0

CS = 1.0 / np.sqrt(3.0)


def alpha_of(b):
    return np.log(2.0) / (b * b)


def bessel(eta, t, eps, b, cs=CS, panels=400, order=32):
    """Eq. exactpules minus rho0, at distances eta (any shape) and time t."""
    a = alpha_of(b)
    xmax = np.sqrt(4.0 * a * 45.0)  # exp(-xi^2/(4a)) < 3e-20 beyond
    xg, wg = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(0.0, xmax, panels + 1)
    mid = 0.5 * (edges[1:] + edges[:-1])
    half = 0.5 * (edges[1:] - edges[:-1])
    xi = (mid[:, None] + half[:, None] * xg[None, :]).ravel()
    w = (half[:, None] * wg[None, :]).ravel()
    kern = w * np.exp(-xi * xi / (4.0 * a)) * np.cos(cs * xi * t) * xi
    eta = np.asarray(eta, dtype=np.float64)
    flat = eta.ravel()
    out = np.empty_like(flat)
    step = max(1, 2_000_000 // xi.size)
    for s in range(0, flat.size, step):
        e = flat[s:s + step]
        out[s:s + step] = j0(e[:, None] * xi[None, :]) @ kern
    return (eps / (2.0 * a)) * out.reshape(eta.shape)


def periodic(nx, ny, xc, yc, t, eps, b, U0=0.0, cs=CS, gamma=None):
    """Density perturbation at the nodes of a periodic nx x ny lattice at time
    t for a pulse centred at (xc, yc) at t = 0.  gamma(k) -> damping per unit
    time of the acoustic mode at wavenumber k (None: inviscid)."""
    a = alpha_of(b)
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    k = np.sqrt(kx * kx + ky * ky)
    amp = (np.pi * eps / a) * np.exp(-k * k / (4.0 * a)) * np.cos(cs * k * t)
    if gamma is not None:
        amp = amp * np.exp(-gamma(k) * t)
    shift = np.exp(-1j * (kx * (xc + U0 * t) + ky * yc))
    return np.real(np.fft.ifft2(amp * shift))


def nyquist_leak(b):
    """Relative size of the Gaussian spectrum at the Nyquist wavenumber."""
    a = alpha_of(b)
    kn = np.pi
    return float(np.exp(-kn * kn / (4.0 * a)))
