"""CPU oracle of the D2Q9 MRT lattice Boltzmann step (FP64).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py, never by the product path.  It shares no code
with the CUDA library.

* the step, init and moments run in plain C (lbm_oracle.c, Eq. blbs of
  section 2.1 with the MRT collision of section 2.1 and the D2Q9 equilibrium
  moments of section 2.3);
* ``oracle.vn`` builds the von Neumann amplification matrix of section 4.1
  from the printed Psi of section 2.3;
* ``oracle.pulse`` evaluates the Gaussian-pulse solution of section 5.2;
* ``oracle.modified`` runs the recursive algorithm of section 2.2 (the
  modified equations of the linearized scheme) and the cost functions and
  parameter minimization of sections 3.2 and 4.2.

Relaxation rates are given here in the paper's moment order
(rho, jx, jy, e, eps, qx, qy, pxx, pxy); ``s_paper`` builds that vector.
"""
import ctypes
import os

import numpy as np

from . import build as _build

Q = 9
_lib = None


def load():
    """Build (if needed) and load liboracle.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_long]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_init_eq.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        lib.orc_moments.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        lib.orc_collide.argtypes = [dp, dp]
        lib.orc_meq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_matrices.argtypes = [dp, dp]
        lib.orc_velocities.argtypes = [ctypes.POINTER(ctypes.c_int)] * 2
        lib.orc_run_source.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_long,
                                       ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.orc_run_source.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_get_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def s_paper(s_e, s_eps, s_q, s_nu):
    """S = diag(0,0,0,s_e,s_eps,s_q,s_q,s_nu,s_nu) (section 2.3)."""
    return np.array([0.0, 0.0, 0.0, s_e, s_eps, s_q, s_q, s_nu, s_nu])


def set_threads(n):
    load().orc_set_threads(int(n))


def threads():
    return load().orc_get_threads()


def velocities():
    cx = (ctypes.c_int * Q)()
    cy = (ctypes.c_int * Q)()
    load().orc_velocities(cx, cy)
    return np.array(list(cx)), np.array(list(cy))


def matrices():
    """(M, M^-1) as used by the oracle's collision."""
    M = np.zeros(Q * Q)
    Mi = np.zeros(Q * Q)
    load().orc_matrices(_p(M), _p(Mi))
    return M.reshape(Q, Q), Mi.reshape(Q, Q)


def meq(rho, jx, jy):
    out = np.zeros(Q)
    load().orc_meq(float(rho), float(jx), float(jy), _p(out))
    return out


def collide(s, f):
    """One collision at one node; returns the post-collision populations."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    g = np.array(f, dtype=np.float64)
    load().orc_collide(_p(s), _p(g))
    return g


def init_eq(rho, ux, uy):
    """f = f^eq(rho, u) on a lattice; inputs (ny, nx), output (9, ny, nx)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ux = np.ascontiguousarray(ux, dtype=np.float64)
    uy = np.ascontiguousarray(uy, dtype=np.float64)
    ny, nx = rho.shape
    f = np.zeros((Q, ny, nx))
    load().orc_init_eq(nx, ny, _p(rho), _p(ux), _p(uy), _p(f))
    return f


def run(f, s, nsteps):
    """Advance populations f (9, ny, nx) by nsteps; returns a new array."""
    f = np.array(f, dtype=np.float64, order="C")
    s = np.ascontiguousarray(s, dtype=np.float64)
    _, ny, nx = f.shape
    rc = load().orc_run(nx, ny, _p(s), _p(f), int(nsteps))
    if rc != 0:
        raise RuntimeError("orc_run failed (%d)" % rc)
    return f


def run_source(f, s, nsteps, source, t0=0, rho0=1.0):
    """orc_run with the point source of section 5.1: source = (x, y,
    amplitude, period); the node is reset to f^eq(rho0 + amplitude
    sin(2 pi t / period), 0) before each step's collision."""
    f = np.array(f, dtype=np.float64, order="C")
    s = np.ascontiguousarray(s, dtype=np.float64)
    _, ny, nx = f.shape
    x, y, amp, period = source
    rc = load().orc_run_source(nx, ny, _p(s), _p(f), int(nsteps), int(t0), int(x), int(y),
                               float(rho0), float(amp), float(period))
    if rc != 0:
        raise RuntimeError("orc_run_source failed (%d)" % rc)
    return f


_lib_ext = None


def run_ext(f, s, nsteps):
    """As run, with the collision and streaming in extended precision (the
    same C source built with long double arithmetic; FP64 in and out).  The
    reference for GPU paths whose FP64 rounding differs from the plain
    oracle's."""
    global _lib_ext
    if _lib_ext is None:
        lib = ctypes.CDLL(_build.build(ext=True))
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_long]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib_ext = lib
    _lib_ext.orc_set_threads(threads())
    f = np.array(f, dtype=np.float64, order="C")
    s = np.ascontiguousarray(s, dtype=np.float64)
    _, ny, nx = f.shape
    rc = _lib_ext.orc_run(nx, ny, _p(s), _p(f), int(nsteps))
    if rc != 0:
        raise RuntimeError("orc_run (extended) failed (%d)" % rc)
    return f


def moments(f):
    """(rho, ux, uy) of populations f (9, ny, nx)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, ny, nx = f.shape
    rho = np.zeros((ny, nx))
    ux = np.zeros((ny, nx))
    uy = np.zeros((ny, nx))
    load().orc_moments(nx, ny, _p(f), _p(rho), _p(ux), _p(uy))
    return rho, ux, uy


def window_run(rho, ux, uy, s, nsteps, x, y):
    """Populations at time nsteps of node (x, y) of a large periodic lattice.

    A node after T steps depends only on the initial field within distance
    T (one node per step), so the plain periodic oracle is run on the
    (2T+3)-wide window around (x, y) cut out of the initial macroscopic
    fields; wrong data entering from the window's own wrap cannot reach the
    centre.  Along a dimension no longer than the window the whole periodic
    extent is kept (its wrap is then the true one).  Returns the 9
    populations of the node.
    """
    ny, nx = rho.shape
    h = int(nsteps) + 1
    if 2 * h + 1 < ny:
        ys, cy = np.arange(y - h, y + h + 1) % ny, h
    else:
        ys, cy = np.arange(ny), y
    if 2 * h + 1 < nx:
        xs, cx = np.arange(x - h, x + h + 1) % nx, h
    else:
        xs, cx = np.arange(nx), x
    sel = (ys[:, None], xs[None, :])
    f = init_eq(rho[sel], ux[sel], uy[sel])
    f = run(f, s, nsteps)
    return f[:, cy, cx].copy()
