"""Python binding of liblbm.so (include/lbm.h), same names, marshalling only.

Every step of the lattice Boltzmann path runs in the CUDA library; this
module converts arguments (numpy arrays for host data, torch CUDA tensors or
raw integers for device pointers and streams) and turns error codes into
``LbmError``.  There is no fallback: if liblbm.so is missing the import
fails.
"""
import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

LBM_OK, LBM_PENDING = 0, 1
LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE = -1, -2, -3, -4
LBM_ETIMEOUT, LBM_ENOTFOUND, LBM_ECLOSED = -5, -6, -7
LBM_F64, LBM_F32DEV, LBM_F16DEV, LBM_BF16DEV, LBM_F64DEV = 0, 1, 2, 3, 4
LBM_INIT_FIELDS, LBM_INIT_GAUSSIAN, LBM_INIT_PLANE = 0, 1, 2
DTYPES = {"f64": LBM_F64, "f32": LBM_F32DEV, "f16": LBM_F16DEV, "bf16": LBM_BF16DEV,
          "f64dev": LBM_F64DEV}

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class lbm_info_t(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pitch", ctypes.c_int),
                ("dtype", ctypes.c_int), ("elem_bytes", ctypes.c_int), ("t", ctypes.c_long),
                ("qscale", ctypes.c_double), ("S_paper", ctypes.c_double * 9),
                ("device_bytes", ctypes.c_size_t)]


class lbm_request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("S", ctypes.c_double * 9),
                ("rho0", ctypes.c_double), ("u0", ctypes.c_double * 2),
                ("dtype", ctypes.c_int), ("steps", ctypes.c_long),
                ("init_kind", ctypes.c_int), ("init_params", ctypes.c_double * 8),
                ("rho", _dp), ("ux", _dp), ("uy", _dp)]


class lbm_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("admitted", ctypes.c_longlong),
                ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("generations", ctypes.c_longlong), ("resident", ctypes.c_int),
                ("peak_resident", ctypes.c_int), ("resident_bytes", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("lattice_updates", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("variant", ctypes.c_int)]


class lbm_cost_spec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("order", ctypes.c_int), ("part", ctypes.c_int),
                ("reference", ctypes.c_int), ("u0", ctypes.c_double),
                ("fixed_speed", ctypes.c_int)]


LBM_COST_F, LBM_COST_G = 0, 1
LBM_PART_ALL, LBM_PART_ODD, LBM_PART_EVEN = 0, 1, 2
LBM_REF_NS, LBM_REF_EULER, LBM_REF_NS_BULK = 0, 1, 2
SIGMA_NAMES = ("sigma_e", "sigma_eps", "sigma_q", "sigma_nu")


_SIGS = {
    "lbm_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp,
                                  ctypes.c_int, ctypes.POINTER(_vp)]),
    "lbm_init_field": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbm_init_field_dev": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_init_analytic": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
    "lbm_step": (ctypes.c_int, [_vp, ctypes.c_long]),
    "lbm_tune": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_int)]),
    "lbm_set_source": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double]),
    "lbm_batch_tune": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_int)]),
    "lbm_set_variant": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_batch_set_variant": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_batch_get_variant": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_resident": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_const_table": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "lbm_get_variant": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "lbm_opt_cost": (ctypes.c_int, [ctypes.POINTER(lbm_cost_spec), ctypes.c_int, _dp, _dp]),
    "lbm_opt_minimize": (ctypes.c_int, [ctypes.POINTER(lbm_cost_spec), _dp, ctypes.c_uint, _dp,
                                        _dp, _dp, _dp, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_size": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_batch_init_packed": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbm_batch_moments_packed": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbm_moments": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbm_moments_dev": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_destroy": (ctypes.c_int, [_vp]),
    "lbm_get_populations": (ctypes.c_int, [_vp, _dp]),
    "lbm_set_populations": (ctypes.c_int, [_vp, _dp]),
    "lbm_set_stream": (ctypes.c_int, [_vp, _vp]),
    "lbm_sync": (ctypes.c_int, [_vp]),
    "lbm_drift": (ctypes.c_int, [_vp, _dp]),
    "lbm_drift_pop_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, _dp, _vp]),
    "lbm_info": (ctypes.c_int, [_vp, ctypes.POINTER(lbm_info_t)]),
    "lbm_set_allocator": (ctypes.c_int, [_vp, _vp, _vp]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_host_alloc": (ctypes.c_void_p, [ctypes.c_size_t]),
    "lbm_host_free": (ctypes.c_int, [ctypes.c_void_p]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "lbm_vn_eigs": (ctypes.c_int, [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp,
                                   ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_step": (ctypes.c_int, [_vp, ctypes.c_long]),
    "lbm_batch_drift": (ctypes.c_int, [_vp, _dp]),
    "lbm_batch_init_fields": (ctypes.c_int, [_vp, ctypes.POINTER(_dp), ctypes.POINTER(_dp),
                                             ctypes.POINTER(_dp)]),
    "lbm_batch_moments": (ctypes.c_int, [_vp, ctypes.POINTER(_dp), ctypes.POINTER(_dp),
                                         ctypes.POINTER(_dp)]),
    "lbm_batch_destroy": (ctypes.c_int, [_vp]),
    "lbm_batch_solve_packed": (ctypes.c_int, [_vp, ctypes.c_long, _dp, _dp, _dp, _dp, _dp, _dp,
                                              _dp]),
    "lbm_slabs_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp,
                                        ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_vp)]),
    "lbm_slabs_rows": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    "lbm_slabs_init_field": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbm_slabs_set_populations": (ctypes.c_int, [_vp, _dp]),
    "lbm_slabs_step": (ctypes.c_int, [_vp, ctypes.c_long]),
    "lbm_slabs_moments": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbm_slabs_get_populations": (ctypes.c_int, [_vp, _dp]),
    "lbm_slabs_drift": (ctypes.c_int, [_vp, _dp]),
    "lbm_slabs_destroy": (ctypes.c_int, [_vp]),
    "lbm_slab_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       _dp, ctypes.c_double, _dp, ctypes.c_int,
                                       ctypes.POINTER(_vp)]),
    "lbm_slab_halo_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_slab_pack": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "lbm_slab_unpack": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "lbm_batch_wait": (ctypes.c_int, [_vp, _dp]),
    "lbm_debug_bounds": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint), ctypes.c_int]),
    "lbm_debug_bounds_selftest": (ctypes.c_int, []),
    "lbm_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_long, ctypes.POINTER(_vp)]),
    "lbm_submit": (ctypes.c_int, [_vp, ctypes.POINTER(lbm_request),
                                  ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_poll": (ctypes.c_int, [_vp, ctypes.c_longlong, _dp, _dp, _dp, _dp]),
    "lbm_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(lbm_server_stats_t)]),
    "lbm_server_set_policy": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_longlong]),
    "lbm_server_destroy": (ctypes.c_int, [_vp]),
    "lbm_server_done": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
}

_lib = None


def load(path=LIB_PATH):
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("liblbm.so not built: run paper_1107_4543_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class LbmError(RuntimeError):
    def __init__(self, code, where):
        lib = load()
        msg = "%s failed: %s (%d): %s" % (where, lib.lbm_strerror(code).decode(), code,
                                          lib.lbm_last_error().decode())
        super().__init__(msg)
        self.code = code


def _ck(rc, where):
    if rc != LBM_OK:
        raise LbmError(rc, where)
    return rc


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _dev(t):
    """Device pointer of a torch CUDA tensor (float64, contiguous) or an int."""
    if isinstance(t, int):
        return t
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def lbm_strerror(code):
    return load().lbm_strerror(int(code)).decode()


def lbm_last_error():
    return load().lbm_last_error().decode()


def lbm_host_alloc(nbytes):
    """Address of nbytes of page-locked huge-page host memory (raises on
    failure); release it with lbm_host_free."""
    p = load().lbm_host_alloc(int(nbytes))
    if not p:
        raise LbmError(LBM_ENOMEM, "lbm_host_alloc")
    return p


def lbm_host_free(p):
    _ck(load().lbm_host_free(ctypes.c_void_p(p)), "lbm_host_free")


def host_array(shape, dtype=np.float64):
    """A numpy array in page-locked huge-page host memory (lbm_host_alloc),
    released once the array and every view of it are gone."""
    dtype = np.dtype(dtype)
    count = int(np.prod(shape))
    nbytes = max(count * dtype.itemsize, 1)
    p = lbm_host_alloc(nbytes)
    buf = (ctypes.c_char * nbytes).from_address(p)
    weakref.finalize(buf, load().lbm_host_free, ctypes.c_void_p(p))
    return np.frombuffer(buf, dtype=dtype, count=count).reshape(shape)


def lbm_create(nx, ny, S, rho0=1.0, u0=(0.0, 0.0), dtype=LBM_F32DEV):
    """S: 9 rates in Lallemand-Luo order (rho, e, eps, jx, qx, jy, qy, pxx, pxy)."""
    lib = load()
    s = _f64(S, (9,))
    u = _f64(u0, (2,))
    h = _vp()
    _ck(lib.lbm_create(int(nx), int(ny), _ptr(s), float(rho0), _ptr(u),
                       DTYPES.get(dtype, dtype), ctypes.byref(h)), "lbm_create")
    return h


def lbm_destroy(h):
    _ck(load().lbm_destroy(h), "lbm_destroy")


def lbm_info(h):
    info = lbm_info_t()
    _ck(load().lbm_info(h, ctypes.byref(info)), "lbm_info")
    return dict(nx=info.nx, ny=info.ny, pitch=info.pitch, dtype=info.dtype,
                elem_bytes=info.elem_bytes, t=info.t, qscale=info.qscale,
                S_paper=list(info.S_paper), device_bytes=info.device_bytes)


def lbm_init_field(h, rho, ux, uy):
    i = lbm_info(h)
    shp = (i["ny"], i["nx"])
    r, u, v = _f64(rho, shp), _f64(ux, shp), _f64(uy, shp)
    _ck(load().lbm_init_field(h, _ptr(r), _ptr(u), _ptr(v)), "lbm_init_field")


def lbm_init_field_dev(h, rho, ux, uy):
    _ck(load().lbm_init_field_dev(h, _dev(rho), _dev(ux), _dev(uy)), "lbm_init_field_dev")


def lbm_init_analytic(h, kind, params):
    p = np.zeros(8)
    p[:len(params)] = params
    _ck(load().lbm_init_analytic(h, int(kind), _ptr(p)), "lbm_init_analytic")


def lbm_step(h, n):
    _ck(load().lbm_step(h, int(n)), "lbm_step")


def lbm_set_source(h, x, y, amplitude, period):
    _ck(load().lbm_set_source(h, int(x), int(y), float(amplitude), float(period)),
        "lbm_set_source")


LBM_TUNE_VARIANTS = 3


def lbm_tune(h):
    """(times_ms per launch variant, chosen variant)."""
    t = np.zeros(LBM_TUNE_VARIANTS)
    c = ctypes.c_int()
    _ck(load().lbm_tune(h, _ptr(t), ctypes.byref(c)), "lbm_tune")
    return t, c.value


LBM_BATCH_TUNE_VARIANTS = 6


def lbm_set_variant(h, variant):
    _ck(load().lbm_set_variant(h, int(variant)), "lbm_set_variant")


def lbm_batch_set_variant(b, variant):
    _ck(load().lbm_batch_set_variant(b, int(variant)), "lbm_batch_set_variant")


def lbm_get_variant(h):
    v = ctypes.c_int()
    _ck(load().lbm_get_variant(h, ctypes.byref(v)), "lbm_get_variant")
    return v.value


def lbm_batch_get_variant(b):
    v = ctypes.c_int()
    _ck(load().lbm_batch_get_variant(b, ctypes.byref(v)), "lbm_batch_get_variant")
    return v.value


def lbm_batch_resident(b):
    """Per member: whether the batch keeps it in shared memory for all the
    steps of a launch (bool array in member order)."""
    n = lbm_batch_size(b)[0]
    f = np.zeros(n, dtype=np.int32)
    _ck(load().lbm_batch_resident(b, f.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
        "lbm_batch_resident")
    return f.astype(bool)


def lbm_batch_const_table(b):
    """Per member: whether the batched step reads its collision constants
    from the constant-memory table (bool array in member order)."""
    n = lbm_batch_size(b)[0]
    f = np.zeros(n, dtype=np.int32)
    _ck(load().lbm_batch_const_table(b, f.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
        "lbm_batch_const_table")
    return f.astype(bool)


def lbm_batch_tune(b):
    t = np.zeros(LBM_BATCH_TUNE_VARIANTS)
    c = ctypes.c_int()
    _ck(load().lbm_batch_tune(b, _ptr(t), ctypes.byref(c)), "lbm_batch_tune")
    return t, c.value


def lbm_moments(h, out=None):
    """(rho, ux, uy) as (ny, nx) float64 arrays; `out` may supply them."""
    i = lbm_info(h)
    if out is None:
        out = tuple(np.empty((i["ny"], i["nx"])) for _ in range(3))
    for a in out:
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != i["nx"] * i["ny"]:
            raise ValueError("moment outputs must be contiguous float64 ny x nx")
    _ck(load().lbm_moments(h, _ptr(out[0]), _ptr(out[1]), _ptr(out[2])), "lbm_moments")
    return out


def lbm_moments_dev(h, rho, ux, uy):
    _ck(load().lbm_moments_dev(h, _dev(rho), _dev(ux), _dev(uy)), "lbm_moments_dev")


def lbm_get_populations(h):
    i = lbm_info(h)
    f = np.empty((9, i["ny"], i["nx"]))
    _ck(load().lbm_get_populations(h, _ptr(f)), "lbm_get_populations")
    return f


def lbm_set_populations(h, f):
    i = lbm_info(h)
    a = _f64(f, (9, i["ny"], i["nx"]))
    _ck(load().lbm_set_populations(h, _ptr(a)), "lbm_set_populations")


def lbm_set_stream(h, stream):
    """stream: an int cudaStream_t, a torch.cuda.Stream, or None."""
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    _ck(load().lbm_set_stream(h, stream), "lbm_set_stream")


def lbm_sync(h):
    _ck(load().lbm_sync(h), "lbm_sync")


def lbm_drift(h):
    """[sum rho', sum jx', sum jy', non-finite count]; a non-zero count is
    reported in the last entry (the C call returns LBM_EUNSTABLE)."""
    out = np.zeros(4)
    rc = load().lbm_drift(h, _ptr(out))
    if rc not in (LBM_OK, LBM_EUNSTABLE):
        raise LbmError(rc, "lbm_drift")
    return out


def lbm_drift_pop_noalloc(f_dev, nx, ny, rho0=1.0, j0=(0.0, 0.0), stream=None):
    """lbm_drift's sums over caller-owned FP64 populations (device pointer or
    contiguous CUDA tensor of 9 x ny x nx doubles), allocating nothing."""
    out = np.zeros(4)
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    rc = load().lbm_drift_pop_noalloc(_dev(f_dev), int(nx), int(ny), float(rho0), float(j0[0]),
                                      float(j0[1]), _ptr(out), stream)
    if rc not in (LBM_OK, LBM_EUNSTABLE):
        raise LbmError(rc, "lbm_drift_pop_noalloc")
    return out


def lbm_set_allocator(alloc_fn=None, free_fn=None, ctx=None):
    """alloc_fn / free_fn: ctypes function pointers or None (cudaMalloc)."""
    a = ctypes.cast(alloc_fn, _vp) if alloc_fn is not None else None
    f = ctypes.cast(free_fn, _vp) if free_fn is not None else None
    _ck(load().lbm_set_allocator(a, f, ctx), "lbm_set_allocator")


def lbm_vn_eigs(kx, ky, U, V, S):
    """Eigenvalues (n, 9) complex of G(k) for n cases; S is (n, 9) or (9,)
    in Lallemand-Luo order.  Raises if some QR iteration did not converge."""
    kx = _f64(np.atleast_1d(kx))
    n = kx.size
    ky, U, V = (_f64(np.broadcast_to(np.asarray(a, dtype=np.float64), (n,))) for a in (ky, U, V))
    S = _f64(np.broadcast_to(np.asarray(S, dtype=np.float64), (n, 9)))
    out = np.empty((n, 18))
    bad = ctypes.c_int()
    _ck(load().lbm_vn_eigs(n, _ptr(kx), _ptr(ky), _ptr(U), _ptr(V), _ptr(S), _ptr(out),
                           ctypes.byref(bad)), "lbm_vn_eigs")
    return out.view(np.complex128)  # (re, im) pairs: (n, 9) complex, no copy


def lbm_batch_create(handles):
    arr = (_vp * len(handles))(*[h.value if isinstance(h, _vp) else h for h in handles])
    b = _vp()
    _ck(load().lbm_batch_create(len(handles), arr, ctypes.byref(b)), "lbm_batch_create")
    return b


def lbm_batch_step(b, n):
    _ck(load().lbm_batch_step(b, int(n)), "lbm_batch_step")


def lbm_batch_drift(b, n):
    """(n, 4) array: lbm_drift's sums for each of the batch's n members."""
    out = np.zeros((n, 4))
    rc = load().lbm_batch_drift(b, _ptr(out))
    if rc not in (LBM_OK, LBM_EUNSTABLE):
        raise LbmError(rc, "lbm_batch_drift")
    return out


def _ptr_array(arrays):
    return (_dp * len(arrays))(*[_ptr(a) for a in arrays])


def lbm_batch_init_fields(b, fields):
    """fields: one (rho, ux, uy) triple of C-contiguous float64 (ny, nx)
    arrays per member, in member order."""
    for f in fields:
        for a in f:
            if a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("fields must be contiguous float64 arrays")
    _ck(load().lbm_batch_init_fields(b, _ptr_array([f[0] for f in fields]),
                                     _ptr_array([f[1] for f in fields]),
                                     _ptr_array([f[2] for f in fields])),
        "lbm_batch_init_fields")


def lbm_batch_moments(b, outs):
    """outs: one (rho, ux, uy) triple of writable contiguous float64 (ny, nx)
    arrays per member, filled in place."""
    for f in outs:
        for a in f:
            if a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("outputs must be contiguous float64 arrays")
    _ck(load().lbm_batch_moments(b, _ptr_array([f[0] for f in outs]),
                                 _ptr_array([f[1] for f in outs]),
                                 _ptr_array([f[2] for f in outs])), "lbm_batch_moments")
    return outs


def lbm_batch_size(b):
    """(members, total nodes) of the batch."""
    m, n = ctypes.c_int(), ctypes.c_longlong()
    _ck(load().lbm_batch_size(b, ctypes.byref(m), ctypes.byref(n)), "lbm_batch_size")
    return m.value, n.value


def _packed(b, arrays, what):
    n = lbm_batch_size(b)[1]
    for a in arrays:
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
            raise ValueError("%s must be contiguous float64 arrays of %d values" % (what, n))


def lbm_batch_init_packed(b, rho, ux, uy):
    """rho, ux, uy: contiguous float64 arrays of lbm_batch_size(b)[1] values,
    member k's (ny, nx) field at the sum of nx*ny of the members before it."""
    _packed(b, (rho, ux, uy), "fields")
    _ck(load().lbm_batch_init_packed(b, _ptr(rho), _ptr(ux), _ptr(uy)), "lbm_batch_init_packed")


def lbm_batch_moments_packed(b, out=None):
    """Every member's rho, ux, uy in packed arrays (filled in place if out is
    given)."""
    if out is None:
        n = lbm_batch_size(b)[1]
        out = tuple(np.empty(n) for _ in range(3))
    _packed(b, out, "outputs")
    _ck(load().lbm_batch_moments_packed(b, _ptr(out[0]), _ptr(out[1]), _ptr(out[2])),
        "lbm_batch_moments_packed")
    return out


def lbm_batch_solve_packed(b, n, fields_in, fields_out, drift_out=None):
    """Queue one whole solve of every member (upload, equilibrium init, n
    steps, drift sums, moments, download) without waiting; fields_in and
    fields_out are (rho, ux, uy) triples of packed contiguous float64 arrays
    (as lbm_batch_init_packed), drift_out an (members, 4) float64 array or
    None.  The arrays must stay alive and untouched until lbm_batch_wait."""
    _packed(b, fields_in, "fields")
    _packed(b, fields_out, "outputs")
    dp = None
    if drift_out is not None:
        m = lbm_batch_size(b)[0]
        if (drift_out.dtype != np.float64 or not drift_out.flags.c_contiguous
                or drift_out.size != 4 * m):
            raise ValueError("drift_out must be a contiguous float64 array of %d values" % (4 * m))
        dp = _ptr(drift_out)
    _ck(load().lbm_batch_solve_packed(b, int(n), _ptr(fields_in[0]), _ptr(fields_in[1]),
                                      _ptr(fields_in[2]), _ptr(fields_out[0]),
                                      _ptr(fields_out[1]), _ptr(fields_out[2]), dp),
        "lbm_batch_solve_packed")


# ------------------------------------------------------------- slabs
def lbm_slabs_create(nx, ny, S, rho0=1.0, u0=(0.0, 0.0), dtype=LBM_F32DEV, nslabs=2,
                     devices=None):
    """One nx x ny periodic lattice split into nslabs y-slabs (devices: one
    CUDA device index per slab, default the current device)."""
    Sa = _f64(S, (9,))
    u = _f64(u0, (2,))
    dev = None
    if devices is not None:
        if len(devices) != nslabs:
            raise ValueError("one device per slab")
        dev = (ctypes.c_int * nslabs)(*devices)
    s = _vp()
    _ck(load().lbm_slabs_create(int(nx), int(ny), _ptr(Sa), float(rho0), _ptr(u), int(dtype),
                                int(nslabs), dev, ctypes.byref(s)), "lbm_slabs_create")
    return s


def lbm_slabs_rows(s, k):
    """(first row, rows, device) of slab k."""
    y0, r, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _ck(load().lbm_slabs_rows(s, int(k), ctypes.byref(y0), ctypes.byref(r), ctypes.byref(d)),
        "lbm_slabs_rows")
    return y0.value, r.value, d.value


def lbm_slabs_init_field(s, rho, ux, uy):
    rho, ux, uy = (_f64(a) for a in (rho, ux, uy))
    _ck(load().lbm_slabs_init_field(s, _ptr(rho), _ptr(ux), _ptr(uy)), "lbm_slabs_init_field")


def lbm_slabs_set_populations(s, f):
    f = _f64(f)
    _ck(load().lbm_slabs_set_populations(s, _ptr(f)), "lbm_slabs_set_populations")


def lbm_slabs_step(s, n):
    _ck(load().lbm_slabs_step(s, int(n)), "lbm_slabs_step")


def lbm_slabs_moments(s, ny, nx):
    rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
    _ck(load().lbm_slabs_moments(s, _ptr(rho), _ptr(ux), _ptr(uy)), "lbm_slabs_moments")
    return rho, ux, uy


def lbm_slabs_get_populations(s, ny, nx):
    f = np.empty((9, ny, nx))
    _ck(load().lbm_slabs_get_populations(s, _ptr(f)), "lbm_slabs_get_populations")
    return f


def lbm_slabs_drift(s):
    out = np.zeros(4)
    rc = load().lbm_slabs_drift(s, _ptr(out))
    if rc not in (LBM_OK, LBM_EUNSTABLE):
        raise LbmError(rc, "lbm_slabs_drift")
    return out


def lbm_slabs_destroy(s):
    _ck(load().lbm_slabs_destroy(s), "lbm_slabs_destroy")


def lbm_slab_create(nx, ny_total, y0, rows, S, rho0=1.0, u0=(0.0, 0.0), dtype=LBM_F32DEV):
    """Handle of rows [y0, y0 + rows) of an nx x ny_total periodic lattice,
    for one slab per process; the caller exchanges its halo rows."""
    Sa = _f64(S, (9,))
    u = _f64(u0, (2,))
    h = _vp()
    _ck(load().lbm_slab_create(int(nx), int(ny_total), int(y0), int(rows), _ptr(Sa), float(rho0),
                               _ptr(u), int(dtype), ctypes.byref(h)), "lbm_slab_create")
    return h


def lbm_slab_halo_bytes(h):
    n = ctypes.c_size_t()
    _ck(load().lbm_slab_halo_bytes(h, ctypes.byref(n)), "lbm_slab_halo_bytes")
    return n.value


def lbm_slab_pack(h, reverse, to_below, to_above):
    """Copy the slab's outgoing rows into two device buffers (torch CUDA
    tensors or device addresses) of lbm_slab_halo_bytes bytes each."""
    _ck(load().lbm_slab_pack(h, int(bool(reverse)), _vp(_dev(to_below)), _vp(_dev(to_above))),
        "lbm_slab_pack")


def lbm_slab_unpack(h, reverse, from_below, from_above):
    _ck(load().lbm_slab_unpack(h, int(bool(reverse)), _vp(_dev(from_below)),
                               _vp(_dev(from_above))), "lbm_slab_unpack")


def lbm_debug_bounds(reset=False):
    """The debug build's index-check word (0: no failed check); raises on a
    library built without the checks."""
    w = ctypes.c_uint()
    _ck(load().lbm_debug_bounds(ctypes.byref(w), int(bool(reset))), "lbm_debug_bounds")
    return w.value


def lbm_debug_bounds_selftest():
    _ck(load().lbm_debug_bounds_selftest(), "lbm_debug_bounds_selftest")


BATCH_PHASES = ("h2d_ms", "init_ms", "steps_ms", "drift_ms", "moments_ms", "d2h_ms")


def lbm_batch_wait(b):
    """Wait for the queued solves; returns the device times per phase (dict
    keyed by BATCH_PHASES; each the median over the solves queued since the
    previous wait, the last 32 at most) and "unstable": whether a drift array
    passed since the previous wait reports non-finite populations (as
    lbm_batch_drift, that is a result, not an error).  Invalid input fields
    raise LbmError (LBM_EINVAL)."""
    ms = np.zeros(6)
    rc = load().lbm_batch_wait(b, _ptr(ms))
    if rc not in (LBM_OK, LBM_EUNSTABLE):
        raise LbmError(rc, "lbm_batch_wait")
    out = dict(zip(BATCH_PHASES, (float(x) for x in ms)))
    out["unstable"] = rc == LBM_EUNSTABLE
    return out


def cost_spec(kind="F", order=5, part="all", reference=None, u0=0.2, fixed_speed=False):
    """lbm_cost_spec from names: kind 'F' / 'G', part 'all' / 'odd' / 'even',
    reference 'ns' / 'euler' / 'ns-bulk' (default 'ns' for F, 'euler' for G)."""
    if reference is None:
        reference = "ns" if kind == "F" else "euler"
    return lbm_cost_spec(
        {"F": LBM_COST_F, "G": LBM_COST_G}[kind], int(order),
        {"all": LBM_PART_ALL, "odd": LBM_PART_ODD, "even": LBM_PART_EVEN}[part],
        {"ns": LBM_REF_NS, "euler": LBM_REF_EULER, "ns-bulk": LBM_REF_NS_BULK}[reference],
        float(u0), 1 if fixed_speed else 0)


def lbm_opt_cost(spec, sigmas):
    """Costs of candidates: sigmas (n, 4) = (sigma_e, sigma_eps, sigma_q,
    sigma_nu) per row -> (n,) array."""
    sig = _f64(np.atleast_2d(np.asarray(sigmas, dtype=np.float64)))
    if sig.ndim != 2 or sig.shape[1] != 4:
        raise ValueError("sigmas must have shape (n, 4)")
    out = np.empty(sig.shape[0])
    _ck(load().lbm_opt_cost(ctypes.byref(spec), sig.shape[0], _ptr(sig), _ptr(out)),
        "lbm_opt_cost")
    return out


def lbm_opt_minimize(spec, sigmas, free, lo, hi):
    """Minimize over the sigmas named in `free` (others held at `sigmas`)
    within [lo, hi] (dicts by name).  Returns (dict of the four sigmas,
    cost, number of cost evaluations)."""
    s_in = _f64(np.asarray([sigmas[k] for k in SIGMA_NAMES], dtype=np.float64))
    mask = 0
    lo_a = np.zeros(4)
    hi_a = np.ones(4)
    for i, k in enumerate(SIGMA_NAMES):
        if k in free:
            mask |= 1 << i
            lo_a[i] = lo[k]
            hi_a[i] = hi[k]
    s_out = np.empty(4)
    c = ctypes.c_double()
    ev = ctypes.c_int()
    _ck(load().lbm_opt_minimize(ctypes.byref(spec), _ptr(s_in), mask, _ptr(lo_a), _ptr(hi_a),
                                _ptr(s_out), ctypes.byref(c), ctypes.byref(ev)),
        "lbm_opt_minimize")
    return dict(zip(SIGMA_NAMES, s_out.tolist())), c.value, ev.value


def lbm_batch_destroy(b):
    _ck(load().lbm_batch_destroy(b), "lbm_batch_destroy")


def lbm_server_create(hbm_budget_bytes, chunk_steps=100):
    s = _vp()
    _ck(load().lbm_server_create(int(hbm_budget_bytes), int(chunk_steps), ctypes.byref(s)),
        "lbm_server_create")
    return s


LBM_SERVE_FIFO, LBM_SERVE_SHORTEST = 0, 1


def lbm_server_set_policy(s, policy=LBM_SERVE_FIFO, max_resident_nodes=0):
    _ck(load().lbm_server_set_policy(s, int(policy), int(max_resident_nodes)),
        "lbm_server_set_policy")


def make_request(nx, ny, S, steps, dtype=LBM_F32DEV, rho0=1.0, u0=(0.0, 0.0),
                 init_kind=LBM_INIT_GAUSSIAN, init_params=(), fields=None):
    r = lbm_request()
    r.nx, r.ny = int(nx), int(ny)
    r.S[:] = [float(v) for v in S]
    r.rho0 = float(rho0)
    r.u0[:] = [float(u0[0]), float(u0[1])]
    r.dtype = DTYPES.get(dtype, dtype)
    r.steps = int(steps)
    r.init_kind = int(init_kind)
    p = list(init_params) + [0.0] * (8 - len(init_params))
    r.init_params[:] = [float(v) for v in p]
    keep = None
    if fields is not None:
        keep = tuple(_f64(a, (ny, nx)) for a in fields)
        r.rho, r.ux, r.uy = (_ptr(a) for a in keep)
    return r, keep


def lbm_submit(s, req):
    """req: an lbm_request (see make_request).  Returns the request id."""
    rid = ctypes.c_longlong()
    _ck(load().lbm_submit(s, ctypes.byref(req), ctypes.byref(rid)), "lbm_submit")
    return rid.value


def lbm_poll(s, rid, nx=None, ny=None):
    """(code, rho, ux, uy, latency_s).  With nx, ny the finished fields are
    returned as (ny, nx) arrays; without them they are discarded.  Arrays are
    None unless code == LBM_OK."""
    lat = ctypes.c_double()
    if nx is None:
        rc = load().lbm_poll(s, ctypes.c_longlong(rid), None, None, None, ctypes.byref(lat))
        if rc == LBM_OK:
            return rc, None, None, None, lat.value
    else:
        rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
        rc = load().lbm_poll(s, ctypes.c_longlong(rid), _ptr(rho), _ptr(ux), _ptr(uy),
                             ctypes.byref(lat))
        if rc == LBM_OK:
            return rc, rho, ux, uy, lat.value
    if rc == LBM_PENDING:
        return rc, None, None, None, None
    raise LbmError(rc, "lbm_poll")


def lbm_server_stats(s):
    st = lbm_server_stats_t()
    _ck(load().lbm_server_stats(s, ctypes.byref(st)), "lbm_server_stats")
    return {k: getattr(st, k) for k, _ in lbm_server_stats_t._fields_}


def lbm_server_done(s, cap=4096):
    """Ids of the requests finished since the previous call (at most cap)."""
    ids = (ctypes.c_longlong * cap)()
    n = ctypes.c_int()
    _ck(load().lbm_server_done(s, ids, cap, ctypes.byref(n)), "lbm_server_done")
    return list(ids[:n.value])


def lbm_server_destroy(s):
    _ck(load().lbm_server_destroy(s), "lbm_server_destroy")
