"""Thin Python binding of the RIDG C ABI (include/ridg.h).

Functions carry the C names and only marshal arguments: every step of the RIDG path runs
in the CUDA kernels of lib/libridg.so.  Host arrays are numpy float64 arrays; device
arrays are torch CUDA float64 tensors (passed by pointer).  If the library is missing the
import of this module fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libridg.so")

RIDG_OK, RIDG_EINVAL, RIDG_ENOMEM, RIDG_ECUDA, RIDG_ENONFINITE, RIDG_ENOCONV, RIDG_ETIMEOUT, \
    RIDG_ESTATE, RIDG_ETOOBIG = range(9)
RIDG_FLUX_ADVECTION, RIDG_FLUX_BURGERS, RIDG_FLUX_EULER = range(3)
RIDG_PREC_FP64, RIDG_PREC_MIXED_BF16, RIDG_PREC_MIXED_FP32, RIDG_PREC_MIXED_TF32, \
    RIDG_PREC_MIXED_FP16 = range(5)

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class ridg_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class ridg_flux(C.Structure):
    _fields_ = [("kind", C.c_int), ("vel", C.c_double * 3), ("gamma", C.c_double)]


class ridg_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("slices", C.c_int), ("newton_max_iters", C.c_int),
                ("newton_tol", C.c_double), ("stream", C.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class ridg_info_t(C.Structure):
    _fields_ = [("dim", C.c_int), ("order", C.c_int), ("m", C.c_int), ("theta_s", C.c_int),
                ("theta_t", C.c_int), ("cells", C.c_longlong), ("dt", C.c_double),
                ("t", C.c_double), ("steps", C.c_longlong), ("newton_unconverged", C.c_longlong),
                ("newton_iters_max", C.c_int), ("precision", C.c_int), ("slices", C.c_int),
                ("newton_iters_total", C.c_longlong), ("newton_hist", C.c_longlong * 16),
                ("mass", C.c_double * 4)]


class ridg_profile_t(C.Structure):
    _fields_ = [("predict_ms", C.c_double), ("correct_ms", C.c_double), ("step_ms", C.c_double),
                ("launches_per_step", C.c_int)]


EXPORTS = {
    "ridg_create": (C.c_int, [C.POINTER(ridg_mesh), C.c_int, C.POINTER(ridg_flux), C.c_double,
                              C.POINTER(ridg_options), C.POINTER(C.c_void_p)]),
    "ridg_destroy": (None, [C.c_void_p]),
    "ridg_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "ridg_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "ridg_set_dt": (C.c_int, [C.c_void_p, C.c_double]),
    "ridg_set_final_time": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_longlong)]),
    "ridg_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "ridg_correct": (C.c_int, [C.c_void_p]),
    "ridg_step": (C.c_int, [C.c_void_p, C.c_int]),
    "ridg_sync": (C.c_int, [C.c_void_p]),
    "ridg_info": (C.c_int, [C.c_void_p, C.POINTER(ridg_info_t)]),
    "ridg_profile_step": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(ridg_profile_t)]),
    "ridg_mass": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "ridg_l2_error": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "ridg_check_bounded_wait": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "ridg_l2_error_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_int, C.c_int,
                                        C.c_int, C.c_void_p, C.POINTER(C.c_double)]),
    "ridg_batch_create": (C.c_int, [C.c_int, C.POINTER(ridg_mesh), C.POINTER(C.c_int),
                                    C.POINTER(ridg_flux), C.c_double, C.POINTER(ridg_options),
                                    C.POINTER(C.c_void_p)]),
    "ridg_batch_destroy": (None, [C.c_void_p]),
    "ridg_batch_instance": (C.c_void_p, [C.c_void_p, C.c_int]),
    "ridg_batch_set_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "ridg_batch_get_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "ridg_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "ridg_batch_schedule": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ridg_batch_autotune": (C.c_int, [C.c_void_p, C.c_char_p]),
    "ridg_batch_sync": (C.c_int, [C.c_void_p]),
    "ridg_autotune": (C.c_int, [C.c_void_p, C.c_char_p]),
    "ridg_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]),
    "ridg_tune_load": (C.c_int, [C.c_char_p]),
    "ridg_tune_lookup": (C.c_int, [C.c_char_p, C.POINTER(C.c_int)]),
    "ridg_shard_create": (C.c_int, [C.POINTER(ridg_mesh), C.c_int, C.POINTER(ridg_flux), C.c_double,
                                    C.POINTER(ridg_options), C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_void_p)]),
    "ridg_shard_destroy": (None, [C.c_void_p]),
    "ridg_shard_slab": (C.c_void_p, [C.c_void_p, C.c_int]),
    "ridg_shard_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "ridg_shard_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "ridg_shard_step": (C.c_int, [C.c_void_p, C.c_int]),
    "ridg_shard_sync": (C.c_int, [C.c_void_p]),
    "ridg_strerror": (C.c_char_p, [C.c_int]),
    "ridg_last_error": (C.c_char_p, [C.c_void_p]),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"RIDG CUDA library not built ({path}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load()


class RidgError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{_lib.ridg_strerror(status).decode()} ({status}): {msg}")
        self.status = status


def _check(status, h=None, allow=()):
    if status != RIDG_OK and status not in allow:
        msg = _lib.ridg_last_error(h).decode() if h else ""
        raise RidgError(status, msg)
    return status


def _ptr(a):
    """(pointer, on_device) of a float64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data_as(C.c_void_p), 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(type(a))


def make_mesh(dim, n, lo=None, hi=None):
    m = ridg_mesh()
    m.dim = dim
    for d in range(3):
        m.n[d] = int(n[d]) if d < dim else 1
        m.lo[d] = float(lo[d]) if (lo is not None and d < dim) else 0.0
        m.hi[d] = float(hi[d]) if (hi is not None and d < dim) else 1.0
    return m


def make_flux(kind="advection", vel=(0.0, 0.0, 0.0), gamma=1.4):
    f = ridg_flux()
    f.kind = {"advection": RIDG_FLUX_ADVECTION, "burgers": RIDG_FLUX_BURGERS,
              "euler": RIDG_FLUX_EULER}[kind]
    for d in range(3):
        f.vel[d] = float(vel[d]) if d < len(vel) else 0.0
    f.gamma = float(gamma)
    return f


def torch_allocator(device=None, stream=0):
    """Device allocator callbacks that draw from torch's caching allocator."""
    import torch
    dev = torch.cuda.current_device() if device is None else device

    @ALLOC_FN
    def _alloc(nbytes, user):
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)

    @FREE_FN
    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return _alloc, _free


def make_options(precision=RIDG_PREC_FP64, slices=0, newton_max_iters=0, newton_tol=0.0,
                 stream=None, allocator=None):
    o = ridg_options()
    o.precision = precision
    o.slices = slices
    o.newton_max_iters = newton_max_iters
    o.newton_tol = newton_tol
    o.stream = stream
    if allocator is not None:
        o.alloc, o.free = allocator
    return o


# ----- the C entry points with the same names -------------------------------------------
def ridg_create(mesh, order, flux, cfl, opt=None):
    h = C.c_void_p()
    _check(_lib.ridg_create(C.byref(mesh), int(order), C.byref(flux), float(cfl),
                            C.byref(opt) if opt is not None else None, C.byref(h)))
    return h


def ridg_destroy(h):
    _lib.ridg_destroy(h)


def ridg_set_state(h, q):
    p, dev = _ptr(q)
    return _check(_lib.ridg_set_state(h, p, dev), h)


def ridg_get_state(h, q):
    p, dev = _ptr(q)
    return _check(_lib.ridg_get_state(h, p, dev), h)


def ridg_set_dt(h, dt):
    return _check(_lib.ridg_set_dt(h, float(dt)), h)


def ridg_set_final_time(h, T):
    n = C.c_longlong()
    _check(_lib.ridg_set_final_time(h, float(T), C.byref(n)), h)
    return n.value


def ridg_predict(h, w_out=None):
    if w_out is None:
        return _check(_lib.ridg_predict(h, None, 0), h, allow=(RIDG_ENOCONV,))
    p, dev = _ptr(w_out)
    return _check(_lib.ridg_predict(h, p, dev), h, allow=(RIDG_ENOCONV,))


def ridg_correct(h):
    return _check(_lib.ridg_correct(h), h)


def ridg_step(h, n=1):
    return _check(_lib.ridg_step(h, int(n)), h)


def ridg_sync(h):
    return _check(_lib.ridg_sync(h), h, allow=(RIDG_ENOCONV,))


def ridg_info(h):
    i = ridg_info_t()
    _check(_lib.ridg_info(h, C.byref(i)), h)
    out = {k: getattr(i, k) for k, _ in ridg_info_t._fields_}
    out["newton_hist"] = list(i.newton_hist)
    out["mass"] = list(i.mass)[: i.m]
    return out


def ridg_profile_step(h, n=1):
    p = ridg_profile_t()
    _check(_lib.ridg_profile_step(h, int(n), C.byref(p)), h, allow=(RIDG_ENOCONV,))
    return {k: getattr(p, k) for k, _ in ridg_profile_t._fields_}


def ridg_mass(h, m=1):
    out = (C.c_double * m)()
    _check(_lib.ridg_mass(h, out), h)
    return np.array(out[:])


def ridg_l2_error(h, x):
    p, dev = _ptr(x)
    e = C.c_double()
    _check(_lib.ridg_l2_error(h, p, dev, C.byref(e)), h)
    return e.value


def ridg_check_bounded_wait(stream=None):
    """Run the bounded-wait check; returns (status, seconds): RIDG_ETIMEOUT is the expected
    status (the wait gave up and reported it)."""
    sec = C.c_double(0.0)
    st = _lib.ridg_check_bounded_wait(stream, C.byref(sec))
    return st, sec.value


def ridg_l2_error_noalloc(q, x, cells, m, dim, order, stream=None):
    """Relative L2 error of device arrays q and x with no device allocation (fixed scratch).

    q holds cells * m * (order+1)^dim and x cells * m * (order+2)^dim doubles, both on the
    current CUDA device (the C side launches there and uses that device's scratch);
    `stream` is a torch.cuda.Stream, a raw cudaStream_t as int, or None (legacy stream)."""
    import torch
    pq, dq = _ptr(q)
    px, dx = _ptr(x)
    if not (dq and dx):
        raise ValueError("ridg_l2_error_noalloc takes device arrays")
    cells, m, dim, order = int(cells), int(m), int(dim), int(order)
    if dim < 1 or dim > 3 or m < 1 or order < 0 or cells < 1:
        raise ValueError("bad sizes")
    if q.numel() != cells * m * (order + 1) ** dim or x.numel() != cells * m * (order + 2) ** dim:
        raise ValueError(f"sizes do not match: q {q.numel()}, x {x.numel()} for {cells} cells, "
                         f"m={m}, dim={dim}, order={order}")
    cur = torch.cuda.current_device()
    if q.device.index != cur or x.device.index != cur:
        raise ValueError("q and x must be on the current CUDA device")
    if isinstance(stream, torch.cuda.Stream):
        stream = stream.cuda_stream
    e = C.c_double()
    _check(_lib.ridg_l2_error_noalloc(pq, px, cells, m, dim, order,
                                      C.c_void_p(stream) if stream else None, C.byref(e)))
    return e.value


def ridg_autotune(h, cache_path=None):
    return _check(_lib.ridg_autotune(h, cache_path.encode() if cache_path else None), h)


def ridg_get_tuning(h):
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(_lib.ridg_get_tuning(h, C.byref(a), C.byref(b), C.byref(c)), h)
    return {"gemm3_slots": a.value, "corr3_block": b.value, "newton_grid": c.value}


def ridg_tune_load(path):
    return _check(_lib.ridg_tune_load(path.encode()))


def ridg_tune_lookup(key):
    """The cached value of key, or None."""
    v = C.c_int()
    return v.value if _lib.ridg_tune_lookup(key.encode(), C.byref(v)) == RIDG_OK else None


class Shard:
    """A linear-advection mesh sharded into slabs along its slowest axis (ridg_shard_*)."""

    def __init__(self, dim, n, order, vel, cfl, count, lo=None, hi=None, precision=RIDG_PREC_FP64,
                 slices=0, devices=None):
        mesh = make_mesh(dim, n, lo, hi)
        flux = make_flux("advection", vel)
        opt = make_options(precision=precision, slices=slices)
        devs = (C.c_int * count)(*devices) if devices else None
        s = C.c_void_p()
        _check(_lib.ridg_shard_create(C.byref(mesh), int(order), C.byref(flux), float(cfl),
                                      C.byref(opt), int(count), devs, C.byref(s)))
        self.s = s
        self.count = count

    def slab(self, i):
        return C.c_void_p(_lib.ridg_shard_slab(self.s, int(i)))

    def set_state(self, q):
        p, dev = _ptr(q)
        return _check(_lib.ridg_shard_set_state(self.s, p, dev))

    def get_state(self, q):
        p, dev = _ptr(q)
        return _check(_lib.ridg_shard_get_state(self.s, p, dev))

    def step(self, n=1):
        return _check(_lib.ridg_shard_step(self.s, int(n)))

    def sync(self):
        return _check(_lib.ridg_shard_sync(self.s))

    def close(self):
        if self.s:
            _lib.ridg_shard_destroy(self.s)
            self.s = None


def ridg_batch_create(meshes, orders, flux, cfl, opt=None):
    n = len(meshes)
    ms = (ridg_mesh * n)(*meshes)
    os_ = (C.c_int * n)(*[int(o) for o in orders])
    b = C.c_void_p()
    _check(_lib.ridg_batch_create(n, ms, os_, C.byref(flux), float(cfl),
                                  C.byref(opt) if opt is not None else None, C.byref(b)))
    return b


def ridg_batch_destroy(b):
    _lib.ridg_batch_destroy(b)


def ridg_batch_instance(b, i):
    return C.c_void_p(_lib.ridg_batch_instance(b, int(i)))


def ridg_batch_set_state(b, i, q):
    p, dev = _ptr(q)
    return _check(_lib.ridg_batch_set_state(b, int(i), p, dev))


def ridg_batch_get_state(b, i, q):
    p, dev = _ptr(q)
    return _check(_lib.ridg_batch_get_state(b, int(i), p, dev))


def ridg_batch_schedule(b):
    sch, ln = C.c_int(), C.c_int()
    _check(_lib.ridg_batch_schedule(b, C.byref(sch), C.byref(ln)))
    return {"schedule": sch.value, "launches_per_step": ln.value}


def ridg_batch_autotune(b, cache_path=None):
    return _check(_lib.ridg_batch_autotune(b, cache_path.encode() if cache_path else None),
                  allow=(RIDG_ENOCONV,))


def ridg_batch_step(b, n=1):
    return _check(_lib.ridg_batch_step(b, int(n)))


def ridg_batch_sync(b):
    """Wait for the batch; RIDG_ENOCONV (returned, not raised) when Newton hit its cap in
    some instance (see each instance's ridg_info)."""
    return _check(_lib.ridg_batch_sync(b), allow=(RIDG_ENOCONV,))


# ----- convenience wrapper ---------------------------------------------------------------
class Solver:
    """Owns one handle, its CUDA stream (a torch stream) and torch-allocated state."""

    def __init__(self, dim, n, order, flux="advection", vel=(0.0, 0.0, 0.0), cfl=0.3,
                 lo=None, hi=None, gamma=1.4, precision=RIDG_PREC_FP64, slices=0,
                 newton_max_iters=0, newton_tol=0.0, use_torch_allocator=True):
        import torch
        self.torch = torch
        self.stream = torch.cuda.Stream()
        self._alloc = torch_allocator(stream=self.stream.cuda_stream) if use_torch_allocator else None
        self.opt = make_options(precision, slices, newton_max_iters, newton_tol,
                                C.c_void_p(self.stream.cuda_stream), self._alloc)
        self.mesh = make_mesh(dim, n, lo, hi)
        self.flux = make_flux(flux, vel, gamma)
        self.h = ridg_create(self.mesh, order, self.flux, cfl, self.opt)
        info = ridg_info(self.h)
        self.dim, self.order, self.m = dim, order, info["m"]
        self.theta_s, self.theta_t, self.cells = info["theta_s"], info["theta_t"], info["cells"]

    def close(self):
        if self.h:
            ridg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, q):
        return ridg_set_state(self.h, q)

    def get_state(self, out=None):
        if out is None:
            out = np.empty((self.cells, self.m * self.theta_s))
        ridg_get_state(self.h, out)
        return out

    def predict(self, out=None):
        """The centre prediction of every cell; `last_status` is RIDG_ENOCONV when Newton hit
        its iteration cap somewhere (the prediction is still complete)."""
        if out is None:
            out = np.empty((self.cells, self.m * self.theta_t))
        self.last_status = ridg_predict(self.h, out)
        return out

    def correct(self):
        return ridg_correct(self.h)

    def step(self, n=1):
        return ridg_step(self.h, n)

    def sync(self):
        self.last_status = ridg_sync(self.h)
        return self.last_status

    def info(self):
        return ridg_info(self.h)

    def set_dt(self, dt):
        return ridg_set_dt(self.h, dt)

    def autotune(self, cache_path=None):
        return ridg_autotune(self.h, cache_path)

    def tuning(self):
        return ridg_get_tuning(self.h)

    def set_final_time(self, T):
        return ridg_set_final_time(self.h, T)

    def mass(self):
        return ridg_mass(self.h, self.m)

    def profile_step(self, n=1):
        return ridg_profile_step(self.h, n)

    def l2_error(self, x):
        return ridg_l2_error(self.h, x)
