"""ctypes binding of the C ABI in include/img.h (argument marshalling only).

Every computation happens in the CUDA library; this module converts numpy
arrays or torch CUDA tensors into pointers and status codes into exceptions.
It raises when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

IMG_OK, IMG_EINVAL, IMG_ENOMEM, IMG_ENOTPD, IMG_ENOTCONV, IMG_ETIMEOUT, IMG_ECUDA = range(7)
COST_LS, COST_PWLS = 0, 1
BOUND_MF, BOUND_MVDR = 0, 1
INFLATE_NONE, INFLATE_RATIO, INFLATE_STD = 0, 1, 2
C64, C128 = 0, 1
PREC_FP32, PREC_F16X3, PREC_BF16X3 = 0, 1, 2
SNAP_MF, SNAP_MVDR, SNAP_ASSC = 0, 1, 2
MAX_SNAPSHOTS = 32
SET_L, SET_U, SET_F = 0, 1, 2

EXPORTS = ("img_params_default", "img_create", "img_set_covariance", "img_dirty",
           "img_mvdr_bound", "img_solve", "img_get_sets", "img_get_gradient", "img_get_events",
           "img_psi",
           "img_psi_adj", "img_ls_image", "img_check_wait", "img_snapshot_image", "img_snapshot_ls_image", "img_prepare_batch", "img_solve_batch", "img_psi_noalloc",
           "img_server_params_default", "img_server_create", "img_server_reserve", "img_server_submit",
           "img_server_wait", "img_server_destroy", "img_destroy", "img_status_str")


class ImgParams(C.Structure):
    _fields_ = [("p", C.c_int), ("n_l", C.c_int), ("n_m", C.c_int),
                ("ant_xyz", C.POINTER(C.c_double)), ("l", C.POINTER(C.c_double)),
                ("m", C.POINTER(C.c_double)), ("lambda_", C.c_double),
                ("cost", C.c_int), ("bound", C.c_int), ("bias_c", C.c_int), ("inflate", C.c_int),
                ("alpha", C.c_double), ("kappa", C.c_double), ("eps_floor", C.c_double),
                ("lsqr_atol", C.c_double), ("lsqr_btol", C.c_double),
                ("lsqr_maxit", C.c_int), ("max_outer", C.c_int), ("feas_tol", C.c_double),
                ("precision", C.c_int), ("support_cap", C.c_int), ("stream", C.c_void_p)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("outer", C.c_int), ("lsqr_iters", C.c_int),
                ("n_free", C.c_int), ("n_upper", C.c_int), ("converged", C.c_int),
                ("lambda_min", C.c_double), ("op_flops", C.c_double),
                ("cyc_total", C.c_double), ("cyc_gradient", C.c_double),
                ("cyc_lsqr", C.c_double), ("cyc_lsqr_fwd", C.c_double),
                ("cyc_lsqr_adj", C.c_double), ("cyc_aux", C.c_double * 6),
                ("t_begin_ns", C.c_double), ("t_end_ns", C.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["cyc_aux"] = list(self.cyc_aux)
        return d


class ServerParams(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_inflight_jobs", C.c_int),
                ("max_batch", C.c_int), ("n_streams", C.c_int), ("max_pixels", C.c_int)]


class ImgError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_str(code)} ({code})")


_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load the CUDA library; raise when it is absent (no CPU fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {_build.LIB} is not built; run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        _build.build()
    lib = C.CDLL(_build.LIB)
    vp, i, ll, dp = C.c_void_p, C.c_int, C.c_longlong, C.c_void_p
    lib.img_params_default.argtypes = [C.POINTER(ImgParams)]
    lib.img_params_default.restype = None
    lib.img_create.argtypes = [C.POINTER(ImgParams), C.POINTER(vp)]
    lib.img_create.restype = i
    lib.img_set_covariance.argtypes = [vp, dp, i, ll, i]
    lib.img_set_covariance.restype = i
    for name in ("img_dirty", "img_mvdr_bound"):
        getattr(lib, name).argtypes = [vp, dp, i]
        getattr(lib, name).restype = i
    lib.img_solve.argtypes = [vp, dp, C.POINTER(SolveInfo), i]
    lib.img_solve.restype = i
    lib.img_ls_image.argtypes = [vp, i, dp, C.POINTER(SolveInfo), i]
    lib.img_ls_image.restype = i
    lib.img_check_wait.argtypes = [C.c_uint, i]
    lib.img_snapshot_image.restype = i
    lib.img_snapshot_image.argtypes = [C.POINTER(vp), i, i, dp, i]
    lib.img_snapshot_ls_image.restype = i
    lib.img_snapshot_ls_image.argtypes = [C.POINTER(vp), i, i, dp, C.POINTER(SolveInfo), i]
    lib.img_check_wait.restype = i
    lib.img_get_sets.argtypes = [vp, dp]
    lib.img_get_sets.restype = i
    lib.img_get_gradient.argtypes = [vp, dp]
    lib.img_get_gradient.restype = i
    lib.img_get_events.argtypes = [vp, dp, dp, i, C.POINTER(i)]
    lib.img_get_events.restype = i
    lib.img_psi.argtypes = [vp, dp, dp, i]
    lib.img_psi.restype = i
    lib.img_psi_adj.argtypes = [vp, dp, dp, i]
    lib.img_psi_adj.restype = i
    lib.img_prepare_batch.argtypes = [C.POINTER(vp), i]
    lib.img_prepare_batch.restype = i
    lib.img_solve_batch.argtypes = [C.POINTER(vp), i, C.POINTER(dp), C.POINTER(SolveInfo), i]
    lib.img_solve_batch.restype = i
    lib.img_psi_noalloc.argtypes = [i, i, i, dp, dp, dp, C.c_double, dp, dp, vp]
    lib.img_psi_noalloc.restype = i
    lib.img_server_params_default.argtypes = [C.POINTER(ServerParams)]
    lib.img_server_params_default.restype = None
    lib.img_server_create.argtypes = [C.POINTER(ServerParams), C.POINTER(vp)]
    lib.img_server_create.restype = i
    lib.img_server_reserve.argtypes = [vp, C.POINTER(ImgParams), i]
    lib.img_server_reserve.restype = i
    lib.img_server_submit.argtypes = [vp, C.POINTER(ImgParams), dp, i, ll, C.POINTER(ll)]
    lib.img_server_submit.restype = i
    lib.img_server_wait.argtypes = [vp, ll, dp, C.POINTER(SolveInfo), C.c_double, C.POINTER(C.c_double)]
    lib.img_server_wait.restype = i
    lib.img_server_destroy.argtypes = [vp]
    lib.img_server_destroy.restype = None
    lib.img_destroy.argtypes = [vp]
    lib.img_destroy.restype = None
    lib.img_status_str.argtypes = [i]
    lib.img_status_str.restype = C.c_char_p
    _LIB = lib
    return lib


def status_str(code: int) -> str:
    try:
        return load().img_status_str(code).decode()
    except Exception:  # library missing: still format the code
        return f"status {code}"


def _check(code: int, where: str, allow=()):
    if code != IMG_OK and code not in allow:
        raise ImgError(code, where)
    return code


def _ptr(a) -> int:
    """Address of a contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"]
        return a.ctypes.data
    return int(a.data_ptr())


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def default_params() -> ImgParams:
    prm = ImgParams()
    load().img_params_default(C.byref(prm))
    return prm


class Imager:
    """One imaging job on the GPU (wraps an img_ctx)."""

    def __init__(self, ant_xyz, l, m, lam: float = 1.0, **kw):
        self._lib = load()
        self.ant = np.ascontiguousarray(ant_xyz, dtype=np.float64)
        self.l = np.ascontiguousarray(l, dtype=np.float64)
        self.m = np.ascontiguousarray(m, dtype=np.float64)
        prm = default_params()
        prm.p = self.ant.shape[0]
        prm.n_l = self.l.shape[0]
        prm.n_m = self.m.shape[0]
        prm.ant_xyz = self.ant.ctypes.data_as(C.POINTER(C.c_double))
        prm.l = self.l.ctypes.data_as(C.POINTER(C.c_double))
        prm.m = self.m.ctypes.data_as(C.POINTER(C.c_double))
        prm.lambda_ = float(lam)
        for k, v in kw.items():
            if k == "stream":
                prm.stream = C.c_void_p(int(v))
            else:
                setattr(prm, k, v)
        self.prm = prm
        self.p, self.Q = prm.p, prm.n_l * prm.n_m
        h = C.c_void_p()
        _check(self._lib.img_create(C.byref(prm), C.byref(h)), "img_create")
        self.h = h

    @classmethod
    def from_job(cls, job, **kw):
        obj = cls(job.ant_xyz, job.l, job.m, job.lam, **kw)
        obj.set_covariance(job.R, job.N)
        return obj

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self._lib.img_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_covariance(self, R, N: int):
        if _is_device(R):
            import torch
            dt = C128 if R.dtype == torch.complex128 else C64
            code = self._lib.img_set_covariance(self.h, _ptr(R), dt, int(N), 1)
        else:
            R = np.asfortranarray(R)
            dt = C128 if R.dtype == np.complex128 else C64
            if R.dtype not in (np.complex64, np.complex128):
                R = np.asfortranarray(R, dtype=np.complex128)
                dt = C128
            code = self._lib.img_set_covariance(self.h, R.ctypes.data, dt, int(N), 0)
        _check(code, "img_set_covariance")

    def _qvec(self, fn, out, name, allow=()):
        if out is None:
            out = np.empty(self.Q, dtype=np.float64)
        code = fn(self.h, _ptr(out), 1 if _is_device(out) else 0)
        _check(code, name, allow)
        return out

    def dirty(self, out=None):
        return self._qvec(self._lib.img_dirty, out, "img_dirty")

    def mvdr_bound(self, out=None):
        return self._qvec(self._lib.img_mvdr_bound, out, "img_mvdr_bound")

    def ls_image(self, maxit=0, out=None):
        """Unconstrained LS / WLS image, every pixel free (img_ls_image)."""
        if out is None:
            out = np.empty(self.Q, dtype=np.float64)
        info = SolveInfo()
        _check(self._lib.img_ls_image(self.h, int(maxit), _ptr(out), C.byref(info), 1 if _is_device(out) else 0),
               "img_ls_image")
        return out, info

    def solve(self, out=None, allow=(IMG_ENOTCONV,)):
        if out is None:
            out = np.empty(self.Q, dtype=np.float64)
        info = SolveInfo()
        code = self._lib.img_solve(self.h, _ptr(out), C.byref(info), 1 if _is_device(out) else 0)
        _check(code, "img_solve", allow)
        return out, info

    def sets(self):
        out = np.empty(self.Q, dtype=np.uint8)
        _check(self._lib.img_get_sets(self.h, out.ctypes.data), "img_get_sets")
        return out

    def gradient(self):
        out = np.empty(self.Q, dtype=np.float64)
        _check(self._lib.img_get_gradient(self.h, out.ctypes.data), "img_get_gradient")
        return out

    def events(self, capacity: int = 1 << 20):
        """Decision log [(kind, pixel, value)], kind 0 free / 1 to L / 2 to U."""
        n = C.c_int()
        _check(self._lib.img_get_events(self.h, None, None, 0, C.byref(n)), "img_get_events")
        m = min(n.value, capacity)
        ev = np.empty(m, dtype=np.int32)
        val = np.empty(m, dtype=np.float64)
        _check(self._lib.img_get_events(self.h, ev.ctypes.data, val.ctypes.data, m, C.byref(n)),
               "img_get_events")
        return [(int(e) >> 24, int(e) & 0xFFFFFF, float(v)) for e, v in zip(ev, val)]

    def psi(self, x, out=None, wait=True):
        """K = unvect(Psi x) (p x p, column-major).  Host arrays, or CUDA
        tensors (float64 x, complex128 out) that stay on the device; with
        wait=False a device call returns once queued on the context stream."""
        if _is_device(x):
            if out is None:
                raise ValueError("device input needs a device output")
            _check(self._lib.img_psi(self.h, _ptr(x), _ptr(out), 1 if wait else 2), "img_psi")
            return out
        x = np.ascontiguousarray(x, dtype=np.float64)
        K = np.empty((self.p, self.p), dtype=np.complex128, order="F")
        _check(self._lib.img_psi(self.h, x.ctypes.data, K.ctypes.data, 0), "img_psi")
        return K

    def psi_adj(self, U, out=None, wait=True):
        """Re(a_i^H U a_i) for every pixel.  Host arrays, or CUDA tensors
        (complex128 U column-major, float64 out) that stay on the device; with
        wait=False a device call returns once queued on the context stream."""
        if _is_device(U):
            if out is None:
                raise ValueError("device input needs a device output")
            _check(self._lib.img_psi_adj(self.h, _ptr(U), _ptr(out), 1 if wait else 2), "img_psi_adj")
            return out
        U = np.asfortranarray(U, dtype=np.complex128)
        out = np.empty(self.Q, dtype=np.float64)
        _check(self._lib.img_psi_adj(self.h, U.ctypes.data, out.ctypes.data, 0), "img_psi_adj")
        return out


def check_wait(polls: int, arrive: bool) -> int:
    """Bounded-wait self-test (img_check_wait); returns the status code."""
    return load().img_check_wait(int(polls), 1 if arrive else 0)


def psi_noalloc(p, n_l, n_m, ant_xyz, l, m, lam, x, Kout, stream=0):
    """Allocation-free forward operator; every array argument is a device
    pointer (torch CUDA tensor or integer address).  Returns the status."""
    lib = load()
    a = [v if isinstance(v, int) else _ptr(v) for v in (ant_xyz, l, m, x, Kout)]
    return lib.img_psi_noalloc(int(p), int(n_l), int(n_m), a[0], a[1], a[2], float(lam), a[3], a[4],
                               C.c_void_p(int(stream)) if stream else None)


def prepare_batch(imagers):
    """Factor and bound several jobs in single launches."""
    lib = load()
    n = len(imagers)
    hs = (C.c_void_p * n)(*[im.h.value for im in imagers])
    _check(lib.img_prepare_batch(hs, n), "img_prepare_batch")


def snapshot_image(imagers, kind=None, out=None):
    """Dirty image over K snapshots, one Imager per snapshot
    (img_snapshot_image): kind SNAP_MF, SNAP_MVDR (default) or SNAP_ASSC."""
    lib = load()
    kind = SNAP_MVDR if kind is None else int(kind)
    n = len(imagers)
    if out is None:
        out = np.empty(imagers[0].Q if n else 0, dtype=np.float64)
    hs = (C.c_void_p * max(n, 1))(*[im.h.value for im in imagers])
    code = lib.img_snapshot_image(hs, n, kind, _ptr(out), 1 if _is_device(out) else 0)
    _check(code, "img_snapshot_image")
    return out


def snapshot_ls_image(imagers, maxit=0, out=None):
    """Unconstrained LS / WLS image over K snapshots, one Imager per snapshot
    (img_snapshot_ls_image); returns (image, SolveInfo)."""
    lib = load()
    n = len(imagers)
    if out is None:
        out = np.empty(imagers[0].Q if n else 0, dtype=np.float64)
    hs = (C.c_void_p * max(n, 1))(*[im.h.value for im in imagers])
    info = SolveInfo()
    code = lib.img_snapshot_ls_image(hs, n, int(maxit), _ptr(out), C.byref(info), 1 if _is_device(out) else 0)
    _check(code, "img_snapshot_ls_image")
    return out, info


def solve_batch(imagers, outs=None, allow=(IMG_ENOTCONV,)):
    """Solve several jobs in one launch; returns (images, infos)."""
    lib = load()
    n = len(imagers)
    if outs is None:
        outs = [np.empty(im.Q, dtype=np.float64) for im in imagers]
    dev = 1 if _is_device(outs[0]) else 0
    hs = (C.c_void_p * n)(*[im.h.value for im in imagers])
    ps = (C.c_void_p * n)(*[_ptr(o) for o in outs])
    infos = (SolveInfo * n)()
    code = lib.img_solve_batch(hs, n, ps, infos, dev)
    _check(code, "img_solve_batch", allow)
    return outs, list(infos)


class Server:
    """Continuous-batching job server (wraps img_server)."""

    def __init__(self, hbm_budget_bytes=None, max_inflight_jobs=0, max_batch=0, n_streams=0,
                 max_pixels=0):
        self._lib = load()
        sp = ServerParams()
        self._lib.img_server_params_default(C.byref(sp))
        if hbm_budget_bytes is not None:
            sp.hbm_budget_bytes = int(hbm_budget_bytes)
        sp.max_inflight_jobs = int(max_inflight_jobs)
        sp.max_batch = int(max_batch)
        if n_streams:
            sp.n_streams = int(n_streams)
        if max_pixels:
            sp.max_pixels = int(max_pixels)
        h = C.c_void_p()
        _check(self._lib.img_server_create(C.byref(sp), C.byref(h)), "img_server_create")
        self.h = h
        self._Q = {}

    def reserve(self, job, count: int, **kw):
        """Pre-create `count` pooled contexts shaped like `job`."""
        ant = np.ascontiguousarray(job.ant_xyz, dtype=np.float64)
        l = np.ascontiguousarray(job.l, dtype=np.float64)
        m = np.ascontiguousarray(job.m, dtype=np.float64)
        prm = default_params()
        prm.p, prm.n_l, prm.n_m = ant.shape[0], l.shape[0], m.shape[0]
        prm.ant_xyz = ant.ctypes.data_as(C.POINTER(C.c_double))
        prm.l = l.ctypes.data_as(C.POINTER(C.c_double))
        prm.m = m.ctypes.data_as(C.POINTER(C.c_double))
        prm.lambda_ = float(job.lam)
        for k, v in kw.items():
            setattr(prm, k, v)
        _check(self._lib.img_server_reserve(self.h, C.byref(prm), int(count)), "img_server_reserve")

    def submit(self, ant_xyz, l, m, lam, R, N, **kw) -> int:
        ant = np.ascontiguousarray(ant_xyz, dtype=np.float64)
        l = np.ascontiguousarray(l, dtype=np.float64)
        m = np.ascontiguousarray(m, dtype=np.float64)
        prm = default_params()
        prm.p, prm.n_l, prm.n_m = ant.shape[0], l.shape[0], m.shape[0]
        prm.ant_xyz = ant.ctypes.data_as(C.POINTER(C.c_double))
        prm.l = l.ctypes.data_as(C.POINTER(C.c_double))
        prm.m = m.ctypes.data_as(C.POINTER(C.c_double))
        prm.lambda_ = float(lam)
        for k, v in kw.items():
            setattr(prm, k, v)
        Rf = np.asfortranarray(R, dtype=np.complex128)
        jid = C.c_longlong()
        _check(self._lib.img_server_submit(self.h, C.byref(prm), Rf.ctypes.data, C128, int(N),
                                           C.byref(jid)), "img_server_submit")
        self._Q[jid.value] = prm.n_l * prm.n_m
        return jid.value

    def submit_job(self, job, **kw) -> int:
        return self.submit(job.ant_xyz, job.l, job.m, job.lam, job.R, job.N, **kw)

    def wait(self, job_id: int, timeout_ms: float = 600_000.0, allow=(IMG_ENOTCONV,)):
        """(image, info, latency_ms) of a finished job."""
        out = np.empty(self._Q[job_id], dtype=np.float64)
        info = SolveInfo()
        lat = C.c_double()
        code = self._lib.img_server_wait(self.h, int(job_id), out.ctypes.data, C.byref(info),
                                         float(timeout_ms), C.byref(lat))
        _check(code, "img_server_wait", allow)
        del self._Q[job_id]
        return out, info, lat.value

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self._lib.img_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
