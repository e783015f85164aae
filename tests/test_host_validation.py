"""Host-side argument validation of the C ABI, exercised without a GPU.

Every check here runs before the library touches CUDA, so it needs no
device; on a machine without one, a valid context request fails loudly with
IMG_ECUDA (there is no CPU fallback)."""
import ctypes as C

import numpy as np
import pytest

from paper_1505_01348_gb300 import _lib as L


@pytest.fixture(scope="module")
def lib():
    return L.load(build_if_missing=True)


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


class _Params:
    """A valid problem (p = 4 antennas on a plane, 3 x 2 grid) whose fields a
    test then breaks one at a time."""

    def __init__(self):
        self.ant = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [1.0, 1.0, 0.0]])
        self.l = np.array([-0.1, 0.0, 0.1])
        self.m = np.array([-0.1, 0.1])
        self.prm = L.default_params()
        self.prm.p, self.prm.n_l, self.prm.n_m = 4, 3, 2
        self._bind()
        self.prm.lambda_ = 1.0

    def _bind(self):
        dp = C.POINTER(C.c_double)
        self.prm.ant_xyz = self.ant.ctypes.data_as(dp)
        self.prm.l = self.l.ctypes.data_as(dp)
        self.prm.m = self.m.ctypes.data_as(dp)


def _create(lib, P):
    h = C.c_void_p()
    code = lib.img_create(C.byref(P.prm), C.byref(h))
    if h.value:
        lib.img_destroy(h)
    return code


BREAK = [
    ("p too small", lambda P: setattr(P.prm, "p", 1)),
    ("p too large", lambda P: setattr(P.prm, "p", 385)),
    ("empty grid", lambda P: setattr(P.prm, "n_l", 0)),
    ("grid above 2^24 pixels", lambda P: (setattr(P.prm, "n_l", 1 << 13), setattr(P.prm, "n_m", 1 << 12))),
    ("no positions", lambda P: setattr(P.prm, "ant_xyz", None)),
    ("wavelength zero", lambda P: setattr(P.prm, "lambda_", 0.0)),
    ("wavelength NaN", lambda P: setattr(P.prm, "lambda_", float("nan"))),
    ("unknown cost", lambda P: setattr(P.prm, "cost", 2)),
    ("unknown bound", lambda P: setattr(P.prm, "bound", 2)),
    ("unknown inflation", lambda P: setattr(P.prm, "inflate", 3)),
    ("unknown arithmetic", lambda P: setattr(P.prm, "precision", 3)),
    ("negative kappa", lambda P: setattr(P.prm, "kappa", -1.0)),
    ("negative LSQR tolerance", lambda P: setattr(P.prm, "lsqr_atol", -1e-6)),
    ("negative iteration cap", lambda P: setattr(P.prm, "lsqr_maxit", -1)),
    ("feasibility tolerance 1", lambda P: setattr(P.prm, "feas_tol", 1.0)),
    ("negative support capacity", lambda P: setattr(P.prm, "support_cap", -1)),
    ("non-finite position", lambda P: P.ant.__setitem__((2, 0), np.inf)),
    ("non-planar array", lambda P: P.ant.__setitem__((1, 2), 0.5)),
    ("non-finite grid line", lambda P: P.l.__setitem__(1, np.nan)),
]


@pytest.mark.parametrize("name,brk", BREAK, ids=[b[0] for b in BREAK])
def test_create_rejects_each_bad_field(lib, name, brk):
    P = _Params()
    brk(P)
    assert _create(lib, P) == L.IMG_EINVAL


def test_create_null_arguments(lib):
    P = _Params()
    h = C.c_void_p()
    assert lib.img_create(None, C.byref(h)) == L.IMG_EINVAL
    assert lib.img_create(C.byref(P.prm), None) == L.IMG_EINVAL


@pytest.mark.skipif(_has_gpu(), reason="a device is present")
def test_valid_problem_without_a_device_fails_loudly(lib):
    P = _Params()
    assert _create(lib, P) == L.IMG_ECUDA
    with pytest.raises(L.ImgError) as e:
        L.Imager(P.ant, P.l, P.m)
    assert e.value.code == L.IMG_ECUDA


def test_calls_on_a_null_context(lib):
    out = np.zeros(6)
    dp = out.ctypes.data_as(C.POINTER(C.c_double))
    R = np.eye(4, dtype=np.complex128)
    assert lib.img_set_covariance(None, R.ctypes.data, L.C128, 100, 0) == L.IMG_EINVAL
    assert lib.img_dirty(None, dp, 0) == L.IMG_EINVAL
    assert lib.img_mvdr_bound(None, dp, 0) == L.IMG_EINVAL
    assert lib.img_solve(None, dp, None, 0) == L.IMG_EINVAL
    assert lib.img_ls_image(None, 10, dp, None, 0) == L.IMG_EINVAL
    lib.img_destroy(None)                                    # NULL-safe


def test_batch_and_snapshot_argument_checks(lib):
    out = np.zeros(6)
    dp = out.ctypes.data_as(C.POINTER(C.c_double))
    none = (C.c_void_p * 2)()
    # empty or NULL handle lists
    assert lib.img_prepare_batch(None, 1) == L.IMG_EINVAL
    assert lib.img_prepare_batch(none, 0) == L.IMG_EINVAL
    # snapshot entry points: count, kind, output and handles are checked first
    assert lib.img_snapshot_image(None, 2, L.SNAP_MF, dp, 0) == L.IMG_EINVAL
    assert lib.img_snapshot_image(none, 0, L.SNAP_MF, dp, 0) == L.IMG_EINVAL
    assert lib.img_snapshot_image(none, L.MAX_SNAPSHOTS + 1, L.SNAP_MF, dp, 0) == L.IMG_EINVAL
    assert lib.img_snapshot_image(none, 2, 7, dp, 0) == L.IMG_EINVAL
    assert lib.img_snapshot_image(none, 2, L.SNAP_MVDR, None, 0) == L.IMG_EINVAL
    assert lib.img_snapshot_image(none, 2, L.SNAP_MVDR, dp, 0) == L.IMG_EINVAL    # NULL handles
    assert lib.img_snapshot_ls_image(None, 2, 10, dp, None, 0) == L.IMG_EINVAL
    assert lib.img_snapshot_ls_image(none, 2, 10, None, None, 0) == L.IMG_EINVAL
    assert lib.img_snapshot_ls_image(none, 0, 10, dp, None, 0) == L.IMG_EINVAL


def test_wait_selftest_range(lib):
    assert lib.img_check_wait(0, 1) == L.IMG_EINVAL
    assert lib.img_check_wait((1 << 26) + 1, 1) == L.IMG_EINVAL


def test_server_null_arguments(lib):
    sp = L.ServerParams()
    lib.img_server_params_default(C.byref(sp))
    s = C.c_void_p()
    assert lib.img_server_create(None, C.byref(s)) == L.IMG_EINVAL
    assert lib.img_server_create(C.byref(sp), None) == L.IMG_EINVAL
    job = C.c_longlong()
    P = _Params()
    R = np.eye(4, dtype=np.complex128)
    assert lib.img_server_submit(None, C.byref(P.prm), R.ctypes.data, L.C128, 100, C.byref(job)) == L.IMG_EINVAL
    lib.img_server_destroy(None)                              # NULL-safe
