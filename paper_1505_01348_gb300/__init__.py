"""GB300 bounded least-squares radio imager (active set + LSQR on Khatri-Rao
operators), a CUDA library behind the C ABI of include/img.h.

Importing the package does not load the library; the first call does, and it
raises when the library has not been built.

The job server launches independent groups on many streams; CUDA maps
streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 unless set), and
streams sharing a queue serialise.  The package raises the default to 32 when
it is imported before CUDA is initialised and the variable is unset.
"""
import os as _os

_os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
from ._lib import (BOUND_MF, BOUND_MVDR, C64, C128, COST_LS, COST_PWLS, IMG_ECUDA, IMG_EINVAL,
                   IMG_ENOMEM, IMG_ENOTCONV, IMG_ENOTPD, IMG_ETIMEOUT, IMG_OK, INFLATE_NONE, INFLATE_RATIO, INFLATE_STD, PREC_BF16X3,
                   PREC_FP32, PREC_F16X3, SET_F, SET_L, SET_U, SNAP_ASSC, SNAP_MF, SNAP_MVDR,
                   MAX_SNAPSHOTS, ImgError, Imager, SolveInfo, load, prepare_batch, snapshot_image, snapshot_ls_image,
                   solve_batch, Server)

__all__ = ["Imager", "Server", "solve_batch", "prepare_batch", "snapshot_image", "snapshot_ls_image", "load", "ImgError", "SolveInfo", "COST_LS", "COST_PWLS",
           "BOUND_MF", "BOUND_MVDR", "INFLATE_NONE", "INFLATE_RATIO", "INFLATE_STD", "C64",
           "C128", "PREC_FP32", "PREC_F16X3", "PREC_BF16X3", "SET_L", "SET_U", "SET_F",
           "IMG_OK", "IMG_EINVAL", "IMG_ENOMEM", "IMG_ENOTPD", "IMG_ENOTCONV", "IMG_ETIMEOUT", "IMG_ECUDA",
           "SNAP_MF", "SNAP_MVDR", "SNAP_ASSC", "MAX_SNAPSHOTS"]
