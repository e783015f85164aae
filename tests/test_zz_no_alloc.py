"""The allocation-free forward operator img_psi_noalloc, for callers that
cannot allocate device memory, against the allocating img_psi and against
the oracle's Psi x.

The entry point keeps its working set in a static device array shared by
every call, so two calls in a row with different sizes must not see each
other's leftovers, and the largest accepted sizes (p = 64 on a 256 x 256 or
256 x 255 grid) fill that array.  This file is collected last so a run that
stops at the first failure has run every other test first."""
import numpy as np
import pytest

import synth
from oracle import imager as O

pytestmark = pytest.mark.gpu

TOL = 1e-5      # operator tolerance of the FP32 path


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _device_psi(G, torch, job, x):
    dev = torch.device("cuda", 0)
    ant = torch.from_numpy(np.ascontiguousarray(job.ant_xyz)).to(dev)
    l = torch.from_numpy(np.ascontiguousarray(job.l)).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(job.m)).to(dev)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    K = torch.zeros(job.p * job.p, dtype=torch.complex128, device=dev)
    code = G._lib.psi_noalloc(job.p, job.n_l, job.n_m, ant, l, m, job.lam, xd, K)
    assert code == G.IMG_OK, code
    return K.cpu().numpy().reshape(job.p, job.p, order="F")


def _oracle_psi(job, x):
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    return O.unvect(O.psi_apply(A, x), job.p)


def test_noalloc_matches_img_psi_twice():
    torch = pytest.importorskip("torch")
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    rng = np.random.default_rng(9)
    for job in (synth.custom(71, 48, 40, 37, 3, 600, radius=4.0),
                synth.custom(72, 13, 9, 22, 2, 300, radius=2.0)):
        x = rng.random(job.Q)
        im = G.Imager.from_job(job, precision=G.PREC_FP32)
        ref = im.psi(x)
        im.close()
        got = _device_psi(G, torch, job, x)
        assert _rel(got, ref) <= TOL
        assert _rel(got, _oracle_psi(job, x)) <= TOL


def test_noalloc_fills_its_capacity_after_a_smaller_call():
    """A small call, then the largest accepted shapes, which use every
    partial matrix and the full steering tables of the static array."""
    torch = pytest.importorskip("torch")
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    rng = np.random.default_rng(10)
    for job in (synth.custom(73, 9, 7, 5, 2, 200, radius=2.0),
                synth.custom(74, 64, 256, 256, 4, 1000, radius=8.0),
                synth.custom(75, 13, 6, 4, 2, 300, radius=2.0),
                synth.custom(76, 64, 256, 255, 4, 1000, radius=8.0)):
        x = rng.random(job.Q)
        im = G.Imager.from_job(job, precision=G.PREC_FP32)
        ref = im.psi(x)
        im.close()
        got = _device_psi(G, torch, job, x)
        assert _rel(got, ref) <= TOL
        assert _rel(got, _oracle_psi(job, x)) <= TOL


def test_noalloc_rejects_sizes_beyond_capacity():
    pytest.importorskip("torch")
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    lib = G._lib.load()
    # p = 65 is over the fixed capacity: rejected before any device work
    assert lib.img_psi_noalloc(65, 8, 8, 1, 1, 1, 1.0, 1, 1, None) == G._lib.IMG_ENOMEM
    assert lib.img_psi_noalloc(16, 300, 8, 1, 1, 1, 1.0, 1, 1, None) == G._lib.IMG_ENOMEM
    assert lib.img_psi_noalloc(16, 8, 8, 0, 1, 1, 1.0, 1, 1, None) == G._lib.IMG_EINVAL
