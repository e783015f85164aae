"""Failure detection on the GPU without a fault: the bounded mbarrier wait
that every tensor-core kernel uses runs out on a barrier nothing arrives at,
the kernel frees its tensor memory on its normal exit path and reports
IMG_ETIMEOUT, and the device keeps working."""
import numpy as np
import pytest

import synth
from oracle import imager as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    return G


def test_wait_runs_out_and_reports(G):
    from paper_1505_01348_gb300._lib import check_wait
    assert check_wait(1000, arrive=False) == G.IMG_ETIMEOUT
    assert check_wait(1000, arrive=True) == G.IMG_OK
    for _ in range(3):                         # repeatable, nothing left behind
        assert check_wait(200, arrive=False) == G.IMG_ETIMEOUT
    assert check_wait(0, arrive=False) == G.IMG_EINVAL
    assert check_wait(1 << 27, arrive=False) == G.IMG_EINVAL


def test_device_usable_after_timeouts(G):
    from paper_1505_01348_gb300._lib import check_wait
    assert check_wait(500, arrive=False) == G.IMG_ETIMEOUT
    job = synth.custom(3, 40, 16, 12, 2, 400, radius=4.0)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    im = G.Imager.from_job(job, precision=1)
    d = im.dirty()
    im.close()
    ref = np.real(np.einsum("ki,kl,li->i", A.conj(), job.R, A))
    assert np.linalg.norm(d - ref) <= 1e-5 * np.linalg.norm(ref)


def test_host_side_injections(G):
    """Corrupted inputs are rejected before any launch; iteration caps stop
    the solve with IMG_ENOTCONV and a valid partial image."""
    job = synth.custom(5, 12, 10, 10, 3, 800, radius=4.0)
    im = G.Imager(job.ant_xyz, job.l, job.m)
    bad = job.R.copy()
    bad[2, 3] = np.nan
    bad[3, 2] = np.nan
    with pytest.raises(G.ImgError) as e:
        im.set_covariance(bad, job.N)
    assert e.value.code == G.IMG_EINVAL
    im.close()
    for prec in (0, 1):
        im = G.Imager.from_job(job, precision=prec, max_outer=1)
        sigma, info = im.solve()
        assert info.status == G.IMG_ENOTCONV and info.converged == 0
        assert info.outer <= 1
        assert np.all(np.isfinite(sigma)) and np.all(sigma >= 0)
        assert np.all(sigma <= im.mvdr_bound() * (1 + 1e-5))
        im.close()
        im = G.Imager.from_job(job, precision=prec, lsqr_maxit=1)
        sigma, info = im.solve()          # may or may not converge; must stay valid
        assert np.all(np.isfinite(sigma)) and np.all(sigma >= 0)
        im.close()
