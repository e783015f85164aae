"""K > 1 snapshots on the GPU: the MF, MVDR and ASSC dirty images over K
snapshots (img_snapshot_image) against the K-snapshot FP64 oracle, with the
array turned between snapshots and one covariance per snapshot (Sec. II,
Sec. III-C, Sec. III-D, eq. ASSC0)."""
import numpy as np
import pytest

import synth
from oracle import imager as O
from oracle import snapshots as S

pytestmark = pytest.mark.gpu

PREC_TOL = {0: 1e-5, 1: 1e-5, 2: 1e-4}


@pytest.fixture(scope="module")
def G():
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    return G


def _imagers(G, job, **kw):
    return [G.Imager(job.ant_xyz[k], job.l, job.m, job.lam, **kw) for k in range(job.K)]


def _set_cov(ims, job):
    for k, im in enumerate(ims):
        im.set_covariance(job.R[k], job.N)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("shape", [(16, 20, 12, 2), (48, 17, 9, 3), (64, 24, 16, 4), (96, 12, 10, 2)])
def test_snapshot_images_match_oracle(G, shape, prec):
    p, nl, nm, K = shape
    job = synth.snapshots_custom(300 + p + K, p, nl, nm, 4, 4 * p + 200, K, dtheta=0.3,
                                 radius=8.0, snr_db=0.0)
    for bias_c in (0, 1):
        As = S.steering_stack(job.ant_xyz, job.l, job.m, job.lam)
        ref = S.bounds_k(As, S.khatri_rao_stack(As), job.R, job.N, O.Params(bias_c=bias_c))
        ims = _imagers(G, job, precision=prec, bias_c=bias_c)
        _set_cov(ims, job)
        got = {kind: G.snapshot_image(ims, kind) for kind in (G.SNAP_MF, G.SNAP_MVDR, G.SNAP_ASSC)}
        for im in ims:
            im.close()
        tol = PREC_TOL[prec]
        for kind, r in ((G.SNAP_MF, ref.dirty), (G.SNAP_MVDR, ref.mvdr), (G.SNAP_ASSC, ref.assc)):
            assert _rel(got[kind], r) <= tol, (kind, _rel(got[kind], r))
            assert np.max(np.abs(got[kind] - r) / r) <= 10 * tol
        if bias_c == 0:
            # ASSC <= MVDR <= MF, up to the arithmetic's error
            assert np.all(got[G.SNAP_ASSC] <= got[G.SNAP_MVDR] * (1 + 10 * tol))
            assert np.all(got[G.SNAP_MVDR] <= got[G.SNAP_MF] * (1 + 10 * tol))


def test_one_and_repeated_snapshots_reproduce_the_single_snapshot_images(G):
    job = synth.custom(41, 32, 20, 14, 3, 600, radius=6.0)
    im = G.Imager.from_job(job, precision=1, bias_c=1)
    d = im.dirty()
    mv = im.mvdr_bound()
    for K in (1, 2, 4):
        ims = [im] * K
        np.testing.assert_array_equal(G.snapshot_image(ims, G.SNAP_MF), d)
        np.testing.assert_array_equal(G.snapshot_image(ims, G.SNAP_MVDR), mv)
        np.testing.assert_array_equal(G.snapshot_image(ims, G.SNAP_ASSC), mv)
    im.close()


def test_device_output_equals_host_output(G):
    torch = pytest.importorskip("torch")
    job = synth.snapshots_custom(52, 40, 16, 16, 3, 800, 3)
    ims = _imagers(G, job, precision=1)
    _set_cov(ims, job)
    for kind in (G.SNAP_MF, G.SNAP_MVDR, G.SNAP_ASSC):
        host = G.snapshot_image(ims, kind)
        dev = torch.empty(job.Q, dtype=torch.float64, device="cuda")
        G.snapshot_image(ims, kind, out=dev)
        np.testing.assert_array_equal(dev.cpu().numpy(), host)
    for im in ims:
        im.close()


def test_snapshot_image_argument_errors(G):
    job = synth.snapshots_custom(53, 12, 10, 8, 2, 300, 2)
    ims = _imagers(G, job)
    _set_cov(ims, job)

    def code(fn):
        with pytest.raises(G.ImgError) as e:
            fn()
        return e.value.code

    assert code(lambda: G.snapshot_image([], G.SNAP_MF, out=np.empty(job.Q))) == G.IMG_EINVAL
    assert code(lambda: G.snapshot_image(ims, 7)) == G.IMG_EINVAL
    assert code(lambda: G.snapshot_image([ims[0]] * (G.MAX_SNAPSHOTS + 1))) == G.IMG_EINVAL
    # a context without a covariance
    fresh = G.Imager(job.ant_xyz[1], job.l, job.m, job.lam)
    assert code(lambda: G.snapshot_image([ims[0], fresh])) == G.IMG_EINVAL
    # a different N, a different grid, a different bias constant
    fresh.set_covariance(job.R[1], job.N + 1)
    assert code(lambda: G.snapshot_image([ims[0], fresh])) == G.IMG_EINVAL
    fresh.close()
    other = G.Imager(job.ant_xyz[1], job.l, job.m[:-1], job.lam)
    other.set_covariance(job.R[1], job.N)
    assert code(lambda: G.snapshot_image([ims[0], other])) == G.IMG_EINVAL
    other.close()
    other = G.Imager(job.ant_xyz[1], job.l, job.m, job.lam, bias_c=1)
    other.set_covariance(job.R[1], job.N)
    assert code(lambda: G.snapshot_image([ims[0], other])) == G.IMG_EINVAL
    other.close()
    # still usable after the errors
    out = G.snapshot_image(ims, G.SNAP_MVDR)
    assert np.all(np.isfinite(out)) and np.all(out > 0)
    for im in ims:
        im.close()
