"""K > 1 snapshots on the GPU against the K-snapshot FP64 oracle, with the
array turned between snapshots and one covariance per snapshot (Sec. II):
the MF, MVDR and ASSC dirty images over K snapshots (img_snapshot_image;
Sec. III-C, Sec. III-D, eq. ASSC0) and the unconstrained LS / WLS image of
the stacked model (img_snapshot_ls_image; Sec. III-B/C, Sec. V-A LSQR)."""
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


# ---------------------------------------------------------------- K-snapshot LS / WLS image
def _oracle_ls(job, cost):
    """The K-snapshot oracle's LSQR on the explicit stacked operator (FP64,
    tolerances 1e-12): full column rank, so the LS / WLS image is unique."""
    As = S.steering_stack(job.ant_xyz, job.l, job.m, job.lam)
    Psi = S.khatri_rao_stack(As)
    bnd = S.bounds_k(As, Psi, job.R, job.N, O.Params(cost=cost))
    prob = S.cost_problem_k(As, Psi, job.R, bnd, cost)
    res = O.lsqr(prob.M, prob.b, 1e-12, 1e-12, 2000)
    assert res.istop in (1, 2)
    return prob, prob.to_sigma * res.x


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("cost", [0, 1])
@pytest.mark.parametrize("shape", [(16, 8, 8, 2), (24, 12, 10, 3)])
def test_snapshot_ls_image_matches_oracle(G, shape, cost, prec):
    p, nl, nm, K = shape
    job = synth.snapshots_custom(60 + p, p, nl, nm, 3, 20 * p, K, dtheta=0.3, radius=4.0, snr_db=5.0)
    prob, ref = _oracle_ls(job, cost)
    ims = _imagers(G, job, cost=cost, precision=prec, lsqr_atol=1e-7, lsqr_btol=1e-7)
    _set_cov(ims, job)
    sigma, info = G.snapshot_ls_image(ims, maxit=600)
    for im in ims:
        im.close()
    assert info.converged == 1
    tol = 1e-4 if prec != 2 else 1e-3
    assert _rel(sigma, ref) <= tol
    # optimality of the GPU image in FP64 on the stacked operator
    x = sigma / prob.to_sigma
    g = np.real(prob.M.conj().T @ (prob.b - prob.M @ x))
    g0 = np.real(prob.M.conj().T @ prob.b)
    assert np.linalg.norm(g) <= 10 * tol * np.linalg.norm(g0)


def test_snapshot_ls_image_one_snapshot_equals_ls_image(G):
    job = synth.custom(45, 20, 10, 9, 3, 400, radius=4.0, snr_db=5.0)
    for cost in (0, 1):
        im = G.Imager.from_job(job, cost=cost, precision=1, lsqr_atol=1e-7, lsqr_btol=1e-7)
        a, ia = im.ls_image(maxit=300)
        b, ib = G.snapshot_ls_image([im], maxit=300)
        im.close()
        assert abs(ia.lsqr_iters - ib.lsqr_iters) <= 10
        assert _rel(b, a) <= 1e-5


def test_snapshot_ls_image_errors(G):
    job = synth.snapshots_custom(54, 12, 8, 8, 2, 300, 2)
    a = G.Imager(job.ant_xyz[0], job.l, job.m, job.lam, cost=0)
    b = G.Imager(job.ant_xyz[1], job.l, job.m, job.lam, cost=1)
    a.set_covariance(job.R[0], job.N)
    with pytest.raises(G.ImgError) as e:
        G.snapshot_ls_image([a, b])              # b holds no covariance
    assert e.value.code == G.IMG_EINVAL
    b.set_covariance(job.R[1], job.N)
    with pytest.raises(G.ImgError) as e:
        G.snapshot_ls_image([a, b])              # different costs
    assert e.value.code == G.IMG_EINVAL
    b.close()
    out, info = G.snapshot_ls_image([a, a], maxit=40)
    assert np.all(np.isfinite(out)) and 1 <= info.lsqr_iters <= 40
    a.close()
