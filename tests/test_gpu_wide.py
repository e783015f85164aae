"""Wide arrays (64 < p <= 384): the streamed tensor-core adjoint (operand B
chunked in global memory, bulk-copied into shared memory per 64-column K
chunk; up to p = 256) and the (tile, unit) work-item adjoint (256 < p <=
384) against the definitions, evaluated directly in FP64.

* dirty image d_i = a_i^H R a_i and MVDR bound C / (a_i^H R^-1 a_i)
  (Sec. IV-A, Eq. 24), every pixel, ragged tiles and p not a multiple of 8;
* Psi^H vect(U) = Re diag(A^H U A) (Eq. 16) for a random Hermitian U;
* Psi x = vect(A diag(x) A^H) (Eq. 15, the tensor-core Gram-block forward,
  up to 12 blocks at p = 330) for signed, sparse and wide-range x;
* a solve whose bounds come from this operator (solver on CUDA cores) against
  the oracle image;
* one batch mixing wide and narrow arrays equals the jobs run one by one.
"""
import numpy as np
import pytest

import synth
from oracle import imager as O

pytestmark = pytest.mark.gpu

PREC_TOL = {1: 1e-5, 2: 1e-4}
IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def G():
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    return G


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _direct_bounds(job, bias_c):
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    d = np.real(np.einsum("ki,kl,li->i", A.conj(), job.R, A))
    h = np.real(np.einsum("ki,kl,li->i", A.conj(), np.linalg.inv(job.R), A))
    C = job.N / (job.N - job.p) if bias_c else 1.0
    return A, d, C / h


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("shape", [(65, 21, 13), (96, 24, 20), (128, 16, 16), (130, 9, 31),
                                   (200, 17, 11), (256, 20, 12), (300, 13, 11), (384, 9, 10)])
def test_wide_dirty_and_mvdr(G, shape, prec):
    p, nl, nm = shape
    job = synth.custom(700 + p, p, nl, nm, 4, 4 * p + 100, radius=8.0, snr_db=0.0)
    _, ref_d, ref_mv = _direct_bounds(job, 1)
    im = G.Imager.from_job(job, bias_c=1, precision=prec)
    d = im.dirty()
    mv = im.mvdr_bound()
    im.close()
    tol = PREC_TOL[prec]
    assert _rel(d, ref_d) <= tol
    assert np.max(np.abs(d - ref_d) / ref_d) <= 10 * tol
    assert _rel(mv, ref_mv) <= tol
    C = job.N / (job.N - job.p)
    assert np.all(mv / C <= d * (1 + 1e-5))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("p", [72, 160, 256, 288, 330])
def test_wide_psi_adjoint(G, p, prec):
    job = synth.custom(9, p, 19, 14, 2, 4 * p + 100, radius=6.0)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    rng = np.random.default_rng(p)
    X = rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p))
    U = X + X.conj().T
    im = G.Imager.from_job(job, precision=prec)
    y = im.psi_adj(U)
    # adjoint identity against the forward operator (tensor-core Gram blocks)
    x = rng.random(job.Q)
    K = im.psi(x)
    im.close()
    ref = np.real(np.einsum("ki,kl,li->i", A.conj(), U, A))
    assert _rel(y, ref) <= PREC_TOL[prec]
    lhs = np.real(np.vdot(O.vect(K), O.vect(U)))
    assert abs(lhs - float(x @ y)) <= PREC_TOL[prec] * np.linalg.norm(K) * np.linalg.norm(U)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("p,nl,nm", [(65, 21, 13), (96, 24, 20), (128, 16, 16), (200, 17, 11), (256, 20, 12),
                                    (288, 15, 13), (330, 9, 14)])
@pytest.mark.parametrize("kind", ["signed", "sparse", "range"])
def test_wide_forward(G, p, nl, nm, prec, kind):
    job = synth.custom(900 + p, p, nl, nm, 2, 4 * p + 100, radius=6.0)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    rng = np.random.default_rng(p + nl)
    if kind == "signed":
        x = rng.standard_normal(job.Q)
    elif kind == "sparse":
        x = np.zeros(job.Q)
        idx = rng.choice(job.Q, 7, replace=False)
        x[idx] = rng.uniform(0.5, 2.0, 7)
    else:
        x = 10.0 ** rng.uniform(-4, 2, job.Q)
    im = G.Imager.from_job(job, precision=prec)
    K = im.psi(x)
    im.close()
    ref = (A * x[None, :]) @ A.conj().T
    assert _rel(K, ref) <= PREC_TOL[prec]
    np.testing.assert_allclose(K, K.conj().T, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("cost", [0, 1])
def test_wide_solve_matches_oracle(G, cost):
    job = synth.custom(77, 96, 20, 18, 5, 3000, radius=10.0, snr_db=0.0)
    prm = O.Params(cost=cost, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5)
    ref = O.image_job(job, prm)
    im = G.Imager.from_job(job, cost=cost, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5, precision=1)
    sigma, info = im.solve()
    im.close()
    assert info.converged == 1
    assert _rel(sigma, ref.solve.sigma) <= IMG_TOL
    assert np.all(sigma >= 0)


def test_wide_and_narrow_batch_equals_single(G):
    shapes = [(96, 20, 16), (40, 24, 24), (160, 12, 12), (64, 16, 20), (256, 8, 8)]
    jobs = [synth.custom(800 + j, p, nl, nm, 4, 4 * p + 200, radius=8.0)
            for j, (p, nl, nm) in enumerate(shapes)]
    singles = []
    for job in jobs:
        im = G.Imager.from_job(job, precision=1)
        singles.append((im.dirty(), im.solve()[0]))
        im.close()
    ims = [G.Imager.from_job(job, precision=1) for job in jobs]
    outs, infos = G.solve_batch(ims)
    for im, out, (d, s) in zip(ims, outs, singles):
        np.testing.assert_array_equal(im.dirty(), d)
        np.testing.assert_array_equal(out, s)
        im.close()


def test_operators_stream_ordered_device_mode(G):
    """on_device = 2: device buffers, work queued on the context's stream and
    no host wait; after a device synchronisation the results equal the
    waiting calls' results bit for bit (p = 48 and 128, both operators)."""
    torch = pytest.importorskip("torch")
    for p in (48, 128):
        job = synth.custom(950 + p, p, 20, 12, 3, 4 * p + 100, radius=6.0)
        rng = np.random.default_rng(p)
        X = rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p))
        U = X + X.conj().T
        x = rng.standard_normal(job.Q)
        im = G.Imager.from_job(job, precision=1)
        Ud = torch.tensor(np.asfortranarray(U).T.copy(), dtype=torch.complex128, device="cuda")
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        y1 = torch.empty(job.Q, dtype=torch.float64, device="cuda")
        y2 = torch.empty_like(y1)
        K1 = torch.empty((p, p), dtype=torch.complex128, device="cuda")
        K2 = torch.empty_like(K1)
        im.psi_adj(Ud, y1)
        im.psi(xd, K1)
        im.psi_adj(Ud, y2, wait=False)
        im.psi(xd, K2, wait=False)
        torch.cuda.synchronize()
        im.close()
        assert torch.equal(y1, y2)
        assert torch.equal(K1, K2)
        # and the host-array calls agree with the device ones
        im = G.Imager.from_job(job, precision=1)
        np.testing.assert_array_equal(im.psi_adj(U), y1.cpu().numpy())
        im.close()
