"""CUDA path against the FP64 oracle, through the C ABI.

Tolerances: operators (dirty image, MVDR bound, Psi, Psi^H) <= 1e-5
relative; images <= 1e-4 relative L2, with the same final pixel sets."""
import numpy as np
import pytest

import synth
from oracle import imager as O

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
IMG_TOL = 1e-4
# operator tolerance per arithmetic: FP32 CUDA cores, FP16x3 and BF16x3 tensor cores
PREC_TOL = {0: 1e-5, 1: 1e-5, 2: 1e-4}


@pytest.fixture(scope="module")
def G():
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    return G


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _oracle_ops(job):
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    return A, Psi


# ---------------------------------------------------------------- operators
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("shape", [(16, 32, 32), (7, 13, 11), (33, 9, 17), (64, 8, 8), (64, 40, 41)])
def test_dirty_and_mvdr_match_oracle(G, shape, prec):
    p, nl, nm = shape
    job = synth.custom(100 + p, p, nl, nm, 3, 4 * p + 50, radius=5.0, snr_db=0.0)
    A, Psi = _oracle_ops(job)
    prm = O.Params(bias_c=1)
    b = O.bounds(A, Psi, job.R, job.N, prm)
    im = G.Imager.from_job(job, bias_c=1, precision=prec)
    d = im.dirty()
    mv = im.mvdr_bound()
    tol = PREC_TOL[prec]
    assert _rel(d, b.dirty) <= tol
    assert np.max(np.abs(d - b.dirty) / b.dirty) <= 10 * tol
    assert _rel(mv, b.mvdr) <= tol
    assert np.all(mv / b.C <= d * (1 + 1e-5))      # Cauchy-Schwarz holds for C = 1
    im.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("p", [9, 48, 64])
def test_psi_pair_matches_explicit_khatri_rao(G, prec, p):
    job = synth.custom(5, p, 21, 13, 2, 400 + 4 * p, radius=3.0)
    A, Psi = _oracle_ops(job)
    im = G.Imager.from_job(job, precision=prec)
    rng = np.random.default_rng(1)
    x = rng.random(job.Q)
    K = im.psi(x)
    ref = O.unvect(Psi @ x, job.p)
    assert _rel(K, ref) <= OP_TOL
    X = rng.standard_normal((job.p, job.p)) + 1j * rng.standard_normal((job.p, job.p))
    U = X + X.conj().T
    y = im.psi_adj(U)
    refy = np.real(Psi.conj().T @ O.vect(U))
    assert _rel(y, refy) <= PREC_TOL[prec]
    # adjoint identity on the GPU operators: <Psi x, U> = <x, Psi^H U>
    lhs = np.real(np.vdot(O.vect(K), O.vect(U)))
    rhs = float(x @ y)
    assert abs(lhs - rhs) <= PREC_TOL[prec] * np.linalg.norm(O.vect(K)) * np.linalg.norm(O.vect(U))
    im.close()


# ---------------------------------------------------------------- solve
def _oracle_image(job, cost, kappa, eps_floor):
    prm = O.Params(cost=cost, kappa=kappa, eps_floor=eps_floor, feas_tol=1e-5)
    return O.image_job(job, prm)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("cost", [0, 1])
def test_tiny_solve_matches_oracle(G, cost, prec):
    job = synth.tiny()
    ref = _oracle_image(job, cost, 6.0, 1e-6)
    im = G.Imager.from_job(job, cost=cost, kappa=6.0, eps_floor=1e-6, precision=prec)
    sigma, info = im.solve()
    assert info.converged == 1
    assert _rel(sigma, ref.solve.sigma) <= IMG_TOL
    np.testing.assert_array_equal(im.sets(), ref.solve.sets)
    assert np.all(sigma >= 0)
    im.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("seed", [41, 42])
def test_ragged_solve_matches_oracle(G, seed, prec):
    job = synth.custom(seed, 11, 19, 13, 4, 800, radius=4.0, snr_db=0.0)
    ref = _oracle_image(job, 1, 6.0, 1e-6)
    im = G.Imager.from_job(job, kappa=6.0, eps_floor=1e-6, precision=prec)
    sigma, info = im.solve()
    assert info.converged == 1
    assert _rel(sigma, ref.solve.sigma) <= IMG_TOL
    np.testing.assert_array_equal(im.sets(), ref.solve.sets)
    im.close()


def test_batch_equals_single(G):
    jobs = [synth.custom(60 + j, 8 + 3 * j, 12 + j, 10, 3, 500, radius=4.0) for j in range(4)]
    singles = []
    for job in jobs:
        im = G.Imager.from_job(job)
        singles.append(im.solve()[0])
        im.close()
    ims = [G.Imager.from_job(job) for job in jobs]
    outs, infos = G.solve_batch(ims)
    for a, b, inf in zip(outs, singles, infos):
        np.testing.assert_array_equal(a, b)
        assert inf.converged == 1
    for im in ims:
        im.close()


# ---------------------------------------------------------------- errors
def test_not_positive_definite_is_reported(G):
    job = synth.custom(3, 4, 5, 5, 1, 100)
    im = G.Imager(job.ant_xyz, job.l, job.m)
    R = np.array([[1, 2, 0, 0], [2, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], dtype=np.complex128)
    im.set_covariance(R, 100)
    with pytest.raises(G.ImgError) as e:
        im.dirty()
    assert e.value.code == G.IMG_ENOTPD
    im.close()


def test_invalid_arguments(G):
    job = synth.custom(3, 4, 5, 5, 1, 100)
    with pytest.raises(G.ImgError):
        G.Imager(job.ant_xyz, job.l, job.m, lam=-1.0)
    ant = job.ant_xyz.copy()
    ant[0, 2] = 1.0
    with pytest.raises(G.ImgError):
        G.Imager(ant, job.l, job.m)
    im = G.Imager(job.ant_xyz, job.l, job.m)
    with pytest.raises(G.ImgError):
        im.solve()                        # no covariance yet
    with pytest.raises(G.ImgError):
        im.set_covariance(job.R, 4)       # N <= p
    bad = job.R.copy()
    bad[0, 1] += 1.0                      # not Hermitian
    with pytest.raises(G.ImgError):
        im.set_covariance(bad, 100)
    im.close()
