"""Unconstrained LS / WLS image (every pixel free, img_ls_image) against the
FP64 oracle's LSQR on the explicit operator (Sec. III-B/C images, Sec. V-A
LSQR): full-column-rank problems (Q < p^2) whose least-squares solution is
unique, so both converge to the same image; the GPU image also satisfies the
normal equations M^H (b - M x) = 0 evaluated in FP64."""
import numpy as np
import pytest

import synth
from oracle import imager as O

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def G():
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    return G


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _oracle(job, cost):
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    bnd = O.bounds(A, Psi, job.R, job.N, O.Params(cost=cost))
    prob = O.cost_problem(A, Psi, job.R, bnd, cost)
    res = O.lsqr(prob.M, prob.b, 1e-12, 1e-12, 2000)
    assert res.istop in (1, 2)
    return prob, prob.to_sigma * res.x


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("cost", [0, 1])
@pytest.mark.parametrize("shape", [(16, 8, 8), (24, 12, 10)])
def test_ls_image_matches_oracle(G, shape, cost, prec):
    p, nl, nm = shape
    job = synth.custom(40 + p, p, nl, nm, 3, 20 * p, radius=4.0, snr_db=5.0)
    prob, ref = _oracle(job, cost)
    im = G.Imager.from_job(job, cost=cost, precision=prec, lsqr_atol=1e-7, lsqr_btol=1e-7)
    sigma, info = im.ls_image(maxit=600)
    im.close()
    assert info.converged == 1
    tol = IMG_TOL if prec != 2 else 1e-3
    assert _rel(sigma, ref) <= tol
    # optimality of the GPU image in FP64: ||M^H r|| small against ||M^H b||
    x = sigma / prob.to_sigma
    g = np.real(prob.M.conj().T @ (prob.b - prob.M @ x))
    g0 = np.real(prob.M.conj().T @ prob.b)
    assert np.linalg.norm(g) <= 10 * tol * np.linalg.norm(g0)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("cost", [0, 1])
@pytest.mark.parametrize("shape", [(72, 14, 12), (130, 12, 11)])
def test_ls_image_wide_arrays_match_oracle(G, shape, cost, prec):
    """p > 64: the tensor-core arithmetics run the streamed adjoint and the
    Gram-block forward (two B units at Kp = 160)."""
    p, nl, nm = shape
    job = synth.custom(60 + p, p, nl, nm, 3, 20 * p, radius=8.0, snr_db=5.0)
    prob, ref = _oracle(job, cost)
    im = G.Imager.from_job(job, cost=cost, precision=prec, lsqr_atol=1e-7, lsqr_btol=1e-7)
    sigma, info = im.ls_image(maxit=600)
    im.close()
    assert info.converged == 1
    tol = IMG_TOL if prec != 2 else 1e-3
    assert _rel(sigma, ref) <= tol
    x = sigma / prob.to_sigma
    g = np.real(prob.M.conj().T @ (prob.b - prob.M @ x))
    g0 = np.real(prob.M.conj().T @ prob.b)
    assert np.linalg.norm(g) <= 10 * tol * np.linalg.norm(g0)


def test_ls_image_errors_and_repeat(G):
    job = synth.custom(7, 12, 8, 8, 2, 500, radius=3.0)
    im = G.Imager(job.ant_xyz, job.l, job.m)
    with pytest.raises(G.ImgError) as e:
        im.ls_image()
    assert e.value.code == G.IMG_EINVAL
    im.set_covariance(job.R, job.N)
    a, _ = im.ls_image(maxit=50)
    b, _ = im.ls_image(maxit=50)
    np.testing.assert_array_equal(a, b)          # buffers reused, same result
    im.close()
