"""Pins of the oracle's streamed operator form (Psi never stored, Sec. V-B).

The streamed form applies Psi x = vect(A diag(x) A^H) and
Psi^H vect(U) = Re vecdiag(A^H U A).  Each pin checks it against a route that
does not use these identities: explicit Kronecker columns kron(conj(a_i), a_i),
the explicit Kronecker weighting conj(L^-1) kron L^-1, closed forms of the
gradient at sigma = 0, the explicit-form Table I run, and scipy's bounded
least squares (BVLS) for the exact optimum."""
import numpy as np
import scipy.optimize as so

import synth
from oracle import imager as O


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _herm(rng, p):
    X = rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p))
    return X + X.conj().T


def _job_ops(seed=31, p=9, nl=7, nm=6):
    job = synth.custom(seed, p, nl, nm, 3, 800, radius=3.0, snr_db=3.0)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    return job, A


def test_streamed_forward_equals_kronecker_columns():
    rng = np.random.default_rng(1)
    _, A = _job_ops()
    Psi = np.stack([np.kron(A[:, i].conj(), A[:, i]) for i in range(A.shape[1])], axis=1)
    x = rng.standard_normal(A.shape[1])
    assert _rel(O.psi_apply(A, x), Psi @ x) < 1e-13


def test_streamed_adjoint_equals_kronecker_columns_and_blocks():
    rng = np.random.default_rng(2)
    _, A = _job_ops(p=11, nl=13, nm=9)
    Psi = np.stack([np.kron(A[:, i].conj(), A[:, i]) for i in range(A.shape[1])], axis=1)
    U = _herm(rng, A.shape[0])
    ref = np.real(Psi.conj().T @ O.vect(U))
    old = O.STREAM_BLOCK
    try:
        for blk in (old, 7, 1):          # pixel blocking is a memory bound only
            O.STREAM_BLOCK = blk
            assert _rel(O.psi_adjoint(A, U), ref) < 1e-13
    finally:
        O.STREAM_BLOCK = old


def test_streamed_adjoint_identity():
    rng = np.random.default_rng(3)
    _, A = _job_ops(p=14, nl=10, nm=10)
    x = rng.standard_normal(A.shape[1])
    U = _herm(rng, A.shape[0])
    lhs = float(np.real(np.vdot(O.psi_apply(A, x), O.vect(U))))
    rhs = float(x @ O.psi_adjoint(A, U))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_streamed_pwls_operator_equals_kronecker_weighting():
    rng = np.random.default_rng(4)
    job, A = _job_ops(p=8, nl=6, nm=5)
    prm = O.Params(cost=O.COST_PWLS)
    bnd = O.bounds(A, None, job.R, job.N, prm)
    prob = O.cost_problem(A, None, job.R, bnd, O.COST_PWLS)
    Linv = np.linalg.inv(np.linalg.cholesky(job.R))
    W = np.kron(Linv.conj(), Linv)                       # explicit Kronecker weighting
    Psi = np.stack([np.kron(A[:, i].conj(), A[:, i]) for i in range(A.shape[1])], axis=1)
    Mref = (W @ Psi) / bnd.D[None, :]
    S = np.array([0, 3, 4, 11, 29])
    v = rng.standard_normal(S.size)
    op = prob.cols(S)
    assert _rel(op.matvec(v), Mref[:, S] @ v) < 1e-12
    u = W @ O.vect(_herm(rng, job.p))
    assert _rel(op.rmatvec(u), np.real(Mref[:, S].conj().T @ u)) < 1e-12
    assert _rel(prob.b, W @ O.vect(job.R)) < 1e-12


def test_streamed_gradient_at_zero_is_minus_the_dirty_images():
    # eq. gls: g(0) = -sigma_MF;  eq. gmvdr: g(0) = -M^H b = -h/D = -C/h = -sigma_MVDR
    job, A = _job_ops(p=10, nl=9, nm=8)
    for cost, bias_c in ((O.COST_LS, 0), (O.COST_PWLS, 0), (O.COST_PWLS, 1)):
        prm = O.Params(cost=cost, bias_c=bias_c)
        bnd = O.bounds(A, None, job.R, job.N, prm)
        prob = O.cost_problem(A, None, job.R, bnd, cost)
        g0 = O.gradient(prob, np.zeros(A.shape[1]))
        # the beamformer outputs, written without the operator identities
        Rinv = np.linalg.inv(job.R)
        mf = np.array([np.real(a.conj() @ job.R @ a) for a in A.T])
        C = job.N / (job.N - job.p) if bias_c else 1.0
        mv = np.array([C / np.real(a.conj() @ Rinv @ a) for a in A.T])
        ref = mf if cost == O.COST_LS else mv
        assert _rel(-g0, ref) < 1e-11


def test_streamed_bounds_equal_explicit():
    job, A = _job_ops(p=12, nl=11, nm=7)
    prm = O.Params()
    b0 = O.bounds(A, O.khatri_rao_psi(A), job.R, job.N, prm)
    b1 = O.bounds(A, None, job.R, job.N, prm)
    for f in ("dirty", "h", "mvdr", "D", "gamma", "eps"):
        assert _rel(getattr(b1, f), getattr(b0, f)) < 1e-13, f


def test_streamed_solve_follows_the_explicit_path():
    for seed, cost, kappa in ((41, O.COST_PWLS, 6.0), (42, O.COST_LS, 6.0), (43, O.COST_PWLS, 0.0)):
        job = synth.custom(seed, 12, 11, 10, 4, 900, radius=4.0, snr_db=0.0)
        prm = O.Params(cost=cost, kappa=kappa, eps_floor=1e-6, feas_tol=1e-5)
        r0 = O.image_job(job, prm)
        r1 = O.image_job(job, prm, streamed=True)
        assert r1.solve.events == r0.solve.events
        np.testing.assert_array_equal(r1.solve.sets, r0.solve.sets)
        assert r1.solve.outer == r0.solve.outer
        assert _rel(r1.solve.sigma, r0.solve.sigma) < 1e-9


def test_streamed_solve_is_the_bounded_ls_optimum():
    # kappa = 0: the exact bounded-LS optimum, independently by BVLS on the
    # real-embedded explicit problem
    for cost in (O.COST_LS, O.COST_PWLS):
        job = synth.custom(44, 9, 5, 4, 3, 2000, radius=3.0, snr_db=5.0)
        prm = O.Params(cost=cost, kappa=0.0, eps_floor=1e-12)
        A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
        bnd = O.bounds(A, None, job.R, job.N, prm)
        prob = O.cost_problem(A, None, job.R, bnd, cost)
        res = O.active_set(prob, bnd.eps, prm)
        assert res.converged
        Psi = O.khatri_rao_psi(A)
        if cost == O.COST_LS:
            M, b = Psi, O.vect(job.R)
        else:
            Linv = np.linalg.inv(np.linalg.cholesky(job.R))
            W = np.kron(Linv.conj(), Linv)
            M, b = (W @ Psi) / bnd.D[None, :], W @ O.vect(job.R)
        Mr = np.vstack([M.real, M.imag])
        br = np.concatenate([b.real, b.imag])
        ref = so.lsq_linear(Mr, br, bounds=(np.zeros(M.shape[1]), prob.upper), method="bvls",
                            tol=1e-14, lsmr_tol=None, max_iter=5000).x
        assert _rel(res.x, ref) < 1e-7
