"""Pins of the FP64 oracle against facts the paper and mathematics fix.

None of these re-types an oracle formula: each checks it through a different
route (a matrix identity, a library routine, a closed form, brute force or
Monte Carlo statistics)."""
import itertools
import math

import numpy as np
import pytest
import scipy.optimize as sopt

import synth
from oracle import imager as O


def _job(seed=11, p=6, n_l=4, n_m=3, n_src=2, N=500, snr_db=0.0):
    return synth.custom(seed, p, n_l, n_m, n_src, N, radius=3.0, snr_db=snr_db)


# ---------------------------------------------------------------- steering
def test_steering_unit_norm_and_closed_form():
    ant = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 0.0], [2.0, 0.5, 0.0]])
    l = np.array([-0.25, 0.0, 0.25])
    m = np.array([0.0, 0.5])
    A = O.steering_matrix(ant, l, m, 1.0)
    assert A.shape == (4, 6)
    np.testing.assert_allclose(np.linalg.norm(A, axis=0), 1.0, rtol=0, atol=1e-15)
    # pixel i = i_l + n_l i_m: i = 2 is (l=0.25, m=0): antenna (1,0,0) sees exp(-j pi/2) = -j
    assert abs(A[0, 2] - (-1j) / 2.0) < 1e-15
    # antenna (0,1,0) depends on m only: pixel 4 = (l=0, m=0.5) -> exp(-j pi) = -1
    assert abs(A[1, 4] - (-1.0) / 2.0) < 1e-15
    assert abs(A[1, 3] - A[1, 5]) < 1e-15            # same m row
    # antenna at the origin is phase-free
    np.testing.assert_allclose(A[2], 0.5, atol=1e-15)
    # wavelength scales phase: (2, 0.5) at (0.25, 0.5) with lam=2 -> -2pi(0.5+0.25)/2
    A2 = O.steering_matrix(ant, l, m, 2.0)
    assert abs(A2[3, 5] - np.exp(-1j * 2 * np.pi * 0.75 / 2.0) / 2.0) < 1e-15


def test_steering_w_term():
    ant = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 0.0]])
    l = np.array([0.6])
    m = np.array([0.0])
    A = O.steering_matrix(ant, l, m, 1.0)
    assert abs(A[0, 0] - np.exp(-2j * np.pi * 0.8) / math.sqrt(2)) < 1e-15


# ---------------------------------------------------------------- Khatri-Rao
def test_khatri_rao_properties():
    rng = np.random.default_rng(0)
    p, Q = 5, 7
    A = rng.standard_normal((p, Q)) + 1j * rng.standard_normal((p, Q))
    Psi = O.khatri_rao_psi(A)
    x = rng.standard_normal(Q)
    # (B^T o A) x = vect(A diag(x) B) with B = A^H
    np.testing.assert_allclose(Psi @ x, (A @ np.diag(x) @ A.conj().T).reshape(-1, order="F"),
                               rtol=1e-13, atol=1e-13)
    # vectdiag(A^H X A) = (conj(A) o A)^H vect(X)
    X = rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p))
    np.testing.assert_allclose(Psi.conj().T @ X.reshape(-1, order="F"),
                               np.diag(A.conj().T @ X @ A), rtol=1e-13, atol=1e-13)


def test_adjoint_identity():
    job = _job(p=8, n_l=5, n_m=5)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(job.Q)
    Y = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    Y = Y + Y.conj().T
    y = O.vect(Y)
    lhs = np.real(np.vdot(Psi @ x, y))
    rhs = float(x @ np.real(Psi.conj().T @ y))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


# ---------------------------------------------------------------- dirty / MVDR
def test_dirty_is_beamformer_output():
    job = _job(p=7, n_l=6, n_m=4, n_src=3)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    d = O.dirty_mf(Psi, job.R)
    for i in range(job.Q):
        a = A[:, i]
        assert abs(d[i] - np.real(a.conj() @ job.R @ a)) < 1e-12 * abs(d[i])
    assert np.all(d > 0)


def test_mvdr_bound_chain_and_inverse():
    job = _job(p=8, n_l=7, n_m=5, n_src=3)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    b = O.bounds(A, Psi, job.R, job.N, O.Params(bias_c=0))
    Rinv = np.linalg.inv(job.R)
    h_ref = np.real(np.einsum("ki,kl,li->i", A.conj(), Rinv, A))
    np.testing.assert_allclose(b.h, h_ref, rtol=1e-12)
    # 0 <= sigma_MVDR <= sigma_MF (Cauchy-Schwarz, Sec. III-D)
    assert np.all(b.mvdr > 0)
    assert np.all(b.mvdr <= b.dirty * (1 + 1e-12))
    # bias constant and D (eq. D, K=1)
    b2 = O.bounds(A, Psi, job.R, job.N, O.Params(bias_c=1))
    assert b2.C == pytest.approx(job.N / (job.N - 8))
    np.testing.assert_allclose(b2.mvdr, b.mvdr * b2.C, rtol=1e-14)
    np.testing.assert_allclose(b2.D, b.h ** 2 / b2.C, rtol=1e-14)


def test_mvdr_equals_jacobi_preconditioned_wls_dirty_image():
    """Sec. III-B: for K = 1, D_WLS^{-1} sigma_WLS equals the MVDR dirty image."""
    job = _job(p=6, n_l=4, n_m=4, n_src=2)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    Rinv = np.linalg.inv(job.R)
    G = np.kron(Rinv.T, Rinv)
    s_wls = np.real(Psi.conj().T @ G @ O.vect(job.R))
    H_wls = np.real(Psi.conj().T @ G @ Psi)
    b = O.bounds(A, Psi, job.R, job.N, O.Params())
    np.testing.assert_allclose(s_wls / np.diag(H_wls), b.mvdr, rtol=1e-10)
    np.testing.assert_allclose(np.diag(H_wls), b.D, rtol=1e-10)


def test_pwls_operator_is_whitened_khatri_rao():
    job = _job(p=5, n_l=3, n_m=4, n_src=2)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    b = O.bounds(A, Psi, job.R, job.N, O.Params())
    prob = O.cost_problem(A, Psi, job.R, b, O.COST_PWLS)
    Linv = np.linalg.inv(np.linalg.cholesky(job.R))
    W = np.kron(Linv.conj(), Linv)
    np.testing.assert_allclose(prob.M, W @ Psi @ np.diag(1.0 / b.D), rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(prob.b, W @ O.vect(job.R), rtol=1e-10, atol=1e-13)
    Rinv = np.linalg.inv(job.R)
    np.testing.assert_allclose(W.conj().T @ W, np.kron(Rinv.T, Rinv), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(prob.upper, b.D * b.gamma, rtol=1e-15)


@pytest.mark.parametrize("cost", [O.COST_LS, O.COST_PWLS])
def test_gradient_at_zero_is_minus_dirty(cost):
    """eq. gls / eq. gmvdr at sigma = 0 give the negated MF / MVDR dirty image."""
    job = _job(p=7, n_l=5, n_m=4, n_src=3)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    b = O.bounds(A, Psi, job.R, job.N, O.Params(cost=cost, bias_c=1))
    prob = O.cost_problem(A, Psi, job.R, b, cost)
    g = O.gradient(prob, np.zeros(job.Q))
    ref = b.dirty if cost == O.COST_LS else b.mvdr
    np.testing.assert_allclose(g, -ref, rtol=1e-10)


# ---------------------------------------------------------------- LSQR
def _embed(M, b):
    return np.vstack([M.real, M.imag]), np.concatenate([b.real, b.imag])


def test_lsqr_matches_lstsq_full_rank():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((40, 9)) + 1j * rng.standard_normal((40, 9))
    b = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    res = O.lsqr(M, b, 1e-14, 1e-14, 200)
    Mr, br = _embed(M, b)
    ref = np.linalg.lstsq(Mr, br, rcond=None)[0]
    np.testing.assert_allclose(res.x, ref, rtol=1e-9, atol=1e-11)
    assert res.istop in (1, 2)


def test_lsqr_min_norm_on_rank_deficient():
    rng = np.random.default_rng(6)
    B = rng.standard_normal((30, 4)) + 1j * rng.standard_normal((30, 4))
    C = rng.standard_normal((4, 8))
    M = B @ C                                  # rank 4 (real coefficient mixing)
    b = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    res = O.lsqr(M, b, 1e-14, 1e-14, 400)
    Mr, br = _embed(M, b)
    ref = np.linalg.pinv(Mr) @ br
    np.testing.assert_allclose(res.x, ref, rtol=1e-7, atol=1e-9)


def test_lsqr_zero_rhs_and_empty():
    M = np.ones((4, 2), dtype=complex)
    assert np.all(O.lsqr(M, np.zeros(4, complex), 1e-12, 1e-12, 10).x == 0)
    assert O.lsqr(np.zeros((4, 0), complex), np.ones(4, complex), 1e-12, 1e-12, 10).x.size == 0


# ---------------------------------------------------------------- active set
def _problem(job, cost, prm):
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    bnd = O.bounds(A, Psi, job.R, job.N, prm)
    return bnd, O.cost_problem(A, Psi, job.R, bnd, cost)


@pytest.mark.parametrize("cost", [O.COST_LS, O.COST_PWLS])
def test_first_free_pixel_is_dirty_argmax(cost):
    """Sec. IV-C: from sigma = 0 the first pixel freed is the dirty-image peak."""
    job = synth.tiny()
    prm = O.Params(cost=cost, max_outer=2)
    bnd, prob = _problem(job, cost, prm)
    res = O.active_set(prob, bnd.eps, prm)
    ref = bnd.dirty if cost == O.COST_LS else bnd.mvdr
    assert res.events[0] == ("free", int(np.argmax(ref)))


def _kkt_ok(prob, res, tol):
    g = O.gradient(prob, res.x)
    F = res.sets == O.SET_F
    L = res.sets == O.SET_L
    U = res.sets == O.SET_U
    scale = np.max(np.abs(O.gradient(prob, np.zeros_like(res.x))))
    assert np.all(np.abs(g[F]) <= tol * scale)
    assert np.all(g[L] >= -tol * scale)
    assert np.all(-g[U] >= -tol * scale)
    assert np.all(res.x >= -1e-12) and np.all(res.x <= prob.upper * (1 + 1e-12))


def _bvls(prob):
    Mr, br = _embed(prob.M, prob.b)
    return sopt.lsq_linear(Mr, br, bounds=(np.zeros(prob.M.shape[1]), prob.upper),
                           method="bvls", tol=1e-15, max_iter=10000).x


@pytest.mark.parametrize("cost", [O.COST_LS, O.COST_PWLS])
@pytest.mark.parametrize("seed", [21, 22, 23])
def test_exact_solve_matches_dense_bvls(cost, seed):
    job = synth.custom(seed, 9, 8, 8, 3, 400, radius=2.0, snr_db=3.0)
    prm = O.Params(cost=cost, kappa=0.0, eps_floor=1e-11)
    bnd, prob = _problem(job, cost, prm)
    res = O.active_set(prob, bnd.eps, prm)
    assert res.converged
    _kkt_ok(prob, res, 1e-8)
    ref = _bvls(prob)
    np.testing.assert_allclose(res.x, ref, rtol=1e-6, atol=1e-8 * np.max(prob.upper))


@pytest.mark.parametrize("cost", [O.COST_LS, O.COST_PWLS])
def test_exact_solve_matches_brute_force_partitions(cost):
    """Enumerate all 3^Q (L, U, F) partitions; the optimum is the unique
    feasible KKT point (strictly convex for full column rank)."""
    job = synth.custom(31, 4, 3, 2, 2, 300, radius=1.5, snr_db=0.0)
    prm = O.Params(cost=cost, kappa=0.0, eps_floor=1e-11, bound=O.BOUND_MVDR)
    bnd, prob = _problem(job, cost, prm)
    Mr, br = _embed(prob.M, prob.b)
    Q = Mr.shape[1]
    assert np.linalg.matrix_rank(Mr) == Q
    best = None
    for labels in itertools.product(range(3), repeat=Q):
        lab = np.array(labels)
        x = np.where(lab == O.SET_U, prob.upper, 0.0)
        F = np.nonzero(lab == O.SET_F)[0]
        if F.size:
            rhs = br - Mr @ x
            x[F] = np.linalg.lstsq(Mr[:, F], rhs, rcond=None)[0]
        if np.any(x < -1e-12) or np.any(x > prob.upper + 1e-12):
            continue
        g = Mr.T @ (Mr @ x - br)
        ok = (np.all(np.abs(g[F]) < 1e-9) and np.all(g[lab == O.SET_L] >= -1e-9)
              and np.all(g[lab == O.SET_U] <= 1e-9))
        if ok:
            best = x
            break
    assert best is not None
    res = O.active_set(prob, bnd.eps, prm)
    assert res.converged
    np.testing.assert_allclose(res.x, best, rtol=1e-7, atol=1e-10)


def test_kappa_solution_is_relaxed_kkt_and_feasible():
    job = synth.tiny()
    for cost in (O.COST_LS, O.COST_PWLS):
        prm = O.Params(cost=cost)
        bnd, prob = _problem(job, cost, prm)
        res = O.active_set(prob, bnd.eps, prm)
        assert res.converged
        g = O.gradient(prob, res.x)
        lam = np.where(res.sets == O.SET_U, -g, g)
        act = res.sets != O.SET_F
        assert np.all(lam[act] >= -bnd.eps[act])
        assert np.all(res.x >= 0) and np.all(res.x <= prob.upper)
        F = res.sets == O.SET_F
        assert np.max(np.abs(g[F])) <= 1e-6 * np.max(np.abs(bnd.dirty))
        assert np.all(res.sigma <= bnd.gamma * (1 + 1e-12))


# ---------------------------------------------------------------- statistics
def test_monte_carlo_bias_and_variances():
    """Appendix A: with E{R_hat^-1} = N/(N-p) R^-1 the scaled C/h is unbiased to
    first order; Var(sigma_MF) = (a^H R a)^2/N; Var(sigma_MVDR) ~ sigma^2/(N-p-1).
    The exact complex-Wishart mean of 1/(a^H R_hat^-1 a) is (N-p+1)/N times
    1/(a^H R^-1 a), which the first-order constant C = N/(N-p) matches to
    1/(N-p); N is chosen so that residual is well inside the tolerance."""
    rng = np.random.default_rng(77)
    p, N, T = 4, 400, 3000
    X = rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p))
    R = X @ X.conj().T / p + np.eye(p)
    a = np.exp(-2j * np.pi * rng.random(p)) / math.sqrt(p)
    Lr = np.linalg.cholesky(R)
    A = a[:, None]
    Psi = O.khatri_rao_psi(A)
    mv, mv1, mf = [], [], []
    for _ in range(T):
        G = (rng.standard_normal((p, N)) + 1j * rng.standard_normal((p, N))) / math.sqrt(2)
        Y = Lr @ G
        Rh = Y @ Y.conj().T / N
        bnd = O.bounds(A, Psi, Rh, N, O.Params(bias_c=1))
        mv.append(bnd.mvdr[0])
        mv1.append(O.bounds(A, Psi, Rh, N, O.Params(bias_c=0)).mvdr[0])
        mf.append(bnd.dirty[0])
    mv, mv1, mf = np.array(mv), np.array(mv1), np.array(mf)
    true_mv = 1.0 / np.real(a.conj() @ np.linalg.solve(R, a))
    true_mf = np.real(a.conj() @ R @ a)
    assert abs(mv.mean() / true_mv - 1.0) < 0.003
    assert abs(mv1.mean() / true_mv - (N - p + 1) / N) < 0.003      # C = 1 is biased low
    assert abs(mf.mean() / true_mf - 1.0) < 0.005
    assert abs(mf.std() / (true_mf / math.sqrt(N)) - 1.0) < 0.06
    assert abs(mv.std() / (true_mv / math.sqrt(N - p - 1)) - 1.0) < 0.06


# ---------------------------------------------------------------- degenerate cases
@pytest.mark.parametrize("cost", [O.COST_LS, O.COST_PWLS])
@pytest.mark.parametrize("bound", [O.BOUND_MF, O.BOUND_MVDR])
def test_single_pixel_closed_form(cost, bound):
    """Q = 1: the bounded problem is a scalar least squares clipped to
    [0, gamma].  With ||a|| = 1 the CLS minimiser is a^H R a (the dirty image)
    and the WLS minimiser is 1 / (a^H R^-1 a) (the MVDR image, C = 1); both
    exceed or equal the MVDR bound, so with that bound the image is the bound,
    and with the MF bound it is the unclipped minimiser."""
    job = synth.custom(81, 5, 1, 1, 1, 400, radius=2.0)
    a = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)[:, 0]
    d = float(np.real(a.conj() @ job.R @ a))
    mv = 1.0 / float(np.real(a.conj() @ np.linalg.solve(job.R, a)))
    prm = O.Params(cost=cost, bound=bound, kappa=0.0, eps_floor=1e-12, feas_tol=1e-9)
    res = O.image_job(job, prm)
    assert res.solve.converged
    if bound == O.BOUND_MVDR:
        expect = mv
    else:
        expect = d if cost == O.COST_LS else mv
    assert abs(res.solve.sigma[0] - expect) <= 1e-9 * expect
    assert res.solve.events[0] == ("free", 0)


def test_two_antenna_array():
    """p = 2, the smallest array: the bounds and an exact solve agree with
    dense BVLS on the explicit operator."""
    job = synth.custom(82, 2, 3, 2, 1, 300, radius=1.0, snr_db=5.0)
    for cost in (O.COST_LS, O.COST_PWLS):
        prm = O.Params(cost=cost, kappa=0.0, eps_floor=1e-11)
        bnd, prob = _problem(job, cost, prm)
        assert np.all(bnd.mvdr <= bnd.dirty * (1 + 1e-12))
        res = O.active_set(prob, bnd.eps, prm)
        assert res.converged
        _kkt_ok(prob, res, 1e-8)
