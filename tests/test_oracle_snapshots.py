"""Pins of the K-snapshot oracle against facts the paper and mathematics fix.

Each check takes a route other than the oracle's own: the block-diagonal
form of the data model, the beamformer definitions with a dense inverse, a
generalised eigenproblem, closed forms for one source (Sherman-Morrison),
dense bounded least squares, brute force over partitions, or Monte Carlo."""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as sopt

import synth
from oracle import imager as O
from oracle import snapshots as S


def _setup(job, prm):
    As = S.steering_stack(job.ant_xyz, job.l, job.m, job.lam)
    Psi = S.khatri_rao_stack(As)
    bnd = S.bounds_k(As, Psi, job.R, job.N, prm)
    return As, Psi, bnd


def _long(As, i):
    """a_i = vect(A^i) = [a_{i,1}; ...; a_{i,K}] (eq. longa)."""
    return np.concatenate([A[:, i] for A in As])


def _ik_circ(As, i):
    """(I_K o A^i): column k holds a_{i,k} in block k, zeros elsewhere."""
    K = len(As)
    p = As[0].shape[0]
    V = np.zeros((K * p, K), dtype=np.complex128)
    for k in range(K):
        V[k * p:(k + 1) * p, k] = As[k][:, i]
    return V


# ---------------------------------------------------------------- data model
def test_stacked_operator_is_the_block_diagonal_model():
    """Psi sigma stacks vect(A_k diag(sigma) A_k^H), and the blocks are those of
    sum_q sigma_q (I_K o A^q)(I_K o A^q)^H (eq. blockdiagtilde)."""
    job = synth.snapshots_custom(3, 5, 3, 3, 2, 300, 3, dtheta=0.4, radius=3.0)
    As = S.steering_stack(job.ant_xyz, job.l, job.m, job.lam)
    Psi = S.khatri_rao_stack(As)
    rng = np.random.default_rng(1)
    sig = rng.random(job.Q)
    big = np.zeros((job.K * job.p, job.K * job.p), dtype=np.complex128)
    for q in range(job.Q):
        V = _ik_circ(As, q)
        big += sig[q] * (V @ V.conj().T)
    p = job.p
    blocks = [big[k * p:(k + 1) * p, k * p:(k + 1) * p] for k in range(job.K)]
    np.testing.assert_allclose(big, sla.block_diag(*blocks), atol=1e-14)
    ref = np.concatenate([b.reshape(-1, order="F") for b in blocks])
    np.testing.assert_allclose(Psi @ sig, ref, rtol=1e-13, atol=1e-13)
    # the snapshots really differ: the array turned between them
    assert np.max(np.abs(As[0] - As[1])) > 0.1


def test_adjoint_identity_stacked():
    job = synth.snapshots_custom(4, 6, 4, 3, 2, 300, 2)
    As = S.steering_stack(job.ant_xyz, job.l, job.m, job.lam)
    Psi = S.khatri_rao_stack(As)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(job.Q)
    Us = []
    for _ in range(job.K):
        X = rng.standard_normal((job.p, job.p)) + 1j * rng.standard_normal((job.p, job.p))
        Us.append(X + X.conj().T)
    u = S.vect_stack(np.stack(Us))
    lhs = np.vdot(Psi @ x, u)
    rhs = float(x @ np.real(Psi.conj().T @ u))
    assert abs(lhs.imag) < 1e-12 * abs(lhs) + 1e-12
    assert abs(lhs.real - rhs) <= 1e-12 * abs(rhs)
    # Psi^H u = sum_k Re diag(A_k^H U_k A_k)   (vectdiag identity, per block)
    ref = sum(np.real(np.diag(As[k].conj().T @ Us[k] @ As[k])) for k in range(job.K))
    np.testing.assert_allclose(np.real(Psi.conj().T @ u), ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- beamformers
def test_mf_and_mvdr_are_beamformer_outputs():
    """MF: w = a_i / sqrt(K), output w^H R w (Sec. III-C, R block-diagonal).
    MVDR: w = sqrt(K) R^{-1} a_i / (a_i^H R^{-1} a_i) (eq. wmvdr), which meets
    w^H a_i = sqrt(K); its output is the MVDR image with C = 1."""
    job = synth.snapshots_custom(6, 7, 5, 4, 3, 800, 3, dtheta=0.3, snr_db=-3.0)
    As, Psi, bnd = _setup(job, O.Params(bias_c=0))
    R = sla.block_diag(*job.R)
    Rinv = np.linalg.inv(R)
    K = job.K
    for i in range(job.Q):
        a = _long(As, i)
        w = a / math.sqrt(K)
        assert abs(np.real(np.vdot(w, R @ w)) - bnd.dirty[i]) <= 1e-12 * bnd.dirty[i]
        w = math.sqrt(K) * (Rinv @ a) / np.real(np.vdot(a, Rinv @ a))
        assert abs(np.vdot(w, a) - math.sqrt(K)) < 1e-10
        assert abs(np.real(np.vdot(w, R @ w)) - bnd.mvdr[i]) <= 1e-10 * bnd.mvdr[i]


def test_assc_is_the_tightest_beamformer_bound():
    """eq. ASSC0: min over w of w^H R w subject to
    w^H (I_K o A^i)(I_K o A^i)^H w = 1 is 1 / lambda_max of the pencil
    (B, R) with B = (I_K o A^i)(I_K o A^i)^H, computed by a dense generalised
    Hermitian eigensolver; it lies below the MVDR and the MF images."""
    job = synth.snapshots_custom(8, 6, 4, 4, 3, 800, 3, dtheta=0.5, snr_db=-3.0)
    As, Psi, bnd = _setup(job, O.Params(bias_c=0))
    R = sla.block_diag(*job.R)
    for i in range(job.Q):
        V = _ik_circ(As, i)
        lam = sla.eigh(V @ V.conj().T, R, eigvals_only=True)
        assert abs(1.0 / lam[-1] - bnd.assc[i]) <= 1e-10 * bnd.assc[i]
    assert np.all(bnd.assc <= bnd.mvdr * (1 + 1e-12))
    assert np.all(bnd.mvdr <= bnd.dirty * (1 + 1e-12))


def test_single_source_closed_forms():
    """True covariances R_k = s a_{i,k} a_{i,k}^H + n I: by Sherman-Morrison,
    a^H R_k^{-1} a = (1 - s c_k / (n + s)) / n with c_k = |a_{j,k}^H a_{i,k}|^2.
    At the source pixel MF = MVDR = ASSC = s + n; elsewhere
    MF_j = mean_k(s c_k) + n, MVDR_j = 1 / mean_k(h_k), ASSC_j = 1 / max_k h_k."""
    K, p, n_l, n_m = 3, 9, 6, 5
    job = synth.snapshots_custom(12, p, n_l, n_m, 0, 1000, K, dtheta=0.6, radius=4.0)
    As = S.steering_stack(job.ant_xyz, job.l, job.m, job.lam)
    Psi = S.khatri_rao_stack(As)
    i, s, n = 7, 4.0, 0.5
    Rs = np.stack([s * np.outer(As[k][:, i], As[k][:, i].conj()) + n * np.eye(p)
                   for k in range(K)])
    bnd = S.bounds_k(As, Psi, Rs, 1000, O.Params(bias_c=0))
    for j in range(job.Q):
        c = np.array([abs(np.vdot(As[k][:, j], As[k][:, i])) ** 2 for k in range(K)])
        h = (1.0 - s * c / (n + s)) / n
        np.testing.assert_allclose(bnd.dirty[j], np.mean(s * c) + n, rtol=1e-12)
        np.testing.assert_allclose(bnd.mvdr[j], 1.0 / np.mean(h), rtol=1e-11)
        np.testing.assert_allclose(bnd.assc[j], 1.0 / np.max(h), rtol=1e-11)
    for v in (bnd.dirty[i], bnd.mvdr[i], bnd.assc[i]):
        assert abs(v - (s + n)) < 1e-11
    # D_ii = (sum_k h)^2 / K with C = 1 (eq. D)
    h_i = np.full(K, 1.0 / (s + n))
    assert abs(bnd.D[i] - h_i.sum() ** 2 / K) < 1e-12


def test_one_snapshot_reduces_to_the_single_snapshot_oracle():
    job = synth.custom(14, 7, 5, 4, 3, 500, radius=3.0)
    for bias_c in (0, 1):
        for bound in (O.BOUND_MF, O.BOUND_MVDR):
            prm = O.Params(bias_c=bias_c, bound=bound, inflate=O.INFLATE_STD)
            A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
            ref = O.bounds(A, O.khatri_rao_psi(A), job.R, job.N, prm)
            As = [A]
            got = S.bounds_k(As, S.khatri_rao_stack(As), job.R[None], job.N, prm)
            for f in ("dirty", "mvdr", "D", "std_mf", "std_mvdr", "gamma", "eps"):
                np.testing.assert_allclose(getattr(got, f), getattr(ref, f), rtol=1e-13)
            np.testing.assert_allclose(got.assc, ref.mvdr, rtol=1e-13)


# ---------------------------------------------------------------- costs
@pytest.mark.parametrize("cost", [O.COST_LS, O.COST_PWLS])
def test_gradient_at_zero_is_minus_dirty_image(cost):
    """From sigma = 0 the CLS gradient is minus the MF image (the 1/(2K)
    scaling of eq. CLS) and the PWLS gradient is minus the MVDR image (the WLS
    dirty image is the MVDR image, Sec. III-E)."""
    job = synth.snapshots_custom(15, 8, 5, 5, 3, 900, 2, dtheta=0.4)
    prm = O.Params(cost=cost, bias_c=1)
    As, Psi, bnd = _setup(job, prm)
    prob = S.cost_problem_k(As, Psi, job.R, bnd, cost)
    g = O.gradient(prob, np.zeros(job.Q))
    ref = bnd.dirty if cost == O.COST_LS else bnd.mvdr
    np.testing.assert_allclose(-g, ref, rtol=1e-11)


def test_pwls_operator_is_blockwise_whitened_psi():
    """Block k of M equals (R_k^{-T/2} kron R_k^{-1/2}) (conj(A_k) o A_k) D^{-1}
    up to a unitary factor per block: compare Gram matrices M^H M, built with
    the Hermitian inverse square roots and explicit Kronecker products."""
    job = synth.snapshots_custom(16, 5, 3, 4, 2, 600, 2, dtheta=0.3, radius=3.0)
    prm = O.Params(cost=O.COST_PWLS)
    As, Psi, bnd = _setup(job, prm)
    prob = S.cost_problem_k(As, Psi, job.R, bnd, O.COST_PWLS)
    G = np.zeros((job.Q, job.Q), dtype=np.complex128)
    bw = []
    for k in range(job.K):
        Ri = sla.fractional_matrix_power(job.R[k], -0.5)
        W = np.kron(Ri.T, Ri)
        Mk = W @ O.khatri_rao_psi(As[k]) / bnd.D[None, :]
        G += Mk.conj().T @ Mk
        bw.append(W @ O.vect(job.R[k]))
    np.testing.assert_allclose(prob.M.conj().T @ prob.M, G, rtol=1e-9, atol=1e-9 * np.abs(G).max())
    bw = np.concatenate(bw)
    # M^H b agrees too (the data side of the whitening)
    Mfull = np.concatenate([np.kron(sla.fractional_matrix_power(job.R[k], -0.5).T,
                                    sla.fractional_matrix_power(job.R[k], -0.5))
                            @ O.khatri_rao_psi(As[k]) for k in range(job.K)]) / bnd.D[None, :]
    np.testing.assert_allclose(prob.M.conj().T @ prob.b, Mfull.conj().T @ bw, rtol=1e-9,
                               atol=1e-9 * np.abs(Mfull.conj().T @ bw).max())


def _embed(M, b):
    return np.vstack([M.real, M.imag]), np.concatenate([b.real, b.imag])


@pytest.mark.parametrize("cost", [O.COST_LS, O.COST_PWLS])
@pytest.mark.parametrize("bound", [O.BOUND_MVDR, S.BOUND_ASSC])
def test_exact_solve_matches_dense_bvls(cost, bound):
    job = synth.snapshots_custom(40 + cost, 8, 7, 6, 3, 500, 2, dtheta=0.4, radius=2.0,
                                 snr_db=3.0)
    prm = O.Params(cost=cost, bound=bound, kappa=0.0, eps_floor=1e-11)
    As, Psi, bnd = _setup(job, prm)
    prob = S.cost_problem_k(As, Psi, job.R, bnd, cost)
    res = O.active_set(prob, bnd.eps, prm)
    assert res.converged
    Mr, br = _embed(prob.M, prob.b)
    ref = sopt.lsq_linear(Mr, br, bounds=(np.zeros(job.Q), prob.upper), method="bvls",
                          tol=1e-15, max_iter=10000).x
    np.testing.assert_allclose(res.x, ref, rtol=1e-6, atol=1e-8 * np.max(prob.upper))


@pytest.mark.parametrize("cost", [O.COST_LS, O.COST_PWLS])
def test_exact_solve_matches_brute_force_partitions(cost):
    job = synth.snapshots_custom(51, 4, 3, 2, 2, 300, 2, dtheta=0.5, radius=1.5)
    prm = O.Params(cost=cost, kappa=0.0, eps_floor=1e-11)
    As, Psi, bnd = _setup(job, prm)
    prob = S.cost_problem_k(As, Psi, job.R, bnd, cost)
    Mr, br = _embed(prob.M, prob.b)
    Q = Mr.shape[1]
    assert np.linalg.matrix_rank(Mr) == Q
    best = None
    for labels in itertools.product(range(3), repeat=Q):
        lab = np.array(labels)
        x = np.where(lab == O.SET_U, prob.upper, 0.0)
        F = np.nonzero(lab == O.SET_F)[0]
        if F.size:
            x[F] = np.linalg.lstsq(Mr[:, F], br - Mr @ x, rcond=None)[0]
        if np.any(x < -1e-12) or np.any(x > prob.upper + 1e-12):
            continue
        g = Mr.T @ (Mr @ x - br)
        if (np.all(np.abs(g[F]) < 1e-9) and np.all(g[lab == O.SET_L] >= -1e-9)
                and np.all(g[lab == O.SET_U] <= 1e-9)):
            best = x
            break
    assert best is not None
    res = O.active_set(prob, bnd.eps, prm)
    assert res.converged
    np.testing.assert_allclose(res.x, best, rtol=1e-7, atol=1e-10)


@pytest.mark.parametrize("cost", [O.COST_LS, O.COST_PWLS])
def test_repeated_snapshot_gives_the_single_snapshot_optimum(cost):
    """K copies of one snapshot scale the CLS cost by nothing and the PWLS cost
    by K, and leave the MVDR bound and the image unchanged (kappa = 0)."""
    job = synth.custom(61, 7, 6, 5, 3, 700, radius=3.0, snr_db=3.0)
    prm = O.Params(cost=cost, kappa=0.0, eps_floor=1e-11)
    ref = O.image_job(job, prm)
    K = 3
    got = S.image_k(np.stack([job.ant_xyz] * K), job.l, job.m, job.lam,
                    np.stack([job.R] * K), job.N, prm)
    assert got.solve.converged and ref.solve.converged
    np.testing.assert_allclose(got.bounds.mvdr, ref.bounds.mvdr, rtol=1e-12)
    np.testing.assert_allclose(got.solve.sigma, ref.solve.sigma, rtol=1e-6,
                               atol=1e-9 * np.max(ref.solve.sigma))


def test_kappa_solution_detects_the_sources():
    """kappa = 6 on a two-snapshot job with strong on-grid sources: every
    freed pixel passes the relaxed KKT test and the brightest true source
    is freed first (argmax of the MVDR image)."""
    job = synth.snapshots_custom(71, 12, 10, 10, 3, 5000, 2, dtheta=0.3, radius=6.0,
                                 snr_db=5.0)
    prm = O.Params(cost=O.COST_PWLS)
    res = S.image_snapshot_job(job, prm)
    assert res.solve.converged
    assert res.solve.events[0] == ("free", int(np.argmax(res.bounds.mvdr)))
    assert np.all(res.solve.sigma >= 0)
    assert np.all(res.solve.sigma <= res.bounds.gamma * (1 + 1e-12))
    assert int(np.argmax(res.solve.sigma)) == int(np.argmax(job.sigma_true))


def test_assc_with_std_inflation_is_rejected():
    job = synth.snapshots_custom(3, 5, 3, 3, 1, 300, 2)
    with pytest.raises(ValueError):
        _setup(job, O.Params(bound=S.BOUND_ASSC, inflate=O.INFLATE_STD))


# ---------------------------------------------------------------- statistics
def test_monte_carlo_k_snapshot_variances():
    """Appendix A for K = 2 independent snapshots: the MF image has variance
    (1/(N K^2)) sum_k (a_k^H R_k a_k)^2; the bias-corrected MVDR image is
    unbiased to first order with variance
    K^2 sum_k h_k^2 / ((N-p-1) (sum_k h_k)^4), h_k = a_k^H R_k^{-1} a_k."""
    rng = np.random.default_rng(91)
    p, N, T, K = 4, 400, 2500, 2
    Rt, Lt, a = [], [], []
    for k in range(K):
        X = rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p))
        Rk = X @ X.conj().T / p + (1.0 + k) * np.eye(p)
        Rt.append(Rk)
        Lt.append(np.linalg.cholesky(Rk))
        a.append(np.exp(-2j * np.pi * rng.random(p)) / math.sqrt(p))
    As = [ak[:, None] for ak in a]
    Psi = S.khatri_rao_stack(As)
    mv, mf, std_mv, std_mf = [], [], [], []
    for _ in range(T):
        Rh = []
        for k in range(K):
            G = (rng.standard_normal((p, N)) + 1j * rng.standard_normal((p, N))) / math.sqrt(2)
            Y = Lt[k] @ G
            Rh.append(Y @ Y.conj().T / N)
        bnd = S.bounds_k(As, Psi, np.stack(Rh), N, O.Params(bias_c=1))
        mv.append(bnd.mvdr[0])
        mf.append(bnd.dirty[0])
        std_mv.append(bnd.std_mvdr[0])
        std_mf.append(bnd.std_mf[0])
    mv, mf = np.array(mv), np.array(mf)
    h = np.array([np.real(np.vdot(a[k], np.linalg.solve(Rt[k], a[k]))) for k in range(K)])
    s = np.array([np.real(np.vdot(a[k], Rt[k] @ a[k])) for k in range(K)])
    true_mv = K / h.sum()
    true_mf = s.mean()
    assert abs(mv.mean() / true_mv - 1.0) < 0.004
    assert abs(mf.mean() / true_mf - 1.0) < 0.005
    sd_mf = math.sqrt(np.sum(s * s) / (N * K * K))
    sd_mv = math.sqrt(K * K * np.sum(h * h) / ((N - p - 1) * h.sum() ** 4))
    assert abs(mf.std() / sd_mf - 1.0) < 0.07
    assert abs(mv.std() / sd_mv - 1.0) < 0.07
    # the per-draw estimates scatter around the same values
    assert abs(np.mean(std_mf) / sd_mf - 1.0) < 0.02
    assert abs(np.mean(std_mv) / sd_mv - 1.0) < 0.03


def test_mvdr_alpha_and_upper_bound_chain_with_true_covariances():
    """Sec. III-D (eq. MVDRUB2): alpha = w^H (I_K o A^i)(I_K o A^i)^H w >= 1 for
    the MVDR beamformer, computed with dense matrices and equal to
    K sum_k h_k^2 / (sum_k h_k)^2; hence with the true covariances
    R_k = sum_q s_q a_{q,k} a_{q,k}^H + n I every bound sits above the true
    sky: sigma <= ASSC <= MVDR <= MF at every pixel (C = 1)."""
    K, p, n_l, n_m = 3, 8, 7, 6
    job = synth.snapshots_custom(95, p, n_l, n_m, 4, 1000, K, dtheta=0.4, radius=5.0)
    As = S.steering_stack(job.ant_xyz, job.l, job.m, job.lam)
    Psi = S.khatri_rao_stack(As)
    s = job.sigma_true
    Rt = np.stack([(As[k] * s[None, :]) @ As[k].conj().T + job.noise_var * np.eye(p) for k in range(K)])
    bnd = S.bounds_k(As, Psi, Rt, 1000, O.Params(bias_c=0))
    R = sla.block_diag(*Rt)
    Rinv = np.linalg.inv(R)
    for i in range(job.Q):
        a = _long(As, i)
        w = math.sqrt(K) * (Rinv @ a) / np.real(np.vdot(a, Rinv @ a))
        V = _ik_circ(As, i)
        alpha = float(np.real(np.vdot(w, V @ (V.conj().T @ w))))
        h = bnd.hk[:, i]
        assert alpha >= 1.0 - 1e-12
        assert abs(alpha - K * np.sum(h * h) / np.sum(h) ** 2) <= 1e-10 * alpha
    tol = 1e-12 * np.max(bnd.dirty)
    assert np.all(s <= bnd.assc + tol)
    assert np.all(bnd.assc <= bnd.mvdr + tol)
    assert np.all(bnd.mvdr <= bnd.dirty + tol)
    # the bounds are not slack everywhere: at a source pixel the MVDR bound is close
    i = int(np.argmax(s))
    assert bnd.mvdr[i] < 1.5 * s[i] + job.noise_var


def test_stored_k_snapshot_bounds_record_is_the_oracle_output():
    """tests/golden/snapshots_extended_bounds.npz (written by
    tests/golden/make_golden.py) holds the seeded stand-in for the paper's
    extended-source simulation and the oracle's K-snapshot MF, MVDR and
    ASSC images for it; recomputing them from the stored inputs reproduces
    the stored values."""
    import os
    z = np.load(os.path.join(os.path.dirname(__file__), "golden", "snapshots_extended_bounds.npz"))
    As = S.steering_stack(z["ant_xyz"], z["l"], z["m"], float(z["lam"]))
    bnd = S.bounds_k(As, S.khatri_rao_stack(As), z["R"], int(z["N"]), O.Params(bias_c=int(z["bias_c"])))
    for key in ("dirty", "mvdr", "assc"):
        np.testing.assert_allclose(getattr(bnd, key), z[key], rtol=1e-12)
    job = synth.snapshots_extended()
    np.testing.assert_allclose(job.R, z["R"], rtol=0, atol=1e-12 * np.abs(z["R"]).max())   # the recipe's inputs


def test_stored_k_snapshot_solve_record_is_a_relaxed_kkt_point():
    """tests/golden/snapshots_mid_pwls.npz (K = 2, p = 48, 48x48, PWLS,
    kappa = 6): the stored bounds are the oracle's for the stored inputs, and
    the stored image satisfies what Table I guarantees at its exit - feasible
    (0 <= sigma <= gamma), the free-set gradient near zero and every active
    pixel's multiplier above -eps (Sec. IV-C)."""
    import os
    z = np.load(os.path.join(os.path.dirname(__file__), "golden", "snapshots_mid_pwls.npz"))
    prm = O.Params(cost=int(z["cost"]), kappa=float(z["kappa"]), eps_floor=float(z["eps_floor"]),
                   feas_tol=float(z["feas_tol"]))
    As = S.steering_stack(z["ant_xyz"], z["l"], z["m"], float(z["lam"]))
    Psi = S.khatri_rao_stack(As)
    bnd = S.bounds_k(As, Psi, z["R"], int(z["N"]), prm)
    for key in ("dirty", "mvdr", "assc", "gamma"):
        np.testing.assert_allclose(getattr(bnd, key), z[key], rtol=1e-12)
    assert bool(z["converged"])
    prob = S.cost_problem_k(As, Psi, z["R"], bnd, prm.cost)
    sigma, sets = z["sigma"], z["sets"]
    assert np.all(sigma >= 0) and np.all(sigma <= bnd.gamma * (1 + 1e-12))
    x = sigma / prob.to_sigma
    g = O.gradient(prob, x)
    lam = np.where(sets == O.SET_U, -g, g)
    act = sets != O.SET_F
    assert np.all(lam[act] >= -bnd.eps[act] * (1 + 1e-9))
    F = sets == O.SET_F
    assert np.max(np.abs(g[F])) <= 1e-5 * np.max(np.abs(bnd.mvdr))
    assert int(F.sum()) == int(np.sum(z["events"][:, 0] == 0)) - int(np.sum(z["events"][:, 0] == 1))
