"""K = 1 pins of the two upper-bound inflations of the oracle's bounds():
gamma = (1 + alpha) sigma_hat (Sec. III-D) and gamma = sigma_hat + alpha std
(Appendix A), for the matched-filter and the MVDR bound.

Independent routes: a one-source sky with the true covariance
R = s a0 a0^H + s2 I, whose MF and MVDR images follow in closed form from the
Sherman-Morrison formula (no Cholesky, no operator), and a Monte Carlo of the
sample covariance, where the inflated bound must cover the true image with
the probability a Gaussian error of the stated standard deviation gives
(Phi(2) = 0.977 for alpha = 2)."""
import math

import numpy as np

import synth
from oracle import imager as O


def _one_source(p=8, n=9, s=4.0, s2=1.0, seed=3):
    rng = np.random.default_rng(seed)
    ant = synth.disk_layout(p, 3.0, rng)
    l = m = synth.grid(n)
    A = O.steering_matrix(ant, l, m, 1.0)
    i0 = (n * n) // 2 + 1
    a0 = A[:, i0]
    R = s * np.outer(a0, a0.conj()) + s2 * np.eye(p)
    return A, R, i0, s, s2


def _closed_forms(A, i0, s, s2):
    """MF and MVDR images at the true R by Sherman-Morrison (unit-norm a):
    a^H R a = s |rho|^2 + s2,  a^H R^-1 a = (1 - s |rho|^2 / (s2 + s)) / s2."""
    rho2 = np.abs(A[:, i0].conj() @ A) ** 2
    mf = s * rho2 + s2
    mvdr = s2 * (s2 + s) / (s2 + s - s * rho2)
    return mf, mvdr


def test_ratio_inflation_equals_the_closed_form():
    A, R, i0, s, s2 = _one_source()
    mf, mvdr = _closed_forms(A, i0, s, s2)
    alpha = 0.37
    for bound, ref in ((O.BOUND_MF, mf), (O.BOUND_MVDR, mvdr)):
        prm = O.Params(bound=bound, inflate=O.INFLATE_RATIO, alpha=alpha)
        b = O.bounds(A, None, R, 1000, prm)
        np.testing.assert_allclose(b.gamma, (1 + alpha) * ref, rtol=1e-10)
        # the source pixel: both images equal s + s2 (unit norm)
        assert abs(b.gamma[i0] - (1 + alpha) * (s + s2)) <= 1e-10 * (s + s2)


def test_uninflated_bound_equals_the_closed_form():
    A, R, i0, s, s2 = _one_source()
    mf, mvdr = _closed_forms(A, i0, s, s2)
    b0 = O.bounds(A, None, R, 1000, O.Params(bound=O.BOUND_MF))
    b1 = O.bounds(A, None, R, 1000, O.Params(bound=O.BOUND_MVDR))
    np.testing.assert_allclose(b0.gamma, mf, rtol=1e-10)
    np.testing.assert_allclose(b1.gamma, mvdr, rtol=1e-10)


def _coverage(bound, bias_c, alpha=2.0, draws=1500, N=400, seed=11):
    A, R, i0, s, s2 = _one_source()
    mf, mvdr = _closed_forms(A, i0, s, s2)
    truth = mf if bound == O.BOUND_MF else mvdr
    p = R.shape[0]
    Lr = np.linalg.cholesky(R)
    rng = np.random.default_rng(seed)
    pix = np.array([i0, 0, 17])                   # the source, a corner, a sidelobe
    cover = np.zeros(len(pix))
    widths, errs = [], []
    for _ in range(draws):
        G = (rng.standard_normal((p, N)) + 1j * rng.standard_normal((p, N))) / math.sqrt(2.0)
        Y = Lr @ G
        Rh = (Y @ Y.conj().T) / N
        prm = O.Params(bound=bound, inflate=O.INFLATE_STD, alpha=alpha, bias_c=bias_c)
        b = O.bounds(A, None, Rh, N, prm)
        base = b.dirty if bound == O.BOUND_MF else b.mvdr
        cover += b.gamma[pix] >= truth[pix]
        widths.append((b.gamma - base)[pix] / alpha)
        errs.append(base[pix] - truth[pix])
    return cover / draws, np.mean(widths, axis=0), np.std(errs, axis=0)


def test_std_inflation_covers_the_truth_mf():
    cov, width, spread = _coverage(O.BOUND_MF, 0)
    assert np.all(cov >= 0.95) and np.all(cov <= 0.995), cov
    # the std the bound adds is the spread of the estimate (10 %)
    np.testing.assert_allclose(width, spread, rtol=0.1)


def test_std_inflation_covers_the_truth_mvdr_unbiased():
    # with C = N / (N - p) the MVDR estimate is unbiased to first order
    cov, width, spread = _coverage(O.BOUND_MVDR, 1)
    assert np.all(cov >= 0.95) and np.all(cov <= 0.995), cov
    np.testing.assert_allclose(width, spread, rtol=0.1)
