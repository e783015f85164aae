"""Graph-driven tensor-core solver (64 < p <= 384) against the FP64 oracle.

Above p = 64 a tensor-core solve runs the Table I loop as one CUDA graph
whose kernels apply the operators in (tile, unit) work items.  Each case
checks, against the oracle run with the same thresholds and feasibility
tolerance (streamed operator form: Psi is never stored), that the GPU's
decision path (every freed and clamped pixel in order) is a path of the
method: the oracle replays it and admits each decision, allowing only ties
within 1e-6 of the problem's scale (the tolerance boundary of the
multiplier and feasibility tests); the final pixel sets and the image
(within 1e-4 relative L2) must then match the oracle along that path.
Shapes cover one, two, three and four operator units (Kp = 96, 128, 160,
288, 384), odd p and ragged grids."""
import numpy as np
import pytest

import synth
from oracle import imager as O

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
TIE_TOL = 1e-6      # decisions closer than this (relative to scale) are ties


@pytest.fixture(scope="module")
def G():
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    return G


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# (seed, p, n_l, n_m, sources, N, array radius, cost, arithmetic)
CASES = [
    (501, 72, 24, 20, 5, 3000, 8.0, O.COST_PWLS, 1),      # Kp = 96: one unit
    (502, 100, 20, 18, 4, 3000, 10.0, O.COST_LS, 1),      # Kp = 128: one unit of 256 rows
    (503, 150, 18, 16, 4, 4000, 12.0, O.COST_PWLS, 1),    # Kp = 160: two units
    (504, 97, 17, 13, 3, 3000, 8.0, O.COST_PWLS, 1),      # odd p, ragged tiles
    (505, 288, 20, 18, 4, 5000, 20.0, O.COST_PWLS, 1),    # Kp = 288: three units
    (506, 330, 12, 13, 3, 5000, 20.0, O.COST_LS, 1),      # Kp = 384 (no split of 352)
    (507, 128, 22, 21, 5, 4000, 12.0, O.COST_PWLS, 2),    # BF16x3
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[1]}_{'pwls' if c[7] else 'ls'}_m{c[8]}" for c in CASES])
def test_wide_solve_follows_the_oracle(G, case):
    seed, p, nl, nm, nsrc, N, rad, cost, prec = case
    job = synth.custom(seed, p, nl, nm, nsrc, N, radius=rad, snr_db=0.0)
    prm = O.Params(cost=cost, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5)
    im = G.Imager.from_job(job, cost=cost, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5, precision=prec)
    sigma, info = im.solve()
    log = [(k, q) for k, q, _ in im.events()]
    sets = im.sets()
    im.close()
    assert info.converged == 1
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    bnd = O.bounds(A, None, job.R, job.N, prm)
    prob = O.cost_problem(A, None, job.R, bnd, cost)
    rep = O.active_set_follow(prob, bnd.eps, prm, log, tol=TIE_TOL)
    assert not rep.violations, (rep.violations[:3], rep.max_margin)
    assert rep.result.converged
    assert info.outer == rep.result.outer
    np.testing.assert_array_equal(sets, rep.result.sets)
    assert _rel(sigma, rep.result.sigma) <= IMG_TOL


def test_wide_solve_repeats_bit_for_bit(G):
    job = synth.custom(511, 96, 20, 16, 4, 3000, radius=10.0, snr_db=0.0)
    im = G.Imager.from_job(job, kappa=6.0, eps_floor=1e-6, precision=1)
    a, ia = im.solve()
    b, ib = im.solve()
    im.close()
    np.testing.assert_array_equal(a, b)
    assert ia.outer == ib.outer and ia.lsqr_iters == ib.lsqr_iters


def test_wide_and_narrow_jobs_in_one_batch(G):
    """A batch mixing one-CTA jobs (p <= 64) and graph-driven jobs (p > 64)
    gives every job the image it gets alone."""
    jobs = [synth.custom(520 + j, p, n, n - 2, 4, 3000, radius=10.0)
            for j, (p, n) in enumerate([(48, 24), (96, 20), (160, 18), (64, 22)])]
    singles = []
    for job in jobs:
        im = G.Imager.from_job(job, precision=1)
        singles.append(im.solve()[0])
        im.close()
    ims = [G.Imager.from_job(job, precision=1) for job in jobs]
    outs, infos = G.solve_batch(ims)
    for a, b, inf in zip(outs, singles, infos):
        np.testing.assert_array_equal(a, b)
        assert inf.converged == 1
    for im in ims:
        im.close()


def test_wide_solve_reports_max_outer(G):
    """A pass cap ends the graph's loop with IMG_ENOTCONV and the image of the
    last feasible point, as in the one-CTA solver."""
    job = synth.custom(530, 80, 16, 16, 5, 3000, radius=8.0)
    prm = O.Params(cost=O.COST_PWLS, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5, max_outer=7)
    ref = O.image_job(job, prm, streamed=True)
    im = G.Imager.from_job(job, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5, max_outer=7, precision=1)
    sigma, info = im.solve()
    im.close()
    assert info.status == G.IMG_ENOTCONV and info.outer == 7
    assert info.outer == ref.solve.outer and not ref.solve.converged
    assert _rel(sigma, ref.solve.sigma) <= IMG_TOL
