"""The oracle's decision-log replay (used to check path-dependent GPU runs)
accepts the oracle's own path and rejects a planted wrong decision."""
import numpy as np

import synth
from oracle import imager as O


def _setup(cost):
    job = synth.custom(17, 12, 14, 12, 4, 900, radius=4.0, snr_db=0.0)
    prm = O.Params(cost=cost, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    bnd = O.bounds(A, Psi, job.R, job.N, prm)
    prob = O.cost_problem(A, Psi, job.R, bnd, cost)
    return prm, bnd, prob


def _log_of(res):
    out = []
    for e in res.events:
        if e[0] == "free":
            out.append((0, e[1]))
        else:
            out.append((1 if e[2] == O.SET_L else 2, e[1]))
    return out


def test_replay_of_own_path_is_exact():
    for cost in (O.COST_LS, O.COST_PWLS):
        prm, bnd, prob = _setup(cost)
        res = O.active_set(prob, bnd.eps, prm)
        rep = O.active_set_follow(prob, bnd.eps, prm, _log_of(res))
        assert not rep.violations
        assert rep.ties == 0
        np.testing.assert_array_equal(rep.result.sets, res.sets)
        np.testing.assert_allclose(rep.result.sigma, res.sigma, rtol=0, atol=0)


def test_replay_rejects_a_wrong_free_decision():
    prm, bnd, prob = _setup(O.COST_PWLS)
    res = O.active_set(prob, bnd.eps, prm)
    log = _log_of(res)
    # plant: free the dimmest pixel of the MVDR image first instead of the brightest
    log[0] = (0, int(np.argmin(bnd.mvdr)))
    rep = O.active_set_follow(prob, bnd.eps, prm, log)
    assert rep.violations and rep.violations[0][0] == "free"


def test_replay_rejects_early_stop():
    prm, bnd, prob = _setup(O.COST_LS)
    res = O.active_set(prob, bnd.eps, prm)
    log = _log_of(res)[:3]
    rep = O.active_set_follow(prob, bnd.eps, prm, log)
    assert any(v[0] == "stop" for v in rep.violations)


def _clamp_case(seed=30):
    # LS cost; seed 30's path clamps two pixels to U (each while it is the
    # only free pixel), seed 31's clamps a pixel while others are free
    job = synth.custom(seed, 12, 14, 12, 4, 900, radius=4.0, snr_db=0.0)
    prm = O.Params(cost=O.COST_LS, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    bnd = O.bounds(A, Psi, job.R, job.N, prm)
    prob = O.cost_problem(A, Psi, job.R, bnd, prm.cost)
    res = O.active_set(prob, bnd.eps, prm)
    log = _log_of(res)
    k = next(i for i, e in enumerate(log) if e[0] in (1, 2))
    return prm, bnd, prob, res, log, k


def test_replay_accepts_its_own_clamps():
    prm, bnd, prob, res, log, k = _clamp_case()
    assert log[k][0] == 2
    rep = O.active_set_follow(prob, bnd.eps, prm, log)
    assert not rep.violations and rep.ties == 0


def test_replay_rejects_a_clamp_to_the_wrong_set():
    prm, bnd, prob, res, log, k = _clamp_case()
    log[k] = (1, log[k][1])                  # plant: the pixel moves to L, its direction is positive
    rep = O.active_set_follow(prob, bnd.eps, prm, log)
    assert rep.violations and rep.violations[0][0] == "clamp-set"


def test_replay_rejects_a_clamp_of_the_wrong_pixel():
    prm, bnd, prob, res, log, _ = _clamp_case(31)
    # a clamp decision taken while at least two pixels are free
    free, plant = [], None
    for k, (kind, q) in enumerate(log):
        if kind == 0:
            free.append(q)
            continue
        if len(free) >= 2:
            plant = (k, next(o for o in free if o != q))
            break
        free.remove(q)
    assert plant is not None
    k, other = plant
    log[k] = (log[k][0], other)              # plant: another free pixel blocks the step
    rep = O.active_set_follow(prob, bnd.eps, prm, log)
    assert rep.violations and rep.violations[0][0] in ("clamp", "clamp-set")


def test_replay_rejects_a_clamp_of_a_pixel_not_free():
    prm, bnd, prob, res, log, k = _clamp_case()
    freed = {q for kind, q in log[:k] if kind == 0}
    other = next(q for q in range(prob.Q) if q not in freed)
    log[k] = (log[k][0], other)
    rep = O.active_set_follow(prob, bnd.eps, prm, log)
    assert rep.violations and rep.violations[0][0] == "clamp-not-free"
