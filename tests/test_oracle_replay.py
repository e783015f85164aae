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
