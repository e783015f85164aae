"""The 256 x 256, p = 288 workload (six clusters of 48 antennas within 200
wavelengths, 50 point sources and 3 Gaussian blobs, N = 1e4, SNR 0 dB)
against the stored oracle record of its first 400 Table I passes
(tests/golden/large_pwls_t.npz, written by tests/golden/make_golden.py with
the streamed oracle).

The GPU runs the same 400 passes (max_outer) on the record's covariance.
Its dirty and MVDR images must match the oracle's within 1e-5; its decision
log must be a path the oracle admits when it replays it (ties within 1e-6
of scale); the pixel sets and the image must match the oracle's along that
path (1e-4)."""
import os

import numpy as np
import pytest

from oracle import imager as O

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
OP_TOL = 1e-5
IMG_TOL = 1e-4
TIE_TOL = 1e-6


@pytest.fixture(scope="module")
def G():
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    return G


@pytest.fixture(scope="module")
def rec():
    return np.load(os.path.join(HERE, "golden", "large_pwls_t.npz"))


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _prm(rec):
    return O.Params(cost=int(rec["cost"]), kappa=float(rec["kappa"]), eps_floor=float(rec["eps_floor"]),
                    feas_tol=float(rec["feas_tol"]), max_outer=int(rec["max_outer"]))


@pytest.mark.parametrize("prec", [1, 2])
def test_large_first_passes_follow_the_record(G, rec, prec):
    prm = _prm(rec)
    im = G.Imager(rec["ant_xyz"], rec["l"], rec["m"], float(rec["lam"]), cost=prm.cost, kappa=prm.kappa,
                  eps_floor=prm.eps_floor, feas_tol=prm.feas_tol, max_outer=prm.max_outer, precision=prec)
    im.set_covariance(rec["R"], int(rec["N"]))
    assert _rel(im.dirty(), rec["dirty"]) <= OP_TOL
    assert _rel(im.mvdr_bound(), rec["mvdr"]) <= OP_TOL
    sigma, info = im.solve()
    log = [(k, q) for k, q, _ in im.events()]
    sets = im.sets()
    im.close()
    assert info.status == G.IMG_ENOTCONV and info.outer == int(rec["outer"])
    # the record itself (its own path): sets and image agree already
    np.testing.assert_array_equal(sets, rec["sets"])
    assert _rel(sigma, rec["sigma"]) <= IMG_TOL
    # the GPU's path is admissible: the oracle replays it
    A = O.steering_matrix(rec["ant_xyz"], rec["l"], rec["m"], float(rec["lam"]))
    bnd = O.bounds(A, None, rec["R"], int(rec["N"]), prm)
    prob = O.cost_problem(A, None, rec["R"], bnd, prm.cost)
    rep = O.active_set_follow(prob, bnd.eps, prm, log, tol=TIE_TOL)
    assert not rep.violations, (rep.violations[:3], rep.max_margin)
    np.testing.assert_array_equal(sets, rep.result.sets)
    assert _rel(sigma, rep.result.sigma) <= IMG_TOL
