"""Parity on the benchmark workloads' shapes and the other configurations.

* 128x128, p = 64 (the bench image): dirty/MVDR on every pixel and the full
  PWLS and CLS solves against stored FP64 oracle records (tests/golden),
  including the decision path.
* Path-dependent solves (kappa = 6) on mid-size jobs: the GPU decision log is
  replayed through the oracle, every decision must be admissible (the
  oracle's own choice or a tie within tolerance) and the images must agree.
* Uneven batches (channels of p in {48, 64, 96} and 64..128 grids), the
  large array (p = 288) and serving-size jobs: operators on sampled pixels,
  computed one by one by the oracle's definitions.
"""
import os

import numpy as np
import pytest

import synth
from oracle import imager as O

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
OP_TOL = 1e-5
IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def G():
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    return G


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _oracle_log(events):
    out = []
    for e in events:
        if e[0] == 0:
            out.append((0, int(e[1])))
        else:
            out.append((1 if e[2] == O.SET_L else 2, int(e[1])))
    return out


# ---------------------------------------------------------------- golden records
@pytest.mark.parametrize("name", ["mid_pwls", "mid_ls"])
@pytest.mark.parametrize("prec", [0, 1])
def test_bench_image_matches_oracle_record(G, name, prec):
    path = os.path.join(HERE, "golden", f"{name}.npz")
    g = np.load(path)
    if "feas_tol" not in g.files:
        pytest.skip("record written without feasibility tolerance")
    im = G.Imager(g["ant_xyz"], g["l"], g["m"], float(g["lam"]), cost=int(g["cost"]),
                  kappa=float(g["kappa"]), eps_floor=float(g["eps_floor"]),
                  feas_tol=float(g["feas_tol"]), precision=prec)
    im.set_covariance(g["R"], int(g["N"]))
    d = im.dirty()
    mv = im.mvdr_bound()
    assert _rel(d, g["dirty"]) <= OP_TOL
    assert _rel(mv, g["mvdr"]) <= OP_TOL
    sigma, info = im.solve()
    assert info.converged == 1
    gpu_log = [(k, p) for k, p, _ in im.events()]
    assert gpu_log == _oracle_log(g["events"]), "decision path differs from the oracle's"
    assert _rel(sigma, g["sigma"]) <= IMG_TOL
    np.testing.assert_array_equal(im.sets(), g["sets"])
    im.close()


# ---------------------------------------------------------------- replayed paths
def _replay_case(G, job, cost, prec):
    prm = O.Params(cost=cost, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5)
    im = G.Imager.from_job(job, cost=cost, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5, precision=prec)
    sigma, info = im.solve()
    log = [(k, p) for k, p, _ in im.events()]
    im.close()
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    bnd = O.bounds(A, Psi, job.R, job.N, prm)
    prob = O.cost_problem(A, Psi, job.R, bnd, cost)
    rep = O.active_set_follow(prob, bnd.eps, prm, log, tol=1e-6)
    return sigma, info, rep


@pytest.mark.parametrize("seed", [201, 202, 203])
@pytest.mark.parametrize("cost", [0, 1])
def test_replayed_path_is_admissible_and_matches(G, seed, cost):
    job = synth.custom(seed, 40, 48, 40, 8, 4000, radius=12.0, snr_db=0.0)
    sigma, info, rep = _replay_case(G, job, cost, prec=1)
    assert info.converged == 1
    assert not rep.violations, rep.violations[:3]
    assert rep.result.converged
    assert _rel(sigma, rep.result.sigma) <= IMG_TOL


# ---------------------------------------------------------------- other shapes
def _sampled_bounds(job, idx, bias_c=0):
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)[:, idx]
    d = np.real(np.einsum("ki,kl,li->i", A.conj(), job.R, A))
    Rinv = np.linalg.inv(job.R)
    h = np.real(np.einsum("ki,kl,li->i", A.conj(), Rinv, A))
    C = job.N / (job.N - job.p) if bias_c else 1.0
    return d, C / h


@pytest.mark.parametrize("c", [0, 7, 21, 63])
def test_uneven_channel_operators(G, c):
    job = synth.batch_channel(c)
    rng = np.random.default_rng(c)
    idx = rng.choice(job.Q, 300, replace=False)
    ref_d, ref_mv = _sampled_bounds(job, idx)
    for prec in (0, 1):
        im = G.Imager.from_job(job, precision=prec)
        d, mv = im.dirty(), im.mvdr_bound()
        im.close()
        assert _rel(d[idx], ref_d) <= OP_TOL
        assert _rel(mv[idx], ref_mv) <= OP_TOL


def test_uneven_batch_equals_single_jobs(G):
    """Channels of different p, grid and wavelength in one batch (one launch
    per arithmetic group) give the same images as solving them one by one."""
    jobs = [synth.custom(300 + j, p, n, n, 6, 4000, radius=10.0)
            for j, (p, n) in enumerate([(48, 40), (64, 48), (96, 32), (20, 56)])]
    singles = []
    for job in jobs:
        im = G.Imager.from_job(job, precision=1)
        singles.append(im.solve()[0])
        im.close()
    ims = [G.Imager.from_job(job, precision=1) for job in jobs]
    outs, infos = G.solve_batch(ims)
    for a, b in zip(outs, singles):
        np.testing.assert_array_equal(a, b)
    for im in ims:
        im.close()


def test_large_array_operators_sampled(G):
    """p = 288 in 6 clusters, 256x256 grid: dirty and MVDR images on sampled
    pixels (the tensor-core path needs p <= 64, so this is the FP32 path)."""
    job = synth.large()
    rng = np.random.default_rng(4)
    idx = rng.choice(job.Q, 200, replace=False)
    ref_d, ref_mv = _sampled_bounds(job, idx)
    im = G.Imager.from_job(job, precision=1)
    d, mv = im.dirty(), im.mvdr_bound()
    im.close()
    assert _rel(d[idx], ref_d) <= OP_TOL
    assert _rel(mv[idx], ref_mv) <= OP_TOL
    assert np.all(mv <= d * (1 + 1e-5))


@pytest.mark.parametrize("j", [0, 1, 2, 3, 4, 5])
def test_serving_jobs_operators_sampled(G, j):
    job = synth.serve_job(j)
    rng = np.random.default_rng(j)
    idx = rng.choice(job.Q, 200, replace=False)
    ref_d, ref_mv = _sampled_bounds(job, idx)
    im = G.Imager.from_job(job, precision=1)
    d, mv = im.dirty(), im.mvdr_bound()
    im.close()
    assert _rel(d[idx], ref_d) <= OP_TOL
    assert _rel(mv[idx], ref_mv) <= OP_TOL
