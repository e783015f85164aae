"""Write FP64-oracle reference records for full-size parity tests.

Each record stores the synthetic inputs (so the GPU test consumes exactly the
covariance the oracle saw, independent of the platform's BLAS rounding) and
the oracle's outputs.  Only synth/ and oracle/ are used here.

    python tests/golden/make_golden.py mid_pwls
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth                       # noqa: E402
from oracle import imager as O     # noqa: E402
from oracle import snapshots as S  # noqa: E402

RECORDS = {
    # 128x128 grid, p = 64 log-spiral, 20 points + Gaussian blob, N = 1e4,
    # PWLS with the MVDR bound, kappa = 6 (the bench workload's image)
    "mid_pwls": dict(maker=lambda: synth.mid(), prm=O.Params(cost=O.COST_PWLS, kappa=6.0,
                                                                eps_floor=1e-6, feas_tol=1e-5)),
    "mid_ls": dict(maker=lambda: synth.mid(), prm=O.Params(cost=O.COST_LS, kappa=6.0,
                                                            eps_floor=1e-6, feas_tol=1e-5)),
    # K = 2 snapshots, p = 100 disk, 64x64 grid, a point source and two
    # extended structures (the stand-in for the paper's extended-source
    # simulation): the K-snapshot MF, MVDR and ASSC images only (C = 1); the
    # bounded solve of this sky takes the oracle well over an hour
    # K = 2 snapshots, p = 48 disk of radius 20, 48x48 grid, 15 point sources
    # U[1, 10], SNR 0 dB, N = 1e4, the array turned 0.2 rad between
    # snapshots: PWLS with the K-snapshot MVDR bound, kappa = 6
    "snapshots_mid_pwls": dict(maker=lambda: synth.snapshots_custom(7148, 48, 48, 48, 15, 10_000, 2,
                                                                    dtheta=0.2, radius=20.0, snr_db=0.0),
                               prm=O.Params(cost=O.COST_PWLS, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5)),
    "snapshots_extended_bounds": dict(maker=lambda: synth.snapshots_extended(),
                                      prm=O.Params(cost=O.COST_PWLS), bounds_only=True),
    # 256x256 grid, p = 288 in six clusters within 200 wavelengths, 50 points
    # + 3 Gaussian blobs, N = 1e4, SNR 0 dB: PWLS with the MVDR bound,
    # kappa = 6, by the streamed oracle (the explicit Psi would hold 87 GB).
    # "large_pwls_t" stops after the first 400 passes of Table I (max_outer)
    "large_pwls": dict(maker=lambda: synth.large(), streamed=True,
                       prm=O.Params(cost=O.COST_PWLS, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5)),
    "large_pwls_t": dict(maker=lambda: synth.large(), streamed=True,
                         prm=O.Params(cost=O.COST_PWLS, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5,
                                      max_outer=400)),
    # the first 100 passes (the FP32 arm of the arithmetic sweep, whose
    # one-CTA CUDA-core solver takes minutes for 400 passes at p = 288)
    "large_pwls_t100": dict(maker=lambda: synth.large(), streamed=True,
                            prm=O.Params(cost=O.COST_PWLS, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5,
                                         max_outer=100)),
    # the same solve with LSQR stopped at atol = btol = 1e-6 (the tolerance the
    # GPU uses) instead of 1e-12: how far two FP64 runs of the method end apart
    # when only the subproblem accuracy differs
    "large_pwls_tol6": dict(maker=lambda: synth.large(), streamed=True,
                            prm=O.Params(cost=O.COST_PWLS, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5,
                                         lsqr_atol=1e-6, lsqr_btol=1e-6)),
}


def make(name: str) -> str:
    rec = RECORDS[name]
    job = rec["maker"]()
    prm = rec["prm"]
    t0 = time.time()
    snap = hasattr(job, "K")
    out = os.path.join(HERE, f"{name}.npz")
    if rec.get("bounds_only"):
        As = S.steering_stack(job.ant_xyz, job.l, job.m, job.lam)
        bnd = S.bounds_k(As, S.khatri_rao_stack(As), job.R, job.N, prm)
        np.savez_compressed(out, K=job.K, ant_xyz=job.ant_xyz, l=job.l, m=job.m, lam=job.lam, R=job.R,
                            N=job.N, bias_c=prm.bias_c, dirty=bnd.dirty, mvdr=bnd.mvdr, assc=bnd.assc,
                            oracle_seconds=time.time() - t0)
        return out
    if snap:
        res = S.image_snapshot_job(job, prm)
    else:
        last = [time.time()]

        def progress(outer, nf, its):
            if time.time() - last[0] > 60:
                last[0] = time.time()
                print(f"{name}: pass {outer}, |F| {nf}, LSQR iterations {its}, "
                      f"{time.time() - t0:.0f} s", flush=True)

        res = O.image_job(job, prm, streamed=rec.get("streamed", False), progress=progress)
    dt = time.time() - t0
    extra = dict(assc=res.bounds.assc, K=job.K) if snap else {}
    np.savez_compressed(
        out, **extra, ant_xyz=job.ant_xyz, l=job.l, m=job.m, lam=job.lam, R=job.R, N=job.N,
        cost=prm.cost, kappa=prm.kappa, eps_floor=prm.eps_floor, feas_tol=prm.feas_tol,
        dirty=res.bounds.dirty, mvdr=res.bounds.mvdr, gamma=res.bounds.gamma,
        sigma=res.solve.sigma, sets=res.solve.sets, outer=res.solve.outer,
        lsqr_iters=res.solve.lsqr_iters, converged=res.solve.converged, max_outer=prm.max_outer,
        events=np.array([(0 if e[0] == "free" else 1, e[1], e[2] if len(e) > 2 else -1)
                         for e in res.solve.events], dtype=np.int64),
        oracle_seconds=dt)
    return out


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(RECORDS)):
        print(make(n))
