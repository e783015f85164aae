"""Benchmark: bounded least-squares images per second on one GB300.

Headline workload (one step): a batch of B independent 256x256-pixel images
from a 288-antenna array (six clusters of 48 within 200 wavelengths), each
sky 50 lognormal point sources plus 3 Gaussian blobs (FWHM 4-10 px), SNR
0 dB, N = 10^4 samples, each image through the whole hot path: Cholesky of
R_hat, matched-filter dirty image, MVDR bound, and the preconditioned-WLS
active-set solve with LSQR subproblems (kappa = 6).  The second workload
("mid": 128x128 pixels, 64-antenna log-spiral, 20 points plus a blob) is
reported inside the same line.  Inputs are seeded synthetic data.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--workload large|mid]
    python bench.py --impl reference      # the FP64 CPU oracle, bounded sample

Under torchrun each rank solves its own batch (jobs are independent: weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# independent launch groups of the job server run on many streams; give them
# as many hardware queues as CUDA allows (must precede CUDA initialisation)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "images/s"
WORKLOADS = {
    "large": "pwls-mvdr 256x256 p=288 (6 clusters of 48 within 200 lambda), 50 points + 3 Gaussian blobs, "
             "N=1e4, SNR 0 dB, kappa=6",
    "mid": "pwls-mvdr 128x128 p=64 log-spiral, 20 points + blob, N=1e4, kappa=6",
}
WORKLOAD = WORKLOADS["large"]
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workload
def rank_seeds(rank: int, B: int, workload: str = "large"):
    """Seeds of the B images rank `rank` solves: disjoint across ranks (the
    images are independent, so ranks are replicas on different data)."""
    base = 4000 if workload == "large" else 2000
    return [base + 100_000 * rank + j for j in range(B)]


def make_jobs(seeds, workload: str = "large"):
    import synth
    if workload == "large":
        return [synth.large(seed=s) for s in seeds]
    return [synth.mid(seed=s) for s in seeds]


def default_batch(workload: str, steps: int, sms: int) -> int:
    """Images per step.  mid: two per SM (one CTA each).  large: each image
    is a graph of kernels spread over the GPU, and the solves in flight
    overlap: 8 give 0.42 images/s, 16 give 0.54, 24 give 0.55 and 32 fall
    back to 0.49 (their working sets no longer share L2); the batch shrinks
    (to 4 at least) when many steps are asked for, to keep the timed region
    near a minute."""
    if workload == "mid":
        return 2 * sms
    return max(4, min(16, 48 // max(steps, 1)))


def reduce_max(value: float, device=None) -> float:
    """Max over ranks (the job is as slow as its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sm_count() -> int:
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


PRECISIONS = {"fp32": 0, "f16x3": 1, "bf16x3": 2}


def fp32_alu_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 CUDA-core peak: 128 FMA lanes per SM, 2 flops each."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def run_ours(args, rank: int, world: int):
    import torch
    import paper_1505_01348_gb300 as G

    G.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = args.workload
    B = args.batch or default_batch(wl, args.steps, sm_count())
    jobs = make_jobs(rank_seeds(rank, B, wl), wl)
    stream = torch.cuda.Stream(device=dev)
    prec = PRECISIONS[args.precision]
    # one-CTA jobs (mid) share the launching stream; graph-driven jobs
    # (large) each get a stream so that their solves run side by side
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(B - 1)] if wl == "large" else [stream] * B
    ims = [G.Imager(j.ant_xyz, j.l, j.m, j.lam, stream=st.cuda_stream, precision=prec)
           for j, st in zip(jobs, streams)]
    # column-major complex128 bytes of each R_hat, resident on the device
    R_dev = [torch.from_numpy(np.ascontiguousarray(j.R.ravel(order="F"))).to(dev) for j in jobs]
    sig_dev = [torch.empty(j.Q, dtype=torch.float64, device=dev) for j in jobs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step_device():
        for im, R, j in zip(ims, R_dev, jobs):
            im.set_covariance(R, j.N)
        G.prepare_batch(ims)
        return G.solve_batch(ims, outs=sig_dev)[1]

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step_device()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = ClockSampler(dev.index)
        clk.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        infos_all = []
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))                      # L2 flush, outside the events
            e0, e1, e2 = ev[k]
            e0.record(stream)
            for im, R, j in zip(ims, R_dev, jobs):
                im.set_covariance(R, j.N)
            G.prepare_batch(ims)
            e1.record(stream)
            _, infos = G.solve_batch(ims, outs=sig_dev)
            e2.record(stream)
            infos_all.append(infos)
        torch.cuda.synchronize()
        clocks = clk.stop()
    t_step = [e0.elapsed_time(e2) / 1e3 for e0, _, e2 in ev]
    t_prep = [e0.elapsed_time(e1) / 1e3 for e0, e1, _ in ev]
    t_solve = [e1.elapsed_time(e2) / 1e3 for _, e1, e2 in ev]
    total = reduce_max(sum(t_step), dev)
    flops = [sum(i.op_flops for i in infos) for infos in infos_all]
    # kernels each wide solve executed (its report's cyc_aux[0]) plus the
    # batch's factor / bounds launches, per step
    launches = [[float(i.cyc_aux[0]) for i in infos] + [4.0] for infos in infos_all] if wl == "large" else None
    conv = sum(i.converged for infos in infos_all for i in infos)
    outer = float(np.mean([i.outer for infos in infos_all for i in infos]))

    # ---------------- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pin = [torch.empty(j.p * j.p, dtype=torch.complex128).pin_memory() for j in jobs]
        for t, j in zip(pin, jobs):
            t.numpy()[:] = j.R.ravel(order="F")
        pin_np = [t.numpy().reshape(j.p, j.p, order="F") for t, j in zip(pin, jobs)]
        host_out = [torch.empty(j.Q, dtype=torch.float64).pin_memory().numpy() for j in jobs]
        ke = 1 if wl == "large" else max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            for im, R, j in zip(ims, pin_np, jobs):
                im.set_covariance(R, j.N)
            G.prepare_batch(ims)
            G.solve_batch(ims, outs=host_out)
        torch.cuda.synchronize()
        te = reduce_max((time.perf_counter() - t0) / ke, dev)
        e2e = {"value": world * B / te, "unit": METRIC,
               "h2d_bytes_per_step": int(sum(j.R.nbytes for j in jobs)),
               "d2h_bytes_per_step": int(sum(j.Q * 8 for j in jobs)),
               "ms_per_step": te * 1e3}
    for im in ims:
        im.close()

    res = {
        "workload": wl, "p": jobs[0].p, "n": jobs[0].n_l,
        "B": B, "total": total, "t_step": t_step, "t_solve": t_solve, "t_prep": t_prep, "launches": launches,
        "prep_flops": float(sum(2 * 8.0 * j.p * j.p * j.Q for j in jobs)), "flops": flops,
        "conv": conv, "outer": outer, "clocks": clocks, "e2e": e2e,
        "sms": sm_count(),
    }
    return res


# ---------------------------------------------------------------- serving
def unit_kp(p: int) -> int:
    """Padded feature count of the tensor-core operand: p rounded up to 32,
    and above p = 256 further up until it splits into at most 8 units of a
    multiple of 16 rows, each unit at most 128."""
    kp = (p + 31) // 32 * 32
    if p <= 256:
        return kp
    while not any(kp % nu == 0 and (kp // nu) % 16 == 0 for nu in range((kp + 127) // 128, 9)):
        kp += 32
    return kp


def run_operators(args, cases=((64, 256), (128, 256), (256, 256), (256, 512), (288, 256)), reps: int = 20):
    """Operator pair img_psi_adj / img_psi on full n x n grids: p = 64, 128
    and 256 on 256x256 (the serving mix's largest grid), p = 256 on 512x512
    and p = 288 on 256x256; up to p = 256 the adjoint runs the streamed,
    warp-specialised tensor-core kernel and at p = 288 the solver's (tile,
    unit) work-item kernel; the forward forms tensor-core Gram blocks at
    every p.
    Adjoint Psi^H (Eq. 16): the streamed tensor-core kernel; each call reduces
    max |U|, writes the chunked operand image from the complex128 U and runs
    the adjoint; calls are queued back to back on one stream and timed with
    CUDA events.
    Useful flops: 8 p^2 Q; issued: the three split products on the padded
    2Kp x 2Kp operand, 3 * 2 * 128 * (2Kp)^2 per 128-pixel tile.  Forward
    Psi x (Eq. 15) as tensor-core Gram blocks: useful 4 p^2 Q (Hermitian
    half), issued 3 * 2 * 128 * N per pixel for every 128 x N block formed."""
    import torch
    import paper_1505_01348_gb300 as G
    import synth

    prec = PRECISIONS[args.precision]
    if prec == 0:
        return None
    pk = measured_peaks()
    peak = float(pk.get("bf16_tflops") or 1900.0)
    out_d = {"grids": "n x n pixels per case (key p<p>_<n>)", "precision": args.precision,
             "kernels": "k_psi_adj_wide (adjoint), k_fwd_wide (forward)",
             "per_call": ("adjoint: max |U| reduction + operand image + adjoint (U read in place); forward: "
                          "FP32 weights + max |w| + Gram blocks + ordered partial sums into K"),
             "peak_tflops": peak,
             "peak_basis": "measured dense BF16 burst (FP16 runs at the BF16 rate)"}
    st = torch.cuda.Stream()
    for p, n in cases:
        job = synth.custom(7000 + p, p, n, n, 20, 10_000, radius=50.0)
        # the context works on this stream, so events recorded on it bracket the calls
        im = G.Imager.from_job(job, precision=prec, stream=st.cuda_stream)
        U = torch.tensor(np.asfortranarray(job.R).T.copy(), dtype=torch.complex128, device="cuda")
        out = torch.empty(job.Q, dtype=torch.float64, device="cuda")
        for _ in range(3):
            im.psi_adj(U, out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            im.psi_adj(U, out, wait=False)
        e1.record(st)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        im.close()
        kp = unit_kp(p)
        tiles = ((n + 7) // 8) * ((n + 15) // 16) if p <= 256 else (job.Q + 127) // 128
        useful = 8.0 * p * p * job.Q
        issued = 3 * 2.0 * 128 * (2 * kp) ** 2 * tiles
        rec = {"adjoint_us_per_call": t * 1e6, "adjoint_useful_tflops": useful / t / 1e12,
               "adjoint_issued_tflops": issued / t / 1e12, "adjoint_issued_frac": issued / t / 1e12 / peak}
        # forward Psi x (Gram blocks of 128 x <=256 features over 64-pixel stages)
        x = torch.rand(job.Q, dtype=torch.float64, device="cuda")
        K = torch.empty((p, p), dtype=torch.complex128, device="cuda")
        im2 = G.Imager.from_job(job, precision=prec, stream=st.cuda_stream)
        for _ in range(3):
            im2.psi(x, K)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            im2.psi(x, K, wait=False)
        e1.record(st)
        torch.cuda.synchronize()
        tf = e0.elapsed_time(e1) / 1e3 / reps
        im2.close()
        nf = 2 * ((p + 31) // 32 * 32)
        blocks = [(m, nb) for m in range((nf + 127) // 128) for nb in range((nf + 255) // 256)
                  if 256 * nb + min(256, nf - 256 * nb) - 1 >= 128 * m]
        pix = ((n + 7) // 8) * ((n + 7) // 8) * 64
        fissued = sum(3 * 2.0 * 128 * min(256, nf - 256 * nb) * pix for _, nb in blocks)
        fuseful = 4.0 * p * p * job.Q
        rec.update({"forward_us_per_call": tf * 1e6, "forward_useful_tflops": fuseful / tf / 1e12,
                    "forward_issued_tflops": fissued / tf / 1e12, "forward_issued_frac": fissued / tf / 1e12 / peak})
        out_d[f"p{p}_{n}"] = rec
    return out_d


def run_ls_images(args, iters: int = 100):
    """Unconstrained WLS image with every pixel free (img_ls_image): LSQR
    on M = W Psi D^-1 over all Q pixels, a fixed 100 iterations (stopping
    tolerances 0).  Each iteration applies the forward (4 p^2 Q useful flops)
    and the adjoint (8 p^2 Q) to the whole image; wall time of the call,
    including the factor and bounds it starts with."""
    import paper_1505_01348_gb300 as G
    import synth

    prec = PRECISIONS[args.precision]
    out = {"iterations": iters, "precision": args.precision, "cost": "pwls"}
    for name, job in (("bench_128x128_p64", synth.mid()),
                      ("p256_256x256", synth.custom(7256, 256, 256, 256, 20, 10_000, radius=50.0))):
        im = G.Imager.from_job(job, precision=prec, lsqr_atol=0.0, lsqr_btol=0.0)
        im.ls_image(maxit=5)                       # warm-up (allocations, kernels)
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            _, info = im.ls_image(maxit=iters)
            ts.append(time.perf_counter() - t0)
        im.close()
        t = min(ts)
        out[name] = {"s_per_image": t, "images_s": 1.0 / t, "lsqr_iters": info.lsqr_iters,
                     "useful_operator_tflops": info.op_flops / t / 1e12}
    return out


def _steer64(ant, l, m, lam, il, im):
    """FP64 steering vectors of pixels (il, im), unit norm, -j sign (the data
    model's definition; host check values, no oracle code)."""
    n = np.sqrt(np.maximum(0.0, 1.0 - l[il] ** 2 - m[im] ** 2))
    dirs = np.stack([l[il], m[im], n])
    return np.exp(-2j * np.pi * (ant @ dirs) / lam) / np.sqrt(ant.shape[0])


def run_snapshots(args, iters: int = 100):
    """K > 1 snapshots on the stand-in for the paper's extended-source
    simulation (p = 100 antennas in a disk, K = 2 snapshots with the array
    turned 0.05 rad between them, 64x64 grid, a point source and two extended
    structures, N = 10^4): the K-snapshot MF, MVDR and ASSC images
    (img_snapshot_image, including both snapshots' factor and bounds, which a
    new covariance clears) and the K-snapshot WLS image
    (img_snapshot_ls_image, a fixed 100 LSQR iterations, stopping tolerances
    0).  Wall time per call, best of 3; the three images' relative L2 errors
    on 256 sampled pixels against FP64 values evaluated here."""
    import paper_1505_01348_gb300 as G
    import synth

    prec = PRECISIONS[args.precision]
    job = synth.snapshots_extended()
    out = {"workload": "p=100 disk, K=2 snapshots (0.05 rad apart), 64x64 grid, point + 2 extended "
                       "structures, N=1e4, pwls", "precision": args.precision}
    ims = [G.Imager(job.ant_xyz[k], job.l, job.m, job.lam, precision=prec, lsqr_atol=0.0, lsqr_btol=0.0)
           for k in range(job.K)]
    try:
        ts = []
        kinds = (G.SNAP_MF, G.SNAP_MVDR, G.SNAP_ASSC)
        for _ in range(3):
            for k, im in enumerate(ims):
                im.set_covariance(job.R[k], job.N)
            t0 = time.perf_counter()
            imgs = [G.snapshot_image(ims, kind) for kind in kinds]
            ts.append(time.perf_counter() - t0)
        out["images_mf_mvdr_assc_s"] = min(ts)
        try:
            # FP64 check values on 256 sampled pixels, evaluated here from the
            # definitions (C = 1): (1/K) sum d_k, K / sum h_k, 1 / max h_k
            idx = np.random.default_rng(13).choice(job.Q, 256, replace=False)
            dk, hk = [], []
            for k in range(job.K):
                Ak = _steer64(job.ant_xyz[k], job.l, job.m, job.lam, idx % job.n_l, idx // job.n_l)
                dk.append(np.real(np.einsum("ki,kl,li->i", Ak.conj(), job.R[k], Ak)))
                hk.append(np.real(np.einsum("ki,kl,li->i", Ak.conj(), np.linalg.inv(job.R[k]), Ak)))
            dk, hk = np.array(dk), np.array(hk)
            refs = (dk.mean(axis=0), job.K / hk.sum(axis=0), 1.0 / hk.max(axis=0))
            out["sampled_rel_err_mf_mvdr_assc"] = [
                float(np.linalg.norm(img[idx] - r) / np.linalg.norm(r)) for img, r in zip(imgs, refs)]
        except Exception as e:                       # the timing above stands either way
            out["sampled_rel_err_mf_mvdr_assc"] = f"{type(e).__name__}: {e}"
        G.snapshot_ls_image(ims, maxit=5)              # warm-up (kernel attributes, scratch)
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            _, info = G.snapshot_ls_image(ims, maxit=iters)
            ts.append(time.perf_counter() - t0)
        t = min(ts)
        out["ls_image"] = {"s_per_image": t, "images_s": 1.0 / t, "lsqr_iters": info.lsqr_iters,
                           "useful_operator_tflops": info.op_flops / t / 1e12}
    finally:
        for im in ims:
            im.close()
    return out


def run_precision(args):
    """Arithmetic sweep against FP64 on the 256x256, p = 288 workload:
    relative L2 errors of the dirty and MVDR images (all pixels) against the
    stored FP64 oracle record, and the first 400 Table I passes of the solve
    against the oracle's record of the same 400 passes (image error, same
    final sets, LSQR iterations); then the 128x128, p = 64 image (whole
    solve) against its stored record."""
    import paper_1505_01348_gb300 as G
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    big = np.load(os.path.join(ROOT, "tests", "golden", "large_pwls_t.npz"))
    gold = np.load(os.path.join(ROOT, "tests", "golden", "mid_pwls.npz"))
    out = {"large": ("256x256, p = 288: bounds and the first Table I passes (400; the FP32 arm 100) vs the "
                     "stored FP64 oracle records of those passes"),
           "mid": "bench image 128x128, p = 64, PWLS, whole solve vs the stored FP64 oracle record",
           "mid_oracle_outer_passes": int(gold["outer"]), "mid_oracle_lsqr_iters": int(gold["lsqr_iters"]),
           "not_built": "TF32x3 and FP64 arithmetic"}

    def solve(rec, prec, max_outer=0):
        im = G.Imager(rec["ant_xyz"], rec["l"], rec["m"], float(rec["lam"]), cost=int(rec["cost"]),
                      kappa=float(rec["kappa"]), eps_floor=float(rec["eps_floor"]),
                      feas_tol=float(rec["feas_tol"]), precision=prec, max_outer=max_outer)
        im.set_covariance(rec["R"], int(rec["N"]))
        d, mv = im.dirty(), im.mvdr_bound()
        t0 = time.perf_counter()
        sigma, info = im.solve()
        ts = time.perf_counter() - t0
        sets = im.sets()
        im.close()
        return d, mv, sigma, info, sets, ts

    big100 = np.load(os.path.join(ROOT, "tests", "golden", "large_pwls_t100.npz"))
    for name, prec in sorted(PRECISIONS.items(), key=lambda kv: kv[1]):
        # the FP32 arm runs the one-CTA CUDA-core solver: its 100 first passes
        rec = big100 if prec == 0 else big
        npass = int(rec["max_outer"])
        d, mv, sigma, info, sets, ts = solve(rec, prec, npass)
        _, _, sig2, info2, _, ts2 = solve(gold, prec)
        out[name] = {"large_dirty_rel": rel(d, big["dirty"]), "large_mvdr_rel": rel(mv, big["mvdr"]),
                     "large_passes": npass, "large_image_rel": rel(sigma, rec["sigma"]),
                     "large_sets_equal": bool(np.array_equal(sets, rec["sets"])),
                     "large_lsqr_iters": int(info.lsqr_iters),
                     "large_oracle_lsqr_iters": int(rec["lsqr_iters"]), "large_solve_s": ts,
                     "mid_image_rel": rel(sig2, gold["sigma"]), "mid_outer_passes": int(info2.outer),
                     "mid_lsqr_iters": int(info2.lsqr_iters), "mid_solve_s": ts2}
    return out


def _serve_stream(G, pool, prec, rate, seconds, reserve_wide, reserve_narrow, seed=77):
    """Poisson arrivals of the pool's jobs (cycled) into the continuous-batching
    server; latencies are the server's submit-to-done times."""
    distinct = len(pool)
    rng = np.random.default_rng(seed)
    n = int(rate * seconds)
    gaps = rng.exponential(1.0 / rate, n)
    srv = G.Server(hbm_budget_bytes=120 << 30)
    shapes = {}
    for j in pool:
        shapes.setdefault((j.p, j.n_l, j.n_m), j)
    for (p, _, _), j in shapes.items():                 # pool contexts before the clock starts
        srv.reserve(j, reserve_wide if p > 64 else reserve_narrow, precision=prec)
    ids = []
    t0 = time.perf_counter()
    t_next = t0
    for k in range(n):
        t_next += gaps[k]
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit_job(pool[k % distinct], precision=prec))
    lat = []
    for jid in ids:
        _, info, ms = srv.wait(jid)
        lat.append(ms)
    t_end = time.perf_counter()
    srv.close()
    lat = np.array(lat)
    return {"rate_jobs_s": rate, "jobs": n, "offered_s": seconds, "images_s": n / (t_end - t0),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max())}


def run_serve(args, full_rate: float = 3.0, full_seconds: float = 30.0, tc_rate: float = 200.0,
              tc_seconds: float = 10.0, distinct: int = 48):
    """Serving under load.  full: the whole job mix (p in {32, 64, 128, 256},
    grids 64^2 .. 256^2), at the highest Poisson rate measured to keep up
    (about 3.4 jobs/s served when 4 are offered); tc_subset: the jobs with
    p <= 64 at 200 jobs/s.  The plain per-job FP32 path (one img_solve at a
    time) is timed on the p <= 64 subset: on the full mix its p = 256 jobs run
    the one-CTA CUDA-core solver for hours."""
    import synth
    import paper_1505_01348_gb300 as G
    prec = PRECISIONS[args.precision]
    full_pool = [synth.serve_job(j) for j in range(distinct)]
    full = _serve_stream(G, full_pool, prec, full_rate, full_seconds, 16, 64)
    full["mix"] = (f"{distinct} distinct seeded jobs cycled: p in {{32,64,128,256}}, 64^2, 128^2 or 256^2 grid, "
                   "5-50 sources, N=1e4; arrivals Poisson; 200 jobs/s is beyond one GPU for this mix")
    tc_pool = [synth.serve_job_tc(j) for j in range(distinct)]
    tc = _serve_stream(G, tc_pool, prec, tc_rate, tc_seconds, 16, 2 * sm_count())
    tc["mix"] = f"{distinct} distinct seeded jobs cycled: p in {{32,64}}, 64^2 or 128^2 grid, 5-50 sources"
    sample = tc_pool[:6]
    t1 = time.perf_counter()
    for job in sample:
        im = G.Imager.from_job(job, precision=0)
        im.solve()
        im.close()
    per_job = len(sample) / (time.perf_counter() - t1)
    return {"precision": args.precision, "full_mix": full, "tc_subset": tc,
            "per_job_fp32_images_s": per_job,
            "per_job_fp32_sample": f"{len(sample)} jobs of the p <= 64 subset, one img_solve at a time"}


def run_batch(args, channels: int = 64):
    """The uneven 64-channel batch (p in {48, 64, 96}, grids 64^2 .. 128^2,
    wavelength 1 .. 1.5): factor and bounds in one launch per arithmetic
    group, the p <= 64 channels in one solver launch (a CTA each), the p = 96
    channels as solve graphs side by side on their own streams; timed per
    arithmetic after a warm call."""
    import torch
    import synth
    import paper_1505_01348_gb300 as G
    jobs = [synth.batch_channel(c) for c in range(channels)]
    out = {"channels": channels, "p_counts": {str(p): sum(1 for j in jobs if j.p == p) for p in (48, 64, 96)}}
    for name, prec in (("fp32", 0), ("f16x3", 1), ("bf16x3", 2)):
        streams = [torch.cuda.Stream() for _ in jobs]
        ims = [G.Imager(j.ant_xyz, j.l, j.m, j.lam, precision=prec, stream=st.cuda_stream)
               for j, st in zip(jobs, streams)]
        for rep in range(2):
            for im, j in zip(ims, jobs):
                im.set_covariance(j.R, j.N)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.prepare_batch(ims)
            _, infos = G.solve_batch(ims)
            dt = time.perf_counter() - t0
        out[name] = {"s_per_batch": dt, "images_s": channels / dt,
                     "converged": int(sum(i.converged for i in infos))}
        for im in ims:
            im.close()
    return out


# ---------------------------------------------------------------- oracle timing
def oracle_sample(budget_passes: int = 40, seed: int = 2000):
    """Time the FP64 oracle on one image of the same workload: full setup
    (steering, explicit Psi, bounds, PWLS operator) plus the first
    `budget_passes` passes of the Table I loop.  Returns (t_setup, t_per_pass)."""
    import synth
    from oracle import imager as O
    job = synth.mid(seed=seed)
    prm = O.Params(cost=O.COST_PWLS, kappa=6.0, eps_floor=1e-6, max_outer=budget_passes)
    t0 = time.perf_counter()
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    Psi = O.khatri_rao_psi(A)
    bnd = O.bounds(A, Psi, job.R, job.N, prm)
    prob = O.cost_problem(A, Psi, job.R, bnd, prm.cost)
    t1 = time.perf_counter()
    res = O.active_set(prob, bnd.eps, prm, record=False)
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / max(res.outer, 1), res.outer


def oracle_passes_per_image() -> float:
    """Table I passes the oracle itself needs for this workload's image
    (seed 2000), read from the committed oracle record."""
    path = os.path.join(ROOT, "tests", "golden", "mid_pwls.npz")
    try:
        return float(np.load(path)["outer"])
    except OSError:
        return 740.0


def profiled_traffic(B: int):
    """DRAM bytes of one k_solve launch from the committed ncu summary (a
    304-image launch of this workload), scaled to B images; None when absent."""
    path = os.path.join(ROOT, "profiles", "k_solve_f16x3_bench_128x128_p64.md")
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_launch k_solve:"):
                return float(line.split(":")[1]) * B / 304.0
    except OSError:
        pass
    return None


def oracle_sample_large(budget_passes: int = 30, seed: int = 4000):
    """Time the FP64 oracle (streamed operator form: Psi is never stored) on
    one image of the 256x256, p = 288 workload: setup (steering matrix, dirty
    and MVDR images, PWLS operator) plus the first `budget_passes` passes of
    the Table I loop.  Returns (t_setup, t_per_pass, passes)."""
    import synth
    from oracle import imager as O
    job = synth.large(seed=seed)
    prm = O.Params(cost=O.COST_PWLS, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5, max_outer=budget_passes)
    t0 = time.perf_counter()
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    bnd = O.bounds(A, None, job.R, job.N, prm)
    prob = O.cost_problem(A, None, job.R, bnd, prm.cost)
    t1 = time.perf_counter()
    res = O.active_set(prob, bnd.eps, prm, record=False)
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / max(res.outer, 1), res.outer


def oracle_record_large():
    """The oracle's complete image of the 256x256, p = 288 workload (seed
    4000): its Table I passes and wall time, as recorded when
    tests/golden/large_pwls.npz was written; None when absent."""
    path = os.path.join(ROOT, "tests", "golden", "large_pwls.npz")
    try:
        g = np.load(path)
        return {"passes": int(g["outer"]), "lsqr_iters": int(g["lsqr_iters"]),
                "seconds": float(g["oracle_seconds"])}
    except (OSError, KeyError):
        return None


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_line(workload: str, budget_passes: int = 30):
    if workload == "mid":
        ppi = oracle_passes_per_image()
        ts, tp, done = oracle_sample(budget_passes)
        t_img = ts + tp * ppi
        return {"value": 1.0 / t_img, "unit": METRIC, "cores": cpu_cores(), "kind": "oracle",
                "sample": (f"FP64 numpy oracle, one image of the same workload: setup {ts:.1f} s "
                           f"(explicit Psi, bounds, PWLS operator) + first {done} Table I passes "
                           f"at {tp:.3f} s/pass, extrapolated to {ppi:.0f} passes per image "
                           f"(later passes cost more, so this favours the oracle)")}
    rec = oracle_record_large()
    ppi = rec["passes"] if rec else 5600.0
    ts, tp, done = oracle_sample_large(budget_passes)
    t_img = ts + tp * ppi
    line = {"value": 1.0 / t_img, "unit": METRIC, "cores": cpu_cores(), "kind": "oracle",
            "sample": (f"FP64 numpy oracle (streamed operators), one image of the same workload: "
                       f"setup {ts:.1f} s + first {done} Table I passes at {tp:.3f} s/pass, "
                       f"extrapolated to the oracle's {ppi:.0f} passes per image (later passes "
                       f"cost more: this favours the oracle)")}
    if rec:
        line["complete_image"] = {"value": 1.0 / rec["seconds"], "unit": METRIC, "seconds": rec["seconds"],
                                  "passes": rec["passes"], "lsqr_iters": rec["lsqr_iters"],
                                  "where": "the oracle's full solve of seed 4000 when its stored record was "
                                           "written (8-core x86 build host, multithreaded BLAS)"}
    return line


def run_reference(args):
    """Reference arm: the FP64 oracle timed as it stands on the host cores."""
    wl = args.workload
    per_step = []
    if wl == "mid":
        ppi = oracle_passes_per_image()
        for k in range(args.warmup + args.steps):
            ts, tp, done = oracle_sample(budget_passes=12)
            if k >= args.warmup:
                per_step.append(ts + tp * ppi)
        sample = f"per step: oracle setup + 12 Table I passes on one image, extrapolated to {ppi:.0f} passes per image"
    else:
        rec = oracle_record_large()
        ppi = rec["passes"] if rec else 5600.0
        for k in range(args.warmup + args.steps):
            ts, tp, done = oracle_sample_large(budget_passes=8)
            if k >= args.warmup:
                per_step.append(ts + tp * ppi)
        sample = (f"per step: streamed-oracle setup + 8 Table I passes on one image, extrapolated to "
                  f"{ppi:.0f} passes per image (favours the oracle)")
        if rec:
            sample += (f"; the oracle's complete image of this workload took {rec['seconds']:.0f} s "
                       f"({rec['passes']} passes) on the 8-core build host")
    t = float(np.mean(per_step))
    val = 1.0 / t
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": METRIC, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[wl], "batch": 1, "device": "cpu"},
        "cpu_baseline": {"value": val, "unit": METRIC, "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=0, help="images per step (0: two per SM)")
    ap.add_argument("--precision", default="f16x3", choices=sorted(PRECISIONS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-ops", action="store_true")
    ap.add_argument("--ops-only", action="store_true",
                    help="only the operator and full-image LS measurements (one JSON line)")
    ap.add_argument("--precision-only", action="store_true",
                    help="only the arithmetic sweep against FP64 (one JSON line)")
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import torch
    if args.precision_only:
        if rank == 0:
            import paper_1505_01348_gb300 as G
            G.load()
            print(json.dumps({"precision_sweep": run_precision(args)}), flush=True)
        return
    if args.ops_only:
        if rank == 0:
            import paper_1505_01348_gb300 as G
            G.load()
            print(json.dumps({"operators": run_operators(args), "ls_image": run_ls_images(args)}), flush=True)
        return
    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world)
    mid = None
    if args.workload == "large" and not args.no_ops and world == 1:
        # the 128x128, p = 64 workload as a second, named measurement
        import copy
        a2 = copy.copy(args)
        a2.workload, a2.steps, a2.warmup, a2.batch, a2.no_e2e = "mid", 3, 3, 0, True
        mid = run_ours(a2, rank, world)
    if rank == 0:
        line = summarize(r, args, world)
        if mid is not None:
            m = summarize(mid, a2, world)
            line["mid_workload"] = {k: m[k] for k in ("value", "unit", "ms_per_step", "config", "roofline",
                                                    "converged", "mean_outer_passes", "gpu_launches")}
        if not args.no_ops and world == 1:
            line["operators"] = run_operators(args)
            if PRECISIONS[args.precision] != 0:
                line["ls_image"] = run_ls_images(args)
            line["precision_sweep"] = run_precision(args)
        if not args.no_serve and world == 1:
            line["serve"] = run_serve(args)
        if not args.no_ops and world == 1:
            line["batch_64_channels"] = run_batch(args)
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline_line(args.workload)
        if not args.no_ops and world == 1:
            try:
                line["snapshots"] = run_snapshots(args)
            except Exception as e:                   # reported in the line, never fatal
                line["snapshots"] = {"error": f"{type(e).__name__}: {e}"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def summarize(r, args, world):
    """The JSON line of one run_ours result."""
    K = args.steps
    B = r["B"]
    total = r["total"]
    value = world * B * K / total
    t_solve = float(np.mean(r["t_solve"]))
    t_prep = float(np.mean(r["t_prep"]))
    flops = float(np.mean(r["flops"]))
    mhz = r["clocks"]["sm_max_mhz"] or 2070.0
    achieved = flops / t_solve / 1e12
    pk = measured_peaks()
    wl = r["workload"]
    if args.precision == "fp32":
        bound, peak = "alu", fp32_alu_peak_tflops(r["sms"], mhz)
        basis = f"FP32 CUDA cores: {r['sms']} SMs x 128 lanes x 2 flops x {mhz:.0f} MHz"
    else:
        bound = "tensor"
        if pk.get("bf16_tflops_sustained"):
            peak = float(pk["bf16_tflops_sustained"])
            basis = ("measured dense BF16 tensor peak, sustained (FP16 runs at the BF16 rate); "
                     "achieved counts algorithmic flops, the split products execute 3x")
        else:
            peak = 1700.0
            basis = "fallback sustained BF16 tensor peak (no measured peaks file)"
    if wl == "large":
        kernel = "k_ws_* (the solve graph: all its kernels, B solves in flight)"
        traffic = None
        launches = int(sum(r["launches"][-1])) if r.get("launches") else None
    else:
        kernel = "k_solve"
        traffic = profiled_traffic(B) if args.precision == "f16x3" else None
        launches = 4 * K
    return {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total / K * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else f"{args.precision}+f32acc",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[wl], "batch_per_gpu": B, "n_l": r["n"], "n_m": r["n"], "p": r["p"],
                   "cost": "pwls", "bound": "mvdr", "precision": args.precision,
                   "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"dp{world} (independent images)"},
        "roofline": {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": basis + " (of measured)" if pk else basis},
        "solve_ms_per_step": t_solve * 1e3,
        "prepare_ms_per_step": t_prep * 1e3,
        "prepare_tflops": r["prep_flops"] / t_prep / 1e12,
        "converged": r["conv"], "mean_outer_passes": r["outer"],
        "gpu_launches": launches if launches is not None else 4 * K,
        "clocks": r["clocks"],
        "e2e": r["e2e"],
    }


if __name__ == "__main__":
    main()
