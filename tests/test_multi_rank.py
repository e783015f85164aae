"""Multi-GPU host logic on CPU ranks (gloo, world size 2).

Across images: images are independent, so ranks solve disjoint seeds and the
job time is the max over ranks; no data-path collective exists.
Within one image: the pixels are sharded over the ranks, and Table I with
LSQR runs with one all-reduce of the p x p forward sum per product, scalar
all-reduces for LSQR's norms and a global (value, index) minimum for each
decision; its result equals the single-rank oracle's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.rank_seeds(rank, 5)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    t = bench.reduce_max(1.0 + rank)
    # each rank's inputs are generated locally from its own seeds
    import synth
    job = synth.custom(seeds[0], 6, 5, 4, 2, 100)
    hs = [None] * world
    dist.all_gather_object(hs, float(abs(job.R).sum()))
    if rank == 0:
        out.put((gathered, t, hs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, t, hs = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert set(gathered[0]).isdisjoint(gathered[1])
    assert len(gathered[0]) == len(gathered[1]) == 5
    assert t == 2.0
    assert hs[0] != hs[1]


def test_single_rank_max_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5


# ---------------------------------------------------------------- pixel sharding
# Within-image sharding of the method across ranks: rank r owns the pixels
# i with i % world == r.  The forward Psi x over a pixel set is the sum of
# the ranks' partial p x p matrices (one all-reduce of p^2 complex); the
# adjoint needs only the replicated p x p operand (no exchange); LSQR's
# vector norms are scalar all-reduces; the multiplier test and the step pick
# a global (value, index) minimum.  The sets and every scalar are replicated,
# so every rank takes the same decisions.  This runs Table I sharded on CPU
# ranks with the oracle's streamed operators and compares with one rank.

def _sharded_solve(rank, world, job, cost):
    import numpy as np
    from oracle import imager as O
    prm = O.Params(cost=cost, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5)
    A = O.steering_matrix(job.ant_xyz, job.l, job.m, job.lam)
    bnd = O.bounds(A, None, job.R, job.N, prm)
    prob = O.cost_problem(A, None, job.R, bnd, cost)
    Q = prob.Q
    own = np.arange(Q) % world == rank

    def allsum(x):
        t = torch.from_numpy(np.ascontiguousarray(np.atleast_1d(x)).view(np.float64).copy())
        dist.all_reduce(t)
        out = t.numpy().view(np.complex128 if np.iscomplexobj(x) else np.float64)
        return out if np.ndim(x) else float(out[0])

    def argmin_global(val, idx):
        objs = [None] * world
        dist.all_gather_object(objs, (float(val), int(idx)))
        return min(objs)

    def fwd(S, xS):                                   # M[:, S] x_S, sharded over S
        m = own[S]
        part = prob.apply(S[m], xS[m]) if m.any() else np.zeros(prob.b.shape, np.complex128)
        return allsum(part)

    def lsqr(F, b):                                   # LSQR on M[:, F], F sharded
        mine = own[F]
        op = prob.cols(F[mine])
        n = F.size
        x = np.zeros(n)
        beta = float(np.linalg.norm(b))
        bnorm = beta
        if beta == 0.0:
            return x, 0
        u = b / beta
        v = np.zeros(n)
        v[mine] = op.rmatvec(u)
        alpha = np.sqrt(allsum(np.sum(v[mine] ** 2)))
        if alpha == 0.0:
            return x, 0
        v /= alpha
        w = v.copy()
        phibar, rhobar, anorm2 = beta, alpha, 0.0
        maxit = 4 * n + 20
        it = 0
        for it in range(1, maxit + 1):
            u = fwd(F, v) - alpha * u
            beta = float(np.linalg.norm(u))
            if beta > 0.0:
                u = u / beta
            anorm2 += alpha * alpha + beta * beta
            vn = np.zeros(n)
            vn[mine] = op.rmatvec(u)
            v = vn - beta * v
            alpha = np.sqrt(allsum(np.sum(v[mine] ** 2)))
            if alpha > 0.0:
                v = v / alpha
            rho = np.hypot(rhobar, beta)
            c, s = rhobar / rho, beta / rho
            theta = s * alpha
            rhobar = -c * alpha
            phi = c * phibar
            phibar = s * phibar
            x = x + (phi / rho) * w
            w = v - (theta / rho) * w
            xnorm = np.sqrt(allsum(np.sum(x[mine] ** 2)))
            anorm = np.sqrt(anorm2)
            if phibar <= prm.lsqr_btol * bnorm + prm.lsqr_atol * anorm * xnorm:
                break
            if phibar * alpha * abs(c) <= prm.lsqr_atol * anorm * phibar:
                break
        # the ranks hold x on their own pixels; gather the rest (replicated state)
        return allsum(np.where(mine, x, 0.0)), it

    x = np.zeros(Q)
    sets = np.full(Q, O.SET_L, np.int8)
    up = prob.upper
    flag, i_min, outer, events = True, -1, 0, []
    tau = prm.feas_tol
    while outer < 10 * Q + 100:
        outer += 1
        if flag:
            F = np.nonzero(sets == O.SET_F)[0]
            U = np.nonzero(sets == O.SET_U)[0]
            z = np.zeros(0)
            if F.size:
                b_sub = prob.b - fwd(U, x[U])
                z, _ = lsqr(F, b_sub)
            if np.all(z >= -tau * up[F]) and np.all(z <= (1.0 + tau) * up[F]):
                x[F] = np.clip(z, 0.0, up[F])
                flag = False
                S = np.nonzero(x)[0]
                r = prob.b - fwd(S, x[S])
                g = np.zeros(Q)
                g[own] = -prob.cols(np.nonzero(own)[0]).rmatvec(r)
                lam = np.where(sets == O.SET_U, -g, g)
                cand = own & (sets != O.SET_F) & (lam < -bnd.eps)
                lv, li = (float(lam[cand].min()), int(np.nonzero(cand)[0][np.argmin(lam[cand])])) \
                    if cand.any() else (np.inf, Q)
                lv, li = argmin_global(lv, li)
                if li == Q:
                    break
                i_min = li
            else:
                pdir = z - x[F]
                mu = np.full(F.size, np.inf)
                mu[pdir > 0] = (up[F][pdir > 0] - x[F][pdir > 0]) / pdir[pdir > 0]
                mu[pdir < 0] = -x[F][pdir < 0] / pdir[pdir < 0]
                m = own[F]
                loc = (float(mu[m].min()), int(F[m][np.argmin(mu[m])])) if m.any() else (np.inf, Q)
                mu_max, ic = argmin_global(*loc)
                k = int(np.nonzero(F == ic)[0][0])
                x[F] = x[F] + mu_max * pdir
                sets[ic] = O.SET_U if pdir[k] > 0 else O.SET_L
                x[ic] = up[ic] if pdir[k] > 0 else 0.0
                events.append(("clamp", ic, int(sets[ic])))
                flag = True
        else:
            sets[i_min] = O.SET_F
            events.append(("free", i_min))
            flag = True
    return prob.to_sigma * x, sets, events, outer


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    res = []
    for seed, cost in ((61, 1), (62, 0)):
        job = synth.custom(seed, 10, 11, 9, 4, 900, radius=4.0, snr_db=0.0)
        res.append(_sharded_solve(rank, world, job, cost))
    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_pixel_sharded_solve_equals_one_rank():
    import numpy as np
    import synth
    from oracle import imager as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for k, (seed, cost) in enumerate(((61, 1), (62, 0))):
        job = synth.custom(seed, 10, 11, 9, 4, 900, radius=4.0, snr_db=0.0)
        ref = O.image_job(job, O.Params(cost=cost, kappa=6.0, eps_floor=1e-6, feas_tol=1e-5), streamed=True)
        for r in (0, 1):
            sigma, sets, events, outer = got[r][k]
            assert events == ref.solve.events
            assert outer == ref.solve.outer
            np.testing.assert_array_equal(sets, ref.solve.sets)
            assert np.linalg.norm(sigma - ref.solve.sigma) <= 1e-9 * np.linalg.norm(ref.solve.sigma)
