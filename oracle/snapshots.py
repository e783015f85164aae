"""FP64 CPU oracle of the imager over K > 1 snapshots.

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import or run this module;
no product code calls it or shares code with it.

The single-snapshot oracle (``oracle.imager``) fixes K = 1.  This module
follows the paper's K-snapshot data model and bounds, reusing the
single-snapshot steering, Khatri-Rao, LSQR and active-set steps unchanged:

* stacked model r = Psi sigma + r_n with Psi = [conj(A_k) o A_k]_k
  (Sec. II, eq. vectRtotal) and r_hat = [vect(R_hat_k)]_k (eq. def:brh);
* MF dirty image (1/K) sum_k a_{i,k}^H R_hat_k a_{i,k} (Sec. III-C);
* unbiased MVDR bound C / ((1/K) sum_k a_{i,k}^H R_hat_k^{-1} a_{i,k})
  (Sec. III-D) and the preconditioner D = (1/(K C)) diag^2(A^H R^{-1} A)
  (eq. D), i.e. D_ii = (sum_k h_{i,k})^2 / (K C);
* the tightest linear-beamformer bound, ASSC: min_k 1/h_{i,k}
  (eq. ASSC0, Appendix B), with the bias constant C applied per snapshot;
* variances of Appendix A for K snapshots;
* CLS cost 1/(2K) ||r_hat - Psi sigma||^2 (eq. CLS) and the PWLS cost with
  per-snapshot whitening (eq. preWLS).

Readings where the paper is silent or ambiguous:

* The weighting (R_hat^{-T/2} kron R_hat^{-1/2}) of eq. def:vecfWLS is
  written with the block-diagonal R_hat of eq. blockdiagtilde, whose
  Kronecker product does not match the length K p^2 of r_hat.  It is read
  as acting on each snapshot's block: r_hat_k is weighted with
  (R_hat_k^{-T/2} kron R_hat_k^{-1/2}).  This is the reading under which the
  WLS dirty image is the MVDR image, as the paper states, and under which
  eq. D is the Jacobi preconditioner.
* Var(sigma_MVDR) (Appendix A) is evaluated with h_{i,k} / C standing in for
  a^H R_k^{-1} a, as the single-snapshot oracle does; for K = 1 this is
  sigma_MVDR^2 / (N - p - 1).
* The ASSC bound has no variance formula in the paper: it is offered
  uninflated only (INFLATE_STD with it raises ValueError).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from oracle import imager as O

BOUND_ASSC = 2


def steering_stack(ant_xyz_k: np.ndarray, l: np.ndarray, m: np.ndarray,
                   lam: float) -> list:
    """A_k (p x Q) for each snapshot k: the single-snapshot steering model
    with snapshot k's antenna positions (Sec. II: the response a_{q,k}
    changes with k as the Earth turns)."""
    return [O.steering_matrix(ant_xyz_k[k], l, m, lam) for k in range(ant_xyz_k.shape[0])]


def khatri_rao_stack(As: list) -> np.ndarray:
    """Psi = [conj(A_1) o A_1; ...; conj(A_K) o A_K] (eq. vectRtotal), (K p^2) x Q."""
    return np.concatenate([O.khatri_rao_psi(A) for A in As], axis=0)


def vect_stack(Rs: np.ndarray) -> np.ndarray:
    """r_hat = [vect(R_hat_1); ...; vect(R_hat_K)] (eq. def:brh)."""
    return np.concatenate([O.vect(Rs[k]) for k in range(Rs.shape[0])]).astype(np.complex128)


@dataclass
class BoundsK(O.Bounds):
    hk: np.ndarray = None      # (K, Q): h_{i,k} = a_{i,k}^H R_hat_k^{-1} a_{i,k}
    assc: np.ndarray = None    # C / max_k h_{i,k}  (eq. ASSC0)
    K: int = 1


def bounds_k(As: list, Psi: np.ndarray, Rs: np.ndarray, N: int, prm: O.Params) -> BoundsK:
    """Dirty images, bounds, preconditioner and thresholds for K snapshots.

    * sigma_MF = (1/K) Psi^H r_hat                          Sec. III-C
    * sigma_MVDR = C K / sum_k h_{i,k}                       Sec. III-D, eq. C
    * D_ii = (sum_k h_{i,k})^2 / (K C)                       eq. D
    * sigma_ASSC = C / max_k h_{i,k}                         eq. ASSC0
    * Var(sigma_MF) = (1/(N K^2)) sum_k (a_{i,k}^H R_hat_k a_{i,k})^2     Appendix A
    * Var(sigma_MVDR) = K^2 C^2 sum_k h^2 / ((N-p-1) (sum_k h)^4)       Appendix A
    * gamma and eps as for one snapshot (Sec. III-D, Appendix A, Sec. IV-C)."""
    K = len(As)
    p = As[0].shape[0]
    dirty = np.real(Psi.conj().T @ vect_stack(Rs)) / K
    mf_k = np.stack([np.real(np.einsum("ki,kl,li->i", As[k].conj(), Rs[k], As[k]))
                     for k in range(K)])
    hk = np.stack([O.mvdr_h(As[k], Rs[k]) for k in range(K)])
    hs = hk.sum(axis=0)
    C = O.bias_constant(N, p, prm.bias_c)
    mv = C * K / hs
    D = hs * hs / (K * C)
    assc = C / hk.max(axis=0)
    std_mf = np.sqrt(np.sum(mf_k * mf_k, axis=0) / N) / K
    dof = N - p - 1
    if dof > 0:
        std_mv = K * C * np.sqrt(np.sum(hk * hk, axis=0)) / (hs * hs * math.sqrt(dof))
    else:
        std_mv = np.full_like(mv, np.inf)
    if prm.bound == O.BOUND_MF:
        base, sd = dirty, std_mf
    elif prm.bound == O.BOUND_MVDR:
        base, sd = mv, std_mv
    elif prm.bound == BOUND_ASSC:
        base, sd = assc, None
    else:
        raise ValueError("unknown bound")
    if prm.inflate == O.INFLATE_RATIO:
        gamma = (1.0 + prm.alpha) * base
    elif prm.inflate == O.INFLATE_STD:
        if sd is None:
            raise ValueError("the ASSC bound has no variance to inflate by")
        gamma = base + prm.alpha * sd
    else:
        gamma = base.copy()
    if prm.cost == O.COST_LS:
        eps = np.maximum(prm.kappa * std_mf, prm.eps_floor * float(np.max(dirty)))
    else:
        eps = np.maximum(prm.kappa * std_mv, prm.eps_floor * float(np.max(mv)))
    return BoundsK(dirty, hs, mv, D, std_mf, std_mv, gamma, eps, C, hk=hk, assc=assc, K=K)


def cost_problem_k(As: list, Psi: np.ndarray, Rs: np.ndarray, bnd: BoundsK,
                   cost: int) -> O.CostProblem:
    """min 1/2 ||b - M x||^2, 0 <= x <= upper, for K snapshots.

    CLS (eq. CLS): 1/(2K) ||r_hat - Psi sigma||^2, i.e. M = Psi / sqrt(K),
    b = r_hat / sqrt(K); the gradient at sigma = 0 is then minus the MF dirty
    image, as for one snapshot.
    PWLS (eq. preWLS): block k of M is conj(L_k^{-1} A_k) o (L_k^{-1} A_k) D^{-1}
    and block k of b is vect(L_k^{-1} R_hat_k L_k^{-H}), with R_hat_k = L_k L_k^H
    (per-snapshot whitening; the weighted norm equals the one with
    R_hat_k^{-1/2}); x = D sigma."""
    K = len(As)
    if cost == O.COST_LS:
        s = 1.0 / math.sqrt(K)
        return O.CostProblem(Psi * s, vect_stack(Rs) * s, bnd.gamma.copy(),
                             np.ones_like(bnd.gamma))
    p = As[0].shape[0]
    Mb, bb = [], []
    for k in range(K):
        Lc = O.cholesky_lower(Rs[k])
        Linv = sla.solve_triangular(Lc, np.eye(p, dtype=np.complex128), lower=True)
        Mb.append(O.khatri_rao_psi(Linv @ As[k]))
        bb.append(O.vect(Linv @ Rs[k] @ Linv.conj().T))
    M = np.concatenate(Mb, axis=0) / bnd.D[None, :]
    return O.CostProblem(M, np.concatenate(bb), bnd.D * bnd.gamma, 1.0 / bnd.D)


@dataclass
class ImageResultK:
    bounds: BoundsK
    solve: O.SolveResult


def image_k(ant_xyz_k, l, m, lam, Rs, N, prm: O.Params) -> ImageResultK:
    """Full pipeline for one K-snapshot job: bounds, then the active set of
    Table I with LSQR on the stacked operator."""
    As = steering_stack(ant_xyz_k, l, m, lam)
    Psi = khatri_rao_stack(As)
    bnd = bounds_k(As, Psi, Rs, N, prm)
    prob = cost_problem_k(As, Psi, Rs, bnd, prm.cost)
    res = O.active_set(prob, bnd.eps, prm)
    return ImageResultK(bnd, res)


def image_snapshot_job(job, prm: O.Params) -> ImageResultK:
    return image_k(job.ant_xyz, job.l, job.m, job.lam, job.R, job.N, prm)
