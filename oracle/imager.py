"""FP64 CPU oracle of the bounded least-squares imager.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import or run this
module.  The product path (the CUDA library and its Python binding) never
calls it and shares no code with it.

Everything is plain numpy/scipy in float64 / complex128, written to be read
against the paper (Sardarabadi, Leshem, van der Veen, "Radio astronomical
image formation using constrained least squares and Krylov subspaces"):

* steering vectors, Sec. II and Sec. IV-D steering model, unit norm;
* the Khatri-Rao operator Psi = conj(A) o A built column by column
  (Sec. III-A, eq. bAt; properties listed in Sec. I notation);
* matched-filter dirty image, eq. mfdimg;
* MVDR bound with bias constant C and variances, eq. wmvdr, eq. UBMVDRV,
  eq. D and Appendix A;
* CLS (eq. CLS) and preconditioned WLS (eq. preWLS) costs, gradients
  eq. gls / eq. gmvdr;
* the active-set method of Table I with the step of eq. mumax;
* LSQR (Paige & Saunders 1982, referenced in Sec. V-A) on the
  Golub-Kahan recurrences eq. initbeta .. eq. lanczos.

Two equivalent forms of the operator are available.  The explicit form builds
Psi (or M) column by column and multiplies by it; it is the form every pin
starts from.  The streamed form never stores Psi (Sec. V-B: the operator is
applied through the steering vectors): Psi x = vect(A diag(x) A^H) and
Psi^H vect(U) = Re vecdiag(A^H U A), the Khatri-Rao properties of the
notation section, evaluated on the columns a product needs.  It is what
makes the 256 x 256, p = 288 workload computable (its explicit Psi would
hold 87 GB).

Readings where the paper is silent or ambiguous (documented beside each use):
steering sign -j; K = 1 snapshot; detection threshold eps_i = kappa * std_i
with a relative floor; ties resolved to the smallest pixel index; cold-start
LSQR; non-strict feasibility.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

COST_LS = 0
COST_PWLS = 1
BOUND_MF = 0
BOUND_MVDR = 1
INFLATE_NONE = 0
INFLATE_RATIO = 1     # gamma = (1 + alpha) * dirty              (Sec. III-D)
INFLATE_STD = 2       # gamma = dirty + alpha * std(dirty)        (Appendix A)

SET_L, SET_U, SET_F = 0, 1, 2


# ---------------------------------------------------------------- Sec. II
def pixel_directions(l: np.ndarray, m: np.ndarray):
    """Pixel i = i_l + n_l * i_m (column-major vect of the image)."""
    n_l = l.shape[0]
    Q = n_l * m.shape[0]
    idx = np.arange(Q)
    ll = l[idx % n_l]
    mm = m[idx // n_l]
    nn = np.sqrt(np.maximum(0.0, 1.0 - ll * ll - mm * mm))
    return ll, mm, nn


def steering_matrix(ant_xyz: np.ndarray, l: np.ndarray, m: np.ndarray,
                    lam: float) -> np.ndarray:
    """A (p x Q): a_i = p^{-1/2} exp(-j 2 pi <x_k, s_i> / lam).

    Sec. IV-D gives the model with +j; the sign is a convention that only
    conjugates every covariance, and -j is used on both the data and the
    imaging side.  Normalisation a_i^H a_i = 1 (Sec. III-A)."""
    p = ant_xyz.shape[0]
    ll, mm, nn = pixel_directions(l, m)
    phase = -2.0 * np.pi * (np.outer(ant_xyz[:, 0], ll) + np.outer(ant_xyz[:, 1], mm)
                            + np.outer(ant_xyz[:, 2], nn)) / lam
    return np.exp(1j * phase) / math.sqrt(p)


def vect(X: np.ndarray) -> np.ndarray:
    """Column stacking (notation section)."""
    return X.reshape(-1, order="F")


def unvect(x: np.ndarray, p: int) -> np.ndarray:
    return x.reshape(p, p, order="F")


# ---------------------------------------------------------------- Sec. III
def khatri_rao_psi(A: np.ndarray) -> np.ndarray:
    """Psi = conj(A) o A (eq. bAt with K = 1): column i is kron(conj(a_i), a_i),
    which equals vect(a_i a_i^H)."""
    p, Q = A.shape
    Psi = np.empty((p * p, Q), dtype=np.complex128)
    for i in range(Q):
        Psi[:, i] = np.kron(A[:, i].conj(), A[:, i])
    return Psi


# Pixels per block in the streamed products: a memory bound only; every
# pixel's value is computed on its own, so blocking changes no arithmetic.
STREAM_BLOCK = 4096


def psi_apply(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Psi x = vect(A diag(x) A^H) without forming Psi (notation section:
    (conj(B) o A) x = vect(A diag(x) B^H), here with B = A)."""
    return vect((A * x[None, :]) @ A.conj().T)


def psi_adjoint(A: np.ndarray, U: np.ndarray) -> np.ndarray:
    """Psi^H vect(U) = Re vecdiag(A^H U A) without forming Psi (notation
    section: (conj(B) o A)^H vect(U) = vecdiag(A^H U B), here B = A); the
    imaginary part vanishes for Hermitian U and is dropped explicitly."""
    Q = A.shape[1]
    out = np.empty(Q)
    for i0 in range(0, Q, STREAM_BLOCK):
        Ab = A[:, i0:i0 + STREAM_BLOCK]
        out[i0:i0 + Ab.shape[1]] = np.real(np.sum(Ab.conj() * (U @ Ab), axis=0))
    return out


class KhatriRaoCols:
    """The operator M_S = (conj(B_S) o B_S) diag(dinv_S) on a pixel subset S
    in streamed form (Sec. V-B): B_S = T A_S with T = I (CLS) or L^{-1}
    (PWLS, by the mixed-product rule), dinv = 1 (CLS) or 1/D (PWLS).
      matvec(v)  = vect(B_S diag(dinv_S v) B_S^H)
      rmatvec(u) = dinv_S * Re vecdiag(B_S^H U B_S),  U = unvect(u)."""

    def __init__(self, B: np.ndarray, dinv: np.ndarray):
        self.B = B
        self.dinv = dinv
        self.shape = (B.shape[0] * B.shape[0], B.shape[1])

    def matvec(self, v: np.ndarray) -> np.ndarray:
        return psi_apply(self.B, self.dinv * v)

    def rmatvec(self, u: np.ndarray) -> np.ndarray:
        return self.dinv * psi_adjoint(self.B, unvect(u, self.B.shape[0]))


def dirty_mf(Psi: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Matched-filter dirty image, eq. mfdimg: (1/K) Psi^H r_hat, K = 1."""
    return np.real(Psi.conj().T @ vect(R))


def cholesky_lower(R: np.ndarray) -> np.ndarray:
    """R = L L^H (raises numpy.linalg.LinAlgError when R is not PD)."""
    return np.linalg.cholesky(R)


def mvdr_h(A: np.ndarray, R: np.ndarray) -> np.ndarray:
    """h_i = a_i^H R^{-1} a_i via the Cholesky factor: ||L^{-1} a_i||^2."""
    Lc = cholesky_lower(R)
    B = sla.solve_triangular(Lc, A, lower=True)
    return np.sum(np.abs(B) ** 2, axis=0)


def bias_constant(N: int, p: int, bias_c: int) -> float:
    """C = N/(N-p) (Appendix A, eq. C) when requested, else 1."""
    return float(N) / float(N - p) if bias_c else 1.0


@dataclass
class Bounds:
    dirty: np.ndarray        # MF dirty image sigma_MF
    h: np.ndarray            # a_i^H R^{-1} a_i
    mvdr: np.ndarray         # C / h  (eq. wmvdr with K=1, bias-corrected form)
    D: np.ndarray            # h^2 / C  (eq. D, K = 1)
    std_mf: np.ndarray       # sqrt(Var(sigma_MF)) (Appendix A)
    std_mvdr: np.ndarray     # sqrt(Var(sigma_MVDR)) (Appendix A)
    gamma: np.ndarray        # upper bound actually used, in sigma units
    eps: np.ndarray          # detection threshold for the chosen cost
    C: float


@dataclass
class Params:
    cost: int = COST_PWLS
    bound: int = BOUND_MVDR
    bias_c: int = 0
    inflate: int = INFLATE_NONE
    alpha: float = 6.0
    kappa: float = 6.0
    eps_floor: float = 1e-12     # eps_i >= eps_floor * max(dirty image of the cost)
    lsqr_atol: float = 1e-12
    lsqr_btol: float = 1e-12
    lsqr_maxit: int = 0          # 0 -> 4 f + 20
    max_outer: int = 0           # 0 -> 10 Q + 100 passes of the Table I loop
    feas_tol: float = 0.0        # z within feas_tol * upper of a bound is feasible


def bounds(A: np.ndarray, Psi: np.ndarray, R: np.ndarray, N: int,
           prm: Params) -> Bounds:
    """Dirty images, upper bounds, preconditioner D and thresholds.

    * sigma_MF = Psi^H vect(R)                      eq. mfdimg
      (Psi = None: the streamed form Re vecdiag(A^H R A))
    * sigma_MVDR = C / (a^H R^{-1} a)               Sec. III-D (unbiased MVDR, K=1)
    * D = (1/(K C)) diag^2(A^H R^{-1} A)            eq. D
    * Var(sigma_MF,i) = (a^H R a)^2 / N             Appendix A (K=1, R -> R_hat)
    * Var(sigma_MVDR,i) = sigma_MVDR,i^2 / (N-p-1)  Appendix A (K=1, with the
      unbiased estimate h/C plugged in for a^H R^{-1} a)
    * gamma: the chosen dirty image, optionally inflated (Sec. III-D or
      Appendix A);  eps_i = kappa * std_i of the cost's dirty image (Sec. IV-C)."""
    p = A.shape[0]
    dirty = dirty_mf(Psi, R) if Psi is not None else psi_adjoint(A, R)
    h = mvdr_h(A, R)
    C = bias_constant(N, p, prm.bias_c)
    mv = C / h
    D = h * h / C
    std_mf = dirty / math.sqrt(N)
    dof = N - p - 1
    std_mv = mv / math.sqrt(dof) if dof > 0 else np.full_like(mv, np.inf)
    if prm.bound == BOUND_MF:
        base, sd = dirty, std_mf
    else:
        base, sd = mv, std_mv
    if prm.inflate == INFLATE_RATIO:
        gamma = (1.0 + prm.alpha) * base
    elif prm.inflate == INFLATE_STD:
        gamma = base + prm.alpha * sd
    else:
        gamma = base.copy()
    if prm.cost == COST_LS:
        eps = prm.kappa * std_mf
        eps = np.maximum(eps, prm.eps_floor * float(np.max(dirty)))
    else:
        eps = prm.kappa * std_mv
        eps = np.maximum(eps, prm.eps_floor * float(np.max(mv)))
    return Bounds(dirty, h, mv, D, std_mf, std_mv, gamma, eps, C)


# ---------------------------------------------------------------- cost operators
@dataclass
class CostProblem:
    """min 1/2 ||b - M x||^2 s.t. 0 <= x <= upper (eq. CLS or eq. preWLS).

    CLS:  M = Psi,             b = vect(R),        x = sigma,    upper = gamma.
    PWLS: M = W Psi D^{-1},    b = W vect(R),      x = D sigma,  upper = D gamma,
          with W = conj(L^{-1}) kron L^{-1}.  W replaces R^{-T/2} kron R^{-1/2}:
          ||W y|| = ||(R^{-T/2} kron R^{-1/2}) y|| for every y because
          W^H W = R^{-T} kron R^{-1}, so cost, gradient and optimum coincide.
    ``to_sigma`` maps the solver variable back to the image (sigma = D^{-1} x)."""
    M: np.ndarray | None
    b: np.ndarray
    upper: np.ndarray
    to_sigma: np.ndarray
    # streamed form (M is None): M = (conj(B) o B) diag(dinv), B = T A
    B: np.ndarray | None = None
    dinv: np.ndarray | None = None

    @property
    def Q(self) -> int:
        return self.M.shape[1] if self.M is not None else self.B.shape[1]

    def cols(self, S: np.ndarray):
        """M[:, S]: a matrix in the explicit form, a KhatriRaoCols otherwise."""
        if self.M is not None:
            return self.M[:, S]
        return KhatriRaoCols(self.B[:, S], self.dinv[S])

    def apply(self, S: np.ndarray, xS: np.ndarray) -> np.ndarray:
        """M[:, S] @ x_S."""
        if self.M is not None:
            return self.M[:, S] @ xS
        return KhatriRaoCols(self.B[:, S], self.dinv[S]).matvec(xS)

    def adjoint(self, r: np.ndarray) -> np.ndarray:
        """Re(M^H r) over every pixel."""
        if self.M is not None:
            return np.real(self.M.conj().T @ r)
        return KhatriRaoCols(self.B, self.dinv).rmatvec(r)


def cost_problem(A: np.ndarray, Psi: np.ndarray | None, R: np.ndarray, bnd: Bounds,
                 cost: int) -> CostProblem:
    """Psi = None selects the streamed form (Psi and M never stored)."""
    p = R.shape[0]
    if cost == COST_LS:
        if Psi is None:
            return CostProblem(None, vect(R).astype(np.complex128), bnd.gamma.copy(),
                               np.ones_like(bnd.gamma), B=A, dinv=np.ones_like(bnd.gamma))
        return CostProblem(Psi, vect(R).astype(np.complex128), bnd.gamma.copy(),
                           np.ones_like(bnd.gamma))
    Lc = cholesky_lower(R)
    Linv = sla.solve_triangular(Lc, np.eye(p, dtype=np.complex128), lower=True)
    if Psi is None:
        return CostProblem(None, vect(Linv @ R @ Linv.conj().T), bnd.D * bnd.gamma, 1.0 / bnd.D,
                           B=Linv @ A, dinv=1.0 / bnd.D)
    # W Psi = (conj(L^-1) kron L^-1)(conj(A) o A) = conj(L^-1 A) o (L^-1 A): the
    # mixed-product rule for Khatri-Rao products (notation section).  The
    # explicit Kronecker route is checked against this one in the tests.
    M = khatri_rao_psi(Linv @ A) / bnd.D[None, :]
    b = vect(Linv @ R @ Linv.conj().T)           # W vect(R) = vect(L^-1 R L^-H)
    return CostProblem(M, b, bnd.D * bnd.gamma, 1.0 / bnd.D)


def gradient(prob: CostProblem, x: np.ndarray) -> np.ndarray:
    """g(x) = -M^H (b - M x), eq. gWLS specialised in eq. gls / eq. gmvdr
    (K = 1).  M^H of a vectorised Hermitian matrix is real; the real part is
    taken explicitly."""
    if prob.M is not None:
        r = prob.b - prob.M @ x
        return -np.real(prob.M.conj().T @ r)
    S = np.nonzero(x)[0]                 # M x = M_S x_S: the other terms are zero
    r = prob.b - prob.apply(S, x[S])
    return -prob.adjoint(r)


# ---------------------------------------------------------------- Sec. V-A
@dataclass
class LsqrResult:
    x: np.ndarray
    iters: int
    istop: int
    rnorm: float
    arnorm: float


def _mv(M, v):
    return M @ v if isinstance(M, np.ndarray) else M.matvec(v)


def _rmv(M, u):
    return np.real(M.conj().T @ u) if isinstance(M, np.ndarray) else M.rmatvec(u)


def lsqr(M, b: np.ndarray, atol: float, btol: float,
         maxit: int) -> LsqrResult:
    """LSQR for min ||b - M x|| over REAL x with complex M and b.
    M is a matrix or an operator with matvec / rmatvec (KhatriRaoCols).

    The u-space is C^{p^2} with the real inner product Re<.,.>; since b and
    every M v are vectorised Hermitian matrices, M^H u is real and the real
    part is taken explicitly.  Bidiagonalisation: eq. initbeta, eq. initu and
    eq. lanczos.  Solution update and stopping rules follow Paige & Saunders
    (1982), cited for the scalar steps in Sec. V-A:
      istop 1: ||r|| <= btol ||b|| + atol ||M|| ||x||
      istop 2: ||M^H r|| <= atol ||M|| ||r||
      istop 3: iteration limit.
    Cold start x0 = 0 (eq. initbeta)."""
    n = M.shape[1]
    x = np.zeros(n)
    if n == 0:
        return LsqrResult(x, 0, 0, float(np.linalg.norm(b)), 0.0)
    beta = float(np.linalg.norm(b))
    bnorm = beta
    if beta == 0.0:
        return LsqrResult(x, 0, 0, 0.0, 0.0)
    u = b / beta
    v = _rmv(M, u)
    alpha = float(np.linalg.norm(v))
    if alpha == 0.0:
        return LsqrResult(x, 0, 2, beta, 0.0)
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    anorm2 = 0.0
    rnorm, arnorm = beta, alpha * beta
    istop, it = 3, 0
    for it in range(1, maxit + 1):
        # Golub-Kahan step, eq. lanczos
        u = _mv(M, v) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0.0:
            u = u / beta
        anorm2 += alpha * alpha + beta * beta
        v = _rmv(M, u) - beta * v
        alpha = float(np.linalg.norm(v))
        if alpha > 0.0:
            v = v / alpha
        # plane rotation eliminating the subdiagonal beta of B
        rho = math.hypot(rhobar, beta)
        c = rhobar / rho
        s = beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        rnorm = phibar
        arnorm = phibar * alpha * abs(c)
        anorm = math.sqrt(anorm2)
        xnorm = float(np.linalg.norm(x))
        if rnorm <= btol * bnorm + atol * anorm * xnorm:
            istop = 1
            break
        if arnorm <= atol * anorm * rnorm:
            istop = 2
            break
    return LsqrResult(x, it, istop, rnorm, arnorm)


# ---------------------------------------------------------------- Table I
@dataclass
class SolveResult:
    sigma: np.ndarray          # image (sigma units)
    x: np.ndarray              # solver variable (sigma or D sigma)
    sets: np.ndarray           # per pixel SET_L / SET_U / SET_F
    outer: int                 # loop passes of Table I
    lsqr_iters: int
    converged: bool
    events: list = field(default_factory=list)   # ('free', i) / ('clamp', i, set)
    grad: np.ndarray | None = None               # last full gradient


def active_set(prob: CostProblem, eps: np.ndarray, prm: Params,
               record: bool = True, progress=None) -> SolveResult:
    """Active-set method of Table I for min 1/2||b - Mx||^2, 0 <= x <= upper.

    Start x = 0, all pixels in L, F empty, flag Freegradient-isnotzero = True.
    While flag or a multiplier is below its threshold:
      if flag: z = argmin over x_F of the equality subproblem
               (eq. subproblemLS / eq. subproblemMVDR, b_sub = b - M_U x_U);
               if z feasible: x_F = z, flag = False, gradient on the active
               set, lambda_L = g_L, lambda_U = -g_U (eq. etaL / eq. etaU);
               else: p = z - x_F, mu_i from eq. mumax, step mu_max, move the
               pixel that reaches its bound to L or U, flag = True.
      else:    move i_min from the active set to F, flag = True.
    Detection (Sec. IV-C): candidates are i in A with lambda_i < -eps_i; the
    candidate with the smallest lambda_i is freed, ties to the smallest index.
    mu ties go to the smallest pixel index; p_i = 0 gives mu_i = +inf.
    Feasibility is non-strict: -tau u_i <= z_i <= (1 + tau) u_i with the
    relative tolerance tau = feas_tol, and an accepted z is clipped into
    [0, u_i].  The paper gives no tolerance; tau matters because the first
    subproblem sits exactly on its bound: one free pixel gives z_i = h_i / C
    against u_i = D_i gamma_i = h_i for PWLS with the MVDR bound (C = 1), and
    z_i = gamma_i for CLS with the MF bound, so the untoleranced test is
    decided by rounding.  progress(outer, n_free, lsqr_total), when given, is
    called after every pass (reporting only)."""
    b, up = prob.b, prob.upper
    Q = prob.Q
    x = np.zeros(Q)
    sets = np.full(Q, SET_L, dtype=np.int8)
    flag = True
    i_min = -1
    outer = 0
    lsqr_total = 0
    events = []
    max_outer = prm.max_outer if prm.max_outer > 0 else 10 * Q + 100
    g = None
    converged = False
    while outer < max_outer:
        outer += 1
        if flag:
            F = np.nonzero(sets == SET_F)[0]
            U = np.nonzero(sets == SET_U)[0]
            if F.size:
                b_sub = b - prob.apply(U, x[U])
                maxit = prm.lsqr_maxit if prm.lsqr_maxit > 0 else 4 * F.size + 20
                res = lsqr(prob.cols(F), b_sub, prm.lsqr_atol, prm.lsqr_btol, maxit)
                lsqr_total += res.iters
                z = res.x
            else:
                z = np.zeros(0)
            tau = prm.feas_tol
            feasible = bool(np.all(z >= -tau * up[F]) and np.all(z <= (1.0 + tau) * up[F]))
            if feasible:
                x[F] = np.clip(z, 0.0, up[F])
                flag = False
                g = gradient(prob, x)
                lam = np.where(sets == SET_U, -g, g)
                cand = (sets != SET_F) & (lam < -eps)
                if not np.any(cand):
                    converged = True
                    break
                lam_c = np.where(cand, lam, np.inf)
                i_min = int(np.argmin(lam_c))          # first index on ties
            else:
                pdir = z - x[F]
                mu = np.full(F.size, np.inf)
                pos = pdir > 0
                neg = pdir < 0
                mu[pos] = (up[F][pos] - x[F][pos]) / pdir[pos]
                mu[neg] = -x[F][neg] / pdir[neg]
                k = int(np.argmin(mu))                 # F is sorted: smallest index
                mu_max = float(mu[k])
                x[F] = x[F] + mu_max * pdir
                i = int(F[k])
                if pdir[k] > 0:
                    sets[i] = SET_U
                    x[i] = up[i]
                else:
                    sets[i] = SET_L
                    x[i] = 0.0
                if record:
                    events.append(("clamp", i, int(sets[i])))
                flag = True
        else:
            sets[i_min] = SET_F
            if record:
                events.append(("free", i_min))
            flag = True
        if progress is not None:
            progress(outer, int(np.count_nonzero(sets == SET_F)), lsqr_total)
    return SolveResult(prob.to_sigma * x, x, sets, outer, lsqr_total, converged,
                       events, g)


# ---------------------------------------------------------------- one image
@dataclass
class ImageResult:
    bounds: Bounds
    solve: SolveResult


def image(ant_xyz, l, m, lam, R, N, prm: Params, streamed: bool = False,
          progress=None) -> ImageResult:
    """Full pipeline for one job: bounds, then the bounded LS solve.
    streamed: never form Psi (the operator is applied through A)."""
    A = steering_matrix(ant_xyz, l, m, lam)
    Psi = None if streamed else khatri_rao_psi(A)
    bnd = bounds(A, Psi, R, N, prm)
    prob = cost_problem(A, Psi, R, bnd, prm.cost)
    res = active_set(prob, bnd.eps, prm, progress=progress)
    return ImageResult(bnd, res)


def image_job(job, prm: Params, streamed: bool = False, progress=None) -> ImageResult:
    return image(job.ant_xyz, job.l, job.m, job.lam, job.R, job.N, prm, streamed, progress)


# ---------------------------------------------------------------- replay
@dataclass
class FollowReport:
    """Outcome of replaying a decision log through the oracle."""
    result: SolveResult
    decisions: int = 0
    ties: int = 0                 # decisions that differ from the oracle's own choice
    violations: list = field(default_factory=list)
    max_margin: float = 0.0       # largest tie margin seen (relative)


def active_set_follow(prob: CostProblem, eps: np.ndarray, prm: Params, log, tol: float = 1e-4
                      ) -> FollowReport:
    """Run Table I (as active_set) but take every discrete decision from `log`
    [(kind, pixel), ...] (kind 0 free, 1 clamp to L, 2 clamp to U; an empty
    remainder means the logged run stopped).  Each logged decision is checked
    against the oracle's own arithmetic: it must be the oracle's choice, or a
    tie within `tol` relative to the quantity's scale:
      free    lambda_j < -eps_j and lambda_j <= lambda_min, within tol * scale
              (scale: largest |gradient| at sigma = 0, the dirty image peak);
      stop    no lambda_i + eps_i below -tol * scale;
      feasible / clamp   z inside / outside its bounds unless within tol of one;
      clamp pixel   mu_j <= mu_max (1 + tol) with the direction's sign.
    Test infrastructure for path-dependent results (kappa > 0): when all
    decisions are admissible, the logged run followed a valid path of the
    method and its image must match the oracle's image along that path."""
    b, up = prob.b, prob.upper
    Q = prob.Q
    x = np.zeros(Q)
    sets = np.full(Q, SET_L, dtype=np.int8)
    rep = FollowReport(result=None)
    scale = float(np.max(np.abs(gradient(prob, np.zeros(Q)))))
    k = 0
    flag = True
    outer = 0
    lsqr_total = 0
    converged = False
    g = None
    free_next = -1
    max_outer = prm.max_outer if prm.max_outer > 0 else 10 * Q + 100
    tau = prm.feas_tol
    while outer < max_outer:
        outer += 1
        if flag:
            F = np.nonzero(sets == SET_F)[0]
            U = np.nonzero(sets == SET_U)[0]
            if F.size:
                b_sub = b - prob.apply(U, x[U])
                maxit = prm.lsqr_maxit if prm.lsqr_maxit > 0 else 4 * F.size + 20
                res = lsqr(prob.cols(F), b_sub, prm.lsqr_atol, prm.lsqr_btol, maxit)
                lsqr_total += res.iters
                z = res.x
            else:
                z = np.zeros(0)
            uF = up[F]
            viol = np.maximum(-z / uF - tau, z / uF - (1.0 + tau)) if F.size else np.zeros(0)
            feas_o = not np.any(viol > 0)
            nxt = log[k] if k < len(log) else None
            feas_l = not (nxt is not None and nxt[0] in (1, 2))
            rep.decisions += 1
            if feas_o != feas_l:
                margin = float(np.max(np.abs(viol))) if viol.size else 0.0
                rep.max_margin = max(rep.max_margin, margin)
                if margin > tol:
                    rep.violations.append(("feasibility", k, margin))
                rep.ties += 1
            if feas_l:
                x[F] = np.clip(z, 0.0, uF)
                flag = False
                g = gradient(prob, x)
                lam = np.where(sets == SET_U, -g, g)
                act = sets != SET_F
                slack = np.where(act, lam + eps, np.inf)
                rep.decisions += 1
                if nxt is None:
                    worst = float(np.min(slack))
                    if worst < -tol * scale:
                        rep.violations.append(("stop", k, worst / scale))
                    converged = True
                    break
                j = int(nxt[1])
                if nxt[0] != 0 or not act[j]:
                    rep.violations.append(("free-kind", k, float("nan")))
                    break
                lam_min = float(np.min(np.where(act & (slack < 0), lam, np.inf)))
                margin = max((lam[j] - lam_min) / scale, slack[j] / scale)
                if np.argmin(np.where(act & (slack < 0), lam, np.inf)) != j:
                    rep.ties += 1
                    rep.max_margin = max(rep.max_margin, margin)
                if margin > tol:
                    rep.violations.append(("free", k, margin))
                free_next = j
                k += 1
            else:
                i = int(nxt[1])
                pos = np.nonzero(F == i)[0]
                if pos.size != 1:
                    rep.violations.append(("clamp-not-free", k, float("nan")))
                    break
                q = int(pos[0])
                pdir = z - x[F]
                mu = np.full(F.size, np.inf)
                pp, pn = pdir > 0, pdir < 0
                mu[pp] = (uF[pp] - x[F][pp]) / pdir[pp]
                mu[pn] = -x[F][pn] / pdir[pn]
                mu_max = float(np.min(mu))
                rep.decisions += 1
                # the blocking pixel goes to U when its direction is positive,
                # to L otherwise (Table I): the logged set must match the sign
                if (nxt[0] == 2) != (pdir[q] > 0):
                    rep.violations.append(("clamp-set", k, float(pdir[q])))
                # and it must be the pixel with the smallest step, up to a tie
                if mu[q] > mu_max * (1 + tol) + 1e-300:
                    rep.violations.append(("clamp", k, float(mu[q] / max(mu_max, 1e-300) - 1)))
                if F[int(np.argmin(mu))] != i:
                    rep.ties += 1
                step = float(mu[q])
                x[F] = x[F] + step * pdir
                if nxt[0] == 2:
                    sets[i] = SET_U
                    x[i] = up[i]
                else:
                    sets[i] = SET_L
                    x[i] = 0.0
                k += 1
                flag = True
        else:
            sets[free_next] = SET_F
            flag = True
    rep.result = SolveResult(prob.to_sigma * x, x, sets, outer, lsqr_total, converged, [], g)
    return rep
