"""Seeded synthetic inputs for the bounded least-squares imager.

This module only *makes data*: antenna layouts, pixel grids, a true sky and a
sample covariance drawn from the data model of Sec. II (the sample-covariance
definition and the covariance model R = A Sigma A^H + R_n).  It holds none of
the imaging method's arithmetic (no dirty images, bounds, operators or
solvers); both the FP64 oracle and the CUDA path consume what it returns.

Positions are in units of the reference wavelength; a job's wavelength
``lam`` scales all phases.  Pixel ``i = i_l + n_l * i_m`` (column-major image
vectorisation).  Every random draw comes from a numpy ``Generator`` seeded by
``(seed, purpose)`` so array, sky and noise streams are independent.

Workload recipes (stand-ins for the paper's LOFAR layout and 3C catalogue,
which are not available):

* ``tiny``   p=16 uniform in a disk of radius 10, 32x32 grid on [-0.5,0.5]^2,
  5 on-grid point sources with powers U[1,10], sigma_n^2 = 1, N = 1000.
* ``mid``    p=64 log-spiral of radius 50, 128x128 grid, 20 point sources with
  lognormal(0,1) powers plus one Gaussian blob (FWHM 6 px, peak 1),
  SNR 0 dB per antenna, N = 10^4.
* ``batch``  one of 64 channels: p in {48,64,96} (prefix of a 96-element
  spiral), n in {64,96,128}, wavelength 1 + 0.5 c/63, 10-40 sources.
* ``large``  p=288 in 6 clusters of 48 within radius 200, 256x256 grid,
  50 point sources plus 3 Gaussian blobs (FWHM U[4,10] px).
* ``serve``  p in {32,64,128,256}, n in {64,128,256}, 5-50 sources.
* ``snapshots_*``  K snapshots of one sky with the array turned by dtheta
  between snapshots (Earth rotation stand-in), independent noise per snapshot.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_ARRAY, _SKY, _NOISE, _PICK = 1, 2, 3, 4


def _rng(seed: int, purpose: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(purpose)])


@dataclass
class Job:
    """One imaging job: instrument, grid and a sample covariance."""

    name: str
    seed: int
    ant_xyz: np.ndarray          # (p, 3) float64, reference-wavelength units
    l: np.ndarray                # (n_l,) direction cosines
    m: np.ndarray                # (n_m,)
    lam: float                   # wavelength in reference units
    R: np.ndarray                # (p, p) complex128 sample covariance, Hermitian
    N: int                       # number of samples behind R
    sigma_true: np.ndarray       # (Q,) true on-grid pixel powers
    noise_var: float
    meta: dict = field(default_factory=dict)

    @property
    def p(self) -> int:
        return self.ant_xyz.shape[0]

    @property
    def n_l(self) -> int:
        return self.l.shape[0]

    @property
    def n_m(self) -> int:
        return self.m.shape[0]

    @property
    def Q(self) -> int:
        return self.n_l * self.n_m


# ---------------------------------------------------------------- layouts
def disk_layout(p: int, radius: float, rng: np.random.Generator) -> np.ndarray:
    r = radius * np.sqrt(rng.random(p))
    th = 2.0 * np.pi * rng.random(p)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(p)], axis=1)


def spiral_layout(p: int, radius: float, rng: np.random.Generator,
                  jitter: float = 0.1) -> np.ndarray:
    k = np.arange(p, dtype=np.float64)
    rot = 2.0 * np.pi * rng.random()
    th = 4.0 * np.pi * k / max(p - 1, 1) + rot
    r = radius ** (k / max(p - 1, 1))
    xy = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    xy += jitter * rng.standard_normal((p, 2))
    return np.concatenate([xy, np.zeros((p, 1))], axis=1)


def cluster_layout(n_clusters: int, per: int, centre_radius: float,
                   cluster_radius: float, rng: np.random.Generator) -> np.ndarray:
    out = []
    centres = disk_layout(n_clusters, centre_radius, rng)
    for c in range(n_clusters):
        pts = disk_layout(per, cluster_radius, rng)
        pts[:, :2] += centres[c, :2]
        out.append(pts)
    return np.concatenate(out, axis=0)


def grid(n: int, half_width: float = 0.5) -> np.ndarray:
    return np.linspace(-half_width, half_width, n)


# ---------------------------------------------------------------- sky
def _distinct_pixels(Q: int, k: int, rng: np.random.Generator) -> np.ndarray:
    return rng.choice(Q, size=k, replace=False)


def gaussian_blob(sky: np.ndarray, n_l: int, n_m: int, centre: int,
                  fwhm_px: float, peak: float) -> None:
    """Add a Gaussian extended source (one on-grid emitter per pixel)."""
    s = fwhm_px / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    cl, cm = centre % n_l, centre // n_l
    rad = int(math.ceil(3.0 * s))
    for dm in range(-rad, rad + 1):
        for dl in range(-rad, rad + 1):
            il, im = cl + dl, cm + dm
            if 0 <= il < n_l and 0 <= im < n_m:
                w = math.exp(-(dl * dl + dm * dm) / (2.0 * s * s))
                if w >= 1e-3:
                    sky[il + n_l * im] += peak * w


# ---------------------------------------------------------------- covariance
def _source_response(ant_xyz: np.ndarray, l: np.ndarray, m: np.ndarray,
                     lam: float) -> np.ndarray:
    """Array response towards (l, m) directions, unit norm per column.

    Data-model side of Sec. II, written independently of any imaging code:
    phase -2*pi*<x_k, s>/lam with s = (l, m, sqrt(1-l^2-m^2)).
    """
    n = np.sqrt(np.maximum(0.0, 1.0 - l * l - m * m))
    dirs = np.stack([l, m, n], axis=0)                    # (3, S)
    ph = -2.0 * np.pi * (ant_xyz @ dirs) / lam            # (p, S)
    return np.exp(1j * ph) / math.sqrt(ant_xyz.shape[0])


def sample_covariance(ant_xyz, l_grid, m_grid, lam, sky, noise_var, N, rng):
    """Draw R_hat = (1/N) Y Y^H with Y = chol(R) G, R = A Sigma A^H + s2 I."""
    p = ant_xyz.shape[0]
    n_l = l_grid.shape[0]
    idx = np.nonzero(sky)[0]
    ls = l_grid[idx % n_l]
    ms = m_grid[idx // n_l]
    At = _source_response(ant_xyz, ls, ms, lam)
    R = (At * sky[idx][None, :]) @ At.conj().T + noise_var * np.eye(p)
    R = 0.5 * (R + R.conj().T)
    C = np.linalg.cholesky(R)
    G = (rng.standard_normal((p, N)) + 1j * rng.standard_normal((p, N))) / math.sqrt(2.0)
    Y = C @ G
    Rh = (Y @ Y.conj().T) / N
    return 0.5 * (Rh + Rh.conj().T)


def _finish(name, seed, ant, l, m, lam, sky, noise_var, N, meta=None) -> Job:
    R = sample_covariance(ant, l, m, lam, sky, noise_var, N, _rng(seed, _NOISE))
    return Job(name=name, seed=seed, ant_xyz=ant, l=l, m=m, lam=lam, R=R, N=N,
               sigma_true=sky, noise_var=noise_var, meta=meta or {})


# ---------------------------------------------------------------- recipes
def tiny(seed: int = 1000, p: int = 16, n: int = 32, n_src: int = 5,
         N: int = 1000) -> Job:
    ant = disk_layout(p, 10.0, _rng(seed, _ARRAY))
    l = m = grid(n)
    rs = _rng(seed, _SKY)
    sky = np.zeros(n * n)
    sky[_distinct_pixels(n * n, n_src, rs)] = rs.uniform(1.0, 10.0, n_src)
    return _finish("tiny", seed, ant, l, m.copy(), 1.0, sky, 1.0, N)


def mid(seed: int = 2000, p: int = 64, n: int = 128, n_src: int = 20,
        N: int = 10_000, blob: bool = True) -> Job:
    ant = spiral_layout(p, 50.0, _rng(seed, _ARRAY))
    l = m = grid(n)
    rs = _rng(seed, _SKY)
    sky = np.zeros(n * n)
    pix = _distinct_pixels(n * n, n_src + 1, rs)
    sky[pix[:n_src]] = rs.lognormal(0.0, 1.0, n_src)
    if blob:
        gaussian_blob(sky, n, n, int(pix[n_src]), 6.0, 1.0)
    noise_var = float(sky.sum()) / p          # SNR 0 dB per antenna
    return _finish("mid", seed, ant, l, m.copy(), 1.0, sky, noise_var, N)


def batch_channel(c: int, seed: int = 3000, N: int = 10_000) -> Job:
    """Channel c of the 64-channel uneven batch."""
    rs = _rng(seed + c, _PICK)
    p = int(rs.choice([48, 64, 96]))
    n = int(rs.choice([64, 96, 128]))
    base = spiral_layout(96, 50.0, _rng(seed, _ARRAY))
    ant = base[:p].copy()
    lam = 1.0 + 0.5 * c / 63.0
    l = m = grid(n)
    sk = _rng(seed + c, _SKY)
    n_src = int(sk.integers(10, 41))
    sky = np.zeros(n * n)
    sky[_distinct_pixels(n * n, n_src, sk)] = sk.lognormal(0.0, 1.0, n_src)
    noise_var = float(sky.sum()) / p
    return _finish("batch", seed + c, ant, l, m.copy(), lam, sky, noise_var, N,
                   {"channel": c})


def large(seed: int = 4000, N: int = 10_000, n: int = 256) -> Job:
    ant = cluster_layout(6, 48, 150.0, 50.0, _rng(seed, _ARRAY))
    l = m = grid(n)
    rs = _rng(seed, _SKY)
    sky = np.zeros(n * n)
    pix = _distinct_pixels(n * n, 53, rs)
    sky[pix[:50]] = rs.lognormal(0.0, 1.0, 50)
    for b in range(3):
        gaussian_blob(sky, n, n, int(pix[50 + b]), float(rs.uniform(4.0, 10.0)), 1.0)
    noise_var = float(sky.sum()) / ant.shape[0]
    return _finish("large", seed, ant, l, m.copy(), 1.0, sky, noise_var, N)


def serve_job(j: int, seed: int = 5000, N: int = 10_000) -> Job:
    rs = _rng(seed + j, _PICK)
    p = int(rs.choice([32, 64, 128, 256]))
    n = int(rs.choice([64, 128, 256]))
    ant = spiral_layout(p, 50.0, _rng(seed + j, _ARRAY))
    l = m = grid(n)
    sk = _rng(seed + j, _SKY)
    n_src = int(sk.integers(5, 51))
    sky = np.zeros(n * n)
    sky[_distinct_pixels(n * n, n_src, sk)] = sk.lognormal(0.0, 1.0, n_src)
    noise_var = float(sky.sum()) / p
    return _finish("serve", seed + j, ant, l, m.copy(), 1.0, sky, noise_var, N,
                   {"job": j})


def custom(seed: int, p: int, n_l: int, n_m: int, n_src: int, N: int,
           radius: float = 10.0, snr_db: float = 0.0,
           half_width: float = 0.5) -> Job:
    """Small jobs of any shape for edge-case and parity tests."""
    ant = disk_layout(p, radius, _rng(seed, _ARRAY))
    l = grid(n_l, half_width)
    m = grid(n_m, half_width)
    rs = _rng(seed, _SKY)
    Q = n_l * n_m
    sky = np.zeros(Q)
    k = min(n_src, Q)
    if k:
        sky[_distinct_pixels(Q, k, rs)] = rs.uniform(1.0, 10.0, k)
    noise_var = max(float(sky.sum()) / p * 10 ** (-snr_db / 10.0), 1e-3)
    return _finish("custom", seed, ant, l, m, 1.0, sky, noise_var, N)


def serve_job_tc(j: int, seed: int = 6000, N: int = 10_000) -> Job:
    """Serving mix restricted to the sizes the tensor-core path takes
    (p in {32, 64}, grid 64x64 or 128x128), 5-50 sources, log-spiral arrays."""
    rs = _rng(seed + j, _PICK)
    p = int(rs.choice([32, 64]))
    n = int(rs.choice([64, 128]))
    ant = spiral_layout(p, 50.0, _rng(seed + j, _ARRAY))
    l = m = grid(n)
    sk = _rng(seed + j, _SKY)
    n_src = int(sk.integers(5, 51))
    sky = np.zeros(n * n)
    sky[_distinct_pixels(n * n, n_src, sk)] = sk.lognormal(0.0, 1.0, n_src)
    noise_var = float(sky.sum()) / p
    return _finish("serve_tc", seed + j, ant, l, m.copy(), 1.0, sky, noise_var, N, {"job": j})


# ---------------------------------------------------------------- K > 1 snapshots
@dataclass
class SnapshotJob:
    """One imaging job observed over K snapshots (Sec. II data model): the
    sky is fixed, the array turns with the Earth between snapshots, and each
    snapshot k has its own sample covariance R_k from N samples."""

    name: str
    seed: int
    ant_xyz: np.ndarray          # (K, p, 3) positions per snapshot, sky-fixed frame
    l: np.ndarray
    m: np.ndarray
    lam: float
    R: np.ndarray                # (K, p, p) complex128 sample covariances
    N: int
    sigma_true: np.ndarray
    noise_var: float
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return self.ant_xyz.shape[0]

    @property
    def p(self) -> int:
        return self.ant_xyz.shape[1]

    @property
    def n_l(self) -> int:
        return self.l.shape[0]

    @property
    def n_m(self) -> int:
        return self.m.shape[0]

    @property
    def Q(self) -> int:
        return self.n_l * self.n_m


def rotate_layout(ant: np.ndarray, theta: float) -> np.ndarray:
    """Turn an array about its local vertical by theta radians.  For an array
    at a pole imaging the zenith region this is the apparent motion of the
    array against the sky between snapshots."""
    c, s = math.cos(theta), math.sin(theta)
    out = ant.copy()
    out[:, 0] = c * ant[:, 0] - s * ant[:, 1]
    out[:, 1] = s * ant[:, 0] + c * ant[:, 1]
    return out


def _finish_snapshots(name, seed, ant0, K, dtheta, l, m, lam, sky, noise_var, N,
                      meta=None) -> SnapshotJob:
    ants = np.stack([rotate_layout(ant0, k * dtheta) for k in range(K)], axis=0)
    Rs = np.stack([sample_covariance(ants[k], l, m, lam, sky, noise_var, N,
                                     np.random.default_rng([int(seed), _NOISE, k]))
                   for k in range(K)], axis=0)
    return SnapshotJob(name=name, seed=seed, ant_xyz=ants, l=l, m=m, lam=lam, R=Rs, N=N,
                       sigma_true=sky, noise_var=noise_var,
                       meta=dict(meta or {}, dtheta=dtheta))


def snapshots_custom(seed: int, p: int, n_l: int, n_m: int, n_src: int, N: int, K: int,
                     dtheta: float = 0.2, radius: float = 10.0, snr_db: float = 0.0,
                     half_width: float = 0.5) -> SnapshotJob:
    """Small K-snapshot jobs for tests: disk array, on-grid point sources with
    powers U[1, 10], noise set by the per-antenna SNR, the array turned by
    dtheta radians from one snapshot to the next."""
    ant = disk_layout(p, radius, _rng(seed, _ARRAY))
    l = grid(n_l, half_width)
    m = grid(n_m, half_width)
    rs = _rng(seed, _SKY)
    Q = n_l * n_m
    sky = np.zeros(Q)
    k = min(n_src, Q)
    if k:
        sky[_distinct_pixels(Q, k, rs)] = rs.uniform(1.0, 10.0, k)
    noise_var = max(float(sky.sum()) / p * 10 ** (-snr_db / 10.0), 1e-3)
    return _finish_snapshots("snapshots_custom", seed, ant, K, dtheta, l, m, 1.0, sky,
                             noise_var, N)


def snapshots_extended(seed: int = 7000, p: int = 100, n: int = 64, K: int = 2,
                       N: int = 10_000, dtheta: float = 0.05) -> SnapshotJob:
    """Stand-in for the extended-source simulation of Sec. VI: p = 100
    antennas at random in a disk, K = 2 snapshots, one strong point source and
    two extended structures of seven Gaussians each (one at the centre, six on
    a hexagon around it), background noise 10 dB below the extended sources.
    The paper's two snapshots are one second apart; dtheta is larger so that
    the two snapshots see visibly different arrays."""
    ant = disk_layout(p, 25.0, _rng(seed, _ARRAY))
    l = m = grid(n)
    rs = _rng(seed, _SKY)
    Q = n * n
    sky = np.zeros(Q)
    sky[int(rs.integers(Q))] = 100.0
    ext_peak = 1.0
    for _ in range(2):
        cl = int(rs.integers(n // 4, 3 * n // 4))
        cm = int(rs.integers(n // 4, 3 * n // 4))
        hexr = max(2, n // 16)
        pts = [(cl, cm)] + [(int(round(cl + hexr * math.cos(t))), int(round(cm + hexr * math.sin(t))))
                            for t in np.arange(6) * (math.pi / 3.0)]
        for il, im in pts:
            if 0 <= il < n and 0 <= im < n:
                gaussian_blob(sky, n, n, il + n * im, 2.0, ext_peak)
    noise_var = ext_peak * 10 ** (-1.0)
    return _finish_snapshots("snapshots_extended", seed, ant, K, dtheta, l, m.copy(), 1.0,
                             sky, noise_var, N)
