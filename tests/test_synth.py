"""The seeded input generators: reproducible, independent streams per
purpose, and the structure each recipe states (array layouts, sky, the
sample covariance of the Sec. II data model, K-snapshot rotation)."""
import numpy as np

import synth


def test_seeded_and_reproducible():
    a = synth.custom(5, 8, 6, 5, 3, 400)
    b = synth.custom(5, 8, 6, 5, 3, 400)
    c = synth.custom(6, 8, 6, 5, 3, 400)
    np.testing.assert_array_equal(a.R, b.R)
    np.testing.assert_array_equal(a.sigma_true, b.sigma_true)
    assert not np.array_equal(a.R, c.R)


def test_sample_covariance_is_hermitian_pd_and_unbiased():
    """R_hat = (1/N) Y Y^H is Hermitian positive definite, and its mean over
    many draws approaches R = A Sigma A^H + s2 I (Sec. II)."""
    job = synth.custom(9, 5, 4, 4, 2, 200, radius=2.0)
    np.testing.assert_allclose(job.R, job.R.conj().T, atol=0)
    assert np.linalg.eigvalsh(job.R).min() > 0
    idx = np.nonzero(job.sigma_true)[0]
    n_l = job.l.shape[0]
    ls, ms = job.l[idx % n_l], job.m[idx // n_l]
    nn = np.sqrt(1 - ls ** 2 - ms ** 2)
    At = np.exp(-2j * np.pi * (job.ant_xyz @ np.stack([ls, ms, nn])) / job.lam) / np.sqrt(job.p)
    R = (At * job.sigma_true[idx]) @ At.conj().T + job.noise_var * np.eye(job.p)
    rng = np.random.default_rng(3)
    acc = np.zeros_like(R)
    T = 400
    for _ in range(T):
        acc += synth.sample_covariance(job.ant_xyz, job.l, job.m, job.lam, job.sigma_true,
                                       job.noise_var, 200, rng)
    err = np.linalg.norm(acc / T - R) / np.linalg.norm(R)
    assert err < 0.02


def test_snapshot_jobs_turn_the_array_and_draw_independent_noise():
    job = synth.snapshots_custom(11, 10, 6, 6, 3, 500, 3, dtheta=0.25)
    assert job.ant_xyz.shape == (3, 10, 3) and job.R.shape == (3, 10, 10)
    r0 = np.linalg.norm(job.ant_xyz[0, :, :2], axis=1)
    for k in range(1, 3):
        np.testing.assert_allclose(np.linalg.norm(job.ant_xyz[k, :, :2], axis=1), r0, rtol=1e-14)
        # angle of every antenna advanced by k * dtheta
        a0 = np.arctan2(job.ant_xyz[0, :, 1], job.ant_xyz[0, :, 0])
        ak = np.arctan2(job.ant_xyz[k, :, 1], job.ant_xyz[k, :, 0])
        np.testing.assert_allclose(np.angle(np.exp(1j * (ak - a0))), 0.25 * k, atol=1e-12)
    assert not np.allclose(job.R[0], job.R[1])
    for k in range(3):
        np.testing.assert_allclose(job.R[k], job.R[k].conj().T, atol=0)
        assert np.linalg.eigvalsh(job.R[k]).min() > 0


def test_extended_source_stand_in():
    job = synth.snapshots_extended(n=32, p=20)
    assert job.K == 2 and job.p == 20 and job.Q == 32 * 32
    assert job.sigma_true.max() == 100.0                      # the strong point source
    ext = job.sigma_true[(job.sigma_true > 0) & (job.sigma_true < 100.0)]
    assert ext.size > 14                                      # 14 Gaussians spread over pixels
    assert abs(job.noise_var - 0.1) < 1e-15                   # 10 dB below the extended sources
