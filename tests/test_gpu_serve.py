"""Continuous-batching server: every job's image is the same whether it runs
alone or mixed with others that arrive while it is on the GPU, and equals the
single-job API's image."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1505_01348_gb300 as G
    G.load(build_if_missing=True)
    return G


def _jobs():
    shapes = [(16, 24, 20), (24, 32, 32), (40, 40, 36), (64, 48, 48), (96, 24, 32), (33, 17, 29)]
    return [synth.custom(500 + k, p, nl, nm, 4, 3000, radius=8.0) for k, (p, nl, nm) in enumerate(shapes)]


def _alone_reference(G, jobs):
    out = []
    for job in jobs:
        im = G.Imager.from_job(job, precision=1)
        out.append(im.solve()[0])
        im.close()
    return out


def test_alone_and_mixed_results_agree(G):
    jobs = _jobs()
    ref = _alone_reference(G, jobs)
    srv = G.Server(max_inflight_jobs=4, max_batch=2, n_streams=3)
    alone = []
    for job in jobs:
        jid = srv.submit_job(job, precision=1)
        alone.append(srv.wait(jid)[0])
    ids = [srv.submit_job(job, precision=1) for job in jobs * 3]   # 18 jobs in flight together
    mixed = [srv.wait(i) for i in ids]
    srv.close()
    for a, r in zip(alone, ref):
        np.testing.assert_array_equal(a, r)
    for k, (img, info, lat) in enumerate(mixed):
        np.testing.assert_array_equal(img, ref[k % len(jobs)])
        assert info.converged == 1
        assert lat > 0


def test_small_budget_admits_as_memory_frees(G):
    jobs = _jobs()[:3]
    ref = _alone_reference(G, jobs)
    srv = G.Server(hbm_budget_bytes=24 << 20, n_streams=2)   # room for about one context
    ids = [srv.submit_job(job, precision=1) for job in jobs]
    got = [srv.wait(i)[0] for i in ids]
    srv.close()
    for a, r in zip(got, ref):
        np.testing.assert_array_equal(a, r)


def test_job_larger_than_budget_is_rejected(G):
    job = synth.custom(9, 64, 128, 128, 3, 1000)
    srv = G.Server(hbm_budget_bytes=1 << 20)
    jid = srv.submit_job(job)
    with pytest.raises(G.ImgError) as e:
        srv.wait(jid)
    assert e.value.code == 2    # IMG_ENOMEM
    srv.close()
