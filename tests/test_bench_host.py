"""Host logic of bench.py on CPU: the JSON line's contract keys and
arithmetic, the images per step and the padded operand width."""
import types

import pytest

import bench


def _fake_result(workload="large", B=16, K=2, total=59.3):
    return {
        "B": B, "total": total, "t_solve": [total / K] * K, "t_prep": [0.04] * K,
        "flops": [3.9e15] * K, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
        "workload": workload, "sms": 152, "n": 256, "p": 288, "prep_flops": 6.6e11,
        "conv": B * K, "outer": 5492.0, "launches": [[1000] * B] * K,
        "e2e": {"value": 0.54, "unit": "images/s", "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1},
    }


def test_summarize_carries_the_contract_keys():
    args = types.SimpleNamespace(steps=2, warmup=3, precision="f16x3")
    r = _fake_result()
    line = bench.summarize(r, args, 1)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "e2e", "gpu_launches"):
        assert k in line, k
    assert line["value"] == pytest.approx(16 * 2 / 59.3)
    assert line["ms_per_step"] == pytest.approx(59.3 / 2 * 1e3)
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert "workload" in line["config"]
    rf = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rf, k
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert rf["achieved"] == pytest.approx(3.9e15 / (59.3 / 2) / 1e12)
    assert line["gpu_launches"] == 16 * 1000


def test_summarize_whole_job_value_scales_with_ranks():
    args = types.SimpleNamespace(steps=2, warmup=3, precision="f16x3")
    one = bench.summarize(_fake_result(), args, 1)
    four = bench.summarize(_fake_result(), args, 4)
    assert four["value"] == pytest.approx(4 * one["value"])
    assert four["config"]["parallelism"] == "dp4 (independent images)"


def test_images_per_step():
    assert bench.default_batch("large", 2, 152) == 16
    assert bench.default_batch("large", 5, 152) == 9
    assert bench.default_batch("large", 50, 152) == 4
    assert bench.default_batch("mid", 2, 152) == 304


@pytest.mark.parametrize("p,kp", [(1, 32), (64, 64), (257, 288), (288, 288), (300, 320), (320, 320),
                                  (330, 384), (352, 384), (384, 384)])
def test_unit_kp(p, kp):
    # p padded to 32 and, above 256, until it splits into units of a multiple
    # of 16 rows, at most 128 each, 8 units at most
    assert bench.unit_kp(p) == kp
    if p > 256:
        assert any(kp % nu == 0 and (kp // nu) % 16 == 0 and kp // nu <= 128 for nu in range(1, 9))
