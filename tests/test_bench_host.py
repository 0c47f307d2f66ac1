"""Host logic of bench.py (no GPU): the roofline object of the dominant
FP32 Dslash class and the replica reduction."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

V5 = 16 * 16 * 16 * 32 * 16


def _classes(ms_plain, ms_fused):
    prof = {"dslash_f32": (696, ms_plain), "dslash_f32_z": (10884, ms_fused)}
    units = {"dslash_f32": 8388, "dslash_f32_z": 130608}
    return prof, units


def test_dominant_class_is_reported_with_the_other_beside_it():
    prof, units = _classes(942.96, 18035.06)
    r = bench.dslash_roofline(prof, units, V5, 6782.8, "measured")
    assert r["kernel"] == "dslash_f32_z" and r["bytes_per_site"] == 300
    # 300 B x 2,097,152 sites x 130,608 fields over 18.035 s
    assert r["achieved"] == pytest.approx(300 * V5 * 130608 / 18.03506 / 1e9, rel=1e-6)
    assert r["frac"] == pytest.approx(r["achieved"] / 6782.8)
    assert r["traffic"] == bench.DSLASH_Z_TRAFFIC_PER_FIELD
    o = r["other_dslash"]
    assert o["kernel"] == "dslash_f32" and o["bytes_per_site"] == 204
    assert o["achieved"] == pytest.approx(204 * V5 * 8388 / 0.94296 / 1e9, rel=1e-6)


def test_plain_class_wins_when_it_takes_longer():
    prof, units = _classes(20000.0, 100.0)
    r = bench.dslash_roofline(prof, units, V5, 6782.8, "measured")
    assert r["kernel"] == "dslash_f32" and r["other_dslash"]["kernel"] == "dslash_f32_z"


def test_missing_classes():
    prof = {"dslash_f32": (5, 1.0), "dslash_f32_z": (0, 0.0)}
    units = {"dslash_f32": 5, "dslash_f32_z": 0}
    r = bench.dslash_roofline(prof, units, V5, 6782.8, "measured")
    assert r["kernel"] == "dslash_f32" and "other_dslash" not in r
    prof["dslash_f32"] = (0, 0.0)
    assert bench.dslash_roofline(prof, units, V5, 6782.8, "measured") is None


def test_replica_reduce_single_process():
    ms_step, value = bench.replica_reduce(1200.0, 3, 12, 1)
    assert ms_step == pytest.approx(400.0)
    assert value == pytest.approx(0.4 / 12)
