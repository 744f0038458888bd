"""The benchmark's report arithmetic on the host: the algorithmic bytes per launch of each
per-search kernel, the choice of the dominant kernel class, and the DRAM traffic records (used
only while the kernel source they were taken from is unchanged)."""
import hashlib
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PK = {"hbm_gbs": 7000.0, "sm_max_mhz": 2000.0}


def res(**kw):
    r = dict(prof={"pick": (10.0, 600), "fields": (30.0, 600), "bound": (70.0, 600), "scan": (50.0, 600),
                   "merge": (72.0, 600)},
             n=600, n_inst=120, R=64, K=120, pairs=179700 * 7680 * 600.0, evald=770 * 7680 * 600.0,
             survivors=190 * 7680 * 600.0, prec="split_bf16", flips="single_pair", pair_scan=1,
             workload="gaussian_n600_120x64", ms=250.0, sms=152)
    r.update(kw)
    return r


def test_merge_bytes_per_launch():
    rl = bench.roofline_merge(res(), PK, "measured")
    searches, K1, W = 7680, 121, 10
    want = searches * (24 * K1 + 8 * W) + 32 * 190 * 7680
    assert rl["bytes_per_launch"] == pytest.approx(want)
    dur = 72.0 / 600 / 1e3
    assert rl["achieved"] == pytest.approx(want / dur / 1e9, rel=1e-3)
    assert rl["frac"] == pytest.approx(rl["achieved"] / 7000.0, rel=1e-3)
    assert rl["kernel"] == "k_merge" and rl["bound"] == "hbm"


def test_bound_bytes_per_launch():
    rl = bench.roofline_bound(res(), PK, "measured")
    assert rl["bytes_per_launch"] == pytest.approx(7680 * (8 * 600 + 8 * 121 * 10))
    assert rl["kernel"] == "k_bound"


def test_sparse_scan_bytes_and_searches():
    rl = bench.roofline(res(), PK)
    assert rl["kernel"] == "k_scan_sparse" and rl["bound"] == "hbm"
    assert rl["searches_per_launch"] == pytest.approx(7680)
    assert rl["bytes_per_launch"] == pytest.approx(7680 * 12 * 600 + 4 * 770 * 7680)


def test_dense_scan_alu_and_fp64_forms():
    rl = bench.roofline(res(pair_scan=2), PK)
    assert rl["kernel"] == "k_scan_pairs" and rl["bound"] == "alu"
    assert rl["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e12, rel=1e-3)
    rl = bench.roofline(res(prec="fp64"), PK)
    assert rl["kernel"] == "k_scan64" and rl["bound"] == "fp64"


def test_traffic_record_used_only_for_its_source_and_workload(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel source\n")
    (tmp_path / "profiles").mkdir()
    rec = {"source": "k.cu", "source_sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
           "workload": "w600", "traffic_bytes_per_launch": 123456}
    (tmp_path / "profiles" / "k_merge_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("w600", "k_merge") == 123456
    assert bench.kernel_traffic("other", "k_merge") is None
    assert bench.kernel_traffic("w600", "k_bound") is None   # no record
    src.write_text("kernel source, changed\n")
    assert bench.kernel_traffic("w600", "k_merge") is None


def test_dominant_class_is_reported():
    rl, others = bench.dominant_roofline(res(), PK, "measured")
    assert rl["kernel"] == "k_merge" and rl["dominant_share"] == pytest.approx(72.0 / 250.0, abs=1e-4)
    assert set(others) == {"k_bound", "k_scan_sparse"}
    r = res()
    r["prof"]["scan"] = (90.0, 600)
    rl, _ = bench.dominant_roofline(r, PK, "measured")
    assert rl["kernel"] == "k_scan_sparse"
    r = res(flips="single")   # no pair scan: bound or merge
    r["prof"]["bound"] = (80.0, 600)
    rl, others = bench.dominant_roofline(r, PK, "measured")
    assert rl["kernel"] == "k_bound" and set(others) == {"k_merge"}
