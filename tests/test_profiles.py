"""The committed DRAM-traffic summaries that bench.py scales into its roofline `traffic` field.

Each profiles/<kernel>_traffic.json names the source region its ncu capture was taken from (a begin
marker and the __global__ function); bench.py reports the traffic only while the region's hash is
unchanged.  These checks need no GPU: the region exists, the hash function finds it, and the stored
bytes per unit are the captured bytes divided by the captured units.
"""
import glob
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def traffic_files():
    return sorted(glob.glob(os.path.join(ROOT, "profiles", "*_traffic.json")))


def test_traffic_files_exist():
    names = {os.path.basename(p) for p in traffic_files()}
    assert {"ns_pair_kernel_traffic.json", "chol_update_kernel_traffic.json",
            "chol_trsm_tc_kernel_traffic.json"} <= names


@pytest.mark.parametrize("path", traffic_files(), ids=os.path.basename)
def test_traffic_summary_is_consistent(bench, path):
    d = json.load(open(path))
    src = d["source"]
    assert os.path.basename(path) == d["kernel"] + "_traffic.json"
    assert src["function"] == d["kernel"]
    h = bench.source_hash(src["file"], src["begin"], src["function"])   # the region exists
    assert len(h) == 16 and len(d["source_sha256_16"]) == 16
    total = d["dram_bytes_read_per_launch"] + d["dram_bytes_write_per_launch"]
    assert d["units_per_launch"] > 0
    assert d["dram_bytes_per_unit"] == pytest.approx(total / d["units_per_launch"], rel=1e-12)
    # the capture was taken with the clocks left alone and on one kernel
    assert "--clock-control none" in d["capture"] and "-c 1" in d["capture"]


def test_traffic_scales_with_units(bench):
    p = os.path.join(ROOT, "profiles", "ns_pair_kernel_traffic.json")
    d = json.load(open(p))
    src = d["source"]
    if bench.source_hash(src["file"], src["begin"], src["function"]) != d["source_sha256_16"]:
        assert bench.traffic_per_launch("ns_pair_kernel", 1000) is None   # stale summaries report nothing
    else:
        assert bench.traffic_per_launch("ns_pair_kernel", 1000) == pytest.approx(1000 * d["dram_bytes_per_unit"])
