"""bench.py --impl reference: the FP64 oracle timed on the host cores on a
bounded sample of the same workload, printed as one JSON line with the bench
line's metric and workload description.  Runs on the CPU (the arm uses no GPU)."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip().splitlines()


@pytest.mark.parametrize("workload", ["riemann", "switchnet"])
def test_reference_line_contract(workload):
    sys.path.insert(0, ROOT)
    import bench
    lines = _run(["--workload", workload, "--steps", "3", "--warmup", "3"])
    d = json.loads(lines[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3
    # every host core runs one single-threaded oracle process
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert "processes" in d["config"]["sampled"] and "cells" in d["config"]["sampled"]
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["unit"] == d["unit"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["dtype"] == "f64" and d["config"]["prec"] == "fp64"
    if workload == "riemann":
        # the same workload description as the bench line of the CUDA path
        ours = bench.describe(bench.make_workload("riemann", 0), "riemann", "fp32")
        assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
        assert d["config"]["workload"] == ours["workload"]
    else:
        assert d["metric"] == bench.SWITCHNET_METRIC and d["unit"] == "cells/s"
        assert d["config"]["workload"] == bench.SWITCHNET_WORKLOAD


def test_reference_runs_on_rank_zero_only():
    assert _run(["--steps", "3", "--warmup", "3"], {"RANK": "1"}) == []


def test_warmup_below_three_is_refused():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--warmup", "2"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode != 0


def test_committed_traffic_belongs_to_the_committed_kernel_sources():
    """The bench reports the DRAM traffic per element under profiles/ only
    when it was captured on the kernel sources as they are (same source
    hash); after a kernel change the line says null until a new capture."""
    sys.path.insert(0, ROOT)
    import bench
    d = json.load(open(os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")))
    for key, e in d["entries"].items():
        wl, prec = key.split("/")
        tr = bench.stored_traffic(prec, wl)
        if e["source_hash"] == bench.source_hash():
            assert tr is not None and 4.0 < tr < 40.0
        else:
            assert tr is None


def test_profile_summaries_name_the_traffic_record_sources():
    """The ncu summaries the stored traffic comes from name the same stage
    kernel sources (source hash) as the traffic record."""
    d = json.load(open(os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")))
    summaries = {"blob/fp32": "stage_kernel_blob256x48_fp32.md", "riemann/fp32": "stage_kernel_riemann128x32_fp32.md"}
    for key, e in d["entries"].items():
        text = open(os.path.join(ROOT, "profiles", summaries[key])).read()
        assert e["source_hash"] in text, key
        # the capture command of the record is the one the summary gives
        log = e["command"].split("--log-file ")[1].split()[0]
        assert log in text, (key, log)
