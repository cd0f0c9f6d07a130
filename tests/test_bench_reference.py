"""bench.py without a GPU: the reference arm (the FP64 oracle's sequential
decoder on the host cores) prints one JSON line with the fields of the
benchmark contract (the same metric, unit and workload as the GPU arm, a
positive rate, the CPU baseline it measured and an end-to-end entry without
device copies), and the decoder's recorded DRAM traffic belongs to the
current decoder sources."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(300)
def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ)
    env.pop("RANK", None)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == bench.workload_name()
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_recorded_traffic_matches_the_decoder_sources():
    # the roofline's DRAM traffic per pixel comes from an ncu capture of the
    # decoder; bench.py reports it only while the decoder's sources hash to
    # the recorded value, so a change to them must come with a new capture
    sys.path.insert(0, ROOT)
    import bench
    for name in bench.DECODER_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_2201_05213_gb300", "csrc", name)), name
    assert bench._csrc_sha() == bench.TRAFFIC_SRC_SHA
    assert 0 < bench.TRAFFIC_B_PER_PX < 64
