"""The bench's own bookkeeping: the ncu traffic figure it reports applies only
to the filter sources it was measured on, and (on a GPU) one small run prints
one JSON line with every key of the line's contract."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_figure_matches_current_sources():
    """The committed traffic figure (profiles/pf_step_kernel_fleet5.json)
    carries the hash of the current filter sources and the variant it was
    taken with; any other variant gives no traffic figure."""
    with open(bench.TRAFFIC_NOTE) as f:
        t = json.load(f)
    assert t["sources"] == bench.pf_source_hash()
    got = bench._pf_traffic(t["variant"], 1000)
    assert got == pytest.approx(float(t["bytes_per_particle"]) * 1000)
    assert bench._pf_traffic("no-such-variant", 1000) is None


def test_source_hash_covers_the_kernel_includes():
    """Every header the filter kernel includes from the library's sources is
    hashed."""
    csrc = os.path.join(ROOT, "paper_2505_08222_gb300", "csrc")
    seen, todo = set(), ["pf_kernel.cuh", "pf_inst_a.cu", "pf_inst_b.cu", "pf_kernel.cu"]
    while todo:
        name = todo.pop()
        if name in seen:
            continue
        seen.add(name)
        for line in open(os.path.join(csrc, name)):
            if line.startswith('#include "'):
                todo.append(line.split('"')[1])
    assert seen <= set(bench.PF_SOURCES), sorted(seen - set(bench.PF_SOURCES))


@pytest.mark.gpu
def test_small_bench_line_has_the_contract_keys():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--envs", "64", "--steps", "3", "--warmup", "3",
           "--no-cpu-baseline", "--train-rows", "200000", "--train-steps", "20", "--round-steps", "5",
           "--eval-steps", "5", "--est-candidates", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    out = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(out) == 1
    line = json.loads(out[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["steps"] == 3 and line["warmup"] == 3 and line["value"] > 0
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"], k
    assert line["gpu_launches"] > 0 and "workload" in line["config"]
    assert 0.0 < line["learned"]["rmse_ratio"] and line["seeds_0_4"]["min"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and line["e2e"]["d2h_bytes_per_step"] > 0
    assert 0.0 < line["learned"]["seeds_0_4"]["fresh_ping_steps"]["rmse_ratio"]
    # the TransfMAPPO update measurement
    ppo = line["ppo"]
    assert ppo["value"] > 0 and ppo["ms_per_update"] > 0 and ppo["collect_ms"] > 0
    assert ppo["roofline"]["bound"] in ("tensor", "alu") and 0.0 < ppo["roofline"]["frac"] < 1.5
    assert all(v == v for v in ppo["stats_last_minibatch"]["actor"] + ppo["stats_last_minibatch"]["critic"])
