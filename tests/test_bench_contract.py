"""The bench's JSON line (reference arm, which needs no GPU): one line with the keys the
contract names, on the small C1 workload so that it runs in seconds."""

import json
import os
import subprocess
import sys

from tests.conftest import ROOT


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "C1",
                          "--steps", "3", "--warmup", "1"], capture_output=True, text=True, timeout=300, env=env,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-500:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "workload" in d["config"]


def test_reference_arm_reports_the_threads_it_used():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "C1",
                          "--steps", "2", "--warmup", "1", "--oracle-threads", "2"], capture_output=True, text=True,
                         timeout=300, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-500:]
    d = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    assert d["cpu_baseline"]["cores"] == 2 and "2 BLAS threads" in d["cpu_baseline"]["sample"]


def test_serving_timeline_has_one_record_per_step():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_2306_08967_gb300.serving import Request

    def req(rid, sid, k, t_arr, step, t_issue, t_done):
        z = np.zeros(k, np.int32)
        r = Request(rid, sid, z, z, np.ones(k, np.int8), t_arr)
        r.step, r.t_issue, r.t_done = step, t_issue, t_done
        return r

    reqs = [(req(0, 3, 5, 0.10, 0, 0.11, 0.20), 0), (req(1, 1, 2, 0.05, 0, 0.11, 0.20), 0),
            (req(2, 3, 7, 0.15, 1, 0.21, 0.30), 1), (req(3, 2, 1, 0.40, None, None, None), 1)]
    tl = bench.serving_timeline(reqs)
    assert [e["step"] for e in tl] == [0, 1]
    assert tl[0]["requests"] == 2 and tl[0]["edges"] == 7 and tl[0]["graphs"] == [1, 3]
    assert tl[0]["first_arrival_s"] == 0.05 and tl[0]["t_issue_s"] == 0.11 and tl[0]["t_done_s"] == 0.20
    assert tl[1]["requests"] == 1 and tl[1]["edges"] == 7 and tl[1]["phase"] == 1
    json.dumps(tl)                                   # JSON-ready


def test_cpu_baseline_leg_runs_the_oracle_in_a_subprocess(tmp_path):
    # the default bench's cpu_baseline and error legs: the oracle in its own process (BLAS
    # threads pinned), its timing as JSON and its final state saved for the error comparison
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from synth import CONFIGS
    state = str(tmp_path / "oracle_state.npz")
    r = bench.oracle_subprocess(CONFIGS["C1"], 4, 5.0, state)
    assert "error" not in r, r
    assert r["kind"] == "oracle" and r["cores"] == bench.ORACLE_THREADS and r["value"] > 0 and r["batches"] >= 1
    z = np.load(state)
    alt = r.get("alt_threads", {}).get("batches") or 0
    assert int(z["batches"]) == 2 + r["batches"] + alt and z["X"].shape[1] == CONFIGS["C1"].d


def test_cpu_baseline_with_two_thread_counts_saves_every_batch_it_ran(tmp_path):
    # batches alternate between the thread counts; the saved state (which the GPU replays for the
    # error comparison) must count the batches of both
    sys.path.insert(0, ROOT)
    import numpy as np
    import pytest
    import bench
    from synth import CONFIGS
    if bench.ORACLE_THREADS < 2 or bench._blas_thread_setter() is None:
        pytest.skip("needs two BLAS thread counts")
    state = str(tmp_path / "oracle_state.npz")
    r = bench.oracle_run(CONFIGS["C1"], 6, 2, 30.0, state, alt_threads=1)
    assert r["alt_threads"]["cores"] == 1 and r["alt_threads"]["batches"] >= 1
    z = np.load(state)
    assert int(z["batches"]) == 2 + r["batches"] + r["alt_threads"]["batches"] == 8


def test_clock_sampler_reads_clocks_and_throttle_reasons(tmp_path, monkeypatch):
    # a stand-in nvidia-smi prints three samples (one under a power cap) and waits to be stopped
    sys.path.insert(0, ROOT)
    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 2070, 2070, 1010.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    import time
    with bench.ClockSampler(0) as clk:
        time.sleep(0.5)
    s = clk.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    # no nvidia-smi at all: the run goes on and says so
    monkeypatch.setenv("PATH", str(tmp_path / "empty"))
    with bench.ClockSampler(0) as clk:
        pass
    assert clk.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
