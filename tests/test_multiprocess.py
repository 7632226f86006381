"""The N > 1 path of bench.py on CPU: two ranks over gloo (GPUs hidden), one
independent replica each, rendezvous at 127.0.0.1, a barrier, and the job
time taken as the maximum over ranks (weak scaling: value = units of all
ranks / slowest rank's time)."""
import json
import os
import socket
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_the_step_time():
    port = _free_port()
    base = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", CUDA_VISIBLE_DEVICES="")
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "mp_replica_helper.py")],
                              env=dict(base, RANK=str(r), LOCAL_RANK=str(r)), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world_size"] == 2
        assert o["ms_max"] == 200.0                      # the slower replica's time
        assert abs(o["value"] - 2 * 3 / 0.2) < 1e-12     # both replicas' steps over it


def test_reference_arm_runs_on_rank_zero_only():
    """bench.py --impl reference under two ranks: rank 0 times the oracle and
    prints the one JSON line, rank 1 exits 0 without work (a small oracle
    sample keeps this test short)."""
    port = _free_port()
    root = os.path.dirname(HERE)
    base = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3", "--ref-n", "8"]
    procs = [subprocess.Popen(cmd, env=dict(base, RANK=str(r), LOCAL_RANK=str(r)), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, cwd=root) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    lines0 = [l for l in outs[0].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not [l for l in outs[1].splitlines() if l.startswith("{")]
    d = json.loads(lines0[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # the line carries the keys of the benchmark's JSON contract
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["n_gpus"] == 2 and d["steps"] == 1 and d["higher_is_better"] is True
    # ms_per_step: the measured time of one timed (sample) step; the value
    # is the full-size rate derived from it by the cell ratio
    assert d["ms_per_step_full_size"] == pytest.approx(1e3 / d["value"], rel=1e-9)
    assert d["ms_per_step"] == pytest.approx(d["cpu_baseline"]["seconds_per_sample"] * 1e3, rel=1e-9)
    assert d["ms_per_step"] * d["steps"] < 300e3
    assert "workload" in d["config"] and not {"model", "global_batch", "seq_len"} & set(d["config"])
    cb = d["cpu_baseline"]
    assert cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["d2h_bytes_per_step"] == 0
