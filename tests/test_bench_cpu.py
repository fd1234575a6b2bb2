"""The benchmark's host-side pieces, without a GPU: the reference arm's JSON
line (the FP64 oracle on a bounded sample of the headline workload) and the
summary of the warm-start leg."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["steps"] == 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and line["unit"] == "matvecs/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_warmstart_summary_keeps_only_solver_arms(monkeypatch):
    import bench

    def fake(train_games, heldout):
        arm = {"iterations": 300, "seconds": 0.25}
        return {"train_games": train_games, "heldout_games": heldout, "loss_first_last": [1.0, 0.5],
                "warm_start": {"rmplus": {"kappa": 0.02, "t0": 0}}, "cold_f32": dict(arm),
                "warm_bf16": dict(arm, iterations=200), "cold_dcfr_f32": dict(arm), "total_seconds": 3.0}

    monkeypatch.setattr(bench, "measure_warmstart", fake)
    s = bench.warmstart_summary(train_games=16, heldout=4)
    assert s["train_games"] == 16 and s["heldout_games"] == 4
    assert s["arms_iterations_seconds"] == {"cold_f32": [300, 0.25], "warm_bf16": [200, 0.25],
                                            "cold_dcfr_f32": [300, 0.25]}


def test_reference_arm_under_torchrun_prints_one_line():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
