"""bench.py's reference arm runs the oracle on the host cores, so its JSON line can be checked
without a GPU: every key of the benchmark line is there, the arm is labelled, and the
end-to-end block carries no host-device traffic.  The config block states whether the workload
exceeds L2."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line_on_cpu():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "64",
                          "--ref-window", "8", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT,
                         env={k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE")})
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "fits in L2" in line["config"]["l2"]  # 64^2 is a small case


def test_config_states_the_l2_relation():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.workload_config(2048, 1)["l2"].startswith("inputs larger than L2")
    assert "fits in L2" in bench.workload_config(64, 1)["l2"]
