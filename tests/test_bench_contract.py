"""bench.py's reference arm (the FP64 oracle on the host) prints one JSON line with
the keys the benchmark contract names (CPU only, a tiny oracle sample)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--cpu-seconds", "1"],
                         check=True, capture_output=True, text=True, cwd=ROOT, timeout=600).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["unit"] == d["unit"]
    # every reported step ran: 1 step of 1 oracle MM iteration, solves/s extrapolated
    # from the oracle's own 217 MM iterations to the 1e-6 gap, named in the line
    assert "217 such iterations" in d["cpu_baseline"]["sample"]
    assert d["config"]["step"] == "1 MM iteration of the oracle"
    assert abs(d["value"] * d["ms_per_step"] / 1000.0 * 217 - 1.0) < 1e-9


def test_kernel_hash_ignores_comments_only():
    """The committed ncu traffic is keyed by a hash of the solve kernel's code with
    comments stripped: a comment edit keeps it, a code edit changes it."""
    import bench
    a = "int x = 1;  // one\n/* block\n comment */\nint y = 2;\n"
    b = "int x = 1;\n\n// another comment\nint y = 2;   \n"
    c = "int x = 1;\nint y = 3;\n"
    assert bench.strip_comments(a) == bench.strip_comments(b) == "int x = 1;\nint y = 2;"
    assert bench.strip_comments(c) != bench.strip_comments(a)
    assert len(bench.kernel_source_hash()) == 16
