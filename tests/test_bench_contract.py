"""bench.py's reference arm (the oracle timed on the host cores) prints one
JSON line with the keys of the bench contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-500:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["unit"] == "DOFs/s" and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["n_gpus"] == 1
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert "workload" in line["config"]


def test_roofline_byte_model():
    """The algorithmic bytes the bench divides by launch time: stored stencil
    words per unknown (the FP32 scalar kernels read the symmetric half, 14 of
    27 in 3D and 5 of 9 in 2D; FP64 data the full stencil; 81 for
    elasticity) and the per-unknown figures of the block kernels."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.stencil_words(3, 4) == 14 and bench.stencil_words(2, 4) == 5
    assert bench.stencil_words(3, 8) == 27 and bench.stencil_words(2, 8) == 9
    assert bench.stencil_words(3, 4, vector=True) == 81
    n, C, w = 1000, 6, 4
    b, f = bench.kernel_work("spmm", n, C, 0, w, S=14)
    assert b == (14 + 2 * C) * w * n and f == 2 * (27 * C + C) * n   # products of the full stencil
    b, f = bench.kernel_work("spmm", n, C, 0, 8, S=27)
    assert b == (27 + 2 * C) * 8 * n and f == 2 * (27 * C + C) * n
    b, _ = bench.kernel_work("orth_update", n, C, 5, w)
    assert b == (2 * 5 * C + 4 * C + 1) * w * n
    assert bench.bmin_per_iteration(1, n, C, 5, w, 14) == ((2 * C + 4) * w + 14 * w) * n
    # one MG chain of two grids with fused nu = 2 Jacobi: (S + 3) w per unknown of each grid
    ns = [10, 100]
    trace = [("init", 0.0), ("jacobi", 1.0), ("jacobi", 1.0), ("check", 0.0)]
    dom, rl, share, tot = bench.roofline(trace, ns, 2, 5, 4, {"hbm_gbs": 1000.0}, None, S=14)
    assert dom == "jacobi" and rl["launches"] == 2
    assert rl["algorithmic_bytes_per_launch"] == (14 + 3) * 4 * (ns[1] + ns[0]) / 2
