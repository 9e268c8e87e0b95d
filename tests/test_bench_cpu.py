"""The bench's CPU-side pieces: the reference arm (the FP64 oracle timed on host cores)
prints one contract JSON line, and the per-kernel algorithmic-byte table covers the
kernels the step launches (no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-sample", "200"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_algorithmic_bytes_cover_the_step_kernels():
    import bench
    sc = dict(n=1000, nd=64, nb=3, C=6, nc=16, n_hits=200000)
    for k in ("k_trace_hemi", "k_bounce", "k_bounce_mc", "k_adj_src", "k_adj_ray", "k_opacity_g", "k_opacity_rec",
              "k_src_fill", "k_pair_fill", "k_bounce_pairs", "k_pair_grad", "k_pair_g", "k_tc_opa", "k_tc_opa_y"):
        b, launches = bench._launch_bytes(k, sc)
        assert b is not None and b > 0 and launches > 0, k
    # the opacity products take one pass of at most 320 columns per pairing: 1,536 columns
    # (the environment map) in five passes, each reading 2 B per hit and pass column
    wide = dict(sc, C=1536)
    b, launches = bench._launch_bytes("k_tc_opa", wide)
    assert launches == 5 * wide["nb"]
    assert b >= wide["n_hits"] * 2 * 320
