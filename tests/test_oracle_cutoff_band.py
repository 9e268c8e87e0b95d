"""Where the GPU tolerance of the hemisphere rays' geometry gradients on the dense Gaussian
bowl comes from (Sec. 6, Eqs. dl-dgeo-0/1), measured on the oracle alone.

The 3-sigma cutoff of the Gaussian model is a discrete event that both sides hold fixed
when they differentiate, and at the cutoff alpha's derivative in q = u^2 + v^2 is not zero
(-o e^{-9/2}/2).  A hit that FP32 keeps and FP64 drops (or the reverse) therefore moves the
geometry gradients far more than it moves B, and a hit's lever on its receiver's frame
grows with its distance.  Two measurements fix the tolerance:

1. The band: q evaluated in float32 by the GPU's formula (ray-plane depth, crossing point,
   local coordinates) against FP64, over every hit of the 1,500-surfel bowl that lies
   within the outer half of the cutoff disc.  Its largest relative error bounds how far
   FP32 can move a cutoff decision: every hit whose q lies farther than that from 9 is
   decided identically on both sides.
2. The effect: the oracle compiled with its cutoff moved by DELTA (above the band's
   maximum) in either direction.  Every decision FP32 could flip is flipped by one of the
   two builds, so the larger change of dL/dp, dL/ds, dL/dtu, dL/dtv bounds what the
   discrete event can do to the GPU's gradients.

TOL_HEMI_DENSE_GAUSS is that bound with a margin of at most 2x for the FP32 accumulation
of the gradients themselves; the GPU test (test_gpu_geometry.py) imports it from here.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

DELTA = 1e-4                 # relative shift of the cutoff (above the FP32 band, measured below)
TOL_HEMI_DENSE_GAUSS = 2e-3  # GPU tolerance of the dense bowl's geometry gradients
GEO_KEYS = ("dp", "ds", "dtu", "dtv")

_CUT = "        if (r2 > 9.0) return;\n        G = exp(-0.5 * r2);"


def bowl():
    """The dense Gaussian case of the GPU test, every input rounded to float32."""
    from paper_2509_18497_gb300 import scenes
    sc = scenes.with_emission(scenes.fruit_bowl(n=1500, L=3, nd=64, nb=3, n_lights=2), seed=3)
    return {k: (v.astype(np.float32).astype(np.float64) if isinstance(v, np.ndarray) and v.dtype == np.float64
                else v) for k, v in sc.items()}


def _q(dt, o, d, pj, nj, uj, vj, su, sv):
    """q = u^2 + v^2 of the crossing of ray o + t d with surfel j's plane, in dtype dt."""
    w = (pj - o).astype(dt)
    den = (nj * d).sum(1).astype(dt)
    h = (nj * w).sum(1).astype(dt)
    t = (h / den).astype(dt)
    x = (t[:, None] * d - w).astype(dt)
    u = ((x * uj).sum(1) / su).astype(dt)
    v = ((x * vj).sum(1) / sv).astype(dt)
    return (u * u + v * v).astype(dt)


def test_fp32_band_of_the_cutoff_is_below_delta():
    from oracle import oracle as O
    sc = bowl()
    orc = O.Oracle(sc).transport()
    h = orc.hits()
    tu, tv, nn = orc.frames()
    p, s, nd = sc["p"], sc["s"], sc["nd"]
    ray = np.repeat(np.arange(sc["n"] * nd), np.diff(h["off"]))
    i, r, j = ray // nd, ray % nd, h["j"]
    outer = h["G"] < np.exp(-0.5 * 4.0)  # q > 4: the outer half of the disc
    i, r, j = i[outer], r[outer], j[outer]
    d = np.array([orc.ray_dir(int(a), nd, int(sc["seed"]), int(b)) for a, b in zip(i, r)])
    args = (p[i], d, p[j], nn[j], tu[j], tv[j], s[j, 0], s[j, 1])
    q64 = _q(np.float64, *args)
    q32 = _q(np.float32, *(a.astype(np.float32) for a in args))
    band = float(np.max(np.abs(q32.astype(np.float64) - q64) / q64))
    assert 0 < band < DELTA, band
    # few hits sit inside the shifted band at all
    assert np.sum(np.abs(q64 - 9.0) < DELTA * 9.0) < 1e-3 * len(q64)


def _oracle_copy(tmp, name, factor):
    src = open(SRC).read()
    assert src.count(_CUT) == 1
    c_path, so_path = os.path.join(tmp, name + ".c"), os.path.join(tmp, name + ".so")
    with open(c_path, "w") as f:
        f.write(src.replace(_CUT, _CUT.replace("9.0", f"(9.0 * {factor!r})"), 1))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", so_path, c_path, "-lm"],
                   check=True, capture_output=True)
    return so_path


_RUN = r"""
import sys, numpy as np
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
from oracle import oracle as O
from test_oracle_cutoff_band import bowl
sc = bowl()
W = np.random.default_rng(12).normal(size=(sc["n"], 16, 6))
g = O.Oracle(sc).transport().geometry_grad(W, E=sc["E"], nb=sc["nb"])
np.savez({out!r}, **{{k: g[k] for k in ("dp", "ds", "dtu", "dtv")}})
"""


@pytest.mark.slow
def test_tolerance_follows_the_oracles_cutoff_sensitivity(tmp_path):
    tmp = str(tmp_path)
    libs = {"base": _oracle_copy(tmp, "base", 1.0), "up": _oracle_copy(tmp, "up", 1.0 + DELTA),
            "down": _oracle_copy(tmp, "down", 1.0 - DELTA)}
    threads = str(max(1, (os.cpu_count() or 3) // 3))
    procs = {}
    for name, so in libs.items():
        out = os.path.join(tmp, name + ".npz")
        code = _RUN.format(root=ROOT, tests=os.path.join(ROOT, "tests"), out=out)
        env = dict(os.environ, ORACLE_LIB=so, OMP_NUM_THREADS=threads)
        procs[name] = (subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT), out)
    for name, (p, _) in procs.items():
        assert p.wait(timeout=1200) == 0, name
    g = {name: np.load(out) for name, (_, out) in procs.items()}
    change = max(float(np.linalg.norm(g[s][k] - g["base"][k]) / np.linalg.norm(g["base"][k]))
                 for s in ("up", "down") for k in GEO_KEYS)
    # the discrete event is visible (so the measurement means something) and the tolerance
    # covers it with a margin of at most 2x
    assert change > 1e-5, change
    assert change <= TOL_HEMI_DENSE_GAUSS <= 2.0 * change, change
