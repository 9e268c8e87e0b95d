"""Directional lights on the GPU (Sec. 5.1: distant lights without the inverse-square
falloff; the 16 x 32 environment map of Sec. 9 as such lights) against the FP64 oracle:
iterates and gradients with a few directional lights and with a small environment map, for
both transports; the full 512-light map on a 2,000-surfel bowl with sampled receivers."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_18497_gb300 import rgs, scenes

from gpu_helpers import rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build
    build.build()


def _directional(sc, n_lights, seed):
    rng = np.random.default_rng(seed)
    out = dict(sc)
    out["light_pos"] = rng.normal(size=(n_lights, 3)).astype(np.float32).astype(np.float64)
    out["light_I"] = rng.uniform(0.5, 3.0, size=(n_lights, 3)).astype(np.float32).astype(np.float64)
    out["light_dir"] = True
    return out


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("maker", [
    lambda: _directional(scenes.with_emission(scenes.fruit_bowl(n=2000, L=2, nd=64, nb=3), seed=1), 4, 2),
    lambda: scenes.with_env_map(scenes.fruit_bowl(n=1200, L=2, nd=64, nb=3), n_theta=4, n_phi=8),
])
def test_directional_lights_match_oracle(maker, pairs):
    sc = maker()
    nc = (sc["L"] + 1) ** 2
    C = 3 * sc["light_pos"].shape[0]
    W = np.random.default_rng(5).normal(size=(sc["n"], nc, C))
    o = run_oracle(sc, W=W, iterates=True, pairs=pairs)
    g = run_gpu(sc, W=W, iterates=True, pairs=pairs)
    for b, (gi, oi) in enumerate(zip(g["iters"], o["iters"])):
        assert rel_l2(gi, oi) <= TOL, b
    keys = ("dE", "dad", "dop", "dlam") if pairs else ("dE", "dad", "dop")
    for key in keys:
        assert rel_l2(g[key], o[key]) <= TOL, key


def test_full_env_map_sampled():
    """The 16 x 32 map (512 lights, C = 1,536 columns) on a 2,000-surfel bowl, batched with
    residual correction: sampled direct terms and first bounces against the oracle, B against
    the FP32 form."""
    sc = scenes.with_env_map(scenes.fruit_bowl(n=2000, L=2, nd=64, nb=3))
    g = run_gpu(sc, iterates=True, precision=rgs.RGS_BF16_FP32ACC_RESCORR)
    orc = O.Oracle(sc)
    recv = np.random.default_rng(3).choice(sc["n"], size=8, replace=False)
    assert rel_l2(g["iters"][0][recv], orc.sample_direct(recv)) <= TOL
    assert rel_l2(g["iters"][1][recv[:2]], orc.sample_bounce1(recv[:2])) <= 5e-3
    f = run_gpu(sc, precision=rgs.RGS_FP32)
    assert rel_l2(g["B"], f["B"]) <= 1e-3
