"""The batched precision modes against the FP64 oracle: bounces gather BF16 copies of the
iterates with FP32 accumulation (relative L2 <= 5e-3), and the residual-corrected form,
whose last bounce gathers FP32 rows (relative L2 <= 1e-3).  BF16 keeps 8 significant bits
(relative rounding 2^-9 ~ 2e-3 per coefficient); the per-hit errors are independent and
average down in the gather, so 5e-3 bounds B; the corrected bounce multiplies the
remaining error by K, whose spectral radius here is below 1/2."""
import numpy as np
import pytest
import torch

from paper_2509_18497_gb300 import rgs, scenes

from gpu_helpers import rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL_BF16, TOL_RESCORR = 5e-3, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build
    build.build()


@pytest.mark.parametrize("L", [3, 2, 1, 0])
def test_batched_modes_forward_and_gradients(L):
    sc = scenes.with_emission(scenes.fruit_bowl(n=3000, L=L, nd=64, nb=3), seed=4)
    nc = (L + 1) ** 2
    W = np.random.default_rng(9).normal(size=(sc["n"], nc, 3))
    o = run_oracle(sc, W=W)
    g = run_gpu(sc, W=W, precision=rgs.RGS_BF16_FP32ACC)
    assert rel_l2(g["B"], o["B"]) <= TOL_BF16
    for key in ("dE", "dad", "dop"):
        assert rel_l2(g[key], o[key]) <= TOL_BF16, key
    c = run_gpu(sc, W=W, precision=rgs.RGS_BF16_FP32ACC_RESCORR)
    assert rel_l2(c["B"], o["B"]) <= TOL_RESCORR
    assert rel_l2(c["B"], o["B"]) < rel_l2(g["B"], o["B"])   # the FP32 sweep helps
    for key in ("dE", "dad", "dop"):
        assert rel_l2(c[key], o[key]) <= TOL_BF16, key


@pytest.mark.parametrize("L", [3, 2])
def test_many_lights_lane_per_column(L):
    """20 lights (C = 60 columns): the lane-per-column kernels, every precision."""
    sc = scenes.with_emission(scenes.fruit_bowl(n=2000, L=L, nd=64, nb=2, n_lights=20), seed=7)
    nc = (L + 1) ** 2
    C = 60
    W = np.random.default_rng(3).normal(size=(sc["n"], nc, C))
    o = run_oracle(sc, W=W)
    for prec, tol in ((rgs.RGS_FP32, 1e-4), (rgs.RGS_BF16_FP32ACC, TOL_BF16), (rgs.RGS_BF16_FP32ACC_RESCORR, TOL_RESCORR)):
        g = run_gpu(sc, W=W, precision=prec)
        assert g["B"].shape == (sc["n"], nc, C)
        assert rel_l2(g["B"], o["B"]) <= tol, prec
        gtol = 1e-4 if prec == rgs.RGS_FP32 else TOL_BF16
        for key in ("dE", "dad", "dop"):
            assert rel_l2(g[key], o[key]) <= gtol, (prec, key)


@pytest.mark.slow
def test_hundred_lights_full_size_sampled():
    """200,000 surfels, 100 lights (C = 300), 256 rays, 4 bounces, batched with residual
    correction: sampled direct terms and first bounces against the oracle computed receiver by
    receiver, and the final B against the FP32 form on the whole scene."""
    from oracle import oracle as O
    sc = scenes.multi_light(n=200000)
    g = run_gpu(sc, iterates=True, precision=rgs.RGS_BF16_FP32ACC_RESCORR)
    orc = O.Oracle(sc)
    rng = np.random.default_rng(1)
    recv = rng.choice(sc["n"], size=24, replace=False)
    assert rel_l2(g["iters"][0][recv], orc.sample_direct(recv)) <= 1e-4
    recv1 = recv[:3]
    assert rel_l2(g["iters"][1][recv1], orc.sample_bounce1(recv1)) <= TOL_BF16
    f = run_gpu(sc, precision=rgs.RGS_FP32)
    assert rel_l2(g["B"], f["B"]) <= TOL_RESCORR
