"""The 1,000,000-surfel large scene at full size (bowl x4 in a value-noise-textured room,
SH degree 3, 512 rays per surfel, 6 bounces, 16 lights), in the configuration the benchmark
times: BF16 gathers with the FP32 residual-correction bounce and automatically checkpointed
iterates.  Sampled receivers of B^(0) and B^(1) (B^(1) recomputed from its checkpoint)
against the oracle computed receiver by receiver; B and the gradients against the FP32
solve of the same transport."""
import numpy as np
import pytest
import torch

from paper_2509_18497_gb300 import api, rgs, scenes

from gpu_helpers import rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_large_scene_full_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_2509_18497_gb300 import build
    build.build()
    sc = scenes.large_scene()
    d = api.upload(sc)
    pipe = api.Pipeline(precision=rgs.RGS_BF16_FP32ACC_RESCORR, checkpoint=-1)
    pipe.build(d)
    pipe.trace(d)
    Bc, st = pipe.solve(d["E"], sc["nb"], stats=True)
    assert st["n_full_rays"] <= 1e-4 * sc["n"] * sc["nd"]
    res = st["residual_norm"]
    assert all(np.isfinite(res)) and all(b < a for a, b in zip(res, res[1:]))
    orc = O.Oracle(sc)
    rng = np.random.default_rng(5)
    recv = rng.choice(sc["n"], size=16, replace=False)
    B0 = rgs.rgs_get_iterate(pipe.transport, 0).double().cpu().numpy()
    assert rel_l2(B0[recv], orc.sample_direct(recv)) <= 1e-4
    B1 = rgs.rgs_get_iterate(pipe.transport, 1).double().cpu().numpy()
    assert rel_l2(B1[recv[:2]], orc.sample_bounce1(recv[:2])) <= 5e-3
    del B0, B1
    gen = torch.Generator(device="cuda").manual_seed(11)
    g = torch.randn((sc["n"], 16, 48), device="cuda", generator=gen)
    gc = [x.double().cpu().numpy() for x in pipe.adjoint(g)]
    Bc = Bc.double().cpu().numpy()
    Bf, _ = pipe.solve(d["E"], sc["nb"], precision=rgs.RGS_FP32)
    assert rel_l2(Bc, Bf.double().cpu().numpy()) <= 1e-3
    del Bf
    gf = [x.double().cpu().numpy() for x in pipe.adjoint(g)]
    for a, b in zip(gc, gf):
        assert np.all(np.isfinite(a))
        assert rel_l2(a, b) <= 1e-3
