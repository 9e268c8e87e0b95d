"""The 32-scene uneven batch at full size (surfel counts log-uniform in [5,000, 300,000],
SH degree 2/3, 128-256 rays, 3-5 bounces, 8 lights each), in the launch configuration the
benchmark times: one rgs_solve_batched call with BF16 gathers and the FP32 residual-
correction bounce, captured in a CUDA graph and autotuned.  Sampled receivers of B^(0) and
B^(1) are checked against the oracle computed receiver by receiver on the smallest, a
middle and the largest scene; every scene's B against its own FP32 solve; and the gradients
after the batched solve against those after the FP32 solve."""
import numpy as np
import pytest
import torch

from paper_2509_18497_gb300 import api, rgs, scenes

from gpu_helpers import rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_RESCORR = 1e-3


def test_uneven_batch_full_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_2509_18497_gb300 import build
    build.build()
    scs = scenes.uneven_batch(32)
    ds = [api.upload(sc) for sc in scs]
    pipes = [api.Pipeline(precision=rgs.RGS_BF16_FP32ACC_RESCORR) for _ in scs]
    for p, d in zip(pipes, ds):
        p.build(d)
        p.trace(d)
    ts = [p.transport for p in pipes]
    Bs, norms = rgs.rgs_solve_batched(ts, [d["E"] for d in ds], [sc["nb"] for sc in scs],
                                      precision=rgs.RGS_BF16_FP32ACC_RESCORR, norms=True)
    Bs = [B.double().cpu().numpy() for B in Bs]
    order = np.argsort([sc["n"] for sc in scs])
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    rng = np.random.default_rng(4)
    for s in picks:
        sc = scs[s]
        orc = O.Oracle(sc)
        recv = rng.choice(sc["n"], size=12, replace=False)
        B0 = rgs.rgs_get_iterate(ts[s], 0).double().cpu().numpy()
        assert rel_l2(B0[recv], orc.sample_direct(recv)) <= 1e-4, s
        B1 = rgs.rgs_get_iterate(ts[s], 1).double().cpu().numpy()
        assert rel_l2(B1[recv[:2]], orc.sample_bounce1(recv[:2])) <= 5e-3, s
    # gradients of the batched-solve transports, kept before the FP32 re-solve below
    Ws = [np.random.default_rng(100 + s).normal(size=(sc["n"], (sc["L"] + 1) ** 2, 24)).astype(np.float32)
          for s, sc in enumerate(scs)]
    gb = {}
    for s in picks:
        gb[s] = [x.double().cpu().numpy() for x in pipes[s].adjoint(torch.as_tensor(Ws[s], device="cuda"))]
    for s, (sc, p, d) in enumerate(zip(scs, pipes, ds)):
        Bf, st = p.solve(d["E"], sc["nb"], stats=True, precision=rgs.RGS_FP32)
        assert rel_l2(Bs[s], Bf.double().cpu().numpy()) <= TOL_RESCORR, s
        assert all(np.isfinite(norms[s])) and len(norms[s]) == sc["nb"]
        if s in gb:
            gf = [x.double().cpu().numpy() for x in p.adjoint(torch.as_tensor(Ws[s], device="cuda"))]
            for a, b in zip(gb[s], gf):
                assert rel_l2(a, b) <= TOL_RESCORR, s
    torch.cuda.synchronize()
