"""rgs_solve_batched: scenes of uneven size, SH degree, ray count and bounce count solved in one
persistent cooperative launch (captured in a CUDA graph), against the oracle and the per-scene
solver; the bounded grid-barrier wait reports a timeout instead of hanging."""
import numpy as np
import pytest
import torch

from paper_2509_18497_gb300 import api, rgs, scenes

from gpu_helpers import rel_l2, run_oracle

pytestmark = pytest.mark.gpu

SPECS = [  # (n, L, nd, nb, seed)
    (1500, 3, 64, 3, 11), (800, 2, 96, 2, 12), (2400, 3, 128, 4, 13), (1100, 2, 64, 3, 14), (300, 3, 32, 1, 15)]


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build
    build.build()
    scs, pipes, ds = [], [], []
    for n, L, nd, nb, seed in SPECS:
        sc = scenes.with_emission(scenes.fruit_bowl(n=n, L=L, nd=nd, nb=nb, n_lights=3, seed=seed), seed=seed)
        d = api.upload(sc)
        p = api.Pipeline()
        p.build(d)
        p.trace(d)
        scs.append(sc)
        pipes.append(p)
        ds.append(d)
    return scs, pipes, ds


@pytest.mark.parametrize("precision,tol", [(rgs.RGS_FP32, 1e-4), (rgs.RGS_BF16_FP32ACC_RESCORR, 1e-3)])
def test_batched_scenes_match_oracle_and_single_solves(batch, precision, tol):
    scs, pipes, ds = batch
    ts = [p.transport for p in pipes]
    Es = [d["E"] for d in ds]
    nbs = [sc["nb"] for sc in scs]
    B1, norms = rgs.rgs_solve_batched(ts, Es, nbs, precision=precision, norms=True)
    B1 = [b.clone() for b in B1]
    B2, _ = rgs.rgs_solve_batched(ts, Es, nbs, precision=precision)  # replays the captured graph
    for a, b in zip(B1, B2):
        assert torch.equal(a, b)
    for sc, p, d, B, nrm in zip(scs, pipes, ds, B1, norms):
        o = run_oracle(sc)
        assert rel_l2(B.double().cpu().numpy(), o["B"]) <= tol
        Bs, st = p.solve(d["E"], sc["nb"], stats=True, precision=precision)
        assert rel_l2(B.double().cpu().numpy(), Bs.double().cpu().numpy()) <= 1e-5
        np.testing.assert_allclose(nrm, st["residual_norm"], rtol=1e-4)


def test_batch_plan_has_one_bucket_per_scene_shape(batch):
    """The autotuned plan (rgs_batch_last_plan): one bucket per distinct (nc, C, rays per
    surfel) of the batch, each with a policy per row precision and the item width it gives."""
    scs, pipes, ds = batch
    ts = [p.transport for p in pipes]
    rgs.rgs_solve_batched(ts, [d["E"] for d in ds], [sc["nb"] for sc in scs],
                          precision=rgs.RGS_BF16_FP32ACC_RESCORR)
    plan = rgs.rgs_batch_last_plan()
    assert plan is not None and plan["autotuned"] and plan["blocks_per_sm"] in (2, 3) and plan["blocks"] > 0
    shapes = {((L + 1) ** 2, 9, nd) for n, L, nd, nb, seed in SPECS}
    assert {(b["nc"], b["C"], b["rays"]) for b in plan["buckets"]} == shapes
    for b in plan["buckets"]:
        assert b["policy_bf16"] in (0, 1, 2) and b["policy_fp32"] in (0, 1, 2)
        assert b["items_bf16"] in (3, 32) and b["items_fp32"] in (3, 32)
        if b["policy_bf16"] == 0:
            assert b["items_bf16"] == 3


def test_adjoint_after_batched_solve(batch):
    scs, pipes, ds = batch
    ts = [p.transport for p in pipes]
    rgs.rgs_solve_batched(ts, [d["E"] for d in ds], [sc["nb"] for sc in scs])
    for sc, p in zip(scs, pipes):
        W = np.random.default_rng(sc["seed"]).normal(size=(sc["n"], (sc["L"] + 1) ** 2, 9))
        dE, dad, dop = p.adjoint(torch.as_tensor(W, dtype=torch.float32, device="cuda"))
        o = run_oracle(sc, W=W)
        for got, key in ((dE, "dE"), (dad, "dad"), (dop, "dop")):
            assert rel_l2(got.double().cpu().numpy(), o[key]) <= 1e-4, key


def test_barrier_wait_limit_reports_timeout(batch):
    scs, pipes, ds = batch
    ts = [p.transport for p in pipes]
    nbs = [sc["nb"] for sc in scs]
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_solve_batched(ts, None, nbs, use_graph=False, autotune=False, spin_limit=1)
    assert e.value.status == 6
    with pytest.raises(rgs.RgsError) as e:  # adjoint refused: the iterates of a timed-out batch are invalid
        rgs.rgs_adjoint(ts[0], torch.zeros((ts[0].n, ts[0].nc, ts[0].C), device="cuda"))
    assert e.value.status == 7
    B, _ = rgs.rgs_solve_batched(ts, None, nbs, use_graph=False)  # the context is still usable
    assert all(torch.isfinite(b).all() for b in B)
