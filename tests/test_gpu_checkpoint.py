"""Checkpointed bounce iterates: a solve that keeps only B^(0), B^(s), ... and an adjoint
that recomputes the iterates between checkpoints must give the same B (bit for bit: the
recomputation replays the same deterministic bounce kernels on the same inputs) and the same
gradients up to summation order (the transposed hit index is filled with atomics, and the
opacity sums group the bounces per checkpoint segment), for every stride, precision and
column layout, and still match the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_2509_18497_gb300 import api, rgs, scenes

from gpu_helpers import rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

ORDER_TOL = 2e-6  # FP32 re-association of the same sums


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build
    build.build()


def _grads_close(a, b, tol=ORDER_TOL):
    for key in ("dE", "dad", "dop"):
        assert rel_l2(a[key], b[key]) <= tol, key


@pytest.mark.parametrize("prec", [rgs.RGS_FP32, rgs.RGS_BF16_FP32ACC, rgs.RGS_BF16_FP32ACC_RESCORR])
def test_strides_match_full_storage(prec):
    sc = scenes.with_emission(scenes.fruit_bowl(n=3000, L=3, nd=64, nb=5), seed=2)
    W = np.random.default_rng(5).normal(size=(sc["n"], 16, 3))
    full = run_gpu(sc, W=W, precision=prec, iterates=True)
    for stride in (1, 2, 3, 4, 5):
        ck = run_gpu(sc, W=W, precision=prec, iterates=True, checkpoint=stride)
        assert np.array_equal(ck["B"], full["B"]), stride
        for b in range(sc["nb"] + 1):  # kept or recomputed, every iterate is the same
            assert np.array_equal(ck["iters"][b], full["iters"][b]), (stride, b)
        _grads_close(ck, full)


def test_checkpointed_against_oracle():
    sc = scenes.with_emission(scenes.box_scene(n=1500, nb=6), seed=3)
    W = np.random.default_rng(8).normal(size=(sc["n"], 9, 3))
    o = run_oracle(sc, W=W)
    g = run_gpu(sc, W=W, checkpoint=2)
    assert rel_l2(g["B"], o["B"]) <= 1e-4
    for key in ("dE", "dad", "dop"):
        assert rel_l2(g[key], o[key]) <= 1e-4, key


@pytest.mark.parametrize("prec", [rgs.RGS_FP32, rgs.RGS_BF16_FP32ACC_RESCORR])
def test_many_columns_checkpointed(prec):
    """16 lights (C = 48): the lane-per-column kernels replay the segments too."""
    sc = scenes.with_emission(scenes.fruit_bowl(n=1500, L=3, nd=64, nb=4, n_lights=16), seed=6)
    W = np.random.default_rng(1).normal(size=(sc["n"], 16, 48))
    full = run_gpu(sc, W=W, precision=prec)
    ck = run_gpu(sc, W=W, precision=prec, checkpoint=3)
    assert np.array_equal(ck["B"], full["B"])
    _grads_close(ck, full)


def test_checkpointing_holds_fewer_iterates():
    sc = scenes.fruit_bowl(n=4000, L=3, nd=64, nb=6, n_lights=4)
    full = run_gpu(sc, precision=rgs.RGS_BF16_FP32ACC_RESCORR)
    ck = run_gpu(sc, precision=rgs.RGS_BF16_FP32ACC_RESCORR, checkpoint=3)
    A = sc["n"] * 12 * 16 * 4
    # full: 7 B + 6 Q + 7 BF16 copies; stride 3: checkpoints B^(0), B^(3) + 2 running + 1 Q
    saved = full["info"]["device_bytes"] - ck["info"]["device_bytes"]
    assert saved >= 7 * A, saved


def test_automatic_mode_keeps_everything_when_it_fits():
    sc = scenes.with_emission(scenes.fruit_bowl(n=2000, L=2, nd=64, nb=4), seed=1)
    W = np.random.default_rng(2).normal(size=(sc["n"], 9, 3))
    full = run_gpu(sc, W=W, iterates=True)
    auto = run_gpu(sc, W=W, iterates=True, checkpoint=-1)
    assert np.array_equal(auto["B"], full["B"])
    assert auto["info"]["device_bytes"] == full["info"]["device_bytes"]


def test_set_checkpointing_rejects_bad_strides():
    sc = scenes.box_scene(n=300, nd=32, nb=2)
    d = api.upload(sc)
    pipe = api.Pipeline()
    pipe.build(d)
    pipe.trace(d)
    for bad in (-2, rgs.RGS_MAX_BOUNCES + 1):
        with pytest.raises(rgs.RgsError):
            rgs.rgs_set_checkpointing(pipe.transport, bad)


def test_pool_shared_between_transports_and_trimmed():
    """Adjoints of two scenes, one after the other on one stream, draw the same pooled
    scratch; results equal those of separate runs, also after the pool is trimmed."""
    s1 = scenes.with_emission(scenes.fruit_bowl(n=2500, L=3, nd=64, nb=3), seed=4)
    s2 = scenes.with_emission(scenes.box_scene(n=1200, nb=3), seed=5)
    W1 = np.random.default_rng(1).normal(size=(s1["n"], 16, 3))
    W2 = np.random.default_rng(2).normal(size=(s2["n"], 9, 3))
    a1, a2 = run_gpu(s1, W=W1), run_gpu(s2, W=W2)
    rgs.rgs_trim_workspace()
    b2, b1 = run_gpu(s2, W=W2), run_gpu(s1, W=W1)
    _grads_close(a1, b1)
    _grads_close(a2, b2)


def _budgeted(sc, W, prec, headroom):
    """Solve + adjoint with the automatic checkpoint stride and a memory budget `headroom`
    bytes above what the traced transport holds; returns the results and the number of
    transposed-index builds the adjoint made."""
    d = api.upload(sc)
    pipe = api.Pipeline(precision=prec, checkpoint=-1)
    pipe.build(d)
    pipe.trace(d)
    held = rgs.rgs_transport_info_get(pipe.transport)["device_bytes"]
    rgs.rgs_set_memory_budget(pipe.transport, held + headroom)
    rgs.rgs_profile_reset()
    rgs.rgs_profile_enable(True)
    B, _ = pipe.solve(d["E"], d["nb"])
    g = torch.as_tensor(np.ascontiguousarray(W, np.float32), device="cuda")
    dE, dad, dop = pipe.adjoint(g)
    torch.cuda.synchronize()
    rgs.rgs_profile_enable(False)
    builds = rgs.rgs_profile_report().get("k_src_fill", (0, 0.0))[0]
    out = dict(B=B.double().cpu().numpy(), dE=dE.double().cpu().numpy(), dad=dad.double().cpu().numpy(),
               dop=dop.double().cpu().numpy(), info=rgs.rgs_transport_info_get(pipe.transport))
    return out, builds


@pytest.mark.parametrize("lights,prec", [(1, rgs.RGS_FP32), (1, rgs.RGS_BF16_FP32ACC_RESCORR),
                                         (20, rgs.RGS_BF16_FP32ACC_RESCORR)])
def test_memory_budget_checkpoints_and_splits_the_index(lights, prec):
    """A budget too small for every iterate and the whole transposed index: the solve picks a
    checkpoint stride and the adjoint splits the index into parts rebuilt per transposed
    bounce; the results are those of the unconstrained run (20 lights: the lane-per-column
    adjoint)."""
    sc = scenes.with_emission(scenes.fruit_bowl(n=3000, L=3, nd=64, nb=5, n_lights=lights), seed=3)
    C = 3 * lights
    W = np.random.default_rng(4).normal(size=(sc["n"], 16, C))
    full = run_gpu(sc, W=W, precision=prec)
    tr_bytes = 8 * full["info"]["n_hits"]
    small, builds = _budgeted(sc, W, prec, headroom=tr_bytes // 3)
    assert builds > 1  # the index was built in parts, for every transposed bounce
    assert np.array_equal(small["B"], full["B"])
    _grads_close(small, full)
