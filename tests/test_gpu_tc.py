"""The tensor-core contraction of the batched modes (rgs_set_tensor_cores) against the FP64
oracle, forward and adjoint (Eq. final-radiosity, Eq. final_dL_dE; Sec. 7's many-light
batching).

Each (receiver tile, source) group forms eight 16 x 16 transport blocks in FP32 from the
group's hits and rounds them to BF16 (relative 2^-9); the source rows are BF16 too.  The
rounding errors of the ~10^3 blocks and rows a receiver sums are independent, so they
average down as in the row-gather form: the BF16 bar (5e-3) applies to B and to the
gradients (the transposed bounces also take BF16 y = o c (x) v).  The corrected mode's last
bounce multiplies the BF16 high and low parts of both operands (three products), an
FP32-level application of K to the BF16 iterate, so B meets 1e-3 as in the row-gather
form.  Cases cover one light (16 padded columns: one MMA piece), 20 lights (64 columns) and
100 lights (304 columns: two pieces, 256 + 48), ragged last tiles (n not a multiple of 8)
and the GFSGS opacity model."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_18497_gb300 import rgs, scenes

from gpu_helpers import rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL_FP32, TOL_BF16, TOL_RESCORR = 1e-4, 5e-3, 1e-3
TC = 1  # rgs_set_tensor_cores: the tensor-core form wherever it applies


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build
    build.build()


def _check(sc, W, o, alpha_model=rgs.RGS_ALPHA_GAUSS, mode=TC):
    errs = {}
    for prec, tol in ((rgs.RGS_BF16_FP32ACC, TOL_BF16), (rgs.RGS_BF16_FP32ACC_RESCORR, TOL_RESCORR)):
        g = run_gpu(sc, W=W, precision=prec, tensor_cores=mode, stats=True, alpha_model=alpha_model)
        errs[prec] = rel_l2(g["B"], o["B"])
        assert errs[prec] <= tol, (prec, errs[prec])
        for key in ("dE", "dad", "dop"):
            e = rel_l2(g[key], o[key])
            assert e <= TOL_BF16, (prec, key, e)
        res = g["stats"]["residual_norm"][:sc["nb"]]
        assert all(np.isfinite(res)) and all(x > 0 for x in res)
    assert errs[rgs.RGS_BF16_FP32ACC_RESCORR] < errs[rgs.RGS_BF16_FP32ACC]  # the split bounce helps
    return errs


@pytest.mark.parametrize("n_lights", [1, 20])
def test_tensor_cores_against_oracle(n_lights):
    """Mode 1 (bounces, transposed bounces and the opacity gather's sampled products on the
    tensor cores), mode 2 (the opacity gather as per-(tile, receiver) products instead) and
    mode 3 (the opacity gather as row gathers)."""
    sc = scenes.with_emission(scenes.fruit_bowl(n=2997, L=3, nd=64, nb=3, n_lights=n_lights), seed=4)
    C = 3 * n_lights
    W = np.random.default_rng(9).normal(size=(sc["n"], 16, C))
    o = run_oracle(sc, W=W)
    _check(sc, W, o, mode=1)
    _check(sc, W, o, mode=2)
    _check(sc, W, o, mode=3)


def test_tensor_cores_gfsgs():
    sc = scenes.with_emission(scenes.fruit_bowl(n=1501, L=3, nd=64, nb=2, n_lights=3), seed=6)
    W = np.random.default_rng(2).normal(size=(sc["n"], 16, 9))
    o = run_oracle(sc, W=W, alpha_model=O.ALPHA_GFSGS)
    _check(sc, W, o, alpha_model=rgs.RGS_ALPHA_GFSGS, mode=2)
    _check(sc, W, o, alpha_model=rgs.RGS_ALPHA_GFSGS, mode=3)


def test_tensor_cores_match_row_gathers():
    """The same batched mode through both contractions: equal up to the BF16 rounding of the
    transport blocks (the row-gather form keeps them in FP32)."""
    sc = scenes.fruit_bowl(n=4000, L=3, nd=64, nb=3, n_lights=8)
    W = np.random.default_rng(1).normal(size=(sc["n"], 16, 24))
    a = run_gpu(sc, W=W, precision=rgs.RGS_BF16_FP32ACC_RESCORR, tensor_cores=TC)
    b = run_gpu(sc, W=W, precision=rgs.RGS_BF16_FP32ACC_RESCORR, tensor_cores=0)
    assert rel_l2(a["B"], b["B"]) <= TOL_RESCORR
    for key in ("dE", "dad", "dop"):
        assert rel_l2(a[key], b[key]) <= TOL_BF16, key


def test_opacity_products_respect_the_memory_budget():
    """A memory budget that leaves no room beside the transport for a 64-column pass of y
    rows: the adjoint's opacity gather takes the row gathers instead (mode 3's form, the
    same results), and the gradients still meet the BF16 bar against the oracle."""
    from paper_2509_18497_gb300 import api
    sc = scenes.with_emission(scenes.fruit_bowl(n=2001, L=3, nd=64, nb=2, n_lights=40), seed=3)
    W = np.random.default_rng(6).normal(size=(sc["n"], 16, 120))
    o = run_oracle(sc, W=W)
    g = torch.as_tensor(np.ascontiguousarray(W, np.float32), device="cuda")
    out = {}
    for mode, budget in ((3, False), (1, True)):
        d = api.upload(sc)
        pipe = api.Pipeline(precision=rgs.RGS_BF16_FP32ACC, tensor_cores=mode)
        pipe.build(d)
        pipe.trace(d)
        pipe.solve(d["E"], d["nb"])
        if budget:
            rgs.rgs_set_memory_budget(pipe.transport, rgs.rgs_transport_info_get(pipe.transport)["device_bytes"])
        rgs.rgs_profile_reset()
        rgs.rgs_profile_enable(True)
        dE, dad, dop = pipe.adjoint(g)
        torch.cuda.synchronize()
        rgs.rgs_profile_enable(False)
        rep = rgs.rgs_profile_report()
        assert rep.get("k_tc_opa", (0, 0.0))[0] == 0 and rep.get("k_opacity_g_mc", (0, 0.0))[0] > 0, (mode, rep)
        out[mode] = dop.double().cpu().numpy()
        assert rel_l2(out[mode], o["dop"]) <= TOL_BF16
    assert rel_l2(out[1], out[3]) <= 1e-6


def test_tensor_core_wait_limit_reports_timeout():
    """Failure detection without a GPU fault: with a 1 ns limit the pipeline's waits run out,
    every role stops (after draining its own copies and MMAs) and the solve returns
    RGS_ERR_TIMEOUT; with the default limit the same transport solves again, correctly."""
    from paper_2509_18497_gb300 import api
    sc = scenes.fruit_bowl(n=1200, L=3, nd=64, nb=2, n_lights=8)
    d = api.upload(sc)
    pipe = api.Pipeline(precision=rgs.RGS_BF16_FP32ACC, tensor_cores=TC)
    pipe.build(d)
    pipe.trace(d)
    rgs.rgs_set_wait_limit(pipe.transport, 1)
    with pytest.raises(rgs.RgsError) as err:
        pipe.solve(d["E"], d["nb"])
    assert err.value.status == 6  # RGS_ERR_TIMEOUT
    torch.cuda.synchronize()
    rgs.rgs_set_wait_limit(pipe.transport, 0)
    B, _ = pipe.solve(d["E"], d["nb"])
    ref = run_gpu(sc, precision=rgs.RGS_BF16_FP32ACC, tensor_cores=0)
    assert rel_l2(B.double().cpu().numpy(), ref["B"]) <= TOL_BF16
    # the adjoint (transposed bounces and the sampled-product opacity gather): their waits
    # run out as well
    g = torch.ones((sc["n"], 16, 24), device="cuda")
    rgs.rgs_set_wait_limit(pipe.transport, 1)
    with pytest.raises(rgs.RgsError) as err:
        pipe.adjoint(g)
    assert err.value.status == 6
    torch.cuda.synchronize()
    rgs.rgs_set_wait_limit(pipe.transport, 0)
    dE, dad, dop = pipe.adjoint(g)
    ref = run_gpu(sc, W=np.ones((sc["n"], 16, 24)), precision=rgs.RGS_BF16_FP32ACC, tensor_cores=0)
    assert rel_l2(dop.double().cpu().numpy(), ref["dop"]) <= TOL_BF16


@pytest.fixture(scope="module")
def hundred():
    """100 lights (C = 300) on a 2,000-surfel bowl with 64 rays and 3 bounces: small enough for
    the oracle's full forward and adjoint."""
    sc = scenes.with_emission(scenes.multi_light(n=2000, nd=64, nb=3), seed=5)
    W = np.random.default_rng(4).normal(size=(sc["n"], 16, 300))
    return sc, W, run_oracle(sc, W=W)


def test_hundred_lights_tensor_cores_full_oracle(hundred):
    sc, W, o = hundred
    _check(sc, W, o, mode=1)
    _check(sc, W, o, mode=2)
    _check(sc, W, o, mode=3)


def test_opacity_products_in_two_column_passes():
    """120 lights (C = 360): the sampled-product opacity gather (mode 1) forms the rays' y rows
    in passes of at most 320 columns, so this case takes two (320 + 40 columns, the second
    padded with zeros to 64).  Against the oracle on every gradient entry, and against the
    row-gather opacity kernels (mode 3) on the same bounces: equal up to the BF16 rounding
    of y and of the source rows."""
    sc = scenes.with_emission(scenes.multi_light(n=603, nd=32, nb=2, n_lights=120), seed=8)
    W = np.random.default_rng(12).normal(size=(sc["n"], 16, 360))
    o = run_oracle(sc, W=W)
    _check(sc, W, o, mode=1)
    a = run_gpu(sc, W=W, precision=rgs.RGS_BF16_FP32ACC, tensor_cores=1)
    b = run_gpu(sc, W=W, precision=rgs.RGS_BF16_FP32ACC, tensor_cores=3)
    assert rel_l2(a["dE"], b["dE"]) <= 1e-6  # the same transposed bounces
    assert rel_l2(a["dop"], b["dop"]) <= TOL_BF16


def test_hundred_lights_fp32_and_row_gathers_full_oracle(hundred):
    """The FP32 form (lane-per-column gathers, 10 column tiles) and the corrected row-gather
    form at C = 300 against the oracle on every entry of B and of the three gradients."""
    sc, W, o = hundred
    f = run_gpu(sc, W=W, precision=rgs.RGS_FP32)
    assert rel_l2(f["B"], o["B"]) <= TOL_FP32
    for key in ("dE", "dad", "dop"):
        assert rel_l2(f[key], o[key]) <= TOL_FP32, key
    c = run_gpu(sc, W=W, precision=rgs.RGS_BF16_FP32ACC_RESCORR, tensor_cores=0)
    assert rel_l2(c["B"], o["B"]) <= TOL_RESCORR
    for key in ("dE", "dad", "dop"):
        assert rel_l2(c[key], o[key]) <= TOL_BF16, key


def test_hundred_lights_partitioned_index_full_oracle(hundred):
    """A memory budget too small for the transposed index (8 bytes per hit) and every iterate:
    the solve checkpoints, the adjoint splits the index into parts rebuilt for every
    transposed bounce, and the FP32 results still match the oracle on every entry."""
    from paper_2509_18497_gb300 import api
    sc, W, o = hundred
    d = api.upload(sc)
    pipe = api.Pipeline(precision=rgs.RGS_FP32, checkpoint=-1)
    pipe.build(d)
    pipe.trace(d)
    info = rgs.rgs_transport_info_get(pipe.transport)
    rgs.rgs_set_memory_budget(pipe.transport, info["device_bytes"] + 8 * info["n_hits"] // 3)
    rgs.rgs_profile_reset()
    rgs.rgs_profile_enable(True)
    B, _ = pipe.solve(d["E"], d["nb"])
    g = torch.as_tensor(np.ascontiguousarray(W, np.float32), device="cuda")
    dE, dad, dop = pipe.adjoint(g)
    torch.cuda.synchronize()
    rgs.rgs_profile_enable(False)
    assert rgs.rgs_profile_report().get("k_src_fill", (0, 0.0))[0] > 1  # built in parts
    assert rel_l2(B.double().cpu().numpy(), o["B"]) <= TOL_FP32
    for key, x in (("dE", dE), ("dad", dad), ("dop", dop)):
        assert rel_l2(x.double().cpu().numpy(), o[key]) <= TOL_FP32, key
