"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerance (FP32 path): relative L2 <= 1e-4 over every (surfel, coefficient, column)
entry of B and of each gradient.  Derivation: FP32 accumulation over <= nd * H ~ 1e4
terms per receiver gives ~1e-6 relative rounding; a hit whose acceptance flips
between FP32 and FP64 at the 3-sigma cutoff or the eps_plane boundary changes one ray
by ~1% of alpha, i.e. ~1e-5 of a receiver, and such flips are rare; the stopping of
compositing below a transmittance of 1e-6 changes results by < 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_18497_gb300 import api, rgs, scenes

from gpu_helpers import rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build
    build.build()
    rgs.load()


def _W(sc, C, seed=9):
    nc = (sc["L"] + 1) ** 2
    return np.random.default_rng(seed).normal(size=(sc["n"], nc, C))


def test_box_scene_forward_all_iterates():
    """Closed box, N=2000, L=2, 64 rays, 3 bounces, 1 light (the small plain-FP32 case)."""
    sc = scenes.box_scene()
    g = run_gpu(sc, iterates=True)
    o = run_oracle(sc, iterates=True)
    for b in range(sc["nb"] + 1):
        assert rel_l2(g["iters"][b], o["iters"][b]) <= TOL, b
    assert rel_l2(g["B"], o["B"]) <= TOL
    # the stored records are the oracle's hits up to the transmittance cut
    h = o["orc"].hits()
    T_before = np.ones_like(h["alpha"])
    for r in range(len(h["off"]) - 1):
        a = h["alpha"][h["off"][r]:h["off"][r + 1]]
        T_before[h["off"][r]:h["off"][r + 1]] = np.concatenate([[1.0], np.cumprod(1 - a)[:-1]])
    kept = int(np.sum(T_before >= 1e-6))
    assert abs(g["info"]["n_hits"] - kept) <= 1e-4 * kept + 10


def test_fruit_bowl_forward_and_gradients():
    """Fruit bowl generator at N=3000, L=3, specular, emission, 3 bounces: B and the
    gradients w.r.t. emission, diffuse albedo and opacity."""
    sc = scenes.with_emission(scenes.fruit_bowl(n=3000, nd=64, nb=3), seed=4)
    W = _W(sc, 3)
    g = run_gpu(sc, W=W)
    o = run_oracle(sc, W=W)
    assert rel_l2(g["B"], o["B"]) <= TOL
    assert rel_l2(g["dE"], o["dE"]) <= TOL
    assert rel_l2(g["dad"], o["dad"]) <= TOL
    assert rel_l2(g["dop"], o["dop"]) <= TOL


def test_multi_light_columns():
    """Five lights as five right-hand-side groups (C = 15), L=2."""
    sc = scenes.with_emission(scenes.random_cluster(n=700, seed=3, L=2, nd=96, nb=2, n_lights=5, extent=2.0), seed=2)
    W = _W(sc, 15)
    g = run_gpu(sc, W=W)
    o = run_oracle(sc, W=W)
    assert g["B"].shape == (700, 9, 15)
    assert rel_l2(g["B"], o["B"]) <= TOL
    for key in ("dE", "dad", "dop"):
        assert rel_l2(g[key], o[key]) <= TOL, key


def test_furnace_exact_on_gpu():
    sc = scenes.furnace_sphere(m=1500, rho=0.6, emission=1.0, nd=64, nb=4)
    g = run_gpu(sc, alpha_model=rgs.RGS_ALPHA_DISC)
    r, e = sc["ad"][0, 0], sc["E"][0, 0, 0]
    expect = e * sum(r ** m for m in range(sc["nb"] + 1))
    np.testing.assert_allclose(g["B"][:, 0, :], expect, rtol=2e-5)
    assert np.abs(g["B"][:, 1:, :]).max() < 1e-5


@pytest.mark.parametrize("L", [0, 1, 2, 3])
def test_sh_degrees_and_ragged_sizes(L):
    """Every SH degree, a surfel count that fills no tile evenly, 32 rays (one warp)."""
    sc = scenes.with_emission(scenes.box_scene(n=1237, L=L, nd=32, nb=2), seed=L)
    W = _W(sc, 3, seed=L)
    g = run_gpu(sc, W=W)
    o = run_oracle(sc, W=W)
    assert rel_l2(g["B"], o["B"]) <= TOL
    for key in ("dE", "dad", "dop"):
        assert rel_l2(g[key], o[key]) <= TOL, key


def test_degenerate_scenes():
    # one surfel: the direct term only (no hits), closed form through the oracle
    sc = scenes.lone_plane(L=3, k=0.6, as_=(0.4, 0.3, 0.2), shin=2.0)
    g = run_gpu(sc)
    o = run_oracle(sc)
    assert rel_l2(g["B"], o["B"]) <= 1e-6
    # no lights: emission only, one column group
    sc = scenes.with_emission(scenes.box_scene(n=500, nd=64, nb=2), seed=1)
    sc = dict(sc, light_pos=np.zeros((0, 3)), light_I=np.zeros((0, 3)))
    W = _W(sc, 3)
    g = run_gpu(sc, W=W)
    o = run_oracle(sc, W=W)
    assert g["B"].shape[2] == 3
    assert rel_l2(g["B"], o["B"]) <= TOL
    for key in ("dE", "dad", "dop"):
        assert rel_l2(g[key], o[key]) <= TOL, key
    # zero bounces: B = S
    sc = dict(scenes.box_scene(n=400, nd=32), nb=0)
    assert rel_l2(run_gpu(sc)["B"], run_oracle(sc)["B"]) <= 1e-5


def test_errors_are_reported_not_raised_on_device():
    sc = scenes.box_scene(n=300, nd=32)
    d = api.upload(sc)
    pipe = api.Pipeline()
    pipe.build(d)
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_trace_transport(pipe.scene, d["light_pos"], d["light_I"], nd=48, seed=0)
    assert e.value.status == 1
    with pytest.raises(rgs.RgsError) as e:  # capacity too small: reported, never overrun
        rgs.rgs_trace_transport(pipe.scene, d["light_pos"], d["light_I"], nd=32, seed=0, hit_capacity=64)
    assert e.value.status == 4
    t = rgs.rgs_trace_transport(pipe.scene, d["light_pos"], d["light_I"], nd=32, seed=0)
    with pytest.raises(rgs.RgsError) as e:  # adjoint before any solve
        rgs.rgs_adjoint(t, torch.zeros((300, 9, 3), device="cuda"))
    assert e.value.status == 7
    bad = dict(d)
    bad["p"] = d["p"].clone()
    bad["p"][7, 1] = float("nan")
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_build_scene(*[bad[k] for k in api.SURFEL_KEYS], sh_degree=2, check_finite=True)
    assert e.value.status == 5
    # the handle and context still work after the reported errors
    B, _ = rgs.rgs_solve(t, None, 1)
    assert torch.isfinite(B).all()


def test_autograd_function_matches_adjoint():
    sc = scenes.with_emission(scenes.box_scene(n=600, nd=32, nb=2), seed=5)
    d = api.upload(sc)
    E = d["E"].clone().requires_grad_(True)
    ad = d["ad"].clone().requires_grad_(True)
    o = d["o"].clone().requires_grad_(True)
    B = api.radiosity(E, ad, o, d, 2)
    W = torch.randn_like(B)
    (B * W).sum().backward()
    ref = run_oracle(sc, W=W.double().cpu().numpy())
    assert rel_l2(E.grad.double().cpu().numpy(), ref["dE"]) <= TOL
    assert rel_l2(ad.grad.double().cpu().numpy(), ref["dad"]) <= TOL
    assert rel_l2(o.grad.double().cpu().numpy(), ref["dop"]) <= TOL


@pytest.mark.slow
def test_fruit_bowl_full_size_sampled():
    """The 50,000-surfel fruit bowl at 256 rays and 4 bounces, in the configuration the
    benchmark times: sampled receivers of the direct term D = B^(0) and of the first
    bounce B^(1) against the oracle computed receiver by receiver, plus the duality
    <W, B^(n)> = <dL/dS, S> that holds at any size."""
    sc = scenes.fruit_bowl(n=50000)
    W = _W(sc, 3)
    g = run_gpu(sc, W=W, iterates=True, stats=True)
    orc = O.Oracle(sc)
    rng = np.random.default_rng(0)
    recv = rng.choice(sc["n"], size=48, replace=False)
    D = orc.sample_direct(recv)
    assert rel_l2(g["iters"][0][recv], D) <= TOL
    recv1 = recv[:12]
    B1 = orc.sample_bounce1(recv1)
    assert rel_l2(g["iters"][1][recv1], B1) <= TOL
    lhs = float(np.sum(W * g["B"]))
    rhs = float(np.sum(g["dE"] * g["iters"][0]))  # one light: u = dL/dE, S = B^(0)
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    assert g["stats"]["n_full_rays"] <= 1e-4 * sc["n"] * sc["nd"]
    res = g["stats"]["residual_norm"]
    assert all(b < a for a, b in zip(res, res[1:]))
