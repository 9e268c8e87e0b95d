"""The center-to-center transport (Sec. 8 approximation: one segment per pair of surfel
centres, V_ji = lambda_j int(alpha_j) T_ij |n_i.w||n_j.w|/r^2) on the GPU against the FP64
oracle: pair lists, iterates, B and the gradients with respect to E, a^d, o and lambda, in
every precision; the closed-sphere furnace closed form."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_18497_gb300 import api, rgs, scenes

from gpu_helpers import rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL, TOL_BF16, TOL_RESCORR = 1e-4, 5e-3, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build
    build.build()


def _with_lam(sc, seed):
    out = dict(sc)
    out["lam"] = np.random.default_rng(seed).uniform(0.5, 1.5, sc["n"]).astype(np.float32).astype(np.float64)
    return out


@pytest.mark.parametrize("maker", [
    lambda: scenes.with_emission(scenes.box_scene(n=900, nb=3), seed=2),
    lambda: _with_lam(scenes.with_emission(scenes.fruit_bowl(n=1500, L=3, nb=3, n_lights=2), seed=3), 4),
    lambda: _with_lam(scenes.with_emission(scenes.random_cluster(n=300, L=2, nb=4, n_lights=3), seed=5), 6),
])
def test_pairs_match_oracle(maker):
    sc = maker()
    nc = (sc["L"] + 1) ** 2
    C = 3 * max(1, sc["light_pos"].shape[0])
    W = np.random.default_rng(7).normal(size=(sc["n"], nc, C))
    o = run_oracle(sc, W=W, iterates=True, pairs=True)
    g = run_gpu(sc, W=W, iterates=True, pairs=True)
    n_or = len(o["orc"].pair_list()["j"])
    assert abs(g["info"]["n_hits"] - n_or) <= max(2, 1e-4 * n_or)  # front-test flips at eps only
    for b, (gi, oi) in enumerate(zip(g["iters"], o["iters"])):
        assert rel_l2(gi, oi) <= TOL, b
    for key in ("dE", "dad", "dop", "dlam"):
        assert rel_l2(g[key], o[key]) <= TOL, key


@pytest.mark.parametrize("prec,tol", [(rgs.RGS_BF16_FP32ACC, TOL_BF16), (rgs.RGS_BF16_FP32ACC_RESCORR, TOL_RESCORR)])
def test_pairs_batched_precisions(prec, tol):
    sc = _with_lam(scenes.with_emission(scenes.fruit_bowl(n=1200, L=3, nb=3, n_lights=2), seed=8), 9)
    W = np.random.default_rng(1).normal(size=(sc["n"], 16, 6))
    o = run_oracle(sc, W=W, pairs=True)
    g = run_gpu(sc, W=W, precision=prec, pairs=True)
    assert rel_l2(g["B"], o["B"]) <= tol
    for key in ("dE", "dad", "dop", "dlam"):
        assert rel_l2(g[key], o[key]) <= TOL_BF16, key


def test_pairs_furnace_closed_form():
    """The oracle's closed-sphere pin on the GPU: B^(n)_00 = e sum_m kappa^m with
    kappa = rho (M-1) s^2 / 4, other coefficients 0 (disc model, o = 1)."""
    m, rho, nb = 600, 0.05, 4
    sc = scenes.furnace_sphere(m=m, rho=rho, emission=1.0, nb=nb)
    g = run_gpu(sc, alpha_model=rgs.RGS_ALPHA_DISC, pairs=True)
    assert g["info"]["n_hits"] == m * (m - 1)
    kappa = sc["ad"][0, 0] * (m - 1) * sc["s"][0, 0] ** 2 / 4.0
    expect = sc["E"][0, 0, 0] * sum(kappa ** q for q in range(nb + 1))
    np.testing.assert_allclose(g["B"][:, 0, :], expect, rtol=1e-5)
    assert np.abs(g["B"][:, 1:, :]).max() <= 1e-5 * expect


def test_pairs_transport_is_not_batched():
    sc = scenes.box_scene(n=300, nb=2)
    d = api.upload(sc)
    p = api.Pipeline(pairs=True)
    p.build(d)
    p.trace(d)
    with pytest.raises(rgs.RgsError):
        rgs.rgs_solve_batched([p.transport], [None], [2])
    # a hemisphere transport is not a center-to-center one
    q = api.Pipeline()
    q.build(d)
    q.trace(d)
    q.solve(None, 2)
    with pytest.raises(rgs.RgsError):
        rgs.rgs_adjoint_pairs(q.transport, torch.zeros((sc["n"], 9, 3), device="cuda"))
