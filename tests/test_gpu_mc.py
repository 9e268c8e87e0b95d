"""The GPU Monte-Carlo TD(0) solver (rgs_mc_solve / rgs_mc_estimate / rgs_mc_groups: Sec. 7,
Alg. 1, App. "Monte-Carlo Solver Details") against the FP64 oracle's or_mc_pick,
or_mc_solve and or_mc_groups on the same center-to-center transport and the same
SplitMix64 keys.

Both sides stream a receiver's pairs in increasing caller index of the source with the same
uniforms, so every draw makes the same pick unless the GPU's FP32 proxy weights move a keep
decision u_k W_k < w_k across its boundary (relative gaps of ~1e-6, which none of these
draws meets: the picks are compared exactly).  The probability of a pick (a ratio of FP32
weights) and the estimate delta = S_a + K_ab Bhat_b / p_b agree to 1e-5 (the FP32 bar of
the transport, 1e-4, with margin to spare).  The unbiasedness identity sum_b p_b delta_b =
S_a + (K Bhat)_a is checked on the GPU's own p and delta, and a short solve (12 steps: the
8 sweeps, then variance-driven receivers) reproduces the oracle's visits exactly and its
means to 1e-4."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_18497_gb300 import api, rgs, scenes

from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build
    build.build()


def _setup(n):
    sc = scenes.with_emission(scenes.random_cluster(n=n, seed=2, L=2, nb=3, n_lights=1), seed=4)
    orc = O.Oracle(sc).pairs()
    d = api.upload(sc)
    pipe = api.Pipeline(pairs=True)
    pipe.build(d)
    pipe.trace(d)
    return sc, orc, d, pipe


@pytest.fixture(scope="module")
def cluster():
    """48 surfels: the draws (the dense interreflection of this cloud makes K's spectral
    radius exceed 1, so its Neumann series and any solver of it diverge)."""
    return _setup(48)


@pytest.fixture(scope="module")
def small():
    """24 surfels (the oracle's own Monte-Carlo pins): a convergent transport for the solvers."""
    return _setup(24)


def _estimates(pipe, d, Bhat, seed, step, groups=0, recv=None):
    Bt = torch.as_tensor(np.ascontiguousarray(Bhat, np.float32), device="cuda")
    rt = None if recv is None else torch.as_tensor(np.asarray(recv, np.int32), device="cuda")
    pick, p, delta = rgs.rgs_mc_estimate(pipe.transport, Bt, seed, step, recv=rt, E=d["E"], groups=groups)
    return pick.cpu().numpy(), p.cpu().numpy(), delta.double().cpu().numpy()


@pytest.mark.parametrize("groups", [0, 3, 6])
@pytest.mark.parametrize("zero_means", [True, False])
def test_estimates_match_the_oracle_draws(cluster, groups, zero_means):
    """Every receiver's draw at step 3 (and step 1 with all means zero: the geometric
    proposal with the floor alone), flat and through K-means groups."""
    sc, orc, d, pipe = cluster
    Bhat = np.zeros(orc._shape()) if zero_means else np.random.default_rng(1).normal(size=orc._shape())
    Bhat = Bhat.astype(np.float32).astype(np.float64)
    step = 1 if zero_means else 3
    pick, p, delta = _estimates(pipe, d, Bhat, 17, step, groups)
    with_pick = 0
    for a in range(sc["n"]):
        k, pk, dk = orc.mc_pick(Bhat, 17, step, a, a, E=sc["E"], groups=groups)
        assert pick[a] == k, (a, pick[a], k)
        if k < 0:
            assert p[a] == 0.0
        else:
            with_pick += 1
            assert p[a] == pytest.approx(pk, rel=1e-5)
        assert np.linalg.norm(delta[a] - dk) <= 1e-5 * max(np.linalg.norm(dk), 1e-30), a
    assert with_pick >= sc["n"] // 2


def test_kmeans_groups_match_the_oracle(cluster):
    sc, orc, d, pipe = cluster
    for G in (3, 6, 11):
        got = rgs.rgs_mc_groups(pipe.transport, G).cpu().numpy()
        np.testing.assert_array_equal(got, orc.mc_groups(G))


@pytest.mark.parametrize("groups", [0, 4])
def test_gpu_estimates_are_unbiased(cluster, groups):
    """For a receiver, every pair the GPU picks over many draws, with the GPU's own p and
    delta: sum p = 1 over the receiver's pairs and sum p delta = S_a + (K Bhat)_a (Eq.
    one-point-estimator), against the oracle's bounce."""
    sc, orc, d, pipe = cluster
    Bhat = np.random.default_rng(2).normal(size=orc._shape()).astype(np.float32).astype(np.float64)
    off = orc.pair_list()["off"]
    S = orc.solve(E=sc["E"], nb=0)
    KB = orc.apply_K(Bhat)[0]
    receivers = [a for a in range(sc["n"]) if off[a + 1] - off[a] >= 3][:3]
    assert receivers
    for a in receivers:
        n_pairs = int(off[a + 1] - off[a])
        pick, p, delta = _estimates(pipe, d, Bhat, 23, 5, groups, recv=[a] * 400000)
        seen = {}
        for k, pk, dk in zip(pick, p, delta):
            seen.setdefault(int(k), (pk, dk))
        assert sorted(seen) == list(range(n_pairs))
        assert sum(pk for pk, _ in seen.values()) == pytest.approx(1.0, rel=1e-5)
        expect = sum(pk * dk for pk, dk in seen.values())
        ref = S[a] + KB[a]
        assert np.linalg.norm(expect - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("groups", [0, 3])
def test_short_solve_reproduces_the_oracle(small, groups):
    """12 steps: the first 8 visit every receiver, the last 4 draw receivers by tracked
    variance.  Same draws, so the same visit counts and the means to the FP32 bar."""
    sc, orc, d, pipe = small
    B, V = rgs.rgs_mc_solve(pipe.transport, 12, seed=9, E=d["E"], groups=groups)
    Bo, Vo = orc.mc_solve(12, seed=9, E=sc["E"], groups=groups)
    np.testing.assert_array_equal(V.cpu().numpy(), Vo)
    assert V.sum().item() == 12 * sc["n"]
    assert rel_l2(B.double().cpu().numpy(), Bo) <= TOL


def test_solver_converges_and_hybrid_source(small):
    """Convergence statistics: the GPU solver's error against the Neumann solution falls
    with the step count like the oracle's (the same estimator), and a given source term
    S_in replaces E + D (the hybrid solver's remaining problem: shoot with the oracle, then
    run the GPU solver on the unshot radiance)."""
    sc, orc, d, pipe = small
    ref = orc.solve(E=sc["E"], nb=300)
    err = {}
    for T in (64, 2048):
        B, _ = rgs.rgs_mc_solve(pipe.transport, T, seed=3, E=d["E"])
        err[T] = rel_l2(B.double().cpu().numpy(), ref)
    Bo, _ = orc.mc_solve(2048, seed=3, E=sc["E"])
    eo = rel_l2(Bo, ref)
    assert err[2048] < err[64] / 3 and err[2048] < 2.0 * eo + 1e-4
    Bh, dB = orc.prog_refine(24, E=sc["E"])
    dBt = torch.as_tensor(np.ascontiguousarray(dB, np.float32), device="cuda")
    Br, _ = rgs.rgs_mc_solve(pipe.transport, 1024, seed=1, S=dBt)
    hybrid = Bh + Br.double().cpu().numpy() - dB
    pure, _ = rgs.rgs_mc_solve(pipe.transport, 1024, seed=1, E=d["E"])
    assert rel_l2(hybrid, ref) < rel_l2(pure.double().cpu().numpy(), ref) / 5


@pytest.mark.parametrize("shots", [0, 1, 5, 24, 400])
def test_progressive_refinement_matches_the_oracle(small, shots):
    """The same surfel shot at every step (the brightest unshot radiance), so Bhat and the
    unshot dB agree with the oracle's to the FP32 bar."""
    sc, orc, d, pipe = small
    Bh, dB = rgs.rgs_prog_refine(pipe.transport, shots, E=d["E"])
    Bho, dBo = orc.prog_refine(shots, E=sc["E"])
    assert rel_l2(Bh.double().cpu().numpy(), Bho) <= TOL
    assert rel_l2(dB.double().cpu().numpy(), dBo) <= TOL if np.linalg.norm(dBo) > 0 else float(dB.abs().max()) == 0.0
    np.testing.assert_array_equal(dB.cpu().numpy() == 0.0, dBo == 0.0)  # the same surfels shot


def test_gpu_hybrid_solver(small):
    """Shooting, then Alg. 1 on the remaining problem, all on the GPU: far less noise than
    Alg. 1 alone for the same steps (Sec. 7)."""
    sc, orc, d, pipe = small
    ref = orc.solve(E=sc["E"], nb=300)
    Bh, dB = rgs.rgs_prog_refine(pipe.transport, 24, E=d["E"])
    Br, _ = rgs.rgs_mc_solve(pipe.transport, 1024, seed=2, S=dB)
    hybrid = (Bh + Br - dB).double().cpu().numpy()
    pure, _ = rgs.rgs_mc_solve(pipe.transport, 1024, seed=2, E=d["E"])
    assert rel_l2(hybrid, ref) < rel_l2(pure.double().cpu().numpy(), ref) / 5


def test_mc_rejects_hemisphere_transports_and_bad_arguments(cluster):
    sc, orc, d, pipe = cluster
    hemi = api.Pipeline()
    hemi.build(d)
    hemi.trace(d)
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_mc_solve(hemi.transport, 4, E=d["E"])
    assert e.value.status == rgs.RGS_ERR_ARG
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_prog_refine(hemi.transport, 4, E=d["E"])
    assert e.value.status == rgs.RGS_ERR_ARG
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_mc_solve(pipe.transport, 4, E=d["E"], groups=2000)
    assert e.value.status == rgs.RGS_ERR_ARG
    Bt = torch.zeros((sc["n"], orc.nc, orc.C), device="cuda")
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_mc_estimate(pipe.transport, Bt, 1, 1, recv=torch.tensor([0, sc["n"]], dtype=torch.int32, device="cuda"),
                            E=d["E"])
    assert e.value.status == rgs.RGS_ERR_ARG
