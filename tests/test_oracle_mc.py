"""Pins of the oracle's Monte-Carlo solver (Sec. 7, Alg. 1; App. "Monte-Carlo Solver
Details") on the center-to-center transport: the one-point estimator is unbiased for the
deterministic bounce, weighted reservoir sampling draws from the proposal, the TD(0)
running mean follows its recursion, the variance-driven selection leaves deterministic
kernels alone, and the solver converges to the Neumann solution (no GPU)."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2509_18497_gb300 import scenes


@pytest.fixture(scope="module")
def cluster():
    sc = scenes.with_emission(scenes.random_cluster(n=24, seed=2, L=2, nb=3, n_lights=1), seed=4)
    return sc, O.Oracle(sc).pairs()


def test_estimator_is_unbiased_for_the_bounce(cluster):
    """sum over a receiver's pairs of p_b * (S_a + K_ab Bhat_b / p_b) = S_a + (K Bhat)_a
    exactly, for any means Bhat (Eq. one-point-estimator)."""
    sc, orc = cluster
    Bhat = np.random.default_rng(0).normal(size=orc._shape())
    S = orc.solve(E=sc["E"], nb=0)
    KB = orc.apply_K(Bhat)[0]
    off = orc.pair_list()["off"]
    with_pairs = [a for a in range(sc["n"]) if off[a + 1] > off[a]]
    for a in with_pairs[:4]:
        w, _ = orc.mc_weights(Bhat, a)
        assert len(w) == off[a + 1] - off[a] and np.all(w > 0)
        seen = {}
        for t in range(1, 20000):  # collect every pick's probability and estimate
            k, pk, delta = orc.mc_pick(Bhat, 7, t, 0, a, E=sc["E"])
            seen.setdefault(k, (pk, delta))
            if len(seen) == len(w):
                break
        assert len(seen) == len(w)
        for k, (pk, _) in seen.items():
            assert pk == pytest.approx(w[k] / w.sum(), rel=1e-12)
        expect = sum(pk * delta for pk, delta in seen.values())
        ref = S[a] + KB[a]
        assert np.linalg.norm(expect - ref) <= 1e-12 * np.linalg.norm(ref)
    lonely = [a for a in range(sc["n"]) if off[a + 1] == off[a]]
    for a in lonely[:2]:  # no source: no pick, and the estimate is S_a itself
        k, pk, delta = orc.mc_pick(Bhat, 7, 1, 0, a, E=sc["E"])
        assert k == -1 and pk == 0.0
        np.testing.assert_allclose(delta, S[a], rtol=1e-15)


@pytest.mark.parametrize("groups", [3, 6])
def test_grouped_proposal_is_unbiased(cluster, groups):
    """Through K-means groups (App. "Monte-Carlo Solver Details"): p_b = p(group) p(b | group)
    sums to 1 over the receiver's pairs and sum p_b delta_b = S_a + (K Bhat)_a exactly."""
    sc, orc = cluster
    assign = orc.mc_groups(groups)
    assert set(assign) == set(range(groups))  # no empty group on this scene
    Bhat = np.random.default_rng(2).normal(size=orc._shape())
    S = orc.solve(E=sc["E"], nb=0)
    KB = orc.apply_K(Bhat)[0]
    off = orc.pair_list()["off"]
    for a in [a for a in range(sc["n"]) if off[a + 1] - off[a] >= 3][:3]:
        n_pairs = off[a + 1] - off[a]
        seen = {}
        for t in range(1, 40000):
            k, pk, delta = orc.mc_pick(Bhat, 5, t, 1, a, E=sc["E"], groups=groups)
            seen.setdefault(k, (pk, delta))
            if len(seen) == n_pairs:
                break
        assert len(seen) == n_pairs
        assert sum(pk for pk, _ in seen.values()) == pytest.approx(1.0, rel=1e-12)
        expect = sum(pk * delta for pk, delta in seen.values())
        ref = S[a] + KB[a]
        assert np.linalg.norm(expect - ref) <= 1e-12 * np.linalg.norm(ref)


def test_reservoir_sampling_draws_from_the_proposal(cluster):
    sc, orc = cluster
    Bhat = np.random.default_rng(1).normal(size=orc._shape())
    a = 5
    w, _ = orc.mc_weights(Bhat, a)
    p = w / w.sum()
    draws = 20000
    cnt = np.zeros(len(w))
    for t in range(draws):
        k, _, _ = orc.mc_pick(Bhat, 11, t, 3, a)
        cnt[k] += 1
    chi2 = ((cnt - draws * p) ** 2 / (draws * p)).sum()
    assert chi2 < stats.chi2.ppf(0.999, len(w) - 1)


def test_proposal_follows_emission_and_geometry(cluster):
    """w_b = geo_ab (lum(|Y(-d)^T Bhat_b|) + floor): with Bhat = 0 the proposal is the
    geometric term alone (floor 1e-9), and scaling one source's mean raises its weight."""
    sc, orc = cluster
    Z = np.zeros(orc._shape())
    w0, fl = orc.mc_weights(Z, 5)
    assert fl == pytest.approx(1e-9)
    pl = orc.pair_list()
    off = pl["off"]
    js = pl["j"][off[5]:off[6]]
    geo = w0 / fl
    assert np.all(geo > 0)
    B1 = Z.copy()
    B1[js[0], 0, :] = 1.0  # the DC band of one source
    w1, _ = orc.mc_weights(B1, 5)
    assert w1[0] > w0[0] * 1e6 and np.allclose(w1[1:] / w0[1:], w1[1] / w0[1])


def test_td0_running_mean_recursion():
    """Two facing surfels, each the other's only source (p = 1): the first 8 steps visit
    every kernel, so B^(t) = (1/t) sum_{s<=t} (S + K B^(s-1)) with B^(0) = 0."""
    sc = scenes.with_emission(scenes.random_cluster(n=2, seed=0, L=2, nb=1, n_lights=1), seed=1)
    sc["p"] = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.4]])
    sc["tu"] = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    sc["tv"] = np.array([[0.0, 1.0, 0.0], [0.0, -1.0, 0.0]])  # n = +z and -z: facing
    sc["light_pos"] = np.array([[0.3, 0.2, 0.2]])
    orc = O.Oracle(sc).pairs()
    assert list(orc.pair_list()["off"]) == [0, 1, 2]
    S = orc.solve(E=sc["E"], nb=0)
    mean, acc = np.zeros(orc._shape()), np.zeros(orc._shape())
    for t in range(1, 9):
        acc += S + orc.apply_K(mean)[0]
        mean = acc / t
        B, D = orc.mc_solve(t, seed=5, E=sc["E"])
        np.testing.assert_allclose(B, mean, rtol=1e-12, atol=1e-15)
        assert np.all(D == t)


def test_variance_selection_and_determinism(cluster):
    sc, orc = cluster
    B1, D1 = orc.mc_solve(256, seed=3, E=sc["E"])
    B2, D2 = orc.mc_solve(256, seed=3, E=sc["E"])
    np.testing.assert_array_equal(B1, B2)
    B3, _ = orc.mc_solve(256, seed=4, E=sc["E"])
    assert not np.array_equal(B1, B3)
    # kernels without sources estimate S exactly every time: zero variance, never drawn
    # again after the 8 sweeps; every step still makes N estimates
    off = orc.pair_list()["off"]
    lonely = np.diff(off) == 0
    assert np.all(D1[lonely] == 8)
    assert D1.sum() == 256 * sc["n"]
    S = orc.solve(E=sc["E"], nb=0)
    np.testing.assert_allclose(B1[lonely], S[lonely], rtol=1e-13)


def test_solver_converges_to_the_neumann_solution(cluster):
    sc, orc = cluster
    ref = orc.solve(E=sc["E"], nb=300)
    err = {}
    for T in (64, 4096):
        B, _ = orc.mc_solve(T, seed=3, E=sc["E"])
        err[T] = np.linalg.norm(B - ref) / np.linalg.norm(ref)
    assert err[4096] < 2e-3 and err[4096] < err[64] / 3


def test_grouped_solver_converges(cluster):
    """The grouped proposal is unbiased but, on this cloud of randomly oriented surfels,
    a poorer match to the integrand (a group's mean normal and centre stand for all its
    members), so it converges more slowly; the mean error over three seeds still falls
    with T."""
    sc, orc = cluster
    ref = orc.solve(E=sc["E"], nb=300)

    def mean_err(T):
        return np.mean([np.linalg.norm(orc.mc_solve(T, seed=sd, E=sc["E"], groups=4)[0] - ref) / np.linalg.norm(ref)
                        for sd in (3, 4, 5)])
    e64, e16k = mean_err(64), mean_err(16384)
    assert e16k < 3e-3 and e16k < e64 / 3


def test_mc_needs_pairs():
    sc = scenes.lone_plane()
    with pytest.raises(RuntimeError):
        O.Oracle(sc).transport().mc_solve(4)


def _neumann(orc, x, nb=400):
    out, cur = x.copy(), x.copy()
    for _ in range(nb):
        cur = orc.apply_K(cur)[0]
        out += cur
    return out


@pytest.mark.parametrize("shots", [0, 1, 5, 24])
def test_progressive_refinement_decomposition(cluster, shots):
    """After any number of shots, B = Bhat + B^r - dB with B^r = dB + K B^r (the remaining
    problem is again the full transport) equals the solution: Sec. 7's decomposition."""
    sc, orc = cluster
    ref = orc.solve(E=sc["E"], nb=400)
    Bh, dB = orc.prog_refine(shots, E=sc["E"])
    full = Bh + _neumann(orc, dB) - dB
    assert np.linalg.norm(full - ref) <= 1e-12 * np.linalg.norm(ref)


def test_progressive_refinement_shoots_the_brightest_and_converges(cluster):
    sc, orc = cluster
    S = orc.solve(E=sc["E"], nb=0)
    lum = np.array([0.2126, 0.7152, 0.0722])[np.arange(orc.C) % 3]
    first = int(np.argmax((np.abs(S) * lum).sum(axis=(1, 2))))
    Bh, dB = orc.prog_refine(1, E=sc["E"])
    assert np.all(dB[first] == 0.0)
    np.testing.assert_array_equal(Bh[first], S[first])  # nothing has reached it yet
    ref = orc.solve(E=sc["E"], nb=400)
    Bh, dB = orc.prog_refine(400, E=sc["E"])
    assert np.linalg.norm(Bh - ref) <= 1e-12 * np.linalg.norm(ref)


def test_hybrid_solver_lowers_the_variance(cluster):
    """Sec. 7's hybrid solver: shooting first and running Alg. 1 on the remaining problem
    (source = the unshot radiance) reaches the solution with far less noise than Alg. 1 on
    the whole problem for the same number of steps."""
    sc, orc = cluster
    ref = orc.solve(E=sc["E"], nb=300)

    def mean_err(shots):
        return np.mean([np.linalg.norm(orc.hybrid_solve(shots, 1024, seed=sd, E=sc["E"]) - ref) / np.linalg.norm(ref)
                        for sd in (1, 2, 3)])
    pure, hybrid = mean_err(0), mean_err(24)
    assert hybrid < 1e-4 and hybrid < pure / 5
    # with nothing left unshot the hybrid returns the shooting result itself
    Bh, dB = orc.prog_refine(400, E=sc["E"])
    np.testing.assert_allclose(orc.hybrid_solve(400, 16, E=sc["E"]), Bh, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n,G", [(24, 3), (24, 6), (300, 8), (300, 20)])
def test_kmeans_groups_equal_an_independent_lloyd(n, G):
    """The grouping of the next-event proposal (App. "Monte-Carlo Solver Details": K-means
    over the surfels) is Lloyd's algorithm on (centre, extent/2 * normal) features from
    evenly spaced seeds.  scikit-learn's Lloyd iteration from the same seeds, run to a
    fixed point, must give the same assignment."""
    cluster_mod = pytest.importorskip("sklearn.cluster")
    sc = scenes.random_cluster(n=n, seed=2, L=2, nb=3, n_lights=1)
    got = O.Oracle(sc).mc_groups(G)
    p = sc["p"].astype(float)
    nrm = np.cross(sc["tu"].astype(float), sc["tv"].astype(float))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    ext = max(float((p.max(axis=0) - p.min(axis=0)).max()), 1e-12)
    feats = np.hstack([p, 0.5 * ext * nrm])
    seeds = feats[[k * n // G for k in range(G)]]
    km = cluster_mod.KMeans(n_clusters=G, init=seeds, n_init=1, algorithm="lloyd", max_iter=50, tol=0.0).fit(feats)
    assert len(set(got)) == G
    np.testing.assert_array_equal(got, km.labels_)
