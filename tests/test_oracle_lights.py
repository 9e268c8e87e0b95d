"""Pins of the oracle's directional lights (Sec. 5.1: lights far away without the
inverse-square falloff; Sec. 9: a 16 x 32 environment map of such lights) against closed
forms, the far-point-light limit, quadrature sums and finite differences (no GPU)."""
import math

import numpy as np

from oracle import oracle as O
from paper_2509_18497_gb300 import scenes

from test_oracle_transport import make_scene


def _dot(a, b):
    return float(np.sum(a * b))


def _directional(sc, dirs, I):
    out = dict(sc)
    out["light_pos"] = np.asarray(dirs, float).reshape(-1, 3)
    out["light_I"] = np.asarray(I, float).reshape(-1, 3)
    out["light_dir"] = True
    return out


def test_lone_plane_directional_closed_form():
    """D_00 = 2 sqrt(pi) (o k a^d / pi) I cos for a diffuse surfel (no 1/r^2); the length of
    the given direction does not matter."""
    base = scenes.lone_plane(L=2, o=0.8, ad=(0.5, 0.3, 0.2), k=1.0)
    w = np.array([0.3, -0.2, 1.5])
    sc = _directional(base, [7.0 * w], [[10.0, 7.0, 4.0]])
    D = O.Oracle(sc).transport().direct()
    cos = w[2] / np.linalg.norm(w)
    expect = 2 * math.sqrt(math.pi) * (sc["o"][0] * sc["ad"][0] / math.pi) * np.array([10.0, 7.0, 4.0]) * cos
    np.testing.assert_allclose(D[0, 0, :], expect, rtol=1e-12)
    np.testing.assert_allclose(D[0, 1:, :], 0.0, atol=1e-15)


def test_directional_shadow_ray_reaches_any_distance():
    """A directional light's shadow ray runs to infinity whatever the length of the given
    direction: a Gaussian occluder 3 units above the receiver, crossed at (dx/s^u, 0) in its
    own frame, multiplies D by 1 - o exp(-(dx/s^u)^2 / 2) although the direction vector is
    only 0.1 long."""
    dx, su, o = 0.02, 0.05, 0.6
    w = np.array([0.0, 0.0, 0.1])
    base = make_scene([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), k=1.0, o=0.8),
                       dict(p=(dx, 0, 3.0), tu=(1, 0, 0), tv=(0, -1, 0), s=(su, 0.05), o=o)])
    lit = _directional(base, [w], [[2.0, 3.0, 4.0]])
    D = O.Oracle(lit).transport().direct()
    free = _directional(make_scene([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), k=1.0, o=0.8)]), [w],
                        [[2.0, 3.0, 4.0]])
    D0 = O.Oracle(free).transport().direct()
    T = 1.0 - o * math.exp(-0.5 * (dx / su) ** 2)
    np.testing.assert_allclose(D[0], D0[0] * T, rtol=1e-12, atol=1e-15)


def test_far_point_light_limit():
    """A point light at distance R along w with intensity I R^2 tends to the directional
    light of intensity I, with an O(size/R) error, in every band (glossy receivers)."""
    sc = scenes.random_cluster(n=40, seed=3, L=3, n_lights=1)
    w = np.array([0.2, 1.0, 0.4])
    w /= np.linalg.norm(w)
    I = np.array([[3.0, 2.0, 1.0]])
    Dd = O.Oracle(_directional(sc, [w], I)).transport().direct()
    errs = []
    for R in (1e3, 1e5):
        s2 = dict(sc)
        s2["light_pos"], s2["light_I"] = (R * w)[None, :], I * R * R
        Dp = O.Oracle(s2).transport().direct()
        errs.append(np.abs(Dp - Dd).max() / np.abs(Dd).max())
    assert errs[1] < 1e-4 and errs[1] < errs[0] / 50


def test_env_map_on_a_plane_with_an_occluder():
    """A diffuse surfel facing +y under a uniform-radiance 16 x 32 map: D_00 =
    o 4 a^d Y00^2 ... = (2 sqrt(pi) o a^d / pi) L sum_cells cos dOmega over the cells above
    the horizon, a midpoint-rule sum within O(dtheta^2) of pi.  An opaque disc (o = 1,
    disc model) of radius a at height h removes exactly the cells whose direction crosses
    it: cos(theta) > h / sqrt(h^2 + a^2)."""
    nt, npf = 16, 32
    th = (np.arange(nt) + 0.5) * math.pi / nt
    ph = (np.arange(npf) + 0.5) * 2 * math.pi / npf
    T, P = np.meshgrid(th, ph, indexing="ij")
    w = np.stack([np.sin(T) * np.cos(P), np.cos(T), np.sin(T) * np.sin(P)], -1).reshape(-1, 3)
    dom = (np.sin(T) * (math.pi / nt) * (2 * math.pi / npf)).reshape(-1)
    Lr = 0.7
    I = np.repeat((Lr * dom)[:, None], 3, axis=1)
    recv = dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 0, -1), o=0.9, ad=(0.4, 0.4, 0.4))
    sc = _directional(make_scene([recv]), w, I)
    D = O.Oracle(sc).transport().direct()
    up = w[:, 1] > 0
    quad = np.sum(w[up, 1] * dom[up])
    assert abs(quad - math.pi) < 0.01 * math.pi
    expect = 2 * math.sqrt(math.pi) * 0.9 * 0.4 / math.pi * Lr * quad
    np.testing.assert_allclose(D[0, 0, 0::3].sum(), expect, rtol=1e-12)   # one channel, summed over the lights
    h, a = 0.5, 0.4
    occ = dict(p=(0, h, 0), tu=(1, 0, 0), tv=(0, 0, 1), s=(a, a), o=1.0)
    sc2 = _directional(make_scene([recv, occ]), w, I)
    D2 = O.Oracle(sc2, alpha_model=O.ALPHA_DISC).transport().direct()
    blocked = up & (w[:, 1] > h / math.hypot(h, a))
    expect2 = 2 * math.sqrt(math.pi) * 0.9 * 0.4 / math.pi * Lr * np.sum(w[up & ~blocked, 1] * dom[up & ~blocked])
    assert blocked.sum() > 0
    np.testing.assert_allclose(D2[0, 0, 0::3].sum(), expect2, rtol=1e-12)


def test_gradients_with_directional_lights():
    """L = <W, B^(n)> under three directional lights: dL/do (through the shadow rays to
    infinity and the hemisphere compositing), dL/da^d and dL/dE against central differences."""
    sc = scenes.with_emission(scenes.random_cluster(n=50, seed=8, L=2, nb=3, n_lights=3), seed=6)
    dirs = np.random.default_rng(4).normal(size=(3, 3))
    sc = _directional(sc, dirs, [[2.0, 1.5, 1.0], [1.0, 1.0, 1.0], [0.5, 1.0, 2.0]])
    orc = O.Oracle(sc).transport()
    W = np.random.default_rng(9).normal(size=(sc["n"], orc.nc, orc.C))
    g = orc.adjoint(W, E=sc["E"], nb=sc["nb"])

    def loss(s2):
        return _dot(W, O.Oracle(s2).transport().solve(E=s2["E"], nb=s2["nb"]))

    def fd(key, idx, h=1e-3):
        def at(hh):
            s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
            s2[key][idx] += hh
            return loss(s2)
        cd = lambda hh: (at(hh) - at(-hh)) / (2 * hh)
        return (4 * cd(h / 2) - cd(h)) / 3

    rng = np.random.default_rng(2)
    scale = {"o": np.abs(g["dop"]).max(), "ad": np.abs(g["dad"]).max(), "E": np.abs(g["dE"]).max()}
    for i in range(sc["n"]):
        assert abs(fd("o", (i,)) - g["dop"][i]) <= 1e-6 * scale["o"]
    for _ in range(16):
        i, ch = rng.integers(sc["n"]), rng.integers(3)
        assert abs(fd("ad", (i, ch)) - g["dad"][i, ch]) <= 1e-6 * scale["ad"]
        i, kk, ch = rng.integers(sc["n"]), rng.integers(9), rng.integers(3)
        assert abs(fd("E", (i, kk, ch)) - g["dE"][i, kk, ch]) <= 1e-6 * scale["E"]


def test_wide_batches_split_by_light():
    """Columns of different lights never mix (Sec. 7's batching of lights as right-hand
    sides): 400 point lights (1,200 columns, more than a 1,024-column row) give, column for
    column, what 2-light subsets of them give on their own; and dL/dB nonzero on those
    columns only gives the subset's gradients."""
    sc = scenes.multi_light(n=40, nd=8, nb=2, n_lights=400)
    orc = O.Oracle(sc).transport()
    C = orc.C
    assert C == 1200
    rng = np.random.default_rng(21)
    B = orc.solve(E=None, nb=sc["nb"])
    for sel in ([0, 1], [398, 399]):
        sub = dict(sc)
        sub["light_pos"] = sc["light_pos"][sel]
        sub["light_I"] = sc["light_I"][sel]
        cols = [3 * k + ch for k in sel for ch in range(3)]
        o2 = O.Oracle(sub).transport()
        B2 = o2.solve(E=None, nb=sc["nb"])
        np.testing.assert_allclose(B[..., cols], B2, rtol=1e-12, atol=1e-300)
        W = np.zeros((sc["n"], 16, C))
        W[..., cols] = rng.normal(size=(sc["n"], 16, 6))
        g_full = orc.adjoint(W)
        g_sub = o2.adjoint(W[..., cols])
        for key in ("dE", "dad", "dop"):
            assert np.abs(g_sub[key]).max() > 0.0, key
            np.testing.assert_allclose(g_full[key], g_sub[key], rtol=1e-10, atol=1e-14 * np.abs(g_sub[key]).max())
