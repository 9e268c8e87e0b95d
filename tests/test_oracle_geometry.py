"""Pins of the oracle's geometry gradients (Eqs. dl-dgeo-0 and dl-dgeo-1) for both
transports: the SH gradient against tangent differences of the SH
(which is itself pinned to scipy), the lone plane's direct term against its closed form,
and the full dL/dp, dL/ds, dL/dtu, dL/dtv against central differences of the whole forward
solve for the Gaussian and GFSGS opacity models, point and directional lights (no GPU)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_18497_gb300 import scenes


@pytest.mark.parametrize("L", [1, 2, 3])
def test_sh_gradient_matches_tangent_differences(L):
    rng = np.random.default_rng(L)
    for _ in range(8):
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        t = np.cross(w, rng.normal(size=3))
        t /= np.linalg.norm(t)
        Y, dY = O.sh_grad(L, w)
        np.testing.assert_allclose(Y, O.sh_eval(L, w), rtol=1e-14, atol=1e-15)

        def Yat(a):
            x = w + a * t
            return O.sh_eval(L, x / np.linalg.norm(x))
        h = 1e-4
        num = (4 * (Yat(h / 2) - Yat(-h / 2)) / h - (Yat(h) - Yat(-h)) / (2 * h)) / 3
        np.testing.assert_allclose(dY.T @ t, num, atol=1e-10)
    # band 1 is linear: Y_1-1 = -c y, Y_10 = c z, Y_11 = -c x (Condon-Shortley phase)
    c = math.sqrt(3.0 / (4.0 * math.pi))
    _, dY = O.sh_grad(1, np.array([0.3, -0.5, math.sqrt(1 - 0.34)]))
    np.testing.assert_allclose(dY[:, 1], [0, -c, 0], atol=1e-15)
    np.testing.assert_allclose(dY[:, 2], [0, 0, c], atol=1e-15)
    np.testing.assert_allclose(dY[:, 3], [-c, 0, 0], atol=1e-15)


def test_lone_plane_position_gradient_closed_form():
    """B_00 = 2 sqrt(pi) (o k a^d / pi) I n.l / |l|^3 with l = p_L - p, so
    dB_00/dp = 2 sqrt(pi) (o k a^d / pi) I (-n / |l|^3 + 3 (n.l) l / |l|^5)."""
    sc = scenes.lone_plane(L=2, o=0.8, ad=(0.5, 0.3, 0.2), k=1.0)
    orc = O.Oracle(sc).pairs()
    W = np.zeros((1, orc.nc, orc.C))
    W[0, 0, 1] = 1.0  # L = B_00 of the green channel
    gg = orc.geometry_grad(W, nb=2)
    lp, I = sc["light_pos"][0], sc["light_I"][0][1]
    l = lp - sc["p"][0]
    r = np.linalg.norm(l)
    n = np.array([0.0, 0.0, 1.0])
    pre = 2 * math.sqrt(math.pi) * sc["o"][0] * sc["ad"][0][1] / math.pi * I
    expect = pre * (-n / r ** 3 + 3 * (n @ l) * l / r ** 5)
    np.testing.assert_allclose(gg["dp"][0], expect, rtol=1e-12)
    np.testing.assert_allclose(gg["ds"][0], 0.0, atol=1e-15)  # nothing depends on the scale
    # the normal: dB_00/dn = pre l / |l|^3 with n = t^u x t^v, t^u = e_x, t^v = e_y, so
    # dL/dtu = (I - e_x e_x^T)(e_y x Gn) and dL/dtv = (I - e_x e_x^T)(I - e_y e_y^T)(Gn x e_x)
    Gn = pre * l / r ** 3
    ex, ey = np.eye(3)[0], np.eye(3)[1]
    Px, Py = np.eye(3) - np.outer(ex, ex), np.eye(3) - np.outer(ey, ey)
    np.testing.assert_allclose(gg["dtu"][0], Px @ np.cross(ey, Gn), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(gg["dtv"][0], Px @ Py @ np.cross(Gn, ex), rtol=1e-12, atol=1e-15)


def _fd_check(sc, alpha_model=O.ALPHA_GAUSS, directional=False, stride=3, keys=(("p", 3), ("s", 2))):
    def make(s2):
        o2 = O.Oracle(s2, alpha_model=alpha_model)
        if directional:
            O.lib().or_set_directional(o2.h, 1)
        return o2.pairs()
    orc = make(sc)
    W = np.random.default_rng(9).normal(size=(sc["n"], orc.nc, orc.C))
    gg = orc.geometry_grad(W, E=sc["E"], nb=sc["nb"])

    def loss(s2):
        return float(np.sum(W * make(s2).solve(E=s2["E"], nb=s2["nb"])))

    def fd(key, idx, h=1e-5):
        def at(hh):
            s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
            s2[key][idx] += hh
            return loss(s2)
        def cd(hh):
            return (at(hh) - at(-hh)) / (2 * hh)
        return (4 * cd(h / 2) - cd(h)) / 3

    # central differences of a loss of size |L0| carry a rounding error of about
    # |L0| eps / h = 1e-11 |L0|; the truncation error of the extrapolated form is far below
    floor = 1e-9 * abs(loss(sc))
    for key, m in keys:
        an = gg["d" + key]
        scale = np.abs(an).max()
        assert scale > 0
        for i in range(0, sc["n"], stride):
            for a in range(m):
                num = fd(key, (i, a))
                assert abs(num - an[i, a]) <= 1e-7 * scale + floor, (key, i, a, num, an[i, a])


def test_geometry_gradients_match_finite_differences():
    sc = scenes.with_emission(scenes.random_cluster(n=40, seed=7, L=2, nb=3, n_lights=2), seed=5)
    _fd_check(sc)


def test_geometry_gradients_gfsgs_and_directional():
    sc = scenes.with_emission(scenes.random_cluster(n=30, seed=3, L=2, nb=3, n_lights=2), seed=5)
    _fd_check(sc, alpha_model=O.ALPHA_GFSGS, stride=4)
    _fd_check(sc, directional=True, stride=4)


def test_frame_gradients_match_finite_differences():
    """dL/dtu and dL/dtv of unnormalised, non-orthogonal frame inputs (carried through
    the Gram-Schmidt construction of Eq. G) against central differences."""
    sc = scenes.with_emission(scenes.random_cluster(n=30, seed=3, L=2, nb=3, n_lights=2), seed=5)
    rng = np.random.default_rng(1)
    sc["tu"] = sc["tu"] * rng.uniform(0.5, 2.0, (sc["n"], 1)) + 0.2 * sc["tv"]
    sc["tv"] = sc["tv"] * rng.uniform(0.5, 2.0, (sc["n"], 1))
    frames = (("tu", 3), ("tv", 3))
    _fd_check(sc, keys=frames)
    _fd_check(sc, alpha_model=O.ALPHA_GFSGS, stride=4, keys=frames)
    _fd_check(sc, directional=True, stride=4, keys=frames)


def _fd_check_hemi(sc, alpha_model=O.ALPHA_GAUSS, stride=3):
    """As _fd_check for the hemisphere-ray transport (smaller steps: the rays move with
    p and the frames, so their hit points do too)."""
    def make(s2):
        return O.Oracle(s2, alpha_model=alpha_model).transport()
    orc = make(sc)
    W = np.random.default_rng(9).normal(size=(sc["n"], orc.nc, orc.C))
    gg = orc.geometry_grad(W, E=sc["E"], nb=sc["nb"])

    def loss(s2):
        return float(np.sum(W * make(s2).solve(E=s2["E"], nb=s2["nb"])))

    def fd(key, idx, h=1e-6):
        def at(hh):
            s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
            s2[key][idx] += hh
            return loss(s2)
        def cd(hh):
            return (at(hh) - at(-hh)) / (2 * hh)
        return (4 * cd(h / 2) - cd(h)) / 3

    floor = 1e-8 * abs(loss(sc))  # rounding of the differences at h = 1e-6
    for key, m in (("p", 3), ("s", 2), ("tu", 3), ("tv", 3)):
        an = gg["d" + key]
        scale = np.abs(an).max()
        assert scale > 0
        for i in range(0, sc["n"], stride):
            for a in range(m):
                num = fd(key, (i, a))
                assert abs(num - an[i, a]) <= 1e-6 * scale + floor, (key, i, a, num, an[i, a])


def test_hemisphere_geometry_gradients_match_finite_differences():
    """The hemisphere-ray transport: every hit point moves with the receiver's centre and
    frame (the rays leave p_i along fixed local directions) and with the source's plane,
    frame and scales; the directional effects act per ray.  Skewed frame inputs."""
    sc = scenes.with_emission(scenes.random_cluster(n=30, seed=3, L=2, nd=16, nb=3, n_lights=2), seed=5)
    rng = np.random.default_rng(1)
    sc["tu"] = sc["tu"] * rng.uniform(0.5, 2.0, (sc["n"], 1)) + 0.2 * sc["tv"]
    sc["tv"] = sc["tv"] * rng.uniform(0.5, 2.0, (sc["n"], 1))
    _fd_check_hemi(sc)
    _fd_check_hemi(scenes.with_emission(scenes.random_cluster(n=24, seed=4, L=2, nd=16, nb=2, n_lights=1), seed=6),
                   alpha_model=O.ALPHA_GFSGS, stride=4)


def test_geometry_gradients_need_a_transport():
    sc = scenes.lone_plane()
    with pytest.raises(RuntimeError):
        O.Oracle(sc).geometry_grad(np.zeros((1, 9, 3)), nb=1)
