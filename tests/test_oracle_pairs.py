"""Pins of the oracle's center-to-center transport (Sec. 8, the approximated forward
rendering equation: one segment per pair of surfel centres) against closed forms,
quadrature, exact special cases, brute force and finite differences (no GPU)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2509_18497_gb300 import scenes

from test_oracle_transport import make_scene


def _dot(a, b):
    return float(np.sum(a * b))


@pytest.mark.parametrize("model", [O.ALPHA_GAUSS, O.ALPHA_DISC])
def test_alpha_area_equals_quadrature(model):
    """int_{P_j} alpha_j dx of App. E for this build's opacity models, by 2-D quadrature
    over the tangent plane in metric coordinates (x = s^u u t^u + s^v v t^v)."""
    sc = make_scene([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), s=(0.07, 0.03), o=0.8)])
    orc = O.Oracle(sc, alpha_model=model)
    su, sv, o = 0.07, 0.03, 0.8
    rmax = 3.0 if model == O.ALPHA_GAUSS else 1.0

    def alpha(y, x):  # metric coordinates x, y in the plane
        r2 = (x / su) ** 2 + (y / sv) ** 2
        if r2 > rmax * rmax:
            return 0.0
        return o * (math.exp(-0.5 * r2) if model == O.ALPHA_GAUSS else 1.0)

    val, err = integrate.dblquad(alpha, -rmax * su, rmax * su,
                                 lambda x: -sv * math.sqrt(max(0.0, rmax ** 2 - (x / su) ** 2)),
                                 lambda x: sv * math.sqrt(max(0.0, rmax ** 2 - (x / su) ** 2)),
                                 epsabs=1e-12, epsrel=1e-10)
    assert abs(orc.alpha_area(0) - val) <= 1e-8 * val


def test_furnace_closed_form():
    """Closed sphere of M inward surfels (disc model, o = 1), pure diffuse rho, uniform
    emission e, no lights.  Every chord stays inside the ball, so no surfel occludes it
    (T = 1), every other surfel is in front of every receiver, and cos_i = cos_j = r/(2R)
    make |n_i.w||n_j.w|/r^2 = 1/(4R^2).  With c_0 = 4 rho and Y00^2 = 1/(4 pi):
        (K B)_00 = rho/pi * sum_j V_ji * B_00 = kappa B_00,  kappa = rho (M-1) s^2 / (4 R^2),
    so B^(n)_00 = e sum_{m<=n} kappa^m exactly and the other coefficients stay 0."""
    for m, rho, nb in ((400, 0.05, 4), (900, 0.02, 6)):
        sc = scenes.furnace_sphere(m=m, rho=rho, emission=1.0, nb=nb)
        orc = O.Oracle(sc, alpha_model=O.ALPHA_DISC).pairs()
        pl = orc.pair_list()
        assert np.all(pl["T"] == 1.0) and len(pl["j"]) == m * (m - 1)
        r32, e32, s32 = sc["ad"][0, 0], sc["E"][0, 0, 0], sc["s"][0, 0]
        kappa = r32 * (m - 1) * s32 * s32 / 4.0
        B = orc.solve(E=sc["E"], nb=nb)
        expect = e32 * sum(kappa ** q for q in range(nb + 1))
        # the centres and frames are float32-rounded, so they sit on the sphere only to
        # ~6e-8 relative; the closed form holds to that rounding
        np.testing.assert_allclose(B[:, 0, :], expect, rtol=1e-6)
        np.testing.assert_allclose(B[:, 1:, :], 0.0, atol=1e-12)


def test_single_occluder_transmittance_and_weight():
    """Receiver at the origin facing +z, source 2 above facing down, one occluder at
    height 1 whose centre is offset by dx in its plane: the segment crosses the occluder
    plane at local radius dx / s^u, so T = 1 - o_k exp(-(dx/s^u)^2 / 2), and
    V = lambda_j A_j T cos_i cos_j / r^2 with cos = 1 and r = 2."""
    dx, su, ok, lam = 0.03, 0.05, 0.7, 1.7
    sc = make_scene([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0)),
                     dict(p=(0, 0, 2), tu=(0, 1, 0), tv=(1, 0, 0), s=(0.04, 0.06), o=0.9),
                     dict(p=(dx, 0, 1), tu=(1, 0, 0), tv=(0, 1, 0), s=(su, 0.05), o=ok)])
    orc = O.Oracle(sc).pairs(lam=np.array([1.0, lam, 1.0]))
    pl = orc.pair_list()
    i0 = slice(pl["off"][0], pl["off"][1])
    js = list(pl["j"][i0])
    assert js == [1, 2]  # both are in front of the receiver
    T = pl["T"][i0][0]
    assert abs(T - (1.0 - ok * math.exp(-0.5 * (dx / su) ** 2))) <= 1e-14
    A = 0.9 * 2 * math.pi * 0.04 * 0.06 * (1 - math.exp(-4.5))
    assert abs(pl["V"][i0][0] - lam * A * T / 4.0) <= 1e-14
    # nothing occludes the receiver -> occluder segment (the occluder faces +z: the
    # receiver at the origin is behind it, so the occluder has no pair towards it)
    i2 = slice(pl["off"][2], pl["off"][3])
    assert list(pl["j"][i2]) == [1]


def test_coplanar_neighbours_of_the_source_do_not_occlude():
    """A second surfel in the source's plane overlapping its centre: its plane is within
    eps_plane of the segment's far end, so it does not occlude the source."""
    sc = make_scene([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0)),
                     dict(p=(0.1, 0, 1), tu=(0, 1, 0), tv=(1, 0, 0), s=(0.2, 0.2)),
                     dict(p=(0.12, 0.01, 1), tu=(0, 1, 0), tv=(1, 0, 0), s=(0.2, 0.2))])
    orc = O.Oracle(sc).pairs()
    pl = orc.pair_list()
    assert np.all(pl["T"][pl["off"][0]:pl["off"][1]] == 1.0)
    # the same neighbour moved 0.4 eps_plane towards the receiver: the segment now crosses its
    # plane before reaching the source, and only the eps_plane rule keeps it from occluding
    # (while one moved 3 eps_plane towards the receiver does occlude)
    eps = O.Oracle(sc).eps_plane
    for shift, occludes in ((0.4, False), (3.0, True)):
        sc2 = make_scene([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0)),
                          dict(p=(0.1, 0, 1), tu=(0, 1, 0), tv=(1, 0, 0), s=(0.2, 0.2)),
                          dict(p=(0.12, 0.01, 1 - shift * eps), tu=(0, 1, 0), tv=(1, 0, 0), s=(0.2, 0.2))])
        pl = O.Oracle(sc2).pairs().pair_list()
        j = list(pl["j"][pl["off"][0]:pl["off"][1]])
        T = pl["T"][pl["off"][0] + j.index(1)]
        assert (T < 1.0) == occludes


def test_adjoint_identity_and_dense_solve():
    sc = scenes.random_cluster(n=90, seed=5, L=2, n_lights=2)
    sc = dict(sc, ad=sc["ad"] * 0.5)
    orc = O.Oracle(sc).pairs(lam=np.random.default_rng(3).uniform(0.5, 1.5, sc["n"]))
    rng = np.random.default_rng(0)
    u = rng.normal(size=(sc["n"], orc.nc, orc.C))
    v = rng.normal(size=(sc["n"], orc.nc, orc.C))
    Kv, _ = orc.apply_K(v)
    KTu = orc.apply_KT(u)
    assert abs(_dot(KTu, v) - _dot(u, Kv)) <= 1e-12 * np.abs(KTu).sum() * np.abs(v).max()
    E = rng.uniform(0, 0.3, size=(sc["n"], 9, 3))
    B = orc.solve(E=E, nb=300)
    S = orc.solve(E=E, nb=0)
    for col in range(orc.C):
        K = orc.dense_K(col)
        assert np.max(np.abs(np.linalg.eigvals(K))) < 0.9
        x = np.linalg.solve(np.eye(K.shape[0]) - K, S[:, :, col].reshape(-1))
        np.testing.assert_allclose(B[:, :, col].reshape(-1), x, rtol=1e-10, atol=1e-12 * np.abs(x).max())


def test_bvh_equals_brute_force():
    sc = scenes.box_scene(n=600)
    a = O.Oracle(sc, use_bvh=True).pairs().pair_list()
    b = O.Oracle(sc, use_bvh=False).pairs().pair_list()
    assert np.array_equal(a["off"], b["off"]) and np.array_equal(a["j"], b["j"])
    np.testing.assert_array_equal(a["T"], b["T"])


def test_gradients_match_finite_differences():
    """L = <W, B^(n)> of the center-to-center solve: analytic dL/dE, dL/da^d, dL/do and
    dL/dlambda against Richardson-extrapolated central differences."""
    sc = scenes.with_emission(scenes.random_cluster(n=50, seed=7, L=2, nb=3, n_lights=2), seed=5)
    lam = np.random.default_rng(2).uniform(0.5, 1.5, sc["n"])
    orc = O.Oracle(sc).pairs(lam=lam)
    W = np.random.default_rng(9).normal(size=(sc["n"], orc.nc, orc.C))
    g = orc.adjoint(W, E=sc["E"], nb=sc["nb"])

    def loss(s2, lam2):
        o2 = O.Oracle(s2).pairs(lam=lam2)
        return _dot(W, o2.solve(E=s2["E"], nb=s2["nb"]))

    def fd(f, h=1e-3):
        def cd(hh):
            return (f(+hh) - f(-hh)) / (2 * hh)
        return (4 * cd(h / 2) - cd(h)) / 3

    def perturb(key, idx, hh):
        s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
        s2[key][idx] += hh
        return s2

    rng = np.random.default_rng(1)
    checks = [("o", (i,), g["dop"][i]) for i in range(sc["n"])]
    checks += [("lam", (i,), g["dlam"][i]) for i in range(sc["n"])]
    for _ in range(32):
        i, ch = rng.integers(sc["n"]), rng.integers(3)
        checks.append(("ad", (i, ch), g["dad"][i, ch]))
        i, kk, ch = rng.integers(sc["n"]), rng.integers(9), rng.integers(3)
        checks.append(("E", (i, kk, ch), g["dE"][i, kk, ch]))
    scale = {key: max(abs(v) for k2, _, v in checks if k2 == key) for key in ("o", "lam", "ad", "E")}
    for key, idx, an in checks:
        if key == "lam":
            def f(hh, i=idx[0]):
                l2 = lam.copy()
                l2[i] += hh
                return loss(sc, l2)
        else:
            def f(hh, key=key, idx=idx):
                return loss(perturb(key, idx, hh), lam)
        num = fd(f)
        assert abs(num - an) <= 1e-6 * scale[key], (key, idx, num, an)


def test_center_to_center_is_the_small_surfel_limit_of_the_hemisphere_transport():
    """Sec. 8 replaces the area integral of Eq. before-final-radiosity by one segment
    between centres, an approximation for surfels small against their distance.  A glossy
    receiver and a tilted, off-axis Gaussian emitter of scale s at distance D: the two
    transports' B^(1) must differ by a term of second order in s/D (the 1/r^2 and cosine
    factors vary quadratically across the emitter), so (B_hemi / B_pairs - 1)(D/s)^2 stays
    the same constant at every distance.  A constant relative error in either transport (a
    lost factor of the alpha integral, a cosine, 1/pi) adds a term growing like (D/s)^2 and
    breaks that.  2^20 stratified rays keep the hemisphere estimate's own error below a
    tenth of the compared term."""
    s, L, nc = 0.08, 2, 9
    d = np.array([0.5, 0.2, 1.0]) / np.linalg.norm([0.5, 0.2, 1.0])
    nrm = -d + np.array([0.3, -0.1, 0.0])
    nrm /= np.linalg.norm(nrm)
    tu = np.cross(nrm, [0.0, 1.0, 0.0])
    tu /= np.linalg.norm(tu)
    tv = np.cross(nrm, tu)
    E = np.zeros((2, nc, 3))
    E[1, 0], E[1, 2], E[1, 3] = (1.0, 2.0, 3.0), (0.4, 0.1, -0.2), (0.2, -0.3, 0.1)
    c00, chigh = [], []
    for D in (0.5, 0.7, 1.0, 1.4):
        sc = make_scene([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), k=0.6, as_=(0.3, 0.3, 0.3), shin=3.0),
                         dict(p=D * d, tu=tu, tv=tv, s=(s, 0.6 * s), o=0.9)], L=L, nd=1 << 20, E=E)
        Bh = O.Oracle(sc).transport().solve(E=sc["E"], nb=1)[0]
        Bp = O.Oracle(sc).pairs().solve(E=sc["E"], nb=1)[0]
        k = (D / s) ** 2
        c00.append((Bh[0] / Bp[0] - 1.0) * k)
        q = np.argmax(np.abs(Bp[1:]))
        chigh.append((Bh[1:] - Bp[1:]).ravel()[q] / np.abs(Bp[1:]).ravel()[q] * k)
    c00, chigh = np.array(c00), np.array(chigh)
    assert np.all(np.abs(c00) < 4.0) and np.all(np.abs(chigh) < 4.0)
    np.testing.assert_allclose(c00, np.broadcast_to(c00.mean(axis=0), c00.shape), rtol=0.15)
    np.testing.assert_allclose(chigh, chigh.mean(), rtol=0.15)
