"""Pins of the oracle's transport, solve and gradients against closed forms, exact
special cases, brute force and finite differences (no GPU)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_18497_gb300 import scenes

from test_oracle_math import real_sh_scipy


def make_scene(surfels, L=2, nd=64, nb=1, seed=0, lights=(), E=None):
    """Scene from a list of dicts with keys p, tu, tv, s, o, ad, k, as_, shin."""
    keys = ("p", "tu", "tv", "s", "o", "ad", "k", "as_", "shin")
    defaults = dict(s=(0.05, 0.05), o=1.0, ad=(0.5, 0.5, 0.5), k=1.0, as_=(0.0, 0.0, 0.0), shin=1.0)
    sc = {k: np.array([np.asarray(sf.get(k, defaults.get(k)), float) for sf in surfels]) for k in keys}
    sc.update(n=len(surfels), L=L, nd=nd, nb=nb, seed=seed,
              light_pos=np.array([lp for lp, _ in lights], float).reshape(-1, 3),
              light_I=np.array([li for _, li in lights], float).reshape(-1, 3),
              E=None if E is None else np.asarray(E, float))
    return sc


def _dot(a, b):
    return float(np.sum(a * b))


# ------------------------------------------------------------------------ direct term
def test_lone_plane_diffuse_closed_form():
    sc = scenes.lone_plane(L=2, o=0.8, ad=(0.5, 0.3, 0.2), k=1.0)
    orc = O.Oracle(sc).transport()
    D = orc.direct()
    lp, I = sc["light_pos"][0], sc["light_I"][0]
    r = np.linalg.norm(lp)
    cos = lp[2] / r
    expect = 2 * math.sqrt(math.pi) * (sc["o"][0] * sc["ad"][0] / math.pi) * I * cos / r ** 2
    np.testing.assert_allclose(D[0, 0, :], expect, rtol=1e-12)
    np.testing.assert_allclose(D[0, 1:, :], 0.0, atol=1e-15)   # a diffuse lobe has no l>0 bands


@pytest.mark.parametrize("L", [2, 3])
def test_lone_plane_specular_equals_projected_brdf(L):
    """D_lm = o * <f(w_I, .), Y_lm> * I cos / r^2 with f the diffuse + clamped Phong BRDF
    (Eq. brdf), projected by quadrature in a frame aligned with the lobe axis and an
    independent SH implementation."""
    k, ad, as_, s, o = 0.35, np.array([0.4, 0.5, 0.6]), np.array([0.5, 0.4, 0.3]), 2.0, 0.9
    sc = scenes.lone_plane(L=L, o=o, ad=ad, k=k, as_=as_, shin=s, light_pos=(0.4, -0.7, 1.1))
    k, ad, as_, s, o = sc["k"][0], sc["ad"][0], sc["as_"][0], sc["shin"][0], sc["o"][0]
    orc = O.Oracle(sc).transport()
    D = orc.direct()
    lp, I = sc["light_pos"][0], sc["light_I"][0]
    r = np.linalg.norm(lp)
    d = lp / r                               # direction to the light
    nrm = np.array([0, 0, 1.0])
    axis = 2 * (nrm @ d) * nrm - d           # mirror direction: the lobe axis
    e1 = np.cross(axis, [1.0, 0, 0]); e1 /= np.linalg.norm(e1)
    e2 = np.cross(axis, e1)
    x, w = np.polynomial.legendre.leggauss(40)
    t = 0.5 * (x + 1)
    wt = 0.5 * w
    nphi = 64
    proj = np.zeros((L + 1) ** 2)
    for ti, wi in zip(t, wt):
        st = math.sqrt(1 - ti * ti)
        for q in range(nphi):
            ph = 2 * math.pi * (q + 0.5) / nphi
            om = ti * axis + st * (math.cos(ph) * e1 + math.sin(ph) * e2)
            proj += wi * (2 * math.pi / nphi) * (s + 1) / (2 * math.pi) * ti ** s * real_sh_scipy(L, om)
    cos = nrm @ d
    for ch in range(3):
        f_coef = (1 - k) * as_[ch] * proj
        f_coef[0] += k * ad[ch] / math.pi * 2 * math.sqrt(math.pi)
        np.testing.assert_allclose(D[0, :, ch], o * f_coef * I[ch] * cos / r ** 2, rtol=1e-9, atol=1e-12)


def test_direct_term_shadowed_by_occluder():
    """A Gaussian occluder on the light segment multiplies the direct term by 1 - alpha."""
    rec = dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), o=0.7)
    occ = dict(p=(0.1, 0.05, 1.0), tu=(0, 1, 0), tv=(1, 0, 0), s=(0.2, 0.3), o=0.6)
    lights = [((0.0, 0.0, 2.0), (5.0, 5.0, 5.0))]
    D_open = O.Oracle(make_scene([rec], lights=lights)).transport().direct()
    D_occ = O.Oracle(make_scene([rec, occ], lights=lights)).transport().direct()
    # the light ray hits the occluder plane z=1 at (0,0,1): local (u,v) = (-0.05/0.2, -0.1/0.3)
    u, v = (0.0 - 0.05) / 0.2, (0.0 - 0.1) / 0.3
    alpha = 0.6 * math.exp(-0.5 * (u * u + v * v))
    np.testing.assert_allclose(D_occ[0], D_open[0] * (1 - alpha), rtol=1e-12)


# ----------------------------------------------------------------- hemisphere transport
def _disc_pair(H, R, src_E, rec_kw=None, src_extra=None, nd=16384, L=2):
    rec = dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), s=(0.01, 0.01), o=0.8, ad=(0.2, 0.5, 0.9), k=1.0)
    rec.update(rec_kw or {})
    src = dict(p=(0, 0, H), tu=(0, 1, 0), tv=(1, 0, 0), s=(R, R), o=1.0, ad=(0, 0, 0), k=1.0)
    src.update(src_extra or {})
    nc = (L + 1) ** 2
    E = np.zeros((2, nc, 3))
    E[1] = src_E
    sc = make_scene([rec, src], L=L, nd=nd, nb=1, E=E)
    return sc, O.Oracle(sc, alpha_model=O.ALPHA_DISC).transport()


def test_disc_form_factor():
    """Receiver below a facing disc of uniform radiance: B_00 = o rho e F with the disc
    form factor F = R^2 / (H^2 + R^2), within the stratified sampling error."""
    H, R, e = 1.0, 0.6, 2.0
    Es = np.zeros((9, 3)); Es[0] = e
    sc, orc = _disc_pair(H, R, Es)
    B = orc.solve(E=sc["E"], nb=1)
    F = R * R / (H * H + R * R)
    np.testing.assert_allclose(B[0, 0, :], 0.8 * np.array([0.2, 0.5, 0.9]) * e * F, rtol=3e-3)
    np.testing.assert_allclose(B[0, 1:, :], 0.0, atol=1e-14)


def test_disc_directional_emission_sign():
    """Source emitting only Y_10 (radiance e c1 w_z): the receiver sees it along -d, so
    B_00 = o 4 rho Y00 e c1 (-int_cap cos^2 dw) (Sec. 3.1: B_i(t_i, -w))."""
    H, R, e = 1.0, 0.8, 1.5
    Es = np.zeros((9, 3)); Es[2] = e
    sc, orc = _disc_pair(H, R, Es)
    B = orc.solve(E=sc["E"], nb=1)
    c1 = math.sqrt(3 / (4 * math.pi))
    cm = H / math.sqrt(H * H + R * R)
    cap = 2 * math.pi * (1 - cm ** 3) / 3
    expect = 0.8 * 4 * np.array([0.2, 0.5, 0.9]) * (0.5 / math.sqrt(math.pi)) * e * c1 * (-cap)
    np.testing.assert_allclose(B[0, 0, :], expect, rtol=3e-3)


def test_specular_transport_matches_area_quadrature():
    """Tilted, off-axis emitting disc and a glossy receiver: every band of B^(1) equals
    o c_l int_disc Y_lm(R_i w) L |n_i.w| |n_j.w| / r^2 dA (area form of Eq.
    before-final-radiosity), computed here by polar quadrature over the disc."""
    L = 3
    nc = (L + 1) ** 2
    k, ad, as_, s, o = 0.4, np.array([0.6, 0.5, 0.4]), np.array([0.5, 0.45, 0.3]), 2.0, 0.9
    c = np.array([[4 * k * ad[ch] + (1 - k) * as_[ch] if l == 0 else (1 - k) * as_[ch] * O.phong_rho(l, s)
                   for ch in range(3)] for l in range(L + 1)])
    center = np.array([0.6, 0.2, 1.0])
    nj = -center / np.linalg.norm(center) + np.array([0.2, -0.1, 0.0])
    nj /= np.linalg.norm(nj)
    tu = np.cross(nj, [0, 1.0, 0]); tu /= np.linalg.norm(tu)
    tv = np.cross(nj, tu)                       # tu x tv = nj
    R, e = 0.35, 1.0
    Es = np.zeros((nc, 3)); Es[0] = e
    sc, orc = _disc_pair(0, R, Es, rec_kw=dict(o=o, ad=ad, k=k, as_=as_, shin=s),
                         src_extra=dict(p=center, tu=tu, tv=tv), nd=65536, L=L)
    B = orc.solve(E=sc["E"], nb=1)
    # area quadrature over the disc
    x, w = np.polynomial.legendre.leggauss(48)
    rho = 0.5 * R * (x + 1)
    wr = 0.5 * R * w
    npsi = 96
    acc = np.zeros(nc)
    nrm = np.array([0, 0, 1.0])
    Lrad = e * 0.5 / math.sqrt(math.pi)     # isotropic radiance of the DC emission
    for rr, wrr in zip(rho, wr):
        for q in range(npsi):
            ps = 2 * math.pi * (q + 0.5) / npsi
            X = center + rr * (math.cos(ps) * tu + math.sin(ps) * tv)
            dist = np.linalg.norm(X)
            om = X / dist
            ci = nrm @ om
            if ci <= 0:
                continue
            Rw = 2 * ci * nrm - om
            acc += wrr * rr * (2 * math.pi / npsi) * real_sh_scipy(L, Rw) * Lrad * ci * abs(nj @ om) / dist ** 2
    expect = np.array([[o * c[int(math.isqrt(kk)), ch] * acc[kk] for ch in range(3)] for kk in range(nc)])
    scale = np.abs(expect).max()
    np.testing.assert_allclose(B[0], expect, atol=4e-3 * scale)
    assert np.abs(expect[1:]).max() > 0.05 * scale   # the glossy bands are exercised


def test_compositing_order_and_weights():
    """Eq. L_I: hits are taken in depth order with a_h = alpha_h prod_{k<h}(1-alpha_k);
    near-equal depths are ordered by surfel index."""
    rec = dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0))
    far = dict(p=(0, 0, 2), tu=(0, 1, 0), tv=(1, 0, 0), s=(1, 1), o=0.5)
    near = dict(p=(0, 0, 1), tu=(0, 1, 0), tv=(1, 0, 0), s=(1, 1), o=0.3)
    orc = O.Oracle(make_scene([rec, far, near]))
    j, t, a, G = orc.trace_ray(0, [0, 0, 0], [0, 0, 1.0])
    assert list(j) == [2, 1] and np.allclose(t, [1, 2])
    np.testing.assert_allclose(a, [0.3, 0.5])
    # nearly coplanar pair (depths 1e-9 apart): ordered by index, not by depth
    twin_far = dict(p=(0, 0, 1 + 1e-9), tu=(0, 1, 0), tv=(1, 0, 0), s=(1, 1), o=0.4)
    orc = O.Oracle(make_scene([rec, twin_far, near]))
    j, t, a, G = orc.trace_ray(0, [0, 0, 0], [0, 0, 1.0])
    assert list(j) == [1, 2]
    # depths 1e-4 apart are no tie: depth order even though the nearer has the larger index
    gap_far = dict(p=(0, 0, 1 + 1e-4), tu=(0, 1, 0), tv=(1, 0, 0), s=(1, 1), o=0.4)
    j, *_ = O.Oracle(make_scene([rec, gap_far, near])).trace_ray(0, [0, 0, 0], [0, 0, 1.0])
    assert list(j) == [2, 1]
    # (nearly) coplanar with the ray origin: ignored (|n_j.(p_j - o)| <= eps_plane)
    for dz in (0.0, 1e-7):
        side = dict(p=(0.3, 0, dz), tu=(1, 0, 0), tv=(0, 1, 0), s=(1, 1), o=1.0)
        orc = O.Oracle(make_scene([rec, side, near]))
        assert orc.eps_plane > 1e-6
        j, *_ = orc.trace_ray(0, [0, 0, 0], [0.6, 0, 0.8])
        assert 1 not in list(j)
    # ... but a plane just above eps_plane is hit
    side = dict(p=(0.3, 0, 1e-4), tu=(1, 0, 0), tv=(0, 1, 0), s=(1, 1), o=1.0)
    j, *_ = O.Oracle(make_scene([rec, side, near])).trace_ray(0, [0, 0, 0], [0.6, 0, 0.8])
    assert 1 in list(j)


def test_furnace_exact():
    """Closed sphere, disc opacity model, o=1, pure diffuse rho, uniform emission e:
    B^(n)_00 = e sum_{m<=n} rho^m for every surfel, independent of Nd and seed."""
    rho, e = 0.6, 1.0
    for nd, seed, nb in ((64, 0, 3), (128, 5, 5)):
        sc = scenes.furnace_sphere(m=1500, rho=rho, emission=e, nd=nd, nb=nb, seed=seed)
        orc = O.Oracle(sc, alpha_model=O.ALPHA_DISC).transport()
        B = orc.solve(E=sc["E"], nb=nb)
        r32, e32 = sc["ad"][0, 0], sc["E"][0, 0, 0]      # the float32-rounded inputs
        expect = e32 * sum(r32 ** m for m in range(nb + 1))
        np.testing.assert_allclose(B[:, 0, :], expect, rtol=1e-12)
        np.testing.assert_allclose(B[:, 1:, :], 0.0, atol=1e-12)


def test_energy_bounds():
    sc = scenes.box_scene(n=1500, pure_diffuse=True)
    orc = O.Oracle(sc).transport()
    h = orc.hits()
    sums = np.add.reduceat(h["a"], h["off"][:-1][np.diff(h["off"]) > 0])
    assert sums.max() <= 1.0 + 1e-14 and h["a"].min() >= 0.0
    # DC row sums of the diffuse K are <= rho_i o_i
    ones = np.zeros((sc["n"], 9, 3)); ones[:, 0, :] = 1.0
    KB, _ = orc.apply_K(ones)
    rho = sc["ad"] * sc["k"][:, None]
    assert np.all(KB[:, 0, :] <= rho * sc["o"][:, None] + 1e-14)
    # E = 0, diffuse: B_00 >= 0 and non-decreasing with the number of bounces
    prev = None
    for nb in range(4):
        B = orc.solve(nb=nb)
        assert B[:, 0, :].min() >= 0.0
        if prev is not None:
            assert np.all(B[:, 0, :] >= prev - 1e-14)
        prev = B[:, 0, :]


def test_neumann_series_equals_dense_solve():
    sc = scenes.random_cluster(n=100, seed=2, L=2, nd=64, n_lights=2)
    sc = dict(sc, ad=sc["ad"] * 0.8)
    orc = O.Oracle(sc).transport()
    E = np.random.default_rng(1).uniform(0, 0.3, size=(sc["n"], 9, 3))
    B = orc.solve(E=E, nb=400)
    S = orc.solve(E=E, nb=0)
    for col in range(orc.C):
        K = orc.dense_K(col)
        assert np.max(np.abs(np.linalg.eigvals(K))) < 0.9
        x = np.linalg.solve(np.eye(K.shape[0]) - K, S[:, :, col].reshape(-1))
        np.testing.assert_allclose(B[:, :, col].reshape(-1), x, rtol=1e-10, atol=1e-12 * np.abs(x).max())
        # the gather form and the assembled dense matrix are the same operator
        KB, _ = orc.apply_K(S)
        np.testing.assert_allclose(KB[:, :, col].reshape(-1), K @ S[:, :, col].reshape(-1), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("maker", [lambda: scenes.box_scene(n=2000), lambda: scenes.random_cluster(n=150, n_lights=3)])
def test_adjoint_identity(maker):
    sc = maker()
    orc = O.Oracle(sc).transport()
    rng = np.random.default_rng(0)
    u = rng.normal(size=(sc["n"], orc.nc, orc.C))
    v = rng.normal(size=(sc["n"], orc.nc, orc.C))
    Kv, _ = orc.apply_K(v)
    KTu = orc.apply_KT(u)
    lhs, rhs = _dot(KTu, v), _dot(u, Kv)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), np.abs(KTu).sum() * np.abs(v).max())


def _loss(sc, W, alpha_model=O.ALPHA_GAUSS):
    orc = O.Oracle(sc, alpha_model=alpha_model).transport()
    return _dot(W, orc.solve(E=sc["E"], nb=sc["nb"]))


def test_gradients_match_finite_differences():
    """L = <W, B^(n)>: analytic dL/dE, dL/da^d, dL/do against Richardson-extrapolated
    central differences (h = 1e-3 and h/2) on 64 parameters of each kind."""
    sc = scenes.with_emission(scenes.random_cluster(n=60, seed=4, L=2, nd=64, nb=3, n_lights=2), seed=3)
    orc = O.Oracle(sc).transport()
    W = np.random.default_rng(9).normal(size=(sc["n"], orc.nc, orc.C))
    g = orc.adjoint(W, E=sc["E"], nb=sc["nb"])
    rng = np.random.default_rng(11)

    def fd(setter, h=1e-3):
        def cd(hh):
            return (_loss(setter(+hh), W) - _loss(setter(-hh), W)) / (2 * hh)
        return (4 * cd(h / 2) - cd(h)) / 3

    def perturb(key, idx, hh):
        s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
        s2[key][idx] += hh
        return s2

    checks = []
    for i in range(sc["n"]):
        checks.append(("o", (i,), g["dop"][i]))
    for _ in range(64):
        i, ch = rng.integers(sc["n"]), rng.integers(3)
        checks.append(("ad", (i, ch), g["dad"][i, ch]))
        i, kk, ch = rng.integers(sc["n"]), rng.integers(9), rng.integers(3)
        checks.append(("E", (i, kk, ch), g["dE"][i, kk, ch]))
    scale = {key: max(abs(v) for k2, _, v in checks if k2 == key) for key in ("o", "ad", "E")}
    worst = 0.0
    for key, idx, an in checks:
        num = fd(lambda hh: perturb(key, idx, hh))
        worst = max(worst, abs(num - an) / scale[key])
        assert abs(num - an) <= 1e-6 * scale[key], (key, idx, num, an)
    assert worst < 1e-6


def test_closed_form_brdf_gradient_is_the_converged_limit():
    """Eq. final-dl-dbrdf (dL/dc = dL/dE (B-E)/c) is exact only at convergence: the exact
    truncated-series gradient approaches it geometrically as the bounce count grows."""
    sc = scenes.with_emission(scenes.random_cluster(n=80, seed=6, L=2, nd=64, n_lights=1), seed=2)
    orc = O.Oracle(sc).transport()
    W = np.random.default_rng(1).normal(size=(sc["n"], orc.nc, orc.C))
    diffs = []
    for nb in (2, 4, 8, 16, 32):
        exact = orc.adjoint(W, E=sc["E"], nb=nb)["dc"]
        closed = orc.brdf_grad_closed_form(W, E=sc["E"], nb=nb)
        diffs.append(np.abs(exact - closed).max() / np.abs(closed).max())
    assert all(b < a for a, b in zip(diffs, diffs[1:]))
    assert diffs[-1] < 1e-6


@pytest.mark.parametrize("maker", [lambda: scenes.box_scene(n=2000), lambda: scenes.fruit_bowl(n=3000, nd=64)])
def test_bvh_equals_brute_force(maker):
    sc = maker()
    a = O.Oracle(sc, use_bvh=True).transport()
    b = O.Oracle(sc, use_bvh=False).transport()
    ha, hb = a.hits(), b.hits()
    assert np.array_equal(ha["off"], hb["off"]) and np.array_equal(ha["j"], hb["j"])
    for key in ("alpha", "a", "t"):
        assert np.array_equal(ha[key], hb[key])
    assert a.num_shadow_hits() == b.num_shadow_hits()
    np.testing.assert_array_equal(a.direct(), b.direct())
