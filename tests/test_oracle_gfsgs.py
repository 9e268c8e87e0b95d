"""Pins of the oracle's GFSGS opacity model (App. E: alpha = 1 - exp(-0.03279 (g G)^3.4))
and of its closed-form integral through the Ein function (no GPU)."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O
from paper_2509_18497_gb300 import scenes

from test_oracle_transport import make_scene


def _dot(a, b):
    return float(np.sum(a * b))


def test_ein_against_scipy():
    """Ein(x) = E1(x) + ln x + gamma for x > 0 (scipy's exponential integral), both sides of
    the oracle's switch between its series and its continued fraction."""
    for x in np.concatenate([np.logspace(-4, 0.3, 25), np.linspace(1.9, 2.1, 9), np.logspace(0.31, 2, 25)]):
        ref = special.exp1(x) + math.log(x) + np.euler_gamma
        assert abs(O.ein(x) - ref) <= 1e-13 * max(1.0, abs(ref)), x
    # small x: Ein(x) = x - x^2/4 + x^3/18 - ...
    x = 1e-3
    assert abs(O.ein(x) - (x - x * x / 4 + x ** 3 / 18)) <= x ** 4 / 96 * 1.01   # the next term


@pytest.mark.parametrize("g", [0.8, 2.0, 4.0])
def test_gfsgs_alpha_area_equals_quadrature(g):
    """int alpha_j dx over the tangent plane, alpha = 1 - exp(-0.03279 (g e^{-r^2/2})^3.4),
    in metric coordinates, against App. E's closed form (2 pi / 3.4) s^u s^v Ein(0.03279 g^3.4)."""
    su, sv = 0.06, 0.04
    sc = make_scene([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), s=(su, sv), o=g)])
    orc = O.Oracle(sc, alpha_model=O.ALPHA_GFSGS)

    def integrand(r):  # polar, in units of s
        return 2 * math.pi * r * (-math.expm1(-0.03279 * (g * math.exp(-0.5 * r * r)) ** 3.4))

    val, _ = integrate.quad(integrand, 0.0, 12.0, epsabs=1e-14, epsrel=1e-12, limit=200)
    val *= su * sv
    assert abs(orc.alpha_area(0) - val) <= 1e-9 * val


def test_gfsgs_occluder_on_the_direct_term():
    """A lone plane under a light with a GFSGS occluder crossing the shadow ray at local
    radius rho: the direct term falls by alpha = 1 - exp(-0.03279 (g e^{-rho^2/2})^3.4), and the
    receiver's own factor is alpha_i(p_i) = 1 - exp(-0.03279 g_i^3.4)."""
    g_i, g_k, dx, s_k = 3.0, 2.5, 0.02, 0.05
    recv = dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), o=g_i, ad=(0.5, 0.5, 0.5))
    occ = dict(p=(dx, 0, 1), tu=(1, 0, 0), tv=(0, 1, 0), s=(s_k, s_k), o=g_k)
    light = ((0, 0, 2), (10, 10, 10))
    D0 = O.Oracle(make_scene([recv], lights=[light]), alpha_model=O.ALPHA_GFSGS).transport().direct()
    D1 = O.Oracle(make_scene([recv, occ], lights=[light]), alpha_model=O.ALPHA_GFSGS).transport().direct()
    a_k = -math.expm1(-0.03279 * (g_k * math.exp(-0.5 * (dx / s_k) ** 2)) ** 3.4)
    np.testing.assert_allclose(D1[0], D0[0] * (1 - a_k), rtol=1e-13)
    a_i = -math.expm1(-0.03279 * g_i ** 3.4)
    expect = 2 * math.sqrt(math.pi) * (a_i * 0.5 / math.pi) * 10 / 4.0   # cos = 1, r = 2
    np.testing.assert_allclose(D0[0, 0, :], expect, rtol=1e-12)


@pytest.mark.parametrize("pairs", [False, True])
def test_gfsgs_gradients_match_finite_differences(pairs):
    """dL/do under the GFSGS model (hits, shadow rays, receiver factor; for the
    center-to-center transport the Ein source term and the occluders), dL/da^d, dL/dE."""
    sc = scenes.with_emission(scenes.random_cluster(n=40, seed=11, L=2, nb=3, n_lights=2), seed=2)
    sc["o"] = np.random.default_rng(5).uniform(1.0, 5.0, sc["n"])

    def make(s2):
        orc = O.Oracle(s2, alpha_model=O.ALPHA_GFSGS)
        return orc.pairs() if pairs else orc.transport()

    orc = make(sc)
    W = np.random.default_rng(9).normal(size=(sc["n"], orc.nc, orc.C))
    g = orc.adjoint(W, E=sc["E"], nb=sc["nb"])

    def fd(key, idx, h=1e-3):
        def at(hh):
            s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
            s2[key][idx] += hh
            return _dot(W, make(s2).solve(E=s2["E"], nb=s2["nb"]))
        cd = lambda hh: (at(hh) - at(-hh)) / (2 * hh)
        return (4 * cd(h / 2) - cd(h)) / 3

    sop, sad, sE = (np.abs(g[k]).max() for k in ("dop", "dad", "dE"))
    for i in range(sc["n"]):
        assert abs(fd("o", (i,)) - g["dop"][i]) <= 1e-6 * sop, i
    rng = np.random.default_rng(1)
    for _ in range(12):
        i, ch = rng.integers(sc["n"]), rng.integers(3)
        assert abs(fd("ad", (i, ch)) - g["dad"][i, ch]) <= 1e-6 * sad
        i, kk, ch = rng.integers(sc["n"]), rng.integers(9), rng.integers(3)
        assert abs(fd("E", (i, kk, ch)) - g["dE"][i, kk, ch]) <= 1e-6 * sE
