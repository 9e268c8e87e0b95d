"""Pins of the oracle's building blocks against things fixed outside it: quadrature,
an independent SH library (scipy), closed forms and published generator outputs."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def real_sh_scipy(L, d):
    """Real SH with the Condon-Shortley phase from scipy's complex SH (independent
    implementation): Y_lm = sqrt2 Re Y_l^m (m>0), sqrt2 Im Y_l^|m| (m<0), Y_l^0 (m=0)."""
    d = np.asarray(d, float)
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    out = np.zeros((L + 1) ** 2)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            y = special.sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                v = math.sqrt(2.0) * y.real
            elif m < 0:
                v = math.sqrt(2.0) * y.imag
            else:
                v = y.real
            out[l * l + l + m] = v
    return out


def sphere_quadrature(nt=64, nphi=128):
    """Gauss-Legendre in cos(theta) x uniform in phi: exact for band-limited products."""
    x, w = np.polynomial.legendre.leggauss(nt)
    phis = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    dirs, wts = [], []
    for ct, wt in zip(x, w):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            dirs.append((st * math.cos(ph), st * math.sin(ph), ct))
            wts.append(wt * 2 * math.pi / nphi)
    return np.array(dirs), np.array(wts)


def test_sh_matches_independent_library():
    rng = np.random.default_rng(3)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        np.testing.assert_allclose(O.sh_eval(5, d), real_sh_scipy(5, d), atol=1e-13, rtol=1e-12)


def test_sh_ordering_and_low_order_closed_forms():
    # Sec. 3.2: ordering [Y00, Y1-1, Y10, Y11, ...]; explicit Cartesian forms (3DGS/2DGS signs)
    d = np.array([0.36, -0.48, 0.8])
    x, y, z = d
    Y = O.sh_eval(2, d)
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    c2 = 0.5 * math.sqrt(15.0 / math.pi)
    ref = [c0, -c1 * y, c1 * z, -c1 * x, c2 * x * y, -c2 * y * z,
           0.25 * math.sqrt(5 / math.pi) * (3 * z * z - 1), -c2 * x * z, 0.5 * c2 * (x * x - y * y)]
    np.testing.assert_allclose(Y, ref, rtol=1e-13, atol=1e-15)


def test_sh_orthonormal_by_quadrature():
    L = 6
    dirs, w = sphere_quadrature()
    Ys = np.array([O.sh_eval(L, d) for d in dirs])
    G = (Ys * w[:, None]).T @ Ys
    np.testing.assert_allclose(G, np.eye((L + 1) ** 2), atol=1e-12)


def test_sh_reflection_and_parity_identities():
    rng = np.random.default_rng(5)
    L = 4
    sign_m = np.array([(-1) ** abs(m) for l in range(L + 1) for m in range(-l, l + 1)], float)
    sign_l = np.array([(-1) ** l for l in range(L + 1) for m in range(-l, l + 1)], float)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        # mirror about the z axis (x,y,z) -> (-x,-y,z) multiplies Y_lm by (-1)^m (Eq. sh-brdf)
        np.testing.assert_allclose(O.sh_eval(L, [-d[0], -d[1], d[2]]), sign_m * O.sh_eval(L, d), atol=1e-14)
        # Ybar(w) = Y(-w) = (-1)^l Y(w)
        np.testing.assert_allclose(O.sh_eval(L, -d), sign_l * O.sh_eval(L, d), atol=1e-14)


def _funk_hecke_phong(l, s):
    """h_l = 2 pi int_0^1 (s+1)/(2 pi) t^s P_l(t) dt by adaptive quadrature."""
    val, err = integrate.quad(lambda t: (s + 1.0) * t ** s * special.eval_legendre(l, t), 0.0, 1.0,
                              epsabs=1e-14, epsrel=1e-13, limit=200)
    return val


@pytest.mark.parametrize("s", [1.0, 1.5, 2.7, 3.2, 10.0])
def test_phong_coefficients_equal_funk_hecke_quadrature(s):
    for l in range(9):
        assert abs(O.phong_rho(l, s) - _funk_hecke_phong(l, s)) < 1e-11


def test_phong_coefficients_golden():
    for line in open(os.path.join(GOLDEN, "phong_rho.txt")):
        if line.startswith("#") or not line.strip():
            continue
        s, l, num, den = (int(v) for v in line.split())
        assert O.phong_rho(l, s) == pytest.approx(num / den, abs=1e-15)


def test_diffuse_coefficient_is_4k_ad():
    # App. A: c00 = 4 k a^d + (1-k) a^s ; diffuse part k a^d / pi projected by Funk-Hecke
    sc = dict(n=1, L=3, p=[[0, 0, 0]], tu=[[1, 0, 0]], tv=[[0, 1, 0]], s=[[0.1, 0.1]], o=[1.0],
              ad=[[0.3, 0.5, 0.7]], k=[0.7], as_=[[0.2, 0.1, 0.05]], shin=[2.0])
    sc = {k: (np.array(v, float) if isinstance(v, list) else v) for k, v in sc.items()}
    c = O.Oracle(sc).brdf()[0]
    fh0 = 2 * math.pi * 2.0 * 0.7 * np.array([0.3, 0.5, 0.7]) / math.pi   # 2pi int_{-1}^{1} k a^d/pi dt
    np.testing.assert_allclose(c[0], fh0 + 0.3 * np.array([0.2, 0.1, 0.05]), rtol=1e-14)
    for l in (1, 2, 3):
        np.testing.assert_allclose(c[l], 0.3 * np.array([0.2, 0.1, 0.05]) * _funk_hecke_phong(l, 2.0), rtol=1e-10)


def test_splitmix64_golden():
    gamma = 0x9E3779B97F4A7C15
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, val = line.split()
        assert O.splitmix64((int(k) * gamma) % 2 ** 64) == int(val, 16)


def test_jitter_is_uniform_on_24_bit_grid():
    """The stratum jitter is uniform on [0, 1) in steps of 2^-24 (App. B's stratified
    sampling needs the full unit interval per stratum): a Kolmogorov-Smirnov test over
    20,000 keys, and every value on the 24-bit grid."""
    v = np.array([O.jitter(3, i, r, dim) for i in range(2500) for r in range(4) for dim in range(2)])
    assert np.all((v >= 0.0) & (v < 1.0))
    np.testing.assert_array_equal(v * 2.0 ** 24, np.floor(v * 2.0 ** 24))
    assert stats.kstest(v, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("nd", [32, 64, 128, 192, 256, 512])
def test_ray_strata_and_cosine_moments(nd):
    """Stratified cosine-weighted hemisphere directions: ray r lies in its own stratum
    (a, b) and the pi/Nd-weighted moments match int cos^k cos dw = 2 pi / (k+2)."""
    rng = np.random.default_rng(nd)
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    a0 = np.array([1.0, 0, 0]) if abs(nrm[0]) < 0.9 else np.array([0, 1.0, 0])
    tu = np.cross(nrm, a0)
    tu /= np.linalg.norm(tu)
    tv = np.cross(nrm, tu)
    sc = dict(n=1, L=0, p=np.zeros((1, 3)), tu=tu[None], tv=tv[None], s=np.full((1, 2), 0.1), o=np.ones(1),
              ad=np.full((1, 3), 0.5), k=np.ones(1), as_=np.zeros((1, 3)), shin=np.ones(1))
    orc = O.Oracle(sc)
    na = O.strata_a(nd)
    assert na * na <= nd < 4 * na * na and nd % na == 0
    nb = nd // na
    cos = []
    for r in range(nd):
        d = orc.ray_dir(0, nd, 7, r)
        assert abs(np.linalg.norm(d) - 1) < 1e-14
        cz = d @ nrm
        assert cz > 0
        u1 = 1 - cz * cz
        u2 = (math.atan2(d @ tv, d @ tu) / (2 * math.pi)) % 1.0
        a, b = r // nb, r % nb
        assert a / na - 1e-12 <= u1 < (a + 1) / na + 1e-12
        assert b / nb - 1e-12 <= u2 < (b + 1) / nb + 1e-12 or (b == nb - 1 and u2 < 1e-12)
        cos.append(cz)
    cos = np.array(cos)
    for kpow in (0, 1, 2, 4):
        est = math.pi / nd * np.sum(cos ** kpow)
        assert abs(est - 2 * math.pi / (kpow + 2)) < 4.0 / na * 2 * math.pi / (kpow + 2)
