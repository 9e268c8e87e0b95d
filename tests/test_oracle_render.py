"""Pins of the oracle's image formation (Eq. L_I for a pinhole camera, the image the
paper's rasterizer produces from the solved radiance): disc coverage against an
independent ray-plane computation, the composite of stacked surfels, the radiance leaving
towards the camera (front and back of a Y10 emitter), and the transpose (no GPU)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_18497_gb300 import scenes

from test_oracle_transport import make_scene

C1 = math.sqrt(3.0 / (4.0 * math.pi))
Y00 = 0.5 / math.sqrt(math.pi)
CAM = [0.0, 0.0, 2.0, 0.0, 0.0, -1.0, 0.0, 1.0, 0.0]  # at z = 2 looking down -z, y up


def _oracle(surfels, alpha_model=O.ALPHA_GAUSS):
    sc = make_scene(surfels, L=1, nb=0)
    return O.Oracle(sc, alpha_model=alpha_model).transport()


def _pixel_dirs(W, H, fov):
    """The pinhole's ray directions: forward -z, right +x, up +y, pixel centres."""
    th = math.tan(0.5 * fov)
    xs = (2.0 * (np.arange(W) + 0.5) / W - 1.0) * th * W / H
    ys = (1.0 - 2.0 * (np.arange(H) + 0.5) / H) * th
    d = np.stack(np.broadcast_arrays(xs[None, :], ys[:, None], -np.ones((H, W))), -1)
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def test_disc_coverage_and_value():
    s = 0.3
    orc = _oracle([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), s=(s, s), o=1.0)], alpha_model=O.ALPHA_DISC)
    B = np.zeros((1, 4, 3))
    B[0, 0] = (1.0, 2.0, 3.0)
    W, H, fov = 41, 31, 0.5
    img = orc.render(B, CAM, W, H, fov)
    d = _pixel_dirs(W, H, fov)
    t = 2.0 / -d[..., 2]  # the plane z = 0 from z = 2
    r2 = (t * d[..., 0]) ** 2 + (t * d[..., 1]) ** 2
    inside = r2 <= s * s
    assert inside.sum() > 20 and (~inside).sum() > 20
    np.testing.assert_allclose(img[inside], np.broadcast_to(np.array([1.0, 2.0, 3.0]) * Y00, img[inside].shape), rtol=1e-12)
    np.testing.assert_array_equal(img[~inside], 0.0)


def test_offset_disc_lands_where_the_pinhole_puts_it():
    """A disc up and to the right of the optical axis covers exactly the pixels whose
    rays (pixel (x, y) with x to the right and y down) meet it: the image is not mirrored
    in either axis."""
    s, cx, cy = 0.12, 0.25, 0.2
    orc = _oracle([dict(p=(cx, cy, 0), tu=(1, 0, 0), tv=(0, 1, 0), s=(s, s), o=1.0)], alpha_model=O.ALPHA_DISC)
    B = np.zeros((1, 4, 3))
    B[0, 0] = (1.0, 1.0, 1.0)
    W, H, fov = 40, 30, 0.6
    img = orc.render(B, CAM, W, H, fov)
    d = _pixel_dirs(W, H, fov)
    t = 2.0 / -d[..., 2]
    inside = (t * d[..., 0] - cx) ** 2 + (t * d[..., 1] - cy) ** 2 <= s * s
    ys, xs = np.nonzero(inside)
    assert inside.sum() > 10 and ys.max() < H // 2 and xs.min() >= W // 2  # upper right quadrant
    np.testing.assert_array_equal(img[..., 0] > 0.0, inside)


def test_camera_up_need_not_be_perpendicular():
    """Only the plane of forward and up matters: the true up is right x forward, so an up
    vector tilted towards the view direction renders the same image."""
    orc = _oracle([dict(p=(0.2, 0.1, 0), tu=(1, 0, 0), tv=(0, 1, 0), s=(0.2, 0.1), o=0.9)])
    B = np.zeros((1, 4, 3))
    B[0, 0], B[0, 2] = (1.0, 2.0, 3.0), (0.3, 0.2, 0.1)
    tilted = CAM[:6] + [0.0, 1.0, 0.7]
    np.testing.assert_allclose(orc.render(B, tilted, 24, 18, 0.7), orc.render(B, CAM, 24, 18, 0.7),
                               rtol=1e-12, atol=1e-14)


def test_gaussian_centre_and_stacked_composite():
    W = H = 21  # odd: the centre pixel's ray is the axis
    fov = 0.6
    # one Gaussian surfel: the axis meets it at its centre, alpha = o
    orc = _oracle([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), s=(0.2, 0.2), o=0.7)])
    B = np.zeros((1, 4, 3))
    B[0, 2] = (1.0, 0.5, 0.25)  # Y10 only
    img = orc.render(B, CAM, W, H, fov)
    np.testing.assert_allclose(img[H // 2, W // 2], 0.7 * C1 * B[0, 2], rtol=1e-12)
    # two discs on the axis: front alpha 0.4, back 0.9 -> 0.4 c_f + 0.6 * 0.9 c_b
    orc = _oracle([dict(p=(0, 0, 0.5), tu=(1, 0, 0), tv=(0, 1, 0), s=(0.2, 0.2), o=0.4),
                   dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), s=(0.2, 0.2), o=0.9)], alpha_model=O.ALPHA_DISC)
    B = np.zeros((2, 4, 3))
    B[0, 0], B[1, 0] = 1.0, 2.0
    img = orc.render(B, CAM, W, H, fov)
    np.testing.assert_allclose(img[H // 2, W // 2], (0.4 * 1.0 + 0.6 * 0.9 * 2.0) * Y00, rtol=1e-12)


def test_radiance_towards_the_camera_front_and_back():
    """The pixel shows B(-d): a Y10 emitter seen from +z gives +c1 b, from -z gives -c1 b."""
    W = H = 11
    fov = 0.4
    orc = _oracle([dict(p=(0, 0, 0), tu=(1, 0, 0), tv=(0, 1, 0), s=(0.2, 0.2), o=1.0)], alpha_model=O.ALPHA_DISC)
    B = np.zeros((1, 4, 3))
    B[0, 2] = 1.0
    front = orc.render(B, CAM, W, H, fov)[H // 2, W // 2]
    back = orc.render(B, [0.0, 0.0, -2.0, 0.0, 0.0, 1.0, 0.0, 1.0, 0.0], W, H, fov)[H // 2, W // 2]
    np.testing.assert_allclose(front, C1, rtol=1e-12)
    np.testing.assert_allclose(back, -C1, rtol=1e-12)


def test_render_adjoint_identity():
    sc = scenes.random_cluster(n=60, seed=1, L=2, nb=1, n_lights=2)
    orc = O.Oracle(sc).transport()
    rng = np.random.default_rng(3)
    B = rng.normal(size=orc._shape())
    W, H, fov = 48, 32, 0.9
    cam = [0.5, 0.5, 3.0, 0.0, 0.0, -1.0, 0.0, 1.0, 0.0]
    Wimg = rng.normal(size=(H, W, orc.C))
    lhs = float(np.sum(orc.render(B, cam, W, H, fov) * Wimg))
    rhs = float(np.sum(B * orc.render_adjoint(Wimg, cam, W, H, fov)))
    assert abs(lhs) > 0
    assert lhs == pytest.approx(rhs, rel=1e-12)
