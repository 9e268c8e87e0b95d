"""Image formation on the GPU (rgs_render / rgs_render_adjoint: Eq. L_I for the rays of a
pinhole camera, the image the paper's rasterizer draws from the solved radiance, and its
transpose) against the FP64 oracle's or_render / or_render_adjoint on the same radiance.

Both sides composite the same hits in the same order (the transport's hit rules, near-equal
depths ordered by caller index); the GPU evaluates them in FP32.  A hit flips across the
cutoff only when its FP32 radius lands within a few ulps of it (a flipped hit weighs
o e^{-4.5} ~ 1 % of the pixel), which none of these cameras meets, so the image and dL/dB
agree to the FP32 bar (1e-4 relative L2) and every pixel to 1e-4 of the image's largest
value.  The GPU's own render and adjoint trace identical rays, so <render(B), G> =
<B, render_adjoint(G)> holds to FP32 summation rounding."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_18497_gb300 import api, rgs, scenes

from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build
    build.build()


def _look_at(eye, at, up=(0.0, 1.0, 0.0)):
    eye = np.asarray(eye, float)
    f = np.asarray(at, float) - eye
    return list(eye) + list(f / np.linalg.norm(f)) + list(up)


CAM_BOWL = _look_at((0.3, 2.6, 4.4), (0.0, 0.5, 0.0))
CAM_LOW = _look_at((-3.0, 0.9, -2.2), (0.2, 0.6, 0.1))


def _pair(sc, alpha_gpu, alpha_orc):
    d = api.upload(sc)
    pipe = api.Pipeline(alpha_gpu, rgs.RGS_FP32)
    pipe.build(d)
    pipe.trace(d)
    orc = O.Oracle(sc, alpha_model=alpha_orc).transport()
    return pipe, orc


def _compare(pipe, orc, B, G, cam, W, H, fov):
    img_o = orc.render(B, cam, W, H, fov)
    dB_o = orc.render_adjoint(G, cam, W, H, fov)
    Bt = torch.as_tensor(B.astype(np.float32), device="cuda")
    Gt = torch.as_tensor(G.astype(np.float32), device="cuda")
    img = rgs.rgs_render(pipe.transport, Bt, cam, W, H, fov)
    dB = rgs.rgs_render_adjoint(pipe.transport, Gt, cam, W, H, fov)
    torch.cuda.synchronize()
    img_g = img.double().cpu().numpy()
    dB_g = dB.double().cpu().numpy()
    assert np.abs(img_o).max() > 0.0 and np.count_nonzero(img_o[..., 0]) > W * H // 10  # the camera sees the scene
    assert rel_l2(img_g, img_o) <= TOL_FP32, rel_l2(img_g, img_o)
    assert np.abs(img_g - img_o).max() <= TOL_FP32 * np.abs(img_o).max()
    np.testing.assert_array_equal(img_g == 0.0, img_o == 0.0)  # the same pixels see nothing
    assert rel_l2(dB_g, dB_o) <= TOL_FP32, rel_l2(dB_g, dB_o)
    lhs = float(np.sum(img_g * G))
    rhs = float(np.sum(B.astype(np.float32).astype(np.float64) * dB_g))
    assert lhs == pytest.approx(rhs, rel=1e-5)
    return img_g, dB_g


@pytest.mark.parametrize("alpha", [(rgs.RGS_ALPHA_GAUSS, O.ALPHA_GAUSS), (rgs.RGS_ALPHA_DISC, O.ALPHA_DISC),
                                   (rgs.RGS_ALPHA_GFSGS, O.ALPHA_GFSGS)], ids=["gauss", "disc", "gfsgs"])
def test_render_of_the_solved_bowl(alpha):
    """The oracle's solved radiance of the bowl scene (SH degree 3, 3 columns), rendered by
    both sides from above at 67 x 45 pixels (ragged against the 128-thread blocks)."""
    sc = scenes.fruit_bowl(n=2997, L=3, nd=64, nb=2, n_lights=1)
    pipe, orc = _pair(sc, *alpha)
    B = orc.solve(E=sc.get("E"), nb=sc["nb"])
    G = np.random.default_rng(3).normal(size=(45, 67, orc.C))
    _compare(pipe, orc, B, G, CAM_BOWL, 67, 45, 0.8)


def test_render_of_a_hundred_light_radiance():
    """300 columns (ten 32-column lane passes), random radiance, a grazing camera: long
    depth-ordered hit lists through the bowl's shells."""
    sc = scenes.multi_light(n=2000, L=3, nd=32, nb=1, n_lights=100)
    pipe, orc = _pair(sc, rgs.RGS_ALPHA_GAUSS, O.ALPHA_GAUSS)
    rng = np.random.default_rng(5)
    B = rng.normal(size=(sc["n"], 16, orc.C))
    G = rng.normal(size=(24, 40, orc.C))
    _compare(pipe, orc, B, G, CAM_LOW, 40, 24, 1.1)


def test_render_degenerate_images():
    """One pixel; a camera looking away from the scene (every pixel 0, dL/dB 0); a rejected
    field of view and a non-finite camera leave the outputs untouched."""
    sc = scenes.fruit_bowl(n=997, L=1, nd=32, nb=1, n_lights=1)
    pipe, orc = _pair(sc, rgs.RGS_ALPHA_GAUSS, O.ALPHA_GAUSS)
    rng = np.random.default_rng(7)
    B = rng.normal(size=(sc["n"], 4, orc.C))
    Bt = torch.as_tensor(B.astype(np.float32), device="cuda")
    one = rgs.rgs_render(pipe.transport, Bt, CAM_BOWL, 1, 1, 0.5).double().cpu().numpy()
    np.testing.assert_allclose(one, orc.render(B, CAM_BOWL, 1, 1, 0.5), rtol=1e-4, atol=1e-6)
    away = _look_at((0.0, 3.0, 6.0), (0.0, 3.0, 12.0))
    img = rgs.rgs_render(pipe.transport, Bt, away, 16, 9, 1.0)
    assert float(img.abs().max()) == 0.0
    dB = rgs.rgs_render_adjoint(pipe.transport, torch.ones((9, 16, orc.C), device="cuda"), away, 16, 9, 1.0)
    assert float(dB.abs().max()) == 0.0
    keep = torch.full((4, 4, orc.C), 7.0, device="cuda")
    for fov, cam, status in ((0.0, CAM_BOWL, rgs.RGS_ERR_ARG), (math.pi, CAM_BOWL, rgs.RGS_ERR_ARG),
                             (0.5, CAM_BOWL[:8] + [float("nan")], rgs.RGS_ERR_NONFINITE)):
        with pytest.raises(rgs.RgsError) as e:
            rgs.rgs_render(pipe.transport, Bt, cam, 4, 4, fov, img_out=keep)
        assert e.value.status == status
    assert float((keep - 7.0).abs().max()) == 0.0
