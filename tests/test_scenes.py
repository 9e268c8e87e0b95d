"""The seeded workload generators: shapes, ranges and invariants of the synthetic scenes
(they carry no transport arithmetic, so these are plain checks of what they place)."""
import math

import numpy as np

from paper_2509_18497_gb300 import scenes


def _frames_ok(sc):
    tu, tv = sc["tu"], sc["tv"]
    assert np.allclose(np.linalg.norm(tu, axis=1), 1.0, atol=1e-6)
    assert np.allclose(np.linalg.norm(tv, axis=1), 1.0, atol=1e-6)
    assert np.allclose(np.sum(tu * tv, axis=1), 0.0, atol=1e-6)


def test_value_noise_range_lattice_and_smoothness():
    rng = np.random.default_rng(0)
    x = rng.uniform(-50, 50, size=(20000, 3))
    v = scenes.value_noise(x)
    assert v.min() >= 0.0 and v.max() < 1.0
    assert 0.3 < v.mean() < 0.7
    # on lattice points the noise is the corner hash itself
    ip = np.floor(x[:50])
    assert np.allclose(scenes.value_noise(ip), scenes._lattice_hash(*(ip.astype(np.int64).T), 0))
    # smoothstep blending: continuous across a cell face
    a = np.array([[2.0 - 1e-9, 0.3, 0.7]])
    b = np.array([[2.0 + 1e-9, 0.3, 0.7]])
    assert abs(scenes.value_noise(a)[0] - scenes.value_noise(b)[0]) < 1e-6
    # different salts decorrelate the channels
    assert abs(np.corrcoef(scenes.value_noise(x, 0), scenes.value_noise(x, 1))[0, 1]) < 0.1


def test_large_scene_layout():
    n = 30000
    sc = scenes.large_scene(n=n)
    assert sc["n"] == n and sc["L"] == 3 and sc["nd"] == 512 and sc["nb"] == 6
    assert sc["light_pos"].shape == (16, 3)
    _frames_ok(sc)
    # every light inside the room (x, z in [-10, 10], y in [0, 20]), white, intensity in [5, 20]
    lp = sc["light_pos"]
    assert np.all(np.abs(lp[:, [0, 2]]) < 10.0) and np.all((lp[:, 1] > 0.0) & (lp[:, 1] < 20.0))
    assert np.all(sc["light_I"] >= 5.0) and np.all(sc["light_I"] <= 20.0)
    assert np.all(sc["light_I"][:, 0] == sc["light_I"][:, 1])
    # wall surfels: on the walls or the ceiling, facing the room, albedo 0.2 + 0.6 * noise
    p = sc["p"]
    n_hat = np.cross(sc["tu"], sc["tv"])
    on_wall = (np.abs(np.abs(p[:, 0]) - 10.0) < 1e-4) | (np.abs(np.abs(p[:, 2]) - 10.0) < 1e-4) | \
              (np.abs(p[:, 1] - 20.0) < 1e-4)
    assert on_wall.sum() > n // 2  # walls dominate the area
    inward = -np.sign(np.where(np.abs(np.abs(p[:, 0]) - 10.0) < 1e-4, p[:, 0], 0.0))
    xs = on_wall & (np.abs(np.abs(p[:, 0]) - 10.0) < 1e-4)
    assert np.all(np.sign(n_hat[xs, 0]) == inward[xs])
    ad_w = sc["ad"][on_wall]
    assert ad_w.min() >= 0.2 - 1e-6 and ad_w.max() <= 0.8 + 1e-6
    expect = 0.2 + 0.6 * np.stack([scenes.value_noise(0.5 * p[on_wall], c) for c in range(3)], axis=1)
    assert np.allclose(ad_w, expect, atol=1e-6)
    # energy bound of the BRDF mixture holds for every surfel
    mix = sc["k"][:, None] * sc["ad"] + (1.0 - sc["k"][:, None]) * sc["as_"]
    assert mix.max() <= 0.95 + 1e-6
    # the bowl inside keeps the fruit-bowl scale x4: ground square [-8, 8]^2 at y = 0
    ground = np.abs(p[:, 1]) < 1e-6
    assert ground.any() and np.all(np.abs(p[ground][:, [0, 2]]) <= 8.0 + 1e-6)


def test_uneven_batch_counts():
    scs = scenes.uneven_batch(32)
    ns = np.array([sc["n"] for sc in scs])
    assert len(scs) == 32 and ns.min() >= 5000 and ns.max() <= 300000
    assert {sc["L"] for sc in scs} <= {2, 3} and {sc["nd"] for sc in scs} <= {128, 192, 256}
    assert {sc["nb"] for sc in scs} <= {3, 4, 5}
    assert all(sc["light_pos"].shape == (8, 3) for sc in scs)
    # log-uniform draw: the log-counts spread over the range
    lg = np.log(ns)
    assert lg.min() < math.log(2e4) and lg.max() > math.log(1e5)
