"""Seeded synthetic scene generators.

This module only *places* Gaussian surfels, materials and point lights; it holds
none of the transport arithmetic (no SH, no BRDF coefficients, no rays). Both the
CUDA path and the FP64 oracle read the arrays it produces, so every value is
rounded to float32 first and carried as float64: the two sides see bit-identical
inputs.

A scene is a dict of numpy float64 arrays in the user layout of the C ABI:

    p[N,3]  tu[N,3]  tv[N,3]  s[N,2]  o[N]  ad[N,3]  k[N]  as_[N,3]  shin[N]
    E[N,nc,3] (or None)   light_pos[NL,3]   light_I[NL,3]
    and the solver settings  L (SH degree), nd (rays / surfel), nb (bounces), seed.

Workload recipes follow the paper's scene types (an enclosed box with objects, an
object-in-bowl scene with interreflection, point lights; Sec. 9 and Sec. 10 of the
paper); the public datasets the paper evaluates on are not available, these
seeded scenes stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

F32 = np.float32


def _f(x):
    """Round to float32 and carry as float64 (identical inputs for both sides)."""
    return np.asarray(x, dtype=np.float64).astype(F32).astype(np.float64)


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _tangent_basis(n):
    """Right-handed in-plane basis (e1, e2) with e1 x e2 = n, for unit normals n[M,3]."""
    a = np.where(np.abs(n[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    e1 = _unit(np.cross(n, a))
    e2 = np.cross(n, e1)
    return e1, e2


def _rotated_frame(n, rng):
    """Tangent frame (tu, tv) rotated by a uniform random angle about n; tu x tv = n."""
    e1, e2 = _tangent_basis(n)
    th = rng.uniform(0.0, 2.0 * math.pi, size=(n.shape[0], 1))
    c, s = np.cos(th), np.sin(th)
    tu = c * e1 + s * e2
    tv = -s * e1 + c * e2
    return tu, tv


def _split_counts(areas, n):
    """Integer counts proportional to area that sum to n (largest remainder)."""
    areas = np.asarray(areas, dtype=np.float64)
    raw = areas / areas.sum() * n
    cnt = np.floor(raw).astype(np.int64)
    rem = n - cnt.sum()
    order = np.argsort(-(raw - cnt), kind="stable")
    cnt[order[:rem]] += 1
    return cnt


def fibonacci_sphere(m, radius=1.0, center=(0.0, 0.0, 0.0)):
    k = np.arange(m, dtype=np.float64)
    y = 1.0 - 2.0 * (k + 0.5) / m
    r = np.sqrt(np.maximum(0.0, 1.0 - y * y))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    pts = np.stack([r * np.cos(phi), y, r * np.sin(phi)], axis=1)
    return pts * radius + np.asarray(center, dtype=np.float64)


# --------------------------------------------------------------------------- faces
class _Rect:
    """Planar rectangle: origin + a*ea + b*eb, a in [0,la], b in [0,lb], normal n."""

    def __init__(self, origin, ea, eb, la, lb, normal):
        self.o = np.asarray(origin, np.float64)
        self.ea = _unit(np.asarray(ea, np.float64)[None])[0]
        self.eb = _unit(np.asarray(eb, np.float64)[None])[0]
        self.la, self.lb = float(la), float(lb)
        self.n = _unit(np.asarray(normal, np.float64)[None])[0]

    def area(self):
        return self.la * self.lb

    def sample(self, m, rng):
        a = rng.uniform(0.0, self.la, size=(m, 1))
        b = rng.uniform(0.0, self.lb, size=(m, 1))
        p = self.o + a * self.ea + b * self.eb
        return p, np.repeat(self.n[None], m, axis=0)


class _Sphere:
    """Full sphere (outward normals) or the lower hemisphere (y <= centre) with
    inward or outward normals."""

    def __init__(self, center, radius, lower_half=False, inward=False):
        self.c = np.asarray(center, np.float64)
        self.r = float(radius)
        self.half = lower_half
        self.inward = inward

    def area(self):
        a = 4.0 * math.pi * self.r ** 2
        return a / 2 if self.half else a

    def sample(self, m, rng):
        v = _unit(rng.normal(size=(m, 3)))
        if self.half:
            v[:, 1] = -np.abs(v[:, 1])
        p = self.c + self.r * v
        n = -v if self.inward else v
        return p, n


def _materials(rng, m, ad_lo, ad_hi, o_lo, o_hi, L, pure_diffuse):
    ad = rng.uniform(ad_lo, ad_hi, size=(m, 3))
    o = rng.uniform(o_lo, o_hi, size=m)
    if pure_diffuse:
        k = np.ones(m)
        as_ = np.zeros((m, 3))
        shin = np.ones(m)
    else:
        k = rng.uniform(0.6, 1.0, size=m)
        as_ = rng.uniform(0.1, 0.4, size=(m, 3))
        # keep k*ad + (1-k)*as <= 0.95 per channel (energy bound of the mixture)
        cap = (0.95 - k[:, None] * ad) / np.maximum(1.0 - k[:, None], 1e-12)
        as_ = np.minimum(as_, np.maximum(cap, 0.0))
        shin = rng.uniform(1.0, max(1.0, (L + 1) ** 2 / 5.0), size=m)
    return ad, o, k, as_, shin


def _assemble(parts, counts, rng, scale_fn, ad_rng, o_rng, L, pure_diffuse):
    ps, ns = [], []
    for part, c in zip(parts, counts):
        if c == 0:
            continue
        p, n = part.sample(int(c), rng)
        ps.append(p)
        ns.append(n)
    p = np.concatenate(ps)
    n = np.concatenate(ns)
    m = p.shape[0]
    tu, tv = _rotated_frame(n, rng)
    s = scale_fn(m)
    ad, o, k, as_, shin = _materials(rng, m, ad_rng[0], ad_rng[1], o_rng[0], o_rng[1], L, pure_diffuse)
    return dict(p=p, tu=tu, tv=tv, s=s, o=o, ad=ad, k=k, as_=as_, shin=shin)


def _finish(sc, L, nd, nb, seed, light_pos, light_I, E=None, name=""):
    out = {key: _f(v) for key, v in sc.items()}
    out.update(
        L=int(L), nd=int(nd), nb=int(nb), seed=int(seed), name=name,
        light_pos=_f(np.asarray(light_pos, np.float64).reshape(-1, 3)),
        light_I=_f(np.asarray(light_I, np.float64).reshape(-1, 3)),
        E=None if E is None else _f(E),
    )
    out["n"] = out["p"].shape[0]
    return out


# --------------------------------------------------------------------------- scenes
def box_scene(n=2000, seed=0, L=2, nd=64, nb=3, pure_diffuse=False):
    """Closed box: unit cube with 5 walls (front z=0 open) and two inner cubes.

    Walls face the interior; cube faces face outward; cube bottoms are omitted.
    Scales U[0.02,0.05], opacity U[0.9,1], diffuse albedo U[0.3,0.8]^3, one point
    light at (0.5, 0.95, 0.5) with intensity 10.
    """
    rng = np.random.default_rng(seed)
    parts = [
        _Rect((0, 0, 0), (0, 0, 1), (1, 0, 0), 1, 1, (0, 1, 0)),    # floor
        _Rect((0, 1, 0), (1, 0, 0), (0, 0, 1), 1, 1, (0, -1, 0)),   # ceiling
        _Rect((0, 0, 1), (1, 0, 0), (0, 1, 0), 1, 1, (0, 0, -1)),   # back
        _Rect((0, 0, 0), (0, 1, 0), (0, 0, 1), 1, 1, (1, 0, 0)),    # left
        _Rect((1, 0, 0), (0, 0, 1), (0, 1, 0), 1, 1, (-1, 0, 0)),   # right
    ]
    for center, side, rot in (((0.3, 0.15, 0.35), 0.3, 0.0), ((0.7, 0.125, 0.65), 0.25, math.radians(30.0))):
        c = np.asarray(center, np.float64)
        h = side / 2
        cr, sr = math.cos(rot), math.sin(rot)
        R = np.array([[cr, 0, sr], [0, 1, 0], [-sr, 0, cr]])  # rotation about +y
        ex, ey, ez = R @ np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), R @ np.array([0, 0, 1.0])
        faces = [
            (c + h * ey - h * ex - h * ez, ez, ex, ey),   # top (+y)
            (c + h * ex - h * ey - h * ez, ey, ez, ex),   # +x
            (c - h * ex - h * ey - h * ez, ez, ey, -ex),  # -x
            (c + h * ez - h * ey - h * ex, ex, ey, ez),   # +z
            (c - h * ez - h * ey - h * ex, ey, ex, -ez),  # -z
        ]
        for o0, ea, eb, nn in faces:
            parts.append(_Rect(o0, ea, eb, side, side, nn))
    counts = _split_counts([q.area() for q in parts], n)
    sc = _assemble(parts, counts, rng, lambda m: rng.uniform(0.02, 0.05, size=(m, 2)),
                   (0.3, 0.8), (0.9, 1.0), L, pure_diffuse)
    return _finish(sc, L, nd, nb, seed, [[0.5, 0.95, 0.5]], [[10.0, 10.0, 10.0]], name="box")


def _bowl_parts(rng, scale=1.0):
    R_out, R_in = 1.0 * scale, 0.98 * scale
    c0 = np.array([0.0, 1.0 * scale, 0.0])
    parts = [
        _Rect((-2 * scale, 0, 2 * scale), (0, 0, -1), (1, 0, 0), 4 * scale, 4 * scale, (0, 1, 0)),  # ground
        _Sphere(c0, R_in, lower_half=True, inward=True),   # bowl, inner layer
        _Sphere(c0, R_out, lower_half=True, inward=False),  # bowl, outer layer
    ]
    radii = np.sort(rng.uniform(0.1, 0.3, size=12))[::-1] * scale
    centers = []
    for r in radii:
        for _ in range(100000):
            c = np.array([rng.uniform(-R_in, R_in), rng.uniform(0.0, 1.0 * scale), rng.uniform(-R_in, R_in)])
            if np.linalg.norm(c - c0) + r > R_in - 0.01 * scale:
                continue
            if any(np.linalg.norm(c - c2) < r + r2 + 0.01 * scale for c2, r2 in centers):
                continue
            centers.append((c, r))
            break
        else:  # pragma: no cover - the packing is loose enough that this never triggers
            raise RuntimeError("sphere packing failed")
    for c, r in centers:
        parts.append(_Sphere(c, r))
    return parts


def fruit_bowl(n=50000, seed=0, L=3, nd=256, nb=4, n_lights=1, pure_diffuse=False,
               light_intensity=None, scale=1.0):
    """Object-in-bowl scene: ground square [-2,2]^2 at y=0, a hemispherical bowl shell
    (inner and outer layers 0.02 apart, centre (0,1,0), radius 1) and 12 non-overlapping
    spheres of radius U[0.1,0.3] inside the cavity.

    Per-axis scale = U[0.4,0.9]*sqrt(A/N), diffuse albedo U[0.1,0.9]^3, opacity
    U[0.5,1]. One light at (0,3,0) with intensity 10, or `n_lights` lights on a
    Fibonacci sphere of radius 3 around (0,0.5,0) with white intensity U[5,20].
    """
    rng = np.random.default_rng(seed)
    parts = _bowl_parts(rng, scale)
    areas = [q.area() for q in parts]
    counts = _split_counts(areas, n)
    spacing = math.sqrt(sum(areas) / n)
    sc = _assemble(parts, counts, rng, lambda m: rng.uniform(0.4, 0.9, size=(m, 2)) * spacing,
                   (0.1, 0.9), (0.5, 1.0), L, pure_diffuse)
    if n_lights == 1:
        lp = np.array([[0.0, 3.0 * scale, 0.0]])
        li = np.full((1, 3), 10.0 if light_intensity is None else light_intensity)
    else:
        lp = fibonacci_sphere(n_lights, 3.0 * scale, (0.0, 0.5 * scale, 0.0))
        w = rng.uniform(5.0, 20.0, size=(n_lights, 1))
        li = np.repeat(w, 3, axis=1)
    return _finish(sc, L, nd, nb, seed, lp, li, name=f"fruit_bowl_{n}")


def multi_light(n=200000, seed=0, n_lights=100, L=3, nd=256, nb=4):
    """Many-light batch on the fruit-bowl generator (all lights are right-hand sides)."""
    return fruit_bowl(n=n, seed=seed, L=L, nd=nd, nb=nb, n_lights=n_lights)


def uneven_batch(count=32, base_seed=1000, n_lights=8, scale=1.0):
    """Independent fruit-bowl scenes with log-uniform surfel counts in [5e3, 3e5] (times
    `scale`, for reduced profiling cases), SH degree 2 or 3, 128/192/256 rays per surfel and
    3-5 bounces."""
    out = []
    for s in range(count):
        rng = np.random.default_rng(base_seed + s)
        ns = int(round(math.exp(rng.uniform(math.log(5e3), math.log(3e5))) * scale))
        L = int(rng.choice([2, 3]))
        nd = int(rng.choice([128, 192, 256]))
        nb = int(rng.choice([3, 4, 5]))
        out.append(fruit_bowl(n=ns, seed=base_seed + s, L=L, nd=nd, nb=nb, n_lights=n_lights))
    return out


def _lattice_hash(ix, iy, iz, salt):
    """Integer lattice hash -> [0, 1): a 32-bit multiply-xorshift mix of the three
    coordinates (wrapped to uint32) and a salt."""
    m = np.uint64(0xFFFFFFFF)
    h = (ix.astype(np.int64).astype(np.uint64) * np.uint64(0x8DA6B343)) & m
    h ^= (iy.astype(np.int64).astype(np.uint64) * np.uint64(0xD8163841)) & m
    h ^= (iz.astype(np.int64).astype(np.uint64) * np.uint64(0xCB1AB31F)) & m
    h ^= np.uint64(salt) & m
    h = (h ^ (h >> np.uint64(16))) * np.uint64(0x7FEB352D) & m
    h = (h ^ (h >> np.uint64(15))) * np.uint64(0x846CA68B) & m
    h ^= h >> np.uint64(16)
    return (h & m).astype(np.float64) / 4294967296.0


def value_noise(x, salt=0):
    """Value noise on the integer lattice: hashed corner values blended trilinearly with
    smoothstep weights. x: [M,3] -> [M] in [0, 1)."""
    x = np.asarray(x, np.float64)
    i0 = np.floor(x)
    f = x - i0
    w = f * f * (3.0 - 2.0 * f)
    i0 = i0.astype(np.int64)
    out = np.zeros(x.shape[0])
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                wt = ((w[:, 0] if dx else 1.0 - w[:, 0]) * (w[:, 1] if dy else 1.0 - w[:, 1])
                      * (w[:, 2] if dz else 1.0 - w[:, 2]))
                out += wt * _lattice_hash(i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz, salt)
    return out


def large_scene(n=1000000, seed=0, L=3, nd=512, nb=6, n_lights=16, scale=4.0, room=20.0):
    """The fruit bowl scaled by `scale` inside a room: four walls and a ceiling of side
    `room` (x, z in [-room/2, room/2], y in [0, room]) facing inward, whose diffuse albedo
    is 0.2 + 0.6 * value_noise(0.5 * x) per channel (three lattice salts). Surfel counts
    are proportional to area over all parts, scales U[0.4,0.9]*sqrt(A/N) as in fruit_bowl.
    `n_lights` white lights U[5,20] on a Fibonacci sphere of radius 0.4*room centred at
    mid-height, so that every light is inside the room."""
    rng = np.random.default_rng(seed)
    parts = _bowl_parts(rng, scale)
    h = room / 2.0
    walls = [
        _Rect((-h, room, -h), (1, 0, 0), (0, 0, 1), room, room, (0, -1, 0)),  # ceiling
        _Rect((-h, 0, -h), (0, 1, 0), (1, 0, 0), room, room, (0, 0, 1)),      # z = -h
        _Rect((-h, 0, h), (1, 0, 0), (0, 1, 0), room, room, (0, 0, -1)),      # z = +h
        _Rect((-h, 0, -h), (0, 0, 1), (0, 1, 0), room, room, (1, 0, 0)),      # x = -h
        _Rect((h, 0, -h), (0, 1, 0), (0, 0, 1), room, room, (-1, 0, 0)),      # x = +h
    ]
    parts = parts + walls
    areas = [q.area() for q in parts]
    counts = _split_counts(areas, n)
    spacing = math.sqrt(sum(areas) / n)
    sc = _assemble(parts, counts, rng, lambda m: rng.uniform(0.4, 0.9, size=(m, 2)) * spacing,
                   (0.1, 0.9), (0.5, 1.0), L, False)
    n_wall = int(sum(counts[-len(walls):]))
    pw = sc["p"][-n_wall:]
    tex = np.stack([value_noise(0.5 * pw, salt=c) for c in range(3)], axis=1)
    ad = sc["ad"].copy()
    ad[-n_wall:] = 0.2 + 0.6 * tex
    k, as_ = sc["k"], sc["as_"].copy()
    cap = (0.95 - k[-n_wall:, None] * ad[-n_wall:]) / np.maximum(1.0 - k[-n_wall:, None], 1e-12)
    as_[-n_wall:] = np.minimum(as_[-n_wall:], np.maximum(cap, 0.0))
    sc["ad"], sc["as_"] = ad, as_
    lp = fibonacci_sphere(n_lights, 0.4 * room, (0.0, h, 0.0))
    li = np.repeat(rng.uniform(5.0, 20.0, size=(n_lights, 1)), 3, axis=1)
    return _finish(sc, L, nd, nb, seed, lp, li, name=f"large_{n}")


def env_map(n_theta=16, n_phi=32, sun=(0.35, 0.8, 0.45), seed=0):
    """An environment map on an n_theta x n_phi latitude-longitude grid as directional lights
    (the paper's 16 x 32 map of distant lights without inverse-square falloff): one light per
    cell centre, direction from the polar angle theta (from +y) and azimuth phi, intensity =
    radiance x the cell's solid angle sin(theta) dtheta dphi.  Radiance: a sky gradient
    0.4 + 0.6 max(0, y) plus a sun lobe 8 max(0, w.sun)^16, per channel tinted by a seeded
    colour in [0.8, 1].  Returns (directions [M,3], intensities [M,3])."""
    rng = np.random.default_rng(seed)
    tint = rng.uniform(0.8, 1.0, size=3)
    th = (np.arange(n_theta) + 0.5) * math.pi / n_theta
    ph = (np.arange(n_phi) + 0.5) * 2.0 * math.pi / n_phi
    T, P = np.meshgrid(th, ph, indexing="ij")
    w = np.stack([np.sin(T) * np.cos(P), np.cos(T), np.sin(T) * np.sin(P)], axis=-1).reshape(-1, 3)
    s = _unit(np.asarray(sun, np.float64)[None])[0]
    rad = 0.4 + 0.6 * np.maximum(0.0, w[:, 1]) + 8.0 * np.maximum(0.0, w @ s) ** 16
    dom = (np.sin(T) * (math.pi / n_theta) * (2.0 * math.pi / n_phi)).reshape(-1)
    return w, (rad * dom)[:, None] * tint[None, :]


def with_env_map(sc, n_theta=16, n_phi=32, seed=0):
    """The scene lit by `env_map` instead of its point lights (directional lights)."""
    w, I = env_map(n_theta, n_phi, seed=seed)
    out = dict(sc)
    out["light_pos"], out["light_I"] = _f(w), _f(I)
    out["light_dir"] = True
    out["name"] = sc.get("name", "") + f"_env{n_theta}x{n_phi}"
    return out


def with_emission(sc, seed=1, scale=0.5, dc_only=False):
    """Attach a seeded emission E[N,nc,3] (used by the gradient tests)."""
    rng = np.random.default_rng(seed)
    nc = (sc["L"] + 1) ** 2
    E = rng.uniform(0.0, scale, size=(sc["n"], nc, 3))
    if dc_only:
        E[:, 1:, :] = 0.0
    else:
        E[:, 1:, :] *= 0.2
    out = dict(sc)
    out["E"] = _f(E)
    return out


# ------------------------------------------------------------------ analytic test scenes
def furnace_sphere(m=2000, rho=0.6, emission=1.0, L=2, nd=64, nb=4, seed=0):
    """Closed unit sphere tiled by `m` inward-facing surfels at Fibonacci points, for the
    `disc` opacity model: disc radius twice the mean spacing, opacity 1, pure diffuse
    albedo `rho`, uniform emission (DC coefficient `emission`), no lights."""
    p = fibonacci_sphere(m)
    n = -p
    rng = np.random.default_rng(seed)
    tu, tv = _rotated_frame(n, rng)
    spacing = math.sqrt(4.0 * math.pi / m)
    nc = (L + 1) ** 2
    E = np.zeros((m, nc, 3))
    E[:, 0, :] = emission
    sc = dict(p=p, tu=tu, tv=tv, s=np.full((m, 2), 2.0 * spacing), o=np.ones(m),
              ad=np.full((m, 3), rho), k=np.ones(m), as_=np.zeros((m, 3)), shin=np.ones(m))
    return _finish(sc, L, nd, nb, seed, np.zeros((0, 3)), np.zeros((0, 3)), E=E, name="furnace")


def lone_plane(L=2, o=0.8, ad=(0.5, 0.3, 0.2), k=1.0, as_=(0.0, 0.0, 0.0), shin=1.0,
               light_pos=(0.3, -0.2, 1.5), light_I=(10.0, 7.0, 4.0), nd=64):
    """One surfel at the origin facing +z, one point light, nothing else."""
    sc = dict(p=np.zeros((1, 3)), tu=np.array([[1.0, 0, 0]]), tv=np.array([[0, 1.0, 0]]),
              s=np.array([[0.05, 0.05]]), o=np.array([o]), ad=np.array([ad], np.float64),
              k=np.array([k]), as_=np.array([as_], np.float64), shin=np.array([shin]))
    return _finish(sc, L, nd, 1, 0, [light_pos], [light_I], name="lone_plane")


def random_cluster(n=120, seed=0, L=2, nd=64, nb=3, n_lights=2, extent=1.0, pure_diffuse=False):
    """Small random cloud of surfels with random orientations inside a cube, plus a few
    lights: dense interreflection and occlusion at a size where dense solves are cheap."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.0, extent, size=(n, 3))
    nrm = _unit(rng.normal(size=(n, 3)))
    tu, tv = _rotated_frame(nrm, rng)
    s = rng.uniform(0.05, 0.15, size=(n, 2)) * extent
    ad, o, k, as_, shin = _materials(rng, n, 0.2, 0.8, 0.4, 1.0, L, pure_diffuse)
    lp = rng.uniform(-0.5, 1.5, size=(n_lights, 3)) * extent
    li = rng.uniform(2.0, 8.0, size=(n_lights, 3))
    sc = dict(p=p, tu=tu, tv=tv, s=s, o=o, ad=ad, k=k, as_=as_, shin=shin)
    return _finish(sc, L, nd, nb, seed, lp, li, name=f"cluster_{n}")
