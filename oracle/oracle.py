"""ctypes binding of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by bench.py's
CPU-baseline / reference legs.  The product path never imports this module.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALPHA_GAUSS, ALPHA_DISC, ALPHA_GFSGS = 0, 1, 2

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)
_lp = ct.POINTER(ct.c_long)


def build(force=False):
    """Compile oracle.c into liboracle.so (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The loaded oracle library.  ORACLE_LIB names a prebuilt copy to load instead (the
    mutation tests run the pins against deliberately broken builds of oracle.c)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("ORACLE_LIB")
            if not path:
                path = build()
            L = ct.CDLL(path)
            L.or_scene_new.restype = ct.c_void_p
            L.or_scene_new.argtypes = [ct.c_int, ct.c_int] + [_dp] * 9 + [ct.c_int, ct.c_int]
            L.or_scene_free.argtypes = [ct.c_void_p]
            L.or_sh_eval.argtypes = [ct.c_int, _dp, _dp]
            L.or_phong_rho.restype = ct.c_double
            L.or_phong_rho.argtypes = [ct.c_int, ct.c_double]
            L.or_splitmix64.restype = ct.c_uint64
            L.or_splitmix64.argtypes = [ct.c_uint64]
            L.or_jitter.restype = ct.c_double
            L.or_jitter.argtypes = [ct.c_uint64] * 4
            L.or_strata_a.restype = ct.c_int
            L.or_strata_a.argtypes = [ct.c_int]
            L.or_eps_plane.restype = ct.c_double
            L.or_eps_plane.argtypes = [ct.c_void_p]
            L.or_frames.argtypes = [ct.c_void_p, _dp, _dp, _dp]
            L.or_brdf.argtypes = [ct.c_void_p, _dp]
            L.or_ray_dir.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_uint64, ct.c_int, _dp]
            L.or_trace_ray.restype = ct.c_int
            L.or_trace_ray.argtypes = [ct.c_void_p, ct.c_int, _dp, _dp, ct.c_double, ct.c_int, _ip, _dp, _dp, _dp]
            L.or_transport.restype = ct.c_int
            L.or_transport.argtypes = [ct.c_void_p, ct.c_int, ct.c_uint64, ct.c_int, _dp, _dp]
            L.or_num_hits.restype = ct.c_long
            L.or_num_hits.argtypes = [ct.c_void_p]
            L.or_num_shadow_hits.restype = ct.c_long
            L.or_num_shadow_hits.argtypes = [ct.c_void_p]
            L.or_get_hits.argtypes = [ct.c_void_p, _lp, _ip, _dp, _dp, _dp, _dp]
            L.or_direct.argtypes = [ct.c_void_p, _dp]
            L.or_apply_K.argtypes = [ct.c_void_p, _dp, _dp, _dp]
            L.or_apply_KT.argtypes = [ct.c_void_p, _dp, _dp]
            L.or_solve.argtypes = [ct.c_void_p, _dp, ct.c_int, _dp, _dp]
            L.or_adjoint.argtypes = [ct.c_void_p, _dp, ct.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
            L.or_set_directional.argtypes = [ct.c_void_p, ct.c_int]
            L.or_ein.restype = ct.c_double
            L.or_ein.argtypes = [ct.c_double]
            L.or_pairs.restype = ct.c_int
            L.or_pairs.argtypes = [ct.c_void_p, _dp, ct.c_int, _dp, _dp]
            L.or_num_pairs.restype = ct.c_long
            L.or_num_pairs.argtypes = [ct.c_void_p]
            L.or_get_pairs.argtypes = [ct.c_void_p, _lp, _ip, _dp, _dp]
            L.or_alpha_area.restype = ct.c_double
            L.or_alpha_area.argtypes = [ct.c_void_p, ct.c_int]
            L.or_brdf_grad_closed_form.argtypes = [ct.c_void_p, _dp, ct.c_int, _dp, _dp]
            L.or_dense_K.argtypes = [ct.c_void_p, ct.c_int, _dp]
            L.or_sample_direct.argtypes = [ct.c_void_p, ct.c_int, _dp, _dp, ct.c_int, _ip, _dp]
            L.or_sample_bounce1.argtypes = [ct.c_void_p, ct.c_int, ct.c_uint64, ct.c_int, _dp, _dp, _dp,
                                            ct.c_int, _ip, _dp]
            L.or_sh_grad.argtypes = [ct.c_int, _dp, _dp, _dp]
            L.or_geometry_grad.restype = ct.c_int
            L.or_geometry_grad.argtypes = [ct.c_void_p, _dp, ct.c_int, _dp, _dp, _dp, _dp, _dp]
            L.or_mc_weights.restype = ct.c_long
            L.or_mc_weights.argtypes = [ct.c_void_p, _dp, ct.c_int, _dp, _dp]
            L.or_mc_pick.restype = ct.c_long
            L.or_mc_pick.argtypes = [ct.c_void_p, _dp, _dp, ct.c_uint64, ct.c_int, ct.c_int, ct.c_int, ct.c_int, _dp,
                                     _dp]
            L.or_mc_solve.restype = ct.c_int
            L.or_mc_solve.argtypes = [ct.c_void_p, _dp, ct.c_int, ct.c_uint64, ct.c_int, _dp, _dp, _dp]
            L.or_mc_groups.argtypes = [ct.c_void_p, ct.c_int, _ip]
            L.or_render.argtypes = [ct.c_void_p, _dp, _dp, ct.c_int, ct.c_int, ct.c_double, _dp]
            L.or_render_adjoint.argtypes = [ct.c_void_p, _dp, _dp, ct.c_int, ct.c_int, ct.c_double, _dp]
            L.or_prog_refine.restype = ct.c_int
            L.or_prog_refine.argtypes = [ct.c_void_p, _dp, ct.c_int, _dp, _dp]
            L.or_num_threads.restype = ct.c_int
            _lib = L
    return _lib


def _d(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    if a is None:
        return ct.cast(None, _dp)
    return a.ctypes.data_as(_dp)


def sh_eval(L, d):
    d = _d(d).reshape(3)
    out = np.zeros((L + 1) ** 2)
    lib().or_sh_eval(L, _ptr(d), _ptr(out))
    return out


def sh_grad(L, d):
    """(Y, dY) at direction d: dY[a, k] = dY_k/d(d_a) of the polynomial form."""
    d = _d(d).reshape(3)
    Y = np.zeros((L + 1) ** 2)
    dY = np.zeros((3, (L + 1) ** 2))
    lib().or_sh_grad(L, _ptr(d), _ptr(Y), _ptr(dY))
    return Y, dY


def phong_rho(l, s):
    return lib().or_phong_rho(int(l), float(s))


def splitmix64(x):
    return int(lib().or_splitmix64(ct.c_uint64(x)))


def jitter(seed, i, r, dim):
    return lib().or_jitter(seed, i, r, dim)


def strata_a(nd):
    return lib().or_strata_a(nd)


def ein(x):
    """Ein(x) = int_0^x (1 - e^{-y}) / y dy (the oracle's own implementation)."""
    return lib().or_ein(float(x))


def num_threads():
    return lib().or_num_threads()


class Oracle:
    """FP64 CPU implementation of the transport, adjoint and gradients of one scene."""

    def __init__(self, sc, alpha_model=ALPHA_GAUSS, use_bvh=True):
        L = lib()
        self.sc = sc
        self.n = int(sc["n"])
        self.L = int(sc["L"])
        self.nc = (self.L + 1) ** 2
        self._keep = [_d(sc[k]) for k in ("p", "tu", "tv", "s", "o", "ad", "k", "as_", "shin")]
        self.h = L.or_scene_new(self.n, self.L, *[_ptr(a) for a in self._keep], int(alpha_model), int(use_bvh))
        if not self.h:
            raise ValueError("oracle: invalid scene")
        L.or_set_directional(self.h, 1 if sc.get("light_dir") else 0)
        self.C = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().or_scene_free(self.h)
                self.h = None
        except Exception:  # pragma: no cover
            pass

    # geometry ------------------------------------------------------------
    @property
    def eps_plane(self):
        return lib().or_eps_plane(self.h)

    def frames(self):
        tu, tv, nn = (np.zeros((self.n, 3)) for _ in range(3))
        lib().or_frames(self.h, _ptr(tu), _ptr(tv), _ptr(nn))
        return tu, tv, nn

    def brdf(self):
        c = np.zeros((self.n, self.L + 1, 3))
        lib().or_brdf(self.h, _ptr(c))
        return c

    def ray_dir(self, i, nd, seed, r):
        d = np.zeros(3)
        lib().or_ray_dir(self.h, i, nd, seed, r, _ptr(d))
        return d

    def trace_ray(self, self_idx, o, d, tmax=np.inf, cap=4096):
        j = np.zeros(cap, np.int32)
        t, a, G = (np.zeros(cap) for _ in range(3))
        o, d = _d(o).reshape(3), _d(d).reshape(3)
        cnt = lib().or_trace_ray(self.h, self_idx, _ptr(o), _ptr(d), float(tmax), cap,
                                 j.ctypes.data_as(_ip), _ptr(t), _ptr(a), _ptr(G))
        cnt = min(cnt, cap)
        return j[:cnt], t[:cnt], a[:cnt], G[:cnt]

    # transport -----------------------------------------------------------
    def transport(self, nd=None, seed=None, light_pos=None, light_I=None):
        nd = self.sc["nd"] if nd is None else nd
        seed = self.sc["seed"] if seed is None else seed
        lp = _d(self.sc["light_pos"] if light_pos is None else light_pos).reshape(-1, 3)
        li = _d(self.sc["light_I"] if light_I is None else light_I).reshape(-1, 3)
        self.nd, self.seed, self.nl = int(nd), int(seed), lp.shape[0]
        self.C = 3 * max(self.nl, 1)
        self._lights = (lp, li)
        lib().or_transport(self.h, self.nd, self.seed, self.nl, _ptr(lp), _ptr(li))
        return self

    def pairs(self, lam=None, light_pos=None, light_I=None):
        """Center-to-center transport (Sec. 8): one segment per pair of surfel centres."""
        lp = _d(self.sc["light_pos"] if light_pos is None else light_pos).reshape(-1, 3)
        li = _d(self.sc["light_I"] if light_I is None else light_I).reshape(-1, 3)
        self.nd, self.seed, self.nl = 0, 0, lp.shape[0]
        self.C = 3 * max(self.nl, 1)
        self._lights = (lp, li)
        self._lam = None if lam is None else _d(lam).reshape(self.n)
        self.pmode = True
        lib().or_pairs(self.h, _ptr(self._lam), self.nl, _ptr(lp), _ptr(li))
        return self

    def pair_list(self):
        L = lib()
        P = L.or_num_pairs(self.h)
        off = np.zeros(self.n + 1, np.int64)
        j = np.zeros(max(P, 1), np.int32)
        V, T = np.zeros(max(P, 1)), np.zeros(max(P, 1))
        L.or_get_pairs(self.h, off.ctypes.data_as(_lp), j.ctypes.data_as(_ip), _ptr(V), _ptr(T))
        return dict(off=off, j=j[:P], V=V[:P], T=T[:P])

    def alpha_area(self, j):
        return lib().or_alpha_area(self.h, int(j))

    def hits(self):
        L = lib()
        H = L.or_num_hits(self.h)
        R = self.n * self.nd
        off = np.zeros(R + 1, np.int64)
        j = np.zeros(max(H, 1), np.int32)
        al, G, a, t = (np.zeros(max(H, 1)) for _ in range(4))
        L.or_get_hits(self.h, off.ctypes.data_as(_lp), j.ctypes.data_as(_ip), _ptr(al), _ptr(G), _ptr(a), _ptr(t))
        return dict(off=off, j=j[:H], alpha=al[:H], G=G[:H], a=a[:H], t=t[:H])

    def num_shadow_hits(self):
        return lib().or_num_shadow_hits(self.h)

    def _shape(self):
        return (self.n, self.nc, self.C)

    def direct(self):
        D = np.zeros(self._shape())
        lib().or_direct(self.h, _ptr(D))
        return D

    def apply_K(self, B):
        B = _d(B).reshape(self._shape())
        out, Q = np.zeros(self._shape()), np.zeros(self._shape())
        lib().or_apply_K(self.h, _ptr(B), _ptr(out), _ptr(Q))
        return out, Q

    def apply_KT(self, V):
        V = _d(V).reshape(self._shape())
        out = np.zeros(self._shape())
        lib().or_apply_KT(self.h, _ptr(V), _ptr(out))
        return out

    def solve(self, E=None, nb=None, iters=False):
        nb = self.sc["nb"] if nb is None else nb
        E = _d(E)
        B = np.zeros(self._shape())
        it = np.zeros((nb + 1,) + self._shape()) if iters else None
        lib().or_solve(self.h, _ptr(E), int(nb), _ptr(B), _ptr(it))
        return (B, it) if iters else B

    def adjoint(self, g, E=None, nb=None):
        nb = self.sc["nb"] if nb is None else nb
        g = _d(g).reshape(self._shape())
        E = _d(E)
        dE = np.zeros((self.n, self.nc, 3))
        dad = np.zeros((self.n, 3))
        dop = np.zeros(self.n)
        dc = np.zeros((self.n, self.L + 1, 3))
        dlam = np.zeros(self.n)
        lib().or_adjoint(self.h, _ptr(E), int(nb), _ptr(g), _ptr(dE), _ptr(dad), _ptr(dop), _ptr(dc), _ptr(dlam))
        out = dict(dE=dE, dad=dad, dop=dop, dc=dc)
        if getattr(self, "pmode", False):
            out["dlam"] = dlam
        return out

    def geometry_grad(self, g, E=None, nb=None):
        """Either transport: dL/dp [N][3], dL/d(s^u, s^v) [N][2] and dL/dtu,
        dL/dtv [N][3] (the frame inputs)."""
        if getattr(self, "C", None) is None:
            raise RuntimeError("geometry gradients need a transport (transport() or pairs())")
        nb = self.sc["nb"] if nb is None else nb
        dp = np.zeros((self.n, 3))
        ds = np.zeros((self.n, 2))
        dtu = np.zeros((self.n, 3))
        dtv = np.zeros((self.n, 3))
        rc = lib().or_geometry_grad(self.h, _ptr(_d(E)), int(nb), _ptr(_d(g).reshape(self._shape())), _ptr(dp), _ptr(ds),
                                    _ptr(dtu), _ptr(dtv))
        if rc != 0:
            raise RuntimeError("geometry gradients need a transport (transport() or pairs())")
        return dict(dp=dp, ds=ds, dtu=dtu, dtv=dtv)

    def mc_solve(self, T, seed=0, E=None, groups=0, S=None):
        """Alg. 1 (Monte-Carlo TD(0) solver with next-event estimation, flat or through
        `groups` K-means groups) on the center-to-center transport: (B [N][nc][C], visits [N])."""
        if not getattr(self, "pmode", False):
            raise RuntimeError("the Monte-Carlo solver runs on the center-to-center transport (pairs())")
        B = np.zeros(self._shape())
        D = np.zeros(self.n)
        S = None if S is None else _d(S).reshape(self._shape())
        lib().or_mc_solve(self.h, _ptr(_d(E)), int(T), ct.c_uint64(seed), int(groups), _ptr(S), _ptr(B), _ptr(D))
        return B, D

    def prog_refine(self, M, E=None):
        """Progressive refinement (shooting) with M shots on the center-to-center transport:
        (Bhat, unshot dB), both [N][nc][C]."""
        if not getattr(self, "pmode", False):
            raise RuntimeError("progressive refinement runs on the center-to-center transport (pairs())")
        Bh, dB = np.zeros(self._shape()), np.zeros(self._shape())
        lib().or_prog_refine(self.h, _ptr(_d(E)), int(M), _ptr(Bh), _ptr(dB))
        return Bh, dB

    def hybrid_solve(self, shots, T, seed=0, E=None, groups=0):
        """Sec. 7's hybrid solver: progressive refinement for `shots` shots, then Alg. 1 on the
        remaining problem (source = the unshot radiance dB): B = Bhat + B^r - dB."""
        Bh, dB = self.prog_refine(shots, E=E)
        Br, _ = self.mc_solve(T, seed=seed, groups=groups, S=dB)
        return Bh + Br - dB

    def mc_groups(self, G):
        """The K-means group of every surfel."""
        out = np.zeros(self.n, np.int32)
        lib().or_mc_groups(self.h, int(G), out.ctypes.data_as(_ip))
        return out

    def mc_weights(self, Bhat, a):
        """The proposal of receiver a under the means Bhat: (unnormalised weights over a's pairs, floor)."""
        Bhat = _d(Bhat).reshape(self._shape())
        off = self.pair_list()["off"]
        w = np.zeros(max(1, int(off[a + 1] - off[a])))
        fl = ct.c_double(0.0)
        n = lib().or_mc_weights(self.h, _ptr(Bhat), int(a), _ptr(w), ct.byref(fl))
        return w[:n], fl.value

    def mc_pick(self, Bhat, seed, t, q, a, E=None, groups=0):
        """One next-event estimate: (picked pair index within a's pairs, its probability, delta)."""
        Bhat = _d(Bhat).reshape(self._shape())
        p = ct.c_double(0.0)
        delta = np.zeros((self.nc, self.C))
        k = lib().or_mc_pick(self.h, _ptr(_d(E)), _ptr(Bhat), ct.c_uint64(seed), int(t), int(q), int(a), int(groups),
                             ct.byref(p), _ptr(delta))
        return int(k), p.value, delta

    def render(self, B, cam, W, H, fov):
        """Eq. L_I for a pinhole camera cam = (o, forward, up): image [H][W][C] of the radiance B."""
        if getattr(self, "C", None) is None:
            raise RuntimeError("render needs a transport (its column count)")
        img = np.zeros((H, W, self.C))
        lib().or_render(self.h, _ptr(_d(B).reshape(self._shape())), _ptr(_d(np.asarray(cam, float).reshape(9))),
                        int(W), int(H), float(fov), _ptr(img))
        return img

    def render_adjoint(self, dimg, cam, W, H, fov):
        """The transpose of render: dL/dB [N][nc][C] from dL/dimg [H][W][C]."""
        if getattr(self, "C", None) is None:
            raise RuntimeError("render needs a transport (its column count)")
        dB = np.zeros(self._shape())
        lib().or_render_adjoint(self.h, _ptr(_d(dimg).reshape(H, W, self.C)),
                                _ptr(_d(np.asarray(cam, float).reshape(9))), int(W), int(H), float(fov), _ptr(dB))
        return dB

    def brdf_grad_closed_form(self, g, E=None, nb=None):
        nb = self.sc["nb"] if nb is None else nb
        dc = np.zeros((self.n, self.L + 1, 3))
        lib().or_brdf_grad_closed_form(self.h, _ptr(_d(E)), int(nb), _ptr(_d(g).reshape(self._shape())), _ptr(dc))
        return dc

    def dense_K(self, col):
        m = self.n * self.nc
        K = np.zeros((m, m))
        lib().or_dense_K(self.h, int(col), _ptr(K))
        return K

    def sample_direct(self, recv, light_pos=None, light_I=None):
        lp = _d(self.sc["light_pos"] if light_pos is None else light_pos).reshape(-1, 3)
        li = _d(self.sc["light_I"] if light_I is None else light_I).reshape(-1, 3)
        recv = np.ascontiguousarray(recv, dtype=np.int32)
        out = np.zeros((len(recv), self.nc, 3 * lp.shape[0]))
        lib().or_sample_direct(self.h, lp.shape[0], _ptr(lp), _ptr(li), len(recv), recv.ctypes.data_as(_ip), _ptr(out))
        return out

    def sample_bounce1(self, recv, E=None, nd=None, seed=None, light_pos=None, light_I=None):
        nd = self.sc["nd"] if nd is None else nd
        seed = self.sc["seed"] if seed is None else seed
        lp = _d(self.sc["light_pos"] if light_pos is None else light_pos).reshape(-1, 3)
        li = _d(self.sc["light_I"] if light_I is None else light_I).reshape(-1, 3)
        recv = np.ascontiguousarray(recv, dtype=np.int32)
        out = np.zeros((len(recv), self.nc, 3 * lp.shape[0]))
        lib().or_sample_bounce1(self.h, int(nd), int(seed), lp.shape[0], _ptr(lp), _ptr(li), _ptr(_d(E)),
                                len(recv), recv.ctypes.data_as(_ip), _ptr(out))
        return out
