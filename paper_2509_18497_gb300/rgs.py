"""Python binding of librgs (include/rgs.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does nothing but
check tensor placement/shape/dtype, pass raw device pointers and the current CUDA
stream, and turn a non-zero rgs_status into an exception.  All computation runs in
the CUDA kernels of librgs.so; there is no CPU or PyTorch fallback: if the library
is missing, importing the binding's entry points raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librgs.so")

RGS_MAX_SH_DEGREE = 3
RGS_MAX_BOUNCES = 64
RGS_ALPHA_GAUSS, RGS_ALPHA_DISC, RGS_ALPHA_GFSGS = 0, 1, 2
RGS_FP32, RGS_BF16_FP32ACC, RGS_BF16_FP32ACC_RESCORR = 0, 1, 2

STATUS = {0: "RGS_OK", 1: "RGS_ERR_ARG", 2: "RGS_ERR_CUDA", 3: "RGS_ERR_OOM", 4: "RGS_ERR_CAPACITY",
          5: "RGS_ERR_NONFINITE", 6: "RGS_ERR_TIMEOUT", 7: "RGS_ERR_STATE"}
(RGS_OK, RGS_ERR_ARG, RGS_ERR_CUDA, RGS_ERR_OOM, RGS_ERR_CAPACITY, RGS_ERR_NONFINITE, RGS_ERR_TIMEOUT,
 RGS_ERR_STATE) = range(8)

# names exported by librgs.so, as declared in include/rgs.h
EXPORTS = ("rgs_build_scene", "rgs_trace_transport", "rgs_solve", "rgs_adjoint", "rgs_get_iterate",
           "rgs_transport_info_get", "rgs_destroy_transport", "rgs_destroy_scene", "rgs_profile_enable",
           "rgs_profile_reset", "rgs_profile_report", "rgs_launch_count", "rgs_status_string",
           "rgs_last_error", "rgs_abi_version", "rgs_residual_norm_noalloc", "rgs_solve_batched",
           "rgs_set_checkpointing", "rgs_trim_workspace", "rgs_set_memory_budget", "rgs_set_tensor_cores",
           "rgs_set_wait_limit", "rgs_contraction_info", "rgs_render", "rgs_render_adjoint",
           "rgs_mc_solve", "rgs_mc_estimate", "rgs_mc_groups", "rgs_prog_refine", "rgs_batch_last_plan",
           "rgs_trace_pairs",
           "rgs_adjoint_pairs", "rgs_adjoint_pairs_geometry", "rgs_adjoint_geometry")


class RgsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class rgs_surfels(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("sh_degree", ct.c_int32)] + [
        (k, ct.c_void_p) for k in ("p", "tu", "tv", "s", "o", "ad", "k", "as_", "shin")]


class rgs_build_opts(ct.Structure):
    _fields_ = [("alpha_model", ct.c_int32), ("check_finite", ct.c_int32)]


class rgs_lights(ct.Structure):
    _fields_ = [("n_lights", ct.c_int32), ("directional", ct.c_int32), ("pos", ct.c_void_p), ("intensity", ct.c_void_p)]


class rgs_trace_opts(ct.Structure):
    _fields_ = [("nd", ct.c_int32), ("reserved0", ct.c_int32), ("seed", ct.c_uint64), ("hit_capacity", ct.c_int64)]


class rgs_pair_opts(ct.Structure):
    _fields_ = [("lambda_", ct.c_void_p)]


class rgs_solve_stats(ct.Structure):
    _fields_ = [("n_bounces", ct.c_int32), ("n_cols", ct.c_int32),
                ("residual_norm", ct.c_double * RGS_MAX_BOUNCES),
                ("n_hits", ct.c_int64), ("n_hit_slots", ct.c_int64), ("n_full_rays", ct.c_int64)]


class rgs_batch_opts(ct.Structure):
    _fields_ = [("precision", ct.c_int32), ("use_graph", ct.c_int32), ("autotune", ct.c_int32),
                ("spin_limit", ct.c_int32)]


class rgs_kernel_time(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int64), ("total_ms", ct.c_double)]


class rgs_transport_info(ct.Structure):
    _fields_ = [(k, ct.c_int32) for k in ("n", "sh_degree", "nc", "n_cols", "nd", "n_lights")] + [
        (k, ct.c_int64) for k in ("n_hits", "n_hit_slots", "n_full_rays", "device_bytes")]


_lib = None


def load(path=LIB_PATH):
    """Load librgs.so (built in-tree by build.py).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librgs.so not found at {path}: run paper_2509_18497_gb300/build.py "
                           "(the CUDA library is required; there is no fallback)")
    L = ct.CDLL(path)
    vp = ct.c_void_p
    L.rgs_build_scene.argtypes = [ct.POINTER(rgs_surfels), ct.POINTER(rgs_build_opts), vp, ct.POINTER(vp)]
    L.rgs_trace_transport.argtypes = [vp, ct.POINTER(rgs_lights), ct.POINTER(rgs_trace_opts), vp, ct.POINTER(vp)]
    L.rgs_solve.argtypes = [vp, vp, ct.c_int32, ct.c_int32, vp, ct.POINTER(rgs_solve_stats), vp]
    L.rgs_adjoint.argtypes = [vp, vp, vp, vp, vp, vp]
    L.rgs_get_iterate.argtypes = [vp, ct.c_int32, vp, vp]
    L.rgs_transport_info_get.argtypes = [vp, ct.POINTER(rgs_transport_info)]
    L.rgs_destroy_transport.argtypes = [vp]
    L.rgs_destroy_transport.restype = None
    L.rgs_destroy_scene.argtypes = [vp]
    L.rgs_destroy_scene.restype = None
    L.rgs_status_string.restype = ct.c_char_p
    L.rgs_status_string.argtypes = [ct.c_int]
    L.rgs_last_error.restype = ct.c_char_p
    L.rgs_abi_version.restype = ct.c_int32
    L.rgs_profile_enable.argtypes = [ct.c_int32]
    L.rgs_profile_enable.restype = None
    L.rgs_profile_reset.argtypes = []
    L.rgs_profile_reset.restype = None
    L.rgs_profile_report.argtypes = [ct.POINTER(rgs_kernel_time), ct.c_int32]
    L.rgs_profile_report.restype = ct.c_int32
    L.rgs_launch_count.restype = ct.c_int64
    L.rgs_residual_norm_noalloc.argtypes = [vp, vp, ct.c_int64, vp, vp]
    L.rgs_solve_batched.argtypes = [ct.POINTER(vp), ct.c_int32, ct.POINTER(vp), ct.POINTER(ct.c_int32),
                                    ct.POINTER(rgs_batch_opts), ct.POINTER(vp), ct.POINTER(ct.c_double), vp]
    L.rgs_solve_batched.restype = ct.c_int
    L.rgs_residual_norm_noalloc.restype = ct.c_int
    L.rgs_set_checkpointing.argtypes = [vp, ct.c_int32]
    L.rgs_set_checkpointing.restype = ct.c_int
    L.rgs_trace_pairs.argtypes = [vp, ct.POINTER(rgs_lights), ct.POINTER(rgs_pair_opts), vp, ct.POINTER(vp)]
    L.rgs_trace_pairs.restype = ct.c_int
    L.rgs_adjoint_pairs.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.rgs_adjoint_pairs.restype = ct.c_int
    L.rgs_adjoint_pairs_geometry.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rgs_adjoint_pairs_geometry.restype = ct.c_int
    L.rgs_adjoint_geometry.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rgs_adjoint_geometry.restype = ct.c_int
    L.rgs_set_memory_budget.argtypes = [vp, ct.c_int64]
    L.rgs_set_memory_budget.restype = ct.c_int
    L.rgs_set_tensor_cores.argtypes = [vp, ct.c_int32]
    L.rgs_set_tensor_cores.restype = ct.c_int
    L.rgs_set_wait_limit.argtypes = [vp, ct.c_int64]
    L.rgs_set_wait_limit.restype = ct.c_int
    L.rgs_contraction_info.argtypes = [vp, ct.POINTER(ct.c_int64), ct.c_int32]
    L.rgs_contraction_info.restype = ct.c_int
    L.rgs_render.argtypes = [vp, vp, ct.POINTER(ct.c_float), ct.c_int32, ct.c_int32, ct.c_float, vp, vp]
    L.rgs_render.restype = ct.c_int
    L.rgs_render_adjoint.argtypes = [vp, vp, ct.POINTER(ct.c_float), ct.c_int32, ct.c_int32, ct.c_float, vp, vp]
    L.rgs_render_adjoint.restype = ct.c_int
    L.rgs_mc_solve.argtypes = [vp, vp, vp, ct.c_int32, ct.c_uint64, ct.c_int32, vp, vp, vp]
    L.rgs_mc_solve.restype = ct.c_int
    L.rgs_mc_estimate.argtypes = [vp, vp, vp, ct.c_uint64, ct.c_int32, ct.c_int32, ct.c_int32, vp, vp, vp, vp, vp]
    L.rgs_mc_estimate.restype = ct.c_int
    L.rgs_prog_refine.argtypes = [vp, vp, ct.c_int32, vp, vp, vp]
    L.rgs_prog_refine.restype = ct.c_int
    L.rgs_mc_groups.argtypes = [vp, ct.c_int32, vp, vp]
    L.rgs_mc_groups.restype = ct.c_int
    L.rgs_batch_last_plan.argtypes = [ct.POINTER(ct.c_int32), ct.c_int32]
    L.rgs_batch_last_plan.restype = ct.c_int32
    L.rgs_trim_workspace.argtypes = []
    L.rgs_trim_workspace.restype = ct.c_int
    for fn in ("rgs_build_scene", "rgs_trace_transport", "rgs_solve", "rgs_adjoint", "rgs_get_iterate",
               "rgs_transport_info_get"):
        getattr(L, fn).restype = ct.c_int
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise RgsError(status, load().rgs_last_error().decode(errors="replace"))


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ct.c_void_p(s.cuda_stream)


def _dev(t, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name}: expected a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
    return ct.c_void_p(t.data_ptr())


class Scene:
    """Owner of an rgs_scene handle (and references to the tensors it was built from)."""

    def __init__(self):
        self.h = ct.c_void_p(None)
        self.n = 0
        self.L = 0
        self._keep = None

    def __del__(self):
        if self.h and _lib is not None:
            _lib.rgs_destroy_scene(self.h)
            self.h = ct.c_void_p(None)


class Transport:
    """Owner of an rgs_transport handle."""

    def __init__(self, scene):
        self.h = ct.c_void_p(None)
        self.scene = scene
        self.C = 3
        self.nb = -1
        self._keep = None

    @property
    def n(self):
        return self.scene.n

    @property
    def nc(self):
        return (self.scene.L + 1) ** 2

    def __del__(self):
        if self.h and _lib is not None:
            _lib.rgs_destroy_transport(self.h)
            self.h = ct.c_void_p(None)


def rgs_build_scene(p, tu, tv, s, o, ad, k, as_, shin, sh_degree, alpha_model=RGS_ALPHA_GAUSS,
                    check_finite=False, stream=None, scene=None):
    """rgs_build_scene: surfel arrays are CUDA float32 tensors in the caller's order."""
    L = load()
    n = int(p.shape[0])
    shapes = dict(p=(n, 3), tu=(n, 3), tv=(n, 3), s=(n, 2), o=(n,), ad=(n, 3), k=(n,), as_=(n, 3), shin=(n,))
    arrs = dict(p=p, tu=tu, tv=tv, s=s, o=o, ad=ad, k=k, as_=as_, shin=shin)
    sf = rgs_surfels(n, int(sh_degree), *[_dev(arrs[key], shapes[key], key) for key in shapes])
    opts = rgs_build_opts(int(alpha_model), int(bool(check_finite)))
    sc = scene if scene is not None else Scene()
    h = ct.c_void_p(sc.h.value)
    _check(L.rgs_build_scene(ct.byref(sf), ct.byref(opts), _stream(stream), ct.byref(h)))
    sc.h = h
    sc.n = n
    sc.L = int(sh_degree)
    sc._keep = arrs
    return sc


def _lights(light_pos, light_I, directional):
    nl = int(light_pos.shape[0])
    return nl, rgs_lights(nl, 1 if directional else 0, _dev(light_pos, (nl, 3), "light_pos") if nl else None,
                          _dev(light_I, (nl, 3), "light_I") if nl else None)


def rgs_trace_transport(scene, light_pos, light_I, nd, seed, hit_capacity=0, stream=None, transport=None,
                        directional=False):
    """rgs_trace_transport: light_pos / light_I are CUDA float32 [NL,3] (NL may be 0); directional:
    light_pos holds directions towards distant lights (no 1/r^2)."""
    L = load()
    nl, lt = _lights(light_pos, light_I, directional)
    opts = rgs_trace_opts(int(nd), 0, int(seed), int(hit_capacity))
    tr = transport if transport is not None else Transport(scene)
    tr.scene = scene
    h = ct.c_void_p(tr.h.value)
    _check(L.rgs_trace_transport(scene.h, ct.byref(lt), ct.byref(opts), _stream(stream), ct.byref(h)))
    tr.h = h
    tr.C = 3 * max(nl, 1)
    tr.nb = -1
    return tr


def rgs_trace_pairs(scene, light_pos, light_I, lam=None, stream=None, transport=None, directional=False):
    """rgs_trace_pairs (center-to-center transport): lam is a CUDA float32 [N] or None (1)."""
    L = load()
    nl, lt = _lights(light_pos, light_I, directional)
    opts = rgs_pair_opts(_dev(lam, (scene.n,), "lambda").value if lam is not None else None)
    tr = transport if transport is not None else Transport(scene)
    tr.scene = scene
    h = ct.c_void_p(tr.h.value)
    _check(L.rgs_trace_pairs(scene.h, ct.byref(lt), ct.byref(opts), _stream(stream), ct.byref(h)))
    tr.h = h
    tr.C = 3 * max(nl, 1)
    tr.nb = -1
    tr.pairs = True
    return tr


def rgs_adjoint_pairs(transport, dL_dB, stream=None):
    """rgs_adjoint_pairs: returns (dL/dE, dL/da^d, dL/do, dL/dlambda)."""
    L = load()
    n, nc, C = transport.n, transport.nc, transport.C
    dE = torch.empty((n, nc, 3), device="cuda", dtype=torch.float32)
    dad = torch.empty((n, 3), device="cuda", dtype=torch.float32)
    dop = torch.empty((n,), device="cuda", dtype=torch.float32)
    dlam = torch.empty((n,), device="cuda", dtype=torch.float32)
    _check(L.rgs_adjoint_pairs(transport.h, _dev(dL_dB, (n, nc, C), "dL_dB"), _dev(dE, (n, nc, 3), "dL_dE"),
                               _dev(dad, (n, 3), "dL_dalbedo"), _dev(dop, (n,), "dL_dopacity"),
                               _dev(dlam, (n,), "dL_dlambda"), _stream(stream)))
    return dE, dad, dop, dlam


def rgs_adjoint_pairs_geometry(transport, dL_dB, stream=None):
    """rgs_adjoint_pairs_geometry: returns (dL/dE, dL/da^d, dL/do, dL/dlambda, dL/dp, dL/ds, dL/dtu, dL/dtv)."""
    L = load()
    n, nc, C = transport.n, transport.nc, transport.C
    dE = torch.empty((n, nc, 3), device="cuda", dtype=torch.float32)
    dad = torch.empty((n, 3), device="cuda", dtype=torch.float32)
    dop = torch.empty((n,), device="cuda", dtype=torch.float32)
    dlam = torch.empty((n,), device="cuda", dtype=torch.float32)
    dp = torch.empty((n, 3), device="cuda", dtype=torch.float32)
    ds = torch.empty((n, 2), device="cuda", dtype=torch.float32)
    dtu = torch.empty((n, 3), device="cuda", dtype=torch.float32)
    dtv = torch.empty((n, 3), device="cuda", dtype=torch.float32)
    _check(L.rgs_adjoint_pairs_geometry(transport.h, _dev(dL_dB, (n, nc, C), "dL_dB"), _dev(dE, (n, nc, 3), "dL_dE"),
                                        _dev(dad, (n, 3), "dL_dalbedo"), _dev(dop, (n,), "dL_dopacity"),
                                        _dev(dlam, (n,), "dL_dlambda"), _dev(dp, (n, 3), "dL_dp"),
                                        _dev(ds, (n, 2), "dL_ds"), _dev(dtu, (n, 3), "dL_dtu"),
                                        _dev(dtv, (n, 3), "dL_dtv"), _stream(stream)))
    return dE, dad, dop, dlam, dp, ds, dtu, dtv


def rgs_adjoint_geometry(transport, dL_dB, stream=None):
    """rgs_adjoint_geometry: returns (dL/dE, dL/da^d, dL/do, dL/dp, dL/ds, dL/dtu, dL/dtv)."""
    L = load()
    n, nc, C = transport.n, transport.nc, transport.C
    f = lambda *shape: torch.empty(shape, device="cuda", dtype=torch.float32)
    dE, dad, dop, dp, ds, dtu, dtv = f(n, nc, 3), f(n, 3), f(n), f(n, 3), f(n, 2), f(n, 3), f(n, 3)
    _check(L.rgs_adjoint_geometry(transport.h, _dev(dL_dB, (n, nc, C), "dL_dB"), _dev(dE, (n, nc, 3), "dL_dE"),
                                  _dev(dad, (n, 3), "dL_dalbedo"), _dev(dop, (n,), "dL_dopacity"),
                                  _dev(dp, (n, 3), "dL_dp"), _dev(ds, (n, 2), "dL_ds"), _dev(dtu, (n, 3), "dL_dtu"),
                                  _dev(dtv, (n, 3), "dL_dtv"), _stream(stream)))
    return dE, dad, dop, dp, ds, dtu, dtv


def rgs_solve(transport, E, n_bounces, B_out=None, stats=False, precision=RGS_FP32, stream=None):
    """rgs_solve: E is CUDA float32 [N,nc,3] or None; returns (B_out [N,nc,C], stats or None)."""
    L = load()
    n, nc, C = transport.n, transport.nc, transport.C
    if B_out is None:
        B_out = torch.empty((n, nc, C), device="cuda", dtype=torch.float32)
    st = rgs_solve_stats() if stats else None
    _check(L.rgs_solve(transport.h, _dev(E, (n, nc, 3), "E") if E is not None else None, int(n_bounces),
                       int(precision), _dev(B_out, (n, nc, C), "B_out"), ct.byref(st) if st is not None else None,
                       _stream(stream)))
    transport.nb = int(n_bounces)
    if st is None:
        return B_out, None
    stats_d = dict(n_bounces=st.n_bounces, n_cols=st.n_cols,
                   residual_norm=[st.residual_norm[b] for b in range(st.n_bounces)],
                   n_hits=st.n_hits, n_hit_slots=st.n_hit_slots, n_full_rays=st.n_full_rays)
    return B_out, stats_d


def rgs_adjoint(transport, dL_dB, dL_dE=None, dL_dalbedo=None, dL_dopacity=None, want=("E", "albedo", "opacity"),
                stream=None):
    """rgs_adjoint: returns (dL/dE [N,nc,3], dL/da^d [N,3], dL/do [N]); entries not in `want` are None."""
    L = load()
    n, nc, C = transport.n, transport.nc, transport.C
    if dL_dE is None and "E" in want:
        dL_dE = torch.empty((n, nc, 3), device="cuda", dtype=torch.float32)
    if dL_dalbedo is None and "albedo" in want:
        dL_dalbedo = torch.empty((n, 3), device="cuda", dtype=torch.float32)
    if dL_dopacity is None and "opacity" in want:
        dL_dopacity = torch.empty((n,), device="cuda", dtype=torch.float32)
    _check(L.rgs_adjoint(transport.h, _dev(dL_dB, (n, nc, C), "dL_dB"),
                         _dev(dL_dE, (n, nc, 3), "dL_dE") if dL_dE is not None else None,
                         _dev(dL_dalbedo, (n, 3), "dL_dalbedo") if dL_dalbedo is not None else None,
                         _dev(dL_dopacity, (n,), "dL_dopacity") if dL_dopacity is not None else None,
                         _stream(stream)))
    return dL_dE, dL_dalbedo, dL_dopacity


def rgs_get_iterate(transport, b, out=None, stream=None):
    L = load()
    n, nc, C = transport.n, transport.nc, transport.C
    if out is None:
        out = torch.empty((n, nc, C), device="cuda", dtype=torch.float32)
    _check(L.rgs_get_iterate(transport.h, int(b), _dev(out, (n, nc, C), "out"), _stream(stream)))
    return out


def rgs_set_checkpointing(transport, stride):
    """0: keep every iterate; s >= 1: keep B^(0), B^(s), ... and recompute in the adjoint;
    -1: automatic (checkpoint only when the full storage does not fit)."""
    _check(load().rgs_set_checkpointing(transport.h, int(stride)))


def rgs_set_memory_budget(transport, nbytes):
    """Bytes the transport may hold with its pooled scratch (0: no budget); steers the
    automatic checkpoint stride and the number of transposed-index parts of the adjoint."""
    _check(load().rgs_set_memory_budget(transport.h, int(nbytes)))


def rgs_set_tensor_cores(transport, mode):
    """Contraction of the batched modes: -1 automatic (tensor cores from 96 columns), 0 the
    row-gather kernels, 1 the tensor-core form wherever it applies (the adjoint's opacity
    gather as sampled products on the tensor cores in both), 2 as 1 with the opacity gather
    as per-(tile, receiver) products, 3 as 1 with the opacity gather as row gathers."""
    _check(load().rgs_set_tensor_cores(transport.h, int(mode)))


def rgs_set_wait_limit(transport, ns):
    """Limit (ns) of every wait in the tensor-core contraction's pipeline (0: default 4 s)."""
    _check(load().rgs_set_wait_limit(transport.h, int(ns)))


def rgs_contraction_info(transport):
    """Pair-tile sizes of the tensor-core contraction: dict of receiver tiles, groups, pairs,
    hits, source tiles and source-tile groups (zeros before the structures are built)."""
    out = (ct.c_int64 * 6)()
    _check(load().rgs_contraction_info(transport.h, out, 6))
    keys = ("tiles", "groups", "pairs", "hits", "src_tiles", "src_groups")
    return {k: int(v) for k, v in zip(keys, out)}


def _cam9(cam):
    c = [float(v) for v in torch.as_tensor(cam, dtype=torch.float64).reshape(-1).tolist()]
    if len(c) != 9:
        raise ValueError("cam must hold 9 numbers: origin, forward, up")
    return (ct.c_float * 9)(*c)


def rgs_render(transport, B, cam, W, H, fov, img_out=None, stream=None):
    """Image [H][W][C] of the radiance B [N][nc][C] (device float32) seen by a pinhole camera
    cam = (origin, forward, up) with vertical field of view fov (Eq. L_I per pixel ray)."""
    n, nc, C = transport.n, transport.nc, transport.C
    pB = _dev(B, (n, nc, C), "B")
    img = torch.empty((H, W, C), dtype=torch.float32, device=B.device) if img_out is None else img_out
    pimg = _dev(img, (H, W, C), "img_out")
    with torch.cuda.device(B.device):
        _check(load().rgs_render(transport.h, pB, _cam9(cam), int(W), int(H), float(fov), pimg, _stream(stream)))
    return img


def rgs_render_adjoint(transport, dimg, cam, W, H, fov, dB_out=None, stream=None):
    """The transpose of rgs_render: dL/dB [N][nc][C] from dL/dimg [H][W][C] (device float32)."""
    n, nc, C = transport.n, transport.nc, transport.C
    pd = _dev(dimg, (H, W, C), "dimg")
    dB = torch.empty((n, nc, C), dtype=torch.float32, device=dimg.device) if dB_out is None else dB_out
    pdB = _dev(dB, (n, nc, C), "dB_out")
    with torch.cuda.device(dimg.device):
        _check(load().rgs_render_adjoint(transport.h, pd, _cam9(cam), int(W), int(H), float(fov), pdB,
                                         _stream(stream)))
    return dB


def _opt_dev(t, shape, name):
    return ct.c_void_p(None) if t is None else _dev(t, shape, name)


def rgs_mc_solve(transport, steps, seed=0, E=None, S=None, groups=0, B_out=None, visits=True, stream=None):
    """Alg. 1's Monte-Carlo TD(0) solver on a center-to-center transport: (B [N][nc][C],
    visits [N] or None), both device float32."""
    n, nc, C = transport.n, transport.nc, transport.C
    dev = torch.device("cuda", torch.cuda.current_device())
    B = torch.empty((n, nc, C), dtype=torch.float32, device=dev) if B_out is None else B_out
    pB = _dev(B, (n, nc, C), "B_out")
    V = torch.empty(n, dtype=torch.float32, device=B.device) if visits else None
    with torch.cuda.device(B.device):
        _check(load().rgs_mc_solve(transport.h, _opt_dev(E, (n, nc, 3), "E"), _opt_dev(S, (n, nc, C), "S"),
                                   int(steps), ct.c_uint64(seed), int(groups), pB,
                                   _opt_dev(V, (n,), "visits"), _stream(stream)))
    return B, V


def rgs_mc_estimate(transport, Bhat, seed, step, recv=None, n_draws=None, E=None, groups=0, stream=None):
    """One step's next-event estimates for the means Bhat: (pick int64 [q], p float64 [q],
    delta float32 [q][nc][C]); receivers recv (int32 device, caller indices) or 0..n_draws-1."""
    n, nc, C = transport.n, transport.nc, transport.C
    pBh = _dev(Bhat, (n, nc, C), "Bhat")
    dev = Bhat.device
    if recv is not None:
        if not (isinstance(recv, torch.Tensor) and recv.is_cuda and recv.dtype == torch.int32 and recv.is_contiguous()):
            raise TypeError("recv: expected a contiguous int32 CUDA tensor")
        q = recv.numel()
    else:
        q = n if n_draws is None else int(n_draws)
    pick = torch.empty(q, dtype=torch.int64, device=dev)
    p = torch.empty(q, dtype=torch.float64, device=dev)
    delta = torch.empty((q, nc, C), dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        _check(load().rgs_mc_estimate(transport.h, _opt_dev(E, (n, nc, 3), "E"), pBh, ct.c_uint64(seed), int(step),
                                      int(groups), int(q),
                                      ct.c_void_p(recv.data_ptr()) if recv is not None else ct.c_void_p(None),
                                      ct.c_void_p(pick.data_ptr()), ct.c_void_p(p.data_ptr()),
                                      ct.c_void_p(delta.data_ptr()), _stream(stream)))
    return pick, p, delta


def rgs_prog_refine(transport, shots, E=None, stream=None):
    """Progressive refinement with `shots` shots: (Bhat, unshot dB), device float32 [N][nc][C]."""
    n, nc, C = transport.n, transport.nc, transport.C
    dev = torch.device("cuda", torch.cuda.current_device())
    Bh = torch.empty((n, nc, C), dtype=torch.float32, device=dev)
    dB = torch.empty((n, nc, C), dtype=torch.float32, device=dev)
    _check(load().rgs_prog_refine(transport.h, _opt_dev(E, (n, nc, 3), "E"), int(shots), _dev(Bh, (n, nc, C), "Bhat"),
                                  _dev(dB, (n, nc, C), "dB"), _stream(stream)))
    return Bh, dB


def rgs_mc_groups(transport, groups, stream=None):
    """The K-means group (int32, caller order) of every surfel, as the grouped proposal uses them."""
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.empty(transport.n, dtype=torch.int32, device=dev)
    _check(load().rgs_mc_groups(transport.h, int(groups), ct.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def rgs_batch_last_plan():
    """The plan of the last rgs_solve_batched call: dict(blocks, blocks_per_sm, autotuned,
    buckets=[dict(nc, C, rays, policy_bf16, policy_fp32, items_bf16, items_fp32)]), or None."""
    L = load()
    m = L.rgs_batch_last_plan(None, 0)
    if m < 0:
        return None
    buf = (ct.c_int32 * m)()
    L.rgs_batch_last_plan(buf, m)
    v = list(buf)
    keys = ("nc", "C", "rays", "policy_bf16", "policy_fp32", "items_bf16", "items_fp32")
    buckets = [dict(zip(keys, v[4 + 7 * k: 11 + 7 * k])) for k in range(v[3])]
    return dict(blocks=v[0], blocks_per_sm=v[1], autotuned=bool(v[2]), buckets=buckets)


def rgs_trim_workspace():
    """Return the unused part of the library's workspace pool to the device."""
    _check(load().rgs_trim_workspace())


def rgs_transport_info_get(transport):
    L = load()
    info = rgs_transport_info()
    _check(L.rgs_transport_info_get(transport.h, ct.byref(info)))
    return {k: getattr(info, k) for k, _ in rgs_transport_info._fields_}


def rgs_abi_version():
    return int(load().rgs_abi_version())


def rgs_profile_enable(on=True):
    load().rgs_profile_enable(1 if on else 0)


def rgs_profile_reset():
    load().rgs_profile_reset()


def rgs_profile_report():
    """{kernel name: (launches, total device ms)} for the launches since the last reset."""
    L = load()
    buf = (rgs_kernel_time * 64)()
    m = L.rgs_profile_report(buf, 64)
    if m < 0:
        raise RgsError(2, L.rgs_last_error().decode(errors="replace"))
    return {buf[q].name.decode(): (int(buf[q].launches), float(buf[q].total_ms)) for q in range(min(m, 64))}


def rgs_launch_count():
    return int(load().rgs_launch_count())


def rgs_residual_norm_noalloc(x, y, norm_out=None, stream=None):
    """rgs_residual_norm_noalloc: FP64 ||x - y||_2 of two equal-size float32 CUDA tensors into a
    float64 CUDA scalar, using the library's static scratch (no device allocation inside)."""
    L = load()
    n = x.numel()
    if norm_out is None:
        norm_out = torch.empty((), device=x.device, dtype=torch.float64)
    if not (norm_out.is_cuda and norm_out.dtype == torch.float64 and norm_out.numel() == 1):
        raise TypeError("norm_out: expected a float64 CUDA scalar")
    for name, t in (("y", y), ("norm_out", norm_out)):
        if t.device != x.device:
            raise ValueError(f"{name} is on {t.device}, x on {x.device}: all three must share one device")
    # the C entry launches on the current device: make it x's
    with torch.cuda.device(x.device):
        _check(L.rgs_residual_norm_noalloc(_dev(x, tuple(x.shape), "x"), _dev(y, tuple(x.shape), "y"), int(n),
                                           ct.c_void_p(norm_out.data_ptr()), _stream(stream)))
    return norm_out


def rgs_solve_batched(transports, E_list, n_bounces, precision=RGS_FP32, use_graph=True, autotune=True,
                      spin_limit=0, B_outs=None, norms=False, stream=None):
    """rgs_solve_batched over a list of traced Transport objects; returns (list of B tensors, norms or None)."""
    m = len(transports)
    for name, seq in (("n_bounces", n_bounces), ("E_list", E_list), ("B_outs", B_outs)):
        if seq is not None and len(seq) != m:
            raise ValueError(f"{name}: {len(seq)} entries for {m} transports")
    L = load()
    hs = (ct.c_void_p * m)(*[t.h.value for t in transports])
    Es = None
    if E_list is not None:
        Es = (ct.c_void_p * m)(*[(_dev(E, (t.n, t.nc, 3), "E").value if E is not None else None)
                                 for t, E in zip(transports, E_list)])
    nbs = (ct.c_int32 * m)(*[int(b) for b in n_bounces])
    if B_outs is None:
        B_outs = [torch.empty((t.n, t.nc, t.C), device="cuda", dtype=torch.float32) for t in transports]
    Bs = (ct.c_void_p * m)(*[_dev(B, (t.n, t.nc, t.C), "B_out").value for t, B in zip(transports, B_outs)])
    nrm = (ct.c_double * (m * RGS_MAX_BOUNCES))() if norms else None
    opts = rgs_batch_opts(int(precision), int(bool(use_graph)), int(bool(autotune)), int(spin_limit))
    _check(L.rgs_solve_batched(hs, m, Es, nbs, ct.byref(opts), Bs, nrm, _stream(stream)))
    for t, b in zip(transports, n_bounces):
        t.nb = int(b)
    out_norms = None
    if norms:
        out_norms = [[nrm[s * RGS_MAX_BOUNCES + b] for b in range(int(n_bounces[s]))] for s in range(m)]
    return B_outs, out_norms
