"""Convenience layer over the C-ABI binding: upload a scene, run build -> trace -> solve
-> adjoint, and torch.autograd.Functions differentiable in emission, diffuse albedo and
opacity (radiosity) and also in the surfels' centres, scales and frames
(radiosity_geometry).  Every numerical step is a librgs.so kernel; this module only moves
tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rgs

SURFEL_KEYS = ("p", "tu", "tv", "s", "o", "ad", "k", "as_", "shin")


def upload(sc, device="cuda"):
    """numpy scene dict (scenes.py layout) -> dict of contiguous float32 CUDA tensors."""
    out = {k: torch.as_tensor(np.ascontiguousarray(sc[k], dtype=np.float32), device=device) for k in SURFEL_KEYS}
    out["light_pos"] = torch.as_tensor(np.ascontiguousarray(sc["light_pos"], np.float32).reshape(-1, 3), device=device)
    out["light_I"] = torch.as_tensor(np.ascontiguousarray(sc["light_I"], np.float32).reshape(-1, 3), device=device)
    out["E"] = None if sc.get("E") is None else torch.as_tensor(np.ascontiguousarray(sc["E"], np.float32), device=device)
    out["lam"] = None if sc.get("lam") is None else torch.as_tensor(np.ascontiguousarray(sc["lam"], np.float32),
                                                                     device=device)
    for key in ("L", "nd", "nb", "seed", "n"):
        out[key] = int(sc[key])
    out["light_dir"] = bool(sc.get("light_dir", False))
    return out


class Pipeline:
    """Reusable handles for one scene shape: build, trace, solve and adjoint in sequence.
    Handles and their buffers are reused across calls; the adjoint's scratch comes from the
    library's stream-ordered pool, which keeps it reserved, so steady-state steps make no
    cudaMalloc inside the library."""

    def __init__(self, alpha_model=rgs.RGS_ALPHA_GAUSS, precision=rgs.RGS_FP32, checkpoint=0, mem_budget=0,
                 pairs=False, tensor_cores=-1):
        self.pairs = pairs  # center-to-center transport (Sec. 8) instead of hemisphere rays
        self.tensor_cores = tensor_cores  # contraction of the batched modes (rgs_set_tensor_cores)
        self.alpha_model = alpha_model
        self.precision = precision
        self.checkpoint = checkpoint  # iterate checkpoint stride (0 all kept, -1 automatic)
        self.mem_budget = mem_budget  # device bytes the transport may hold with its scratch (0: none)
        self.scene = None
        self.transport = None

    def build(self, d, stream=None):
        self.scene = rgs.rgs_build_scene(*[d[k] for k in SURFEL_KEYS], sh_degree=d["L"],
                                         alpha_model=self.alpha_model, stream=stream, scene=self.scene)
        return self.scene

    def trace(self, d, stream=None, hit_capacity=0):
        if self.pairs:
            self.transport = rgs.rgs_trace_pairs(self.scene, d["light_pos"], d["light_I"], lam=d.get("lam"),
                                                 stream=stream, transport=self.transport,
                                                 directional=d.get("light_dir", False))
        else:
            self.transport = rgs.rgs_trace_transport(self.scene, d["light_pos"], d["light_I"], d["nd"], d["seed"],
                                                     hit_capacity=hit_capacity, stream=stream,
                                                     transport=self.transport, directional=d.get("light_dir", False))
        rgs.rgs_set_checkpointing(self.transport, self.checkpoint)
        rgs.rgs_set_memory_budget(self.transport, self.mem_budget)
        rgs.rgs_set_tensor_cores(self.transport, self.tensor_cores)
        return self.transport

    def solve(self, E, nb, B_out=None, stats=False, stream=None, precision=None):
        prec = self.precision if precision is None else precision
        return rgs.rgs_solve(self.transport, E, nb, B_out=B_out, stats=stats, precision=prec, stream=stream)

    def adjoint(self, g, outs=(None, None, None), stream=None):
        return rgs.rgs_adjoint(self.transport, g, *outs, stream=stream)

    def adjoint_pairs(self, g, stream=None):
        """Center-to-center gradients (dL/dE, dL/da^d, dL/do, dL/dlambda)."""
        return rgs.rgs_adjoint_pairs(self.transport, g, stream=stream)

    def adjoint_geometry(self, g, stream=None):
        """Gradients with the geometry ones, either transport:
        (dL/dE, dL/da^d, dL/do, dL/dp, dL/ds, dL/dtu, dL/dtv)."""
        return rgs.rgs_adjoint_geometry(self.transport, g, stream=stream)

    def adjoint_pairs_geometry(self, g, stream=None):
        """Center-to-center gradients with the geometry ones (Eqs. dl-dgeo-0/1):
        (dL/dE, dL/da^d, dL/do, dL/dlambda, dL/dp [N,3], dL/ds [N,2], dL/dtu [N,3], dL/dtv [N,3])."""
        return rgs.rgs_adjoint_pairs_geometry(self.transport, g, stream=stream)

    def step(self, d, g, B_out=None, grads=(None, None, None), stream=None):
        """One full pass of the path: scene build, trace, n bounces, adjoint."""
        self.build(d, stream)
        self.trace(d, stream)
        B, _ = self.solve(d["E"], d["nb"], B_out=B_out, stream=stream)
        return B, self.adjoint(g, grads, stream=stream)


class RadiositySolve(torch.autograd.Function):
    """B = solve(E, a^d, o; geometry, lights) with gradients w.r.t. E, a^d and o.

    forward rebuilds the scene from the given albedo/opacity, traces and runs n bounces;
    backward runs rgs_adjoint (exact gradient of the truncated series)."""

    @staticmethod
    def forward(ctx, E, ad, o, geom, nb, alpha_model=rgs.RGS_ALPHA_GAUSS):
        d = dict(geom)
        d["ad"], d["o"] = ad.detach().contiguous(), o.detach().contiguous()
        pipe = Pipeline(alpha_model)
        pipe.build(d)
        pipe.trace(d)
        B, _ = pipe.solve(E.detach().contiguous() if E is not None else None, int(nb))
        ctx.pipe = pipe
        return B

    @staticmethod
    def backward(ctx, gB):
        dE, dad, do = ctx.pipe.adjoint(gB.contiguous())
        return dE, dad, do, None, None, None


def radiosity(E, ad, o, geom, nb, alpha_model=rgs.RGS_ALPHA_GAUSS):
    return RadiositySolve.apply(E, ad, o, geom, nb, alpha_model)


class RadiositySolveGeometry(torch.autograd.Function):
    """B = solve(E, a^d, o, p, s, tu, tv; the rest of the scene and the lights) with gradients
    with respect to all seven (Eqs. final_dL_dE, final-dl-dbrdf, dl-dgeo-0/1).

    forward rebuilds the scene from the given tensors, traces and runs n bounces (every
    iterate kept: the hemisphere form's geometry gradients read them all); backward runs
    rgs_adjoint_geometry."""

    @staticmethod
    def forward(ctx, E, ad, o, p, s, tu, tv, geom, nb, alpha_model=rgs.RGS_ALPHA_GAUSS, pairs=False):
        d = dict(geom)
        for key, v in (("ad", ad), ("o", o), ("p", p), ("s", s), ("tu", tu), ("tv", tv)):
            d[key] = v.detach().contiguous()
        pipe = Pipeline(alpha_model, pairs=pairs)
        pipe.build(d)
        pipe.trace(d)
        B, _ = pipe.solve(E.detach().contiguous() if E is not None else None, int(nb))
        ctx.pipe = pipe
        return B

    @staticmethod
    def backward(ctx, gB):
        dE, dad, do, dp, ds, dtu, dtv = ctx.pipe.adjoint_geometry(gB.contiguous())
        return dE, dad, do, dp, ds, dtu, dtv, None, None, None, None


def radiosity_geometry(E, ad, o, p, s, tu, tv, geom, nb, alpha_model=rgs.RGS_ALPHA_GAUSS, pairs=False):
    """B differentiable in emission, albedo, opacity, centres, scales and frame inputs."""
    return RadiositySolveGeometry.apply(E, ad, o, p, s, tu, tv, geom, nb, alpha_model, pairs)
