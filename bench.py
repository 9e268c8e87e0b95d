#!/usr/bin/env python
"""Throughput of the surfel light-transport hot path on one or more GB300s.

A step is one pass of the whole path on the 50,000-surfel fruit-bowl scene (SH degree
3, 256 hemisphere rays per surfel, 4 bounces, one point light): scene build (frames,
BRDF coefficients, Morton sort, BVH), hemisphere and shadow-ray tracing with alpha
compositing, the bounce iteration, and the adjoint (transposed bounces, emission,
albedo and opacity gradients).  Metric: surfel x light x bounces per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs the same workload on its own GPU (replicas; the path
does not shard) and rank 0 prints one JSON line.  `--impl reference` times the FP64
CPU oracle on host cores instead (a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "surfel·light·bounces/s, fwd+adjoint, batched vs plain FP32 on GB300 at ≤1e-3 rel err"
UNIT = "surfel·light·bounces/s"
WORKLOAD = ("fruit bowl: 50,000 Gaussian surfels on 12 spheres in a hemispherical bowl on a ground plane, "
            "SH degree 3 (16 x RGB), 256 stratified hemisphere rays/surfel, 4 bounces, 1 point light, "
            "FP32, forward + adjoint (emission, albedo, opacity gradients)")
MULTI_WORKLOAD = ("multi-light batch: 200,000 fruit-bowl surfels, 100 point lights on a Fibonacci sphere of radius 3 "
                  "(intensity U[5,20]) as 300 right-hand sides, SH degree 3, 256 rays/surfel, 4 bounces, "
                  "forward + adjoint")
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _src_sha(name):
    with open(os.path.join(ROOT, "paper_2509_18497_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# DRAM bytes per launch from one ncu capture (profiles/), keyed by kernel; valid only
# while the kernel's source file is unchanged since the capture.
NCU_TRAFFIC = {
    "k_trace_hemi": {"bytes_per_launch": 0.834729e9 + 2.153428e9, "n": 10000, "src_sha": "35405e494984794e"},
}


def algorithmic_bytes(kernel, info, n, nd, nb, C, nc):
    """Compulsory HBM bytes of one launch of `kernel` (reads + writes, each array once)."""
    A = n * C * nc * 4          # one [N][C][nc] float array
    H = info["n_hits"]
    rays = n * nd
    tile = A * 3 // C           # one 3-column tile of such an array
    if kernel == "k_bounce":      # records + counts + directions + B^(k-1) + S in; Q, B^(k) out
        return H * 8 + rays * (4 + 8 + 16) + 4 * A
    if kernel == "k_adj_src":     # transposed records, (direction, y) per ray, offsets; v^(a) tile out, u tile r+w
        return H * 8 + rays * 32 + (n + 1) * 8 + 3 * tile
    if kernel == "k_adj_ray":     # directions + v^(a-1) tile in; y per ray out
        return rays * 32 + tile
    if kernel == "k_opacity_g":   # records (j) + counts + directions; 4 iterates of v and B tiles; g per hit out
        return H * (8 + 4) + rays * (4 + 8 + 16) + 2 * min(nb, 4) * tile
    if kernel == "k_opacity_rec":  # records (j, a) + G + g per hit, counts; dL/do
        return H * (8 + 4 + 4) + rays * (4 + 8) + n * 4
    tiles = (C + 31) // 32
    A16 = n * C * 16 * 2        # BF16 copy of an iterate (rows padded to 16)
    if kernel == "k_bounce_mc":   # per 32-column tile: records, counts, offsets, directions; iterate rows once
        return tiles * (H * 8 + rays * (4 + 8 + 16)) + A16 + 4 * A + A16
    if kernel == "k_opacity_g_mc":  # per tile: records + ray data; 4 iterates of v (FP32) and B (BF16); g per hit
        return tiles * (H * (8 + 4) + rays * (4 + 8 + 16)) + min(nb, 4) * (A + A16)
    if kernel == "k_adj_src_mc":  # per tile: transposed records, directions, y; v tile out, u r+w
        return tiles * (H * 8 + rays * (16 + 128) + (n + 1) * 8) + 3 * A
    if kernel == "k_trace_hemi":  # scene (64 B/surfel + 64 B/node) in; records, counts, directions out
        return n * 64 + (n - 1) * 64 + H * 12 + rays * (4 + 8 + 16) + n * 4
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.p = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


def cpu_baseline(n_sample, threads=None):
    """The FP64 oracle as it stands, timed on the host cores: full pipeline (transport,
    4 bounces, adjoint with all gradients) on an n_sample-surfel scene of the same
    generator, 256 rays/surfel, SH degree 3, one light."""
    import numpy as np

    from oracle import oracle as O
    from paper_2509_18497_gb300 import scenes

    sc = scenes.fruit_bowl(n=n_sample)
    W = np.random.default_rng(0).normal(size=(sc["n"], 16, 3))
    t0 = time.perf_counter()
    orc = O.Oracle(sc).transport()
    orc.adjoint(W, E=None, nb=sc["nb"])  # runs the solve (with iterates) and the adjoint
    dt = time.perf_counter() - t0
    units = sc["n"] * 1 * sc["nb"]
    return {"value": units / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"fruit-bowl generator at {n_sample} surfels (same SH degree, rays, bounces, light), "
                      f"full forward + adjoint in {dt:.1f} s"}, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n_sample = args.ref_sample
    for _ in range(args.warmup):
        cpu_baseline(n_sample)
    total, units = 0.0, 0
    cb = None
    for _ in range(args.steps):
        cb, dt = cpu_baseline(n_sample)
        total += dt
        units += n_sample * 1 * 4
    value = units / total
    cb = dict(cb, value=value)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_surfels": n_sample},
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=50000, help="surfel count (default: the 50,000-surfel workload)")
    ap.add_argument("--workload", default="fruit_bowl", choices=["fruit_bowl", "multi_light"],
                    help="fruit_bowl: 1 light (default); multi_light: 200,000 surfels and 100 lights")
    ap.add_argument("--cpu-sample", type=int, default=6000, help="surfels of the timed oracle sample")
    ap.add_argument("--ref-sample", type=int, default=1500, help="surfels per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2509_18497_gb300 import api, build, rgs, scenes

    build.build()
    rgs.load()
    if args.workload == "multi_light":
        sc = scenes.multi_light(n=200000 if args.n == 50000 else args.n)
    else:
        sc = scenes.fruit_bowl(n=args.n)
    n, nd, nb, nc, nl = sc["n"], sc["nd"], sc["nb"], 16, sc["light_pos"].shape[0]
    C = 3 * nl
    units_per_step = n * nl * nb

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    d = api.upload(sc, device=dev)
    g = torch.as_tensor(np.random.default_rng(1).normal(size=(n, nc, C)).astype(np.float32), device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def make(precision):
        B = torch.empty((n, nc, C), device=dev)
        grads = (torch.empty((n, nc, 3), device=dev), torch.empty((n, 3), device=dev), torch.empty((n,), device=dev))
        return api.Pipeline(precision=precision), B, grads

    # batched form (BF16 gathers, FP32 accumulation, one FP32 residual-correction bounce)
    # and the plain FP32 form, on the same inputs
    forms = {"batched": make(rgs.RGS_BF16_FP32ACC_RESCORR), "plain": make(rgs.RGS_FP32)}
    for pipe, B, grads in forms.values():
        for _ in range(max(args.warmup, 3)):
            pipe.step(d, g, B_out=B, grads=grads)
    torch.cuda.synchronize()
    info = rgs.rgs_transport_info_get(forms["batched"][0].transport)
    # accuracy of the batched form against the FP32 form (which the tests hold to 1e-4 of the oracle)
    Bb, Bp = forms["batched"][1].double(), forms["plain"][1].double()
    rel_err = float(torch.linalg.norm(Bb - Bp) / torch.linalg.norm(Bp))
    grad_err = max(float(torch.linalg.norm(a.double() - b.double()) / torch.linalg.norm(b.double()))
                   for a, b in zip(forms["batched"][2], forms["plain"][2]))

    def timed(form, profile):
        pipe, B, grads = forms[form]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            rgs.rgs_profile_reset()
            rgs.rgs_profile_enable(True)
        launches0 = rgs.rgs_launch_count()
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()  # evict L2 between steps (outside the step's events)
            ev[k][0].record(stream)
            pipe.step(d, g, B_out=B, grads=grads)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        launches = rgs.rgs_launch_count() - launches0
        prof = None
        if profile:
            rgs.rgs_profile_enable(False)
            prof = rgs.rgs_profile_report()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_s = sum(step_ms) / 1e3
        if world > 1:
            t = torch.tensor([total_s], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_s = float(t.item())
            dist.barrier()
        return units_per_step * args.steps * world / total_s, step_ms, launches, prof, t_wall

    # the headline is the batched form when it meets the 1e-3 accuracy gate, else plain
    headline = "batched" if rel_err <= 1e-3 else "plain"
    other = "plain" if headline == "batched" else "batched"
    clocks = Clocks(local)
    value, step_ms, launches, prof, t_wall = timed(headline, True)
    clk = clocks.stop()
    value_o, step_ms_o, _, _, _ = timed(other, False)
    value_b, value_p = (value, value_o) if headline == "batched" else (value_o, value)
    step_ms_b, step_ms_p = (step_ms, step_ms_o) if headline == "batched" else (step_ms_o, step_ms)
    pipe, B, grads = forms[headline]

    # ---------------------------------------------------------- end to end (host buffers)
    host = {k: d[k].cpu().pin_memory() for k in api.SURFEL_KEYS + ("light_pos", "light_I")}
    g_host = g.cpu().pin_memory()
    outs_host = [torch.empty(B.shape, pin_memory=True)] + [torch.empty(x.shape, pin_memory=True) for x in grads]
    d_e2e = dict(d)
    h2d = sum(v.numel() * 4 for v in host.values()) + g_host.numel() * 4
    d2h = sum(x.numel() * 4 for x in outs_host)
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        e2e_ev[k][0].record(stream)
        for key, v in host.items():
            d_e2e[key] = v.to(dev, non_blocking=True)
        g_dev = g_host.to(dev, non_blocking=True)
        Bk, gr = pipe.step(d_e2e, g_dev)
        for dst, src in zip(outs_host, (Bk,) + tuple(gr)):
            dst.copy_(src, non_blocking=True)
        e2e_ev[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_s = sum(a.elapsed_time(b) for a, b in e2e_ev) / 1e3
    if world > 1:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = units_per_step * args.steps * world / e2e_s

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---------------------------------------------------------- roofline of the dominant kernel
    peak, peak_kind = _peaks()
    kernels = {k: {"launches_per_step": c / args.steps, "ms_per_step": ms / args.steps,
                   "share": ms / max(1e-9, sum(v[1] for v in prof.values()))} for k, (c, ms) in prof.items()}
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    c_dom, ms_dom = prof[dom]
    alg = algorithmic_bytes(dom, info, n, nd, nb, C, nc)
    avg_ms = ms_dom / c_dom
    achieved = alg / (avg_ms * 1e-3) / 1e9 if alg else None
    src_file = {"k_bounce": "rgs_solve.cu", "k_adj_src": "rgs_adjoint.cu", "k_adj_ray": "rgs_adjoint.cu",
                "k_bounce_mc": "rgs_manycol.cu", "k_opacity_g_mc": "rgs_manycol.cu", "k_adj_src_mc": "rgs_manycol.cu",
                "k_opacity_g": "rgs_adjoint.cu", "k_opacity_rec": "rgs_adjoint.cu",
                "k_trace_hemi": "rgs_trace.cu"}.get(dom)
    traffic = None
    if dom in NCU_TRAFFIC and src_file and NCU_TRAFFIC[dom]["src_sha"] == _src_sha(src_file):
        traffic = NCU_TRAFFIC[dom]["bytes_per_launch"] * (n / NCU_TRAFFIC[dom]["n"])
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "algorithmic_bytes": alg, "avg_launch_ms": avg_ms, "peak_source": peak_kind}

    cb = None
    if not args.no_cpu_baseline and world == 1:
        cb, _ = cpu_baseline(args.cpu_sample)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3),
            "ms_per_step": sum(step_ms) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16-gather/f32-acc" if headline == "batched" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == "fruit_bowl" else MULTI_WORKLOAD, "n_surfels": n, "sh_degree": 3, "rays_per_surfel": nd, "bounces": nb,
                       "lights": nl, "precision": headline, "l2": "flushed between steps (512 MiB write)",
                       "parallelism": f"replicas x{world}", "hit_records": info["n_hits"]},
            "batched_vs_plain": {"batched": value_b, "plain": value_p, "speedup": value_b / value_p,
                                 "batched_rel_l2_vs_fp32": rel_err, "batched_grad_rel_l2_vs_fp32": grad_err,
                                 "plain_ms_per_step": sum(step_ms_p) / args.steps,
                                 "batched_ms_per_step": sum(step_ms_b) / args.steps},
            "roofline": roofline, "cpu_baseline": cb,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches), "clocks": clk, "wall_s_timed": t_wall, "kernels": kernels}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
