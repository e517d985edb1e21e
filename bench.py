#!/usr/bin/env python
"""Benchmark of the SaLF ray-cast hot path on GB300.

Headline: Mrays/s for a 1920x1080 pinhole camera (60 deg horizontal FOV, one
ray per pixel) over the seeded 2,000,000-voxel synthetic driving scene (FP32
records, Eq. 1 density), forward only.  Extra sections on the same JSON line:
128x2048 spinning LiDAR and 1920x1080 190-degree fisheye on the same scene,
forward + adjoint for 8 cameras 960x640 on a 1M-voxel BF16 scene, and the
continuous-batching server on a 4M-voxel BF16 scene (p50 / p99 latency).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl salf|reference]
N > 1 runs as independent replicas (launched with torch.distributed.run), one
per GPU: rays are independent, nothing is exchanged.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Mrays/s, 1080p pinhole camera, 2M-voxel driving scene (FP32, forward)"
WORKLOAD = "pinhole 1920x1080, 60deg hFOV, 1 ray/pixel, driving scene 2,000,000 voxels (seed 2)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SOURCES = ["paper_2507_18713_gb300/csrc/render.cu", "paper_2507_18713_gb300/csrc/traverse.cuh",
                  "paper_2507_18713_gb300/csrc/salf_internal.h"]
RASTER_SOURCES = KERNEL_SOURCES + ["paper_2507_18713_gb300/csrc/raster.cu"]
FALLBACK_HBM_GBS = 6800.0

# algorithmic bytes (Eq. 1-2 record scalars read per visit, outputs per ray)
B_FIELD_EXP_F32 = 25 * 4
B_FIELD_EXP_INT_F32 = 29 * 4
B_FIELD_EXP_BF16 = 25 * 2
B_OUT_CAMERA = 20
B_OUT_LIDAR = 12


def kernel_hash(workload: str = "camera") -> str:
    """Hash of the sources of the kernel a workload times (ncu traffic figures
    are only used while it matches)."""
    h = hashlib.sha256()
    for f in (RASTER_SOURCES if workload == "raster" else KERNEL_SOURCES):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def hbm_peak():
    try:
        p = json.load(open(PEAKS_FILE))
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def driving_camera():
    return synth.pinhole(1920, 1080, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))


def driving_lidar():
    return synth.lidar(128, 2048, synth.lidar_pose((0.0, 0.0, 1.9), 0.0),
                       synth.lidar_pose((1.0, 0.0, 1.9), 0.02), t0=0.0, t1=0.1)


def driving_fisheye():
    return synth.fisheye(1920, 1080, 190.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))


WORKLOADS = {
    "camera": dict(sensor=driving_camera, b_field=B_FIELD_EXP_F32, b_out=B_OUT_CAMERA,
                   want_intensity=False, outputs=("rgb", "depth", "opacity"), metric=METRIC,
                   workload=WORKLOAD),
    "lidar": dict(sensor=driving_lidar, b_field=B_FIELD_EXP_INT_F32, b_out=B_OUT_LIDAR,
                  want_intensity=True, outputs=("depth", "opacity", "intensity"),
                  metric="Mrays/s, 128x2048 spinning LiDAR, 2M-voxel driving scene (FP32, forward)",
                  workload="spinning LiDAR 128 beams x 2048 azimuths, elevation -25..+15 deg, "
                           "per-ray pose, range + intensity, driving scene 2,000,000 voxels (seed 2)"),
    "fisheye": dict(sensor=driving_fisheye, b_field=B_FIELD_EXP_F32, b_out=B_OUT_CAMERA,
                    want_intensity=False, outputs=("rgb", "depth", "opacity"),
                    metric="Mrays/s (valid rays), 1080p 190-degree fisheye, 2M-voxel driving scene",
                    workload="equidistant fisheye 1920x1080 190deg, driving scene 2,000,000 voxels"),
    "raster": dict(sensor=driving_camera, b_field=B_FIELD_EXP_F32, b_out=B_OUT_CAMERA,
                   want_intensity=False, outputs=("rgb", "depth", "opacity"),
                   metric="Mrays/s, 1080p pinhole camera by tile rasterisation, 2M-voxel driving "
                          "scene (FP32, forward)",
                   workload=WORKLOAD + ", tile rasteriser (projection, tile lists, radix sort, "
                            "16x16 tiles)"),
}


# --------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id_for(torch, dev: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev] if vis else str(dev)


# --------------------------------------------------------------------- replicas

def replica_throughput(local_ms: float, local_units: int, steps: int, dist=None, device="cpu"):
    """Whole-job throughput of N independent replicas: every rank processed
    local_units per step for `steps` steps in local_ms; the job took the
    slowest rank's time.  Returns (units per second, max ms over ranks)."""
    t = local_ms
    units = local_units
    if dist is not None and dist.is_initialized():
        import torch
        v = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        u = torch.tensor([local_units], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        t, units = float(v.item()), int(u.item())
    return units * steps / (t * 1e-3), t


# --------------------------------------------------------------------- timing

def timed_renders(torch, fn, steps, warmup, flush):
    """Per-step CUDA-event durations (ms) of fn(), L2 flushed between steps."""
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in evs:
        flush.zero_()
        a.record(st)
        fn()
        b.record(st)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def visits_of(torch, gscene, sensor, want_intensity=False):
    out = gscene.render(sensor, saved=True, outputs=("opacity",), want_intensity=want_intensity)
    torch.cuda.synchronize()
    s = out["saved"]
    return int(s[:, 7].double().sum().item()), out


def section(torch, P, gscene, sensor, steps, warmup, flush, b_field, b_out, want_intensity=False,
            rays_counted=None):
    R = sensor["width"] * sensor["height"]
    outputs = ("rgb", "depth", "opacity") if sensor["kind"] != "lidar" else ("depth", "opacity", "intensity")
    out = {k: torch.empty((R, 3) if k == "rgb" else (R,), device="cuda") for k in outputs}
    fn = lambda: gscene.render(sensor, outputs=outputs, out=out, valid=False,
                               want_intensity=want_intensity)
    ms = timed_renders(torch, fn, steps, warmup, flush)
    nvis, sv = visits_of(torch, gscene, sensor, want_intensity)
    n_rays = R if rays_counted is None else rays_counted
    avg = sum(ms) / len(ms)
    bytes_alg = nvis * b_field + R * b_out
    return dict(ms=avg, ms_median=statistics.median(ms), rays=n_rays,
                mrays_s=n_rays / (avg * 1e-3) / 1e6, fps=1e3 / avg, visits=nvis,
                visits_per_ray=nvis / R, bytes_alg=bytes_alg,
                achieved_gbs=bytes_alg / (avg * 1e-3) / 1e9)


# --------------------------------------------------------------------- extras

def bench_backward(torch, P, steps, warmup, flush, peak):
    sc = synth.driving_scene(1_000_000, seed=4, ground_extent=141.4, n_actors=140)
    g = P.Scene(sc, dtype="bf16")
    cams = [synth.pinhole(960, 640, 60.0, synth.camera_pose_looking(
        (5.0 * math.cos(k * math.pi / 4), 5.0 * math.sin(k * math.pi / 4), 1.7), k * math.pi / 4))
        for k in range(8)]
    gen = torch.Generator(device="cuda").manual_seed(4)
    targets = [torch.rand((960 * 640, 3), device="cuda", generator=gen) for _ in cams]
    dparams = torch.zeros((sc.n, 32), device="cuda")
    R = 960 * 640
    outs = [dict(rgb=torch.empty((R, 3), device="cuda"), saved=torch.empty((R, 8), device="cuda"))
            for _ in cams]
    grads = [torch.empty((R, 3), device="cuda") for _ in cams]
    inv = 1.0 / (R * 3 * len(cams))

    def step():
        # the 8 cameras in one forward launch and one adjoint launch
        dparams.zero_()
        g.render_batch(cams, outputs=("rgb",), saved=True, valid=False, outs=outs)
        for o, tg, gr in zip(outs, targets, grads):
            torch.sub(o["rgb"], tg, out=gr).mul_(2 * inv)
        g.backward_batch(cams, [o["saved"] for o in outs], d_rgb=grads, d_params=dparams)

    ms = timed_renders(torch, step, max(3, steps // 20), warmup, flush)
    g.check()
    avg = sum(ms) / len(ms)
    # the adjoint kernel alone (one batched launch over the 8 cameras), with its
    # algorithmic bytes: per visit the BF16 record's 25 used scalars (50 B) and
    # 25 FP32 gradient scalars added (100 B); per ray dL/drgb (12 B) and the
    # saved totals (32 B)
    visits = sum(int(o["saved"][:, 7].double().sum().item()) for o in outs)
    adj = lambda: g.backward_batch(cams, [o["saved"] for o in outs], d_rgb=grads,
                                   d_params=dparams)
    ms_adj = timed_renders(torch, adj, max(3, steps // 20), warmup, flush)
    avg_adj = sum(ms_adj) / len(ms_adj)
    b_adj = visits * (B_FIELD_EXP_BF16 + 4 * 25) + len(cams) * R * (12 + 32)
    ach = b_adj / (avg_adj * 1e-3) / 1e9
    return dict(workload="8 pinhole 960x640, driving scene 1,000,000 voxels (seed 4), BF16 "
                "records, FP32 grads, MSE vs U[0,1] targets; salf_render_rays_batch + "
                "salf_render_backward_batch (one launch each for the 8 cameras)",
                ms_per_step=avg, mrays_s=len(cams) * R / (avg * 1e-3) / 1e6,
                adjoint=dict(kernel="k_backward<BF16,EXP>, the 8 cameras in one launch",
                             ms_per_launch=avg_adj, ms_per_camera=avg_adj / len(cams),
                             visits_per_ray=visits / (len(cams) * R),
                             roofline=dict(bound="hbm", achieved=ach, peak=peak, unit="GB/s",
                                           frac=ach / peak, bytes_per_launch=b_adj,
                                           note="per visit 50 B BF16 record + 100 B of gradient "
                                                "scalars (25 x 4 B), per ray 12 B dL/drgb + "
                                                "32 B saved totals; visits counted by the "
                                                "forward kernel; bytes and time of the one "
                                                "launch")))


def bench_refine(torch, P, flush):
    """One densify/prune step (Sec. III-C) of the training scene: the 8 training
    cameras render with alpha maxima and back-propagate an MSE loss, then the
    top 5% of voxels by colour-gradient L1 norm split, alpha < 0.001 prunes,
    and the scene is rebuilt from the new voxel list."""
    sc = synth.driving_scene(1_000_000, seed=4, ground_extent=141.4, n_actors=140)
    g = P.Scene(sc, dtype="bf16")
    cams = [synth.pinhole(960, 640, 60.0, synth.camera_pose_looking(
        (5.0 * math.cos(k * math.pi / 4), 5.0 * math.sin(k * math.pi / 4), 1.7), k * math.pi / 4))
        for k in range(8)]
    gen = torch.Generator(device="cuda").manual_seed(4)
    R = 960 * 640
    params = torch.from_numpy(sc.params.astype(np.float32)).cuda()
    dparams = torch.zeros((sc.n, 32), device="cuda")
    ma = torch.zeros(sc.n, device="cuda")
    for cam in cams:
        o = g.render(cam, outputs=("rgb",), saved=True, valid=False, max_alpha=ma)
        tg = torch.rand((R, 3), device="cuda", generator=gen)
        g.backward(cam, o["saved"], d_rgb=(o["rgb"] - tg).mul_(2.0 / (R * 3 * len(cams))),
                   d_params=dparams)
    l1 = dparams[:, 4:13].abs().sum(dim=1)
    thr = float(torch.quantile(l1[l1 > 0][:1 << 24].float(), 0.95).item())
    torch.cuda.synchronize()
    ms = {}
    reps = 5
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vs, counts = g.refine(params, dparams, ma, thr, 1e-3)
        t1 = time.perf_counter()
        g2 = P.Scene(vs, dtype="bf16", params=vs.params)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ms.setdefault("plan_apply", []).append((t1 - t0) * 1e3)
        ms.setdefault("rebuild", []).append((t2 - t1) * 1e3)
        g2.close()
    # Eq. 7 L_reg over the scene's face-adjacent pairs (loss and gradient)
    loss = torch.zeros(1, device="cuda")
    reg = statistics.median(timed_renders(
        torch, lambda: g.reg_loss(params, 1.0, 1.0, 1.0, grads=dparams, loss=loss), 20, 3, flush))
    g.check()
    return dict(workload="training scene 1,000,000 voxels (seed 4), BF16; alpha maxima and "
                "gradients from the 8 training cameras (960x640); split the top 5% by colour-"
                "gradient L1 norm, prune alpha < 0.001",
                counts=counts, split_threshold=thr, reg_loss_ms=reg,
                plan_apply_ms=statistics.median(ms["plan_apply"]),
                rebuild_ms=statistics.median(ms["rebuild"]),
                note="plan + apply on the GPU (includes the one host wait for the counts); rebuild "
                     "= salf_build_scene from the device-resident voxel list (device build)")


def bench_serving(torch, P, duration_s=10.0, seed=6, n_streams=4):
    sc = synth.driving_scene(4_000_000, seed=3, ground_layers=2, n_actors=600)
    g = P.Scene(sc, dtype="bf16")
    rng = np.random.default_rng(seed)
    kinds = ([("pinhole", 1920, 1080)] * 8 + [("fisheye", 1280, 960)] * 4 + [("pano", 4096, 1024)] * 2
             + [("lidar", 2048, 128)] * 4 + [("lidar", 1024, 64)] * 2)
    events = []
    for si, (k, w, h) in enumerate(kinds):
        t = rng.exponential(0.1)
        while t < duration_s:
            events.append((t, si))
            t += rng.exponential(0.1)
    events.sort()

    def make(si):
        k, w, h = kinds[si]
        yaw = si * 2 * math.pi / len(kinds) + rng.normal(0, 0.05)
        pos = (rng.normal(0, 0.5), rng.normal(0, 0.5), 1.7 + rng.normal(0, 0.05))
        if k == "pinhole":
            return synth.pinhole(w, h, 60.0, synth.camera_pose_looking(pos, yaw))
        if k == "fisheye":
            return synth.fisheye(w, h, 190.0, synth.camera_pose_looking(pos, yaw))
        if k == "pano":
            return synth.panorama(w, h, synth.camera_pose_looking(pos, yaw))
        return synth.lidar(h, w, synth.lidar_pose((pos[0], pos[1], 1.9), yaw),
                           synth.lidar_pose((pos[0] + 1.0, pos[1], 1.9), yaw + 0.02), t0=0.0, t1=0.1)

    reqs = [(t, make(si)) for t, si in events]
    total_rays = sum(s["width"] * s["height"] for _, s in reqs)
    # continuous batching
    srv = P.Server(g, mem_budget_bytes=2 << 30, n_streams=n_streams)
    warm = [srv.submit(s, want_intensity=s["kind"] == "lidar") for _, s in reqs[:8]]
    for t in warm:
        srv.poll(t, -1)
        srv.release(t)
    srv.close()
    srv = P.Server(g, mem_budget_bytes=2 << 30, n_streams=n_streams)
    import queue
    q: "queue.Queue" = queue.Queue()

    def consumer():   # a client that reads each result as soon as it is done
        while True:
            t = q.get()
            if t is None:
                return
            srv.poll(t, -1)
            srv.release(t)

    th = threading.Thread(target=consumer)
    th.start()
    t0 = time.perf_counter()
    for at, s in reqs:
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        q.put(srv.submit(s, want_intensity=s["kind"] == "lidar"))
    q.put(None)
    th.join()
    t_end = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    # sequential plain rendering of the same trace (one render at a time)
    lat = []
    t0 = time.perf_counter()
    for at, s in reqs:
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        g.render(s, want_intensity=s["kind"] == "lidar")
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t0 - at) * 1e3)
    t_seq = time.perf_counter() - t0
    # saturation: the same requests offered all at once (closed loop)
    sat = reqs[:min(len(reqs), 400)]
    sat_rays = sum(s["width"] * s["height"] for _, s in sat)
    srv = P.Server(g, mem_budget_bytes=2 << 30, n_streams=n_streams)
    q2: "queue.Queue" = queue.Queue()

    def consumer2():
        while True:
            t = q2.get()
            if t is None:
                return
            srv.poll(t, -1)
            srv.release(t)

    th = threading.Thread(target=consumer2)
    th.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _, s in sat:
        q2.put(srv.submit(s, want_intensity=s["kind"] == "lidar"))
    q2.put(None)
    th.join()
    t_sat_b = time.perf_counter() - t0
    st_sat = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _, s in sat:
        g.render(s, want_intensity=s["kind"] == "lidar")
        torch.cuda.synchronize()
    t_sat_s = time.perf_counter() - t0
    lat.sort()
    q = lambda p: lat[min(len(lat) - 1, int(math.ceil(p * len(lat))) - 1)]
    return dict(workload=f"20 sensors at 10 Hz Poisson for {duration_s:.0f} s, driving scene "
                "4,000,000 voxels (seed 3), BF16 records", requests=len(reqs),
                offered_mrays_s=total_rays / duration_s / 1e6,
                streams=n_streams,
                batched=dict(p50_ms=st["p50_ms"], p99_ms=st["p99_ms"], launches=st["launches"],
                             requests_per_launch=st["requests_launched"] / max(1, st["launches"]),
                             max_batch=st["max_batch"], mixed_launches=st["mixed_launches"],
                             mrays_s=total_rays / t_end / 1e6, wall_s=t_end),
                sequential=dict(p50_ms=q(0.5), p99_ms=q(0.99), mrays_s=total_rays / t_seq / 1e6,
                                wall_s=t_seq),
                saturated=dict(requests=len(sat), rays=sat_rays,
                               batched_mrays_s=sat_rays / t_sat_b / 1e6,
                               batched_launches=st_sat["launches"],
                               requests_per_launch=st_sat["requests_launched"]
                               / max(1, st_sat["launches"]),
                               mixed_launches=st_sat["mixed_launches"],
                               batched_p50_ms=st_sat["p50_ms"], batched_p99_ms=st_sat["p99_ms"],
                               sequential_mrays_s=sat_rays / t_sat_s / 1e6,
                               note="all requests offered at once; sequential = one "
                                    "salf_render_rays per request in arrival order, "
                                    "waiting for each"))


# --------------------------------------------------------------------- oracle

def oracle_rate(scene_or, sensor, n_sample, seed, outputs=None):
    """Rays per second of the oracle on the host cores; `outputs`, if a dict,
    receives the rendered rays (idx) and their outputs."""
    import oracle
    R = sensor["width"] * sensor["height"]
    n_sample = min(n_sample, R)
    idx = None if n_sample >= R else synth.sample_ray_indices(R, n_sample, seed)
    t = time.perf_counter()
    out = oracle.render(scene_or, sensor, idx=idx)
    dt = time.perf_counter() - t
    if outputs is not None:
        outputs.update(out, idx=np.arange(R) if idx is None else idx)
    return n_sample / dt / 1e6, dt, oracle.num_threads()


def bf16_storage_error(torch, P, sc, osc, cam, ref):
    """Error of BF16 record storage against the FP64 oracle on the FP32
    records, per output: the 1080p frame the CPU baseline rendered, and a
    seeded sample of the LiDAR sweep (range, intensity)."""
    import oracle
    g16 = P.Scene(sc, dtype="bf16")
    res = {}

    def stats(a, b):
        e = np.abs(np.asarray(a, np.float64) - b).ravel()
        return dict(max=float(e.max()), mean=float(e.mean()),
                    p999=float(np.quantile(e, 0.999)))

    idx = ref["idx"]
    o = g16.render(cam, outputs=("rgb", "depth", "opacity"))
    torch.cuda.synchronize()
    for k in ("rgb", "depth", "opacity"):
        res[f"camera_{k}"] = stats(o[k].cpu().numpy()[idx], ref[k])
    lid = driving_lidar()
    li = synth.sample_ray_indices(lid["width"] * lid["height"], 65536, 98)
    rl = oracle.render(osc, lid, idx=li, want_intensity=True)
    ol = g16.render(lid, outputs=("depth", "opacity", "intensity"), want_intensity=True)
    torch.cuda.synchronize()
    for k, name in (("depth", "range"), ("opacity", "opacity"), ("intensity", "intensity")):
        res[f"lidar_{name}"] = stats(ol[k].cpu().numpy()[li], rl[k])
    g16.check()
    g16.close()
    return dict(note="BF16 records (GPU) vs the FP64 oracle on the FP32 records; absolute "
                     "errors (depth / range in metres); the tolerance for arithmetic parity "
                     "(FP32 records, or the oracle on dequantised records) is 1e-4 / 1e-3 m",
                camera_rays=int(len(idx)), lidar_rays=int(len(li)), **res)


def run_reference(args):
    """The FP64 CPU oracle on the host cores, same workload and metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    sc = synth.driving_scene(2_000_000, seed=2)
    osc = oracle.OracleScene(sc)
    cam = driving_camera()
    R = cam["width"] * cam["height"]
    rate, _, cores = oracle_rate(osc, cam, 8192, 100)
    budget_s = 150.0
    # whole 1080p frames per step when the run fits the time budget, else an
    # equal seeded sample of each frame's rays
    per_step = int(max(1024, min(R, rate * 1e6 * budget_s / max(1, args.steps + args.warmup))))
    for w in range(args.warmup):
        oracle_rate(osc, cam, per_step, 200 + w)
    times = []
    for k in range(args.steps):
        _, dt, _ = oracle_rate(osc, cam, per_step, 300 + k)
        times.append(dt)
    tot = sum(times)
    value = per_step * args.steps / tot / 1e6
    what = "the whole 1080p frame per step" if per_step == R else \
        f"{per_step} seeded rays of the 1080p frame per step"
    line = dict(metric=METRIC, value=value, unit="Mrays/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=tot / args.steps * 1e3, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference",
                config=dict(workload=WORKLOAD, sample=what),
                cpu_baseline=dict(value=value, unit="Mrays/s", cores=cores, kind="oracle",
                                  sample=what),
                e2e=dict(value=value, unit="Mrays/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


# --------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="salf", choices=["salf", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="headline only")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--workload", default="camera", choices=["camera", "lidar", "fisheye", "raster"],
                    help="sensor of the headline line (default: the 1080p camera by ray "
                         "casting; raster: the same camera by tile rasterisation)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_2507_18713_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    P.load()
    ctx = P.Context(local)

    sc = synth.driving_scene(2_000_000, seed=2)
    g = P.Scene(sc, dtype="f32", ctx=ctx)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # 2x L2
    wl = WORKLOADS[args.workload]
    cam = wl["sensor"]()
    want_int = wl["want_intensity"]
    outs = wl["outputs"]
    R = cam["width"] * cam["height"]
    out = {k: torch.empty((R, 3) if k == "rgb" else (R,), device="cuda") for k in outs}
    raster = args.workload == "raster"
    if raster:
        fn = lambda: g.render_raster(cam, out=out, outputs=outs, valid=False)
        rstats = {}
        g.render_raster(cam, out=out, outputs=outs, valid=False, stats=rstats)
        launches_per_step = rstats["kernels"]
    else:
        fn = lambda: g.render(cam, out=out, outputs=outs, valid=False, want_intensity=want_int)
        launches_per_step = 1

    sampler = ClockSampler(gpu_id_for(torch, local))
    for _ in range(args.warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ms = timed_renders(torch, fn, args.steps, 0, flush)
    clocks = sampler.stop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    g.check()
    n_counted = R
    if args.workload == "fisheye":
        n_counted = int(g.render(cam, outputs=("opacity",))["valid"].sum().item())
    rate, tot_ms = replica_throughput(sum(ms), n_counted, args.steps, dist, "cuda")
    avg = tot_ms / args.steps
    value = rate / 1e6

    nvis, _ = visits_of(torch, g, cam, want_int)
    bytes_alg = nvis * wl["b_field"] + R * wl["b_out"]
    peak, peak_kind = hbm_peak()
    achieved = bytes_alg / (avg * 1e-3) / 1e9
    traffic = None
    inst = None
    l2_bytes = None
    try:
        ent = json.load(open(TRAFFIC_FILE)).get(args.workload, {})
        if ent.get("kernel_hash") == kernel_hash(args.workload):
            traffic = ent.get("dram_bytes_per_launch")
            inst = ent.get("warp_inst_per_launch")
            l2_bytes = ent.get("l2_bytes_per_launch")
    except Exception:
        pass
    # L2 read bandwidth of this GPU (streaming reads of a 96 MiB buffer resident in L2; smaller
    # buffers give each thread too few loads per pass to reach it): the kernels take most of
    # their bytes from L1 and L2, so their L2 traffic is set against it
    l2_peak = None
    try:
        from paper_2507_18713_gb300 import _lib as _L2
        import ctypes as _C
        _g = _C.c_double(0.0)
        if _L2.load().salf_measure_l2_read(local, 96 << 20, 20, _C.byref(_g)) == 0:
            l2_peak = _g.value
    except Exception:
        pass
    # issue fraction: warp instructions of the launch (ncu smsp__inst_executed.sum)
    # over the issue slots of its duration (4 schedulers per SM, one
    # instruction per cycle each, at the median SM clock seen in the run)
    issue_frac = None
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    if inst and clocks.get("sm_mhz"):
        issue_frac = inst / (n_sm * 4 * clocks["sm_mhz"] * 1e6 * avg * 1e-3)
    from paper_2507_18713_gb300 import _lib as _L
    param_bytes = int(_L.load().salf_launch_param_bytes())

    # end to end through the C ABI with host output buffers (pinned)
    host = {k: torch.empty((R, 3) if k == "rgb" else (R,), dtype=torch.float32, pin_memory=True)
            for k in outs}
    if raster:  # device outputs, then copies into the pinned host buffers
        def e2e_call():
            g.render_raster(cam, out=out, outputs=outs, valid=False)
            for k in outs:
                host[k].copy_(out[k], non_blocking=True)
            torch.cuda.synchronize()
        e2e_how = "salf_render_raster, then copies of the outputs into pinned host buffers"
    else:
        def e2e_call():
            g.render_host(cam, out=host, want_intensity=want_int)
        e2e_how = ("HostFrames: salf_render_rays into device buffers on one stream, each "
                   "frame's outputs copied into page-locked host buffers by the copy engine on "
                   "a second stream while the next frame renders (two frames in flight, each in "
                   "its own buffers); every frame's results are in host memory, and waited for, "
                   "inside the timed region")
    e2e_steps = max(10, args.steps // 4)
    # synchronous calls, one frame at a time
    for _ in range(args.warmup):
        e2e_call()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_call()
    e2e_sync_s = time.perf_counter() - t0
    e2e_sync_value = world * n_counted * e2e_steps / e2e_sync_s / 1e6
    if raster:
        e2e_value = e2e_sync_value
    else:
        # pipelined: frame i renders into buffer set i % 2 while frame i - 1 finishes
        host2 = {k: torch.empty_like(v).pin_memory() for k, v in host.items()}
        sets = (host, host2)
        st = torch.cuda.current_stream()
        evs = (torch.cuda.Event(), torch.cuda.Event())

        def e2e_frames(n):
            for i in range(n):
                b = i & 1
                if i >= 2:
                    evs[b].synchronize()  # frame i - 2 is in host memory; its buffers are free
                g.render_host(cam, out=sets[b], want_intensity=want_int, sync=False, stream=st)
                evs[b].record(st)
            for i in range(max(0, n - 2), n):
                evs[i & 1].synchronize()

        e2e_frames(max(2, args.warmup))
        t0 = time.perf_counter()
        e2e_frames(e2e_steps)
        e2e_inplace_value = world * n_counted * e2e_steps / (time.perf_counter() - t0) / 1e6

        # device outputs + copy engine (HostFrames): frame i renders while frame i - 1 copies
        frames = P.HostFrames(g, cam, outputs=outs, depth=2, want_intensity=want_int)

        def e2e_copy_frames(n):
            prev = None
            for _ in range(n):
                slot = frames.submit(cam)
                if prev is not None:
                    frames.result(prev)  # frame i - 1 is in host memory
                prev = slot
            frames.result(prev)

        e2e_copy_frames(max(2, args.warmup))
        t0 = time.perf_counter()
        e2e_copy_frames(e2e_steps)
        e2e_s = time.perf_counter() - t0
        e2e_value = world * n_counted * e2e_steps / e2e_s / 1e6

    line = dict(metric=wl["metric"], value=value, unit="Mrays/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=avg, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=wl["workload"], l2="flushed between timed steps (256 MiB write)",
                            parallelism=f"replicas x{world}", fps=1e3 / avg,
                            visits_per_ray=nvis / R, t_min=1e-4),
                roofline=dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s",
                              frac=achieved / peak, traffic=traffic, issue_frac=issue_frac,
                              peak_source=f"{peak_kind} hbm_gbs",
                              bytes_per_launch=bytes_alg,
                              kernel="k_raster<F32,EXP> (whole pipeline timed)" if raster
                              else "k_forward<F32,EXP>",
                              note="bytes = visits x record scalars read + outputs per ray; "
                                   "visits counted by the kernel",
                              l2=dict(peak_gbs=l2_peak,
                                      bytes_per_launch=l2_bytes,
                                      achieved_gbs=(l2_bytes / (avg * 1e-3) / 1e9
                                                    if l2_bytes else None),
                                      frac=(l2_bytes / (avg * 1e-3) / 1e9 / l2_peak
                                            if l2_bytes and l2_peak else None),
                                      note="L2 traffic of the launch (ncu lts__t_sectors.sum x "
                                           "32 B, from the profile of these kernel sources) "
                                           "against the L2 read bandwidth measured here")),
                e2e=dict(value=e2e_value, unit="Mrays/s", sync_value=e2e_sync_value,
                         inplace_pipelined_value=None if raster else e2e_inplace_value,
                         h2d_bytes_per_step=param_bytes,
                         d2h_bytes_per_step=R * 4 * (len(outs) + 2 * ("rgb" in outs)),
                         how=e2e_how,
                         h2d_note="the launch's kernel parameters (sensor and request "
                                  "descriptor): rays are generated on the device and the scene "
                                  "is resident"),
                gpu_launches=args.steps * launches_per_step, clocks=clocks)

    if not args.no_extras and rank == 0:
        def extra(name, fn):
            try:
                line[name] = fn()
            except Exception as e:  # an extra section never costs the headline
                line[name] = {"error": f"{type(e).__name__}: {e}"}

        def issue_of(name, r):
            # warp instructions of the launch (ncu, at the current kernel sources)
            # over the issue slots of its measured duration
            try:
                ent = json.load(open(TRAFFIC_FILE)).get(name, {})
                if ent.get("kernel_hash") != kernel_hash(name) or not clocks.get("sm_mhz"):
                    return
                inst = ent["warp_inst_per_launch"]
                r["dram_bytes_per_launch"] = ent.get("dram_bytes_per_launch")
                r["issue_frac"] = inst / (n_sm * 4 * clocks["sm_mhz"] * 1e6 * r["ms"] * 1e-3)
            except Exception:
                pass

        def lidar_section():
            r = section(torch, P, g, driving_lidar(), max(50, args.steps // 4), args.warmup, flush,
                        B_FIELD_EXP_INT_F32, B_OUT_LIDAR, want_intensity=True)
            r["workload"] = "spinning LiDAR 128x2048, per-ray pose, intensity, same scene"
            r["roofline_frac"] = r["achieved_gbs"] / peak
            issue_of("lidar", r)
            return r

        def fisheye_section():
            fe = driving_fisheye()
            n_valid = int(g.render(fe, outputs=("opacity",))["valid"].sum().item())
            r = section(torch, P, g, fe, max(50, args.steps // 4), args.warmup, flush,
                        B_FIELD_EXP_F32, B_OUT_CAMERA, rays_counted=n_valid)
            r["workload"] = "equidistant fisheye 1920x1080 190deg, valid rays counted"
            r["roofline_frac"] = r["achieved_gbs"] / peak
            issue_of("fisheye", r)
            return r

        def raster_section():
            # Sec. V efficiency trade-off: ray casting vs tile rasterisation of
            # the same pinhole camera at four resolutions (outputs are equal)
            res = []
            for (w, h) in ((480, 270), (960, 540), (1920, 1080), (3840, 2160)):
                cam_r = synth.pinhole(w, h, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))
                n = w * h
                o = {k: torch.empty((n, 3) if k == "rgb" else (n,), device="cuda")
                     for k in ("rgb", "depth", "opacity")}
                st = {}
                g.render_raster(cam_r, out=o, valid=False, stats=st)
                k = max(20, args.steps // 10)
                ray_ms = statistics.median(timed_renders(
                    torch, lambda: g.render(cam_r, out=o, valid=False), k, args.warmup, flush))
                ras_ms = statistics.median(timed_renders(
                    torch, lambda: g.render_raster(cam_r, out=o, valid=False), k, args.warmup,
                    flush))
                res.append(dict(resolution=f"{w}x{h}", ray_ms=ray_ms, raster_ms=ras_ms,
                                ray_mrays_s=n / ray_ms / 1e3, raster_mrays_s=n / ras_ms / 1e3,
                                pairs=st["pairs"], visible_voxels=st["visible_voxels"],
                                faster="raster" if ras_ms < ray_ms else "ray"))
            return dict(workload="pinhole 60deg hFOV at (0,0,1.7) looking +x, driving scene "
                        "2,000,000 voxels (seed 2), FP32; median ms per frame, L2 flushed",
                        note="raster time includes projection, tile lists, sort and the one "
                             "host wait for the list size", points=res)

        def secondary_section():
            # Sec. V-C / Fig. 1: reflection and shadow rays spawned at the 1080p
            # frame's expected hit points, then traced through the same scene
            R = cam["width"] * cam["height"]
            prim = g.render(cam, outputs=("depth", "opacity"))
            rays = torch.empty((R, 8), device="cuda")
            o = {k: torch.empty((R, 3) if k == "rgb" else (R,), device="cuda")
                 for k in ("rgb", "depth", "opacity")}
            res = dict(workload="1080p pinhole frame of the driving scene; rays spawned where "
                       "opacity >= 0.5; L2 flushed; median ms")
            for kind, kw in (("reflect", {}), ("shadow", dict(light_dir=(0.4, 0.3, 1.0)))):
                gen = lambda: g.secondary_rays(cam, prim["depth"], prim["opacity"], kind=kind,
                                               out=rays, **kw)
                ms_gen = timed_renders(torch, gen, 20, args.warmup, flush)
                gen()
                torch.cuda.synchronize()
                spawned = int(rays[:, 3:6].abs().sum(dim=1).gt(0).sum().item())
                sen = P.rays_sensor(rays)
                tr = lambda: g.render(sen, outputs=("rgb", "depth", "opacity"), out=o, valid=False)
                ms_tr = timed_renders(torch, tr, 20, args.warmup, flush)
                t = statistics.median(ms_tr)
                res[kind] = dict(spawned=spawned, generate_ms=statistics.median(ms_gen),
                                 trace_ms=t, trace_mrays_s=spawned / (t * 1e-3) / 1e6)
            g.check()
            return res

        def actors_section():
            # Sec. IV-A: the same frames with 24 moving car-sized actors on the road
            tracks = synth.actor_tracks(24, seed=5)
            shapes = [(4.4, 1.9, 1.6), (3.9, 1.8, 1.5), (4.8, 2.0, 1.8)] * 8
            acts = [(P.Scene(synth.actor_shell(*d, seed=100 + k), ctx=ctx), p0, p1, (k + 1) << 22)
                    for k, (d, (p0, p1)) in enumerate(zip(shapes, tracks))]
            res = {}
            for name, sen, wi, outs_ in (("camera_1080p", cam if args.workload == "camera"
                                          else driving_camera(), False, ("rgb", "depth", "opacity")),
                                         ("lidar_128x2048", driving_lidar(), True,
                                          ("depth", "opacity", "intensity"))):
                n = sen["width"] * sen["height"]
                o = {k: torch.empty((n, 3) if k == "rgb" else (n,), device="cuda") for k in outs_}
                k = max(20, args.steps // 10)
                with_ms = statistics.median(timed_renders(
                    torch, lambda: g.render_actors(sen, acts, out=o, outputs=outs_, valid=False,
                                                   want_intensity=wi), k, args.warmup, flush))
                without_ms = statistics.median(timed_renders(
                    torch, lambda: g.render(sen, out=o, outputs=outs_, valid=False,
                                            want_intensity=wi), k, args.warmup, flush))
                res[name] = dict(with_actors_ms=with_ms, static_only_ms=without_ms,
                                 mrays_s=n / with_ms / 1e3)
            g.check()
            return dict(workload="driving scene 2,000,000 voxels (seed 2) + 24 car shells "
                        "(2.4k-3.2k voxels each, FP32) on lane tracks moving up to 15 m/s over "
                        "the 0.1 s exposure (seed 5); median ms per frame, L2 flushed",
                        note="static_only uses the ray kernel without actors", **res)

        extra("lidar", lidar_section)
        extra("fisheye", fisheye_section)
        extra("raster_vs_ray", raster_section)
        extra("secondary", secondary_section)
        extra("actors", actors_section)
        del g
        torch.cuda.empty_cache()
        extra("train_step", lambda: bench_backward(torch, P, args.steps, args.warmup, flush, peak))
        torch.cuda.empty_cache()
        extra("refine", lambda: bench_refine(torch, P, flush))
        torch.cuda.empty_cache()
        extra("serving", lambda: bench_serving(torch, P, args.serve_seconds))

    if rank == 0:
        try:
            import oracle
            oracle.build()
            osc = oracle.OracleScene(sc)
            n_s = R if args.workload in ("camera", "raster") else 131072
            ref = {}
            rate, dt, cores = oracle_rate(osc, cam, n_s, 99, outputs=ref)
            line["cpu_baseline"] = dict(value=rate, unit="Mrays/s", cores=cores, kind="oracle",
                                        sample=(f"the whole {cam['width']}x{cam['height']} frame"
                                                if n_s == R else f"{n_s} seeded rays of the frame")
                                        + f" ({dt:.1f} s wall)")
            if not args.no_extras and args.workload in ("camera", "raster"):
                try:
                    line["bf16_error"] = bf16_storage_error(torch, P, sc, osc, cam, ref)
                except Exception as e:
                    line["bf16_error"] = {"error": f"{type(e).__name__}: {e}"}
        except Exception as e:  # the baseline is reported, never required
            line["cpu_baseline"] = dict(value=None, unit="Mrays/s", cores=None, kind="oracle",
                                        sample=f"failed: {e}")
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
