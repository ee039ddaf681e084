"""Benchmark: one training step of hierarchical 3D Gaussian splatting on the 10M-splat
city workload at 3840x2160 with 16 KD subsets (forward, L1 loss, backward, Adam).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload city|object|tiny]

Prints one JSON line.  `value` is Mpix/s over all ranks (pixels rendered and
back-propagated per second of device time, inputs resident in HBM); `e2e` is the same
metric through the public training-step API with each step's target image copied from
pinned host memory and the loss read back.  `--impl reference` times the FP64 CPU
oracle on this host's cores on a bounded pixel sample of the same workload and
extrapolates to the full frame.  With N > 1 (torchrun) every rank trains its own replica
on its own cameras (the path does not shard on one GPU: replicas only).  The city run
also reports `serving`: p50/p99 latency and Mpix/s of the batched render server and of
the plain one-request-per-launch path on a Poisson stream over a 5M-splat scene.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd+Adam Mpix/s, 10M Gaussians, 3840x2160, 16 KD subsets"
WORKLOAD_NAMES = {"city": "city-10M-3840x2160-K16", "object": "object-1M-1600x1060-K8", "tiny": "tiny-4k-128px-K2",
                  "city-small": "city-1M-1920x1080-K16", "city-100m": "city-100M-3840x2160-K64"}
UNIT = "Mpix/s"
FP32_LANES_PER_SM = 128
MUFU_PER_SM_CLK = 16     # ex2 results per SM per clock (the SFU rate)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t_end = time.perf_counter() + 3.0      # sampling is running before the timed region starts
            while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
                time.sleep(0.005)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        for ln in self.lines[1:] if len(self.lines) > 1 else self.lines:   # the first predates the region
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- workloads
def make_workload(name, device):
    from paper_2406_11836_gb300 import workloads as W
    if name == "city":
        return W.city_10m(device=device)
    if name == "object":
        return W.object_1m(device=device)
    if name == "city-small":
        return W.city_10m(device=device, n=1_000_000, width=1920, height=1080, n_views=4)
    if name == "city-100m":
        return W.city_100m(device=device)
    return W.tiny(device=device)


# --------------------------------------------------------------------------- CPU oracle timing
def oracle_step_estimate(wl, budget_s=20.0, cam_index=0, threads=None):
    """Time the FP64 oracle on a bounded sample of one training step and extrapolate to
    the full frame: forward (Eq. 2) and adjoint over S sampled pixels with every splat
    projected, at two sample sizes to separate the per-pixel cost from the fixed cost;
    Adam (numpy float64) on 1% of the parameters, scaled."""
    from oracle import oracle as O
    from paper_2406_11836_gb300 import workloads as W
    cam = wl.cameras[cam_index]
    HW = cam.width * cam.height
    host = wl.scene.to("cpu")

    def run(S):
        pix = W.sample_pixels(cam.width, cam.height, S, seed=123)
        t0 = time.perf_counter()
        out = O.render(host, cam, pix=pix)
        g = np.sign(out["C"] - 0.5) / (3.0 * HW)
        O.adjoint(host, cam, g, pix=pix)
        return time.perf_counter() - t0

    S1 = 64
    t_start = time.perf_counter()
    t1 = run(S1)
    # grow the second sample until its extra pixels cost at least half the fixed part
    # (so the per-pixel slope is measured, not noise), within the time budget
    S2, t2 = min(8 * S1, HW), None
    while True:
        t2 = run(S2)
        spent = time.perf_counter() - t_start
        if t2 - t1 >= 0.5 * t1 or S2 >= min(16384, HW) or spent + 2.2 * t2 > budget_s:
            break
        S2 = min(4 * S2, HW)
    c = max((t2 - t1) / (S2 - S1), 1e-9)
    fixed = max(t1 - c * S1, 0.0)
    n_par = sum(int(t.numel()) for t in host.tensors())
    m = max(n_par // 100, 1)
    r = np.random.default_rng(0)
    p, gr = r.normal(size=m), r.normal(size=m)
    t0 = time.perf_counter()
    O.adam_step(p, gr, np.zeros(m), np.zeros(m), 1, 1e-3)
    t_adam = (time.perf_counter() - t0) * (n_par / m)
    step_s = fixed + c * HW + t_adam
    cores = threads or int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"{host.n} splats projected twice (forward, adjoint); blend+adjoint on {S1} and {S2} sampled "
              f"pixels, per-pixel cost extrapolated linearly to {cam.width}x{cam.height}; Adam on {m} of {n_par} "
              f"parameters, scaled; {t1 + t2:.1f} s of CPU work")
    return {"value": HW / step_s / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "step_s_extrapolated": step_s}


# --------------------------------------------------------------------------- roofline of the dominant kernel
# Algorithmic work per (pixel, splat) pair of the blend kernels, as the method counts it:
#   forward:  ~30 FP32 operations + 1 ex2 per evaluated pair (Mahalanobis distance through the
#             conic, the truncation tests, alpha, weight, colour and transmittance updates)
#   backward: ~70 FP32 operations + 1 ex2 per evaluated pair (the forward's replay plus the
#             adjoint of sigma and the 2D mean, conic, opacity and colour gradients)
# and per instance / pixel the bytes each must move (records once per staged instance, the
# partial maps, dL/dC, the per-splat 2D gradients).  The kernel's own finer count (an FMA as
# two operations: 14 per evaluated pair, +11 forward / +40 backward per contributing pair) is
# reported beside it.
FLOPS_PER_PAIR = {"blend_fwd": 30, "blend_bwd": 70}
FLOPS_EVAL = 14
FLOPS_CONTRIB = {"blend_fwd": 11, "blend_bwd": 40}


def sm_count():
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def stage_roofline(name, ms, launches, cnt, peaks, peak_src, geom):
    """Roofline of one pass: min-time bound = max(bytes / HBM peak, FP32 ops / FP32 peak,
    ex2 / SFU peak) over its launches; frac = bound / measured time."""
    avg_s = ms / 1e3 / launches
    sms = geom["sms"]
    clock_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6          # FLOP/s
    mufu_peak = sms * MUFU_PER_SM_CLK * clock_mhz * 1e6                 # ex2/s
    hbm = peaks["hbm_gbs"] * 1e9
    HW, K = geom["pixels"], geom["K"]
    per = lambda key: cnt.get(key, 0) / max(launches, 1)               # per launch
    flops = mufu = 0.0
    own = None
    if name == "blend_fwd":
        P = per("fwd_pairs")
        flops, mufu = FLOPS_PER_PAIR[name] * P, P
        # staged records; per pixel the image (and the partial maps when the forward writes them)
        byts = 36 * per("fwd_instances_staged") + (0 if geom.get("flat_backward") else 16 * K * HW) + 16 * HW
        own = FLOPS_EVAL * P + FLOPS_CONTRIB[name] * per("fwd_contrib")
    elif name == "blend_bwd":
        P = per("bwd_pairs")
        flops, mufu = FLOPS_PER_PAIR[name] * P, P
        # the backward replays the lists the forward staged; per pixel dL/dC and the image
        # (flat form) or dL/dC and the partial maps (per-subset form)
        per_pixel = 24 if geom.get("flat_backward") else 12 + 16 * K
        byts = per_pixel * HW + 36 * per("fwd_instances_staged") + 36 * per("visible")
        own = FLOPS_EVAL * P + FLOPS_CONTRIB[name] * per("bwd_contrib")
    else:
        I, Nv = per("instances"), per("visible")
        byts = {"instance_sort": 24 * I, "depth_sort": 24 * Nv, "emit": 8 * I, "ranges": 4 * I,
                "project": 44 * geom["N"] + 192 * Nv + 76 * Nv, "project_bwd": 48 * Nv + 236 * Nv * 2,
                "adam": 28 * geom["params"]}.get(name, 0.0)
    t_hbm, t_fp32, t_mufu = byts / hbm, flops / fp32_peak, mufu / mufu_peak
    t_min = max(t_hbm, t_fp32, t_mufu)
    if t_fp32 >= t_hbm and t_fp32 >= t_mufu and flops > 0:
        out = {"kernel": name, "bound": "alu", "achieved": flops / avg_s / 1e12, "peak": fp32_peak / 1e12,
               "unit": "TFLOP/s", "frac": t_min / avg_s,
               "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {clock_mhz:.0f} MHz (derived)",
               "peak_kind": "derived from unit counts and the measured max SM clock"}
    else:
        out = {"kernel": name, "bound": "hbm", "achieved": byts / avg_s / 1e9, "peak": peaks["hbm_gbs"],
               "unit": "GB/s", "frac": t_min / avg_s, "peak_kind": "of " + peak_src}
    out.update({"algorithmic_bytes": byts, "algorithmic_flops": flops, "ex2": mufu,
                "bound_ms": {"hbm": t_hbm * 1e3, "fp32": t_fp32 * 1e3, "sfu": t_mufu * 1e3},
                "avg_launch_ms": avg_s * 1e3, "launches": launches})
    if own is not None:
        out["own_count_tflops"] = own / avg_s / 1e12
    if name == "instance_sort":
        out["implementation_bytes"] = 20 * I * geom.get("sort_passes", 3)
    return out


def roofline(prof, peaks, peak_src, source, traffic_table, geom, workload=None):
    stages = prof["stages"]
    cnt = prof["counters"]
    cand = {k: v for k, v in stages.items() if v[1] > 0}
    dom = max(cand, key=lambda k: cand[k][0])
    out = stage_roofline(dom, cand[dom][0], cand[dom][1], cnt, peaks, peak_src, geom)
    t = traffic_table.get(dom)
    ok = t and t.get("source_sha") == source.get(t.get("source")) and t.get("workload") == workload
    out["traffic"] = t["dram_bytes_per_launch"] if ok else None
    # the next passes by time, same arithmetic (context for the dominant one)
    others = sorted(cand, key=lambda k: -cand[k][0])[1:4]
    out["next"] = {k: {kk: v for kk, v in stage_roofline(k, cand[k][0], cand[k][1], cnt, peaks, peak_src, geom).items()
                       if kk in ("bound", "achieved", "unit", "frac", "avg_launch_ms")} for k in others}
    for k in others:
        tk = traffic_table.get(k)
        if tk and tk.get("source_sha") == source.get(tk.get("source")) and tk.get("workload") == workload:
            out["next"][k]["traffic"] = tk["dram_bytes_per_launch"]
    return out


def _source_hashes():
    out = {}
    for f in ("raster.cu", "sort.cu", "project.cu", "adam.cu"):
        p = os.path.join(ROOT, "paper_2406_11836_gb300", "csrc", f)
        out[f] = hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]
    return out


def _traffic_table():
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


# --------------------------------------------------------------------------- serving
def run_serving(requests=3000, warm=200, rates=(200.0, 300.0), budget_gb=32, burst=400, device=None, lanes=4,
                max_slots=4):
    """Serving on the 5M-splat city scene (K=8): a seeded Poisson stream of mixed-resolution
    requests against the batched server and the plain one-request-per-launch server, at each
    offered rate of `rates` (the same requests, arrival gaps scaled; the first rate is the
    headline).  Latency = host time from submit to completion; Mpix/s = pixels of all
    requests over the wall time from the first arrival to the last completion.  The
    saturation figure submits `burst` requests at once."""
    import torch
    from paper_2406_11836_gb300 import rgs
    from paper_2406_11836_gb300 import workloads as W
    warm = min(warm, requests // 4)
    burst = min(burst, requests)
    wl = W.serving_5m(device=device)
    g = rgs.scene_c(wl.scene)
    kd = rgs.kd_partition(wl.scene, wl.depth_L)
    streams = {rate: W.request_stream(requests, rate_hz=rate, seed=7) for rate in rates}
    ring = 32   # output buffers per resolution, reused round robin
    outs = {(w, h): [torch.empty(3, h, w, device=device) for _ in range(ring)] for (w, h) in W.RESOLUTIONS}
    res = {}
    # batched: `lanes` concurrent lanes of up to `max_slots` requests per batch; lanes_only: the
    # same lanes with one request per batch (concurrency without batching; headline rate only);
    # plain: one request at a time through the render entry point
    # every server is sized for the stream's largest request (3840x2160)
    big = dict(max_width=max(w for w, _ in W.RESOLUTIONS), max_height=max(h for _, h in W.RESOLUTIONS))
    modes = {"batched": dict(max_slots=max_slots, lanes=lanes, plain=False, **big),
             "lanes_only": dict(max_slots=1, lanes=lanes, plain=False, **big),
             "plain": dict(max_slots=max_slots, lanes=lanes, plain=True, **big)}

    def measure(srv, stream):
        tickets = []
        t0 = time.perf_counter()
        for k, (ta, cam) in enumerate(stream):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0001)
            tickets.append((srv.submit(cam, outs[(cam.width, cam.height)][k % ring]), cam.width * cam.height))
        lats = [srv.wait(t, timeout_s=600) for t, _ in tickets]
        span = time.perf_counter() - t0
        L = np.array(lats[warm:])
        by_res = {}
        for (w, h) in W.RESOLUTIONS:
            Lr = np.array([lt for lt, (_, c) in zip(lats[warm:], stream[warm:]) if (c.width, c.height) == (w, h)])
            if len(Lr):
                by_res[f"{w}x{h}"] = {"p50_ms": float(np.percentile(Lr, 50)), "p99_ms": float(np.percentile(Lr, 99)),
                                      "n": int(len(Lr))}
        return {"p50_ms": float(np.percentile(L, 50)), "p99_ms": float(np.percentile(L, 99)),
                "mean_ms": float(L.mean()), "mpix_s": sum(px for _, px in tickets) / span / 1e6,
                "requests_measured": int(len(L)), "by_resolution": by_res}

    for mode, kw in modes.items():
        srv = rgs.Server(kd, g, rgs.default_opts(), int(budget_gb) << 30, keepalive=wl.scene, **kw)
        for (w, h), bufs in outs.items():     # warm every resolution once
            srv.wait(srv.submit(W.look_at((6.0, 6.0, 5.0), (0, 0, 0), w, h), bufs[0]))
        for ri, rate in enumerate(rates):
            if ri > 0 and mode == "lanes_only":
                continue
            st0 = srv.stats()
            entry = measure(srv, streams[rate])
            st = srv.stats()
            entry["mean_batch"] = (st["completed"] - st0["completed"]) / max(st["batches"] - st0["batches"], 1)
            if ri == 0:
                res[mode] = entry
            else:
                res.setdefault("rates", {}).setdefault(f"{rate:g}", {})[mode] = entry
        # saturation: everything queued at once
        st = srv.stats()
        sub = streams[rates[0]][:burst]
        t1 = time.perf_counter()
        bt = [srv.submit(cam, outs[(cam.width, cam.height)][k % ring]) for k, (_, cam) in enumerate(sub)]
        for t in bt:
            srv.wait(t, timeout_s=600)
        sat = sum(c.width * c.height for _, c in sub) / (time.perf_counter() - t1) / 1e6
        st2 = srv.stats()
        srv.close()
        sat_batches = max(st2["batches"] - st["batches"], 1)
        res[mode].update({"saturation_mpix_s": sat,
                          "saturation_mean_batch": (st2["completed"] - st["completed"]) / sat_batches,
                          "requeued": st2["requeued"], "max_slots": kw["max_slots"],
                          "lanes": 1 if kw["plain"] else lanes})
    torch.cuda.synchronize()
    res["config"] = {"workload": "serve-5M-K8", "splats": int(g.n), "subsets": kd.K,
                     "arrivals": f"Poisson, {requests} requests ({warm} warm-up) at each rate",
                     "rates_hz": list(rates), "resolutions": [f"{w}x{h}" for w, h in W.RESOLUTIONS],
                     "budget_gb": budget_gb, "max_slots": max_slots, "lanes": lanes,
                     "offered_mpix_s": {f"{r:g}": r * float(np.mean([w * h for w, h in W.RESOLUTIONS])) / 1e6
                                        for r in rates}}
    return res


def run_serve_only(args, rank, world, local_rank):
    """--workload serve: the serving measurement alone (one JSON line)."""
    import torch
    from paper_2406_11836_gb300 import build as B
    B.build()
    torch.cuda.set_device(local_rank)
    res = run_serving(requests=args.serve_requests, device=torch.device("cuda", local_rank))
    if rank == 0:
        b = res["batched"]
        print(json.dumps({"metric": "serve Mpix/s (5M Gaussians, K=8, Poisson 200 req/s, mixed resolutions)",
                          "value": b["mpix_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
                          "p50_ms": b["p50_ms"], "p99_ms": b["p99_ms"], "serving": res}), flush=True)


# --------------------------------------------------------------------------- multi-rank host logic
def shard_cameras(cams, rank, world):
    """Replicas: rank r renders cameras r, r + world, ... (a rank left without one reuses all)."""
    return cams[rank::world] or list(cams)


def reduce_max(vals, world, device="cpu"):
    """Element-wise max over ranks (the slowest rank's times); identity for one rank."""
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_mpix_s(world, steps, pix_per_step, ms_total):
    """Pixels of every rank's steps over the slowest rank's time, in Mpix/s (weak scaling)."""
    return world * steps * pix_per_step / (ms_total / 1e3) / 1e6


# --------------------------------------------------------------------------- arms
def partition_report(trainer) -> dict:
    """Subset balance of the median KD partition the step ran with, against a fixed grid of
    the same depth (untimed; the analogue of the paper's subset-balance table)."""
    from paper_2406_11836_gb300 import partition as Pt
    from paper_2406_11836_gb300 import workloads as W
    p = trainer.p
    scene = W.Scene(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"], trainer.sh_degree)
    keys = ("owned_max_over_mean", "owned_min_over_mean", "members_max_over_mean", "overlap")
    med = Pt.balance(trainer.kd, p["means"])
    grid = Pt.balance(Pt.kd_grid(scene, trainer.kd.L), p["means"])
    return {"subsets": med["subsets"], "median_kd": {k: round(med[k], 4) for k in keys},
            "fixed_grid": {k: round(grid[k], 4) for k in keys}}


def foot_reading_report(trainer, cams) -> dict:
    """Cost of the perpendicular-foot reading of x_i (Sec. 3.2) against the depth-plane
    reading the step uses: the forward with partial maps over every view, each timed with
    CUDA events (untimed warm-up pass first), then once more with per-stage timing.  The
    foot forward sorts every (tile, subset) run by a per-tile bound of the foot's ray
    parameter and restores each pixel's order in a 64-entry buffer; `overflow` counts the
    contributors that buffer blended early (0: exact order).  The foot reading's backward
    is timed on two views (`backward_ms`)."""
    import torch
    from paper_2406_11836_gb300 import rgs
    g = trainer.gaussians()
    opts = trainer.opts
    kd = trainer.kd
    dev = trainer.flat.device
    H, Wd = cams[0].height, cams[0].width
    tiles = ((H + 15) // 16) * ((Wd + 15) // 16)
    out = {"partial_C": torch.empty(kd.K, 3, H, Wd, device=dev), "partial_T": torch.empty(kd.K, H, Wd, device=dev),
           "image": torch.empty(3, H, Wd, device=dev), "T_final": torch.empty(H, Wd, device=dev),
           "tile_depth": torch.empty(tiles, kd.K, device=dev)}
    foot_out = {k: out[k] for k in ("partial_C", "partial_T", "image", "T_final")}
    ws = trainer.ws
    stream = torch.cuda.current_stream()

    def plane(c):
        rgs.render_fwd(kd, g, c, opts, ws, out=out)
        return 0

    def foot(c):
        return rgs.render_fwd_foot(kd, g, c, opts, ws, out=foot_out)["overflow"]

    res = {}
    for name, fn in (("depth_plane", plane), ("foot", foot)):
        for c in cams:
            fn(c)
        torch.cuda.synchronize()
        ms, over = [], 0
        for c in cams:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            over += fn(c)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        rgs.profile_enable(timing=True, counters=False)
        rgs.profile_read(reset=True)
        for c in cams:
            fn(c)
        torch.cuda.synchronize()
        prof = rgs.profile_read(reset=True)
        rgs.profile_enable(False, False)
        res[name] = {"forward_ms": round(float(np.mean(ms)), 3),
                     "stages_ms": {k: round(v[0] / len(cams), 3) for k, v in prof["stages"].items() if v[1] > 0},
                     "instances_per_view": prof["counters"]["instances"] / len(cams)}
        if name == "foot":
            res[name]["overflow_per_view"] = over / len(cams)
    res["views"] = len(cams)
    res["foot_over_depth_plane"] = round(res["foot"]["forward_ms"] / res["depth_plane"]["forward_ms"], 3)
    # the foot reading's backward (lists re-derived, per-pixel order replayed, pair adjoints
    # added with atomics, projection backward) after its image-only forward, on the first
    # two views with a seeded dL/dC; compare with variants.bwd_recompute (the depth-plane
    # backward that re-derives its lists)
    grads = [torch.zeros_like(t) for t in (trainer.p["means"], trainer.p["log_scales"], trainer.p["quats"],
                                           trainer.p["opacity_logits"], trainer.p["sh"])]
    gen = torch.Generator(device=dev).manual_seed(3)
    dL = (torch.randint(0, 2, (3, H, Wd), generator=gen, device=dev).float() * 2 - 1) / float(H * Wd)
    img = torch.empty(3, H, Wd, device=dev)
    bms, bover = [], 0
    bviews = cams[:2]
    for timed in (False, True):
        for c in bviews:
            rgs.render_fwd_foot(kd, g, c, opts, ws, partials=False, out={"image": img, "T_final": out["T_final"]})
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            o = rgs.render_bwd_foot(kd, g, c, opts, img, dL, grads, ws)
            e1.record(stream)
            torch.cuda.synchronize()
            if timed:
                bms.append(e0.elapsed_time(e1))
                bover += o
    res["foot"]["backward_ms"] = round(float(np.mean(bms)), 3)
    res["foot"]["backward_views"] = len(bviews)
    res["foot"]["backward_overflow_per_view"] = bover / len(bviews)
    del grads
    return res


def sort_passes(L, H, W):
    """Radix passes of the (tile, subset) instance sort: two wide passes for keys of 17 to 20
    bits, 8-bit digits otherwise."""
    tiles = ((H + 15) // 16) * ((W + 15) // 16)
    bits = max(0, (tiles - 1).bit_length()) + L
    return 2 if 16 < bits <= 20 else -(-bits // 8)


def variant_report(trainer, cams, targets, args) -> dict:
    """Untimed-for-the-headline comparisons on the same views (CUDA events on the launching
    stream, after a warm-up pass over every view):
      exact_partials: the step with every subset blended on every ray it meets (the partial
                      maps are the whole Eq. 3-4), against the headline's occlusion culling;
      backward_flat / backward_subsets: the step with the other backward form than the
                      headline's (flat: image-only forward and one replay of each pixel's
                      concatenated list; subsets: partial maps and the merge adjoint);
      one_group:      the headline step with the image-only forward binned in one group of
                      view ranks (group_binning = 0) instead of two;
      bwd_recompute:  the backward with a workspace that does not hold the forward's lists,
                      so it re-derives them (projection, binning, sorting) with the forward's
                      per-(tile, subset) depth table culling splats behind saturated tiles."""
    import torch
    from paper_2406_11836_gb300 import rgs
    stream = torch.cuda.current_stream()
    n = max(len(cams), 4)
    res = {}

    def timed(fn):
        for i in range(len(cams)):
            fn(i)
        torch.cuda.synchronize()
        rgs.profile_enable(timing=True, counters=False)
        rgs.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(n):
            fn(i)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = rgs.profile_read(reset=True)
        rgs.profile_enable(False, False)
        return e0.elapsed_time(e1) / n, {k: round(v[0] / n, 3) for k, v in prof["stages"].items() if v[1] > 0}

    step = lambda i: trainer.step(cams[i % len(cams)], targets[i % len(cams)], return_loss=False)
    saved, saved_bwd = trainer.opts, trainer.backward
    trainer.opts, trainer.backward = rgs.default_opts(cull_occluded=0), "subsets"
    ms, st = timed(step)
    res["exact_partials"] = {"ms_per_step": round(ms, 3), "stages_ms": st}
    # the other backward form than the headline's, same culled forward
    trainer.opts = saved
    trainer.backward = "flat" if saved_bwd == "subsets" else "subsets"
    ms, st = timed(step)
    res[f"backward_{trainer.backward}"] = {"ms_per_step": round(ms, 3), "stages_ms": st}
    trainer.backward = saved_bwd
    # the image-only forward binned in one group
    one = rgs.default_opts(cull_occluded=saved.cull_occluded, group_binning=0)
    trainer.opts = one
    ms, st = timed(step)
    res["one_group"] = {"ms_per_step": round(ms, 3), "stages_ms": st}
    trainer.opts = saved

    g = trainer.gaussians()
    ws2 = rgs.Workspace(trainer.flat.device)
    outs = {}

    def fwd(i):
        c = cams[i % len(cams)]
        outs[i % len(cams)] = rgs.render_fwd(trainer.kd, g, c, trainer.opts, trainer.ws, image=True)

    def bwd(i):
        c = cams[i % len(cams)]
        o = outs[i % len(cams)]
        dL = torch.sign(o["image"] - targets[i % len(cams)]).div_(float(o["image"].numel()))
        rgs.render_bwd(trainer.kd, g, c, trainer.opts, o["partial_C"], o["partial_T"], dL, trainer.grads(), ws2,
                       tile_depth=o["tile_depth"])

    rec = []
    rgs.profile_read(reset=True)
    for rep in range(2):   # a pass to warm up, then the timed one
        for i in range(len(cams)):
            fwd(i)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            rgs.profile_enable(timing=rep == 1, counters=False)
            e0.record(stream)
            bwd(i)
            e1.record(stream)
            torch.cuda.synchronize()
            rgs.profile_enable(False, False)
            if rep == 1:
                rec.append(e0.elapsed_time(e1))
    prof = rgs.profile_read(reset=True)
    trainer.grad.zero_()
    res["bwd_recompute"] = {"bwd_ms": round(float(np.mean(rec)), 3),
                            "stages_ms": {k: round(v[0] / len(cams), 3) for k, v in prof["stages"].items() if v[1] > 0},
                            "instances_per_view": prof["counters"]["instances"] / len(cams)}
    del outs, ws2
    torch.cuda.empty_cache()
    return res


def batch_report(device, B=4, steps=6) -> dict:
    """Training steps over B views per step (the object 1M workload: 1M splats, 1600x1060,
    8 subsets, SH degree 3): Trainer.step_batch through one batched launch sequence
    (rgs_render_batch_fwd/bwd) against the same steps view by view.  CUDA events on the
    launching stream around `steps` steps after two warm-up steps, each mode on a fresh
    trainer from the same scene."""
    import torch
    from paper_2406_11836_gb300 import workloads as W
    from paper_2406_11836_gb300.render import Trainer
    wl = W.object_1m(device=device)
    cams = wl.cameras[:B]
    targets = [W.target_image(c.width, c.height, seed=2000 + i, device=device) for i, c in enumerate(cams)]
    stream = torch.cuda.current_stream()
    res = {"workload": "object-1M-1600x1060-K8", "views_per_step": B, "steps": steps}
    for mode in ("sequential", "batched"):
        tr = Trainer(wl.scene, wl.depth_L, device=device, batched_views=(mode == "batched"))
        for _ in range(2):
            tr.step_batch(cams, targets, return_loss=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            tr.step_batch(cams, targets, return_loss=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        pix = sum(c.width * c.height for c in cams)
        res[mode] = {"ms_per_step": round(ms, 3), "mpix_s": round(pix / (ms / 1e3) / 1e6, 1)}
        del tr
        torch.cuda.empty_cache()
    res["batched_over_sequential"] = round(res["batched"]["mpix_s"] / res["sequential"]["mpix_s"], 3)
    return res


class OracleOneThread:
    """The oracle's step estimate with one host thread, in a fresh interpreter with
    OMP_NUM_THREADS=1 that touches no GPU; started at the beginning of the run so that its
    CPU time (about two minutes on the city workload) overlaps the GPU measurements."""

    def __init__(self, workload, budget_s=10.0):
        code = ("import json, sys; sys.path.insert(0, %r); import bench; "
                "wl = bench.make_workload(%r, 'cpu'); "
                "print(json.dumps(bench.oracle_step_estimate(wl, budget_s=%r, threads=1)))"
                % (ROOT, workload, budget_s))
        env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
        self.proc = subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                     text=True, env=env)

    def result(self, timeout_s=600) -> dict:
        try:
            out, _ = self.proc.communicate(timeout=timeout_s)
            d = json.loads(out.strip().splitlines()[-1])
            return {"value": d["value"], "unit": d["unit"], "cores": 1, "sample": d["sample"]}
        except Exception as e:   # reported, never fatal
            self.proc.kill()
            return {"unavailable": f"{type(e).__name__}: {e}"[:200]}


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2406_11836_gb300 import build as B
    B.build()
    from paper_2406_11836_gb300 import rgs
    from paper_2406_11836_gb300 import workloads as W
    from paper_2406_11836_gb300.render import Trainer

    one_thread = (OracleOneThread(args.workload, budget_s=args.cpu_budget / 2)
                  if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.profile_only else None)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = make_workload(args.workload, dev)
    cams = shard_cameras(wl.cameras, rank, world)
    H, Wd = cams[0].height, cams[0].width
    trainer = Trainer(wl.scene, wl.depth_L, device=dev)
    del wl.scene
    targets = [W.target_image(c.width, c.height, seed=1000 + i, device=dev) for i, c in enumerate(cams)]
    stream = torch.cuda.current_stream()

    def step(i):
        return trainer.step(cams[i % len(cams)], targets[i % len(cams)], return_loss=False)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    peaks, peak_src = _peaks()

    # ---- exact replay of the timed steps with the pair counters on (untimed): the counts
    # give the algorithmic work of the timed launches; the state is then restored
    counts = {}
    if not args.profile_only:
        ck = trainer.checkpoint()
        rgs.profile_enable(timing=False, counters=True)
        rgs.profile_read(reset=True)
        for i in range(args.steps):
            step(args.warmup + i)
        torch.cuda.synchronize()
        counts = rgs.profile_read(reset=True)["counters"]
        rgs.profile_enable(False, False)
        trainer.restore(ck)
        del ck
        torch.cuda.synchronize()

    # ---- device-timed region (inputs resident in HBM)
    rgs.profile_enable(timing=True, counters=False)
    rgs.profile_read(reset=True)
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    prof = rgs.profile_read(reset=True)
    rgs.profile_enable(False, False)
    prof["counters"] = dict(counts, kernel_launches=prof["counters"]["kernel_launches"])
    launches_timed = prof["counters"]["kernel_launches"]

    if args.profile_only:
        if rank == 0:
            print(json.dumps({"profile_only": True, "ms_per_step": ms / args.steps,
                              "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof["stages"].items()
                                                     if v[1] > 0}}), flush=True)
        return
    # ---- end to end through the public step API with host inputs
    pinned = [t.cpu().pin_memory() for t in targets]
    dev_target = torch.empty_like(targets[0])
    for j in range(max(len(cams), args.warmup)):           # untimed passes warm the loss path on every view
        dev_target.copy_(pinned[j % len(cams)], non_blocking=True)
        float(trainer.step(cams[j % len(cams)], dev_target, return_loss=True).item())
    torch.cuda.synchronize()
    host_ms = []
    # each step's target is copied from pinned host memory inside the timed region, on a
    # copy stream one step ahead of the step that uses it (two device buffers); a buffer is
    # refilled only after the step that used it returned its loss to the host
    bufs = [dev_target, torch.empty_like(dev_target)]
    copy_stream = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    main_stream = torch.cuda.current_stream()

    def prefetch(slot, view):
        with torch.cuda.stream(copy_stream):
            bufs[slot].copy_(pinned[view], non_blocking=True)
            ready[slot].record(copy_stream)

    e2e_clocks = ClockSampler(local_rank)
    e2e_clocks.start()
    t0 = time.perf_counter()
    prefetch(0, args.warmup % len(cams))
    for i in range(args.steps):
        ts = time.perf_counter()
        j = (args.warmup + i) % len(cams)
        if i + 1 < args.steps:
            prefetch((i + 1) & 1, (args.warmup + i + 1) % len(cams))
        main_stream.wait_event(ready[i & 1])
        loss = trainer.step(cams[j], bufs[i & 1], return_loss=True)
        float(loss.item())
        host_ms.append((time.perf_counter() - ts) * 1e3)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_clk = e2e_clocks.stop()
    print("e2e host ms per step:", [round(x, 1) for x in host_ms], file=sys.stderr)

    ms_max, e2e_ms_max = reduce_max([ms, e2e_s * 1e3], world, dev)
    pix_per_step = H * Wd
    value = whole_job_mpix_s(world, args.steps, pix_per_step, ms_max)
    e2e = whole_job_mpix_s(world, args.steps, pix_per_step, e2e_ms_max)
    geom = {"sms": sm_count(), "pixels": H * Wd, "K": trainer.kd.K, "N": trainer.n, "params": int(trainer.flat.numel()),
            "sort_passes": sort_passes(trainer.kd.L, H, Wd), "flat_backward": trainer.backward == "flat"}
    rl = roofline(prof, peaks, peak_src, _source_hashes(), _traffic_table(), geom, WORKLOAD_NAMES[args.workload])
    line = {
        "metric": METRIC if args.workload == "city" else f"fwd+bwd+Adam Mpix/s ({args.workload})",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded city-like scene and cameras)",
        "config": {"workload": WORKLOAD_NAMES[args.workload],
                   "splats": trainer.n, "width": Wd, "height": H, "subsets": trainer.kd.K, "sh_degree": trainer.sh_degree,
                   "step": "render fwd + L1 loss + render bwd + Adam", "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 (parameters, gradients and Adam state {trainer.n * 59 * 16 / 1e9:.1f} GB, "
                         "instance buffers several GB)"},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(targets[0].numel() * 4),
                "d2h_bytes_per_step": 4, "clocks": e2e_clk},
        "gpu_launches": int(launches_timed),
        "roofline": rl,
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof["stages"].items() if v[1] > 0},
        "counters_per_step": {k: v / args.steps for k, v in prof["counters"].items()},
        "clocks": clk,
    }
    if rank == 0:
        line["partition"] = partition_report(trainer)
    if rank == 0 and world == 1 and not args.no_variants:
        line["variants"] = variant_report(trainer, cams, targets, args)
    if rank == 0 and world == 1 and not args.no_foot:
        line["foot_reading"] = foot_reading_report(trainer, cams)
    if rank == 0 and world == 1 and not args.no_batches and args.workload == "city":
        line["view_batches"] = batch_report(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        wl_host = make_workload(args.workload, "cpu")
        line["cpu_baseline"] = oracle_step_estimate(wl_host, budget_s=args.cpu_budget)
        line["cpu_baseline"]["one_thread"] = one_thread.result() if one_thread else None
    if args.workload == "city" and not args.no_serve and world == 1:
        del trainer, targets, pinned, dev_target
        torch.cuda.empty_cache()
        line["serving"] = run_serving(requests=args.serve_requests, device=dev)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    import torch  # noqa: F401  (only for the generators)
    from paper_2406_11836_gb300 import workloads as W  # noqa: F401
    wl = make_workload(args.workload, "cpu")
    cam = wl.cameras[0]
    HW = cam.width * cam.height
    budget = max(5.0, 150.0 / max(args.steps + args.warmup, 1))
    vals = []
    est = None
    for i in range(args.warmup + args.steps):
        est = oracle_step_estimate(wl, budget_s=budget, cam_index=i % len(wl.cameras))
        if i >= args.warmup:
            vals.append(est["step_s_extrapolated"])
    step_s = float(np.mean(vals))
    value = HW / step_s / 1e6
    line = {"impl": "reference", "metric": METRIC if args.workload == "city" else f"fwd+bwd+Adam Mpix/s ({args.workload})",
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded city-like scene and cameras)",
            "config": {"workload": WORKLOAD_NAMES[args.workload], "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": est["cores"], "kind": "oracle",
                             "sample": est["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("city", "object", "tiny", "city-small", "city-100m", "serve"),
                    default="city")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-foot", action="store_true", help="skip the foot-reading forward comparison")
    ap.add_argument("--no-batches", action="store_true",
                    help="skip the batched multi-view training comparison (object 1M workload)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the exact-partials step and the recomputing backward comparisons")
    ap.add_argument("--serve-requests", type=int, default=3000, help="requests of the serving stream at each rate")
    ap.add_argument("--profile-only", action="store_true",
                    help="warm-up and timed steps only (no counter replay, end-to-end loop, CPU baseline or "
                         "serving): for launch lists under a profiler; its numbers are not bench values")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.workload == "serve":
        run_serve_only(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
