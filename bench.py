"""Benchmark: room-scale FP32 training step of the sparse-dense SDF renderer on one B300 (or N replicas).

Workload (synthetic stand-in for the paper's ScanNet rooms): a 6x6x3 m room with 10 seeded boxes / cylinders,
1 cm voxels in 8^3 blocks, blocks activated from 50 analytic 640x480 depth maps with a 4-voxel band; FP32 SDF,
RGB and fusion weight per voxel.  One step = 2^18 rays x 128 stratified samples through the fused
forward + L1 colour/depth loss + backward kernel, the loss reduction, and an Adam update of every voxel.

Prints one JSON line (see the keys below).  `--impl reference` times the CPU FP64 oracle instead.
"""
from __future__ import annotations

import argparse
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

METRIC = "fwd+bwd rays/s and samples/s on sparse-dense SDF grid; HBM GB/s; p50/p99 ms"
VS, BAND, N_VIEWS, W, H = 0.01, 4, 50, 640, 480
N_SAMPLES = 128
BETA = 0.5 * VS
LAMBDA_D = 0.1


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50,
                   help="timed steps (50 room steps are about 80 ms of device time, so that one stalled step moves "
                        "the mean by little)")
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--rays", type=int, default=1 << 18)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--parallel", default="replicas", choices=["replicas", "dp"],
                   help="N > 1: independent replicas (each rank its own batch), or one batch sharded by rays over "
                        "the ranks with an all-reduce of the gradients before the replicated optimiser step")
    p.add_argument("--no-prepare", action="store_true",
                   help="room step without the preparation pipeline (each batch ordered and walked inside its own "
                        "step instead of beside the previous step's optimiser)")
    p.add_argument("--no-extra", action="store_true",
                   help="room line without the precision / serving / apartment sub-measurements")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU baseline sample")
    p.add_argument("--views", type=int, default=N_VIEWS)
    p.add_argument("--max-blocks", type=int, default=80_000, help="grid capacity (room: 53,855 active blocks)")
    p.add_argument("--config", default="room", choices=["room", "room_bf16_sem", "serve", "apartment", "fusion",
                                                              "query", "crf"],
                   help="room: the headline training step; the others are the precision, serving and apartment "
                        "workloads (one JSON line each)")
    p.add_argument("--requests", type=int, default=2000, help="serve: requests per arrival rate")
    p.add_argument("--serve-scenes", default="0,1,2,3,4,5,6,7",
                   help="serve: which of the eight serving rooms to register (comma-separated indices)")
    p.add_argument("--order", default="pixel", choices=["pixel", "drawn"],
                   help="ray order inside a batch: grouped by view and pixel (a per-image loader) or as drawn")
    p.add_argument("--ray-order", default="auto", choices=["auto", "given", "surface"],
                   help="processing order of the fused pass (train_step_rays ray_order): auto puts batches of "
                        ">= 65536 rays in surface order on the GPU inside the step")
    return p.parse_args()


def _order_launches(args, n: int) -> int:
    """Kernels the surface ordering adds to a training step (bucket keys, bucket scan, scatter)."""
    return 3 if args.ray_order == "surface" or (args.ray_order == "auto" and n >= 65536) else 0


def _train_launches(args, n: int) -> int:
    """Kernels of one training pass: traversal, render (records), render (rays with more cells than a record
    holds), loss sum -- plus the surface ordering's."""
    return 4 + _order_launches(args, n)


def _stats(xs):
    """Median and p10 / p90 (and the mean) of per-step times in ms."""
    a = np.asarray(xs, np.float64)
    return {"median": round(float(np.median(a)), 4), "p10": round(float(np.percentile(a, 10)), 4),
            "p90": round(float(np.percentile(a, 90)), 4), "mean": round(float(a.mean()), 4)}


def _peak():
    """Measured HBM copy bandwidth (GB/s) and its source."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p))["hbm_gbs"], "measured"
    return 6400.0, "fallback"


def reduce_max(x: float, device=None) -> float:
    """Max of x over all ranks (identity without torch.distributed); the timing rule takes the slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = device if (device is not None and dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rays_per_s(world: int, rays_per_rank: int, ms_per_step_max: float) -> float:
    """Whole-job throughput: the rays all ranks processed in one step over the slowest rank's step time."""
    return world * rays_per_rank / (ms_per_step_max / 1e3)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


# ----------------------------------------------------------------------------------------------------------
# Workload construction
# ----------------------------------------------------------------------------------------------------------
def build_workload(sdg, torch, device, n_views, rays_per_step, n_batches=4, seed=0, max_blocks=80_000,
                   order="pixel"):
    import synth
    sc = synth.scene_room(seed)
    poses = synth.random_poses(sc, n_views, seed=seed)
    K = synth.intrinsics(W, H)
    t0 = time.time()
    depths = [synth.depth_map(sc, T, W, H, K, device=device) for T in poses]
    torch.cuda.synchronize()
    t_depth = time.time() - t0
    G = sdg.Grid(VS, max_blocks, beta=BETA)
    # activation: timed separately, all 50 maps in one batch (one synchronisation)
    depth_all = torch.stack(depths).contiguous()
    T_all = np.stack([np.asarray(T, np.float64) for T in poses])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    G.activate_depth_frames(depth_all, K, T_all, BAND)
    ev1.record()
    torch.cuda.synchronize()
    act_ms = ev0.elapsed_time(ev1)
    nb = G.num_blocks
    keys = G.keys().cpu().numpy()
    vals = synth.fill_grid(sc, keys, VS, BAND, device=device)
    A = sdg._abi
    geo = G.channel(A.GROUP_GEO)
    geo[:nb, :, 0] = vals["sdf"].to(torch.float32)
    geo[:nb, :, 1:4] = vals["rgb"].to(torch.float32)
    G.channel(A.GROUP_WEIGHT)[:nb, :, 0] = 1.0
    del vals
    batches = []
    for b in range(n_batches):
        tb = synth.training_batch(sc, poses, W, H, K, rays_per_step, seed=1000 * seed + b, device=device,
                                  order=order)
        batches.append({k: v.contiguous() for k, v in tb.items()})
    torch.cuda.synchronize()
    return {"scene": sc, "poses": poses, "K": K, "grid": G, "keys": keys, "batches": batches, "act_ms": act_ms,
            "depth_s": t_depth}


# ----------------------------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ----------------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "power_w_max": max(power) if power else None, "samples": len(sm)}


# ----------------------------------------------------------------------------------------------------------
# CPU oracle leg (baseline and algorithmic byte counts)
# ----------------------------------------------------------------------------------------------------------
def oracle_grid(wl, torch, sdg):
    import oracle
    G = wl["grid"]
    A = sdg._abi
    nb = G.num_blocks
    geo = G.channel(A.GROUP_GEO)[:nb].double().cpu().numpy()
    return oracle.Grid(VS, BETA).set(wl["keys"], geo[..., 0], geo[..., 1:4])


def cpu_leg(O, batch, seconds, N=N_SAMPLES):
    """Times the oracle's forward + loss + backward on successive 256-ray chunks of the batch until `seconds`
    of CPU time are spent; returns rays/s and the sample description."""
    import oracle
    perm = np.random.default_rng(0).permutation(batch["rays"].shape[0])   # a sample spread over all views
    rays = batch["rays"].cpu().numpy()[perm]
    t_rgb = batch["rgb"].double().cpu().numpy()[perm]
    t_d = batch["depth"].double().cpu().numpy()[perm]
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds and done < len(rays):
        sl = slice(done, min(done + 256, len(rays)))
        out = O.render(rays[sl], N, seed=0, ray_id0=done)
        _, g = oracle.loss(out["rgb"], out["depth"], t_rgb[sl], t_d[sl], LAMBDA_D)
        O.backward(rays[sl], N, g["rgb"], g["depth"], seed=0, ray_id0=done)
        done = sl.stop
    el = time.perf_counter() - t0
    return done / el, done, el


def bytes_per_ray(O, batch, n=1024, N=N_SAMPLES):
    """Algorithmic bytes per ray of the fused training kernel, from the oracle's count of the distinct voxels
    and blocks each ray's stencils touch: voxels x (16 B read + 16 B grad read + 16 B grad write),
    blocks x 40 B (16-B hash slot + 24 B of neighbour table on average... counted as 40 B), ray 32 B,
    targets 16 B, loss 4 B."""
    idx = np.linspace(0, batch["rays"].shape[0] - 1, n).astype(np.int64)   # spread over all views of the batch
    rays = batch["rays"][idx].cpu().numpy()
    vx, bl = O.count_touched(rays, N, seed=0)
    per_ray = vx * 48.0 + bl * 40.0 + 32 + 16 + 4
    return float(per_ray.mean()), float(vx.mean()), float(bl.mean())


# Sources of the fused training kernel: a DRAM-traffic capture is valid only for the build it was taken on.
KERNEL_SOURCES = ["paper_2305_13220_b300/csrc/render_core.cuh", "paper_2305_13220_b300/csrc/render_kernels.cuh",
                  "paper_2305_13220_b300/csrc/common.cuh", "paper_2305_13220_b300/csrc/render_inst_f32_bwd.cu"]


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(kernel: str):
    """(DRAM bytes per launch, note) from the ncu capture summarised in profiles/<kernel>_traffic.txt.  The file
    records the hash of the kernel's sources it was captured on; a capture of other sources gives (None, why)."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    if not os.path.exists(p):
        return None, "no capture"
    val, sha = None, None
    for ln in open(p):
        if ln.startswith("traffic_bytes_per_launch:"):
            try:
                val = float(ln.split(":", 1)[1])
            except ValueError:
                val = None
        if ln.startswith("source_sha16:"):
            sha = ln.split(":", 1)[1].strip()
    cur = kernel_source_hash()
    if sha != cur:
        return None, f"capture is of other kernel sources ({sha}, built {cur}): traffic not reported"
    return val, f"ncu capture of these sources ({cur})"


# ----------------------------------------------------------------------------------------------------------
# Serving measurement (p50 / p99 latency)
# ----------------------------------------------------------------------------------------------------------
def serve_leg(sdg, torch, wl, n_requests=200, seed=0):
    import synth
    srv = sdg.Server(hbm_budget_bytes=2 << 30, max_slots=32, n_streams=4, chunk_rays=4096, max_batch_rays=1 << 18)
    sid = srv.add_scene(wl["grid"])
    rng = np.random.default_rng(seed)
    res = [(160, 120), (320, 240), (640, 480), (1280, 960)]
    sc = wl["scene"]
    poses = synth.random_poses(sc, 16, seed=77)
    # warm-up
    t = srv.submit(sid, 120, 160, synth.intrinsics(160, 120), poses[0], n_samples=N_SAMPLES)
    srv.wait(t, 120000)
    srv.release(t)
    # open loop at a rate of about 80% of a quick capacity estimate
    t0 = time.perf_counter()
    tk = [srv.submit(sid, 480, 640, synth.intrinsics(640, 480), poses[i % 16], n_samples=N_SAMPLES, seed=i)
          for i in range(8)]
    for t in tk:
        srv.wait(t, 120000)
        srv.release(t)
    cap_rays_s = 8 * 640 * 480 / (time.perf_counter() - t0)
    mean_rays = np.mean([w * h for w, h in res])
    rate = 0.8 * cap_rays_s / mean_rays
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    sizes = [res[int(rng.integers(0, 4))] for _ in range(n_requests)]
    start = time.perf_counter()
    lat, rays = _open_loop(srv, n_requests, arrivals,
                           lambda i: (sid, sizes[i][1], sizes[i][0], synth.intrinsics(*sizes[i]), poses[i % 16]), start)
    elapsed = time.perf_counter() - start
    srv.close()
    return {"requests": n_requests, "rate_req_s": round(rate, 2), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "rays_per_s": round(rays / elapsed, 1),
            "resolutions": "uniform over 160x120, 320x240, 640x480, 1280x960", "samples_per_ray": N_SAMPLES,
            "arrivals": "Poisson at 0.8x measured saturated capacity"}


# ----------------------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    import paper_2305_13220_b300 as sdg
    device = f"cuda:{local}"
    dp_mode = args.parallel == "dp" and world > 1
    # data parallel: every rank holds the same grid and batch and renders its shard of it
    wl = build_workload(sdg, torch, device, args.views, args.rays, seed=0 if dp_mode else rank,
                        max_blocks=args.max_blocks, order=args.order)
    G = wl["grid"]
    n = args.rays
    stream = torch.cuda.current_stream()
    loss_sum = torch.zeros(1, device=device)

    # Preparation pipeline: batch i + 1's ordering and traversal are enqueued (on the grid's auxiliary stream)
    # after batch i's training pass and before its optimiser step, so they run beside the HBM-bound optimiser.
    # prep[0] is the slot batch i was prepared in (None: not prepared).
    pipelined = not args.no_prepare and not dp_mode
    prep = [None]

    def train(b, seed, ev=None):
        sdg.train_step_rays(G, b["rays"], b["rgb"], b["depth"], n_samples=N_SAMPLES, seed=seed,
                            lambda_depth=LAMBDA_D, loss_sum=loss_sum, ray_order=args.ray_order, prepared=prep[0])
        if ev is not None:
            ev.record(stream)

    def prepare_next(b_next):
        if pipelined and b_next is not None:
            slot = 0 if prep[0] is None else 1 - prep[0]
            sdg.train_prepare(G, b_next["rays"], b_next["depth"], slot, ray_order=args.ray_order)
            prep[0] = slot
        else:
            prep[0] = None

    def step(b, b_next=None):
        if dp_mode:
            from paper_2305_13220_b300 import dp
            dp.data_parallel_step(G, b["rays"], b["rgb"], b["depth"], rank, world, n_samples=N_SAMPLES,
                                  seed=stepno[0], lambda_depth=LAMBDA_D, loss_sum=loss_sum, ray_order=args.ray_order)
            return
        train(b, stepno[0])
        prepare_next(b_next)
        G.adam_step(lr=1e-3)

    nb_ = len(wl["batches"])
    stepno = [0]
    for i in range(args.warmup):
        stepno[0] = i
        step(wl["batches"][i % nb_], wl["batches"][(i + 1) % nb_])
    torch.cuda.synchronize()
    # phase timing, all with CUDA events on the grid's stream: the training pass (ordering, traversal, render
    # kernels, loss sum), the render kernels alone (recorded by the library around them), the optimiser
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    kev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    for e in kev:  # the events exist once recorded
        e[0].record(stream)
        e[1].record(stream)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(K):
        b = wl["batches"][(args.warmup + i) % nb_]
        stepno[0] = 1000 + i
        G.set_pass_events(kev[i][0], kev[i][1])
        evs[i][0].record(stream)
        if dp_mode:  # this rank's shard, then the gradient all-reduce with the optimiser step
            from paper_2305_13220_b300 import dp
            dp.shard_train(G, b["rays"], b["rgb"], b["depth"], rank, world, n_samples=N_SAMPLES, seed=stepno[0],
                           lambda_depth=LAMBDA_D, loss_sum=loss_sum, ray_order=args.ray_order)
            evs[i][1].record(stream)
            dp.all_reduce_grads(G)
        else:
            train(b, stepno[0], evs[i][1])
            prepare_next(wl["batches"][(args.warmup + i + 1) % nb_])
        G.adam_step(lr=1e-3)
        evs[i][2].record(stream)
    end.record(stream)
    G.set_pass_events()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = reduce_max(start.elapsed_time(end), device)
    train_t = [e[0].elapsed_time(e[1]) for e in evs]
    kern_t = [e[0].elapsed_time(e[1]) for e in kev]
    adam_t = [e[1].elapsed_time(e[2]) for e in evs]
    step_t = [e[0].elapsed_time(e[2]) for e in evs]
    train_ms, kern_ms, adam_ms = (float(np.median(x)) for x in (train_t, kern_t, adam_t))
    ms_step = total_ms / K
    # replicas: every rank a whole batch; data parallel: one batch over all ranks
    value = (n / (ms_step / 1e3)) if dp_mode else aggregate_rays_per_s(world, n, ms_step)

    # the same steps without the preparation pipeline, for comparison (not the headline)
    unprepared_ms = None
    if pipelined:
        prep[0] = None
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        for i in range(K):
            b = wl["batches"][i % nb_]
            sdg.train_step_rays(G, b["rays"], b["rgb"], b["depth"], n_samples=N_SAMPLES, seed=2000 + i,
                                lambda_depth=LAMBDA_D, loss_sum=loss_sum, ray_order=args.ray_order)
            G.adam_step(lr=1e-3)
        u1.record(stream)
        torch.cuda.synchronize()
        unprepared_ms = u0.elapsed_time(u1) / K

    # unfused forward and backward of the same batches (timed apart; not part of the headline step)
    fb = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    for i in range(K):
        b = wl["batches"][i % len(wl["batches"])]
        fb[i][0].record(stream)
        o = sdg.render(G, b["rays"], N_SAMPLES, seed=3000 + i, want_ctx=True)
        fb[i][1].record(stream)
        _, gs = sdg.loss_l1(G, o["rgb"], o["depth"], b["rgb"], b["depth"], lambda_depth=LAMBDA_D)
        sdg.backward(o["ctx"], gs["rgb"], gs["depth"])
        fb[i][2].record(stream)
        o["ctx"].release()
    torch.cuda.synchronize()
    G.zero_grad()
    fwd_t = [e[0].elapsed_time(e[1]) for e in fb]
    bwd_t = [e[1].elapsed_time(e[2]) for e in fb]

    # end to end through the public API: every step's rays and targets are copied from pinned host memory and its
    # loss is read back, inside the timed region.  Two device input buffers: while step k computes on the
    # grid's stream, step k+1's inputs upload on a copy stream (events order the two).
    hb = [{k: v.cpu().pin_memory() for k, v in b.items() if k in ("rays", "rgb", "depth")} for b in wl["batches"]]
    dev_in = [{k: torch.empty_like(v) for k, v in wl["batches"][0].items() if k in ("rays", "rgb", "depth")}
              for _ in range(2)]
    host_loss = torch.empty(1, pin_memory=True)
    h2d = sum(v.numel() * v.element_size() for v in hb[0].values())
    copy_stream = torch.cuda.Stream()
    uploaded = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]

    def upload(i, slot):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(consumed[slot])
            for k in dev_in[slot]:
                dev_in[slot][k].copy_(hb[i % len(hb)][k], non_blocking=True)
            uploaded[slot].record(copy_stream)

    def e2e_steps(count):
        for s_ in range(2):
            consumed[s_].record(stream)
        upload(0, 0)
        prep[0] = None
        stream.wait_event(uploaded[0])
        prepare_next(dev_in[0])
        for i in range(count):
            slot = i % 2
            if i + 1 < count:
                upload(i + 1, 1 - slot)
            stream.wait_event(uploaded[slot])
            stepno[0] = 4000 + i
            train(dev_in[slot], stepno[0])
            if i + 1 < count:
                stream.wait_event(uploaded[1 - slot])  # the next batch's inputs, for its preparation
                prepare_next(dev_in[1 - slot])
            else:
                prep[0] = None
            G.adam_step(lr=1e-3)
            consumed[slot].record(stream)
            host_loss.copy_(loss_sum, non_blocking=True)

    e2e_steps(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_steps(K)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1) / K, device)
    e2e_value = (n / (e2e_ms / 1e3)) if dp_mode else aggregate_rays_per_s(world, n, e2e_ms)

    res = None
    if rank == 0:
        nb = G.num_blocks
        params = nb * 512 * 4
        adam_bytes = params * 32
        line = {"metric": METRIC, "value": round(value, 1), "unit": "rays/s", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
                "scaling": "strong" if dp_mode else "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "room-scale FP32 training step (6x6x3 m room, 10 boxes/cylinders, 1 cm "
                                       "voxels, 8^3 blocks, 4-voxel band from 50 640x480 depth maps; 2^18 rays "
                                       "x 128 stratified samples, L1 colour + 0.1 L1 depth, Adam on every voxel)",
                           "rays_per_step": n, "samples_per_ray": N_SAMPLES, "n_blocks": nb,
                           "ray_order": args.ray_order + (" (surface order, sorted on the GPU inside the step)"
                                                          if _order_launches(args, n) else ""),
                           "voxels": nb * 512, "params": params,
                           "parallelism": (f"dp{world} (ray shards, gradient all-reduce)" if dp_mode else
                                           f"replicas{world}" if world > 1 else "single"),
                           "l2": "inputs larger than L2: each step streams the whole grid and Adam state "
                                 f"({adam_bytes / 1e9:.1f} GB) through HBM"},
                "samples_per_s": round(value * N_SAMPLES, 1),
                "phases": {"train_kernel_ms": round(train_ms, 4), "render_kernels_ms": round(kern_ms, 4),
                           "adam_ms": round(adam_ms, 4), "activation_ms_50_maps": round(wl["act_ms"], 3)},
                "timing": {"step_ms": _stats(step_t), "train_pass_ms": _stats(train_t),
                           "pipeline": ("each batch's ordering and traversal prepared on the grid's auxiliary "
                                        "stream beside the previous step's optimiser (sdg_train_prepare); the "
                                        "same steps unprepared: " + (f"{unprepared_ms:.4f} ms per step"
                                                                    if unprepared_ms else "not run"))
                           if pipelined else "none",
                           "render_kernels_ms": _stats(kern_t), "adam_ms": _stats(adam_t),
                           "unfused_forward_ms": _stats(fwd_t), "unfused_loss_backward_ms": _stats(bwd_t),
                           "note": "CUDA events on the grid's stream; the train pass holds the render kernels "
                                   "and the loss sum (and, without the preparation pipeline, the surface ordering "
                                   "and the traversal); the render kernels are timed by events the library "
                                   "records around them (sdg_grid_set_pass_events)"},
                "clocks": clk, "gpu_launches": (_train_launches(args, n) + 1) * K,
                "e2e": {"value": round(e2e_value, 1), "unit": "rays/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4}}
        peak, peak_src = _peak()
        adam_gbs = adam_bytes / (adam_ms / 1e3) / 1e9
        O = None
        bpr = None
        if not args.no_cpu_baseline:
            O = oracle_grid(wl, torch, sdg)
            bpr, vx, bl = bytes_per_ray(O, wl["batches"][0])
            rate, done, el = cpu_leg(O, wl["batches"][0], args.cpu_seconds)
            line["cpu_baseline"] = {"value": round(rate, 2), "unit": "rays/s", "cores": 1, "kind": "oracle",
                                    "sample": f"{done} rays of the first batch (fwd + L1 loss + bwd, FP64, "
                                              f"single thread, {el:.1f} s)"}
            del O
        if bpr:
            kern_gbs = bpr * n / (kern_ms / 1e3) / 1e9
            traffic, tnote = read_traffic("k_render_train")
            line["roofline"] = {"kernel": "k_render_train", "bound": "hbm", "achieved": round(kern_gbs, 1),
                                "peak": peak, "unit": "GB/s", "frac": round(kern_gbs / peak, 4), "traffic": traffic,
                                "traffic_note": tnote, "peak_source": peak_src,
                                "algorithmic_bytes_per_launch": round(bpr * n),
                                "launch_ms_median": round(kern_ms, 4),
                                "note": "the fused training pass's render kernels (records kernel + in-warp "
                                        "kernel for rays beyond the record capacity), algorithmic bytes from the "
                                        "oracle's count over their median duration; over the training pass as "
                                        f"timed (train_pass_ms) {bpr * n / (train_ms / 1e3) / 1e9:.1f} GB/s"}
            line["roofline_other"] = {"kernel": "k_opt_f32", "achieved": round(adam_gbs, 1),
                                      "frac": round(adam_gbs / peak, 4), "unit": "GB/s",
                                      "algorithmic_bytes_per_launch": adam_bytes}
            line["train_kernel_bytes_per_ray"] = {"value": round(bpr, 1), "distinct_voxels": round(vx, 1),
                                                  "distinct_blocks": round(bl, 2), "rays_counted": 1024}
        else:
            line["roofline"] = {"kernel": "k_opt_f32", "bound": "hbm", "achieved": round(adam_gbs, 1), "peak": peak,
                                "unit": "GB/s", "frac": round(adam_gbs / peak, 4), "traffic": None,
                                "peak_source": peak_src, "algorithmic_bytes_per_launch": adam_bytes,
                                "note": "run without the oracle's byte count (--no-cpu-baseline): the optimiser"}
        if world == 1 and not args.no_extra:
            # the other workloads, measured after the headline step (each with its own grid)
            line["precision"] = measure_precision(args, compact=True)
            if not args.no_serve:
                line["serve"] = measure_serve(args, compact=True)
            line["apartment"] = measure_apartment(args, compact=True)
        elif not args.no_serve:
            line["serve"] = serve_leg(sdg, torch, wl)
        res = line
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return res


# ----------------------------------------------------------------------------------------------------------
# Other workloads: precision variant, serving, apartment
# ----------------------------------------------------------------------------------------------------------
def _prepared_steps(sdg, G, batches, train, ray_order):
    """A step function over `batches` in cyclic order, pipelined as the room step is: after each batch's training
    pass the next batch's ordering and traversal are enqueued on the grid's auxiliary stream (sdg_train_prepare),
    beside the optimiser step.  train(batch, seed, prepared_slot) runs the training pass."""
    st = {"k": 0, "slot": None}

    def step(_b, seed):
        nb = len(batches)
        b, nxt = batches[st["k"] % nb], batches[(st["k"] + 1) % nb]
        train(b, seed, st["slot"])
        slot = 0 if st["slot"] is None else 1 - st["slot"]
        sdg.train_prepare(G, nxt["rays"], nxt["depth"], slot, ray_order=ray_order)
        st["slot"] = slot
        st["k"] += 1
        G.adam_step(lr=1e-3)
    return step


def _timed_steps(torch, step, batches, K, W_):
    for i in range(W_):
        step(batches[i % len(batches)], i)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for i in range(K):
        step(batches[i % len(batches)], 1000 + i)
    s1.record()
    torch.cuda.synchronize()
    return s0.elapsed_time(s1) / K


def _phase_times(torch, sdg, G, batches, K, train):
    """Median CUDA-event times of the training pass, of its render kernels (events the library records around
    them) and of the optimiser step."""
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    for e in ev:  # the library records the pass events; they exist once recorded here
        e[3].record()
        e[4].record()
    for i in range(K):
        G.set_pass_events(ev[i][3], ev[i][4])
        ev[i][0].record()
        train(batches[i % len(batches)], 2000 + i)
        ev[i][1].record()
        G.adam_step(lr=1e-3)
        ev[i][2].record()
    G.set_pass_events()
    torch.cuda.synchronize()
    return {"train_kernel_ms": round(float(np.median([e[0].elapsed_time(e[1]) for e in ev])), 4),
            "render_kernels_ms": round(float(np.median([e[3].elapsed_time(e[4]) for e in ev])), 4),
            "adam_ms": round(float(np.median([e[1].elapsed_time(e[2]) for e in ev])), 4)}


def _activate_views(sdg, torch, G, sc, poses, K, device, band):
    """Activates the grid from the views' depth maps in one batch; returns its time in ms (maps made beforehand)."""
    import synth
    depth_all = torch.stack([synth.depth_map(sc, T, W, H, K, device=device) for T in poses]).contiguous()
    T_all = np.stack([np.asarray(T, np.float64) for T in poses])
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    G.activate_depth_frames(depth_all, K, T_all, band)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    del depth_all
    return ms


def _fill(sdg, torch, G, sc, vs, band, device, n_sem=0):
    import synth
    A = sdg._abi
    keys = G.keys().cpu().numpy()
    nb = len(keys)
    vals = synth.fill_grid(sc, keys, vs, band, n_sem=n_sem, device=device)
    if G.rgb_dtype == "f32":
        geo = G.channel(A.GROUP_GEO)
        geo[:nb, :, 0] = vals["sdf"].to(torch.float32)
        geo[:nb, :, 1:4] = vals["rgb"].to(torch.float32)
    else:
        G.channel(A.GROUP_SDF)[:nb, :, 0] = vals["sdf"].to(torch.float32)
        ch = G.channel(A.GROUP_RGB)
        ch[:nb, :, 0:3] = vals["rgb"].to(torch.bfloat16)
        ch[:nb, :, 3] = 0
    if n_sem:
        G.channel(A.GROUP_SEM)[:nb] = vals["sem"].to(torch.bfloat16)
    return keys, vals


def _line(value, unit, K, W_, ms, config, **extra):
    d = {"metric": METRIC, "value": round(value, 1), "unit": unit, "n_gpus": 1, "steps": K, "warmup": W_,
         "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
         "dtype": "f32", "data": "synthetic", "config": config}
    d.update(extra)
    return d


def _open_loop(srv, n_requests, arrivals, make_req, start, n_samples=N_SAMPLES):
    """Submits request i at time arrivals[i] (open loop) while a consumer thread waits for results in order and
    releases them, as a client that reads its frames would.  Returns (latencies ms, rays rendered)."""
    import queue
    q = queue.Queue()
    lat, tot = [], [0]

    def consume():
        while True:
            item = q.get()
            if item is None:
                return
            t, nr = item
            r = srv.wait(t, 600000)
            lat.append(r.t_done_ms - r.t_submit_ms)
            tot[0] += nr
            srv.release(t)

    th = threading.Thread(target=consume, daemon=True)
    th.start()
    for i in range(n_requests):
        while time.perf_counter() - start < arrivals[i]:
            time.sleep(0.0001)
        s, h, w, Kq, T = make_req(i)
        q.put((srv.submit(s, h, w, Kq, T, n_samples=n_samples, seed=i), h * w))
    q.put(None)
    th.join()
    return np.array(lat), tot[0]


def measure_precision(args, compact=False):
    """Room-scale step with BF16 colour and 20 BF16 semantic logits; per-output errors vs the FP64 oracle over
    every ray of a 4096-ray subset (the oracle fed the GPU's own samples, sdg_debug_trace)."""
    import torch
    import oracle
    import paper_2305_13220_b300 as sdg
    import synth
    device = "cuda:0"
    sc = synth.scene_room(0)
    poses = synth.random_poses(sc, args.views, seed=0)
    K = synth.intrinsics(W, H)
    G = sdg.Grid(VS, args.max_blocks, beta=BETA, rgb_dtype="bf16", n_sem=20)
    _activate_views(sdg, torch, G, sc, poses, K, device, BAND)
    keys, vals = _fill(sdg, torch, G, sc, VS, BAND, device, n_sem=20)
    batches = [synth.training_batch(sc, poses, W, H, K, args.rays, seed=b, device=device, n_sem=20,
                                    order=args.order) for b in range(4)]

    # error table (before any training step changes the grid) on 4096 rays spread over the views: GPU (BF16
    # storage) vs the FP64 oracle on the unrounded generator values, and vs the oracle on the stored (rounded)
    # values (the parity check)
    A = sdg._abi
    nb = len(keys)
    G.zero_grad()
    sub = batches[0]["rays"][torch.linspace(0, args.rays - 1, 4096, device=device).long()].contiguous()
    out = sdg.render(G, sub, N_SAMPLES, seed=0, want_ctx=True)
    tr = sdg.trace(G, sub, N_SAMPLES, seed=0)
    given = {"S": tr["S"].double().cpu().numpy(), "t": tr["t"].cpu().numpy(), "cell": tr["cell"].cpu().numpy()}
    del tr
    n = sub.shape[0]
    gen = torch.Generator(device=device).manual_seed(0)
    seeds = [torch.randn(sh, generator=gen, device=device) * 1e-3 for sh in ((n, 3), (n,), (n,), (n, 20))]
    sdg.backward(out["ctx"], *seeds)
    torch.cuda.synchronize()
    stored = {"sdf": G.channel(A.GROUP_SDF)[:nb, :, 0].double().cpu().numpy(),
              "rgb": G.channel(A.GROUP_RGB)[:nb, :, 0:3].double().cpu().numpy(),
              "sem": G.channel(A.GROUP_SEM)[:nb].double().cpu().numpy()}
    full = {"sdf": vals["sdf"].to(torch.float32).double().cpu().numpy(), "rgb": vals["rgb"].cpu().numpy(),
            "sem": vals["sem"].cpu().numpy()}
    del vals
    got = {k: out[k].double().cpu().numpy() for k in ("rgb", "depth", "opac", "sem")}
    cnt_rays = batches[0]["rays"][np.linspace(0, args.rays - 1, 1024).astype(np.int64)].cpu().numpy()
    ggot = {"sdf": G.channel(A.GROUP_SDF, A.KIND_GRAD)[:nb, :, 0].double().cpu().numpy(),
            "rgb": G.channel(A.GROUP_RGB, A.KIND_GRAD)[:nb, :, 0:3].double().cpu().numpy(),
            "sem": G.channel(A.GROUP_SEM, A.KIND_GRAD)[:nb].double().cpu().numpy()}
    out["ctx"].release()
    rays_np = sub.cpu().numpy()
    sd = [x.double().cpu().numpy() for x in seeds]
    table = {}
    for name, src in (("vs_fp64_unrounded", full), ("vs_fp64_same_bf16_values", stored)):
        O = oracle.Grid(VS, BETA, 20).set(keys, src["sdf"], src["rgb"], src["sem"])
        if src is stored:  # distinct voxels and blocks per ray, for the roofline's algorithmic bytes
            vx, bl = O.count_touched(cnt_rays, N_SAMPLES, seed=0)
        ref = O.render(rays_np, N_SAMPLES, seed=0, given=given)
        row = {k: float(np.abs(got[k] - ref[k]).max()) for k in ("rgb", "depth", "opac", "sem")}
        gref = O.backward(rays_np, N_SAMPLES, sd[0], sd[1], sd[2], sd[3], seed=0, given=given)
        for k in ("sdf", "rgb", "sem"):
            row["grad_" + k + "_rel"] = float(np.abs(ggot[k] - gref[k]).max() / max(np.abs(gref[k]).max(), 1e-30))
        table[name] = row
        del O, ref, gref
    del full, stored, ggot
    G.zero_grad()

    step = _prepared_steps(sdg, G, batches, lambda b, i, slot: sdg.train_step_rays(
        G, b["rays"], b["rgb"], b["depth"], b["sem"], n_samples=N_SAMPLES, seed=i, ray_order=args.ray_order,
        prepared=slot), args.ray_order)

    ms = _timed_steps(torch, step, batches, args.steps, args.warmup)
    phases = _phase_times(torch, sdg, G, batches, args.steps, lambda b, i: sdg.train_step_rays(
        G, b["rays"], b["rgb"], b["depth"], b["sem"], n_samples=N_SAMPLES, seed=i, ray_order=args.ray_order))
    G.close()
    del batches
    torch.cuda.empty_cache()
    rps = args.rays / (ms / 1e3)
    # per distinct voxel: 52 B read (SDF 4, colour 8, 20 BF16 logits 40) and 200 B of gradient read-modify-write
    # (SDF 4, colour 16, logits 80, each read and written); per block 40 B; per ray 32 B, targets 96 B, loss 4 B
    bpr = float((vx * 252.0 + bl * 40.0 + 32 + 96 + 4).mean())
    peak, peak_src = _peak()
    kern_gbs = bpr * args.rays / (phases["render_kernels_ms"] / 1e3) / 1e9
    roof = {"kernel": "k_render_train (BF16 colour, 20 logits)", "bound": "hbm", "achieved": round(kern_gbs, 1),
            "peak": peak, "unit": "GB/s", "frac": round(kern_gbs / peak, 4), "traffic": None,
            "peak_source": peak_src, "algorithmic_bytes_per_launch": round(bpr * args.rays),
            "bytes_per_ray": round(bpr, 1), "distinct_voxels": round(float(vx.mean()), 1),
            "distinct_blocks": round(float(bl.mean()), 2), "launch_ms_median": phases["render_kernels_ms"]}
    if compact:
        return {"workload": "room step, BF16 colour + 20 BF16 logits (FP32 SDF, transmittance, accumulation)",
                "rays_per_s": round(rps, 1), "ms_per_step": round(ms, 4), "phases": phases, "roofline": roof,
                "errors_on_4096_rays_all_compared": table, "steps": args.steps, "warmup": args.warmup}
    return _line(rps, "rays/s", args.steps, args.warmup, ms,
                 {"workload": "precision variant of the room step: BF16 colour + 20 BF16 semantic logits, FP32 "
                              "SDF / transmittance / accumulation", "rays_per_step": args.rays,
                  "samples_per_ray": N_SAMPLES, "n_blocks": nb},
                 dtype="f32+bf16", samples_per_s=round(args.rays * N_SAMPLES / (ms / 1e3), 1), phases=phases,
                 roofline=roof, errors_on_4096_rays_all_compared=table,
                 gpu_launches=(_train_launches(args, args.rays) + 1) * args.steps)


def run_precision(args):
    print(json.dumps(measure_precision(args)), flush=True)


# Serving scenes: rooms of the room-scale kind (boxes and cylinders on the floor), sized and voxelised so that
# their block counts span about 10k to 200k (blocks of the analytic band, 3 voxels).
SERVE_SPECS = [((6, 5, 3), 10, 0.02), ((8, 6, 3), 12, 0.02), ((6, 6, 3), 10, 0.015), ((9, 7, 3), 16, 0.015),
               ((6, 6, 3), 12, 0.01), ((8, 8, 3), 20, 0.01), ((12, 9, 3), 30, 0.01), ((17, 14, 3), 60, 0.01)]


def measure_serve(args, compact=False):
    """8 device-resident rooms (about 10k-200k blocks, 1-2 cm voxels, BF16 colour); Poisson arrivals at 0.5x,
    0.8x and 1.0x of the measured saturated capacity; latency = submit -> result ready (host clock)."""
    import torch
    import paper_2305_13220_b300 as sdg
    import synth
    device = "cuda:0"
    grids, scenes = [], []
    for i in [int(x) for x in args.serve_scenes.split(",")]:
        size, n_obj, vs = SERVE_SPECS[i]
        sc = synth.scene_room(100 + i, size=size, n_objects=n_obj)
        keys = synth.band_blocks(sc, vs, 3, device=device)
        G = sdg.Grid(vs, len(keys), beta=0.5 * vs, rgb_dtype="bf16")
        G.activate_keys(torch.as_tensor(keys, device=device))
        _fill(sdg, torch, G, sc, vs, 3, device)
        grids.append(G)
        scenes.append(sc)
    srv = sdg.Server(hbm_budget_bytes=4 << 30, max_slots=32, n_streams=4, chunk_rays=4096, max_batch_rays=1 << 18)
    ids = [srv.add_scene(G) for G in grids]
    res = [(160, 120), (320, 240), (640, 480), (1280, 960)]
    rng = np.random.default_rng(0)
    poses = [synth.random_poses(sc, 8, seed=50) for sc in scenes]

    def req(i):
        s = int(rng.integers(0, len(ids)))
        w, h = res[int(rng.integers(0, 4))]
        return ids[s], h, w, synth.intrinsics(w, h), poses[s][i % 8]

    # saturated capacity: 64 mixed requests submitted at once
    reqs = [req(i) for i in range(64)]
    t = srv.submit(*reqs[0][:3], reqs[0][3], reqs[0][4], n_samples=N_SAMPLES)
    srv.wait(t, 300000)
    srv.release(t)
    t0 = time.perf_counter()
    tk = [(srv.submit(s, h, w, Kq, T, n_samples=N_SAMPLES, seed=i), h * w) for i, (s, h, w, Kq, T) in enumerate(reqs)]
    rays = 0
    for t, nr in tk:
        srv.wait(t, 300000)
        srv.release(t)
        rays += nr
    cap = rays / (time.perf_counter() - t0)
    mean_rays = np.mean([w * h for w, h in res])
    points = []
    for frac in (0.5, 0.8, 1.0):
        rate = frac * cap / mean_rays
        arr = np.cumsum(rng.exponential(1.0 / rate, size=args.requests))
        start = time.perf_counter()
        lat, nr_tot = _open_loop(srv, args.requests, arr, lambda i: req(i), start)
        el = time.perf_counter() - start
        points.append({"load": frac, "rate_req_s": round(rate, 2), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                       "p99_ms": round(float(np.percentile(lat, 99)), 3), "rays_per_s": round(nr_tot / el, 1),
                       "requests": args.requests})
    st = srv.stats()
    srv.close()
    nblocks = [G.num_blocks for G in grids]
    for G in grids:
        G.close()
    del grids
    torch.cuda.empty_cache()
    if compact:
        return {"workload": f"{len(ids)} rooms, BF16 colour, N = 128, requests uniform over 160x120..1280x960, "
                            "Poisson arrivals at 0.5x / 0.8x / 1.0x of the saturated rate",
                "scene_blocks": nblocks, "saturated_rays_per_s": round(cap, 1), "points": points}
    return _line(cap, "rays/s", len(points), 1, 1e3 * mean_rays / cap,
                 {"workload": f"serving: {len(ids)} device-resident rooms, BF16 colour, 128 samples per ray, "
                              "requests of 160x120 / 320x240 / 640x480 / 1280x960 with Poisson arrivals",
                  "scene_blocks": nblocks},
                 dtype="f32+bf16", saturated_rays_per_s=round(cap, 1), serve_points=points,
                 peak_server_bytes=int(st.peak_bytes_in_use), gpu_launches=int(st.launches))


def run_serve(args):
    print(json.dumps(measure_serve(args)), flush=True)


def measure_apartment(args, compact=False):
    """20x15x3 m apartment (6 rooms, 60 furniture primitives), 1 cm voxels: a full 1280x960 render at 192
    samples per ray, and 2^20-ray training steps (fused pass + Adam)."""
    import torch
    import paper_2305_13220_b300 as sdg
    import synth
    device = "cuda:0"
    sc = synth.scene_apartment(0)
    poses = synth.random_poses(sc, 300, seed=0)
    K = synth.intrinsics(W, H)
    G = sdg.Grid(VS, 1_600_000, beta=BETA)
    act_ms = _activate_views(sdg, torch, G, sc, poses, K, device, BAND)
    keys, vals = _fill(sdg, torch, G, sc, VS, BAND, device)
    del vals
    nb = len(keys)
    # full-frame render, 1280x960 at 192 samples
    Kr = synth.intrinsics(1280, 960)
    frame = synth.view_rays(poses[0], 1280, 960, Kr, device=device)
    for _ in range(2):
        sdg.render(G, frame, 192, seed=0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(5):
        sdg.render(G, frame, 192, seed=i)
    e1.record()
    torch.cuda.synchronize()
    render_ms = e0.elapsed_time(e1) / 5
    batches = [synth.training_batch(sc, poses, W, H, K, 1 << 20, seed=b, device=device, order=args.order)
               for b in range(2)]

    step = _prepared_steps(sdg, G, batches, lambda b, i, slot: sdg.train_step_rays(
        G, b["rays"], b["rgb"], b["depth"], n_samples=N_SAMPLES, seed=i, ray_order=args.ray_order, prepared=slot),
        args.ray_order)
    ms = _timed_steps(torch, step, batches, args.steps, args.warmup)
    torch.cuda.synchronize()
    phases = _phase_times(torch, sdg, G, batches, args.steps, lambda b, i: sdg.train_step_rays(
        G, b["rays"], b["rgb"], b["depth"], n_samples=N_SAMPLES, seed=i, ray_order=args.ray_order))
    G.close()
    del batches, frame
    torch.cuda.empty_cache()
    n = 1 << 20
    render = {"ms": round(render_ms, 3), "rays_per_s": round(1280 * 960 / (render_ms / 1e3), 1),
              "samples_per_s": round(1280 * 960 * 192 / (render_ms / 1e3), 1)}
    if compact:
        return {"workload": "apartment 20x15x3 m, 1 cm voxels, 4-voxel band from 300 depth maps",
                "n_blocks": nb, "train_2p20_rays": {"rays_per_s": round(n / (ms / 1e3), 1), "ms_per_step": round(ms, 4),
                                                    "phases": phases},
                "render_1280x960_n192": render, "activation_ms_300_maps": round(act_ms, 2)}
    return _line(n / (ms / 1e3), "rays/s", args.steps, args.warmup, ms,
                 {"workload": "apartment 20x15x3 m, 6 rooms, 60 furniture primitives, 1 cm voxels, 4-voxel band "
                              "from 300 depth maps; 2^20-ray training steps at 128 samples + 1280x960 render at 192",
                  "n_blocks": nb, "voxels": nb * 512, "rays_per_step": n},
                 render_1280x960_n192=render, activation_ms_300_maps=round(act_ms, 2), phases=phases,
                 gpu_launches=(_train_launches(args, 1 << 20) + 1) * args.steps)


def run_apartment(args):
    print(json.dumps(measure_apartment(args)), flush=True)


_REF = {}  # the reference arm's oracle grid and sample, inherited by forked workers


def _ref_chunk(bounds):
    """Oracle forward + L1 loss + backward of rays [a, b) of the reference sample (in a forked worker)."""
    import oracle
    a, b = bounds
    O, rays, t_rgb, t_d = _REF["O"], _REF["rays"], _REF["rgb"], _REF["depth"]
    t0 = time.perf_counter()
    out = O.render(rays[a:b], N_SAMPLES, seed=0, ray_id0=a)
    _, g = oracle.loss(out["rgb"], out["depth"], t_rgb[a:b], t_d[a:b], LAMBDA_D)
    O.backward(rays[a:b], N_SAMPLES, g["rgb"], g["depth"], seed=0, ray_id0=a)
    return time.perf_counter() - t0


def run_reference(args):
    """Reference arm: the CPU FP64 oracle, as it stands (single-threaded code), run on all host cores as one
    process per core over chunks of rays (fork: every worker shares the parent's oracle grid) and, for context,
    on one core.  Its rays are a seeded sample of the GPU arm's first batch (same scene, block set, voxel values,
    rays and samples); each step is a bounded sample of it.  Rank 0 only."""
    import multiprocessing as mp
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import torch
    import synth
    import oracle
    t_setup = time.perf_counter()
    sc = synth.scene_room(0)
    poses = synth.random_poses(sc, args.views, seed=0)
    K = synth.intrinsics(W, H)
    ks = oracle.KeySet()
    for T in poses:
        ks.add_depth(synth.depth_map(sc, T, W, H, K), K, T, VS, BAND)
    keys = ks.keys()
    vals = synth.fill_grid(sc, keys, VS, BAND)
    O = oracle.Grid(VS, BETA).set(keys, vals["sdf"].to(torch.float32).double().numpy(),
                                  vals["rgb"].to(torch.float32).double().numpy())
    del vals
    # the GPU arm's first batch (build_workload: seed 0, batch 0, per-image order), then a seeded sample of it
    batch = synth.training_batch(sc, poses, W, H, K, args.rays, seed=0, order=args.order)
    perm = np.random.default_rng(0).permutation(args.rays)
    cores = max(1, min(len(os.sched_getaffinity(0)), 64))
    per_core = 128  # rays per core and step: about 0.15 s of oracle work each
    rays_per_step = per_core * cores
    total = (args.warmup + args.steps) * rays_per_step + 256
    sel = perm[:min(total, args.rays)]
    _REF.update(O=O, rays=batch["rays"].numpy()[sel], rgb=batch["rgb"].double().numpy()[sel],
                depth=batch["depth"].double().numpy()[sel])
    setup_s = time.perf_counter() - t_setup
    # one core: 256 rays
    t0 = time.perf_counter()
    _ref_chunk((len(sel) - 256, len(sel)))
    single = 256 / (time.perf_counter() - t0)
    # all cores: each step splits rays_per_step rays over the workers
    ctx = mp.get_context("fork")
    step_s = []
    with ctx.Pool(cores) as pool:
        for i in range(args.warmup + args.steps):
            a = i * rays_per_step
            chunks = [(a + c * per_core, a + (c + 1) * per_core) for c in range(cores)]
            if chunks[-1][1] > len(sel) - 256:
                break
            t0 = time.perf_counter()
            pool.map(_ref_chunk, chunks, chunksize=1)
            if i >= args.warmup:
                step_s.append(time.perf_counter() - t0)
    steps = len(step_s)
    ms = 1e3 * float(np.mean(step_s))
    v = rays_per_step / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": "rays/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "room-scale FP32 training step (6x6x3 m room, 10 boxes/cylinders, 1 cm "
                                   "voxels, 8^3 blocks, 4-voxel band from 50 640x480 depth maps; 2^18 rays "
                                   "x 128 stratified samples, L1 colour + 0.1 L1 depth, Adam on every voxel)",
                       "rays_per_step": rays_per_step, "samples_per_ray": N_SAMPLES, "n_blocks": int(len(keys)),
                       "sample": f"each step: {rays_per_step} rays of the GPU arm's first 2^18-ray batch "
                                 f"(seeded sample, fwd + L1 loss + bwd), {per_core} per core on {cores} cores"},
            "ms_per_full_2p18_step_extrapolated": round(1e3 * args.rays / v, 1),
            "timing": {"step_ms": _stats(1e3 * np.asarray(step_s)), "setup_s": round(setup_s, 1)},
            "single_core_rays_per_s": round(single, 2),
            "cpu_baseline": {"value": round(v, 2), "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} steps x {rays_per_step} rays of the GPU arm's first batch, one "
                                       f"process per core (the oracle's code is single-threaded); one core: "
                                       f"{single:.1f} rays/s"},
            "e2e": {"value": round(v, 2), "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


def run_fusion(args):
    """Volumetric fusion (Eq. 9-11) of the room's RGB-D views into the room grid: frames/s with all views in one
    call and one view per call (an online loop), for an FP32 grid (depth + colour) and a BF16 grid with 20
    logits (depth + colour + labels)."""
    import torch
    import paper_2305_13220_b300 as sdg
    import synth
    device = "cuda:0"
    sc = synth.scene_room(0)
    poses = synth.random_poses(sc, args.views, seed=0)
    K = synth.intrinsics(W, H)
    mu = BAND * VS
    F = len(poses)
    out = {}
    for name, dtype, ns in (("depth_rgb_f32", "f32", 0), ("depth_rgb_sem20_bf16", "bf16", 20)):
        G = sdg.Grid(VS, args.max_blocks, beta=BETA, rgb_dtype=dtype, n_sem=ns)
        _activate_views(sdg, torch, G, sc, poses, K, device, BAND)
        fr = [synth.rgbd_frame(sc, T, W, H, K, n_sem=ns, seed=i, device=device) for i, T in enumerate(poses)]
        depth = torch.stack([f["depth"] for f in fr]).contiguous()
        rgb = torch.stack([f["rgb"] for f in fr]).contiguous()
        sem = torch.stack([f["sem"] for f in fr]).contiguous() if ns else None
        del fr
        Kt = torch.tensor(K, dtype=torch.float32)

        def batch(_b, _i):
            G.fuse(depth, Kt, poses, mu, rgb=rgb, sem=sem)

        def online(_b, _i):
            for i in range(F):
                G.fuse(depth[i], Kt, poses[i], mu, rgb=rgb[i], sem=sem[i] if ns else None)

        ms_batch = _timed_steps(torch, batch, [None], args.steps, args.warmup)
        ms_online = _timed_steps(torch, online, [None], max(args.steps // 4, 2), 1)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        G.fuse_finalize()
        t1.record()
        torch.cuda.synchronize()
        w = G.channel(sdg._abi.GROUP_WEIGHT)[:G.num_blocks, :, 0]
        out[name] = {"frames_per_s_batched": round(F / (ms_batch / 1e3), 1), "ms_per_50_frames": round(ms_batch, 4),
                     "frames_per_s_one_per_call": round(F / (ms_online / 1e3), 1),
                     "finalize_ms": round(t0.elapsed_time(t1), 4), "n_blocks": G.num_blocks,
                     "voxels_fused": int((w > 0).sum().item()),
                     "mean_associations_per_fused_voxel": round(float(w[w > 0].mean().item()) / (args.warmup
                                                                  + args.steps + max(args.steps // 4, 2) + 1), 2)}
        del G, depth, rgb, sem
        torch.cuda.empty_cache()
    main_ = out["depth_rgb_f32"]
    line = _line(main_["frames_per_s_batched"], "frames/s", args.steps, args.warmup, main_["ms_per_50_frames"],
                 {"workload": f"volumetric fusion of {F} 640x480 RGB-D views (analytic depth and colour; 20 noisy "
                              "one-hot logits for the semantic variant) into the room grid (1 cm voxels, 8^3 "
                              f"blocks, 4-voxel band, mu = {mu} m)", "frames_per_call": F},
                 fusion=out, gpu_launches=args.steps,
                 paper_context="50 Hz depth + colour, 30 Hz with labels (RTX 3060, whole fusion step; context)")
    print(json.dumps(line), flush=True)


def run_query(args):
    """The paper's query benchmark on the room grid: SDF and its gradient (one pass, Eq. 16-17) at the k^3 lattice
    points of the block AABB, k = 16..512, and an Eikonal step (loss + gradient scatter) on 2^20 points drawn
    uniformly in the allocated blocks."""
    import torch
    import paper_2305_13220_b300 as sdg
    import synth
    device = "cuda:0"
    sc = synth.scene_room(0)
    poses = synth.random_poses(sc, args.views, seed=0)
    K = synth.intrinsics(W, H)
    G = sdg.Grid(VS, args.max_blocks, beta=BETA)
    _activate_views(sdg, torch, G, sc, poses, K, device, BAND)
    keys, _ = _fill(sdg, torch, G, sc, VS, BAND, device)
    kt = torch.as_tensor(keys, device=device, dtype=torch.float64)
    lo = kt.min(0).values * 8 * VS
    hi = (kt.max(0).values + 1) * 8 * VS
    res = {}
    for k in (16, 32, 64, 128, 256, 512):
        t = (torch.arange(k, device=device, dtype=torch.float64) + 0.5) / k
        zz, yy, xx = torch.meshgrid(t, t, t, indexing="ij")  # x fastest
        xyz = (lo + (hi - lo) * torch.stack([xx, yy, zz], -1).reshape(-1, 3)).to(torch.float32).contiguous()
        del zz, yy, xx
        n = xyz.shape[0]
        sdf = torch.empty(n, device=device)
        grad = torch.empty((n, 3), device=device)

        def q(_b, _i):
            sdg._abi.call("sdg_query", G.handle, xyz.data_ptr(), n, sdf.data_ptr(), grad.data_ptr())

        ms = _timed_steps(torch, q, [None], args.steps, args.warmup)
        valid = int((~torch.isnan(sdf)).sum().item())
        alg = n * (12 + 16) + valid * 8 * 4  # point in, SDF + gradient out, 8 corner SDF values per valid point
        res[str(k)] = {"points": n, "ms": round(ms, 4), "points_per_s": round(n / (ms / 1e3), 1),
                       "valid_points": valid, "alg_gb_s": round(alg / (ms / 1e3) / 1e9, 1)}
        del xyz, sdf, grad
    # Eikonal step on 2^20 points uniform in the allocated blocks
    gen = torch.Generator(device=device)
    gen.manual_seed(11)
    m = 1 << 20
    b = kt[torch.randint(0, len(keys), (m,), device=device, generator=gen)]
    pts = ((b * 8 + torch.rand((m, 3), device=device, generator=gen, dtype=torch.float64) * 8) * VS)
    pts = pts.to(torch.float32).contiguous()
    total = torch.zeros(1, device=device)

    def eik(_b, _i):
        G.eikonal(pts, 0.1, loss_sum=total)

    ms_eik = _timed_steps(torch, eik, [None], args.steps, args.warmup)
    top = res["512"]
    line = _line(top["points_per_s"], "points/s", args.steps, args.warmup, top["ms"],
                 {"workload": "SDF + gradient query (one pass, Eq. 16-17) at the k^3 lattice points of the room grid's "
                              "block AABB (53,855 blocks, 1 cm voxels), k = 16..512; value at k = 512",
                  "points": top["points"]},
                 query=res, eikonal_2p20_points={"ms": round(ms_eik, 4), "points_per_s": round(m / (ms_eik / 1e3), 1)},
                 gpu_launches=args.steps,
                 paper_context="the paper's figure (query time vs NGP-grid, k = 16..512) is not in the text")
    print(json.dumps(line), flush=True)


def run_crf(args):
    """CRF message passing (Eq. 19-22) on the room: 2^18 surface samples of the 50 views (first hits), features
    = position / 0.1 m, colour / 0.1, unit normal (d = 9); the permutohedral-lattice filter of 20 label
    channels and one Potts mean-field update."""
    import torch
    import paper_2305_13220_b300 as sdg
    import synth
    device = "cuda:0"
    sc = synth.scene_room(0)
    poses = synth.random_poses(sc, args.views, seed=0)
    K = synth.intrinsics(W, H)
    n = 1 << 18
    b = synth.training_batch(sc, poses, W, H, K, n, seed=5, device=device, n_sem=20)
    x = b["rays"][:, :3].double() + b["depth"].double()[:, None] * b["rays"][:, 4:7].double()
    eps = 1e-4
    grad = torch.stack([(synth.scene_sdf(sc, x + eps * e) - synth.scene_sdf(sc, x - eps * e)) / (2 * eps)
                        for e in torch.eye(3, dtype=torch.float64, device=device)], -1)
    nrm = grad / grad.norm(dim=-1, keepdim=True).clamp_min(1e-12)
    feat = torch.cat([x / 0.1, b["rgb"].double() / 0.1, nrm], 1).to(torch.float32).contiguous()
    U = (-b["sem"]).contiguous()
    Q = torch.softmax(-U, dim=1).contiguous()
    G = sdg.Grid(VS, 16, beta=BETA)  # stream and scratch owner (the filter does not read the grid's voxels)
    stats = {}

    def filt(_b, _i):
        stats["M"] = G.lattice_filter(feat, Q)[1]

    def mf(_b, _i):
        G.crf_meanfield(feat, U, Q, 1.0)

    ms_f = _timed_steps(torch, filt, [None], args.steps, args.warmup)
    ms_mf = _timed_steps(torch, mf, [None], args.steps, args.warmup)
    line = _line(n / (ms_mf / 1e3), "points/s", args.steps, args.warmup, ms_mf,
                 {"workload": "continuous-CRF mean-field update on 2^18 surface samples of the room (features: "
                              "position/0.1 m, colour/0.1, normal; d = 9; 20 labels), permutohedral lattice",
                  "points": n, "d": 9, "labels": 20},
                 lattice={"points": int(stats["M"]), "filter_ms": round(ms_f, 4),
                          "meanfield_ms": round(ms_mf, 4)},
                 gpu_launches=(6 + 10) * args.steps,
                 note="each call synchronises once: the lattice size sizes the blur launches")
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    single = {"room_bf16_sem", "serve", "apartment", "fusion", "query", "crf"}
    if args.impl != "reference" and args.config in single and int(os.environ.get("WORLD_SIZE", "1")) > 1:
        # one-GPU measurements: under a multi-process launch rank 0 runs them (on its own GPU), the others exit
        if int(os.environ.get("RANK", "0")) != 0:
            return
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "room_bf16_sem":
        run_precision(args)
    elif args.config == "serve":
        run_serve(args)
    elif args.config == "apartment":
        run_apartment(args)
    elif args.config == "fusion":
        run_fusion(args)
    elif args.config == "query":
        run_query(args)
    elif args.config == "crf":
        run_crf(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
