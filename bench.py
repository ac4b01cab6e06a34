"""Benchmark of the FilterGS LoD render path on one GB300 (or N replicas).

One step = one whole frame of the render path (R&L filter, ancestor filter +
compaction, projection + SH + shrink + per-tile pair counts, tile ranges, key
scatter into per-tile buckets, per-tile sort, blending) for one camera pose of the synthetic workload, inputs resident in HBM.

Default workload: the 10M-leaf city tree (~12.5M nodes), 1920x1080, 64-pose
flythrough, adaptive shrinking with tau calibrated over the 64 poses
(lambda_G = 0.2).  Prints ONE JSON line on rank 0.  Beside the headline the
line carries the per-stage times and bandwidths, the blend's ALU roofline, the
end-to-end rate through the C ABI with host buffers, the blend work counters,
the traversal-free filter against the level-by-level baseline, the batched
32-view form, the shrinking study and the differentiable form's backward.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload city|blobs|tiny]
                  [--impl ours|reference] [--no-cpu-baseline] [--no-batch]
                  [--no-study] [--no-backward]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import threading
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STAGES = ["filter_rl", "ancestor_compact", "project", "tile_ranges", "keys", "sort", "blend"]
METRIC = "1080p ms/frame & FPS on 10M-leaf LoD tree; GS-tile pairs/frame; HBM roofline %"


def _json_default(o):
    if isinstance(o, (np.floating,)):
        return float(o)
    if isinstance(o, (np.integer,)):
        return int(o)
    raise TypeError(type(o))


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload(name):
    from paper_2603_23891_gb300 import synth
    if name == "city":
        return (synth.city_tree(), synth.city_cameras(), 3.0,
                "city-10M: 10M-leaf city LoD tree, 1920x1080, 64-pose flythrough, adaptive shrink")
    if name == "blobs":
        return (synth.blob_tree(), synth.blob_cameras(), 3.0,
                "blobs-1M: 1M-leaf blob LoD tree, 1920x1080, 8 poses, adaptive shrink")
    if name == "tiny":
        return (synth.tiny_tree(), [synth.tiny_camera()], 1.0,
                "tiny-4k: 4,096-leaf tree, 256x256, 1 pose, adaptive shrink")
    raise ValueError(name)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region (read from its
    output pipe; nothing is written to disk).  `cmd` replaces the sampler command
    (tests use a fake that prints the same CSV)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index, cmd=None):
        self.idx = device_index
        self.proc = None
        self.lines = []
        self.reader = None
        self.cmd = cmd or ["nvidia-smi", f"--id={device_index}", f"--query-gpu={self.Q}",
                           "--format=csv,noheader,nounits", "-lms", "100"]

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line)

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.reader.join(timeout=5)
        return self.summarise(list(self.lines))

    @staticmethod
    def summarise(lines):
        """Median SM clock, maximum SM clock and the throttle reasons seen."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- roofline

def algorithmic_bytes(tree, M, NP, width, height, sh_floats, E, n_cov, tiles, chunks=None):
    """Bytes the method must move per frame, per stage.  E: selected Gaussians that
    emit pairs, the only ones whose SH colour is evaluated; n_cov: in-frustum
    internal nodes, the only ones whose covariance R&L needs; chunks: 128-node
    chunks whose centres R&L reads (the others lie wholly outside the frustum; all
    three counted on the device; None: every chunk); tiles: screen tiles."""
    N = tree.n
    D = tree.depth
    n_box = (N + 127) // 128
    read = n_box if chunks is None else chunks
    return {
        # chunk boxes, the centres and leaf bits of the chunks read, covariances, P bits out
        "filter_rl": 32.0 * n_box + (12.0 * 128 + 16.0) * read + 24.0 * n_cov + N / 8.0,
        "ancestor_compact": N / 8.0 + 4.0 * D * M + 4.0 * M,
        # id, centre, covariance, opacity + ln opacity in; splat and footprint out;
        # SH rows of the emitting Gaussians; the per-tile pair counts
        "project": M * (4 + 12 + 24 + 8 + 48 + 16) + E * 4 * sh_floats + 4.0 * tiles,
        # counts in; ranges and cursors out
        "tile_ranges": 16.0 * tiles,
        # footprints in; one 8-byte item per pair out
        "keys": 16.0 * M + 8.0 * NP,
        # items in; keys and values out
        "sort": 20.0 * NP,
        "blend": NP * (4.0 + 48.0) + 16.0 * width * height,
    }


def blend_alu_peak(sm_mhz, sms):
    """FP32 lane-ops/s: 128 FP32 lanes per SM per clock."""
    return 128.0 * sms * sm_mhz * 1e6


# FP32 lane operations of Eq. 2 with the 3DGS rules, as the blend computes them
OPS_PER_EVAL = 9.0    # dx, dy, B'dy, C'dy, (C'dy)dy, two FMAs, the two skip tests
OPS_PER_HIT = 24.0    # exp (15: k by one FMA and a subtraction, reduction 2 FMAs, degree-7
                      # Horner 7 FMAs, 2^k 2 integer ops, scaling, range select), alpha,
                      # clamp, 1 - alpha, T update, stop test, weight, 3 colour FMAs


# source files of each frame kernel (a kernel's committed DRAM figure is used only
# while these files are unchanged)
KERNEL_SOURCES = {
    "frame_begin_kernel": ["filter.cu", "fgs_internal.cuh"],
    "filter_pred_kernel": ["filter.cu", "fgs_internal.cuh"],
    "filter_anc_kernel": ["filter.cu", "fgs_internal.cuh"],
    "compact_counted_kernel": ["filter.cu", "fgs_internal.cuh"],
    "project_kernel": ["project.cu", "project_impl.cuh", "pairs_impl.cuh", "fgs_internal.cuh"],
    "tile_scan_kernel": ["pairs.cu", "pairs_impl.cuh", "fgs_internal.cuh"],
    "scatter_kernel": ["pairs.cu", "pairs_impl.cuh", "fgs_internal.cuh"],
    "segsort_kernel": ["pairs.cu", "pairs_impl.cuh", "fgs_internal.cuh"],
    "blend_kernel": ["blend.cu", "blend_impl.cuh", "fgs_internal.cuh"],
}
# the kernels of each bench stage
STAGE_KERNELS = {
    "filter_rl": ["frame_begin_kernel", "filter_pred_kernel"],
    "ancestor_compact": ["filter_anc_kernel", "compact_counted_kernel"],
    "project": ["project_kernel"],
    "tile_ranges": ["tile_scan_kernel"],
    "keys": ["scatter_kernel"],
    "sort": ["segsort_kernel"],
    "blend": ["blend_kernel"],
}


def _kernel_sources_sha(kernel):
    import hashlib
    files = KERNEL_SOURCES.get(kernel)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2603_23891_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """Mean DRAM bytes per launch of `kernel` on the bench workload's timed poses,
    from the committed ncu summary (profiles/traffic.txt: '<kernel> <source
    sha16> <bytes>'), or None if the kernel source changed since it was
    captured."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = _kernel_sources_sha(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) == 3 and parts[0] == kernel and parts[1] == sha:
            return int(parts[2])
    return None


def run_batched(r, torch, filtergs, args):
    """Batched multi-view form: 32 views (8 each at 640x360, 1280x720, 1920x1080,
    3840x2160) over the city tree; autotuned tile / blend-warp shapes, CUDA-graph
    replay, against the same 32 views rendered one call at a time."""
    from paper_2603_23891_gb300 import synth
    cams = synth.city_batch_cameras()
    t0 = time.time()
    choice, tuned_ms = r.batch_autotune(cams, sel_capacity=args.batch_sel_cap,
                                        pair_capacity=args.batch_pair_cap)
    tune_s = time.time() - t0
    total = int(r.batch_offsets[-1])
    rgb = torch.empty(3 * total, dtype=torch.float32, device="cuda")
    T = torch.empty(total, dtype=torch.float32, device="cuda")
    _, _, st, _ = r.render_batch(rgb, T, graph=True, stats=True)
    reps = args.batch_reps
    for _ in range(2):
        r.render_batch(rgb, T, graph=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hold_stream(torch, reps)              # both loops: the host enqueues them behind a spin
    e0.record()
    for _ in range(reps):
        r.render_batch(rgb, T, graph=True)
    e1.record()
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / reps
    # sequential single-view calls, default 16x16 tiles
    r.set_params(tile=(16, 16), blend_warp_w=8)
    outs = {}
    for c in cams:
        if (c.width, c.height) not in outs:
            outs[(c.width, c.height)] = (torch.empty((3, c.height, c.width), device="cuda"),
                                         torch.empty((c.height, c.width), device="cuda"))
    for c in cams[:4]:
        r.set_camera(c)
        r.render(*outs[(c.width, c.height)])
    torch.cuda.synchronize()
    hold_stream(torch, reps * len(cams))
    e0.record()
    for _ in range(reps):
        for c in cams:
            r.set_camera(c)
            r.render(*outs[(c.width, c.height)])
    e1.record()
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / reps
    return {"views": len(cams), "views_per_s": round(len(cams) / (batch_ms * 1e-3), 1),
            "ms_per_batch": round(batch_ms, 3),
            "sequential_views_per_s": round(len(cams) / (seq_ms * 1e-3), 1),
            "sequential_ms": round(seq_ms, 3), "speedup": round(seq_ms / batch_ms, 2),
            "selected_entries": int(st.n_selected), "pairs": int(st.n_pairs),
            "autotune": {f"{w}x{h}": list(v) for (w, h), v in choice.items()},
            "autotune_s": round(tune_s, 2), "graph": True,
            "how": ("CUDA events around reps batch replays and around reps x 32 single-view "
                    "calls, each loop enqueued behind a fixed-length spin (device time, no "
                    "waits for the host)")}


# ----------------------------------------------------------------------------- ours

def shard_poses(n_poses: int, rank: int, world: int) -> list:
    """Views are independent: rank r renders poses r, r + world, r + 2 world, ...
    (one pose at least).  No data crosses ranks."""
    return [k for k in range(n_poses) if k % world == rank] or [rank % n_poses]


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time for a per-rank time: the maximum over ranks."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _time_backward(r, torch, cams, poses, P, G, dL_of, keep, accumulate, flush):
    """Per pose: render (keep or not), the loss gradient, the backward; CUDA
    events around the render and around the backward.  Returns mean ms."""
    stream = torch.cuda.current_stream()
    for w in range(3):
        r.set_camera(cams[poses[w % len(poses)]])
        rgb, _, _ = r.render(keep=keep)
        r.backward(dL_of(poses[w % len(poses)], rgb), P, G, accumulate=accumulate)
    torch.cuda.synchronize()
    fwd, bwd = [], []
    for k in poses:
        hold_stream(torch, 1, min_s=0.01)                 # the host enqueues the pose behind it
        flush.zero_()
        r.set_camera(cams[k])
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        rgb, _, _ = r.render(keep=keep)
        e[1].record(stream)
        dL = dL_of(k, rgb)
        e[2].record(stream)
        r.backward(dL, P, G, accumulate=accumulate)
        e[3].record(stream)
        torch.cuda.synchronize()
        fwd.append(e[0].elapsed_time(e[1]))
        bwd.append(e[2].elapsed_time(e[3]))
    return round(float(np.mean(fwd)), 4), round(float(np.mean(bwd)), 4)


def _tree_params(torch, tree, dev):
    P = {"mu": tree.mu, "log_scale": tree.log_scale, "quat": tree.quat,
         "logit": tree.opacity_logit, "sh": tree.sh}
    return {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev) for k, v in P.items()}


def run_backward(r, torch, filtergs, args):
    """Differentiable form, its configuration: the 1M-leaf blob tree at
    1920x1080 (3-sigma footprint), L2 loss against the image of the same tree
    with every leaf attribute perturbed by N(0, 0.01) (seed 3, parents rebuilt).
    Per pose: forward, dL/drgb = 2 (rgb - target), hand-written backward.  The
    default backward recomputes each pixel's final transmittance by a walk over
    its tile; with the forward's kept state (FGS_RENDER_KEEP) it reads it.
    Accumulate mode (the cut's gradients added into the caller's buffers)."""
    from paper_2603_23891_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    tree, target_tree, cams = synth.blob_tree(), synth.blob_target_tree(), synth.blob_cameras()
    poses = list(range(len(cams)))
    r.set_params(tau_R=3.0, tile=(16, 16), blend_warp_w=8, bg=(0.0, 0.0, 0.0),
                 pair_capacity=args.pair_capacity)
    r.shrink(None)
    r.load_tree(target_tree)
    targets = {}
    for k in poses:
        r.set_camera(cams[k])
        rgb, _, _ = r.render()
        targets[k] = rgb.clone()
    r.load_tree(tree)
    P = _tree_params(torch, tree, dev)
    G = {k: torch.zeros_like(v) for k, v in P.items()}
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    r.update_params(P)
    t1.record()
    torch.cuda.synchronize()
    prep_ms = t0.elapsed_time(t1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    loss = []

    def dL_of(k, rgb):
        d = rgb - targets[k]
        if len(loss) < len(poses):
            loss.append(float((d * d).sum()))
        return 2.0 * d

    out = {}
    for name, keep in (("recompute", False), ("kept_state", True)):
        f, b = _time_backward(r, torch, cams, poses, P, G, dL_of, keep, True, flush)
        out[name] = {"forward_ms": f, "backward_ms": b}
    K3 = (tree.sh_degree + 1) ** 2 * 3
    return {"workload": "blobs-1M, 1920x1080, 8 poses, 3-sigma footprint, L2 loss against the "
                        "tree with leaf attributes perturbed by N(0, 0.01)",
            "nodes": tree.n, "params_per_node": 11 + K3, "ms_per_frame": out["recompute"]["backward_ms"],
            "recompute": out["recompute"], "kept_state": out["kept_state"],
            "prep_params_ms": round(prep_ms, 4), "loss_pose0": loss[0] if loss else None,
            "how": "CUDA events around fgs_render and around fgs_backward per pose (L2 flushed "
                   "before each pose, each pose enqueued behind a 10 ms fixed-length spin), accumulate "
                   "mode; the loss gradient is outside both"}


def run_backward_city(r, torch, tree, cams, poses, args):
    """The backward on the bench workload (city-10M, adaptive shrink), dL/drgb ~
    N(0, 1), both transmittance modes, accumulate mode."""
    dev = torch.device("cuda", torch.cuda.current_device())
    P = _tree_params(torch, tree, dev)
    G = {k: torch.zeros_like(v) for k, v in P.items()}
    W, H = cams[0].width, cams[0].height
    dL = torch.randn((3, H, W), generator=torch.Generator(device=dev).manual_seed(0), device=dev)
    r.update_params(P)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    poses = poses[: min(16, len(poses))]
    out = {}
    for name, keep in (("recompute", False), ("kept_state", True)):
        f, b = _time_backward(r, torch, cams, poses, P, G, lambda k, rgb: dL, keep, True, flush)
        out[name] = {"forward_ms": f, "backward_ms": b}
    return {"workload": "city-10M, 1920x1080, 16 poses, adaptive shrink, dL/drgb ~ N(0, 1)", **out}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2603_23891_gb300 import build, filtergs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    build.build()

    t0 = time.time()
    tree, cams, tau_R, wname = workload(args.workload)
    log(f"[rank {rank}] workload {tree.name}: {tree.n} nodes, {tree.n_leaves} leaves, "
        f"depth {tree.depth} ({time.time() - t0:.1f}s)")
    P = len(cams)
    my_poses = shard_poses(P, rank, world)
    W, H = cams[0].width, cams[0].height

    r = filtergs.Renderer(device=local, tau_R=tau_R, pair_capacity=args.pair_capacity)
    t0 = time.time()
    r.load_tree(tree)
    log(f"[rank {rank}] tree uploaded ({time.time() - t0:.1f}s)")
    t0 = time.time()
    tau, ln_tau, gbars = r.calibrate(cams, args.lambda_g)
    calib_s = time.time() - t0
    log(f"[rank {rank}] calibrated: tau={tau:.5f} ln_tau={ln_tau:.5f} "
        f"mean G={np.nanmean(gbars):.4f} ({calib_s:.2f}s)")
    r.shrink(tau, ln_tau)

    stream = torch.cuda.current_stream()
    rgb = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
    Tt = torch.empty((H, W), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # per-pose work (M, N_P, emitting Gaussians, R&L covariance reads, the blend's
    # work counters) from one counting frame per pose, outside the timed region; the
    # line's per-frame figures average them over the poses the timed steps render
    work = {}
    for k in my_poses:
        r.set_camera(cams[k])
        _, _, st = r.render(rgb, Tt, count=True)
        work[k] = {"M": st.n_selected, "NP": st.n_pairs, "E": st.n_emitting,
                   "cov_nodes": st.filter_cov_nodes, "in_frustum": st.filter_in_frustum,
                   "chunks": st.filter_chunks_read,
                   "evals": st.blend_evals, "hits": st.blend_hits, "entries": st.blend_entries,
                   "active": st.blend_active}
        launches = st.n_launches
    # shrink-off pair counts for context
    r.shrink(None)
    NP_off = []
    for k in my_poses[: min(8, len(my_poses))]:
        r.set_camera(cams[k])
        _, _, st = r.render(rgb, Tt, stats=True)
        NP_off.append(st.n_pairs)
    r.shrink(tau, ln_tau)

    for w in range(args.warmup):
        r.set_camera(cams[my_poses[w % len(my_poses)]])
        r.render(rgb, Tt)
    torch.cuda.synchronize()

    K = args.steps
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    # hold the stream with torch's fixed-length spin kernel while the host enqueues
    # the K steps, so that a step's events never include the GPU waiting for the host
    # to launch its first kernel (the spin runs before the first step's start event)
    hold_s = hold_stream(torch, K)
    for k in range(K):
        flush.zero_()                                     # evict L2 between steps
        r.set_camera(cams[my_poses[k % len(my_poses)]])
        ev_s[k].record(stream)
        r.render(rgb, Tt)
        ev_e[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(K)]
    total_ms = float(sum(step_ms))
    # per-stage durations: the same K steps again, with events between the stages
    # (events between kernels stop the launch overlap, so this pass is separate)
    slot0 = filtergs.fgs_stage_count(r.ctx)
    for k in range(K):
        flush.zero_()
        r.set_camera(cams[my_poses[k % len(my_poses)]])
        r.render(rgb, Tt, stage_events=True)
    torch.cuda.synchronize()
    stage_ms = np.array([filtergs.fgs_stage_times(r.ctx, (slot0 + k) % 256) for k in range(K)])
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, "cuda")

    # end-to-end through the C ABI with pinned host buffers (camera in, image out;
    # the step's result is the image, the transmittance stays on the device):
    # pipelined host outputs (FGS_RENDER_ASYNC), frame k's image copy overlapping
    # frame k + 1's kernels, two host buffers in turn, and one synchronising
    # fgs_sync after the last step inside the timed region; the synchronising
    # host call (render, copy, wait, one frame at a time) is reported beside it
    rgb_h = [torch.empty((3, H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    for w in range(2):
        r.set_camera(cams[my_poses[0]])
        r.render_host(rgb_h[w].numpy())
        r.render_host(rgb_h[w].numpy(), pipelined=True)
    r.sync()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for k in range(K):
        r.set_camera(cams[my_poses[k % len(my_poses)]])
        r.render_host(rgb_h[k % 2].numpy(), pipelined=True)
    r.sync()
    e2e_s = time.perf_counter() - e0
    e1 = time.perf_counter()
    for k in range(K):
        r.set_camera(cams[my_poses[k % len(my_poses)]])
        r.render_host(rgb_h[k % 2].numpy())
    e2e_sync_s = time.perf_counter() - e1
    if world > 1:
        e2e_s = max_over_ranks(e2e_s, dist, "cuda")
        e2e_sync_s = max_over_ranks(e2e_sync_s, dist, "cuda")

    # traversal-free filter vs the serial level-by-level baseline (Eq. 3 / Table 2),
    # same poses, wall time of each call on an idle stream
    filt_par, filt_lw, lw_levels = [], [], 0
    sel_buf = np.zeros(tree.n, np.uint32)
    m_buf = np.zeros(1, np.uint32)
    for k in my_poses[: min(16, len(my_poses))]:
        r.set_camera(cams[k])
        for rep in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            filtergs.fgs_filter(r.ctx, r.stream, sel_buf, tree.n, m_buf, 0)
            t1 = time.perf_counter()
            lw_levels = filtergs.fgs_filter_levelwise(r.ctx, r.stream, sel_buf, tree.n, m_buf, 0)
            t2 = time.perf_counter()
            if rep == 1:
                filt_par.append((t1 - t0) * 1e3)
                filt_lw.append((t2 - t1) * 1e3)

    # the GPU's shrunk images of two poses, for the oracle comparison against the
    # unshrunk render (made in the CPU-baseline leg)
    shrunk_images = {}
    for k in sorted({my_poses[0], my_poses[len(my_poses) // 2]}):
        r.set_camera(cams[k])
        r.render(rgb, Tt)
        torch.cuda.synchronize()
        shrunk_images[k] = rgb.cpu().numpy().copy()

    batched = None
    if args.batch and args.workload == "city":
        batched = run_batched(r, torch, filtergs, args)

    # shrinking study (3 sigma, tau = 1/255, lambda_G sweep) on 8 of the poses
    study = None
    if args.study:
        from paper_2603_23891_gb300 import shrink_study
        r.set_params(tau_R=tau_R, tile=(16, 16), blend_warp_w=8, pair_capacity=args.pair_capacity)
        st_poses = my_poses[:: max(1, len(my_poses) // 8)][:8]
        full = shrink_study.run_study(r, cams, st_poses)
        study = {"poses": full["poses"], "G_bar": full["G_bar"], "settings": [
            {k: row[k] for k in ("setting", "tau", "N_P_mean", "N_P_vs_3sigma", "fps",
                                 "psnr_vs_3sigma_db", "max_abs_vs_3sigma")}
            | {"kpc_below_0.01": row["kpc"]["below_0.01"], "kpc_below_0.05": row["kpc"]["below_0.05"],
               "redundant_0.05_vs_3sigma": row["redundant_0.05_vs_3sigma"]}
            for row in full["settings"]],
            "how": "per setting: mean over the poses; KPC (Eq. 5) of the emitted pairs under that "
                   "footprint; image error against the 3-sigma GPU render of the same pose"}
        r.shrink(tau, ln_tau)

    # last: they replace the tree's attributes by the binary32 parameter map
    backward = None
    if args.backward:
        r.set_params(tau_R=tau_R, tile=(16, 16), blend_warp_w=8, pair_capacity=args.pair_capacity)
        r.shrink(tau, ln_tau)
        backward_city = run_backward_city(r, torch, tree, cams, my_poses, args)
        backward = run_backward(r, torch, filtergs, args)
        backward["city"] = backward_city

    frames = K * world
    fps = frames / (total_ms / 1e3)
    result = None
    if rank == 0:
        timed = [my_poses[k % len(my_poses)] for k in range(K)]

        def timed_mean(key):
            return float(np.mean([work[k][key] for k in timed]))
        M_mean, NP_mean, E_mean = timed_mean("M"), timed_mean("NP"), timed_mean("E")
        cov_mean = timed_mean("cov_nodes")
        chunks_mean = timed_mean("chunks")
        sh_floats = (tree.sh_degree + 1) ** 2 * 3
        n_screen_tiles = ((W + 15) // 16) * ((H + 15) // 16)
        ab = algorithmic_bytes(tree, M_mean, NP_mean, W, H, sh_floats, E_mean, cov_mean, n_screen_tiles,
                               chunks_mean)
        st_mean = stage_ms.mean(axis=0)
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
        stages = {}
        for i, nm in enumerate(STAGES):
            gbs = ab[nm] / (st_mean[i] * 1e-3) / 1e9 if st_mean[i] > 0 else 0.0
            traffic = [profiled_traffic(k) for k in STAGE_KERNELS[nm]]
            stages[nm] = {"ms": round(float(st_mean[i]), 5), "algo_bytes": round(ab[nm]),
                          "GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4),
                          "dram_bytes": None if None in traffic else int(sum(traffic))}
        dom = STAGES[int(np.argmax(st_mean))]
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        if dom == "blend":
            # issue-bound: FP32 lane operations of the evaluations the kernel performs
            ops = OPS_PER_EVAL * timed_mean("evals") + OPS_PER_HIT * timed_mean("hits")
            clk_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
            peak_tf = 128.0 * sms * clk_mhz * 1e6 / 1e12
            ach_tf = ops / (st_mean[STAGES.index("blend")] * 1e-3) / 1e12
            dom_rl = {"bound": "alu", "kernel": "blend_kernel", "achieved": round(ach_tf, 3),
                      "peak": round(peak_tf, 3), "unit": "T FP32 lane-ops/s",
                      "frac": round(ach_tf / peak_tf, 4),
                      "traffic": profiled_traffic("blend_kernel"),
                      "peak_source": f"derived: 128 FP32 lanes x {sms} SMs x {clk_mhz:.0f} MHz",
                      "ops": "FP32 lane operations (a fused multiply-add counts as one): 9 per "
                             "pixel-Gaussian evaluation (offsets, power, the two skip tests), 24 more "
                             "per evaluation that applies alpha (exp, alpha, clamp, T, stop test, "
                             "colour); evaluations and applications counted on the device for the "
                             "timed poses",
                      "ops_per_frame": round(ops),
                      "hbm_view": {"achieved": stages[dom]["GB/s"], "peak": hbm_peak, "unit": "GB/s",
                                   "frac": stages[dom]["frac_hbm"]}}
        else:
            dom_rl = {"bound": "hbm", "kernel": dom, "achieved": stages[dom]["GB/s"],
                      "peak": hbm_peak, "unit": "GB/s", "frac": stages[dom]["frac_hbm"],
                      "traffic": profiled_traffic(dom), "peak_source": peak_src}
        img_bytes = 3 * H * W * 4
        cam_bytes = 4 * 26 + 8
        result = {
            "metric": METRIC, "value": round(fps, 2), "unit": "frames/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(total_ms / K, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator; no trained model or dataset)",
            "config": {"workload": wname, "n_nodes": tree.n, "n_leaves": tree.n_leaves,
                       "depth": tree.depth, "resolution": f"{W}x{H}", "poses": P,
                       "tau_R": tau_R, "lambda_G": args.lambda_g, "tau": tau,
                       "M_mean": round(M_mean, 1), "emitting_mean": round(E_mean, 1),
                       "N_P_mean": round(NP_mean, 1), "rl_cov_nodes_mean": round(cov_mean, 1),
                       "rl_chunks_read_mean": round(chunks_mean, 1),
                       "rl_chunks_total": int((tree.n + 127) // 128),
                       "in_frustum_mean": round(timed_mean("in_frustum"), 1),
                       "work_sample": f"per-frame work averaged over the {K} timed steps' poses "
                                      f"(counted on the device, one counting frame per pose)",
                       "N_P_mean_shrink_off": round(float(np.mean(NP_off)), 1),
                       "l2": "flushed between steps (256 MiB write, outside the step events)",
                       "stream_hold_s": hold_s,
                       "parallelism": f"replicas x{world} (views round-robin)"},
            "stages_ms": {nm: stages[nm]["ms"] for nm in STAGES},
            "stages": stages,
            "roofline": dom_rl,
            "e2e": {"value": round(frames / e2e_s, 2), "unit": "frames/s",
                    "h2d_bytes_per_step": cam_bytes, "d2h_bytes_per_step": img_bytes,
                    "how": "fgs_render with pinned host output buffers, FGS_RENDER_ASYNC (each frame's "
                           "image copy on the context's copy stream overlaps the next frame's "
                           "kernels), wall time of K steps ending with fgs_sync",
                    "synchronous_value": round(frames / e2e_sync_s, 2)},
            "gpu_launches": int(K * launches),
            "blend_work_per_frame": {"entries": round(timed_mean("entries")),
                                     "evaluations": round(timed_mean("evals")),
                                     "alpha_applied": round(timed_mean("hits")),
                                     "entries_with_alpha": round(timed_mean("active"))},
            "filter_vs_levelwise": {
                "parallel_ms": round(float(np.median(filt_par)), 4),
                "levelwise_ms": round(float(np.median(filt_lw)), 4),
                "levels": lw_levels,
                "speedup": round(float(np.median(filt_lw) / np.median(filt_par)), 2),
                "how": "host wall time per call incl. result copy-out, median over poses"},
            "clocks": clk,
            "calibration_s": round(calib_s, 3),
            "batched": batched,
            "backward": backward,
            "shrink_study": study,
            "wall_s_timed": round(wall, 4),
        }
    r.close()
    if world > 1:
        dist.destroy_process_group()
    return result, tree, cams, tau, ln_tau, tau_R, shrunk_images


# ----------------------------------------------------------------------------- oracle

def oracle_sample(tree, cams, tau_R, tau, ln_tau, pose, pix_frac, seed=0):
    """Oracle on one pose: full cut, projection and pairs; per-pixel blending on a random
    fraction of the pixels, scaled to a whole frame.  Returns (seconds per frame, info)."""
    import oracle
    cam = cams[pose]
    p = oracle.Params(tau_R=tau_R, shrink=True, tau=tau, ln_tau=ln_tau)
    t0 = time.perf_counter()
    sel = oracle.filter_dfs(tree, cam, tau_R)
    splat, rect, _ = oracle.project(tree, cam, p, sel)
    keys, vals = oracle.pairs(splat, rect, cam, p)
    t_front = time.perf_counter() - t0
    n = cam.width * cam.height
    rng = np.random.default_rng(seed)
    k = max(1, int(n * pix_frac))
    pix = np.sort(rng.choice(n, size=k, replace=False))
    t0 = time.perf_counter()
    oracle.render_pixels(splat, keys, vals, cam, p, pix)
    t_blend = (time.perf_counter() - t0) * (n / k)
    return t_front + t_blend, {"front_s": t_front, "blend_s_scaled": t_blend, "pixels": k}


CPU_SAMPLE_S = 10.0     # single-thread seconds of whole oracle frames the CPU-baseline leg times
CPU_SAMPLE_MAX = 16     # at most this many poses


HOLD_S_MIN = 0.5        # seconds the stream is held while the host enqueues the timed steps
HOLD_S_PER_STEP = 0.01
HOLD_S_MAX = 5.0


def hold_stream(torch, steps, min_s=HOLD_S_MIN, clock_hz=2.07e9):
    """Enqueue torch's fixed-length spin kernel (a clock-count loop, no flag) on the
    current stream, long enough for the host to enqueue ``steps`` steps behind it
    (at least ``min_s`` seconds).  Returns its nominal length in seconds (0 when
    torch lacks the helper)."""
    spin = getattr(torch.cuda, "_sleep", None)
    if spin is None:
        return 0.0
    s = min(HOLD_S_MAX, max(min_s, HOLD_S_PER_STEP * steps))
    spin(int(s * clock_hz))
    return round(s, 3)


def cpu_sample_poses(n_poses, first):
    """Pose order of the CPU-baseline sample: the poses in ``first``, then every
    eighth pose of the flythrough, then the poses between them."""
    order = list(first)
    for step_off in range(8):
        for k in range(step_off, n_poses, 8):
            if k not in order:
                order.append(k)
    return order


def cpu_baseline(tree, cams, tau_R, tau, ln_tau, shrunk_images):
    """The CPU-baseline leg: the oracle on whole frames, on one thread and on
    every host core (OpenMP; the results are bit-identical).  The single-thread
    run renders poses (those of ``shrunk_images`` first, then spread over the
    flythrough) until CPU_SAMPLE_S seconds are spent or CPU_SAMPLE_MAX poses are
    done; the all-core run renders the same poses.  Untimed, the same leg renders
    the poses of ``shrunk_images`` with the oracle's unshrunk (3-sigma) footprint
    and reports the GPU's shrunk image against it (§3.3: shrinking changes the
    image; reported, not gated)."""
    import oracle
    order = cpu_sample_poses(len(cams), sorted(shrunk_images))
    n_all = oracle.set_threads(0)
    out = {}
    oracle.set_threads(1)
    poses, ts = [], []
    for k in order:
        if len(poses) >= CPU_SAMPLE_MAX or (len(poses) >= len(shrunk_images) and sum(ts) >= CPU_SAMPLE_S):
            break
        t, _ = oracle_sample(tree, cams, tau_R, tau, ln_tau, k, 1.0)
        poses.append(k)
        ts.append(t)
    out["single"] = (len(ts) / sum(ts), sum(ts), 1)
    oracle.set_threads(n_all)
    ts = [oracle_sample(tree, cams, tau_R, tau, ln_tau, k, 1.0)[0] for k in poses]
    out["all"] = (len(ts) / sum(ts), sum(ts), n_all)
    # shrunk GPU image against the unshrunk oracle image, whole frames
    errs = []
    for k in sorted(shrunk_images):
        cam = cams[k]
        p = oracle.Params(tau_R=tau_R)
        fr = oracle.frame(tree, cam, p, blend=True)
        g = shrunk_images[k].astype(np.float64)
        mse = float(np.mean((g - fr.rgb) ** 2))
        errs.append({"pose": k, "psnr_db": round(10 * math.log10(1.0 / mse), 2) if mse > 0 else None,
                     "max_abs": round(float(np.abs(g - fr.rgb).max()), 5),
                     "mean_abs": round(float(np.abs(g - fr.rgb).mean()), 7)})
    v_all, s_all, n = out["all"]
    v_one, s_one, _ = out["single"]
    return {"value": round(v_all, 5), "unit": "frames/s", "cores": n, "kind": "oracle",
            "sample": (f"poses {poses}: {len(poses)} whole frames (LoD cut, projection, pairs, "
                       f"per-pixel blending) on {n} threads, {s_all:.1f}s total"),
            "single_core": {"value": round(v_one, 5), "unit": "frames/s", "cores": 1,
                            "sample": (f"the same {len(poses)} frames on 1 thread, {s_one:.1f}s total "
                                       f"(poses added until {CPU_SAMPLE_S:.0f}s)")},
            "shrink_vs_unshrunk_oracle": {
                "tau": tau, "poses": errs,
                "how": "GPU image at the calibrated tau against the oracle's 3-sigma image of the "
                       "same pose, every pixel (PSNR over [0, 1])"}}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on the machine's host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    oracle.build_lib()
    n_threads = oracle.set_threads(0)
    tree, cams, tau_R, wname = workload(args.workload)
    # Eq. 5-8 on the oracle over every pose, as the GPU arm calibrates
    t0 = time.perf_counter()
    tau, ln_tau, _ = oracle_calibrate_sampled(tree, cams, tau_R)
    calib = time.perf_counter() - t0
    times = []
    for w in range(args.warmup + args.steps):
        t, info = oracle_sample(tree, cams, tau_R, tau, ln_tau, w % len(cams), 1.0 / 64, seed=w)
        if w >= args.warmup:
            times.append(t)
    v = len(times) / sum(times)
    return {"metric": METRIC, "value": round(v, 5), "unit": "frames/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 / v, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator)", "impl": "reference",
            "config": {"workload": wname, "n_nodes": tree.n, "tau": tau,
                       "calibration": f"oracle GTC over all {len(cams)} poses ({calib:.1f}s)"},
            "cpu_baseline": {"value": round(v, 5), "unit": "frames/s", "cores": n_threads,
                             "kind": "oracle",
                             "sample": "per step: one pose, full cut/projection/pairs, "
                                       "per-pixel blend of 1/64 of the pixels scaled to a frame"},
            "e2e": {"value": round(v, 5), "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def oracle_calibrate_sampled(tree, cams, tau_R):
    """Eq. 5-8 on the oracle with KPC from a full-frame render of each pose."""
    import oracle
    gbars = []
    for cam in cams:
        p = oracle.Params(tau_R=tau_R)
        fr = oracle.frame(tree, cam, p, blend=False)
        _, _, kpc = oracle.render(fr.splat, fr.keys, fr.vals, cam, p, want_kpc=True)
        tx, ty = oracle.tiles_of(cam, p)
        _, gbar, _ = oracle.gtc(fr.keys, kpc, tx * ty)
        gbars.append(gbar)
    tau, ln_tau = oracle.tau_from(gbars, 0.2)
    return tau, ln_tau, gbars


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--workload", default="city", choices=["city", "blobs", "tiny"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lambda-g", dest="lambda_g", type=float, default=0.2)
    ap.add_argument("--pair-capacity", type=int, default=64 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--no-backward", dest="backward", action="store_false")
    ap.add_argument("--no-study", dest="study", action="store_false")
    ap.add_argument("--batch-reps", type=int, default=5)
    ap.add_argument("--batch-sel-cap", type=int, default=96 << 20)
    ap.add_argument("--batch-pair-cap", type=int, default=256 << 20)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        res = run_reference(args)
        if res is not None:
            print(json.dumps(res, default=_json_default), flush=True)
        return
    res, tree, cams, tau, ln_tau, tau_R, shrunk_images = run_ours(args)
    if res is None:
        return
    if not args.no_cpu_baseline:
        t0 = time.time()
        res["cpu_baseline"] = cpu_baseline(tree, cams, tau_R, tau, ln_tau, shrunk_images)
        log(f"cpu baseline {time.time() - t0:.1f}s")
    print(json.dumps(res, default=_json_default), flush=True)


if __name__ == "__main__":
    main()
