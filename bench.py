"""Benchmark: Gradient-SDF tracking + fusion on the hashed room workload.

Workload (one "step" = one frame of a SLAM loop): a 640x480 depth frame of a synthetic room
(4x4x3 m, 10 spheres, 6 boxes, noise sigma = 0.0012 z^2) on a smooth 100-frame trajectory,
8^3-block hashed map with 1 cm voxels, T = 5 cm.  Per frame: 10 Gauss-Newton tracking steps
against the map (from the previous frame's estimate), then fusion of the frame at the tracked
pose.  Frame 0 is fused at its true pose.  The first W frames are warm-up, the next K are timed.

value = tracked depth pixels per second per Gauss-Newton iteration over the whole step
        (H*W pixels x 10 iterations x K frames / summed step time);
fused_voxels_per_s = ray-voxel updates per second over the same time.

Rooflines (HBM, against the measured copy bandwidth) are reported for each kernel with two byte
counts.  Per access: a tracking step reads 4 B of depth per pixel and, per usable pixel, one 8 B
block key and the voxel payload (20 B FP32; FP16: 8 B half4 + 4 B W + 4 B block scale; dense grids
have no key); a fusion reads 4 B of depth per pixel and per ray-voxel update probes a key and
read-modify-writes 20 B (the payload, or an FP16 map's frame accumulators, whose distinct voxels the
apply pass then folds).  Compulsory: every distinct voxel and block a pass touches, counted on the
device by gsdf_footprint, read (tracking) or read and written (fusion) once.
Inputs (all depth frames) are resident in HBM before timing; L2 is flushed (a 512 MB write)
between timed steps, outside the timed interval.  e2e repeats the run through the same API
with each frame copied from pinned host memory and the pose read back inside the interval.

Forms (forms_summary holds their headline figures): 64 scenes batched, 50 timed frames, one
gsdf_batch_frame graph per frame (FP32 and FP16 payload) against per-scene calls; the room at 4 mm
for 300 frames with the FP32 and the FP16 payload; the adjoint, bundle adjustment, surface
extraction and the trilinear baseline tracker.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gsdf|reference]
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tracked depth px/s per GN iteration & fused voxels/s; % of HBM peak"
GN_ITERS = 10
SEED = 2
VOXEL = 0.01
HASH_SLOTS = 1 << 18
FALLBACK_HBM_GBS = 6800.0


def workload_name(n_frames):
    return (f"hashed room, 640x480 depth, 8^3 blocks, 1 cm voxels, T=5 cm, {n_frames}-frame spline "
            f"trajectory, {GN_ITERS} GN iterations + 1 fusion per frame")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x, world, device):
    """The largest of a value over the ranks, on every rank (the slowest rank's time bounds the
    whole job).  `device` is where the process group's backend reduces: a CUDA device for NCCL,
    the CPU for gloo."""
    if world == 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, t_max):
    """Whole-job throughput: every rank processes units_per_rank in at most t_max seconds."""
    return world * units_per_rank / t_max


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d and isinstance(d[k], (int, float)):
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# the sources each profiled kernel is compiled from
KERNEL_SOURCES = {
    "track_chain_kernel": ("track.cu", "track_device.cuh", "gsdf_internal.cuh"),
    "integrate_kernel": ("integrate.cu", "integrate_device.cuh", "gsdf_internal.cuh"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2111_13652_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha") != kernel_source_hash(kernel):
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sms, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sms)}


def make_sequence(n_frames, processes=1):
    from paper_2111_13652_gb300 import inputs as I

    return I.room_sequence(seed=SEED, n_frames=n_frames, voxel_size=VOXEL, processes=processes)


# -----------------------------------------------------------------------------------------------
# oracle (CPU) timing: the reference arm and the cpu_baseline leg
# -----------------------------------------------------------------------------------------------


def run_oracle(seq, first, count):
    """Oracle SLAM loop: fuse frame 0 at its true pose, then frames 1..first+count-1 with
    tracking; returns the time of frames first..first+count-1 and their units."""
    from oracle import oracle as O

    om = O.OracleMap(O.params(VOXEL))
    om.integrate(seq.depths[0], seq.cam, seq.poses[0])
    T = seq.poses[0].copy()
    t_sum, visits = 0.0, 0
    for f in range(1, first + count):
        t0 = time.perf_counter()
        for _ in range(GN_ITERS):
            T, _ = om.track_step(seq.depths[f], seq.cam, T)
        st = om.integrate(seq.depths[f], seq.cam, T)
        dt = time.perf_counter() - t0
        if f >= first:
            t_sum += dt
            visits += st.n_visits
    px = seq.cam.width * seq.cam.height * GN_ITERS * count
    return t_sum, px, visits


def _oracle_replica(args):
    """One single-threaded oracle process of the all-core CPU leg: fuse frame 0 and run the frames
    before `first`, wait for every replica, then time frames first..first+count-1."""
    depths, cam, poses, first, count, barrier = args
    from oracle import oracle as O

    om = O.OracleMap(O.params(VOXEL))
    om.integrate(depths[0], cam, poses[0])
    T = poses[0].copy()

    def frame(f, T):
        for _ in range(GN_ITERS):
            T, _ = om.track_step(depths[f], cam, T)
        om.integrate(depths[f], cam, T)
        return T

    for f in range(1, first):
        T = frame(f, T)
    barrier.wait()
    t0 = time.time()
    for f in range(first, first + count):
        T = frame(f, T)
    return t0, time.time(), cam.width * cam.height * GN_ITERS * count


def run_oracle_replicas(seq, first, count, n):
    """The oracle on every host core at once: n independent replicas of run_oracle's loop in spawned
    processes, released together; the units of all of them over the span from the first start to
    the last end."""
    import concurrent.futures as cf
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    k = first + count
    from paper_2111_13652_gb300 import inputs as I

    with I._SingleThreadedChildren(), ctx.Manager() as mgr:
        bar = mgr.Barrier(n)
        job = (seq.depths[:k], seq.cam, [np.asarray(T) for T in seq.poses[:k]], first, count, bar)
        with cf.ProcessPoolExecutor(n, mp_context=ctx) as ex:
            res = list(ex.map(_oracle_replica, [job] * n))
    span = max(r[1] for r in res) - min(r[0] for r in res)
    return sum(r[2] for r in res) / span


def forms_summary(forms):
    """The headline figures of every form, kept short so that they appear early in the line."""
    out = {}
    b = forms.get("batched_64_scenes")
    if b:
        sp = b["split"]
        out["batched_64_scenes"] = {
            "px_per_s": b["value"], "fp16_px_per_s": b["fp16_value"], "plain_px_per_s": b["plain_value"],
            "ms_per_frame": b["ms_per_frame"], "speedup_vs_plain": b["speedup_vs_plain"],
            "fp16_speedup_vs_plain": b["fp16_speedup_vs_plain"],
            "max_pose_error_in_voxels": {k: b["pose_accuracy"][k]["max_in_voxels"]
                                         for k in ("batched", "batched_fp16", "plain")},
            "accuracy_gate": b["pose_accuracy"]["gate_all_scenes_within_2_voxels"],
            "hbm_frac": {m: {k: {kk: sp[m][k][kk]["frac"] for kk in ("per_access", "per_access_usable", "compulsory")
                                 if kk in sp[m][k]} for k in ("track", "fusion")}
                         for m in sp}}
    f = forms.get("fp16_payload_4mm")
    if f:
        last = str(FP16_FRAMES)
        out["fp16_payload_4mm"] = {
            "ms_per_frame": {m: f[m]["ms_per_frame"] for m in ("fp32", "fp16")},
            "voxels": f["fp16"]["voxels"],
            "pose_error_m_at_300": {m: f[m]["pose_error_m"][last] for m in ("fp32", "fp16")},
            "fp16_vs_fp32_at_300_same_poses": {k: f["checkpoints"][last]["fields_fp16_vs_fp32_same_poses"][k]
                                               for k in ("max_dpsi", "mean_dpsi", "max_dghat", "mean_dghat")},
            "hbm_frac": {m: {k: {kk: f[m]["roofline"][k][kk]["frac"] for kk in ("per_access", "per_access_usable", "compulsory")
                                 if kk in f[m]["roofline"][k]} for k in ("track", "fusion")}
                         for m in ("fp32", "fp16")}}
    a = forms.get("adjoint_10_keyframes")
    if a:
        out["adjoint_10_keyframes"] = {"gradient_evaluations_per_s": a["gradient_evaluations_per_s"],
                                       "hbm_frac": a["hbm_frac_energy_and_gradient"]}
    t = forms.get("taylor_vs_trilinear_room640")
    if t:
        out["taylor_vs_trilinear"] = {"tracking_speedup": t["tracking_speedup_taylor_vs_trilinear"]}
    return out


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = max(100, 1 + args.warmup + args.steps)
    seq = make_sequence(1 + args.warmup + args.steps)  # the trajectory's prefix is independent of its length
    first = 1 + args.warmup
    t, px, visits = run_oracle(seq, first, args.steps)
    value = px / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "px/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(n)},
            "fused_voxels_per_s": visits / t,
            "cpu_baseline": {"value": value, "unit": "px/s", "cores": 1, "kind": "oracle",
                             "sample": f"frames {first}..{first + args.steps - 1} of the workload, single-threaded"},
            "e2e": {"value": value, "unit": "px/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -----------------------------------------------------------------------------------------------
# GPU arm
# -----------------------------------------------------------------------------------------------


def gpu_arm(args):
    import torch

    from paper_2111_13652_gb300 import gsdf as G

    rank, world, local = dist_env()
    procs = max(1, min(16, os.cpu_count() or 1))
    batch_scenes = None
    if not args.no_batch_form:
        from paper_2111_13652_gb300 import inputs as I

        # ray-cast the batch workload in a spawned pool before the first CUDA call
        batch_scenes = I.batch_scenes(BATCH_SCENES, 1 + BATCH_WARMUP + BATCH_STEPS, processes=procs)
    fp16_seq = None
    if not args.no_fp16_form:
        from paper_2111_13652_gb300 import inputs as I

        # the 4 mm room: 300 frames at 0.5 cm per frame
        fp16_seq = I.room_sequence(seed=SEED, n_frames=1 + FP16_FRAMES, voxel_size=FP16_VOXEL,
                                   frames_per_segment=75, processes=procs, conditioned_horizon=1 + FP16_FRAMES)
    keyframes = None
    if not args.no_adjoint_form:
        from paper_2111_13652_gb300 import inputs as I

        keyframes = I.keyframes(seed=SEED, n_keyframes=ADJ_KEYFRAMES, stride=ADJ_STRIDE, voxel_size=VOXEL)
    n_frames = max(100, 1 + args.warmup + args.steps)
    seq = make_sequence(n_frames, procs)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    G.load_library()
    H, W = seq.cam.height, seq.cam.width
    K = G.intrinsics(seq.cam)
    stream = torch.cuda.current_stream(dev)
    depths = torch.from_numpy(seq.depths).to(dev)  # inputs resident in HBM
    gt0 = torch.from_numpy(np.ascontiguousarray(seq.poses[0])).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    n_steps_total = args.warmup + args.steps
    first = 1

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def run(e2e: bool):
        m = G.Map(G.make_config(VOXEL, hash_slots=HASH_SLOTS), stream)
        pose = gt0.clone()
        dbuf = torch.empty((H, W), dtype=torch.float32, device=dev)  # depth staging buffer
        dbuf.copy_(depths[0])
        m.integrate(dbuf, K, pose)
        # the graph-replayed calls write fixed statistics buffers; they are copied out per step
        tbuf = m.new_track_stats(GN_ITERS)
        ibuf = m.new_integrate_stats()
        tstats = torch.zeros((args.steps, GN_ITERS, G.TRACK_STATS_BYTES), dtype=torch.uint8, device=dev)
        istats = torch.zeros((args.steps, G.INTEGRATE_STATS_BYTES), dtype=torch.uint8, device=dev)
        host_depth = torch.from_numpy(seq.depths).pin_memory() if e2e else None
        host_pose = torch.empty(16, dtype=torch.float64).pin_memory()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        launches = 0
        for s in range(n_steps_total):
            f = first + s
            timed = s >= args.warmup
            k = s - args.warmup
            if timed and k == 0:
                barrier()
                wall0 = time.perf_counter()
            if timed:
                flush.fill_(s & 0xFF)  # evict L2 before the step (not timed)
                ev[k][0].record(stream)
            dbuf.copy_(host_depth[f] if e2e else depths[f], non_blocking=True)
            if timed:
                ev[k][1].record(stream)
            m.track(dbuf, K, pose, GN_ITERS, tbuf)
            if timed:
                ev[k][2].record(stream)
            m.integrate(dbuf, K, pose, ibuf)
            if e2e:
                host_pose.copy_(pose.view(-1), non_blocking=True)
            if timed:
                ev[k][3].record(stream)
                launches += GN_ITERS + 3  # chained tracking steps, final solve, fusion, statistics kernel
                tstats[k].copy_(tbuf)
                istats[k].copy_(ibuf)
            if e2e:
                stream.synchronize()
        barrier()
        wall = time.perf_counter() - wall0
        m.sync()
        step_ms = np.array([e[0].elapsed_time(e[3]) for e in ev])
        track_ms = np.array([e[1].elapsed_time(e[2]) for e in ev])
        int_ms = np.array([e[2].elapsed_time(e[3]) for e in ev])
        ts = tstats.cpu().numpy()
        ist = istats.cpu().numpy()
        n_valid = np.array([[G.track_stats_from_bytes(ts[k, i]).n_valid for i in range(GN_ITERS)]
                            for k in range(args.steps)])
        visits = np.array([G.integrate_stats_from_bytes(ist[k]).n_visits for k in range(args.steps)])
        blocks = G.integrate_stats_from_bytes(ist[-1]).n_blocks_total
        final_pose = pose.cpu().numpy()
        # distinct voxels and blocks of the last frame's tracking and fusion (compulsory bytes)
        fp_t = m.footprint(G.GSDF_FOOTPRINT_TRACK, dbuf, K, pose)
        fp_f = m.footprint(G.GSDF_FOOTPRINT_FUSE, dbuf, K, pose)
        m.close()
        return dict(step_ms=step_ms, track_ms=track_ms, int_ms=int_ms, n_valid=n_valid, visits=visits,
                    blocks=blocks, wall=wall, launches=launches, pose=final_pose, fp_t=fp_t, fp_f=fp_f)

    with ClockSampler(local) as clk:
        r = run(e2e=False)
        r2 = run(e2e=True)
        forms = {}
        hbm = measured_hbm_peak()[0]
        if batch_scenes is not None:
            forms["batched_64_scenes"] = batch_form(G, torch, dev, stream, batch_scenes, hbm)
        if not args.no_fp16_form:
            forms["fp16_payload_4mm"] = fp16_form(G, torch, dev, stream, fp16_seq, hbm)
        if keyframes is not None:
            forms["adjoint_10_keyframes"] = adjoint_form(G, torch, dev, stream, keyframes, measured_hbm_peak()[0])
            if not args.no_ba_form:
                forms["ba_10_keyframes"] = ba_form(G, torch, dev, stream, keyframes)
        if not args.no_points_form:
            forms["points_room640"] = points_form(G, torch, dev, stream, seq)
        if not args.no_trilinear_form:
            forms["taylor_vs_trilinear_room640"] = trilinear_form(G, torch, dev, stream, seq)
    clocks = clk.summary()
    clocks["window"] = "whole GPU run (warm-up, timed steps, e2e repeat); 100 ms sampling"

    t_total = reduce_max(float(r["step_ms"].sum()) / 1e3, world, dev)
    t_e2e = reduce_max(float(r2["step_ms"].sum()) / 1e3, world, dev)
    px_units = H * W * GN_ITERS * args.steps
    value = job_rate(world, px_units, t_total)
    visits_total = float(r["visits"].sum())
    # roofline of the two kernels; the dominant one (larger share of step time) is reported
    hbm, hbm_kind = measured_hbm_peak()
    # tracking: nominal per-access bytes (40 B per pixel) for `achieved`; the implementation's own
    # per-access count (usable pixels only, its 8 B key) and the compulsory bytes beside it
    track_s = r["track_ms"].sum() / 1e3
    track_nom_gbs = float(track_bytes_nominal("f32", H * W) * GN_ITERS * args.steps / track_s / 1e9)
    track_b = track_bytes("f32", H * W, r["n_valid"])  # per launch (per access, usable pixels)
    track_gbs = float(track_b.sum() / track_s / 1e9)  # 10 launches per interval
    int_b = fuse_bytes("f32", H * W, r["visits"])
    int_gbs = float(int_b.sum() / (r["int_ms"].sum() / 1e3) / 1e9)
    step_s = float(r["track_ms"].mean()) / 1e3 / GN_ITERS
    fuse_s = float(r["int_ms"].mean()) / 1e3
    share_track = float(r["track_ms"].sum() / r["step_ms"].sum())  # the rest: staging copy
    share_int = float(r["int_ms"].sum() / r["step_ms"].sum())
    if share_int >= share_track:
        dom, ach, traffic = "integrate_kernel", int_gbs, profiled_traffic("integrate_kernel")
    else:
        dom, ach, traffic = "track_chain_kernel", track_nom_gbs, profiled_traffic("track_chain_kernel")
    roofline = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
            "kernel": dom, "peak_source": hbm_kind,
            "bytes": "per access (algorithmic): tracking 40 B per pixel (4 B depth + 20 B payload + 16 B hash "
                     "slot, every pixel, no reuse); fusion 4 B per pixel + 48 B (key + 20 B read-modify-write) "
                     "per ray-voxel update",
            "kernels": {"track_chain_kernel": {"GBs": track_nom_gbs, "share": share_track,
                                         "per_access_usable": {"GBs": track_gbs, "frac": track_gbs / hbm,
                                                       "bytes": "4 B per pixel + 28 B (8 B key + 20 B payload) "
                                                                "per usable pixel"},
                                         "us_per_launch": 1e6 * step_s,
                                         "launches": f"{GN_ITERS} chained steps and one final solve per frame; "
                                                     f"time per Gauss-Newton step",
                                         "compulsory": roof(track_bytes("f32", H * W, 0, *r["fp_t"]), step_s, hbm),
                                         "distinct_voxels": r["fp_t"][0]},
                        "integrate_kernel": {"GBs": int_gbs, "share": share_int,
                                             "us_per_launch": 1e6 * fuse_s,
                                             "compulsory": roof(fuse_bytes("f32", H * W, 0, *r["fp_f"]), fuse_s, hbm),
                                             "distinct_voxels": r["fp_f"][0]}},
            "l2_note": "a 640x480 frame's tracking and fusion working set (a few MB) is L2-resident after the "
                       "first Gauss-Newton step; see forms.*.split / roofline for the batched and 4 mm forms"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        first_cpu, count = 1, 3
        t_cpu, px_cpu, _ = run_oracle(seq, first_cpu, count)
        cpu = {"value": px_cpu / t_cpu, "unit": "px/s", "cores": 1, "kind": "oracle",
               "sample": f"frames {first_cpu}..{first_cpu + count - 1} of the same sequence "
                         f"({GN_ITERS} GN steps + fusion each), single-threaded"}
        ncores = os.cpu_count() or 1
        v_all = run_oracle_replicas(seq, first_cpu, count, ncores)
        cpu["all_cores"] = {"value": v_all, "unit": "px/s", "cores": ncores, "kind": "oracle",
                            "sample": f"{ncores} independent single-threaded oracle processes (one per host "
                                      f"core), each on frames {first_cpu}..{first_cpu + count - 1}; "
                                      f"units of all of them over the slowest one's time"}
    if rank == 0:
        gt = seq.poses[first + n_steps_total - 1]
        line = {
            "metric": METRIC, "value": value, "unit": "px/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(n_frames), "l2": "flushed (512 MB write) before every timed step",
                       "parallelism": f"{world} independent replica(s)", "hash_slots": HASH_SLOTS},
            "fused_voxels_per_s": job_rate(world, visits_total, t_total),
            "track_px_per_s_kernel_only": H * W * GN_ITERS * args.steps / (r["track_ms"].sum() / 1e3),
            "roofline": roofline,
            "forms_summary": forms_summary(forms),
            "forms": forms,
            "cpu_baseline": cpu,
            "e2e": {"value": job_rate(world, px_units, t_e2e), "unit": "px/s", "h2d_bytes_per_step": H * W * 4,
                    "d2h_bytes_per_step": 16 * 8},
            "gpu_launches": r["launches"],
            "clocks": clocks,
            "blocks_allocated": int(r["blocks"]),
            "final_pose_error_m": float(np.linalg.norm(r["pose"][:3, 3] - gt[:3, 3])),
            "wall_s_timed_region": r["wall"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


BATCH_SCENES = 64
BATCH_WARMUP = 3
BATCH_STEPS = 50
BATCH_SPLIT_STEPS = 10

# bytes a tracking step and a fusion read or write, per unit, by payload kind ("dense", "f32",
# "f16"); see the roofline paragraphs of the module docstring
SLOT_B = {"dense": 0, "f32": 8, "f16": 8}       # the 8 B block key probed per lookup
PAYLOAD_B = {"dense": 20, "f32": 20, "f16": 16}  # per lookup: float4 + W (FP16: half4 + W + block scale)
VOXEL_B = {"dense": 20, "f32": 20, "f16": 12}    # per distinct voxel (FP16: half4 + W)
BLOCK_B = {"dense": 0, "f32": 8, "f16": 12}      # per distinct block (key; FP16 also its scale)


# Nominal per-access bytes of one tracking lookup per pixel, with no reuse and every pixel counted:
# 4 B of depth, the payload (FP32 20 B; FP16 10 B: psi, gbar and W at 2 B each) and a 16 B hash
# slot (key and block index; none for a dense grid).
NOMINAL_PX_B = {"dense": 4 + 20, "f32": 4 + 20 + 16, "f16": 4 + 10 + 16}


def track_bytes_nominal(kind, n_px):
    """One tracking step, nominal per-access bytes: NOMINAL_PX_B per pixel of the frame."""
    return NOMINAL_PX_B[kind] * n_px


def track_bytes(kind, n_px, n_valid, vox=None, blocks=None):
    """One tracking step: per access (4 B of depth per pixel, one key probe and one payload read per
    usable pixel) or, given the distinct voxels and blocks, compulsory (each read once)."""
    if vox is None:
        return 4 * n_px + (SLOT_B[kind] + PAYLOAD_B[kind]) * n_valid
    return 4 * n_px + VOXEL_B[kind] * vox + BLOCK_B[kind] * blocks


def fuse_bytes(kind, n_px, visits, vox=None, blocks=None):
    """One fusion: per access (4 B of depth per pixel; per ray-voxel update one key probe and a
    20 B read-modify-write of the FP32 payload or, for FP16 maps, of the frame accumulators, whose
    distinct voxels are then folded: sums read and cleared, payload read and written) or compulsory
    (each distinct voxel's payload read and written once, each block's key once)."""
    if vox is None:
        b = 4 * n_px + (8 + 40) * visits
        return b
    return 4 * n_px + 2 * VOXEL_B[kind] * vox + BLOCK_B[kind] * blocks


def fp16_apply_bytes(vox, blocks):
    """The FP16 apply pass per access: each listed block's 512 weight sums, and per distinct voxel
    its sums (read 20 B, cleared 20 B) and payload (read and written, 12 B each)."""
    return 4 * 512 * blocks + (20 + 20 + 12 + 12) * vox


def roof(bytes_per_unit, seconds_per_unit, peak):
    gbs = bytes_per_unit / seconds_per_unit / 1e9
    return {"GBs": gbs, "frac": gbs / peak}


def observable(sc, T):
    """What tracking can determine: the camera position in a room, the camera-frame centre of the
    sphere (at the origin) in a sphere-only scene."""
    T = np.asarray(T)
    return T[:3, :3].T @ (-T[:3, 3]) if sc.dense_dims is not None else T[:3, 3]


def batch_form(G, torch, dev, stream, scenes, hbm):
    """64 independent scenes (160x120..640x480, dense 64^3 spheres and hashed rooms, 1-4 cm voxels):
    each frame runs 10 Gauss-Newton steps and fusion of every scene.  Batched: one gsdf_batch_frame
    per frame (one CUDA graph: persistent tracking launches, persistent fusion, depth pointers
    advanced on the device), with the FP32 payload and with the rooms in FP16; plain: per-scene
    calls.  A split run times the batched tracking and fusion kernels apart for their rooflines."""
    n = len(scenes)
    Ks = [G.intrinsics(sc.cam) for sc in scenes]
    depths = [torch.from_numpy(sc.depths).to(dev) for sc in scenes]  # (F, H, W) per scene, in HBM
    n_px = [sc.cam.width * sc.cam.height for sc in scenes]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    last = BATCH_WARMUP + BATCH_STEPS

    def kinds(fp16):
        return ["dense" if sc.dense_dims is not None else ("f16" if fp16 else "f32") for sc in scenes]

    def make_maps(fp16):
        maps = []
        for sc in scenes:
            if sc.dense_dims is not None:
                cfg = G.make_config(sc.voxel_size, dense_dims=sc.dense_dims, dense_origin=sc.dense_origin,
                                    damping=sc.damping)
            else:
                cfg = G.make_config(sc.voxel_size, hash_slots=sc.hash_slots, damping=sc.damping, fp16=fp16,
                                    max_touched_blocks=sc.hash_slots // 2)
            maps.append(G.Map(cfg, stream))
        return maps

    px_per_iter = sum(n_px)
    out = {}
    for mode in ("batched", "batched_fp16", "plain"):
        maps = make_maps(mode == "batched_fp16")
        poses = [torch.from_numpy(np.ascontiguousarray(sc.poses[0])).to(dev) for sc in scenes]
        istats = torch.zeros((n, G.INTEGRATE_STATS_BYTES), dtype=torch.uint8, device=dev)
        ist_all = torch.zeros((BATCH_STEPS, n, G.INTEGRATE_STATS_BYTES), dtype=torch.uint8, device=dev)
        batch, tiles = None, None
        if mode != "plain":
            batch = G.Batch(maps, stream)
            batch.set_frames([d[0] for d in depths], Ks, poses, integrate_stats=istats)
            batch.set_depth_stride(n_px)
            batch.frame(0)  # frame 0 fused at its true pose; the depth pointers now sit at frame 1
            tiles = batch.autotune()  # untimed: tile size and CTAs per SM for these frame sizes
        else:
            staging = [torch.empty_like(d[0]) for d in depths]
            for s in range(n):
                maps[s].integrate(depths[s][0], Ks[s], poses[s])
        ev = []
        for f in range(1, last + 1):
            timed = f > BATCH_WARMUP
            if timed:
                flush.fill_(f & 0xFF)  # evict L2 (not timed)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            if batch is not None:
                batch.frame(GN_ITERS)
            else:  # each scene through its own handle; a staging buffer keeps gsdf_track a graph replay
                for s in range(n):
                    staging[s].copy_(depths[s][f], non_blocking=True)
                    maps[s].track(staging[s], Ks[s], poses[s], GN_ITERS)
                    maps[s].integrate(staging[s], Ks[s], poses[s], istats[s])
            if timed:
                e1.record(stream)
                ev.append((e0, e1))
                ist_all[f - 1 - BATCH_WARMUP].copy_(istats)
        torch.cuda.synchronize(dev)
        ms = float(sum(a.elapsed_time(b) for a, b in ev))
        ist = ist_all.cpu().numpy()
        visits = sum(G.integrate_stats_from_bytes(ist[k, s]).n_visits for k in range(BATCH_STEPS) for s in range(n))
        final = [p.cpu().numpy() for p in poses]
        err = [float(np.linalg.norm(observable(sc, T) - observable(sc, sc.poses[last]))) for sc, T in zip(scenes, final)]
        status = [int(G.gsdf_sync(m.h)) for m in maps]
        out[mode] = dict(ms=ms, visits=visits, final=final, err=err, tiles=tiles, status=status)
        if batch is not None:
            batch.close()
        for m in maps:
            m.close()
    b, b16, pl = out["batched"], out["batched_fp16"], out["plain"]

    # split run: the batched tracking and fusion kernels timed apart, for their rooflines
    split = {}
    for mode in ("batched", "batched_fp16"):
        fp16 = mode == "batched_fp16"
        maps = make_maps(fp16)
        poses = [torch.from_numpy(np.ascontiguousarray(sc.poses[0])).to(dev) for sc in scenes]
        tstats = torch.zeros((n, G.TRACK_STATS_BYTES), dtype=torch.uint8, device=dev)
        istats = torch.zeros((n, G.INTEGRATE_STATS_BYTES), dtype=torch.uint8, device=dev)
        batch = G.Batch(maps, stream)
        batch.set_frames([d[0] for d in depths], Ks, poses, tstats, istats)
        batch.integrate()
        batch.autotune()
        t_track, t_fuse, valid, visits = 0.0, 0.0, [], []
        for f in range(1, 1 + BATCH_WARMUP + BATCH_SPLIT_STEPS):
            batch.set_frames([d[f] for d in depths], Ks, poses, tstats, istats)
            flush.fill_(f & 0xFF)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            batch.track(GN_ITERS)
            e[1].record(stream)
            batch.integrate()
            e[2].record(stream)
            torch.cuda.synchronize(dev)
            if f > BATCH_WARMUP:
                t_track += e[0].elapsed_time(e[1]) / 1e3
                t_fuse += e[1].elapsed_time(e[2]) / 1e3
                ts, ist = tstats.cpu().numpy(), istats.cpu().numpy()
                # per-step usable pixels: the last step's count (the count barely moves over the steps)
                valid += [G.track_stats_from_bytes(ts[s]).n_valid for s in range(n)]
                visits += [G.integrate_stats_from_bytes(ist[s]).n_visits for s in range(n)]
        # distinct voxels and blocks of the last frame (compulsory bytes), per scene
        fl = BATCH_WARMUP + BATCH_SPLIT_STEPS
        fp_t = [maps[s].footprint(G.GSDF_FOOTPRINT_TRACK, depths[s][fl], Ks[s], poses[s]) for s in range(n)]
        fp_f = [maps[s].footprint(G.GSDF_FOOTPRINT_FUSE, depths[s][fl], Ks[s], poses[s]) for s in range(n)]
        batch.close()
        for m in maps:
            m.close()
        kd = kinds(fp16)
        k_steps = BATCH_SPLIT_STEPS
        valid_mean = np.sum(np.reshape(valid, (k_steps, n)), axis=0) / k_steps
        visits_mean = np.sum(np.reshape(visits, (k_steps, n)), axis=0) / k_steps
        tb_nom = sum(track_bytes_nominal(kd[s], n_px[s]) for s in range(n))
        tb_acc = sum(track_bytes(kd[s], n_px[s], valid_mean[s]) for s in range(n))
        tb_cmp = sum(track_bytes(kd[s], n_px[s], 0, *fp_t[s]) for s in range(n))
        fb_acc = sum(fuse_bytes(kd[s], n_px[s], visits_mean[s]) for s in range(n))
        fb_acc += sum(fp16_apply_bytes(*fp_f[s]) for s in range(n) if kd[s] == "f16")
        fb_cmp = sum(fuse_bytes(kd[s], n_px[s], 0, *fp_f[s]) for s in range(n))
        step_s = t_track / (k_steps * GN_ITERS)
        fuse_s = t_fuse / k_steps
        split[mode] = {
            "track": {"kernel": "batch_track_kernel", "us_per_step": 1e6 * step_s,
                      "bytes_per_step": {"per_access": tb_nom, "per_access_usable": tb_acc, "compulsory": tb_cmp},
                      "per_access": roof(tb_nom, step_s, hbm), "per_access_usable": roof(tb_acc, step_s, hbm),
                      "compulsory": roof(tb_cmp, step_s, hbm),
                      "distinct_voxels": int(sum(x[0] for x in fp_t)), "usable_px": float(np.sum(valid_mean))},
            "fusion": {"kernel": "batch_integrate_kernel" + (" + batch_list16/apply16" if fp16 else ""),
                       "us_per_frame": 1e6 * fuse_s,
                       "bytes_per_frame": {"per_access": fb_acc, "compulsory": fb_cmp},
                       "per_access": roof(fb_acc, fuse_s, hbm), "compulsory": roof(fb_cmp, fuse_s, hbm),
                       "distinct_voxels": int(sum(x[0] for x in fp_f)), "visits": float(np.sum(visits_mean))},
        }

    def acc(r):
        e = np.array(r["err"])
        vs = np.array([sc.voxel_size for sc in scenes])
        worst = int(np.argmax(e / vs))
        return {"mean_m": float(e.mean()), "max_m": float(e.max()), "max_in_voxels": float((e / vs).max()),
                "worst_scene": worst, "scenes_over_2_voxels": int(np.sum(e > 2 * vs)),
                "per_scene_m": [round(x, 5) for x in e.tolist()]}

    def diff(x, y):
        return max(float(np.linalg.norm(observable(sc, p) - observable(sc, q)))
                   for sc, p, q in zip(scenes, x["final"], y["final"]))

    units = px_per_iter * GN_ITERS * BATCH_STEPS
    a_b, a_16, a_pl = acc(b), acc(b16), acc(pl)
    return {
        "workload": f"{n} scenes: 160x120/320x240/480x360/640x480 by index mod 4, dense 64^3 sphere grid "
                    f"(index mod 4 = 0) or hashed room, voxels 1-4 cm; per frame {GN_ITERS} GN steps + fusion of "
                    f"every scene; frame 0 fused at its true pose, {BATCH_WARMUP} warm-up frames, {BATCH_STEPS} "
                    f"timed; L2 flushed before every timed frame",
        "value": units / (b["ms"] / 1e3), "unit": "px/s", "ms_per_frame": b["ms"] / BATCH_STEPS,
        "fused_voxels_per_s": b["visits"] / (b["ms"] / 1e3),
        "fp16_value": units / (b16["ms"] / 1e3), "fp16_ms_per_frame": b16["ms"] / BATCH_STEPS,
        "plain_value": units / (pl["ms"] / 1e3), "plain_ms_per_frame": pl["ms"] / BATCH_STEPS,
        "speedup_vs_plain": pl["ms"] / b["ms"], "fp16_speedup_vs_plain": pl["ms"] / b16["ms"],
        "graph": "one gsdf_batch_frame (one CUDA graph launch) per frame",
        "autotuned": {"tile_px": b["tiles"][0], "ctas_per_sm": b["tiles"][1]},
        "pose_accuracy": {
            "measure": "camera position for rooms; camera-frame sphere centre for sphere-only scenes (rotations "
                       "about the sphere are unobservable); metres, after the last timed frame",
            "batched": a_b, "batched_fp16": a_16, "plain": a_pl,
            "max_diff_batched_vs_plain": diff(b, pl), "max_diff_fp16_vs_fp32": diff(b16, b),
            "gate_all_scenes_within_2_voxels": a_b["scenes_over_2_voxels"] == 0 and a_16["scenes_over_2_voxels"] == 0},
        "map_status": {"batched": max(b["status"]), "batched_fp16": max(b16["status"]), "plain": max(pl["status"])},
        "split": split,
    }


FP16_VOXEL = 0.004
FP16_SLOTS = 1 << 17
FP16_FRAMES = 300
FP16_CHECKS = (1, 10, 100, 300)


def fp16_form(G, torch, dev, stream, seq, hbm):
    """The room at 4 mm voxels (T = 2 cm), 300 frames at 0.5 cm per frame: the per-frame loop with the
    FP32 payload and with the FP16 payload (per-block scale), same frames, same timing rules; pose
    errors at frames 1, 10, 100 and 300, and the FP16 fields against the FP32 fields there."""
    K = G.intrinsics(seq.cam)
    H, W = seq.cam.height, seq.cam.width
    depths = torch.from_numpy(seq.depths).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    out, fields, poses_at = {}, {}, {}
    track_fp32 = torch.zeros((FP16_FRAMES + 1, 4, 4), dtype=torch.float64, device=dev)  # the FP32 run's poses
    for mode in ("fp32", "fp16"):
        m = G.Map(G.make_config(FP16_VOXEL, hash_slots=FP16_SLOTS, fp16=(mode == "fp16"),
                                max_touched_blocks=FP16_SLOTS // 2), stream)
        pose = torch.from_numpy(np.ascontiguousarray(seq.poses[0])).to(dev)
        dbuf = torch.empty((H, W), dtype=torch.float32, device=dev)
        dbuf.copy_(depths[0])
        m.integrate(dbuf, K, pose)
        tstats = m.new_track_stats(GN_ITERS)
        istats = m.new_integrate_stats()
        valid = torch.zeros(FP16_FRAMES, dtype=torch.int64, device=dev)
        visits = torch.zeros(FP16_FRAMES, dtype=torch.int64, device=dev)
        ev = []
        fields[mode], poses_at[mode] = {}, {}
        for f in range(1, FP16_FRAMES + 1):
            flush.fill_(f & 0xFF)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            dbuf.copy_(depths[f], non_blocking=True)
            m.track(dbuf, K, pose, GN_ITERS, tstats)
            e[1].record(stream)
            m.integrate(dbuf, K, pose, istats)
            e[2].record(stream)
            ev.append(e)
            valid[f - 1] = tstats[GN_ITERS - 1].view(torch.int64)[28]  # n_valid of the last step
            visits[f - 1] = istats.view(torch.int64)[1]
            if mode == "fp32":
                track_fp32[f] = pose
            if f in FP16_CHECKS:  # untimed: pose and fields at the checkpoint
                torch.cuda.synchronize(dev)
                poses_at[mode][f] = pose.cpu().numpy()
                v = m.extract()
                fields[mode][f] = v
        torch.cuda.synchronize(dev)
        st = G.gsdf_sync(m.h)
        fp_t = m.footprint(G.GSDF_FOOTPRINT_TRACK, dbuf, K, pose)
        fp_f = m.footprint(G.GSDF_FOOTPRINT_FUSE, dbuf, K, pose)
        t_frame = np.array([e[0].elapsed_time(e[2]) for e in ev]) / 1e3
        t_track = np.array([e[0].elapsed_time(e[1]) for e in ev]) / 1e3
        t_fuse = np.array([e[1].elapsed_time(e[2]) for e in ev]) / 1e3
        kind = "f16" if mode == "fp16" else "f32"
        nv, nvis = valid.cpu().numpy(), visits.cpu().numpy()
        # the last 100 frames (the map at its full size) for the rooflines
        sl = slice(FP16_FRAMES - 100, FP16_FRAMES)
        step_s = float(t_track[sl].mean()) / GN_ITERS
        fuse_s = float(t_fuse[sl].mean())
        tb_nom = track_bytes_nominal(kind, H * W)
        tb_acc = track_bytes(kind, H * W, float(nv[sl].mean()))
        tb_cmp = track_bytes(kind, H * W, 0, *fp_t)
        fb_acc = fuse_bytes(kind, H * W, float(nvis[sl].mean())) + (fp16_apply_bytes(*fp_f) if kind == "f16" else 0)
        fb_cmp = fuse_bytes(kind, H * W, 0, *fp_f)
        out[mode] = {
            "ms_per_frame": 1e3 * float(t_frame.mean()),
            "track_us_per_step": 1e6 * step_s,
            "integrate_us": 1e6 * float(t_fuse.mean()),
            "voxels": int(len(fields[mode][FP16_FRAMES])), "blocks": m.num_blocks(),
            "payload_bytes_per_voxel": VOXEL_B[kind],
            "pose_error_m": {str(c): float(np.linalg.norm(poses_at[mode][c][:3, 3] - seq.poses[c][:3, 3]))
                             for c in FP16_CHECKS},
            "status": int(st),
            "roofline": {
                "track": {"us_per_step": 1e6 * step_s, "per_access": roof(tb_nom, step_s, hbm),
                          "per_access_usable": roof(tb_acc, step_s, hbm),
                          "compulsory": roof(tb_cmp, step_s, hbm), "distinct_voxels": fp_t[0]},
                "fusion": {"us_per_frame": 1e6 * fuse_s, "per_access": roof(fb_acc, fuse_s, hbm),
                           "compulsory": roof(fb_cmp, fuse_s, hbm), "distinct_voxels": fp_f[0]},
                "window": "frames 201..300 (the map at full size); bytes from the last frame's counts"},
        }
        m.close()

    def field_diff(a, b):
        """FP16 against FP32 fields on their common voxels.  The two runs track independently, so
        their poses differ slightly and a voxel at the band edge can take one more or one fewer ray
        in one of them; such voxels set the maximum, the percentiles show the bulk (the FP16 payload
        against the FP64 oracle at identical poses is bounded in the GPU tests)."""
        key = lambda m: ((m[:, 0].astype(np.int64) + (1 << 20)) << 42) | ((m[:, 1].astype(np.int64) + (1 << 20)) << 21) \
            | (m[:, 2].astype(np.int64) + (1 << 20))  # noqa: E731
        _, ia, ib = np.intersect1d(key(a["m"]), key(b["m"]), assume_unique=True, return_indices=True)
        gh = lambda g: g / np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-30)  # noqa: E731
        dpsi = np.abs(a["psi"][ia].astype(np.float64) - b["psi"][ib])
        dg = np.abs(gh(a["g"][ia].astype(np.float64)) - gh(b["g"][ib].astype(np.float64))).max(axis=1)
        pct = lambda x: {p: float(np.percentile(x, q)) for p, q in (("p50", 50), ("p99", 99), ("p999", 99.9))}  # noqa: E731
        return {"common_voxels": len(ia), "only_fp32": len(a) - len(ia), "only_fp16": len(b) - len(ib),
                "max_dpsi": float(dpsi.max()), "mean_dpsi": float(dpsi.mean()), "dpsi": pct(dpsi),
                "max_dghat": float(dg.max()), "mean_dghat": float(dg.mean()), "dghat": pct(dg)}

    # untimed: the FP16 payload fused at the FP32 run's own poses, so that both maps take the same
    # decisions and differ only by the payload's precision
    same = {}
    m = G.Map(G.make_config(FP16_VOXEL, hash_slots=FP16_SLOTS, fp16=True, max_touched_blocks=FP16_SLOTS // 2), stream)
    track_fp32[0] = torch.from_numpy(np.ascontiguousarray(seq.poses[0])).to(dev)
    for f in range(FP16_FRAMES + 1):
        m.integrate(depths[f], K, track_fp32[f])
        if f in FP16_CHECKS:
            same[f] = field_diff(fields["fp32"][f], m.extract())
    m.close()
    checks = {}
    for c in FP16_CHECKS:
        checks[str(c)] = {"pose_diff_fp16_vs_fp32": float(np.abs(poses_at["fp16"][c] - poses_at["fp32"][c]).max()),
                          "fields_fp16_vs_fp32": field_diff(fields["fp32"][c], fields["fp16"][c]),
                          "fields_fp16_vs_fp32_same_poses": same[c]}
    return {
        "workload": f"hashed room at 4 mm voxels (T = 2 cm), 640x480, {FP16_FRAMES} frames at 0.5 cm/frame, "
                    f"{GN_ITERS} GN steps + fusion per frame, every frame timed, L2 flushed before each",
        "fp32": out["fp32"], "fp16": out["fp16"], "checkpoints": checks,
        "speedup_fp16_vs_fp32": out["fp32"]["ms_per_frame"] / out["fp16"]["ms_per_frame"],
    }


TRI_WARMUP = 3
TRI_STEPS = 12


def trilinear_form(G, torch, dev, stream, seq):
    """The paper's comparison (Sec. 6): the same SLAM loop (10 GN steps + fusion per frame) with the
    one-lookup Taylor tracker and with the 8-lookup trilinear direct SDF tracker (Eqs. dir_dist,
    dir_grad), same frames, same timing rules."""
    K = G.intrinsics(seq.cam)
    H, W = seq.cam.height, seq.cam.width
    depths = torch.from_numpy(seq.depths).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    out = {}
    for name, tracker in (("taylor", G.GSDF_TRACKER_TAYLOR), ("trilinear", G.GSDF_TRACKER_TRILINEAR)):
        m = G.Map(G.make_config(VOXEL, hash_slots=HASH_SLOTS, tracker=tracker), stream)
        pose = torch.from_numpy(np.ascontiguousarray(seq.poses[0])).to(dev)
        dbuf = torch.empty((H, W), dtype=torch.float32, device=dev)
        dbuf.copy_(depths[0])
        m.integrate(dbuf, K, pose)
        stats = m.new_track_stats(GN_ITERS)
        ev, nv = [], []
        for f in range(1, 1 + TRI_WARMUP + TRI_STEPS):
            timed = f > TRI_WARMUP
            if timed:
                flush.fill_(f & 0xFF)
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record(stream)
            dbuf.copy_(depths[f], non_blocking=True)
            m.track(dbuf, K, pose, GN_ITERS, stats)
            if timed:
                e[1].record(stream)
            m.integrate(dbuf, K, pose)
            if timed:
                e[2].record(stream)
                ev.append(e)
                nv.append(G.track_stats_from_bytes(stats[GN_ITERS - 1].cpu().numpy()).n_valid)
        torch.cuda.synchronize(dev)
        T = pose.cpu().numpy()
        gt = seq.poses[TRI_WARMUP + TRI_STEPS]
        out[name] = {
            "track_us_per_step": 1e3 * float(np.mean([e[0].elapsed_time(e[1]) for e in ev])) / GN_ITERS,
            "ms_per_frame": float(np.mean([e[0].elapsed_time(e[2]) for e in ev])),
            "pixels_used_per_step": float(np.mean(nv)),
            "pose_error_m": float(np.linalg.norm(T[:3, 3] - gt[:3, 3])),
        }
        m.close()
    return {
        "workload": f"hashed room, 640x480, 1 cm voxels, frames 1..{TRI_WARMUP + TRI_STEPS}, {GN_ITERS} GN steps "
                    f"+ fusion per frame, {TRI_WARMUP} warm-up frames, {TRI_STEPS} timed, L2 flushed before each",
        "taylor": out["taylor"], "trilinear": out["trilinear"],
        "tracking_speedup_taylor_vs_trilinear": out["trilinear"]["track_us_per_step"] / out["taylor"]["track_us_per_step"],
        "paper_context": "30-40 ms vs 100-120 ms per frame for pose estimation on a CPU (Sec. 6): about 3x",
    }


POINTS_FRAMES = 30
POINTS_REPS = 5


def points_form(G, torch, dev, stream, seq):
    """Surface extraction (Sec. 4.3) from the room fused over 30 frames at their true poses:
    gsdf_extract_voxels for comparison, gsdf_extract_points at level 0 and with 2x2x2 upsampling,
    and the marching-cubes mesh (gsdf_extract_mesh).  Each is a synchronous API call that ends with the host copy; wall-clock median of
    five calls after one warm-up call."""
    K = G.intrinsics(seq.cam)
    m = G.Map(G.make_config(VOXEL, hash_slots=HASH_SLOTS), stream)
    for f in range(POINTS_FRAMES):
        m.integrate(torch.from_numpy(seq.depths[f]).to(dev), K, torch.from_numpy(np.ascontiguousarray(seq.poses[f])).to(dev))
    m.sync()
    n_vox = len(m.extract())
    out = {"workload": f"hashed room, 1 cm voxels, fused from frames 0..{POINTS_FRAMES - 1} at their true poses; "
                       f"wall-clock median of {POINTS_REPS} synchronous calls (device work and host copy)",
           "voxels": n_vox}

    def timed(fn):
        fn()
        ts = []
        for _ in range(POINTS_REPS):
            t0 = time.perf_counter()
            r = fn()
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts)), r

    t_vox, _ = timed(lambda: m.extract())
    out["extract_voxels_ms"] = 1e3 * t_vox
    for level in (0, 1):
        cap = n_vox * (8 if level else 1)
        t, pts = timed(lambda: m.extract_points(level, cap))
        out[f"level{level}"] = {"points": int(len(pts)), "ms": 1e3 * t, "points_per_s": len(pts) / t,
                                "voxels_scanned_per_s": n_vox / t}
    t, tri = timed(lambda: m.extract_mesh(4 * n_vox))
    out["mesh"] = {"triangles": int(len(tri)), "ms": 1e3 * t, "triangles_per_s": len(tri) / t,
                   "cubes_scanned_per_s": n_vox / t}
    m.close()
    return out


ADJ_KEYFRAMES = 10
ADJ_STRIDE = 10
ADJ_WARMUP = 3
ADJ_STEPS = 20
ADJ_LAMBDA = 0.5
# algorithmic bytes per adjoint evaluation: per voxel m (12), psi (4), g (12), rho (12) and its
# visibility word (4) read, dE/dpsi, dE/dg, dE/drho (4 + 12 + 12) written; per keyframe pixel its
# depth (4) and its RGB texel (16, each texel counted once)
ADJ_B_PER_VOXEL = 12 + 4 + 12 + 12 + 4 + 4 + 12 + 12
ADJ_B_PER_PX = 4 + 16


BA_ITERS = 10
BA_LAMBDA = 100.0  # sigma_I^2 / sigma_d^2: colour noise ~0.01, depth noise ~1 mm


def ba_form(G, torch, dev, stream, ks):
    """Photometric bundle adjustment (Sec. 4.2, decoupled per-keyframe energies of Eq. rgb_cost_pose,
    plus lambda times the geometric term): the room fused from 10 RGB-D keyframes at their true
    poses; keyframes 1..9 perturbed by 0.3 deg / 3 mm; 10 pose-only iterations of
    gsdf_energy_ba_step, each timed with CUDA events, L2 flushed before each."""
    K = G.intrinsics(ks.cam)
    m = G.Map(G.make_config(ks.voxel_size, hash_slots=HASH_SLOTS), stream)
    P_true = torch.from_numpy(np.stack(ks.poses)).to(dev)
    depths = torch.from_numpy(ks.depths).to(dev)
    for i in range(len(ks.poses)):
        m.integrate(depths[i], K, P_true[i])
    vox = m.extract()
    m.close()
    n = len(vox)
    mm = torch.from_numpy(np.ascontiguousarray(vox["m"]).astype(np.int32)).to(dev)
    psi = torch.from_numpy(np.ascontiguousarray(vox["psi"]).astype(np.float32)).to(dev)
    g = torch.from_numpy(np.ascontiguousarray(vox["g"]).astype(np.float32)).to(dev)
    rng = np.random.default_rng(SEED)
    from paper_2111_13652_gb300 import inputs as I

    poses = [ks.poses[0]] + [I.perturb_pose(T, rng, 0.3, 0.003) for T in ks.poses[1:]]
    P = torch.from_numpy(np.stack(poses)).to(dev)
    en = G.Energy(mm, ks.voxel_size, K, torch.from_numpy(ks.rgbs).to(dev), depths, stream)
    nu = en.visibility(psi, g, P)
    rho = torch.empty((n, 3), dtype=torch.float32, device=dev)
    F = len(ks.poses)
    stats = torch.zeros((BA_ITERS, F, G.TRACK_STATS_BYTES), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ev = []
    for it in range(BA_ITERS):
        flush.fill_(it & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        en.ba_step(psi, g, rho, P, nu, BA_LAMBDA, 1e-4, G.GSDF_BA_POSES, stats[it])
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize(dev)
    t = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    st = stats.cpu().numpy()
    energy = [sum(G.track_stats_from_bytes(st[it, i]).energy for i in range(F)) for it in range(BA_ITERS)]
    Pf = P.cpu().numpy()
    err0 = [float(np.linalg.norm(poses[i][:3, 3] - ks.poses[i][:3, 3])) for i in range(1, F)]
    err1 = [float(np.linalg.norm(Pf[i][:3, 3] - ks.poses[i][:3, 3])) for i in range(1, F)]
    en.close()
    return {
        "workload": f"{F} RGB-D keyframes {ks.cam.width}x{ks.cam.height} of the room, voxels fused on the GPU at "
                    f"{ks.voxel_size * 100:.0f} cm at the true poses; keyframes 1..{F - 1} perturbed by 0.3 deg / 3 mm; "
                    f"{BA_ITERS} pose-only iterations, lambda = {BA_LAMBDA}, damping 1e-4, L2 flushed before each",
        "voxels": n, "ms_per_iteration": t, "ms_per_iteration_and_pose": t / F,
        "energy_first_last": [energy[0], energy[-1]],
        "mean_position_error_m_before_after": [float(np.mean(err0)), float(np.mean(err1))],
        "paper_context": "20-30 ms per iteration and pose on a single-threaded CPU (Sec. 6)",
    }


def adjoint_form(G, torch, dev, stream, ks, hbm_peak):
    """The differentiable form: E = photometric + lambda geometric over the voxels of the room fused
    from 10 RGB-D keyframes (640x480, 1 cm), and its full gradient (psi, g, rho, 10 poses) through
    gsdf_energy_eval; also the same through the torch.autograd.Function (forward + backward)."""
    K = G.intrinsics(ks.cam)
    m = G.Map(G.make_config(ks.voxel_size, hash_slots=HASH_SLOTS), stream)
    P = torch.from_numpy(np.stack(ks.poses)).to(dev)
    depths = torch.from_numpy(ks.depths).to(dev)
    for i in range(len(ks.poses)):
        m.integrate(depths[i], K, P[i])
    vox = m.extract()
    m.close()
    n = len(vox)
    mm = torch.from_numpy(np.ascontiguousarray(vox["m"]).astype(np.int32)).to(dev)
    psi = torch.from_numpy(np.ascontiguousarray(vox["psi"]).astype(np.float32)).to(dev)
    g = torch.from_numpy(np.ascontiguousarray(vox["g"]).astype(np.float32)).to(dev)
    rho = torch.from_numpy(np.random.default_rng(SEED).uniform(0.2, 0.9, (n, 3)).astype(np.float32)).to(dev)
    en = G.Energy(mm, ks.voxel_size, K, torch.from_numpy(ks.rgbs).to(dev), depths, stream)
    nu = en.visibility(psi, g, P)
    pairs = int(np.unpackbits(nu.cpu().numpy().view(np.uint8)).sum())
    # preallocated outputs; one evaluation = one C-ABI call
    E = torch.empty(3, dtype=torch.float64, device=dev)
    dpsi = torch.empty(n, dtype=torch.float32, device=dev)
    dg = torch.empty((n, 3), dtype=torch.float32, device=dev)
    drho = torch.empty((n, 3), dtype=torch.float32, device=dev)
    dT = torch.empty((len(ks.poses), 4, 4), dtype=torch.float64, device=dev)
    dxi = torch.empty((len(ks.poses), 6), dtype=torch.float64, device=dev)
    G.gsdf_energy_set_stream(en.e, stream.cuda_stream)

    def call(grad):
        if grad:
            st = G.gsdf_energy_eval(en.e, psi.data_ptr(), g.data_ptr(), rho.data_ptr(), P.data_ptr(), nu.data_ptr(),
                                    ADJ_LAMBDA, 0, E.data_ptr(), dpsi.data_ptr(), dg.data_ptr(), drho.data_ptr(),
                                    dT.data_ptr(), dxi.data_ptr())
        else:
            st = G.gsdf_energy_eval(en.e, psi.data_ptr(), g.data_ptr(), rho.data_ptr(), P.data_ptr(), nu.data_ptr(),
                                    ADJ_LAMBDA, 0, E.data_ptr())
        if st != 0:
            raise RuntimeError(G.gsdf_status_string(st))

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        ts = []
        for k in range(ADJ_WARMUP + ADJ_STEPS):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            if k >= ADJ_WARMUP:
                ts.append((e0, e1))
        torch.cuda.synchronize(dev)
        return 1e-3 * float(np.mean([a.elapsed_time(b) for a, b in ts]))

    t_vis = timed(lambda: en.visibility(psi, g, P))
    t_energy = timed(lambda: call(False))
    t_grad = timed(lambda: call(True))
    ps, gs, rs, Ps = (x.clone().requires_grad_(True) for x in (psi, g, rho, P))

    def autograd_step():
        for x in (ps, gs, rs, Ps):
            x.grad = None
        G.voxel_energy(ps, gs, rs, Ps, en, nu, ADJ_LAMBDA).backward()

    t_auto = timed(autograd_step)
    E_val = E.cpu().numpy()
    npx = len(ks.poses) * ks.cam.width * ks.cam.height
    bytes_eval = ADJ_B_PER_VOXEL * n + ADJ_B_PER_PX * npx
    en.close()
    return {
        "workload": f"{len(ks.poses)} RGB-D keyframes {ks.cam.width}x{ks.cam.height} of the room (every "
                    f"{ADJ_STRIDE}th frame), voxels fused on the GPU at {ks.voxel_size * 100:.0f} cm, random colours "
                    f"U[0.2, 0.9], lambda = {ADJ_LAMBDA}; {ADJ_WARMUP} warm-up and {ADJ_STEPS} timed evaluations, "
                    f"L2 flushed between them",
        "voxels": n, "visible_pairs": pairs, "keyframe_pixels": npx,
        "visibility_ms": 1e3 * t_vis,
        "energy_only_ms": 1e3 * t_energy,
        "energy_and_gradient_ms": 1e3 * t_grad,
        "autograd_forward_backward_ms": 1e3 * t_auto,
        "gradient_evaluations_per_s": 1.0 / t_grad,
        "algorithmic_bytes_per_evaluation": bytes_eval,
        "hbm_frac_energy_and_gradient": bytes_eval / t_grad / 1e9 / hbm_peak,
        "E": E_val.tolist(),
        "paper_context": "photometric BA 20-30 ms per iteration and pose on a CPU (Sec. 6); here all "
                         f"{len(ks.poses)} poses and every voxel in one evaluation",
    }


def profile_case(case):
    """Small standalone runs of single kernels' workloads, for ncu captures (not benchmark lines):
    batchN / batchN_fp16: the first N scenes of the batch workload (rooms FP16 with _fp16), frame 0
    fused at its true pose, autotuned (not with a _fixed suffix: the default tile choice, so that a
    capture does not depend on timings taken under the profiler), then 4 frames of gsdf_batch_frame
    (10 GN steps + fusion);
    fp16_4mm: the 4 mm room fused with the FP16 payload at its true poses, 9 frames.  Prints the
    event-timed milliseconds per call."""
    import torch

    from paper_2111_13652_gb300 import gsdf as G
    from paper_2111_13652_gb300 import inputs as I

    procs = max(1, min(16, os.cpu_count() or 1))
    if case.startswith("batch"):
        fixed = case.endswith("_fixed")
        fp16 = "_fp16" in case
        n = int(case[len("batch"):].split("_")[0])
        frames = 4
        scenes = I.batch_scenes(n, frames + 1, processes=procs)
        G.load_library()
        dev = torch.device("cuda")
        maps = []
        for sc in scenes:
            if sc.dense_dims is not None:
                cfg = G.make_config(sc.voxel_size, dense_dims=sc.dense_dims, dense_origin=sc.dense_origin,
                                    damping=sc.damping)
            else:
                cfg = G.make_config(sc.voxel_size, hash_slots=sc.hash_slots, damping=sc.damping, fp16=fp16,
                                    max_touched_blocks=sc.hash_slots // 2)
            maps.append(G.Map(cfg))
        depths = [torch.from_numpy(sc.depths).to(dev) for sc in scenes]
        poses = [torch.from_numpy(np.ascontiguousarray(sc.poses[0])).to(dev) for sc in scenes]
        b = G.Batch(maps)
        b.set_frames([d[0] for d in depths], [G.intrinsics(sc.cam) for sc in scenes], poses)
        b.set_depth_stride([sc.cam.width * sc.cam.height for sc in scenes])
        b.frame(0)
        if not fixed:
            b.autotune()
        calls = [lambda: b.frame(GN_ITERS)] * frames
    elif case == "fp16_4mm":
        frames = 9
        seq = I.room_sequence(seed=SEED, n_frames=frames, voxel_size=FP16_VOXEL, frames_per_segment=75,
                              processes=procs)
        G.load_library()
        dev = torch.device("cuda")
        m = G.Map(G.make_config(FP16_VOXEL, hash_slots=FP16_SLOTS, fp16=True, max_touched_blocks=FP16_SLOTS // 2))
        K = G.intrinsics(seq.cam)
        depths = torch.from_numpy(seq.depths).to(dev)
        poses = torch.from_numpy(np.stack(seq.poses)).to(dev)
        calls = [(lambda f=f: m.integrate(depths[f], K, poses[f])) for f in range(frames)]
    else:
        raise SystemExit(f"unknown profile case {case}")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ts = []
    for k, call in enumerate(calls):
        flush.fill_(k & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        ts.append((e0, e1))
    torch.cuda.synchronize()
    print(case, "ms per call:", " ".join(f"{a.elapsed_time(c):.3f}" for a, c in ts), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=95)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="gsdf", choices=["gsdf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch-form", action="store_true")
    ap.add_argument("--no-fp16-form", action="store_true")
    ap.add_argument("--no-adjoint-form", action="store_true")
    ap.add_argument("--no-points-form", action="store_true")
    ap.add_argument("--no-trilinear-form", action="store_true")
    ap.add_argument("--no-ba-form", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    help="run one small standalone case for an ncu capture instead of the benchmark "
                         "(batchN, batchN_fp16, fp16_4mm)")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
