"""Benchmark of the fused Harris chain on synthetic high-speed video (1000 x 800 x 600 u8).

One step = the whole hot path over the 1000-frame volume, inputs already resident in
HBM: the 8-stage chain in the partition the traffic-model planner picks (full fusion),
then per frame the 256 strongest corners and one Lucas-Kanade step against the previous
frame. The volume
(480 MB of frames + 480 MB of mask) is larger than L2, so no flush is needed between
steps. Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the deliberately slow reference) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1509_04394_gb300 import shard  # noqa: E402
from synth import video as sv  # noqa: E402

METRIC = "fused-chain Mpixel/s & HBM roofline fraction vs unfused, 800×600×1000 u8"
UNIT = "Mpixel/s"
E2E_CHUNK = 50  # frames per chunk of the pipelined host-to-host call
GATE_CYCLES = 100_000_000  # SM clock cycles of the blocking kernel ahead of a timed region
SPEC = sv.HSDV_800x600x1000
WORKLOAD = "Harris 8-stage chain, 1000 frames x 800 rows x 600 cols u8, 64 blobs + 32 patches, seed 3"
# Algorithmic FP32 operations per output pixel of the chain, from the stage definitions
# (an FMA counts once): the basis of the ALU roofline of the fused kernel.
OPS_BY_STAGE = {"S1 convert": 1, "S2 Gaussian-H (2 adds, 2 FMAs)": 4, "S3 Gaussian-V": 4,
                "S4 Sobel (Dx 1, Sx 2, Ix 2, Iy 1)": 6, "S5 products": 3, "S6 box 5x5 (3 x (4 + 4) adds)": 24,
                "S7 Harris (det 2, trace 1, response 2)": 5, "S8 threshold + 3x3 max (2 + 2 max3, 2 compares)": 6}
OPS_PER_PX = sum(OPS_BY_STAGE.values())
TUNE_ROWS = [100, 160, 200, 267, 320, 400, 800]  # chunk heights the autotuner tries on the workload


def kernel_counters():
    """ncu counters of the step's dominant kernel (the fused chain with corner lists) from
    profiles/fused_chain_traffic.json, only while its source still hashes to the captured
    version (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "fused_chain_traffic.json")) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for f in ("paper_1509_04394_gb300/csrc/kf_chain.cuh", "paper_1509_04394_gb300/csrc/kf_params.h",
                  "paper_1509_04394_gb300/csrc/kf_groups_a1.cu"):
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        return rec if rec.get("source_sha256") == h.hexdigest() else None
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling (every 200 ms) of one GPU while the benchmark runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id, self.rows, self.proc = gpu_id, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()
        # nvidia-smi's start-up (driver library initialisation) took over a second on some
        # hosts, and the first timed leg after it came out 20-30 ms longer in total while
        # its kernels kept their times: wait for the first sample before going on
        t_end = time.time() + 10.0
        while not self.rows and self.proc.poll() is None and time.time() < t_end:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            time.sleep(0.5)  # its shutdown too, before the next timed leg

    def summary(self, t0: float, t1: float) -> dict:
        rows = [r for (ts, r) in self.rows if t0 <= ts <= t1 and len(r) >= 9]
        if not rows:
            rows = [r for (_, r) in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][2]),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ ranks
def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time (every rank processes its own frame range)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(pixels_per_rank: int, world: int, ms: float) -> float:
    """Whole-job Mpixel/s: the pixels of all ranks over the slowest rank's time."""
    return world * pixels_per_rank / (ms / 1000) / 1e6


# ------------------------------------------------------------------ workload
def make_video(rank: int = 0, world: int = 1, T: int | None = None):
    """Rank `rank`'s frames of one video of world x T frames (T defaults to the workload's
    1000): the T frames it owns and, before them, the one frame that the tracking of its
    first owned frame reads (none for rank 0). Returns (frames [n, H, P], P, owned)."""
    P = sv.pitch_for(SPEC.W)
    T = T or SPEC.T
    s0, t0, t1 = shard.span(world * T, world, rank)
    frames, _ = sv.generate(SPEC, pitch=P, frames=range(s0, t1))
    return frames, P, t1 - t0


def run_profile(args):
    """Small case for profiler captures: `--profile T` runs only the planned fused chain on
    the first T frames (warm-up launches, then `--steps` launches), nothing else."""
    import torch
    from paper_1509_04394_gb300 import build as kbuild
    from paper_1509_04394_gb300 import kfuse as K
    kbuild.build()
    frames_h, P, _ = make_video(0, 1, args.profile)
    T, H, W = frames_h.shape[0], SPEC.H, SPEC.W
    dev = torch.device("cuda:0")
    frames = torch.from_numpy(frames_h).to(dev)
    mask = torch.zeros_like(frames)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    ctx = K.Context(0, precision=K.KF_PREC_F16 if args.f16 else K.KF_PREC_F32)
    if args.rows > 0:
        K.kf_set_chunk_rows(ctx.h, args.rows)
    cuts = args.cuts if args.cuts >= 0 else K.kf_plan(ctx.h, W, H, T)[0]
    if args.track:  # the whole hot path: fused chain with corner lists, selection, LK
        KP = 256
        n_pts = torch.zeros(T, dtype=torch.int32, device=dev)
        idx = torch.zeros((T, KP), dtype=torch.int32, device=dev)
        uu, vv = torch.zeros((T, KP), device=dev), torch.zeros((T, KP), device=dev)
        st = torch.zeros((T, KP), dtype=torch.int32, device=dev)
        ws = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, H, T), dtype=torch.uint8, device=dev)
        for _ in range(args.warmup + args.steps):
            K.kf_track(ctx.h, frames, W, mask, counts, KP, n_pts, idx, uu, vv, st, ws)
    else:
        ws_b = K.kf_workspace_bytes(ctx.h, cuts, W, H, T)
        ws = torch.empty(ws_b, dtype=torch.uint8, device=dev) if ws_b else None
        for _ in range(args.warmup + args.steps):
            K.kf_run(ctx.h, cuts, frames, W, mask, counts, ws)
    torch.cuda.synchronize()
    print(json.dumps({"profile_frames": T, "cuts": cuts, "counts_sum": int(counts.sum())}))


def cpu_oracle_rate(frames: np.ndarray, W: int, budget_s: float = 12.0) -> dict:
    """The FP64 oracle as it stands, on the whole hot path (chain + corner selection +
    LK per frame pair), OpenMP over frame pairs on all host cores, on a bounded prefix of
    the volume sized to about `budget_s` seconds."""
    from oracle import chain as oc
    T, H, P = frames.shape
    t0 = time.perf_counter()
    oc.track_volume(frames[:5], W=W)
    probe = time.perf_counter() - t0
    n = int(max(5, min(T, 1 + budget_s / max(probe / 4, 1e-6))))
    t0 = time.perf_counter()
    _, _, _, _, _, used = oc.track_volume(frames[:n], W=W)
    dt = time.perf_counter() - t0
    return {"value": (n - 1) * H * W / dt / 1e6, "unit": UNIT, "cores": int(used), "kind": "oracle",
            "sample": f"frame pairs of the first {n} of {T} frames ({(n - 1) * H * W / 1e6:.1f} Mpixel), "
                      f"FP64 chain + tracking, {dt:.1f} s"}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    frames, P, _ = make_video()
    from oracle import chain as oc
    T, H, W = SPEC.T, SPEC.H, SPEC.W
    per_step = 25  # frames of the workload per timed step (24 tracked frame pairs)
    for i in range(args.warmup):
        oc.track_volume(frames[(i * per_step) % T:(i * per_step) % T + per_step], W=W)
    times, used = [], 1
    for i in range(args.steps):
        s = (i * per_step) % (T - per_step)
        t0 = time.perf_counter()
        _, _, _, _, _, used = oc.track_volume(frames[s:s + per_step], W=W)
        times.append(time.perf_counter() - t0)
    ms = 1000 * sum(times) / len(times)
    value = (per_step - 1) * H * W / (ms / 1000) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_per_step": f"{per_step} frames ({per_step - 1} tracked pairs)",
                       "impl": "FP64 CPU oracle: chain + corner selection + LK"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(used), "kind": "oracle",
                             "sample": f"{per_step} frames per step of the 1000-frame volume"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist
    from paper_1509_04394_gb300 import build as kbuild
    from paper_1509_04394_gb300 import kfuse as K

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0:
        kbuild.build()
    if world > 1:
        dist.barrier()

    frames_h, P, owned = make_video(rank, world)  # this rank's frame range of one video
    T, H, W = frames_h.shape[0], SPEC.H, SPEC.W
    KP = 256  # tracked points per frame
    frames_pin = torch.from_numpy(frames_h).pin_memory()
    frames = frames_pin.to(dev)
    mask = torch.zeros_like(frames)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    n_pts = torch.zeros(T, dtype=torch.int32, device=dev)
    idx = torch.zeros((T, KP), dtype=torch.int32, device=dev)
    uu = torch.zeros((T, KP), dtype=torch.float32, device=dev)
    vv = torch.zeros((T, KP), dtype=torch.float32, device=dev)
    st = torch.zeros((T, KP), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    ctx = K.Context(local_rank)
    cuts, _ = K.kf_plan(ctx.h, W, H, T)  # traffic-model plan: full fusion
    n_groups = bin(cuts).count("1") + 1
    ws_track = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, H, T), dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(fn, k, w, between=None, gate=True):
        for _ in range(w):
            fn()
        barrier()
        if between:
            between()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if gate:
            # a blocking kernel (a device sleep of about 50 ms) ahead of the first event: the
            # K steps' launches queue up behind it, so a stall of the host while it enqueues
            # them (a shared host's other work) cannot leave the GPU idle inside the timed
            # region. The end-to-end leg runs ungated: host-side work is part of what it times.
            torch.cuda._sleep(GATE_CYCLES)
        ev0.record(stream)
        for _ in range(k):
            fn()
        ev1.record(stream)
        barrier()
        return max_over_ranks(ev0.elapsed_time(ev1) / k, world, dev)

    def step():  # the whole hot path: fused chain, corner selection, LK tracking
        K.kf_track(ctx.h, frames, W, mask, counts, KP, n_pts, idx, uu, vv, st, ws_track, stream)

    # the dominant kernel alone: the fused chain as the planner partitions it, on a
    # context of its own at the height kf_tune_chunk_rows finds for it
    cctx = K.Context(local_rank)

    def chain():
        K.kf_run(cctx.h, cuts, frames, W, mask, counts, None, stream)

    # the executor's tile height for this workload from its autotuner (CUDA-event timing of
    # the fused chain inside the library, on a context of its own), applied to the step
    # (--rows fixes it instead: profiler runs, whose serialised launches would mislead it).
    # The autotuner times the step itself (kf_tune_track_rows): the chain's launch with
    # corner lists takes its jobs by SM kind, and its best height is not the plain chain's
    if args.rows > 0:
        best_rows, best_ms, rows_from = args.rows, None, "fixed (--rows)"
        K.kf_set_chunk_rows(cctx.h, args.rows)
        chain_rows = args.rows
    else:
        chain_rows, _ = K.kf_tune_chunk_rows(cctx.h, frames, W, torch.zeros_like(frames), torch.zeros_like(counts),
                                             TUNE_ROWS, reps=3, stream=stream)
        best_rows, best_ms = K.kf_tune_track_rows(ctx.h, frames, W, mask, counts, KP, n_pts, idx, uu, vv, st,
                                                  ws_track, TUNE_ROWS, reps=3, stream=stream)
        rows_from = "autotuner (kf_tune_track_rows, on the step)"
    K.kf_set_chunk_rows(ctx.h, best_rows)

    # clocks: sample across a ~1.5 s soak and the timed region
    try:
        gid = str(torch.cuda.get_device_properties(dev).uuid)
        gid = gid if gid.startswith("GPU-") else "GPU-" + gid
    except Exception:
        gid = str(local_rank)
    clk = ClockSampler(gid)
    clk.start()
    t_soak = time.time()
    while time.time() - t_soak < 1.5:
        step()
        torch.cuda.synchronize(dev)
    # the step, with each of its kernels bracketed by CUDA events on the launching stream
    K.kf_set_kernel_timing(ctx.h, True)
    ms = timed(step, args.steps, args.warmup, between=lambda: K.kf_kernel_times(ctx.h))
    kt = K.kf_kernel_times(ctx.h)
    K.kf_set_kernel_timing(ctx.h, False)
    mask_step, counts_step = mask.clone(), counts.clone()  # what the timed step wrote
    ms_chain = timed(chain, args.steps, args.warmup)
    chain_same = bool(torch.equal(mask, mask_step) and torch.equal(counts, counts_step))
    # the clocks cover the soak and the timed step and chain; the sampler (an nvidia-smi
    # process polling the driver) is stopped before the end-to-end leg, whose host-side
    # copies and launches it would perturb
    t_b = time.time()
    clk.stop()
    # end to end through the public call: pinned host frames in; mask, counts and tracks
    # out. kf_track_host runs the step in chunks of E2E_CHUNK frames with the copy in of
    # one chunk, the hot path of the previous ones and the copy out of earlier ones on
    # separate streams. The headline delivers the mask bit-packed (packed on the device,
    # 8 pixels a byte, and copied out); the byte-mask form is reported beside it.
    S = ((W * H + 7) // 8 + 15) // 16 * 16
    host = dict(frames=frames_pin, mask=torch.empty((T, S), dtype=torch.uint8).pin_memory(),
                counts=torch.empty_like(counts, device="cpu").pin_memory(),
                n_points=torch.empty_like(n_pts, device="cpu").pin_memory(),
                idx=torch.empty_like(idx, device="cpu").pin_memory(), u=torch.empty_like(uu, device="cpu").pin_memory(),
                v=torch.empty_like(vv, device="cpu").pin_memory(), status=torch.empty_like(st, device="cpu").pin_memory())
    host_b = dict(host, mask=torch.empty_like(frames_pin).pin_memory())
    devb = dict(frames=frames, mask=mask, counts=counts, n_points=n_pts, idx=idx, u=uu, v=vv, status=st)

    def e2e_step():
        K.kf_track_host(ctx.h, host, devb, W, KP, ws_track, chunk=E2E_CHUNK, stream=stream, mask_format=K.KF_MASK_BITS)

    def e2e_bytes_step():
        K.kf_track_host(ctx.h, host_b, devb, W, KP, ws_track, chunk=E2E_CHUNK, stream=stream,
                        mask_format=K.KF_MASK_BYTES)
    # the tile height of the call's chunk launches: the step's, 160 or 200 rows, whichever
    # the call itself measures fastest (a chunk launch is about one wave long, not fifteen);
    # each candidate timed in two interleaved rounds and kept at its faster one, so that one
    # round slowed by other work on the host's link does not decide
    e2e_rows = {}
    for _ in range(2):
        for r in sorted({best_rows, 160, 200}):
            K.kf_set_host_chunk_rows(ctx.h, r)
            ms = timed(e2e_step, 3, 1, gate=False)
            e2e_rows[r] = min(e2e_rows.get(r, ms), ms)
    host_rows = min(e2e_rows, key=e2e_rows.get)
    K.kf_set_host_chunk_rows(ctx.h, host_rows)
    ms_e2e = timed(e2e_step, max(3, args.steps // 2), 1, gate=False)
    m_bits = np.packbits(mask[:, :, :W].reshape(T, -1).cpu().numpy(), axis=1, bitorder="little")
    e2e_same = bool(np.array_equal(host["mask"].numpy()[:, :m_bits.shape[1]], m_bits)
                    and torch.equal(host["idx"], idx.cpu()) and torch.equal(host["u"], uu.cpu()))
    ms_e2e_b = timed(e2e_bytes_step, max(3, args.steps // 2), 1, gate=False)
    e2e_same_b = bool(torch.equal(host_b["mask"], mask.cpu()) and torch.equal(host_b["idx"], idx.cpu()))
    # the FP16-tile form: the same step and chain with the box's row-pair sums in FP16 on chip
    ctx16t = K.Context(local_rank, precision=K.KF_PREC_F16_TILES)
    K.kf_set_chunk_rows(ctx16t.h, best_rows)  # the FP32 step's height
    ctx16 = K.Context(local_rank, precision=K.KF_PREC_F16)
    mask16, counts16 = torch.zeros_like(frames), torch.zeros_like(counts)
    tr16 = (torch.zeros_like(n_pts), torch.zeros_like(idx), torch.zeros_like(uu), torch.zeros_like(vv), torch.zeros_like(st))
    ms_step16 = timed(lambda: K.kf_track(ctx16t.h, frames, W, mask16, counts16, KP, *tr16, ws_track, stream),
                      args.steps, args.warmup)
    mask16_diff = int((mask16 != mask_step).sum())
    ms_chain16 = timed(lambda: K.kf_run(ctx16t.h, 0, frames, W, mask16, counts16, None, stream), args.steps, args.warmup)
    clocks = clk.summary(t_soak, t_b)
    dev_err = K.kf_device_error(ctx.h)

    px = owned * H * W  # pixels this rank owns (the halo frame before them is not counted)
    value = job_rate(px, world, ms)
    hbm_peak, peak_kind = peaks()
    n_corners = int(counts.sum())
    # per-kernel device time inside the timed step (max over ranks)
    kernels = {}
    for name, (n, tot) in kt.items():
        if n:
            kernels[name] = {"launches": n, "ms_per_launch": max_over_ranks(tot / n, world, dev)}
    step_kernel_ms = sum(k["ms_per_launch"] * k["launches"] for k in kernels.values())
    for k in kernels.values():
        k["share"] = k["ms_per_launch"] * k["launches"] / step_kernel_ms
    dom = kernels["chain_corners"]["ms_per_launch"]
    # The dominant kernel is bound by arithmetic (its HBM traffic is ~2 B/px), so its
    # roofline is the FP32 lanes: algorithmic operations per output pixel from the stage
    # definitions (FMA = 1 op): S1 convert 1, S2/S3 Gaussian 4 + 4, S4 Sobel 6, S5
    # products 3, S6 separable 5x5 box 3 x 8, S7 Harris 5, S8 threshold + 3x3 max 6 = 53;
    # peak = the device's SMs x 128 FP32 lanes x the SM clock measured under load.
    sm_mhz = (clocks.get("sm_mhz") or 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    ops_per_px = OPS_PER_PX
    alu_peak = n_sm * 128 * sm_mhz * 1e6 / 1e9  # G lane-ops / s
    alu_ach = px * ops_per_px / (dom / 1000) / 1e9
    # HBM view: frames read once, mask written once, one 8-byte key per corner, the
    # per-frame corner and candidate counts
    alg_bytes = 2 * px + 8 * n_corners + 8 * T
    achieved = alg_bytes / (dom / 1000) / 1e9
    rec = kernel_counters() if T == 1000 else None
    # the counters taken at the step's tile height (each height has its own halo rows and
    # job count), if that height was captured
    rec = (dict(rec["by_rows"][str(best_rows)], kernel=rec["kernel"])
           if rec and str(best_rows) in rec.get("by_rows", {}) else None)
    traffic = rec["dram_bytes_per_launch_1000_frames"] if rec else None
    # issue view: executed warp instructions (ncu) over 152 SMs x 4 schedulers x clock
    issue_peak = n_sm * 4 * sm_mhz * 1e6 / 1e9  # G warp-instructions / s
    issue = None
    if rec:
        ach = rec["warp_instructions_per_launch_1000_frames"] / (dom / 1000) / 1e9
        issue = {"achieved": ach, "peak": issue_peak, "unit": "Gwarp-inst/s", "frac": ach / issue_peak,
                 "peak_kind": f"{n_sm} SMs x 4 schedulers x SM clock",
                 "instructions_per_launch": rec["warp_instructions_per_launch_1000_frames"], "kernel": rec["kernel"]}

    # batched form: the same workload as one video of a persistent-kernel batch (graph replay)
    bws = torch.empty(K.kf_batch_workspace_bytes(ctx.h, [frames], [W], KP), dtype=torch.uint8, device=dev)
    bmask = torch.zeros_like(frames)
    btr = (KP, torch.zeros_like(n_pts), torch.zeros_like(idx), torch.zeros_like(uu), torch.zeros_like(vv),
           torch.zeros_like(st))
    bcounts = torch.zeros_like(counts)
    batch = K.kf_batch_create(ctx.h, [frames], [W], [bmask], [bcounts], bws, [btr])
    ms_batch = timed(lambda: K.kf_batch_run(batch, stream), args.steps, args.warmup)
    batch_same = bool(torch.equal(bmask, mask) and torch.equal(bcounts, counts) and torch.equal(btr[1], n_pts))
    K.kf_batch_destroy(batch)
    del bws

    # unfused sequence (one kernel per stage, volume-wide maps through HBM)
    unf_cuts = (1 << 7) - 1
    ws = torch.empty(K.kf_workspace_bytes(ctx.h, unf_cuts, W, H, T), dtype=torch.uint8, device=dev)
    mask_u = torch.zeros_like(frames)
    counts_u = torch.zeros_like(counts)
    ms_unf = timed(lambda: K.kf_run(ctx.h, unf_cuts, frames, W, mask_u, counts_u, ws, stream), max(3, args.steps // 4), 1)
    same = bool(torch.equal(mask_u, mask) and torch.equal(counts_u, counts))
    unf_bytes = 98 * px  # FP32 maps: sum over stages of input + output bytes per pixel
    # 16-bit maps, unfused (half the intermediate bytes)
    ws16 = torch.empty(K.kf_workspace_bytes(ctx16.h, unf_cuts, W, H, T), dtype=torch.uint8, device=dev)
    ms_unf16 = timed(lambda: K.kf_run(ctx16.h, unf_cuts, frames, W, mask_u, counts_u, ws16, stream),
                     max(3, args.steps // 4), 1)
    del ws, ws16

    ms_e2e_end = timed(e2e_step, max(3, args.steps // 2), 1, gate=False)  # the same call once more, after every other form
    h2d = frames_pin.numel()
    d2h_tracks = sum(t.numel() * t.element_size() for k, t in host.items() if k not in ("frames", "mask"))
    d2h = T * ((W * H + 7) // 8) + d2h_tracks
    d2h_b = host_b["mask"].numel() + d2h_tracks
    tracked = int(n_pts.sum())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames": T, "rows": H, "cols": W, "step": "fused 8-stage chain + "
                   f"top-{KP} corner selection + LK tracking per frame pair", "partition_cuts": cuts,
                   "groups": n_groups, "chunk_rows": best_rows, "chunk_rows_from": rows_from, "cols_per_lane": 4,
                   "l2": "inputs larger than L2 (480 MB frames, 480 MB mask), no flush",
                   "host_gate": "device-timed legs queued behind a ~50 ms blocking kernel before the first event",
                   "parallelism": (f"frame shards x{world} of one {world * owned}-frame video, merged on the host"
                                   if world > 1 else "single GPU")},
        "frames_per_s": world * owned / (ms / 1000),
        "tracked_points_per_s": world * tracked / (ms / 1000),
        "chain_only": {"value": world * px / (ms_chain / 1000) / 1e6, "ms_per_step": ms_chain,
                       "kernel": "group_kernel<1,8> (full fusion, no corner lists), timed alone by kf_run",
                       "chunk_rows": chain_rows,
                       "identical_to_step": chain_same,
                       "hbm_frac": (2 * px + 4 * T) / (ms_chain / 1000) / 1e9 / hbm_peak},
        "roofline": {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "Gop/s",
                     "frac": alu_ach / alu_peak, "traffic": traffic,
                     "peak_kind": f"{n_sm} SMs (read from the device) x 128 FP32 lanes x median SM clock under load",
                     "sm_count": n_sm, "ops_per_px_by_stage": OPS_BY_STAGE,
                     "kernel": "group_kernel<1,8> with corner lists (the step's dominant kernel, timed inside the step)",
                     "ms_per_launch": dom, "ops_per_px": ops_per_px, "algorithmic_ops_per_launch": px * ops_per_px,
                     "algorithmic_bytes_per_launch": alg_bytes},
        "hbm_view": {"achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "peak_kind": peak_kind, "traffic": traffic},
        "issue_view": issue,
        "kernels_in_step": kernels,
        "fp16_form": {"value": world * px / (ms_step16 / 1000) / 1e6, "ms_per_step": ms_step16,
                      "chain_ms": ms_chain16, "step_speedup_over_fp32": ms / ms_step16,
                      "what": "KF_PREC_F16_TILES: the fused chain with the box's row-pair sums in FP16 on chip (FP32 "
                              "window sums), same step", "mask_pixels_differing_from_fp32": mask16_diff},
        "batched_form": {"value": world * px / (ms_batch / 1000) / 1e6, "ms_per_step": ms_batch,
                         "what": "the same step as one video of a persistent-kernel batch replayed from a CUDA graph",
                         "identical_results": batch_same},
        "autotuned_chunk_rows": {"best": best_rows, "step_ms": best_ms, "candidates": TUNE_ROWS},
        "unfused": {"value": world * px / (ms_unf / 1000) / 1e6, "ms_per_step": ms_unf, "kernels": 8,
                    "hbm_frac": unf_bytes / (ms_unf / 1000) / 1e9 / hbm_peak,
                    "bit_identical_to_fused": bool(same and chain_same),
                    "fused_chain_speedup": ms_unf / ms_chain},
        "unfused_f16": {"value": world * px / (ms_unf16 / 1000) / 1e6, "ms_per_step": ms_unf16,
                        "hbm_frac": 50 * px / (ms_unf16 / 1000) / 1e9 / hbm_peak},
        "e2e": {"value": world * px / (ms_e2e / 1000) / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": ms_e2e, "chunk_frames": E2E_CHUNK,
                "chunk_tile_rows": host_rows, "chunk_tile_rows_ms": {str(k): v for k, v in e2e_rows.items()},
                "call": "kf_track_host, KF_MASK_BITS (copy in, hot path on three streams, mask packed 8 px/byte "
                        "on the device, packed mask and tracks copied out)",
                "results_equal_device_step": e2e_same, "ms_per_step_repeated_at_end": ms_e2e_end},
        "e2e_byte_mask": {"value": world * px / (ms_e2e_b / 1000) / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                          "d2h_bytes_per_step": int(d2h_b), "ms_per_step": ms_e2e_b,
                          "call": "kf_track_host, KF_MASK_BYTES", "results_equal_device_step": e2e_same_b},
        "gpu_launches": sum(k["launches"] for k in kernels.values()),  # counted by the library's event pairs
        "device_error": dev_err,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(frames_h, W)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _ranks(x) -> np.ndarray:
    """Ranks 1..n of the values of x, ties given their average rank."""
    x = np.asarray(x, dtype=np.float64)
    order = np.argsort(x, kind="stable")
    r = np.empty(len(x), dtype=np.float64)
    r[order] = np.arange(1, len(x) + 1)
    for v in np.unique(x):
        sel = x == v
        if sel.sum() > 1:
            r[sel] = r[sel].mean()
    return r


def spearman(a, b) -> float:
    ra, rb = _ranks(a), _ranks(b)
    ra, rb = ra - ra.mean(), rb - rb.mean()
    return float((ra * rb).sum() / np.sqrt((ra * ra).sum() * (rb * rb).sum()))


def run_partitions(args):
    """Every contiguous partition of the 8-stage chain timed on 600 frames of 192 x 432
    (seed 2): the traffic model's choice (kf_plan) against the measured best, with the
    model's rank among the measured times, its regret and the rank correlation between
    predicted bytes and measured time (the check Sec. VI's model gets from Sec. VII-B's
    measured No / Two / Full Fusion). Each timed launch starts with L2 flushed."""
    import torch
    from paper_1509_04394_gb300 import build as kbuild
    from paper_1509_04394_gb300 import kfuse as K
    kbuild.build()
    spec = SPEC if args.partitions_full else sv.PARTITIONS_192x432x600
    T, H, W = spec.T, spec.H, spec.W
    P = sv.pitch_for(W)
    fr, _ = sv.generate(spec, pitch=P)
    dev = torch.device("cuda:0")
    frames = torch.from_numpy(fr).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = K.Context(0, precision=K.KF_PREC_F16 if args.f16 else K.KF_PREC_F32)
    parts = K.kf_enumerate(ctx.h)
    plan, plan_bytes = K.kf_plan(ctx.h, W, H, T)
    ws_b = max(K.kf_workspace_bytes(ctx.h, c, W, H, T) for c in parts)
    ws = torch.empty(max(ws_b, 256), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # twice the L2
    mask = torch.zeros_like(frames)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    K.kf_run(ctx.h, 0, frames, W, mask, counts, None, stream)
    ref_mask, ref_counts = mask.clone(), counts.clone()
    reps = max(args.steps, 5)
    rows = []
    for c in parts:
        for _ in range(args.warmup):
            K.kf_run(ctx.h, c, frames, W, mask, counts, ws, stream)
        times = []
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            K.kf_run(ctx.h, c, frames, W, mask, counts, ws, stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        same = bool(torch.equal(mask, ref_mask) and torch.equal(counts, ref_counts))
        rows.append({"cuts": c, "groups": bin(c).count("1") + 1, "ms": statistics.median(times),
                     "model_bytes": K.kf_partition_traffic(ctx.h, c, W, H, T), "identical": same})
    assert K.kf_device_error(ctx.h) == 0
    ms = np.array([r["ms"] for r in rows])
    mb = np.array([r["model_bytes"] for r in rows])
    order = np.argsort(ms)
    best = rows[int(order[0])]
    chosen = next(r for r in rows if r["cuts"] == plan)
    rank = 1 + int(np.sum(ms < chosen["ms"]))
    out = {"workload": f"Harris 8-stage chain, {T} frames x {H} rows x {W} cols u8, seed {spec.seed}, "
                       f"{'16-bit' if args.f16 else 'FP32'} maps",
           "partitions": len(rows), "reps_per_partition": reps, "l2": "flushed before every timed launch",
           "model_choice": {"cuts": plan, "ms": chosen["ms"], "model_bytes": plan_bytes, "measured_rank": rank},
           "measured_best": {"cuts": best["cuts"], "ms": best["ms"], "model_bytes": best["model_bytes"]},
           "regret": chosen["ms"] / best["ms"] - 1.0,
           "spearman_model_bytes_vs_ms": spearman(mb, ms),
           "all_identical_to_full_fusion": all(r["identical"] for r in rows),
           "unfused": next(r for r in rows if r["cuts"] == 127),
           "fastest_10": [rows[int(i)] for i in order[:10]],
           "slowest_3": [rows[int(i)] for i in order[-3:]]}
    if args.partitions_table:
        with open(args.partitions_table, "w") as fh:
            json.dump(rows, fh)
    print(json.dumps(out), flush=True)


BATCH48 = [(16, 192, 432, 600), (16, 480, 640, 300), (12, 800, 600, 1000), (4, 1080, 1920, 120)]  # count, H, W, T


PCHAIN_SIZES = [(256, 256), (512, 512), (1024, 1024)]  # H, W: the paper's resized clips (Sec. VII-A)
PCHAIN_PARTS = {"full_fusion": 0, "two_fusion": 0b0010, "no_fusion": 0b1111}


def pchain_video(dev, H, W, T, seed):
    """RGBA frames [T, H, W, 4] on the device: 64 generated frames, cycled."""
    import torch
    spec = sv.VideoSpec(T=T, H=H, W=W, seed=seed, n_blobs=max(8, H * W // 8000), n_patches=max(8, H * W // 12000))
    g, _ = sv.generate(spec, frames=range(min(T, 64)))
    src = torch.from_numpy(sv.rgba_of(g)).to(dev)
    f = torch.empty((T, H, W, 4), dtype=torch.uint8, device=dev)
    for t0 in range(0, T, src.shape[0]):
        m = min(src.shape[0], T - t0)
        f[t0:t0 + m] = src[:m]
    return f


def run_pchain(args):
    """The paper's own chain (Table II: RGBA to gray, IIR filter, Gaussian, gradient,
    threshold, then Kalman) at the paper's 256^2, 512^2 and 1024^2 x 1000 frames: "No
    Fusion" (five kernels), "Two Fusion" (K1 K2 | K3 K4 K5) and "Full Fusion", each timed
    with CUDA events (inputs larger than L2), with the traffic model's bytes and the HBM
    fraction they imply; K6 (Kalman over the 16 region tracks) timed alone."""
    import torch
    from paper_1509_04394_gb300 import build as kbuild
    from paper_1509_04394_gb300 import kfuse as K
    kbuild.build()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = K.Context(0, harris=False)
    hbm_peak, peak_kind = peaks()
    T = args.pc_frames
    sizes = PCHAIN_SIZES if not args.pc_size else [(args.pc_size, args.pc_size)]
    out = {"workload": f"paper chain K1..K5 + K6 on RGBA video, {T} frames per size (64 generated frames, cycled)",
           "peak_hbm_gbs": hbm_peak, "peak_kind": peak_kind, "sizes": []}
    for i, (H, W) in enumerate(sizes):
        fr = pchain_video(dev, H, W, T, 20 + i)
        mp = (W + 15) // 16 * 16
        mask = torch.zeros((T, H, mp), dtype=torch.uint8, device=dev)
        counts = torch.zeros(T, dtype=torch.int32, device=dev)
        regions = torch.zeros((T, 16, 3), dtype=torch.int32, device=dev)
        px = T * H * W
        row = {"H": H, "W": W, "T": T, "planned_cuts": K.kf_pc_plan(ctx.h, W, H, T)[0]}
        ref = None
        for name, cuts in PCHAIN_PARTS.items():
            ws = torch.empty(K.kf_pc_workspace_bytes(ctx.h, cuts, W, H, T), dtype=torch.uint8, device=dev)
            run = lambda: K.kf_pc_run(ctx.h, cuts, fr, W, mask, counts, regions, ws, stream)  # noqa: E731
            if args.pc_once:
                run()
                torch.cuda.synchronize()
                continue
            for _ in range(args.warmup):
                run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            model = K.kf_pc_traffic(ctx.h, cuts, W, H, T)
            res = (mask.clone(), counts.clone(), regions.clone())
            if ref is None:
                ref = res
            same = all(torch.equal(a, b) for a, b in zip(res, ref))
            row[name] = {"cuts": cuts, "ms": ms, "value": px / (ms / 1000) / 1e6, "unit": "Mpixel/s",
                         "model_bytes": model, "model_bytes_per_px": model / px,
                         "hbm_frac": model / (ms / 1000) / 1e9 / hbm_peak, "identical_to_full_fusion": same}
            del ws
        if not args.pc_once:
            states = torch.zeros((T, 16, 4), dtype=torch.float64, device=dev)
            status = torch.zeros((T, 16), dtype=torch.int32, device=dev)
            K.kf_pc_kalman(ctx.h, regions, states, status, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                K.kf_pc_kalman(ctx.h, regions, states, status, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            row["kalman_ms"] = e0.elapsed_time(e1) / args.steps
            row["full_vs_no_fusion"] = row["no_fusion"]["ms"] / row["full_fusion"]["ms"]
            row["two_vs_no_fusion"] = row["no_fusion"]["ms"] / row["two_fusion"]["ms"]
            row["corners_per_frame"] = float(counts.float().mean())
        out["sizes"].append(row)
        del fr, mask
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


ST_BETAS = (4096, 16384, 65536)
ST_SIDES = (8, 16, 32, 48, 64, 96)


def run_stbox(args):
    """Spatio-temporal boxes against Eq. 6: the group K1, Kt (temporal binomial, reach n),
    K3, K4, K5 on 1024 x 1024 x 1000 RGBA video, run over boxes x * x * t. For each output
    volume beta = x^2 t the sides x in ST_SIDES with t = beta / x^2 are timed (CUDA events,
    inputs larger than L2), next to Sec. VI-D's bytes for the tiling, Eq. 3's data
    utilisation and Eq. 6's optimum; then a free sweep over (x, t) for the best box."""
    import torch
    from paper_1509_04394_gb300 import build as kbuild
    from paper_1509_04394_gb300 import kfuse as K
    kbuild.build()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = K.Context(0, harris=False)
    hbm_peak, peak_kind = peaks()
    T, H, W = args.pc_frames, args.pc_size or 1024, args.pc_size or 1024
    fr = pchain_video(dev, H, W, T, 40)
    mask = torch.zeros((T, H, W), dtype=torch.uint8, device=dev)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    px = T * H * W

    def time_box(n, x, t):
        run = lambda: K.kf_st_run(ctx.h, fr, W, mask, counts, n, x, t, stream)  # noqa: E731
        if args.pc_once:
            run()
            torch.cuda.synchronize()
            return None
        for _ in range(args.warmup):
            run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    def row(n, x, t):
        ms = time_box(n, x, t)
        model, clipped = K.kf_st_traffic(W, H, T, x, t, n)
        r = {"x": x, "t": t, "beta": x * x * t, "smem_bytes": K.kf_st_smem_bytes(n, x), "model_bytes_per_px": model / px,
             "clipped_bytes_per_px": clipped / px, "du_eq3": x * x * t / ((x + 4) ** 2 * (t + n))}
        if ms is not None:
            r.update({"ms": ms, "value": px / (ms / 1000) / 1e6, "hbm_frac": clipped / (ms / 1000) / 1e9 / hbm_peak})
        return r

    out = {"workload": f"spatio-temporal group (gray, temporal binomial, 3x3 Gaussian, Sobel, threshold) on "
                       f"{W}x{H}x{T} RGBA (64 generated frames, cycled)", "unit": "Mpixel/s",
           "peak_hbm_gbs": hbm_peak, "peak_kind": peak_kind, "l2": "inputs larger than L2 (4.2 GB frames)",
           "reaches": []}
    first = {}

    def same_as_first(n):  # every box shape gives the same masks and counts (or it is a bug)
        if args.pc_once:
            return None
        if n not in first:
            first[n] = (mask.clone(), counts.clone())
            return True
        return bool(torch.equal(first[n][0], mask) and torch.equal(first[n][1], counts))

    for n in (2, 4):
        rec = {"n": n, "dx": 2, "dt": n, "fixed_beta": [], "sweep": []}
        for beta in ST_BETAS:
            x6, t6 = K.kf_st_box_eq6(beta, n)
            rows = []
            for x in ST_SIDES:
                t = beta // (x * x)
                if t < 1:
                    continue
                rows.append(row(n, x, t))
                rows[-1]["identical_to_first_box"] = same_as_first(n)
            timed_rows = [r for r in rows if "ms" in r]
            best = min(timed_rows, key=lambda r: r["ms"]) if timed_rows else None
            least = min(rows, key=lambda r: r["clipped_bytes_per_px"])
            rec["fixed_beta"].append({"beta": beta, "eq6_x": x6, "eq6_t": t6, "boxes": rows,
                                      "fastest_x": best["x"] if best else None,
                                      "least_traffic_x": least["x"]})
        for x in (16, 32, 48, 64, 96):
            for t in (4, 8, 16, 32, 64):
                rec["sweep"].append(row(n, x, t))
                rec["sweep"][-1]["identical_to_first_box"] = same_as_first(n)
        timed = [r for r in rec["sweep"] if "ms" in r]
        if timed:
            b = min(timed, key=lambda r: r["ms"])
            rec["best"] = {"x": b["x"], "t": b["t"], "ms": b["ms"], "value": b["value"], "hbm_frac": b["hbm_frac"]}
        out["reaches"].append(rec)
        first.pop(n, None)
    print(json.dumps(out), flush=True)


def run_batch48(args):
    """The batching workload: 48 independent videos of four sizes (9.03 Gpixel) through one
    persistent launch replayed from a CUDA graph, chain + corner selection + LK per video.
    Each video cycles through its first 32 generated frames (generation time bound);
    per-frame cost does not depend on content beyond the corner count."""
    import torch
    from paper_1509_04394_gb300 import build as kbuild
    from paper_1509_04394_gb300 import kfuse as K
    kbuild.build()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = K.Context(0)
    KP = 256
    vids, masks, counts, tracks = [], [], [], []
    seed = 1000
    for (n, H, W, T) in BATCH48:
        P = sv.pitch_for(W)
        for _ in range(n):
            spec = sv.VideoSpec(T=T, H=H, W=W, seed=seed)
            seed += 1
            base, _ = sv.generate(spec, pitch=P, frames=range(min(T, 32)))
            src = torch.from_numpy(base).to(dev)
            f = torch.empty((T, H, P), dtype=torch.uint8, device=dev)
            for t0 in range(0, T, src.shape[0]):
                m = min(src.shape[0], T - t0)
                f[t0:t0 + m] = src[:m]
            vids.append((f, W))
            masks.append(torch.zeros_like(f))
            counts.append(torch.zeros(T, dtype=torch.int32, device=dev))
            tracks.append((KP, torch.zeros(T, dtype=torch.int32, device=dev),
                           torch.zeros((T, KP), dtype=torch.int32, device=dev), torch.zeros((T, KP), device=dev),
                           torch.zeros((T, KP), device=dev), torch.zeros((T, KP), dtype=torch.int32, device=dev)))
    px = sum(f.shape[0] * f.shape[1] * W for f, W in vids)
    # autotuned tile shape per video shape (rows per job; cached), then the persistent
    # launch's resident warps per SM for this batch (cached)
    from paper_1509_04394_gb300 import tuning
    cache = tuning.TuneCache(args.tune_cache)
    name = torch.cuda.get_device_name(dev)
    shape_rows = tuning.batch_rows(ctx.h, vids, cache, name, K.KF_PREC_F32, stream=stream)
    ws = torch.empty(K.kf_batch_workspace_bytes(ctx.h, [v for v, _ in vids], [w for _, w in vids], KP),
                     dtype=torch.uint8, device=dev)
    choices = [shape_rows] + [[r] * len(vids) for r in (200, 267, 400)]
    rows, warps, _ = tuning.batch_launch(ctx.h, vids, masks, counts, ws, tracks, choices, cache, name, stream=stream)
    b = K.kf_batch_create(ctx.h, [v for v, _ in vids], [w for _, w in vids], masks, counts, ws, tracks,
                          chunk_rows=rows, warps_per_sm=warps)

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k
    ms = timed(lambda: K.kf_batch_run(b, stream), args.steps)
    batch_out = [(m.clone(), c.clone(), tr[1].clone(), tr[2].clone()) for m, c, tr in zip(masks, counts, tracks)]
    # the same videos one kf_track call each, each with its own tuned tile height
    wsv = torch.empty(max(K.kf_track_workspace_bytes(ctx.h, w, v.shape[1], v.shape[0]) for v, w in vids),
                      dtype=torch.uint8, device=dev)

    def per_video(assign):
        for (v, w), m, c, tr, r in zip(vids, masks, counts, tracks, assign):
            K.kf_set_chunk_rows(ctx.h, r)
            K.kf_track(ctx.h, v, w, m, c, KP, *tr[1:], wsv, stream)
    # the per-video baseline gets the best of the same tile-height candidates
    seq = {i: timed(lambda: per_video(rc), max(1, args.steps // 2)) for i, rc in enumerate(choices)}
    best_seq = min(seq, key=seq.get)
    ms_seq = seq[best_seq]
    per_video(choices[best_seq])
    same = all(torch.equal(m, bo[0]) and torch.equal(c, bo[1]) and torch.equal(tr[1], bo[2]) and torch.equal(tr[2], bo[3])
               for m, c, tr, bo in zip(masks, counts, tracks, batch_out))
    # the batch before tuning: the context's default tile height, as many warps as fit
    K.kf_set_chunk_rows(ctx.h, 200)
    b0 = K.kf_batch_create(ctx.h, [v for v, _ in vids], [w for _, w in vids], masks, counts, ws, tracks)
    ms_untuned = timed(lambda: K.kf_batch_run(b0, stream), args.steps)
    K.kf_batch_destroy(b0)
    K.kf_batch_destroy(b)
    shapes = {f"{v.shape[1]}x{w}": r for (v, w), r in zip(vids, rows)}
    print(json.dumps({"workload": "48 videos: 16 x 192x432x600, 16 x 480x640x300, 12 x 800x600x1000, "
                                  "4 x 1080x1920x120 u8 (frames cycle every 32)",
                      "gpixel": px / 1e9, "ms_per_step": ms, "value": px / (ms / 1000) / 1e6, "unit": UNIT,
                      "per_video_calls_ms": ms_seq, "per_video_calls_value": px / (ms_seq / 1000) / 1e6,
                      "per_video_calls_ms_by_choice": [seq[i] for i in range(len(choices))],
                      "per_video_best_rows_per_shape": {f"{v.shape[1]}x{w}": r for (v, w), r in
                                                        zip(vids, choices[best_seq])},
                      "batch_over_per_video": ms_seq / ms, "identical_to_per_video": same,
                      "untuned_batch_ms": ms_untuned, "tile_rows_per_shape": shapes, "warps_per_sm": warps,
                      "standalone_tile_rows_per_shape": {f"{v.shape[1]}x{w}": r for (v, w), r in zip(vids, shape_rows)},
                      "device_error": K.kf_device_error(ctx.h)}), flush=True)


def run_costmodel(args):
    """The learned-cost-model workload: 400 random kernel DAGs (12-24 stages) on synthetic
    1080x1920 video; every candidate group of every DAG is timed by the executor on a
    prefix of the video (per-frame cost does not depend on the frame count); the MLP is
    trained on 300 DAGs and ranks partitions of the 100 held out, judged by the measured
    cost of its choice against the measured optimum and against the traffic model."""
    import torch
    from paper_1509_04394_gb300 import build as kbuild
    from paper_1509_04394_gb300 import costmodel as cm
    from paper_1509_04394_gb300 import kfuse as K
    from synth import dags as sd
    kbuild.build()
    dev = torch.device("cuda:0")
    W, H, T = 1920, 1080, args.cm_frames
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=5), pitch=W)
    f = torch.from_numpy(fr).to(dev)
    ctx = K.kf_create(0)
    t0 = time.time()
    meas = [cm.measure(ctx, sd.to_array(sd.random_dag(4000 + s)), f, W, 4000 + s) for s in range(400)]
    t1 = time.time()
    X, y = cm.dataset(meas[:300])
    loss = K.kf_costmodel_train(ctx, X, y, steps=4000, lr=3e-3, seed=1)
    t2 = time.time()
    ev = cm.evaluate(ctx, meas[300:])
    # end-to-end check of the additive model: run the chosen partitions of 10 held-out DAGs
    e2e = []
    for m in meas[300:310]:
        dag = K.kf_dag_create(ctx, m.rows)
        ws = torch.empty(K.kf_dag_workspace_bytes(dag, W, H, T), dtype=torch.uint8, device=dev)
        out = torch.empty((T, H, W), dtype=torch.float32, device=dev)
        row = next(r for r in ev["per_dag"] if r["seed"] == m.seed)
        for name, cuts in row["plans"].items():
            K.kf_dag_run(dag, cuts, f, W, out, ws)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                K.kf_dag_run(dag, cuts, f, W, out, ws)
            e1.record()
            torch.cuda.synchronize()
            e2e.append({"seed": m.seed, "plan": name, "run_ms": e0.elapsed_time(e1) / 3,
                        "sum_of_groups_ms": cm.partition_cost(m, cuts)})
        K.kf_dag_destroy(dag)
        del ws, out
    ev.pop("per_dag")
    ratio = [r["run_ms"] / r["sum_of_groups_ms"] for r in e2e]
    print(json.dumps({"workload": f"400 random DAGs (12-24 stages), 1080x1920 u8, groups timed on {T} frames",
                      "train_dags": 300, "held_out_dags": 100, "train_samples": int(len(y)),
                      "final_std_mse": loss, "measure_s": t1 - t0, "train_s": t2 - t1, **ev,
                      "end_to_end_over_sum_of_groups": {"median": float(np.median(ratio)), "min": float(min(ratio)),
                                                        "max": float(max(ratio)), "runs": len(ratio)}}),
          flush=True)


def run_dagplan(args):
    """Recompute instead of store: on the learned-cost-model workload (400 random DAGs,
    1080x1920, groups timed on a prefix of the video), each of the 100 held-out DAGs is
    planned over contiguous partitions and over plans with inlined (recomputed) nodes by
    two MLPs -- one trained on the 300 training DAGs' contiguous groups, one also on 60
    sampled groups with inlined nodes per training DAG -- and the plans, with the
    measured-best contiguous partition, run end to end (CUDA events); bits compared."""
    import torch
    from paper_1509_04394_gb300 import build as kbuild
    from paper_1509_04394_gb300 import costmodel as cm
    from paper_1509_04394_gb300 import kfuse as K
    from synth import dags as sd
    kbuild.build()
    dev = torch.device("cuda:0")
    W, H, T = 1920, 1080, args.cm_frames
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=5), pitch=W)
    f = torch.from_numpy(fr).to(dev)
    ctx_c, ctx_x = K.kf_create(0), K.kf_create(0)
    meas = [cm.measure(ctx_c, sd.to_array(sd.random_dag(4000 + s)), f, W, 4000 + s) for s in range(400)]
    Xc, yc = cm.dataset(meas[:300])
    inl = [cm.measure_inlined(ctx_c, m.rows, f, W, 9000 + m.seed) for m in meas[:300]]
    Xi = np.concatenate([x for x, _ in inl])
    yi = np.concatenate([y for _, y in inl])
    K.kf_costmodel_train(ctx_c, Xc, yc, steps=4000, lr=3e-3, seed=1)
    K.kf_costmodel_train(ctx_x, np.concatenate([Xc, Xi]).astype(np.float32), np.concatenate([yc, yi]), steps=4000,
                         lr=3e-3, seed=1)
    out_a = torch.empty((T, H, W), dtype=torch.float32, device=dev)
    out_b = torch.empty((T, H, W), dtype=torch.float32, device=dev)

    def run_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    rows = []
    for m in meas[300:]:
        dag = K.kf_dag_create(ctx_c, m.rows)
        ws = torch.empty(K.kf_dag_workspace_bytes(dag, W, H, T), dtype=torch.uint8, device=dev)
        best_cuts = cm.plan_costs(ctx_c, m)["measured"]
        t_best = run_ms(lambda: K.kf_dag_run(dag, best_cuts, f, W, out_a, ws))
        r = {"seed": m.seed, "n": m.n, "best_contiguous_ms": t_best}
        same = True
        for name, ctx in (("mlp", ctx_c), ("mlp_inl", ctx_x)):
            cont = cm.plan_costs(ctx, m)["mlp"]
            cx, xm, _ = K.kf_dag_plan_recompute(dag, W, H, T, model=ctx)
            r[name + "_contiguous_ms"] = run_ms(lambda: K.kf_dag_run(dag, cont, f, W, out_a, ws))
            r[name + "_recompute_ms"] = run_ms(lambda: K.kf_dag_run_x(dag, cx, xm, f, W, out_b, ws))
            r[name + "_inlined"] = bin(xm).count("1")
            same = same and bool(torch.equal(out_a, out_b))
        # measured search: inline one node at a time on top of the measured-best partition
        best_j, t_j = 0, t_best
        for j in range(1, m.n):
            try:
                t = run_ms(lambda: K.kf_dag_run_x(dag, best_cuts, 1 << (j - 1), f, W, out_b, ws), reps=2)
            except K.KfuseError:
                continue
            same = same and bool(torch.equal(out_a, out_b))
            if t < t_j:
                best_j, t_j = j, t
        r["measured_one_inlined_ms"], r["measured_inlined_node"] = t_j, best_j
        r["same_bits"] = same
        rows.append(r)
        K.kf_dag_destroy(dag)
        del ws

    def summary(name):
        x = np.array([q[name + "_recompute_ms"] for q in rows])
        c = np.array([q[name + "_contiguous_ms"] for q in rows])
        best = np.array([q["best_contiguous_ms"] for q in rows])
        used = np.array([q[name + "_inlined"] > 0 for q in rows])
        return {"plans_with_inlined_nodes": int(used.sum()),
                "recompute_over_own_contiguous": {"mean": float((x / c).mean()),
                                                  "mean_where_inlined": float((x / c)[used].mean()) if used.any() else 1.0,
                                                  "min": float((x / c).min()), "max": float((x / c).max())},
                "recompute_over_measured_best_contiguous": {"mean": float((x / best).mean()),
                                                            "faster": int(np.sum(x < best))},
                "contiguous_over_measured_best": float((c / best).mean())}
    print(json.dumps({"workload": f"100 held-out random DAGs (12-24 stages), 1080x1920 u8, {T} frames",
                      "dags": len(rows), "inlined_training_samples": int(len(yi)),
                      "mlp_contiguous_training": summary("mlp"), "mlp_with_inlined_training": summary("mlp_inl"),
                      "measured_one_inlined_over_best_contiguous": {
                          "mean": float(np.mean([q["measured_one_inlined_ms"] / q["best_contiguous_ms"] for q in rows])),
                          "improved_dags": int(sum(q["measured_inlined_node"] > 0 for q in rows)),
                          "min": float(min(q["measured_one_inlined_ms"] / q["best_contiguous_ms"] for q in rows))},
                      "all_bits_equal": all(q["same_bits"] for q in rows), "per_dag": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--rows", type=int, default=0, help="fixed tile height for the step (default: autotuned)")
    ap.add_argument("--profile", type=int, default=0, help="profiler case: fused chain only, on T frames")
    ap.add_argument("--cuts", type=int, default=-1, help="partition for --profile (default: planned)")
    ap.add_argument("--f16", action="store_true", help="FP16 maps for --profile")
    ap.add_argument("--track", action="store_true", help="--profile the whole path with tracking")
    ap.add_argument("--batch48", action="store_true", help="the 48-video batching workload")
    ap.add_argument("--tune-cache", default=os.path.join(ROOT, ".kfuse_tune_cache.json"),
                    help="JSON file of autotuning results (--batch48)")
    ap.add_argument("--costmodel", action="store_true", help="the learned-cost-model workload")
    ap.add_argument("--cm-frames", type=int, default=24, help="frames the groups are timed on (--costmodel; 24 "
                    "frames of 1080 x 1920 make every map between groups larger than L2)")
    ap.add_argument("--pchain", action="store_true", help="the paper's own chain: no / two / full fusion")
    ap.add_argument("--pc-frames", type=int, default=1000, help="frames per size (--pchain)")
    ap.add_argument("--pc-size", type=int, default=0, help="one square size instead of the three (--pchain)")
    ap.add_argument("--pc-once", action="store_true", help="run each partition once, untimed (profiler case)")
    ap.add_argument("--dagplan", action="store_true", help="recompute-vs-store DAG plans (learned costs)")
    ap.add_argument("--partitions", action="store_true", help="all 128 partitions of the chain timed on "
                    "600 x 192 x 432 (traffic model vs measured)")
    ap.add_argument("--partitions-full", action="store_true", help="--partitions on the 1000 x 800 x 600 workload")
    ap.add_argument("--partitions-table", default="", help="--partitions: also write every row to this JSON file")
    ap.add_argument("--stbox", action="store_true", help="spatio-temporal boxes against Eq. 6 (uses --pc-frames, "
                    "--pc-size, --pc-once)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.partitions:
        run_partitions(args)
    elif args.pchain:
        run_pchain(args)
    elif args.stbox:
        run_stbox(args)
    elif args.dagplan:
        run_dagplan(args)
    elif args.costmodel:
        run_costmodel(args)
    elif args.batch48:
        run_batch48(args)
    elif args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
