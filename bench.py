#!/usr/bin/env python
"""Throughput of the stereo hot path (census cost volume -> Dual MM ->
primal-dual refinement) on one synthetic KITTI-shaped frame per step.

One step = one frame of 1242x375 pixels with 128 labels: cost volume, 10 Dual
MM iterations (horizontal + vertical pass each), 100 primal-dual iterations
in 5 warps.  Inputs are resident on the GPU when the timed region starts; L2
is flushed (a 256 MB write) between steps, outside the timed events.

Prints one JSON line (rank 0).  With --impl reference the CPU oracle is timed
instead, on a bounded crop of the same workload.  Under torchrun each rank
solves its own frame (replicas; weak scaling; no collective on the data path).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel·labels/s (discrete+continuous) at 1242×375×128"
UNIT = "Mpixel·labels/s"
CPU_SAMPLE_ROWS = 24


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="kitti", choices=["kitti", "diff", "stream", "batch", "lr", "minorants", "flow"],
                    help="kitti: the plain method on the 1242x375x128 frame (default); "
                         "diff: forward + reverse mode of 200 PD iterations at 512x256x96; "
                         "stream: 60 warm-started frames of 1920x1080x256 (uint16 costs); "
                         "batch: 32 pairs of mixed size and label count in one CUDA graph; "
                         "lr: both views of the 1242x375x128 frame and the consistency check; "
                         "minorants: Dual MM with the hierarchical, naive and iterative minorants; "
                         "flow: optical flow of a 640x480 pair with 64x64 displacements")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, ws: int, device) -> float:
    """The slowest rank's time (an all-reduce MAX; the local value when alone)."""
    if ws <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_step: int, steps: int, ws: int, tot_ms: float) -> float:
    """Whole-job throughput in millions of units per second: every rank solves its
    own frames (replicas, weak scaling), timed by the slowest rank."""
    return units_per_step * steps * ws / (tot_ms / 1e3) / 1e6


# ---------------------------------------------------------------------------
# CPU oracle on a bounded crop (the cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def cpu_sample(rows: int = CPU_SAMPLE_ROWS):
    from paper_1601_06274_gb300 import synthetic as S
    spec = S.KITTI
    sp = S.make_workload(spec, seed=0)
    return sp.left[:rows].copy(), sp.right[:rows].copy(), spec


def time_oracle(left, right, spec):
    from oracle import oracle as O
    O.lib()
    t0 = time.perf_counter()
    O.solve(left, right, spec["L"], spec["dmm_iters"], spec["pd_iters"], nthreads=os.cpu_count())
    return time.perf_counter() - t0


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    left, right, spec = cpu_sample()
    units = left.shape[0] * left.shape[1] * spec["L"]
    for _ in range(args.warmup):
        time_oracle(left, right, spec)
    ts = [time_oracle(left, right, spec) for _ in range(args.steps)]
    tot = sum(ts)
    value = units * args.steps / tot / 1e6
    sample = (f"rows 0-{left.shape[0] - 1} of the 1242x375x128 frame (a {left.shape[1]}x"
              f"{left.shape[0]}x{spec['L']} crop), {spec['dmm_iters']} Dual MM + "
              f"{spec['pd_iters']} PD iterations per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
        "config": {"workload": "kitti-1242x375x128 (cpu crop)", "dmm_iters": spec["dmm_iters"],
                   "pd_iters": spec["pd_iters"]},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        import torch
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(device_index).uuid)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", uuid, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a few hundred ms to start: wait (at most 3 s) for its
        # first sample so that the sampling covers the whole timed region
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# Differentiable form: forward with checkpoints + reverse mode
# ---------------------------------------------------------------------------

DIFF = dict(H=256, W=512, L=96, iters=200, ckpt=20)
DIFF_METRIC = "Mpixel·labels/s (forward+reverse, 200 PD iterations) at 512×256×96"
# algorithmic bytes per pixel of one launch of each PD kernel (float32 state):
# forward iteration: reads u, p, q (5 x 4 B), u0, s1, s2, lo, hi (5 x 4 B), two
# uint8 weights, writes u, p, q (5 x 4 B); reverse iteration: reads state k and
# u_{k+1} (6 x 4 B), the linearisation (5 x 4 B), weights (2 B), the output
# adjoints (5 x 4 B), writes the input adjoints (5 x 4 B) and updates four
# float accumulators (4 x 8 B)
PD_FWD_BYTES = 62
PD_ADJ_BYTES = 118


def run_diff(args):
    import numpy as np
    import torch
    from paper_1601_06274_gb300 import build, dm, synthetic as S
    build.build()
    ws, rank, local = dist_env()
    dev = torch.device("cuda", 0)
    H, W, L, NP, CK = DIFF["H"], DIFF["W"], DIFF["L"], DIFF["iters"], DIFF["ckpt"]
    sp = S.make_pair(H, W, L, planes=8, noise_sigma=2.0, seed=rank)
    ctx = dm.Context(H, W, L, device=str(dev))
    stream = ctx.stream
    ctx.cost_volume(sp.left, sp.right)
    ctx.discrete(10)
    c8, wh_t, wv_t = ctx.cost()
    g = torch.Generator(device=dev).manual_seed(rank)
    cost = (c8.float() + torch.rand(c8.shape, device=dev, generator=g)).contiguous()
    alpha = (0.5 + torch.rand((H, W), device=dev, generator=g)).contiguous()
    gt = torch.from_numpy(sp.gt).to(dev, torch.float32)
    ctx.set_cost_volume_f32(cost)
    ctx.set_data_weights(alpha)
    tape = torch.empty(ctx.tape_bytes(NP, CK), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        ctx.refine_tape(NP, CK, None, tape)      # from the labels of the discrete stage
        u = ctx.disparity()
        gu = torch.sign(u - gt) / u.numel()       # d/du of the L1 loss
        return ctx.refine_backward(gu, tape)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    launches0 = ctx.launch_count()
    clk = Clocks(0)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = ctx.launch_count() - launches0
    tot_ms = sum(a.elapsed_time(b) for a, b in evs)
    units = H * W * L
    value = units * args.steps / (tot_ms / 1e3) / 1e6
    # the plain forward on the same inputs
    pf = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.refine(NP)
        b.record(stream)
        pf.append((a, b))
    torch.cuda.synchronize()
    plain_ms = sum(a.elapsed_time(b) for a, b in pf) / len(pf)
    # end to end: inputs from pinned host memory, gradients back to the host
    h_cost = cost.cpu().pin_memory()
    h_alpha = alpha.cpu().pin_memory()
    h_gc = torch.empty_like(h_cost).pin_memory()
    d_cost = torch.empty_like(cost)
    d_alpha = torch.empty_like(alpha)
    e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            d_cost.copy_(h_cost, non_blocking=True)
            d_alpha.copy_(h_alpha, non_blocking=True)
            ctx.set_cost_volume_f32(d_cost)
            ctx.set_data_weights(d_alpha)
            gc, ga, gl, _ = step()
            h_gc.copy_(gc, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        e_ms.append(a.elapsed_time(b))
    e2e_value = units * args.steps / (sum(e_ms) / 1e3) / 1e6
    # per-kernel averages: one forward and one reverse iteration
    fwd_ev, adj_ev = [], []
    tape2 = ctx.refine_tape(NP, CK, None, tape)
    u = ctx.disparity()
    gu = torch.sign(u - gt) / u.numel()
    for k in range(3):
        a, b, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        flush.fill_(k & 0xff)
        a.record(stream)
        ctx.refine(NP)
        b.record(stream)
        ctx.refine_backward(gu, tape2)
        c2.record(stream)
        fwd_ev.append((a, b))
        adj_ev.append((b, c2))
    torch.cuda.synchronize()
    fwd_it_ms = sum(a.elapsed_time(b) for a, b in fwd_ev) / len(fwd_ev) / NP
    bwd_ms = sum(a.elapsed_time(b) for a, b in adj_ev) / len(adj_ev)
    # the reverse pass runs NP forward (recompute) and NP reverse iterations
    adj_it_ms = (bwd_ms - NP * fwd_it_ms) / NP
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6800.0, "fallback"
    if os.path.exists(peaks_path):
        peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
    achieved = PD_ADJ_BYTES * H * W / (adj_it_ms / 1e3) / 1e9
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the oracle's reverse mode on the first rows of the same inputs
        from oracle import oracle as O
        rows = 32
        wh_c = wh_t[:rows].cpu().numpy().astype(np.float64)
        wv_c = wv_t[:rows].cpu().numpy().astype(np.float64)
        wv_c[-1, :] = 0.0
        u0_c = dm.labels_u16(ctx.labels())[:rows].astype(np.float64)
        t0 = time.perf_counter()
        O.refine_grad(cost[:rows].double().cpu().numpy(), wh_c, wv_c, u0_c, NP,
                      gt[:rows].double().cpu().numpy(), O.Params(),
                      alpha=alpha[:rows].double().cpu().numpy())
        t_cpu = time.perf_counter() - t0
        cpu = {"value": round(rows * W * L / t_cpu / 1e6, 4), "unit": "Mpixel·labels/s",
               "cores": 1, "kind": "oracle",
               "sample": f"rows 0-{rows - 1} ({W}x{rows}x{L}), forward and reverse of {NP} "
                         f"iterations in FP64, {t_cpu:.2f} s"}
    line = {
        "metric": DIFF_METRIC, "value": round(value, 3), "unit": "Mpixel·labels/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "diff-512x256x96", "H": H, "W": W, "L": L, "pd_iters": NP,
                   "checkpoint_every": CK, "warps": 5, "loss": "L1(u, gt)",
                   "grads": ["cost", "alpha", "lambda_r"],
                   "l2": "flushed between steps (256 MB write, outside the timed events)"},
        "plain_forward_ms": round(plain_ms, 4),
        "reverse_over_forward": round(tot_ms / args.steps / plain_ms, 3),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "pd_adjoint_kernel (one reverse iteration, derived: reverse pass "
                               "minus the recompute, per iteration)",
                     "peak_source": peak_src,
                     "fwd_iter_us": round(fwd_it_ms * 1e3, 3),
                     "adj_iter_us": round(adj_it_ms * 1e3, 3)},
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 3), "unit": "Mpixel·labels/s",
                "h2d_bytes_per_step": 4 * H * W * L + 4 * H * W,
                "d2h_bytes_per_step": 4 * H * W * L},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Algorithmic bytes (the hot-path table's compulsory bytes, int16 duals) and
# the bytes of the implementation's own storage
# ---------------------------------------------------------------------------

def survey_pass_bytes(HW: int, L: int) -> dict:
    """Compulsory bytes of one Dual MM pass with int16 duals: the horizontal
    pass reads c (1 B) and lambda_v (2 B) and writes lambda_h (2 B) per
    pixel-label; the vertical pass reads lambda_h and writes lambda_v (2 + 2 B)."""
    return {0: HW * L * 5, 1: HW * L * 4}


def survey_frame_bytes(HW: int, L: int, cost_bytes: int, dmm_iters: int, pd_iters: int,
                       warps: int) -> int:
    """Compulsory bytes of one frame: census + cost (2 B/px read, L cost_bytes
    B/px written), Dual MM at 9 B per pixel-label and iteration (the first
    iteration's lambda_v read skipped), linearisation at 23 B/px per warp and
    60 B/px per primal-dual iteration."""
    return (HW * (2 + L * cost_bytes) + HW * L * (9 * dmm_iters - 2) + HW * 23 * warps
            + HW * 60 * pd_iters)


def dmm_pass_bytes(kernel: int, delta_bytes: int, cost_bytes: int, HW: int, L: int) -> dict:
    """Bytes the implementation's own storage makes a pass move at least.
    Packed kernels (8, 16): the horizontal pass reads the deltas of c +
    lambda_v and c and writes those of lambda_h, the vertical pass reads
    lambda_h and c and writes c + lambda_v (the deltas plus a 4-byte base per
    pixel each; the one-warp kernel reads c only on the vertical pass).  int32
    kernel: the horizontal pass reads c and lambda_v and writes lambda_h, the
    vertical pass reads lambda_h and writes lambda_v."""
    if kernel == 8:
        return {0: HW * ((2 * delta_bytes + cost_bytes) * L + 8),
                1: HW * ((2 * delta_bytes + cost_bytes) * L + 8)}
    if kernel == 16:
        return {0: HW * (2 * delta_bytes * L + 8),
                1: HW * ((2 * delta_bytes + cost_bytes) * L + 8)}
    return {0: HW * L * (cost_bytes + 8), 1: HW * L * 8}


def hbm_peak():
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        return float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def time_passes(ctx, d_left, d_right, iters, reps, flush, stream, warm_prev=None):
    """Average duration of each Dual MM pass (CUDA events on the context's stream)."""
    import torch
    if warm_prev is None:
        ctx.cost_volume(d_left, d_right)
    else:
        ctx.cost_volume(*warm_prev)
        ctx.discrete(iters)
        ctx.cost_volume_warm(d_left, d_right)
    pass_ms = {0: [], 1: []}
    for _ in range(reps):
        for it in range(iters):
            for which in (0, 1):
                flush.fill_(it & 0xff)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.discrete_pass(which)
                b.record(stream)
                pass_ms[which].append((a, b))
        ctx.reset_duals()
    torch.cuda.synchronize()
    return {w: sum(a.elapsed_time(b) for a, b in v) / len(v) for w, v in pass_ms.items()}


def time_stages(ctx, d_left, d_right, dmm_iters, pd_iters, flush, stream, reps=5):
    """Average duration of each stage of one solve (CUDA events on the
    context's stream, L2 flushed before each): the census and cost volume, the
    dmm_iters Dual MM iterations, and the pd_iters refinement iterations."""
    import torch
    ev = {"census_and_cost_volume": [], "dual_mm": [], "refinement": []}

    def rec(name, fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ev[name].append((a, b))

    with torch.cuda.stream(stream):
        for r in range(reps):
            flush.fill_(r & 0xff)
            rec("census_and_cost_volume", lambda: ctx.cost_volume(d_left, d_right))
            flush.fill_(r & 0xff)
            rec("dual_mm", lambda: ctx.discrete(dmm_iters))
            flush.fill_(r & 0xff)
            rec("refinement", lambda: ctx.refine(pd_iters))
    torch.cuda.synchronize()
    out = {k: round(sum(a.elapsed_time(b) for a, b in v) / len(v), 4) for k, v in ev.items()}
    out["refinement_iterations"] = pd_iters
    return out


def refinement_issue(ms, iters):
    """The refinement's single launch against the instruction-issue bound: warp
    instructions of its ncu capture (null once pd.cu has changed) over the
    stage's measured time."""
    inst = NCU_PD_INSTRUCTIONS.get(("pd_res_kernel", iters, source_tag("pd.cu")))
    out = {"kernel": "pd_res_kernel", "bound": "issue", "ms": ms,
           "warp_instructions_per_launch": inst, "issue_frac": None}
    if inst is not None and ms > 0:
        out["issue_frac"] = round(inst / (ms / 1e3) / 1e9 / ISSUE_PEAK_GINST_S, 4)
    return out


def source_tag(kernel_file: str) -> str:
    """First 12 hex digits of the SHA-256 of a kernel's source file: a profile
    figure is used only while the kernel it was captured from is unchanged."""
    path = os.path.join(ROOT, "paper_1601_06274_gb300", "csrc", kernel_file)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:12]


def roofline_line(ctx, avg, HW, L, cost_bytes, kernel_names, workload="kitti"):
    """Roofline of the slower Dual MM pass: achieved = the compulsory bytes of
    the pass (int16 duals) / its average duration; frac_storage uses the bytes
    of the implementation's own storage instead.  traffic and the instruction
    count come from an ncu capture of the same kernel source, else null."""
    kernel, dbytes = ctx.path()
    alg = survey_pass_bytes(HW, L)
    own = dmm_pass_bytes(kernel, dbytes, cost_bytes, HW, L)
    dom = max((0, 1), key=lambda w: avg[w])
    peak, src = hbm_peak()
    sec = avg[dom] / 1e3
    achieved = alg[dom] / sec / 1e9
    name = kernel_names[kernel] + (" horizontal" if dom == 0 else " vertical") + " pass"
    # from 128 labels on, a lane-group pass runs as two kernels: the top levels
    # (one CTA per chain), then the depth-first units on persistent CTAs; the
    # vertical pass at 128 labels stays one kernel
    split = kernel == 8 and L >= 128 and not (L <= 128 and dom == 1)
    key = (workload, name, source_tag(KERNEL_FILES[kernel]))
    line = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": NCU_TRAFFIC.get(key),
            "kernel": name, "peak_source": src, "bytes_per_launch": alg[dom],
            "bytes_rule": "5 B (horizontal) / 4 B (vertical) per pixel-label: int16 duals",
            "frac_storage": round(own[dom] / sec / 1e9 / peak, 4),
            "storage_bytes_per_launch": own[dom],
            "dual_storage": f"{dbytes}-byte deltas" if kernel in (8, 16) else "int32",
            "pass_ms": {"horizontal": round(avg[0], 4), "vertical": round(avg[1], 4)}}
    if split:
        line["kernels"] = ["dmg_kernel (levels down to KL, one CTA per chain)",
                           "dmg_units_kernel (depth-first units, persistent CTAs)"]
    inst = NCU_INSTRUCTIONS.get(key)
    if inst is not None:
        rate = inst / sec / 1e9
        line["issue_frac"] = round(rate / ISSUE_PEAK_GINST_S, 4)
        line["issue"] = {"warp_instructions_per_launch": inst, "achieved_ginst_s": round(rate, 1),
                         "peak_ginst_s": round(ISSUE_PEAK_GINST_S, 1)}
    return line


KERNEL_NAMES = {8: "dmg_kernel", 16: "dmm16_kernel", 32: "dmm_pass_kernel"}
KERNEL_FILES = {8: "dmg_impl.cuh", 16: "dmm16_impl.cuh", 32: "dmm.cu"}
# dram__bytes_read.sum + dram__bytes_write.sum per launch from the ncu captures
# summarised in profiles/, keyed by workload, kernel and the kernel source's tag
# (source_tag) at capture time: a kernel changed since its capture reports null
NCU_TRAFFIC = {
    # profiles/dmg_kernel_kitti_1242x375x128.md (the horizontal pass: its two
    # kernels together)
    ("kitti", "dmg_kernel horizontal pass", "51e0dbb4b9e3"): 317_615_360,
    ("kitti", "dmg_kernel vertical pass", "51e0dbb4b9e3"): 245_022_464,
    # profiles/dmm_alt_staged_kernel_minorants_1242x375x128.md:
    # dram__bytes.sum.per_second x gpu__time_duration.sum of the capture
    ("minorants", "dmm_alt_staged_kernel horizontal pass", "4ac94b722085"): 3_568_100_000,
    ("minorants", "dmm_alt_staged_kernel vertical pass", "4ac94b722085"): 3_343_700_000,
    ("lr", "lr_check_kernel", "68c80f87cd1d"): 3_732_000,
}
# smsp__inst_executed.sum per launch from the same captures: a Dual MM pass is
# bound by instruction issue and latency, so its issue rate is reported beside
# the HBM roofline, against 152 SMs x 4 schedulers x 1 warp-instruction per
# cycle at 2070 MHz
NCU_INSTRUCTIONS = {
    ("kitti", "dmg_kernel horizontal pass", "51e0dbb4b9e3"): 272_887_919,
    ("kitti", "dmg_kernel vertical pass", "51e0dbb4b9e3"): 252_160_776,
}
# the refinement kernel (profiles/pd_res_kernel_kitti_1242x375x128.md): warp
# instructions per launch of 100 iterations, keyed by the source tag of pd.cu
NCU_PD_INSTRUCTIONS = {("pd_res_kernel", 100, "468a4778602a"): 347_755_545}
ISSUE_PEAK_GINST_S = 152 * 4 * 2.070


# ---------------------------------------------------------------------------
# Streaming: 60 warm-started frames of 1920x1080x256 with uint16 costs
# ---------------------------------------------------------------------------

def run_stream(args):
    import numpy as np
    import torch
    from paper_1601_06274_gb300 import build, dm, synthetic as S
    build.build()
    dev = torch.device("cuda", 0)
    spec = S.STREAM
    H, W, L, NF = spec["H"], spec["W"], spec["L"], spec["frames"]
    NI, NP = spec["dmm_iters"], spec["pd_iters"]
    frames = list(S.make_sequence(H, W, L, NF, planes=spec["planes"],
                                  noise_sigma=spec["noise_sigma"], drift=spec["drift"], seed=0))
    d_frames = [(torch.from_numpy(f.left).to(dev), torch.from_numpy(f.right).to(dev))
                for f in frames]
    ctx = dm.Context(H, W, L, dm.default_params(cost_bytes=2), device=str(dev))
    stream = ctx.stream
    d_u = torch.empty((H, W), dtype=torch.float32, device=dev)
    for k in range(args.warmup):
        if k == 0:
            ctx.solve(*d_frames[0], NI, NP, out=d_u)
        else:
            ctx.solve_next(*d_frames[k % NF], NI, NP, out=d_u)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(NF)]
    launches0 = ctx.launch_count()
    clk = Clocks(0)
    with torch.cuda.stream(stream):
        for f in range(NF):
            evs[f][0].record(stream)
            if f == 0:
                ctx.solve(*d_frames[0], NI, NP, out=d_u)      # cold start
            else:
                ctx.solve_next(*d_frames[f], NI, NP, out=d_u)  # warm start from frame f - 1
            evs[f][1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = ctx.launch_count() - launches0
    ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(ms)
    fps = NF / (tot_ms / 1e3)
    cold = []
    for f in range(min(NF, 5)):       # the same frames, each from a cold start
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.solve(*d_frames[f], NI, NP, out=d_u)
        b.record(stream)
        cold.append((a, b))
    torch.cuda.synchronize()
    cold_ms = sum(a.elapsed_time(b) for a, b in cold) / len(cold)
    # warm vs cold lower bound after the iterations on one frame
    ctx.solve(*d_frames[0], NI, NP, out=d_u)
    ctx.solve_next(*d_frames[1], NI, NP, out=d_u)
    lb_warm = ctx.lower_bounds(NI)
    ctx.solve(*d_frames[1], NI, NP, out=d_u)
    lb_cold = ctx.lower_bounds(NI)
    # end to end: pinned host frames in, the disparity back to the host, per frame
    h_frames = [(torch.from_numpy(f.left).pin_memory(), torch.from_numpy(f.right).pin_memory())
                for f in frames]
    h_u = torch.empty((H, W), dtype=torch.float32).pin_memory()
    dl, dr = torch.empty_like(d_frames[0][0]), torch.empty_like(d_frames[0][1])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    with torch.cuda.stream(stream):
        for f in range(NF):
            dl.copy_(h_frames[f][0], non_blocking=True)
            dr.copy_(h_frames[f][1], non_blocking=True)
            if f == 0:
                ctx.solve(dl, dr, NI, NP, out=d_u)
            else:
                ctx.solve_next(dl, dr, NI, NP, out=d_u)
            h_u.copy_(d_u, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_fps = NF / (a.elapsed_time(b) / 1e3)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    avg = time_passes(ctx, *d_frames[1], NI, 1, flush, stream, warm_prev=d_frames[0])
    roof = roofline_line(ctx, avg, H * W, L, 2, KERNEL_NAMES)
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle on the first row of frame 0 (cold start), the whole path
        from oracle import oracle as O
        t0 = time.perf_counter()
        O.solve(frames[0].left[:1].copy(), frames[0].right[:1].copy(), L, NI, NP,
                nthreads=os.cpu_count())
        t_cpu = time.perf_counter() - t0
        cpu = {"value": round(1.0 / H / t_cpu, 6), "unit": "frames/s", "cores": 1,
               "kind": "oracle",
               "sample": f"row 0 of frame 0 ({W}x1x{L}), {NI} Dual MM + {NP} PD iterations, "
                         f"{t_cpu:.2f} s; frames/s = 1 / ({H} x that time)"}
    line = {
        "metric": "frames/s (discrete+continuous), 60 warm-started frames of 1920×1080×256",
        "value": round(fps, 3), "unit": "frames/s", "n_gpus": 1, "steps": NF,
        "warmup": args.warmup, "ms_per_step": round(tot_ms / NF, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int16x2+int32+f32",
        "data": "synthetic",
        "config": {"workload": "stream-1920x1080x256", "H": H, "W": W, "L": L, "frames": NF,
                   "dmm_iters": NI, "pd_iters": NP, "cost": "uint16",
                   "warm_start": "lambda_v of the previous frame",
                   "l2": "inputs larger than L2 (1.06 GB cost volume per frame)"},
        "latency_ms": {"p50": round(float(np.percentile(ms, 50)), 3),
                       "p99": round(float(np.percentile(ms, 99)), 3),
                       "max": round(max(ms), 3), "cold_start_mean": round(cold_ms, 3)},
        "lower_bound_frame1": {"warm": int(lb_warm[-1]), "cold": int(lb_cold[-1]),
                               "warm_first_iter": int(lb_warm[0]),
                               "cold_first_iter": int(lb_cold[0])},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_fps, 3), "unit": "frames/s", "h2d_bytes_per_step": 2 * H * W,
                "d2h_bytes_per_step": 4 * H * W},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Batched form: 32 pairs of mixed size and label count, one captured graph
# ---------------------------------------------------------------------------

def run_batch(args):
    import numpy as np
    import torch
    from paper_1601_06274_gb300 import build, dm, synthetic as S
    build.build()
    dev = torch.device("cuda", 0)
    specs = S.batch_specs(32, seed=0)
    shapes = [(s["H"], s["W"], s["L"]) for s in specs]
    NI, NP = specs[0]["dmm_iters"], specs[0]["pd_iters"]
    pairs = [S.make_workload(s, seed=s["seed"]) for s in specs]
    b = dm.Batch(shapes, device=str(dev))
    lefts = [torch.from_numpy(p.left).to(dev) for p in pairs]
    rights = [torch.from_numpy(p.right).to(dev) for p in pairs]
    cache = os.path.join(tempfile.gettempdir(), "dm_batch_tune.txt")
    t0 = time.perf_counter()
    choice = b.tune(lefts, rights, cache)
    tune_s = time.perf_counter() - t0
    outs = b.outputs()
    b.capture(lefts, rights, NI, NP, outs)
    for _ in range(args.warmup):
        b.replay()
    b.sync()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = b.stream
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    launches0 = b.launch_count()
    clk = Clocks(0)
    for k in range(args.steps):
        with torch.cuda.stream(st):
            flush.fill_(k & 0xff)
            evs[k][0].record(st)
        b.replay()
        with torch.cuda.stream(st):
            evs[k][1].record(st)
    b.sync()
    clocks = clk.stop()
    launches = b.launch_count() - launches0
    tot_ms = sum(a.elapsed_time(c) for a, c in evs)
    units = sum(H * W * L for H, W, L in shapes)
    value = units * args.steps / (tot_ms / 1e3) / 1e6
    # the same 32 pairs one after another through the single-pair path
    ctxs = [dm.Context(H, W, L, device=str(dev)) for H, W, L in shapes]
    for c, l, r in zip(ctxs, lefts, rights):
        c.solve(l, r, NI, NP)
    torch.cuda.synchronize()
    sp_ms = []
    for k in range(max(1, args.steps // 2)):
        flush.fill_(k & 0xff)
        a, c2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for c, l, r in zip(ctxs, lefts, rights):
            c.solve(l, r, NI, NP)
        c2.record()
        torch.cuda.synchronize()
        sp_ms.append(a.elapsed_time(c2))
    single_ms = sum(sp_ms) / len(sp_ms)
    # end to end: pinned host images into the captured buffers, disparities back
    h_l = [torch.from_numpy(p.left).pin_memory() for p in pairs]
    h_r = [torch.from_numpy(p.right).pin_memory() for p in pairs]
    h_u = [torch.empty(o.shape, dtype=torch.float32).pin_memory() for o in outs]
    torch.cuda.synchronize()
    e_ms = []
    for k in range(args.steps):
        a, c2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            a.record(st)
            for i in range(len(pairs)):
                lefts[i].copy_(h_l[i], non_blocking=True)
                rights[i].copy_(h_r[i], non_blocking=True)
        with torch.cuda.stream(st):
            b.replay()
            for i in range(len(pairs)):
                h_u[i].copy_(outs[i], non_blocking=True)
            c2.record(st)
        b.sync()
        e_ms.append(a.elapsed_time(c2))
    e2e_value = units * args.steps / (sum(e_ms) / 1e3) / 1e6
    peak, src = hbm_peak()
    # ---- dominant kernel: one Dual MM pass over all 32 pairs (the persistent
    # lane-group kernel, one launch per group and label class), CUDA events on
    # the batch stream
    pass_ms = {}
    for which in (0, 1):
        evs = []
        for r in range(3):
            with torch.cuda.stream(st):
                flush.fill_(r & 0xff)
                a, c2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                b.discrete_pass(which)
                c2.record(st)
            evs.append((a, c2))
        torch.cuda.synchronize()
        pass_ms[which] = sum(x.elapsed_time(y) for x, y in evs) / len(evs)
    pass_bytes = {0: 0, 1: 0}
    kernels = set()
    for k, (H, W, L) in enumerate(shapes):
        kernels.add({8: "dmg_batch_kernel", 16: "dmm16_batch_kernel"}.get(
            b.pairs[k].path()[0], "dmm_pass_kernel"))
        pb = survey_pass_bytes(H * W, L)
        pass_bytes[0] += pb[0]
        pass_bytes[1] += pb[1]
    dom = max((0, 1), key=lambda w: pass_ms[w])
    ach = pass_bytes[dom] / (pass_ms[dom] / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(ach, 2), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": None,
                "kernel": "+".join(sorted(kernels)) + (" horizontal" if dom == 0 else " vertical")
                          + " pass over all pairs", "peak_source": src,
                "bytes_rule": "5 B (horizontal) / 4 B (vertical) per pixel-label: int16 duals",
                "bytes_per_launch": pass_bytes[dom],
                "pass_ms": {"horizontal": round(pass_ms[0], 4), "vertical": round(pass_ms[1], 4)}}
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle on the first 24 rows of the batch's first pair
        from oracle import oracle as O
        sp0, (H0, W0, L0) = pairs[0], shapes[0]
        rows = min(24, H0)
        t0 = time.perf_counter()
        O.solve(sp0.left[:rows].copy(), sp0.right[:rows].copy(), L0, NI, NP,
                nthreads=os.cpu_count())
        t_cpu = time.perf_counter() - t0
        cpu = {"value": round(rows * W0 * L0 / t_cpu / 1e6, 4), "unit": "Mpixel·labels/s",
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"rows 0-{rows - 1} of pair 0 ({W0}x{rows}x{L0}), {NI} Dual MM + "
                         f"{NP} PD iterations, {t_cpu:.2f} s"}
    line = {
        "metric": "Mpixel·labels/s (discrete+continuous), 32 mixed pairs in one CUDA graph",
        "value": round(value, 3), "unit": "Mpixel·labels/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(tot_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int16x2+int32+f32", "data": "synthetic",
        "config": {"workload": "batch-32-mixed", "pairs": len(shapes),
                   "sizes": sorted({f"{W}x{H}" for H, W, _ in shapes}),
                   "labels": sorted({L for _, _, L in shapes}),
                   "pixel_labels": units, "dmm_iters": NI, "pd_iters": NP,
                   "l2": "flushed between steps (256 MB write, outside the timed events)"},
        "tuning": {"dmm_ctas_per_sm": choice[0], "pd_tile": f"{choice[1]}x{choice[2]}",
                   "pd_ctas_per_sm": choice[3], "group_budget_mb": choice[4],
                   "tune_seconds": round(tune_s, 2)},
        "single_pair_path_ms": round(single_ms, 4),
        "speedup_over_single_pair_path": round(single_ms / (tot_ms / args.steps), 3),
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 3), "unit": "Mpixel·labels/s",
                "h2d_bytes_per_step": sum(2 * H * W for H, W, _ in shapes),
                "d2h_bytes_per_step": sum(4 * H * W for H, W, _ in shapes)},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# Two views and the consistency check at 1242x375x128
# ---------------------------------------------------------------------------

LR_METRIC = "Mpixel·labels/s (two views + consistency check) at 1242×375×128"
# one launch of the check kernel per pixel: reads the left disparity and the
# mirrored right disparity (2 x 4 B), writes the mask (1 B), the checked
# disparity and the right view's disparity in its own columns (2 x 4 B)
LR_CHECK_BYTES = 17


def run_lr(args):
    import numpy as np
    import torch
    from paper_1601_06274_gb300 import build, dm, synthetic as S
    from oracle import oracle as O
    build.build()
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    dev = torch.device("cuda", 0)
    spec = S.KITTI
    H, W, L = spec["H"], spec["W"], spec["L"]
    NI, NP = spec["dmm_iters"], spec["pd_iters"]
    sp = S.make_workload(spec, seed=0)
    d_left = torch.from_numpy(sp.left).to(dev)
    d_right = torch.from_numpy(sp.right).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lr = dm.StereoLR(H, W, L)
    outs = lr.outputs()
    single = dm.Context(H, W, L)
    d_u1 = torch.empty((H, W), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        lr.solve(d_left, d_right, NI, NP, 1.0, outs)
        single.solve(d_left, d_right, NI, NP, out=d_u1)
    torch.cuda.synchronize()

    def frames(fn, stream):
        evs = []
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(k & 0xff)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                evs.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    # ---- timed region: K two-view frames (the right view on its own stream)
    l0 = lr.left.launch_count() + lr.right.launch_count()
    clk = Clocks(0)
    ms = frames(lambda: lr.solve(d_left, d_right, NI, NP, 1.0, outs), lr.left.stream)
    clocks = clk.stop()
    launches = lr.left.launch_count() + lr.right.launch_count() - l0
    lr.sync()
    tot_ms = sum(ms)
    units = H * W * L
    value = job_value(units, args.steps, 1, tot_ms)
    # the same frames through one view, for the cost of the second view and the check
    ms1 = frames(lambda: single.solve(d_left, d_right, NI, NP, out=d_u1), single.stream)
    single.sync()
    u, ok, ur = outs
    pass_frac = float(ok.float().mean())

    # ---- end to end: pinned host images in, checked disparity and mask out
    h_left = torch.from_numpy(sp.left).pin_memory()
    h_right = torch.from_numpy(sp.right).pin_memory()
    h_u = torch.empty((H, W), dtype=torch.float32).pin_memory()
    h_ok = torch.empty((H, W), dtype=torch.uint8).pin_memory()
    cur = torch.cuda.current_stream(dev)
    e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        uu, oo, _ = lr.solve(h_left, h_right, NI, NP, 1.0, outs)
        h_u.copy_(uu, non_blocking=True)
        h_ok.copy_(oo, non_blocking=True)
        b.record(cur)
        torch.cuda.synchronize()
        e_ms.append(a.elapsed_time(b))
    e2e_value = units * args.steps / (sum(e_ms) / 1e3) / 1e6

    # ---- the check kernel alone (HBM-bound): NB launches over rotating buffers
    # (more than L2 in total) replayed from a CUDA graph, so that neither the
    # host's launch latency nor a warm cache enters the per-launch time
    ul = lr.left.disparity()
    um = lr.right.disparity()
    NB = 24
    bufs = [(ul.clone(), um.clone(), (torch.empty_like(ul), torch.empty_like(ok),
                                      torch.empty_like(ul))) for _ in range(NB)]
    side = torch.cuda.Stream(dev)
    side.wait_stream(cur)
    with torch.cuda.stream(side):
        dm.lr_check(bufs[0][0], bufs[0][1], 1.0, bufs[0][2])
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for a_, m_, o_ in bufs:
            dm.lr_check(a_, m_, 1.0, o_)
    chk = []
    for k in range(max(5, args.steps)):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        graph.replay()
        b.record(cur)
        chk.append((a, b))
    torch.cuda.synchronize()
    chk_ms = sum(a.elapsed_time(b) for a, b in chk) / len(chk) / NB
    peak, src = hbm_peak()
    chk_gbs = LR_CHECK_BYTES * H * W / (chk_ms / 1e3) / 1e9
    avg = time_passes(single, d_left, d_right, NI, max(1, args.steps // 2), flush,
                      single.stream)
    roofline = roofline_line(single, avg, H * W, L, 1, KERNEL_NAMES)
    roofline["check_kernel"] = {"kernel": "lr_check_kernel", "us": round(chk_ms * 1e3, 2),
                                "timing": f"{NB} launches on rotating buffers in one graph",
                                "bytes_per_launch": LR_CHECK_BYTES * H * W,
                                "traffic": NCU_TRAFFIC.get(("lr", "lr_check_kernel",
                                                            source_tag("lr.cu"))),
                                "achieved_gbs": round(chk_gbs, 1),
                                "frac": round(chk_gbs / peak, 4)}

    cpu = None
    if not args.no_cpu_baseline:
        left_c, right_c, _ = cpu_sample()
        O.lib()
        t0 = time.perf_counter()
        O.solve_lr(left_c, right_c, L, NI, NP, nthreads=os.cpu_count())
        t_cpu = time.perf_counter() - t0
        cpu = {"value": round(left_c.shape[0] * W * L / t_cpu / 1e6, 4), "unit": UNIT,
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"rows 0-{CPU_SAMPLE_ROWS - 1} ({W}x{CPU_SAMPLE_ROWS}x{L} crop) of the "
                         f"frame, both views ({NI} Dual MM + {NP} PD iterations each) and the "
                         f"check, {t_cpu:.2f} s"}

    line = {
        "metric": LR_METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
        "config": {"workload": "lr-1242x375x128", "H": H, "W": W, "L": L, "dmm_iters": NI,
                   "pd_iters": NP, "max_diff": 1.0, "streams": 2,
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "parallelism": "replicas1"},
        "single_view_ms": round(sum(ms1) / len(ms1), 4),
        "two_view_over_single": round((tot_ms / args.steps) / (sum(ms1) / len(ms1)), 3),
        "pass_fraction": round(pass_frac, 4),
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 2 * H * W,
                "d2h_bytes_per_step": 5 * H * W},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Chain minorants compared: lower bound per Dual MM iteration and time
# ---------------------------------------------------------------------------

MIN_METRIC = "Mpixel·labels/s (10 Dual MM iterations, iterative minorant) at 1242×375×128"
# the alternative minorants' kernel at 128 labels (a multiple of 16: the staged form)
ALT_KERNEL = "dmm_alt_staged_kernel"


def run_minorants(args):
    """The comparison of Sec. 2.3 / App. A (hierarchical, naive and iterative
    minorants: lower bound after each Dual MM iteration) on the synthetic frame,
    with each variant's time per iteration.  One step = 10 Dual MM iterations
    with the iterative minorant (max_pass 3, gamma 1/4)."""
    import torch
    from paper_1601_06274_gb300 import build, dm, synthetic as S
    build.build()
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    dev = torch.device("cuda", 0)
    spec = S.KITTI
    H, W, L = spec["H"], spec["W"], spec["L"]
    NI = spec["dmm_iters"]
    sp = S.make_workload(spec, seed=0)
    d_left = torch.from_numpy(sp.left).to(dev)
    d_right = torch.from_numpy(sp.right).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    results = {}
    ctxs = {}
    for kind in ("hier", "naive", "iterative"):
        ctx = dm.Context(H, W, L)
        ctx.set_minorant(kind)
        ctx.cost_volume(d_left, d_right)
        lb = ctx.discrete(NI, lower_bounds=True)
        ctxs[kind] = ctx
        avg = time_passes(ctx, d_left, d_right, 1, 2, flush, ctx.stream)
        results[kind] = {"lower_bound_per_iteration": [int(v) for v in lb],
                         "pass_ms": {"horizontal": round(avg[0], 4),
                                     "vertical": round(avg[1], 4)},
                         "kernel": KERNEL_NAMES[ctx.path()[0]] if kind == "hier" else
                                   ALT_KERNEL}
    # ---- timed region: K solves of 10 iterations with the iterative minorant
    ctx = ctxs["iterative"]
    for _ in range(args.warmup):
        ctx.cost_volume(d_left, d_right)
        ctx.discrete(NI)
    torch.cuda.synchronize()
    evs = []
    l0 = ctx.launch_count()
    clk = Clocks(0)
    for k in range(args.steps):
        ctx.cost_volume(d_left, d_right)
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(ctx.stream)
        ctx.discrete(NI)
        b.record(ctx.stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = ctx.launch_count() - l0 - 3 * args.steps   # less the cost-volume launches
    ctx.sync()
    ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(ms)
    units = H * W * L
    value = job_value(units, args.steps, 1, tot_ms)
    for kind in ("hier", "naive"):
        c2 = ctxs[kind]
        c2.cost_volume(d_left, d_right)
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(c2.stream)
        c2.discrete(NI)
        b.record(c2.stream)
        torch.cuda.synchronize()
        results[kind]["ms_per_solve"] = round(a.elapsed_time(b), 4)
    results["iterative"]["ms_per_solve"] = round(tot_ms / args.steps, 4)
    # ---- end to end: pinned host images in, the labels back
    h_left = torch.from_numpy(sp.left).pin_memory()
    h_right = torch.from_numpy(sp.right).pin_memory()
    h_lab = torch.empty((H, W), dtype=torch.int16).pin_memory()
    e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(ctx.stream)
        ctx.cost_volume(h_left, h_right)
        ctx.discrete(NI)
        h_lab.copy_(ctx.labels(), non_blocking=True)
        b.record(ctx.stream)
        torch.cuda.synchronize()
        e_ms.append(a.elapsed_time(b))
    e2e_value = units * args.steps / (sum(e_ms) / 1e3) / 1e6
    peak, src = hbm_peak()
    pm = results["iterative"]["pass_ms"]
    bytes_per = dmm_pass_bytes(32, 4, 1, H * W, L)
    dom = 0 if pm["horizontal"] >= pm["vertical"] else 1
    dur = pm["horizontal"] if dom == 0 else pm["vertical"]
    achieved = bytes_per[dom] / (dur / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": ALT_KERNEL + " " + ("horizontal" if dom == 0 else "vertical") + " pass",
                "peak_source": src, "bytes_per_launch": bytes_per[dom]}
    roofline["traffic"] = NCU_TRAFFIC.get(("minorants", roofline["kernel"], source_tag("dmm.cu")))

    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        rows = 8
        cost = O.cost_volume(sp.left[:rows].copy(), sp.right[:rows].copy(), L)
        wh, wv = O.edge_weights(sp.left[:rows].copy())
        t0 = time.perf_counter()
        O.dmm(cost, wh, wv, NI, nthreads=os.cpu_count(), minorant="iterative")
        t_cpu = time.perf_counter() - t0
        cpu = {"value": round(rows * W * L / t_cpu / 1e6, 4), "unit": UNIT,
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"rows 0-{rows - 1} ({W}x{rows}x{L} crop), {NI} Dual MM iterations "
                         f"with the iterative minorant, {t_cpu:.2f} s"}
    line = {
        "metric": MIN_METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "minorants-1242x375x128", "H": H, "W": W, "L": L,
                   "dmm_iters": NI, "iterative": {"max_pass": 3, "gamma": "1/4"},
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "parallelism": "replicas1"},
        "minorants": results, "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 2 * H * W,
                "d2h_bytes_per_step": 2 * H * W,
                "includes": "census and cost volume, 10 Dual MM iterations, labels"},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Optical flow: 640x480, displacements in [-32, 32)^2
# ---------------------------------------------------------------------------

FLOW_METRIC = "Mpixel·labels/s (optical flow, 64×64 displacements) at 640×480"


def run_flow(args):
    """One step = one flow: census and the two decoupled cost volumes, 10 Dual MM
    iterations on each layer (the two layers on two streams), 100 primal-dual
    iterations of the two-component refinement.  The metric counts the K1 x K2
    displacements searched per pixel."""
    import numpy as np
    import torch
    from paper_1601_06274_gb300 import build, dm, synthetic as S
    build.build()
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    dev = torch.device("cuda", 0)
    spec = S.FLOW
    H, W = spec["H"], spec["W"]
    lo1, K1, lo2, K2 = spec["lo1"], spec["K1"], spec["lo2"], spec["K2"]
    NI, NP = spec["dmm_iters"], spec["pd_iters"]
    fp = S.make_flow_workload(spec, seed=0)
    d1_img = torch.from_numpy(fp.img1).to(dev)
    d2_img = torch.from_numpy(fp.img2).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    f = dm.Flow(H, W, lo1, K1, lo2, K2)
    outs = (torch.empty((H, W), dtype=torch.float32, device=dev),
            torch.empty((H, W), dtype=torch.float32, device=dev))
    for _ in range(args.warmup):
        f.solve(d1_img, d2_img, NI, NP, outs)
    torch.cuda.synchronize()
    st = f.layer1.stream
    l0 = f.layer1.launch_count() + f.layer2.launch_count()
    clk = Clocks(0)
    evs = []
    with torch.cuda.stream(st):
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            f.solve(d1_img, d2_img, NI, NP, outs)
            b.record(st)
            evs.append((a, b))
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = f.layer1.launch_count() + f.layer2.launch_count() - l0
    f.sync()
    ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(ms)
    units = H * W * K1 * K2
    value = job_value(units, args.steps, 1, tot_ms)
    # ---- end to end: pinned host frames in, both displacement fields back
    h1 = torch.from_numpy(fp.img1).pin_memory()
    h2 = torch.from_numpy(fp.img2).pin_memory()
    hd1 = torch.empty((H, W), dtype=torch.float32).pin_memory()
    hd2 = torch.empty((H, W), dtype=torch.float32).pin_memory()
    e_ms = []
    with torch.cuda.stream(st):
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            o1, o2 = f.solve(h1, h2, NI, NP, outs)
            hd1.copy_(o1, non_blocking=True)
            hd2.copy_(o2, non_blocking=True)
            b.record(st)
            torch.cuda.synchronize()
            e_ms.append(a.elapsed_time(b))
    e2e_value = units * args.steps / (sum(e_ms) / 1e3) / 1e6
    d1, d2 = outs
    inner = np.s_[40:H - 40, 40:W - 40]
    acc = float(np.mean((np.abs(d1.cpu().numpy() - fp.gt1) < 1.0)[inner] &
                        (np.abs(d2.cpu().numpy() - fp.gt2) < 1.0)[inner]))

    # ---- stages, one at a time on the first layer's stream
    def timed(fn, reps=3):
        out = []
        for r in range(reps):
            flush.fill_(r & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            out.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in out) / len(out)

    with torch.cuda.stream(st):
        cost_ms = timed(lambda: f.cost_volumes(d1_img, d2_img))
        passes = {0: [], 1: []}
        for it in range(2):
            for which in (0, 1):
                passes[which].append(timed(lambda: f.layer1.discrete_pass(which), 1))
        f.cost_volumes(d1_img, d2_img)
        f.discrete(NI)
        refine_ms = timed(lambda: f.refine(NP, outs))
    avg = {w: sum(v) / len(v) for w, v in passes.items()}
    roofline = roofline_line(f.layer1, avg, H * W, K1, 1, KERNEL_NAMES)
    # the decoupled-cost kernel is bound by the integer ALU pipe: its utilisation
    # from the ncu capture of this kernel as built now
    roofline["flow_cost_kernel"] = {"bound": "alu", "sm__pipe_alu_cycles_active_pct": 83.0,
                                    "source": "ncu capture of flow_cost_kernel at 640x480, 64x64"}
    roofline["stage_ms"] = {"census_and_cost_volumes": round(cost_ms, 4),
                            "dual_mm_pass_layer1": {"horizontal": round(avg[0], 4),
                                                    "vertical": round(avg[1], 4)},
                            "refinement_100_iterations": round(refine_ms, 4)}

    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        rows = 12
        t0 = time.perf_counter()
        O.solve_flow(fp.img1[:rows].copy(), fp.img2[:rows].copy(), lo1, K1, lo2, K2, NI, NP,
                     nthreads=os.cpu_count())
        t_cpu = time.perf_counter() - t0
        cpu = {"value": round(rows * W * K1 * K2 / t_cpu / 1e6, 4), "unit": UNIT,
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"rows 0-{rows - 1} of both frames ({W}x{rows}, {K1}x{K2} "
                         f"displacements), the whole flow path, {t_cpu:.2f} s"}
    line = {
        "metric": FLOW_METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
        "config": {"workload": "flow-640x480x64x64", "H": H, "W": W, "d1": [lo1, lo1 + K1 - 1],
                   "d2": [lo2, lo2 + K2 - 1], "dmm_iters": NI, "pd_iters": NP,
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "parallelism": "replicas1"},
        "accuracy_within_1px": round(acc, 4),
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 2 * H * W,
                "d2h_bytes_per_step": 8 * H * W},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "diff":
        run_diff(args)
        return
    if args.workload == "stream":
        run_stream(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "lr":
        run_lr(args)
        return
    if args.workload == "minorants":
        run_minorants(args)
        return
    if args.workload == "flow":
        run_flow(args)
        return
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as distd
        torch.cuda.set_device(local)
        distd.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1601_06274_gb300 import build, dm, synthetic as S
    build.build()
    spec = S.KITTI
    H, W, L = spec["H"], spec["W"], spec["L"]
    NI, NP = spec["dmm_iters"], spec["pd_iters"]
    sp = S.make_workload(spec, seed=rank)
    ctx = dm.Context(H, W, L, device=str(dev))
    stream = ctx.stream
    d_left = torch.from_numpy(sp.left).to(dev)
    d_right = torch.from_numpy(sp.right).to(dev)
    d_u = torch.empty((H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        ctx.solve(d_left, d_right, NI, NP, out=d_u)
    torch.cuda.synchronize()

    # ---- timed region: K frames, events per frame, L2 flushed between frames
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    launches0 = ctx.launch_count()
    barrier()
    torch.cuda.synchronize()
    clk = Clocks(dev.index or 0)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            evs[k][0].record(stream)
            ctx.solve(d_left, d_right, NI, NP, out=d_u)
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    launches = ctx.launch_count() - launches0
    ctx.sync()
    ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = max_over_ranks(sum(ms), ws, dev)
    units = H * W * L
    value = job_value(units, args.steps, ws, tot_ms)

    # ---- end to end through the C ABI with pinned host buffers
    h_left = torch.from_numpy(sp.left).pin_memory()
    h_right = torch.from_numpy(sp.right).pin_memory()
    h_u = torch.empty((H, W), dtype=torch.float32).pin_memory()
    ctx.solve_host(h_left, h_right, NI, NP, h_u)
    e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.solve_host(h_left, h_right, NI, NP, h_u)
        b.record(stream)
        torch.cuda.synchronize()
        e_ms.append(a.elapsed_time(b))
    e2e_value = units * args.steps * ws / (sum(e_ms) / 1e3) / 1e6

    # ---- the same frame replayed from a CUDA graph of the whole solve
    gctx = dm.Context(H, W, L, device=str(dev), stream=torch.cuda.Stream(dev))
    gctx.solve(d_left, d_right, NI, NP)
    g_u = torch.empty((H, W), dtype=torch.float32, device=dev)
    gctx.capture(d_left, d_right, NI, NP, g_u)
    gctx.replay()
    torch.cuda.synchronize()
    g_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(gctx.stream)
        gctx.replay()
        b.record(gctx.stream)
        torch.cuda.synchronize()
        g_ms.append(a.elapsed_time(b))
    graph_ms = sum(g_ms) / len(g_ms)
    gctx.sync()

    # ---- dominant kernel: one Dual MM pass per launch, CUDA events on the ctx stream
    avg = time_passes(ctx, d_left, d_right, NI, max(1, args.steps // 2), flush, stream)
    roofline = roofline_line(ctx, avg, H * W, L, 1, KERNEL_NAMES)
    peak = roofline["peak"]
    frame_bytes = survey_frame_bytes(H * W, L, 1, NI, NP, 5)
    roofline["frame_bytes"] = frame_bytes
    roofline["frame_frac"] = round(frame_bytes / (tot_ms / args.steps / 1e3) / 1e9 / peak, 4)
    roofline["stage_ms"] = time_stages(ctx, d_left, d_right, NI, NP, flush, stream)
    roofline["refinement_kernel"] = refinement_issue(roofline["stage_ms"]["refinement"], NP)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        left_c, right_c, _ = cpu_sample()
        t_cpu = time_oracle(left_c, right_c, spec)
        cpu = {"value": round(left_c.shape[0] * W * L / t_cpu / 1e6, 4), "unit": UNIT,
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"rows 0-{CPU_SAMPLE_ROWS - 1} ({W}x{CPU_SAMPLE_ROWS}x{L} crop) of the "
                         f"frame, {NI} Dual MM + {NP} PD iterations, {t_cpu:.2f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
            "config": {"workload": "kitti-1242x375x128", "H": H, "W": W, "L": L,
                       "dmm_iters": NI, "pd_iters": NP, "warps": 5,
                       "l2": "flushed between steps (256 MB write, outside the timed events)",
                       "parallelism": f"replicas{ws}"},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 2 * H * W,
                    "d2h_bytes_per_step": 4 * H * W},
            "graph_replay_ms_per_step": round(graph_ms, 4),
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
