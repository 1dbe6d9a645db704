"""Benchmark: FOEED inpainting throughput on one GB300 (pixel-updates/s, % HBM roofline).

A step is one complete FOEED inpainting solve of the 2048 x 2048 FP32 phantom
workload (3% mask, sigma 1.5, lambda 0.02, 100 FSI cycles of length 40, cycle
residual every cycle), i.e. every row of the hot path: pre-smoothing, tensor,
Hessian, outer divergence, masked FSI update, residual reduction, cycle driver.
pixel-updates = w * h * cycles * cycle_len per solve, known pixels included.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 (torchrun): every rank solves its own copy of the workload (independent
problems, no collective on the data path); value = all ranks' pixel-updates /
the slowest rank's time ("weak" scaling).
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample (one FSI cycle of the same image) with the same metric.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pixel-updates/s (FOEED FSI solve, 2048x2048 FP32)"
UNIT = "pixel-updates/s"
BYTES_PER_PIXEL_UPDATE = 13  # u^k, u^{k-1}, u^{k+1} in float + uint8 mask
WORKLOAD = 3

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
# of the dominant kernel on the full 2048x2048 workload, and the hash of the
# kernel source it was taken on; reported only while the source is unchanged.
NCU_TRAFFIC = {"source_sha1": "ae657531a038fd4f6fb6f8bd2597053c49cd13c1",
               "bytes_per_launch": 37793536 + 32000}  # from the ncu capture summary of this kernel


def kernel_source_sha1():
    h = hashlib.sha1()
    for fn in ("step_fast.cuh", "foeed_device.cuh", "dispatch.h"):
        with open(os.path.join(ROOT, "paper_2006_10406_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def instance_for_rank(rank: int) -> int:
    """Each rank solves its own independent instance of the workload (seeded by rank)."""
    return rank


def max_over_ranks(value: float, pg, device) -> float:
    """Slowest rank's value (all ranks must call it); identity without a process group."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reference_arm(args, world, rank):
    """FP64 CPU oracle on the host cores: each step is one FSI cycle of the workload."""
    import numpy as np
    import oracle as O
    import synth
    if rank != 0:
        return
    img, mask, p = synth.workload(WORKLOAD)
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    f = img.astype(np.float32).astype(np.float64)
    n = p["cycle_len"]
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.inpaint(0, f, mask, p["sigma"], p["lam"], n, 1)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    per = sum(times) / len(times)
    pu = img.size * n
    value = pu / per
    sample = f"one FSI cycle ({n} FOEED steps) of the {p['w']}x{p['h']} phantom per step, FP64"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": p["name"], "w": p["w"], "h": p["h"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline_leg(p, img, mask, gpu_results=None):
    """The oracle as it stands, on all host cores: a bounded timed sample (five FSI
    cycles of the same image, about ten seconds) and one cycle of length 4 on one
    core. With gpu_results ({name: FP32/FP64 result as a numpy array}), the same
    oracle then runs the whole benchmarked solve (100 cycles of 40, untimed, a few
    minutes) as the reference every GPU result is compared with."""
    import numpy as np
    import oracle as O
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    f = img.astype(np.float32).astype(np.float64)
    n, sample_cycles = p["cycle_len"], 5
    t0 = time.perf_counter()
    O.inpaint(0, f, mask, p["sigma"], p["lam"], n, sample_cycles)
    dt = time.perf_counter() - t0
    # the same oracle on one thread, a shorter sample (one FSI cycle of length 4)
    O.set_threads(1)
    t1 = time.perf_counter()
    O.inpaint(0, f, mask, p["sigma"], p["lam"], 4, 1)
    dt1 = time.perf_counter() - t1
    O.set_threads(cores)
    out = {"value": img.size * n * sample_cycles / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{sample_cycles} FSI cycles ({sample_cycles * n} FOEED steps, FP64) of the {p['w']}x{p['h']} "
                     f"phantom, {dt:.1f} s",
           "single_thread": {"value": img.size * 4 / dt1, "unit": UNIT, "cores": 1,
                             "sample": f"one FSI cycle of 4 steps of the same image, {dt1:.1f} s"}}
    if gpu_results:
        t2 = time.perf_counter()
        ref, st, info = O.inpaint(0, f, mask, p["sigma"], p["lam"], n, p["max_cycles"])
        dt2 = time.perf_counter() - t2

        def psnr(u):
            mse = float(np.mean((u - img) ** 2))
            return float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)

        acc = {"oracle_cycles": info["cycles"], "oracle_s": dt2, "psnr_oracle_db": psnr(ref)}
        for name, u in gpu_results.items():
            u = u.astype(np.float64)
            acc[f"max_abs_{name}_vs_oracle"] = float(np.max(np.abs(u - ref)))
            acc[f"psnr_delta_{name}_vs_oracle_db"] = abs(psnr(u) - psnr(ref))
        out["oracle_reference"] = acc
    return out


def batched_leg(fg, synth, torch, dev, stream):
    """W4: 256 piecewise-smooth images of uneven sizes (sides 128..1024, square and
    2:1, mask density 2-10%, lambda 0.01-0.1), sigma 1, 50 FSI cycles of length 25,
    solved in one launch per step over all tiles, against solving them one by one."""
    import numpy as np
    cases = synth.batched_workload(256)
    imgs = [torch.from_numpy(c[0].astype(np.float32)).to(dev) for c in cases]
    masks = [torch.from_numpy(c[1]).to(dev) for c in cases]
    lams = [float(c[2]) for c in cases]
    n, cycles = 25, 50
    pixels = sum(int(im.numel()) for im in imgs)
    pu = pixels * n * cycles
    fg.set_tile_policy("auto")
    fg.foeed_inpaint_batch(imgs, masks, lams, 1.0, n, 1)  # warm-up: the autotuner times the tile plans here
    plan = fg.last_tile_plan()
    ws = torch.empty(fg.workspace_bytes(1024, 1024, fg.F32), dtype=torch.uint8, device=dev)

    def timed_batch(reps=2):
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            res, _ = fg.foeed_inpaint_batch(imgs, masks, lams, 1.0, n, cycles, stream=stream)
            b.record(stream)
            torch.cuda.synchronize(dev)
            times.append(a.elapsed_time(b))
        return res, min(times)

    outs, ms = timed_batch()
    # the same batch with 64 x 32 tiles for every image (the plan without the autotuner)
    fg.set_tile_policy("h32")
    outs32, ms32 = timed_batch()
    fg.set_tile_policy("auto")
    same_bits = all(bool(torch.equal(x, y)) for x, y in zip(outs, outs32))
    # warm the single-image path once per distinct image size (the autotuner's
    # choice is cached per size), then solve the images one by one; each call
    # captures its own cycle graph (lambda differs per image), as a caller's would
    seen = set()
    for f, m, lam in zip(imgs, masks, lams):
        if tuple(f.shape) not in seen:
            seen.add(tuple(f.shape))
            fg.foeed_inpaint(f, m, lam, 1.0, n, 1, workspace=ws)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    refs = []
    for f, m, lam in zip(imgs, masks, lams):
        ref, _ = fg.foeed_inpaint(f, m, lam, 1.0, n, cycles, workspace=ws, stream=stream)
        refs.append(ref)
    b.record(stream)
    torch.cuda.synchronize(dev)
    seq_ms = a.elapsed_time(b)
    diff = max(float((ref - u).abs().max().item()) for ref, u in zip(refs, outs))
    return {"value": pu / (ms / 1e3), "unit": UNIT, "images": len(imgs), "pixels": pixels, "ms_per_solve": ms,
            "tile_plan": {"images_on_64x16_tiles": plan["images_h16"], "tuned": bool(plan["tuned"]),
                          "us_per_step_all_64x32": plan["us_h32"], "us_per_step_all_64x16": plan["us_h16"],
                          "us_per_step_chosen": plan["us_chosen"]},
            "fixed_64x32_value": pu / (ms32 / 1e3), "fixed_64x32_ms": ms32,
            "autotuned_equals_fixed_bitwise": same_bits,
            "one_by_one_value": pu / (seq_ms / 1e3), "one_by_one_ms": seq_ms,
            "max_abs_diff_vs_one_by_one": diff, "fsi_cycles": cycles, "cycle_len": n}


def convergence_leg(fg, synth, torch, dev, stream):
    """W2 (512 x 512 polygons, 4% mask): FOEED and EED solved until the relative
    change of a cycle falls below 1e-6 (at most 20000 cycles), FP32."""
    import numpy as np
    img, mask, p = synth.workload(2)
    f = torch.from_numpy(img.astype(np.float32)).to(dev)
    m = torch.from_numpy(mask).to(dev)
    imgd = torch.from_numpy(img).to(dev)
    out = {}
    for name, solve in (("foeed", fg.foeed_inpaint), ("eed", fg.eed_inpaint)):
        solve(f, m, p["lam"], p["sigma"], p["cycle_len"], 2, stream=stream)  # capture
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        u, rep = solve(f, m, p["lam"], p["sigma"], p["cycle_len"], p["max_cycles"], tol=p["tol"], stream=stream,
                       raise_on_status=False)
        b.record(stream)
        torch.cuda.synchronize(dev)
        mse, aae, psnr = fg.foeed_errors(u.double(), imgd)
        out[name] = {"converged": rep.converged, "cycles": rep.cycles_run, "last_rel_change": rep.last_rel_change,
                     "ms": a.elapsed_time(b), "psnr_db": psnr, "mse": mse}
    return {"workload": p["name"], "tol": p["tol"], "cycle_len": p["cycle_len"], **out}


def gradient_once(fg, synth, torch, dev, rank, checkpoint_every=16):
    """One warm-up and one timed gradient of the W5 workload (a checkpoint every
    `checkpoint_every` steps; 1 keeps every state)."""
    import numpy as np
    img, mask, p = synth.workload(5)
    f = torch.from_numpy(img.astype(np.float32)).to(dev)
    m = torch.from_numpy(mask).to(dev)
    g = torch.full_like(f, 1e-3)
    args = (f, m, g, p["lam"], p["sigma"], p["cycle_len"], p["max_cycles"])
    fg.foeed_inpaint_vjp(*args, checkpoint_every=checkpoint_every)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    gf, _ = fg.foeed_inpaint_vjp(*args, checkpoint_every=checkpoint_every)
    b.record()
    torch.cuda.synchronize(dev)
    if rank == 0:
        print(json.dumps({"gradient_ms": a.elapsed_time(b), "workload": p["name"], "checkpoint_every": checkpoint_every,
                          "grad_norm": float(gf.norm())}), flush=True)


def batch_once(fg, synth, torch, dev, rank, tile_policy="auto"):
    """One warm-up (one FSI cycle) and one timed solve (two cycles of 25 steps) of
    the W4 batch of 256 images, for profiler launch lists of the batched step."""
    import numpy as np
    cases = synth.batched_workload(256)
    imgs = [torch.from_numpy(c[0].astype(np.float32)).to(dev) for c in cases]
    masks = [torch.from_numpy(c[1]).to(dev) for c in cases]
    lams = [float(c[2]) for c in cases]
    fg.set_tile_policy(tile_policy)
    fg.foeed_inpaint_batch(imgs, masks, lams, 1.0, 25, 1)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fg.foeed_inpaint_batch(imgs, masks, lams, 1.0, 25, 2)
    b.record()
    torch.cuda.synchronize(dev)
    if rank == 0:
        pixels = sum(int(im.numel()) for im in imgs)
        ms = a.elapsed_time(b)
        print(json.dumps({"batch_ms": ms, "images": len(imgs), "pixels": pixels, "steps": 50,
                          "pixel_updates_per_s": pixels * 50 / (ms / 1e3), "tile_plan": fg.last_tile_plan()}),
              flush=True)


def adjoint_leg(fg, synth, torch, dev, stream):
    """W5 tonal optimisation: 1024 x 1024 FP32, 4% mask, 30 FSI cycles of length 20
    unrolled; 20 Adam steps on the stored grey values with the gradient of the
    reconstruction MSE from the hand-written adjoint (checkpoint every 16 steps)."""
    import numpy as np
    img, mask, p = synth.workload(5)
    n, cycles = p["cycle_len"], p["max_cycles"]
    target = torch.from_numpy(img.astype(np.float32)).to(dev)
    md = torch.from_numpy(mask).to(dev)
    known = md.bool()
    f = target.clone().requires_grad_(True)
    opt = torch.optim.Adam([f], lr=2e-3)
    mse = []
    ev = []
    for it in range(21):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        u = fg.foeed_inpaint_diff(f, md, p["lam"], p["sigma"], n, cycles, checkpoint_every=16)
        loss = ((u - target) ** 2).mean()
        if it < 20:
            opt.zero_grad()
            loss.backward()
        b.record(stream)
        torch.cuda.synchronize(dev)
        mse.append(float(loss.item()))
        if it < 20:
            ev.append(a.elapsed_time(b))
            opt.step()
            with torch.no_grad():
                f.clamp_(0.0, 1.0)
    steps = n * cycles
    # one gradient alone, checkpoint every 16 steps (recomputed segments) and every step (all states kept)
    grad_ms = {}
    g = torch.ones_like(target) * 1e-3
    for k in (16, 1):
        fg.foeed_inpaint_vjp(target, md, g, p["lam"], p["sigma"], n, cycles, checkpoint_every=k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fg.foeed_inpaint_vjp(target, md, g, p["lam"], p["sigma"], n, cycles, checkpoint_every=k)
        b.record(stream)
        torch.cuda.synchronize(dev)
        grad_ms[f"checkpoint_every_{k}"] = a.elapsed_time(b)
    # the plain single-image FP32 solve of the same workload (same steps), for comparison
    solve_ms = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fg.foeed_inpaint(target, md, p["lam"], p["sigma"], n, cycles, stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        solve_ms.append(a.elapsed_time(b))
    plain = min(solve_ms)
    return {"iterations": 20, "mse_start": mse[0], "mse_end": mse[-1], "gradient_ms": grad_ms,
            "plain_solve_ms": plain,
            "gradient_over_plain_solve": {k: v / plain for k, v in grad_ms.items()},
            "mse_drop_pct": 100.0 * (mse[0] - mse[-1]) / mse[0],
            "psnr_start_db": float(10 * np.log10(1.0 / mse[0])), "psnr_end_db": float(10 * np.log10(1.0 / mse[-1])),
            "ms_per_iteration": float(np.median(ev)), "unrolled_steps": steps, "checkpoint_every": 16,
            "forward_backward_pixel_steps_per_s": 2 * img.size * steps / (float(np.median(ev)) / 1e3)}


def time_to_mse(fg, solve_one_cycle, imgd, cycles, ms_per_cycle, u_final):
    """Cycles (and device time) until the MSE against the ground truth is within 1% of
    the MSE after all `cycles` cycles. Each FSI cycle restarts from its first iterate,
    so one-cycle solves started from the previous result retrace the full solve
    exactly; the last one is checked against the full solve's output."""
    u, mses = None, []
    for _ in range(cycles):
        u = solve_one_cycle(u)
        mses.append(fg.foeed_errors(u.double(), imgd)[0])
    final = mses[-1]
    m = next(i for i, v in enumerate(mses) if v <= 1.01 * final) + 1
    return {"cycles_to_within_1pct": m, "ms_to_within_1pct": m * ms_per_cycle, "final_mse": final,
            "trajectory_equals_solve": bool((u == u_final).all().item())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-convergence", action="store_true")
    ap.add_argument("--tile-policy", default="auto", choices=["auto", "h32", "h16", "h64", "h8"],
                    help="tile shape of the FP32 step kernel: timed once and kept (auto), or fixed; a fixed "
                         "shape keeps profiler runs, whose serialised launches distort the timing, on the "
                         "shape the benchmark uses")
    ap.add_argument("--minimal", action="store_true",
                    help="only the warm-up and timed solves (for profiler launch lists)")
    ap.add_argument("--checkpoint-every", type=int, default=16,
                    help="checkpoint interval of --gradient-only (1: every state kept, nothing recomputed)")
    ap.add_argument("--gradient-only", action="store_true",
                    help="only one warm-up and one timed gradient of the 1024^2 tonal-optimisation "
                         "workload (for profiler launch lists of the backward kernels)")
    ap.add_argument("--batched-only", action="store_true",
                    help="only one warm-up and one timed two-cycle solve of the 256-image batch "
                         "(for profiler launch lists of the batched step kernel)")
    args = ap.parse_args()
    world, rank, local = dist_setup()

    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import numpy as np
    import torch

    import paper_2006_10406_gb300 as fg
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.gradient_only:
        return gradient_once(fg, synth, torch, dev, rank, args.checkpoint_every)
    if args.batched_only:
        return batch_once(fg, synth, torch, dev, rank, args.tile_policy)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    img, mask, p = synth.workload(WORKLOAD, instance=instance_for_rank(rank))
    W, H, n, cycles = p["w"], p["h"], p["cycle_len"], p["max_cycles"]
    f32 = img.astype(np.float32)
    fd = torch.from_numpy(f32).to(dev)
    md = torch.from_numpy(mask).to(dev)
    ws = torch.empty(fg.workspace_bytes(W, H, fg.F32), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # 2x the 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def solve():
        return fg.foeed_inpaint(fd, md, p["lam"], p["sigma"], n, cycles, workspace=ws, stream=stream)

    fg.set_tile_policy(args.tile_policy)
    tile_plan = None
    for _ in range(args.warmup):
        solve()
        if tile_plan is None:  # the first solve of this size times the tile shapes
            tile_plan = fg.last_tile_plan()
    torch.cuda.synchronize(dev)

    # ---- timed region: K device-resident solves, L2 flushed between them ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            u, rep = solve()
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_total = max_over_ranks(sum(ms), pg, dev)
    ms_per_step = ms_total / args.steps
    pu_per_solve = W * H * cycles * n
    value = pu_per_solve * world / (ms_per_step / 1e3)
    launches_per_solve = 2 + cycles * n + 1
    clocks = clk.summary()

    if args.minimal:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                              "minimal": True}), flush=True)
        if pg:
            pg.destroy_process_group()
        return

    # ---- end to end: host buffers, copies inside the timed region ----
    fh = torch.from_numpy(f32).pin_memory()
    mh = torch.from_numpy(mask).pin_memory()
    uh = torch.empty((H, W), dtype=torch.float32).pin_memory()
    e2e_ms = []
    for i in range(max(2, args.steps // 2)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fd.copy_(fh, non_blocking=True)
        md.copy_(mh, non_blocking=True)
        u, rep = solve()
        uh.copy_(u, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms.append(a.elapsed_time(b))
    e2e_per = sum(e2e_ms) / len(e2e_ms)
    e2e = {"value": pu_per_solve * world / (e2e_per / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": fh.numel() * 4 + mh.numel(), "d2h_bytes_per_step": uh.numel() * 4}

    # ---- roofline of the dominant kernel (fused FOEED step, FP32, R = 5) ----
    peak, peak_kind = measured_peak()
    step_launch_s = (ms_per_step / 1e3) / (cycles * n)  # every step launch of the solve, gaps included
    achieved = BYTES_PER_PIXEL_UPDATE * W * H / step_launch_s / 1e9
    traffic = NCU_TRAFFIC["bytes_per_launch"] if NCU_TRAFFIC["source_sha1"] == kernel_source_sha1() else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "fsi_step_fast<R=5, FOEED, float>",
                "algorithmic_bytes_per_launch": BYTES_PER_PIXEL_UPDATE * W * H}

    extra = {}
    gpu_results = None
    if rank == 0:
        # EED comparison path on the same workload (tau 0.25)
        eed_ms = []
        for i in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fg.eed_inpaint(fd, md, p["lam"], p["sigma"], n, cycles, workspace=ws, stream=stream)
            b.record(stream)
            torch.cuda.synchronize(dev)
            eed_ms.append(a.elapsed_time(b))
        extra["eed"] = {"value": pu_per_solve / (min(eed_ms[1:]) / 1e3), "unit": UNIT,
                        "ms_per_solve": min(eed_ms[1:])}
        if not args.no_accuracy:
            def timed(fn):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                out = fn()
                b.record(stream)
                torch.cuda.synchronize(dev)
                return out[0].clone(), a.elapsed_time(b)

            u32, _ = solve()
            u32 = u32.clone()
            ws64 = torch.empty(fg.workspace_bytes(W, H, fg.F64), dtype=torch.uint8, device=dev)
            fd64 = fd.double()
            fg.foeed_inpaint(fd64, md, p["lam"], p["sigma"], n, 1, workspace=ws64, stream=stream)  # capture
            u64, ms64 = timed(lambda: fg.foeed_inpaint(fd64, md, p["lam"], p["sigma"], n, cycles, workspace=ws64,
                                                       stream=stream))
            fg.foeed_inpaint(fd, md, p["lam"], p["sigma"], n, 1, dtype="f32_f64u", workspace=ws, stream=stream)
            umx, msmx = timed(lambda: fg.foeed_inpaint(fd, md, p["lam"], p["sigma"], n, cycles, dtype="f32_f64u",
                                                       workspace=ws, stream=stream))
            imgd = torch.from_numpy(img).to(dev)
            m32 = fg.foeed_errors(u32.double(), imgd)
            m64 = fg.foeed_errors(u64, imgd)
            mmx = fg.foeed_errors(umx.double(), imgd)
            diff = float((u32.double() - u64).abs().max().item())
            extra["accuracy"] = {"max_abs_f32_vs_f64_gpu": diff, "psnr_f32_db": m32[2], "psnr_f64_db": m64[2],
                                 "psnr_delta_db": abs(m32[2] - m64[2]), "mse_f32": m32[0], "mse_f64": m64[0]}
            gpu_results = {"f32": u32.cpu().numpy(), "f64_gpu": u64.cpu().numpy(),
                           "f32_f64u": umx.cpu().numpy()}
            # the other arithmetic modes of the same solve (the FP64 GPU solve is the parity-tested reference)
            extra["precisions"] = {
                "f64": {"value": pu_per_solve / (ms64 / 1e3), "unit": UNIT, "ms_per_solve": ms64},
                "f32_storage_two_float_update": {
                    "value": pu_per_solve / (msmx / 1e3), "unit": UNIT, "ms_per_solve": msmx,
                    "update": "FSI update in two-float arithmetic (pairs of floats), rounded to float once",
                    "max_abs_vs_f64_gpu": float((umx.double() - u64).abs().max().item()),
                    "psnr_db": mmx[2], "psnr_delta_vs_f64_db": abs(mmx[2] - m64[2])}}
            del ws64, fd64
            # time to within 1% of the final MSE, FOEED against EED (same workload, FP32)
            def one(method):
                def run(u0):
                    return method(fd, md, p["lam"], p["sigma"], n, 1, u0=u0, workspace=ws, stream=stream)[0].clone()
                return run
            u_eed, _ = fg.eed_inpaint(fd, md, p["lam"], p["sigma"], n, cycles, workspace=ws, stream=stream)
            u_eed = u_eed.clone()
            extra["time_to_mse"] = {
                "foeed": time_to_mse(fg, one(fg.foeed_inpaint), imgd, cycles, ms_per_step / cycles, u32),
                "eed": time_to_mse(fg, one(fg.eed_inpaint), imgd, cycles, min(eed_ms[1:]) / cycles, u_eed)}

    if rank == 0 and not args.no_batched:
        extra["batched"] = batched_leg(fg, synth, torch, dev, stream)
    if rank == 0 and not args.no_adjoint:
        extra["adjoint"] = adjoint_leg(fg, synth, torch, dev, stream)
    if rank == 0 and not args.no_convergence:
        extra["convergence"] = convergence_leg(fg, synth, torch, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(p, img, mask, gpu_results)
        if "oracle_reference" in cpu:
            extra["accuracy"].update(cpu.pop("oracle_reference"))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": p["name"], "w": W, "h": H, "mask_density": p["density"], "sigma": p["sigma"],
                       "lambda": p["lam"], "tau": 0.05, "fsi_cycles": cycles, "cycle_len": n,
                       "pixel_updates_per_step": pu_per_solve,
                       "l2": "flushed (256 MB write) between timed steps; the 38 MB working set stays "
                             "L2-resident within a solve",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": launches_per_solve * args.steps, "roofline": roofline,
            "tile_plan": tile_plan,
            "cpu_baseline": cpu, "clocks": clocks, **extra,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
