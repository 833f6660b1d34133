#!/usr/bin/env python3
"""Benchmark: MLUPS of the full per-iteration hot path (the persistent step
kernel: bulk lattice, boundary, critical and auxiliary particle parts) on the
8 x 64^3 orientation-sweep workload, one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp16|bf16]
  python bench.py --impl reference ...   (the CPU oracle on the same workload)

A step is one iteration of the paper's Appendix over all 8 boxes.  The state
(two distribution buffers of 160 MB each in FP32) is larger than the 129 MB L2,
so no flush is done between steps.  Under torchrun each rank runs its own 8
boxes (weak scaling, no collective on the data path).

The line's value is the FP32 leg (or --precision's).  After it, the same
workload runs with FP16 and BF16 deviation storage for the same K steps
("mixed": MLUPS, roofline fraction and ratio to FP32), and one box of the sweep
is run in all three formats against the FP64 oracle for --drag-steps
iterations ("mixed.drag_error_vs_oracle"), and the D3Q27 lattice runs the
same workload in FP32 ("d3q27": MLUPS and the fraction of the HBM roofline at
216 bytes per lattice update, with BGK and with the paper's ghost-mode
collision).  "steps_to_steady" is the learned
warm start on the surrogate workload's evaluation box (128^3, 16 spheroids):
steps until every particle's velocity stays within 1e-2 / 3e-3 / 1e-3 of its
steady value, cold, with the lattice fluid's steady flow only, and warm.
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

BYTES_PER_LUP = {"fp32": 152, "fp16": 76, "bf16": 76}   # 2 * 19 * s, read + write
PREC = {"fp32": 0, "fp16": 1, "bf16": 2}
WORKLOADS = {
    "sweep_8x64": ("sweep_8x64: 8 periodic 64^3 D3Q19 boxes, BGK tau=0.8, one prolate spheroid (8,4,4) per box "
                   "at 0,15,...,90 deg and a random orientation to the force, |F_ext|=5e-4 with counter body force"),
    "squirmer_batch": ("squirmer_batch: 32 periodic cubic D3Q19 boxes of edges drawn from {48,64,96,128} in one "
                       "launch, BGK tau=1, one squirmer spheroid (6,3,3) per box, B1=1e-3, B2/B1 in {-2,0,2}"),
}
WORKLOAD = WORKLOADS["sweep_8x64"]


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


STEP_ITERS = 256   # iterations per launch of the step kernel (the library's chunk)


STEP_SOURCES = ("step_kernel.cu", "boundary_block.cuh", "bulk_tile.cuh", "particle_blocks.cuh", "lattice_common.cuh",
                "lbsph_internal.cuh")


def kernel_hash():
    """Hash of the device sources the persistent step kernel is compiled from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2403_05443_gb300", "csrc")
    for f in STEP_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(precision, nodes):
    """DRAM bytes per iteration of the step kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[precision]
        if e.get("source_hash") != kernel_hash():
            return None
        return float(e["dram_bytes_per_node"]) * nodes
    except Exception:
        return None


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Weak scaling: every rank advances its own nodes_per_rank nodes by steps
    iterations; the job's rate divides all of them by the slowest rank's time."""
    return nodes_per_rank * steps * world / seconds / 1e6


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def cpu_baseline(target_s: float = 12.0, boxes_parts=None):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload."""
    from lb_inputs import sweep_8x64
    from oracle import oracle as O

    boxes, parts = boxes_parts or sweep_8x64(seed=0)
    threads = os.cpu_count() or 1
    sims = [O.Sim(b, p, nthreads=threads) for b, p in zip(boxes, parts)]
    nodes = sum(b["nx"] * b["ny"] * b["nz"] for b in boxes)
    t0 = time.perf_counter()
    for s in sims:
        s.step(1)
    one = time.perf_counter() - t0
    k = max(1, int(target_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    for s in sims:
        s.step(k)
    dt = time.perf_counter() - t0
    return {"value": nodes * k / dt / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"all 8 boxes (2,097,152 nodes), {k} iterations after one warm-up iteration, "
                      f"FP64, OpenMP over {threads} threads, {dt:.1f} s"}


def static_config(args, boxes, world):
    """The workload description both arms print (identical dicts)."""
    nodes = sum(b["nx"] * b["ny"] * b["nz"] for b in boxes)
    return {"workload": WORKLOADS[args.workload], "boxes": len(boxes), "nodes_per_gpu": nodes,
            "precision": args.precision,
            "l2": f"state {2 * nodes * BYTES_PER_LUP[args.precision] // 2 / 1e6:.0f} MB > 129 MB L2; not flushed",
            "parallelism": f"{world} rank(s), {len(boxes)} independent boxes each, no collective"}


def run_reference(args):
    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    if rank != 0:
        return 0
    import lb_inputs
    from oracle import oracle as O

    boxes, parts = getattr(lb_inputs, args.workload)(seed=args.seed)
    threads = os.cpu_count() or 1
    nb = len(boxes)
    sims = [None] * nb
    # each step is a bounded sample: one iteration of one of the boxes, in turn
    # (a box's oracle state is created on its first use, outside the timed steps)
    for i in range(max(args.warmup, nb)):
        k = i % nb
        if sims[k] is None:
            sims[k] = O.Sim(boxes[k], parts[k], nthreads=threads)
        sims[k].step(1)
    nodes = 0
    t0 = time.perf_counter()
    for i in range(args.steps):
        k = i % nb
        sims[k].step(1)
        nodes += boxes[k]["nx"] * boxes[k]["ny"] * boxes[k]["nz"]
    dt = time.perf_counter() - t0
    v = nodes / dt / 1e6
    line = {"impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": static_config(args, boxes, world),
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} single-box iterations of the FP64 oracle, the boxes in "
                                       f"turn ({nodes:,} node updates), OpenMP over {threads} threads"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def drag_error_vs_oracle(steps: int, seed: int = 0):
    """Drag and rotation error of each storage format against the FP64 oracle on
    one box of the sweep (the 45-degree spheroid: drag along and across its
    axis, and a torque-free drift), the velocities averaged over the last 500 of
    `steps` iterations: |U - U_ref| / |U_ref| and |Omega - Omega_ref| a / |U_ref|
    (the rotation's surface speed)."""
    import numpy as np

    import paper_2403_05443_gb300 as pkg
    from lb_inputs import sweep_8x64
    from oracle import oracle as O

    boxes, parts = sweep_8x64(seed=seed)
    b, pl = boxes[3], parts[3]
    avg = min(500, steps // 2)

    def steady(step, read):
        # mean over the last `avg` steps (a node covered a few steps apart on
        # the two sides moves the instantaneous drag by ~1e-3 of itself)
        step(steps - avg)
        acc = []
        for _ in range(avg // 25):
            step(25)
            acc.append(read())
        return {k: np.mean([x[k] for x in acc], axis=0) for k in ("U", "Om")}

    t0 = time.perf_counter()
    ref = O.Sim(b, pl, nthreads=os.cpu_count() or 1)
    r = steady(ref.step, lambda: ref.particle(0))
    t_orc = time.perf_counter() - t0
    ref.close()
    a = max(pl[0]["semi"])
    out = {}
    for name, prec in PREC.items():
        sim = pkg.Simulation([b], [pl], precision=prec, max_semi=8)
        g = steady(sim.step, lambda: sim.particle(0))
        sim.close()
        nU = float(np.linalg.norm(r["U"]))
        out[name] = {"drag": float(np.linalg.norm(g["U"] - r["U"]) / nU),
                     "rotation": float(np.linalg.norm(g["Om"] - r["Om"]) * a / nU)}
    out["sample"] = (f"box 4 of the sweep (64^3, tau 0.8, (8,4,4) at 45 deg, |F| 5e-4), {steps} iterations, "
                     f"means over the last {avg}; GPU storage formats against the FP64 oracle "
                     f"({t_orc:.1f} s on the host)")
    out["U_ref"] = [float(v) for v in r["U"]]
    return out


SURROGATE_WEIGHTS = os.path.join(ROOT, "paper_2403_05443_gb300", "surrogate_config5.npy")


def steps_to_steady_block(args):
    """Steps to steady state of the surrogate workload's evaluation box (128^3,
    16 spheroids with a/b in [1, 4] and b in [3, 5], random orientations,
    forces in random directions with the counter force, tau = 1): cold, the
    lattice fluid's steady flow alone, and warm (that flow plus the network's
    velocities), against the velocities at the end of the cold run.  The
    network is the one trained on the workload's 64^3 resistance runs
    (surrogate_config5.npy, written by `python -m
    paper_2403_05443_gb300.warmstart config5`); without that file a small
    network is trained here first on 96 samples in 32^3 boxes."""
    from paper_2403_05443_gb300 import warmstart as W

    t0 = time.perf_counter()
    if os.path.exists(SURROGATE_WEIGHTS):
        net = W.load_params(SURROGATE_WEIGHTS)
        origin = "surrogate_config5.npy (trained on the workload's 64^3 resistance runs)"
    else:
        import lb_inputs as I
        import numpy as np

        smp = I.resistance_samples(args.seed, 96, 32)
        M = np.zeros((len(smp), 6, 6))
        for tau in (0.8, 1.0, 1.2):
            sub = [i for i, s in enumerate(smp) if s["tau"] == tau]
            if sub:
                steps = int(8 * 32 * 32 / (4 * 3.141592653589793 ** 2 * (tau - 0.5) / 3.0))
                M[sub] = W.measure_mobility([smp[i] for i in sub], steps)[0]
        geoms = np.asarray([W.geom_of(s["a"], s["b"], s["tau"], s["L"], s["e"]) for s in smp])
        x, R = W.targets(*W.augment(geoms, M))
        net, _ = W.train(x, R, steps=1500, seed=args.seed)
        origin = "trained here: 96 samples in 32^3 boxes, 1500 steps (no surrogate_config5.npy)"
    ev = W.evaluate(net, seed=args.seed, eval_n=128, eval_count=16, force=1e-7, every=50, ref_steps=args.steady_steps,
                    eval_tau=1.0, aspect=(1.0, 4.0), b_range=(3.0, 5.0))
    ev.pop("error_curves", None)
    ev["network"] = origin
    ev["seconds_total"] = time.perf_counter() - t0
    return ev


def run_leg(args, pkg, precision, boxes, parts, local, dist, stream, sp, primary, lattice=19, collision=0):
    """Warm-up, autotune and the timed K steps of one storage format (or of the
    D3Q27 lattice, which has no tuner) on the workload; returns its
    measurements (and the simulation, still open)."""
    import torch

    nodes = sum(b["nx"] * b["ny"] * b["nz"] for b in boxes)
    sim = pkg.Simulation(boxes, parts, precision=PREC[precision], max_semi=8, device=local, torch_alloc=True,
                         lattice=lattice, collision=collision)
    sim.step(args.warmup, stream=sp)
    if lattice == 19:
        # launch shape of the step kernel for this workload (untimed; the
        # candidates compute identical values, so this is more warm-up)
        (fetch, gx, _), tune_ms = pkg.lbsph.lb_autotune(sim.ctx, 64, sp)
    else:
        fetch, gx, tune_ms = None, None, [0.0] * 10
    sim.step(args.warmup, stream=sp)           # the kept shape, right before the timed steps
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # an NVTX range around the timed launches (host side, outside the events),
    # so that a profiler can select exactly them (ncu --nvtx --nvtx-include)
    torch.cuda.nvtx.range_push(f"timed_steps_{precision}")
    e0.record(stream)
    sim.step(args.steps, stream=sp)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    per = ms / args.steps / 1e3
    peak, peak_src = measured_peak()
    achieved = (BYTES_PER_LUP[precision] if lattice == 19 else 2 * 27 * 4) * nodes / per / 1e9
    return sim, {"value": whole_job_mlups(nodes, args.steps, env_int("WORLD_SIZE", 1), ms / 1e3),
                 "ms_per_step": ms / args.steps, "achieved_gbs": achieved, "frac": achieved / peak,
                 "peak": peak, "peak_source": peak_src,
                 "tuning": {"units_per_fetch": fetch, "blocks_per_particle": gx,
                            "ms_per_step_gx_1_2_3_d_2d_3d": [round(v, 5) for v in tune_ms[:6]],
                            "ms_per_step_fetch_1_2_4_8": [round(v, 5) for v in tune_ms[6:]]}}


def run_ours(args):
    import numpy as np
    import torch

    import paper_2403_05443_gb300 as pkg
    import lb_inputs

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    boxes, parts = getattr(lb_inputs, args.workload)(seed=args.seed + rank)
    nodes = sum(b["nx"] * b["ny"] * b["nz"] for b in boxes)
    stream = torch.cuda.Stream()                  # every launch and event on this one stream
    torch.cuda.set_stream(stream)
    sp = pkg.lbsph.stream_handle(stream)
    # clocks are sampled from before the first warm-up step to after the last
    # timed leg, so that no idle gap precedes a timed region
    clocks = ClockSampler(local)
    clocks.start()
    sim, lead = run_leg(args, pkg, args.precision, boxes, parts, local, dist, stream, sp, True)
    launches = -(-args.steps // STEP_ITERS)
    traffic = committed_traffic(args.precision, nodes) if args.workload == "sweep_8x64" else None

    # the four parts as separate kernels, serialised with CUDA events between them
    nprof = max(50, min(500, args.steps // 10))
    k_ms, b_ms, c_ms, a_ms = pkg.lb_profile_step(sim.ctx, nprof, sp)

    # end to end through the C ABI: per step, F_ext/T_ext in from pinned host
    # memory, one iteration, all particle records back to pinned host memory
    np_tot = sum(len(p) for p in parts)
    ft_in = torch.empty((np_tot, 6), dtype=torch.float64, pin_memory=True)
    rec_out = torch.empty((np_tot, pkg.lbsph.LB_RECORD_DOUBLES), dtype=torch.float64, pin_memory=True)
    ft_np, rec_np = ft_in.numpy(), rec_out.numpy()
    for i, pl in enumerate(parts):
        ft_np[i, :3] = pl[0]["F_ext"]
        ft_np[i, 3:] = pl[0]["T_ext"]
    ke = max(20, min(400, args.steps // 20))
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        pkg.lb_set_external(sim.ctx, -1, ft_np, sp)
        sim.step(1, stream=sp)
        pkg.lb_get_force_torque(sim.ctx, -1, np_tot, rec_np)
    t_sync = max_over_ranks(time.perf_counter() - t0, dist)
    e2e_sync = whole_job_mlups(nodes, ke, world, t_sync)
    # pipelined: every step's inputs from their own pinned slot and every
    # step's records into their own pinned slot, queued on the stream, one wait
    ft_ring = torch.empty((ke, np_tot, 6), dtype=torch.float64, pin_memory=True)
    ft_ring[:] = ft_in
    rec_ring = torch.empty((ke, np_tot, pkg.lbsph.LB_RECORD_DOUBLES), dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    pkg.lb_step_io(sim.ctx, ke, ft_ring.data_ptr(), rec_ring.data_ptr(), sp)
    stream.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist)
    pkg.lb_synchronize(sim.ctx)
    e2e_v = whole_job_mlups(nodes, ke, world, t_e2e)
    if not np.array_equal(rec_ring[-1].numpy(), pkg.lb_get_force_torque(sim.ctx, -1, np_tot)):
        raise RuntimeError("pipelined records differ from the synchronous read-back")
    sim.close()

    # mixed precision: the same workload and step count with 16-bit storage
    mixed = None
    if args.precision == "fp32" and not args.no_mixed:
        mixed = {}
        for prec in ("fp16", "bf16"):
            s16, leg = run_leg(args, pkg, prec, boxes, parts, local, dist, stream, sp, False)
            s16.close()
            mixed[prec] = {"value": leg["value"], "unit": "MLUPS", "ms_per_step": leg["ms_per_step"],
                           "roofline": {"achieved": leg["achieved_gbs"], "peak": leg["peak"], "unit": "GB/s",
                                        "frac": leg["frac"], "bytes_per_lup": BYTES_PER_LUP[prec]},
                           "tuning": leg["tuning"]}
            mixed[prec]["ratio_vs_fp32"] = leg["value"] / lead["value"]
    # the D3Q27 lattice on the same workload (FP32; two kernels per step)
    d3q27 = None
    if args.precision == "fp32" and not args.no_d3q27:
        s27, leg = run_leg(args, pkg, "fp32", boxes, parts, local, dist, stream, sp, False, lattice=27)
        s27.close()
        d3q27 = {"value": leg["value"], "unit": "MLUPS", "ms_per_step": leg["ms_per_step"],
                 "roofline": {"achieved": leg["achieved_gbs"], "peak": leg["peak"], "unit": "GB/s",
                              "frac": leg["frac"], "bytes_per_lup": 2 * 27 * 4},
                 "ratio_vs_d3q19_fp32": leg["value"] / lead["value"],
                 "kernels": "lattice27_kernel near pass (pull, bounce-back, remap, collision, link sums) and "
                            "particle27_kernel (solve, pose, map, drag matrix) on one stream, bulk27_kernel "
                            "(pull, collision) on the other, per step"}
        # the same with the paper's ghost-mode collision
        s27, leg = run_leg(args, pkg, "fp32", boxes, parts, local, dist, stream, sp, False, lattice=27, collision=1)
        s27.close()
        d3q27["ghost_mode_collision"] = {"value": leg["value"], "unit": "MLUPS", "ms_per_step": leg["ms_per_step"],
                                         "frac": leg["frac"]}
    clk = clocks.stop()

    extra = {}
    if rank == 0 and world == 1 and args.workload == "sweep_8x64" and not args.no_cpu_baseline:
        extra["cpu_baseline"] = cpu_baseline(boxes_parts=(boxes, parts))
        if mixed is not None and args.drag_steps > 0:
            mixed["drag_error_vs_oracle"] = drag_error_vs_oracle(args.drag_steps, seed=args.seed)
    if rank == 0 and world == 1 and args.steady_steps > 0:
        extra["steps_to_steady"] = steps_to_steady_block(args)

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": lead["value"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": lead["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else f"f32 arithmetic, {args.precision} storage",
            "data": "synthetic",
            "config": static_config(args, boxes, world),
            "tuning": lead["tuning"],
            "roofline": {"bound": "hbm", "achieved": lead["achieved_gbs"], "peak": lead["peak"], "unit": "GB/s",
                         "frac": lead["frac"], "traffic": traffic, "peak_source": lead["peak_source"],
                         "kernel": "step_kernel (persistent: bulk pull streaming + BGK/Guo collision, "
                                   "boundary links, particle solve), per iteration",
                         "bytes_per_lup": BYTES_PER_LUP[args.precision],
                         "method": f"CUDA events on the launching stream around the timed region "
                                   f"({launches} launch(es) of up to {STEP_ITERS} iterations)",
                         "parts_ms_separate_kernels": {
                             "bulk": k_ms / nprof, "boundary": b_ms / nprof,
                             "particle_critical": c_ms / nprof, "particle_aux": a_ms / nprof,
                             "method": f"lb_profile_step: the four parts as separate kernels, {nprof} "
                                       "iterations after the timed region, CUDA events between them"}},
            "mixed": mixed,
            "d3q27": d3q27,
            "e2e": {"value": e2e_v, "unit": "MLUPS", "h2d_bytes_per_step": int(ft_in.numel() * 8),
                    "d2h_bytes_per_step": int(rec_out.numel() * 8), "steps": ke,
                    "path": "lb_step_io over all steps: per step F_ext/T_ext in from that step's pinned slot, "
                            "one iteration, all particle records out into that step's pinned slot, queued on "
                            "the stream by the library; one wait at the end",
                    "sync_per_step": {"value": e2e_sync, "unit": "MLUPS",
                                      "path": "lb_set_external(-1) + lb_step(1) + lb_get_force_torque(-1) "
                                              "(waits) per step"}},
            "steps_to_steady": extra.get("steps_to_steady"),
            "gpu_launches": launches,   # step-kernel launches in the timed region
            "clocks": clk,
            "cpu_baseline": extra.get("cpu_baseline"),
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=list(PREC))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workload", default="sweep_8x64", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP16 / BF16 legs")
    ap.add_argument("--no-d3q27", action="store_true", help="skip the D3Q27 leg")
    ap.add_argument("--drag-steps", type=int, default=3000,
                    help="iterations of the drag-error check against the oracle (0: skip)")
    ap.add_argument("--steady-steps", type=int, default=40000,
                    help="length of the cold reference run of the steps-to-steady check (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
