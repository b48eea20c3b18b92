#!/usr/bin/env python3
"""Throughput benchmark of the fused phase-field LB step on GB300.

Workload: 2-D Rayleigh-Taylor instability on a 16384 x 16384 grid (Atwood
0.5, Re = 3000, d = 16384, 32 seeded random interface modes), conservative
Allen-Cahn phase field, consistent-flux hydrodynamics, FP32, periodic in x
with no-flux / no-slip walls in y (Sec. 4.4 of the paper, at the throughput
size).  One benchmark step = one time step of the whole grid = one launch of
the fused kernel; the metric is million lattice updates per second (phase +
flow per node), summed over GPUs.

`python bench.py [--gpus N --steps K --warmup W]` prints one JSON line.
Under torchrun each rank runs its own full-size replica (weak scaling: the
path shards into independent replicas, there is no data-path collective).
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import glob
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "fused-step MLUPS (phase+flow) and % HBM roofline; adjoint/forward time ratio"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6800.0
# GB300's FP64 rate (non-tensor), nominal: the FP64 step is bound by it
FP64_NOMINAL_GFLOPS = 1250.0
PRECISIONS = {  # name: (lbm precision, dtype label, algorithmic bytes per lattice update)
    "fp32": (W.PREC_FP32, "f32", 46 * 4),
    "fp64": (W.PREC_FP64, "f64", 46 * 8),
    # per set and node: FP32 rest population + 8 x 16-bit deviations (20 B),
    # two sets read and written, FP32 history read and written
    "fp16dev": (W.PREC_FP16_DEV, "f32", 2 * 2 * 20 + 2 * 5 * 4),
    "bf16dev": (W.PREC_BF16_DEV, "f32", 2 * 2 * 20 + 2 * 5 * 4),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pflbm", choices=["pflbm", "reference"])
    ap.add_argument("--n", type=int, default=16384, help="grid side")
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-storage-compare", action="store_true",
                    help="skip timing the 16-bit deviation storage beside FP32")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip timing the adjoint against the forward pass")
    ap.add_argument("--adjoint-steps", type=int, default=400)
    ap.add_argument("--adjoint-precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the adjoint against the forward pass (profiling)")
    ap.add_argument("--obstacle-only", action="store_true",
                    help="time only the dam break over the obstacle, beside the same chamber "
                         "without it on both fused kernels (profiling)")
    return ap.parse_args()


def workload_name(n):
    return f"rti_multimode_{n}x{n}_atwood0.5_re3000_ac"


# ---------------------------------------------------------------------------
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            flat = {}

            def walk(o, pre=""):
                if isinstance(o, dict):
                    for k, v in o.items():
                        walk(v, f"{pre}{k}.")
                else:
                    flat[pre[:-1]] = o
            walk(d)
            for k, v in flat.items():
                if "hbm" in k.lower() and isinstance(v, (int, float)) and "sustain" not in k.lower():
                    return float(v), "of measured"
            for k, v in flat.items():
                if "hbm" in k.lower() and isinstance(v, (int, float)):
                    return float(v), "of measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "of fallback"


def profiled_traffic(precision, key=None):
    """DRAM bytes per lattice update of the step kernel, from the committed
    ncu summary (profiles/*.txt line 'dram_bytes_per_lu_<precision>: X');
    `key` reads another per-update figure the same way."""
    key = key or f"dram_bytes_per_lu_{precision}"
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.txt"))):
        for line in open(f):
            m = re.match(rf"\s*{key}\s*:\s*([0-9.eE+-]+)", line)
            if m:
                return float(m.group(1)), os.path.basename(f)
    return None, None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"pflbm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def cpu_baseline(case, seconds, side=512):
    """The FP64 oracle on a bounded sample of the workload: a side x side
    window of the same initial field (centred on the interface, walls at its
    y ends), timed for about `seconds` of host time."""
    import oracle

    n = case.params.nx
    y0 = n // 2 - side // 2
    x0 = n // 2 - side // 2
    sub = case.params.with_(nx=side, ny=side, precision=W.PREC_FP64)
    phi = np.ascontiguousarray(case.phi[y0:y0 + side, x0:x0 + side])
    o = oracle.Oracle(sub)
    o.init_fields(phi)
    o.step(1)

    def timed(limit):
        steps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < limit:
            o.step(2)
            steps += 2
        return steps, time.perf_counter() - t0

    steps, dt = timed(seconds)
    cores = oracle.get_threads()
    oracle.set_threads(1)  # the same oracle on one core, for a fifth of the time
    s1, d1 = timed(seconds / 5)
    oracle.set_threads(cores)
    return {"value": side * side * steps / dt / 1e6, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{side}x{side} window of the {n}x{n} initial field at the interface, "
                      f"{steps} FP64 steps ({dt:.1f} s)",
            "single_core_value": side * side * s1 / d1 / 1e6, "cpu_model": cpu_model()}


def cpu_model() -> str:
    """The host CPU's model name as lscpu reports it (empty if unavailable)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return ""


def run_reference(args):
    """--impl reference: the oracle on the host cores, each step one oracle
    time step of a 256 x 256 window of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    side = 256
    n = args.n
    full = W.rti_multimode(n, precision=W.PREC_FP64)
    y0 = x0 = n // 2 - side // 2
    case = W.Case("rti_window", full.params.with_(nx=side, ny=side),
                  np.ascontiguousarray(full.phi[y0:y0 + side, x0:x0 + side]))
    del full
    o = oracle.Oracle(case.params)
    o.init_fields(case.phi)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = side * side * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(n), "precision": "fp64", "sample_side": side},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"{side}x{side} RTI window with the workload's parameters, "
                                       f"{args.steps} timed FP64 steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks_of(x: float, world: int, dist, device) -> float:
    """The largest of the ranks' values of x (one all-reduce; the job's time
    is its slowest replica's)."""
    if world == 1:
        return x
    import torch

    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, nodes_per_rank: int, steps: int, seconds: float) -> float:
    """Lattice updates of all replicas per second of the slowest one, / 1e6."""
    return world * nodes_per_rank * steps / seconds / 1e6


def adjoint_timing(args, torch):
    """Adjoint/forward time ratio on the adjoint workload (512 x 2048 RTI,
    Atwood 0.5, Re 1000, 8 seeded modes; checkpoints every 100 steps;
    J = phi-weighted vertical centroid), over a shorter horizon than its
    2000 steps.  Wall time with the device synchronised on both sides of the
    forward rollout and of the backward pass (recomputation included); the
    first of two passes warms allocations and kernels up."""
    from paper_2111_00847_gb300.adjoint import centroid_y, interface_phi0, rollout

    prec = W.PREC_FP64 if args.adjoint_precision == "fp64" else W.PREC_FP32
    case = W.rti_adjoint(precision=prec)
    prm = case.params
    every = 100
    out = {}
    for _ in range(2):
        a = torch.tensor(case.notes["a"], dtype=torch.float64, requires_grad=True)
        G = torch.tensor([prm.gx, prm.gy], dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        phiN = rollout(interface_phi0(a, prm.nx, prm.ny, prm.width, prm.phiA, prm.phiB), G, prm,
                       args.adjoint_steps, every)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        centroid_y(phiN).backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out = {"workload": "rti_adjoint_512x2048_atwood0.5_re1000_8modes",
               "precision": args.adjoint_precision, "steps": args.adjoint_steps, "checkpoint_every": every,
               "forward_ms_per_step": (t1 - t0) / args.adjoint_steps * 1e3,
               "backward_ms_per_step": (t2 - t1) / args.adjoint_steps * 1e3,
               "ratio": (t2 - t1) / (t1 - t0),
               "what": "backward = checkpoint recomputation + adjoint steps; wall time, device synchronised"}
    return out


# ---------------------------------------------------------------------------
def obstacle_timing(args, torch, pk, stream, barrier, max_over_ranks, world, peak, compare=False):
    """The dam break over the trapezoidal obstacle, 4096 x 2048 (a = 1024,
    height a/2 at Lx/2), FP32, Allen-Cahn: the phi pass with its fill over the
    region the blocks near the obstacle read, then the TMA step (2 launches a
    step); 5 x K steps after W warm-up steps,
    CUDA events on the simulation's stream.  compare: also the same chamber
    without the obstacle on the TMA and on the register-pipelined kernel."""
    db = W.dam_break_obstacle(nx=4096, ny=2048, precision=W.PREC_FP32)
    nodes = db.params.nx * db.params.ny
    nst = 5 * args.steps

    def run(params, solid):
        sim = pk.Simulation(params, stream=stream)
        if solid is not None:
            sim.set_solid(solid)
        sim.init_fields(db.phi)
        sim.step(args.warmup)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(nst)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        gb = sim.device_bytes / 1e9
        sim.close()
        return ms, gb

    oms, gb = run(db.params, db.solid)
    out = {"dam_break_obstacle_4096x2048": {
        "value": whole_job_mlups(world, nodes, nst, oms / 1e3), "unit": UNIT, "steps": nst,
        "ms_per_step": oms / nst, "solid_fraction": float(db.solid.mean()), "launches_per_step": 2,
        "frac_of_fused_bytes": PRECISIONS["fp32"][2] * nodes * nst / (oms / 1e3) / 1e9 / peak,
        "l2": f"state {gb:.2f} GB > L2"}}
    if compare:
        for name, flags in (("no_obstacle_tma", 0), ("no_obstacle_register_kernel", pk.LBM_FLAG_NO_TMA)):
            ms, _ = run(db.params.with_(flags=flags), None)
            out[name] = {"value": whole_job_mlups(world, nodes, nst, ms / 1e3), "unit": UNIT,
                         "ms_per_step": ms / nst}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.adjoint_only:
        import __graft_entry__

        __graft_entry__.build()
        if rank == 0:
            print(json.dumps({"metric": "adjoint/forward time ratio", "adjoint": adjoint_timing(args, torch)}),
                  flush=True)
        return

    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2111_00847_gb300 as pk

    prec, dtype, bytes_per_lu = PRECISIONS[args.precision]
    n = args.n
    N = n * n

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return max_over_ranks_of(x, world, dist, dev)

    stream = torch.cuda.current_stream(dev)
    peak, peak_src = measured_peak()
    if args.obstacle_only:
        res = obstacle_timing(args, torch, pk, stream, barrier, max_over_ranks, world, peak, compare=True)
        if rank == 0:
            print(json.dumps({"metric": "obstacle step MLUPS", "obstacle_workloads": res}), flush=True)
        return
    case = W.rti_multimode(n, precision=prec)

    def timed_steps(params, label, per_lu_bytes, phi0=None, steps=None):
        """W warm-up steps, then K steps timed with CUDA events on the
        simulation's stream (barrier + synchronize on both sides); the
        roofline of the fused step kernel (one launch per step)."""
        nodes = params.nx * params.ny
        nsteps = args.steps if steps is None else steps
        s = pk.Simulation(params, stream=stream)
        s.init_fields(case.phi if phi0 is None else phi0)
        s.step(args.warmup)
        torch.cuda.synchronize()
        clk_s = ClockSampler(local)
        clk_s.start()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ck = clk_s.stop()
        t_ms = max_over_ranks(e0.elapsed_time(e1))
        launch_s = t_ms / 1e3 / nsteps
        ach = per_lu_bytes * nodes / launch_s / 1e9
        tr, tr_from = profiled_traffic(label)
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": (tr * nodes if tr is not None else None), "peak_source": peak_src,
                "algorithmic_bytes_per_lu": per_lu_bytes, "traffic_source": tr_from}
        return s, t_ms, roof, ck

    # ---- device-resident timed region
    sim, ms, roofline, clk = timed_steps(case.params, args.precision, bytes_per_lu)
    sec = ms / 1e3
    value = whole_job_mlups(world, N, args.steps, sec)

    # ---- end to end through the public API, host buffers, copies inside
    e2e = None
    if not args.no_e2e:
        phi_h = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        phi_h.numpy()[...] = case.phi
        out_h = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.init_fields(phi_h.numpy())
        sim.step(args.steps)
        sim.fields(pk.LBM_PHI, out=out_h.numpy())
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0)
        barrier()
        e2e = {"value": world * N * args.steps / te / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": 8 * N / args.steps, "d2h_bytes_per_step": 8 * N / args.steps,
               "what": "lbm_init_fields(phi from pinned host) + lbm_step(K) + lbm_fields(PHI to pinned host)"}
        del phi_h, out_h
    state_gb = sim.device_bytes / 1e9
    sim.close()
    del sim

    # ---- the wetting-boundary path: droplet spreading at 2048 x 1024 (walls
    # with contact angles 30, 60, 120 degrees on the bottom, x periodic), FP32
    wetting = None
    if args.precision == "fp32" and not args.no_storage_compare:
        wetting = {}
        for th in (30.0, 60.0, 120.0):
            sp = W.droplet_spreading(theta=th, precision=W.PREC_FP32)
            ssim = pk.Simulation(sp.params, stream=stream)
            ssim.init_fields(sp.phi)
            ssim.step(args.warmup)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            nst = 10 * args.steps
            e0.record(stream)
            ssim.step(nst)
            e1.record(stream)
            torch.cuda.synchronize()
            wms = max_over_ranks(e0.elapsed_time(e1))
            nodes = sp.params.nx * sp.params.ny
            wetting[f"droplet_spreading_2048x1024_theta{int(th)}"] = {
                "value": whole_job_mlups(world, nodes, nst, wms / 1e3), "unit": UNIT, "steps": nst,
                "frac": bytes_per_lu * nodes * nst / (wms / 1e3) / 1e9 / peak,
                "l2": f"state {ssim.device_bytes / 1e9:.2f} GB > L2"}
            ssim.close()

    obstacle = None
    if args.precision == "fp32" and not args.no_storage_compare:
        obstacle = obstacle_timing(args, torch, pk, stream, barrier, max_over_ranks, world, peak)

    # ---- the Cahn-Hilliard alternative on the same workload (phi in [-1, 1])
    models = None
    if args.precision == "fp32" and not args.no_storage_compare:
        chp = case.params.with_(phase_model=W.MODEL_CH, phiA=1.0, phiB=-1.0)
        sch, msch, roofch, clkch = timed_steps(chp, "fp32_ch", bytes_per_lu, 2.0 * case.phi - 1.0)
        sch.close()
        del sch
        models = {"cahn_hilliard": {"value": whole_job_mlups(world, N, args.steps, msch / 1e3), "unit": UNIT,
                                    "ms_per_step": msch / args.steps, "roofline": roofch, "clocks": clkch}}
        # the FP64 step (the path held to 1e-12 against the oracle): RTI
        # 8192^2, K/5 steps; bound by GB300's FP64 pipe, not by HBM
        n64 = 8192
        c64 = W.rti_multimode(n64, precision=W.PREC_FP64)
        k64 = max(1, args.steps // 5)
        s64, ms64, roof64, clk64 = timed_steps(c64.params, "fp64", PRECISIONS["fp64"][2], c64.phi, steps=k64)
        s64.close()
        del s64
        lups64 = n64 * n64 * k64 / (ms64 / 1e3)
        fl, fl_from = profiled_traffic("fp64", key="fp64_flops_per_lu")
        ni, _ = profiled_traffic("fp64", key="fp64_inst_per_lu")
        alu = None
        if fl is not None:
            ach = fl * lups64 / 1e9
            alu = {"bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
                   "frac": ach / FP64_NOMINAL_GFLOPS, "traffic": None,
                   "peak_source": "nominal FP64 rate of GB300: 2 FP64 instructions per clock per SM "
                                  "x 152 SMs x 2.07 GHz x 2 flops (no measured FP64 peak)",
                   "flops_per_lu": fl, "flops_source": fl_from}
            if ni is not None:
                # DADD and DMUL hold an FP64 issue slot for one flop: the pipe's
                # own rate, in instructions
                alu["fp64_pipe_frac"] = ni * lups64 / (2 * 152 * 2.07e9)
        models["fp64"] = {"value": whole_job_mlups(world, n64 * n64, k64, ms64 / 1e3), "unit": UNIT,
                          "workload": workload_name(n64), "steps": k64, "ms_per_step": ms64 / k64,
                          "roofline": alu, "hbm_frac": roof64["frac"], "clocks": clk64}

    # ---- the same workload with 16-bit deviation storage (FP32 arithmetic)
    storage = None
    if args.precision == "fp32" and not args.no_storage_compare:
        storage = {}
        for name in ("fp16dev",):
            p16, _, b16 = PRECISIONS[name]
            s16, ms16, roof16, clk16 = timed_steps(case.params.with_(precision=p16), name, b16)
            s16.close()
            del s16
            storage[name] = {"value": world * N * args.steps / (ms16 / 1e3) / 1e6, "unit": UNIT,
                             "ms_per_step": ms16 / args.steps, "roofline": roof16, "clocks": clk16,
                             "gain_vs_fp32": ms / ms16}

    adjoint = None
    if rank == 0 and not args.no_adjoint:
        adjoint = adjoint_timing(args, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(case, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype,
                "data": "synthetic",
                "config": {"workload": workload_name(n), "nx": n, "ny": n,
                           "precision": args.precision, "phase_model": "AC", "flux": "present",
                           "replicas": world, "parallelism": f"replicas{world}",
                           "l2": f"inputs larger than L2 (device state {state_gb:.1f} GB)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps, "clocks": clk, "storage_variants": storage,
                "wetting_workloads": wetting, "obstacle_workloads": obstacle, "model_variants": models,
                "adjoint": adjoint}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
