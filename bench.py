"""Benchmark: Stokes DoF solved per second to a 1e-8 relative residual.

Workload (default): unit cube of 6 Kuhn tetrahedra refined to level 7
(129^3 nodes, 8,291,838 free DoFs), manufactured smooth solution (Sec. 5),
viscosity 1, Dirichlet velocity, zero-mean pressure; all-at-once Uzawa
multigrid V_var(3,3) from a zero initial guess.  One step = set the
right-hand side from device-resident nodal inputs + solve to 1e-8 in the
FP32-V-cycle-in-FP64-refinement mode (the headline); the plain FP64 solve is
timed the same way and reported beside it.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload (the oracle cannot hold level 7 in
seconds); with torchrun, ranks > 0 of the reference arm exit at once.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

# the CPU oracle is timed single-threaded; fix the BLAS pools before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokes DoF solved/s to 1e-8 rel. residual, FP32+refine vs FP64; HBM % of peak"
LEVEL = 7
TOL = 1e-8
# DRAM bytes (read + write) of one k_vel_colour_rhs<float> launch, from an ncu
# capture of `bench.py --roofline-only` at that level (cold caches: ncu
# flushes them before each pass); None where no capture of the current kernel
# exists.  The level-7 capture (47,154,176 bytes) predates the packed
# (row, quarter-row slot) thread mapping of the colour kernels, so it is not
# reported for the current kernel.
TRAFFIC_PER_LAUNCH = {}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _inputs(mesh):
    import workloads as W
    x = mesh.node_coords()
    return W.manufactured_forcing(x), W.manufactured_velocity(x)


def run_gpu(args):
    import torch

    import paper_1511_02134_gb300 as pkg
    import workloads as W

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    pkg.load_library()
    stream = torch.cuda.Stream()
    macro = W.unit_cube()
    mesh = pkg.Mesh(macro.vertices, macro.tets, macro.bc_flags, args.level, stream=stream.cuda_stream)
    nv, npn = mesh.num_dofs()
    dofs = 3 * nv + npn
    f_host, ud_host = _inputs(mesh)
    f_dev = torch.from_numpy(f_host).cuda()
    ud_dev = torch.from_numpy(ud_host).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2

    def step(mode):
        mesh.set_rhs(f_dev, ud_dev)
        _, _, st = mesh.solve(tol=TOL, max_cycles=50, mode=mode, want_solution=False)
        if st.status != 0:
            raise RuntimeError(f"solve did not converge: {st}")
        return st

    def timed(mode, steps, warmup):
        for _ in range(warmup):
            step(mode)
        total_ms, cycles, launches = 0.0, [], 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _barrier(world)
        torch.cuda.synchronize()
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)  # evict L2 between timed steps (not timed)
            stream.synchronize()
            k0 = mesh.kernel_launches()
            e0.record(stream)
            st = step(mode)
            e1.record(stream)
            e1.synchronize()
            launches += mesh.kernel_launches() - k0
            total_ms += e0.elapsed_time(e1)
            cycles.append(st.cycles)
        torch.cuda.synchronize()
        _barrier(world)
        return total_ms, cycles, launches, st

    clocks = ClockSampler(local)
    clocks.start()
    ms32, cyc32, launches32, st32 = timed(pkg.MODE_FP32_IR, args.steps, args.warmup)
    clk = clocks.stop()
    ms64, cyc64, launches64, st64 = timed(pkg.MODE_FP64, max(1, args.steps // 2), max(1, args.warmup // 3))

    ms32_max = _max_over_ranks(ms32, world)
    ms64_max = _max_over_ranks(ms64, world)
    n64 = max(1, args.steps // 2)
    value = world * dofs * args.steps / (ms32_max / 1e3)
    value64 = world * dofs * n64 / (ms64_max / 1e3)

    # ---- end to end through the C ABI with pinned host buffers ----
    f_pin = torch.from_numpy(f_host).pin_memory()
    ud_pin = torch.from_numpy(ud_host).pin_memory()
    n = mesh.num_nodes()
    u_pin = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    p_pin = torch.empty((n,), dtype=torch.float64).pin_memory()
    e2e_ms = 0.0
    for _ in range(args.steps):
        stream.synchronize()
        t0 = time.perf_counter()
        mesh.set_rhs(f_pin, ud_pin)
        mesh.solve(tol=TOL, max_cycles=50, mode=pkg.MODE_FP32_IR, u_out=u_pin, p_out=p_pin)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = _max_over_ranks(e2e_ms, world)
    e2e = {"value": world * dofs * args.steps / (e2e_ms / 1e3), "unit": "DoF/s",
           "h2d_bytes_per_step": int(2 * 3 * n * 8), "d2h_bytes_per_step": int(4 * n * 8)}

    roofline = measure_roofline(mesh, args.level, stream, flush)

    out = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle + f64 refinement", "data": "synthetic",
        "config": {"workload": f"unit cube, 6 Kuhn tetrahedra, level {args.level} ({dofs} free DoFs), manufactured "
                               "solution, V_var(3,3) from zero to 1e-8", "level": args.level, "free_dofs": dofs,
                   "mode": "FP32 V-cycle inside FP64 iterative refinement", "l2": "flushed (256 MB write) "
                   "between timed steps", "parallelism": "replicas" if world > 1 else "single GPU"},
        "cycles": cyc32, "fp64": {"value": value64, "ms_per_step": ms64_max / n64, "cycles": cyc64,
                                  "dtype": "f64"},
        "speedup_fp32ir_vs_fp64": value / value64,
        "roofline": roofline, "clocks": clk, "e2e": e2e, "gpu_launches": launches32,
    }
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(out))
    mesh.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_roofline(mesh, lvl, stream, flush):
    """Roofline of the dominant kernel of the FP32 path: the velocity colour
    sweep with f - B^T p formed at each node (k_vel_colour_rhs<float>) on the
    finest level, timed with CUDA events on the mesh's stream (hhg_time_op).
    Algorithmic bytes of one forward sweep (four colour launches): u read and
    written (2 x 3 x 4 B), f (3 x 4 B), p (4 B) and the node flag (1 B) once per
    node; one colour launch carries a quarter of that."""
    import torch
    peak, peak_kind = _peaks()
    reps = 20
    with torch.cuda.stream(stream):
        flush.fill_(1.0)
    stream.synchronize()
    ms_sweep = mesh.time_op(lvl, "vel_forward_f", precision=1, reps=reps)  # 4 colour launches
    ms_launch = ms_sweep / 4.0
    nodes = mesh.num_nodes(lvl)
    alg_bytes = nodes * (2 * 3 * 4 + 3 * 4 + 4 + 1) / 4.0
    achieved = alg_bytes / (ms_launch / 1e3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": TRAFFIC_PER_LAUNCH.get(lvl),
            "kernel": "k_vel_colour_rhs<float> (level %d)" % lvl, "peak_kind": peak_kind,
            "ms_per_launch": ms_launch, "alg_bytes_per_launch": alg_bytes}


def roofline_only(args):
    """Set up the bench workload, run one FP32+IR solve and print the roofline
    measurement alone (the command the kernel profiles are taken with)."""
    import torch
    import paper_1511_02134_gb300 as pkg
    import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    cube = W.unit_cube()
    mesh = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, args.level, stream=stream.cuda_stream)
    x = mesh.node_coords()
    mesh.set_rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    mesh.solve(tol=TOL, max_cycles=50, mode=pkg.MODE_FP32_IR, want_solution=False)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    print(json.dumps(measure_roofline(mesh, args.level, stream, flush)))
    mesh.close()


def _oracle_sample(level: int, seconds: float):
    """Time the CPU oracle's FP64 solve (as it stands) on the cube at `level`."""
    import workloads as W
    from oracle import multigrid as MG
    H = MG.build_hierarchy(W.unit_cube(), level)
    L = H.levels[level]
    x = L.mesh.xyz
    f, g = L.rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    t_solve, runs, cycles = 0.0, 0, 0
    while t_solve < seconds or runs == 0:
        t0 = time.perf_counter()
        res = MG.solve(H, f, g, tol=TOL, max_cycles=50)
        t_solve += time.perf_counter() - t0
        runs += 1
        cycles = res.cycles
    return L.n_dofs * runs / t_solve, runs, cycles, L.n_dofs


def cpu_baseline(seconds: float, level: int = 5):
    v, runs, cycles, dofs = _oracle_sample(level, seconds)
    return {"value": v, "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": f"unit cube level {level} ({dofs} free DoFs), FP64 V_var(3,3) to 1e-8, {runs} solves "
                      f"x {cycles} cycles, numpy/scipy single thread; setup excluded"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    level = 5
    per = []
    for _ in range(args.warmup):
        _oracle_sample(level, 0.0)
    for _ in range(args.steps):
        v, runs, cycles, dofs = _oracle_sample(level, 0.0)
        per.append(v)
    value = float(np.mean(per))
    sample = (f"unit cube level {level} ({dofs} free DoFs) instead of level {args.level}: FP64 V_var(3,3) to 1e-8 "
              f"by the numpy/scipy oracle, one solve per step, single thread")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dofs / value * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"unit cube, 6 Kuhn tetrahedra, level {args.level}, manufactured solution "
                                  "(oracle on a bounded sample)", "level": level},
           "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=LEVEL)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--roofline-only", action="store_true",
                    help="print only the roofline measurement of the dominant kernel")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import __graft_entry__ as g
    g.build()
    if args.roofline_only:
        roofline_only(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
