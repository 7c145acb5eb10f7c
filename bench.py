"""Benchmark: Stokes DoF solved per second to a 1e-8 relative residual.

Workload (default): unit cube of 6 Kuhn tetrahedra refined to level 9
(513^3 nodes, 535,304,190 free DoFs), manufactured smooth solution (Sec. 5),
viscosity 1, Dirichlet velocity, zero-mean pressure; all-at-once Uzawa
multigrid V_var(3,3) from a zero initial guess.  One step = set the
right-hand side from device-resident nodal inputs + solve to 1e-8 in the
FP32-V-cycle-in-FP64-refinement mode (the headline); the plain FP64 solve is
timed the same way and reported beside it, and the same pair is reported for
the level-7 cube (8,291,838 free DoFs) under "level7" and the level-4 cube
(15,038 free DoFs, latency-bound) under "level4".  "fmg" times full
multigrid (Sec. 5) on the headline level, with its error ratio gamma, its
parallel textbook efficiency E_parTME (with and without the coarse-grid
solves), and the 1e-8 solve started from one FMG pass;
"channel_level6" times the obstacle channel (2.6e8 free DoFs) FP32+IR solve
and "slip_channel_level6" the same channel with free-slip obstacles (Sec. 6.1);
"dform_level7" the D-operator formulation beside the Laplace form.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload (the oracle cannot hold level 9); with
torchrun, ranks > 0 of the reference arm exit at once.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import platform
import subprocess
import sys
import threading
import time

# the CPU oracle is timed single-threaded per process; fix the BLAS pools before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokes DoF solved/s to 1e-8 rel. residual, FP32+refine vs FP64; HBM % of peak"
LEVEL = 9
EXTRA_LEVEL = 7
TOL = 1e-8
ORACLE_LEVEL = 5
# DRAM bytes (read + write) of one launch of the roofline kernel, per lattice
# node of the level, from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of that kernel on the level-8 cube (17 M nodes, a
# few GB on the device: the fields are far larger than L2), scaled to the
# bench level by its node count; None where no capture of the current kernel
# exists.
TRAFFIC_BYTES_PER_NODE = {"k_vel_colour_rhs": (295984384 + 43319040) / 257 ** 3}  # 19.99 B: 339.3 MB / 257^3


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
    """The largest x over the ranks (the job's time is its slowest rank's);
    the tensor lives where the process group's backend wants it."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _inputs(mesh):
    import workloads as W
    x = mesh.node_coords()
    f, ud = W.manufactured_forcing(x), W.manufactured_velocity(x)
    del x
    return f, ud


class LevelBench:
    """One cube level: the mesh, device-resident inputs and the timed steps."""

    def __init__(self, pkg, level, stream, flush, world):
        import torch

        import workloads as W
        self.pkg, self.level, self.stream, self.flush, self.world = pkg, level, stream, flush, world
        macro = W.unit_cube()
        self.mesh = pkg.Mesh(macro.vertices, macro.tets, macro.bc_flags, level, stream=stream.cuda_stream)
        nv, npn = self.mesh.num_dofs()
        self.dofs = 3 * nv + npn
        self.n = self.mesh.num_nodes()
        self.f_host, self.ud_host = _inputs(self.mesh)
        self.f_dev = torch.from_numpy(self.f_host).cuda()
        self.ud_dev = torch.from_numpy(self.ud_host).cuda()

    def step(self, mode, u_out=None, p_out=None):
        self.mesh.set_rhs(self.f_dev, self.ud_dev)
        want = u_out is not None
        _, _, st = self.mesh.solve(tol=TOL, max_cycles=50, mode=mode, u_out=u_out, p_out=p_out,
                                   want_solution=want)
        if st.status != 0:
            raise RuntimeError(f"solve did not converge: {st}")
        return st

    def timed(self, mode, steps, warmup):
        import torch
        for _ in range(warmup):
            self.step(mode)
        total_ms, cycles, launches = 0.0, [], 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _barrier(self.world)
        torch.cuda.synchronize()
        for _ in range(steps):
            with torch.cuda.stream(self.stream):
                self.flush.fill_(1.0)  # evict L2 between timed steps (not timed)
            self.stream.synchronize()
            k0 = self.mesh.kernel_launches()
            e0.record(self.stream)
            st = self.step(mode)
            e1.record(self.stream)
            e1.synchronize()
            launches += self.mesh.kernel_launches() - k0
            total_ms += e0.elapsed_time(e1)
            cycles.append(st.cycles)
        torch.cuda.synchronize()
        _barrier(self.world)
        return _max_over_ranks(total_ms, self.world), cycles, launches

    def pair(self, steps, warmup, steps64, clocks=None):
        """FP32+IR (headline) and FP64, device-timed."""
        pkg = self.pkg
        if clocks:
            clocks.start()
        ms32, cyc32, launches32 = self.timed(pkg.MODE_FP32_IR, steps, warmup)
        clk = clocks.stop() if clocks else None
        ms64, cyc64, _ = self.timed(pkg.MODE_FP64, steps64, 1)
        v32 = self.world * self.dofs * steps / (ms32 / 1e3)
        v64 = self.world * self.dofs * steps64 / (ms64 / 1e3)
        return {"value": v32, "ms_per_step": ms32 / steps, "cycles": cyc32, "launches": launches32,
                "fp64": {"value": v64, "ms_per_step": ms64 / steps64, "cycles": cyc64, "dtype": "f64"},
                "speedup_fp32ir_vs_fp64": v32 / v64, "clocks": clk}

    def e2e(self, steps):
        """The same metric end to end through the C ABI: pinned host inputs in,
        solution out, host<->device copies inside the timed region."""
        import torch
        f_pin = torch.from_numpy(self.f_host).pin_memory()
        ud_pin = torch.from_numpy(self.ud_host).pin_memory()
        u_pin = torch.empty((self.n, 3), dtype=torch.float64).pin_memory()
        p_pin = torch.empty((self.n,), dtype=torch.float64).pin_memory()
        ms = 0.0
        for _ in range(steps):
            self.stream.synchronize()
            t0 = time.perf_counter()
            self.mesh.set_rhs(f_pin, ud_pin)
            self.mesh.solve(tol=TOL, max_cycles=50, mode=self.pkg.MODE_FP32_IR, u_out=u_pin, p_out=p_pin)
            ms += (time.perf_counter() - t0) * 1e3
        ms = _max_over_ranks(ms, self.world)
        del f_pin, ud_pin, u_pin, p_pin
        return {"value": self.world * self.dofs * steps / (ms / 1e3), "unit": "DoF/s",
                "h2d_bytes_per_step": int(2 * 3 * self.n * 8), "d2h_bytes_per_step": int(4 * self.n * 8)}

    def accuracy(self, fmg_reps=3):
        """Errors and FMG, against an FP64 solve to 1e-12 on the same device (the
        FP64 path matches the oracle's iterates and solutions at the levels the
        oracle can hold):
          * err_vs_oracle: the FP32+IR solution (to 1e-8) beside the plain FP64
            solve stopped at the same 1e-8 -- the stopping rule, not the
            precision, sets the pressure error;
          * fmg: full multigrid with one and two V_var(2,2) cycles per level
            (Sec. 5), device time, and gamma = ||I u - u~||_h / ||I u - u_h||_h
            with the mesh-dependent norm of Sec. 5 (I: nodal interpolant of the
            manufactured solution, u~ the FMG result, u_h the discrete solution)."""
        import torch

        import workloads as W
        pkg = self.pkg

        def solve(mode, tol):
            u = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
            p = torch.empty((self.n,), dtype=torch.float64, device="cuda")
            self.mesh.set_rhs(self.f_dev, self.ud_dev)
            _, _, st = self.mesh.solve(tol=tol, max_cycles=60, mode=mode, u_out=u, p_out=p)
            return u, p, st

        def err(a, b):
            d = a - b
            return {"max": float(d.abs().max() / b.abs().max()),
                    "rms": float(d.norm() / b.norm())}

        u_ref, p_ref, st_ref = solve(pkg.MODE_FP64, 1e-12)
        out = {"against": f"FP64 solve to 1e-12 ({st_ref.cycles} cycles) on the same GPU",
               "norms": "max: max |x - x_ref| / max |x_ref|; rms: ||x - x_ref||_2 / ||x_ref||_2, over all nodes"}
        for name, mode in (("fp32_ir", pkg.MODE_FP32_IR), ("fp64_same_tol", pkg.MODE_FP64)):
            u, p, st = solve(mode, TOL)
            out[name] = {"u": err(u, u_ref), "p": err(p, p_ref), "cycles": st.cycles,
                         "rel_residual": st.rel_residual}
            del u, p
        # FMG and gamma_l
        flags = torch.from_numpy(self.mesh.node_flags()).cuda()
        vf = (flags & 2) > 0
        act = (flags & 1) > 0
        x = self.mesh.node_coords()
        ip = torch.from_numpy(W.manufactured_pressure(x)).cuda()
        del x
        h = 1.0 / (1 << self.level)
        iu = self.ud_dev

        def hnorm2(u, p):
            return float((iu[vf] - u[vf]).square().sum() + h * h * (ip[act] - p[act]).square().sum())

        disc = hnorm2(u_ref, p_ref)
        fmg = {"discretisation_error_h": disc ** 0.5}
        for cycles, mode in ((1, pkg.MODE_FP64), (2, pkg.MODE_FP64), (1, pkg.MODE_FP32_IR), (2, pkg.MODE_FP32_IR)):
            u = torch.empty_like(u_ref)
            p = torch.empty_like(p_ref)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            best = None
            for _ in range(fmg_reps):
                torch.cuda.synchronize()
                e0.record(self.stream)
                _, _, st = self.mesh.fmg_solve(self.f_dev, self.ud_dev, cycles=cycles, nu=2, mode=mode, u_out=u,
                                               p_out=p)
                e1.record(self.stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            fmg[("V22" if cycles == 1 else "2V22") + ("_fp64" if mode == pkg.MODE_FP64 else "_fp32ir")] = {
                "ms": best, "value": self.world * self.dofs / (best / 1e3), "unit": "DoF/s",
                "gamma": (hnorm2(u, p) / disc) ** 0.5, "rel_residual": st.rel_residual, "cycles": st.cycles}
            del u, p
        # FMG as the start of the 1e-8 solve: one V_var(2,2) FMG pass with FP32
        # corrections, then FP32+IR cycles from its iterate until the residual is
        # 1e-8 of the zero start's (the bench criterion)
        best, info = None, None
        for _ in range(fmg_reps):
            torch.cuda.synchronize()
            e0.record(self.stream)
            _, _, sf = self.mesh.fmg_solve(self.f_dev, self.ud_dev, cycles=1, nu=2, mode=pkg.MODE_FP32_IR,
                                           want_solution=False)
            _, _, ss = self.mesh.solve(tol=TOL / sf.rel_residual, max_cycles=50, mode=pkg.MODE_FP32_IR,
                                       want_solution=False)
            e1.record(self.stream)
            e1.synchronize()
            if ss.status != 0:
                raise RuntimeError(f"solve from the FMG iterate did not converge: {ss}")
            ms = e0.elapsed_time(e1)
            if best is None or ms < best:
                best, info = ms, (sf.rel_residual, ss.cycles, sf.rel_residual * ss.rel_residual)
        fmg["fmg_start_to_1e-8_fp32ir"] = {
            "ms": best, "value": self.world * self.dofs / (best / 1e3), "unit": "DoF/s",
            "fmg_rel_residual": info[0], "cycles_after_fmg": info[1], "rel_residual": info[2]}
        fmg["parTME"] = self.partme(fmg)
        out_fmg = fmg
        del u_ref, p_ref
        return out, out_fmg

    def partme(self, fmg, reps=10):
        """Parallel textbook multigrid efficiency of the FMG runs (Sec. 5):
        E_parTME = t n_c mu_sm / n = t / t_WU, the FMG time in work units.  One
        work unit is one application of K to all n unknowns; with n_c = 1 GPU
        its time t_WU is that of the finest-level residual kernel ((f, g) - K
        (u, p)) in the precision of the FMG's V-cycles, so mu_sm = n / t_WU.
        "wcg" leaves out the coarse-grid solves: one before the first level and
        one per cycle, each timed alone on the coarsest level (the cycles run
        it inside the cluster-resident kernel of the coarse levels)."""
        lc, lf = self.mesh.coarsest, self.level
        t_wu = {m: self.mesh.time_op(lf, "residual", precision=pr, reps=reps) for m, pr in (("fp64", 0), ("fp32ir", 1))}
        t_cg = {m: self.mesh.time_op(lc, "coarse_solve", precision=pr, reps=reps)
                for m, pr in (("fp64", 0), ("fp32ir", 1))}
        out = {"work_unit": "one application of K on the finest level (the residual kernel), n_c = 1 GPU",
               "t_WU_ms": t_wu, "mu_sm_lups": {m: self.dofs / (t / 1e3) for m, t in t_wu.items()},
               "coarse_solve_ms": t_cg}
        for key in ("V22_fp64", "2V22_fp64", "V22_fp32ir", "2V22_fp32ir"):
            m = "fp64" if key.endswith("fp64") else "fp32ir"
            cycles = 2 if key.startswith("2") else 1
            t = fmg[key]["ms"]
            t_coarse = t_cg["fp64"] + cycles * (lf - lc) * t_cg[m]
            out[key] = {"E_parTME": t / t_wu[m], "E_parTME_wcg": (t - t_coarse) / t_wu[m]}
        return out

    def close(self):
        self.mesh.close()


def run_gpu(args):
    import torch

    import paper_1511_02134_gb300 as pkg

    world, rank, local = _dist()
    if rank == 0 and not args.no_cpu:
        # the oracle's process pool starts before any GPU call (spawned workers)
        cpu = cpu_baseline(args.cpu_seconds)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    pkg.load_library()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2

    steps64 = max(1, args.steps // 4)
    head = LevelBench(pkg, args.level, stream, flush, world)
    res = head.pair(args.steps, args.warmup, steps64, clocks=ClockSampler(local))
    e2e = head.e2e(max(1, args.steps // 4))
    err, fmg = head.accuracy()
    roofline = measure_roofline(head.mesh, args.level, stream, flush)
    dofs = head.dofs
    head.close()
    del head
    channel = channel_solve(pkg, args.channel_level, stream) if args.channel_level else None
    slip_channel = channel_solve(pkg, args.channel_level, stream, slip=True) if args.channel_level else None
    dform = dform_solve(pkg, args.dform_level, stream) if args.dform_level else None

    def side_level(level, bound):
        lb = LevelBench(pkg, level, stream, flush, world)
        r = lb.pair(args.steps, args.warmup, max(1, args.steps // 2))
        side = {"free_dofs": lb.dofs, "value": r["value"], "ms_per_step": r["ms_per_step"],
                "cycles": r["cycles"][:1], "fp64": {k: r["fp64"][k] for k in ("value", "ms_per_step")},
                "speedup_fp32ir_vs_fp64": r["speedup_fp32ir_vs_fp64"]}
        if bound:
            side["roofline"] = measure_roofline(lb.mesh, level, stream, flush, bound=bound)
        side["fp64"]["cycles"] = r["fp64"]["cycles"][:1]
        lb.close()
        return side

    extra = side_level(args.extra_level, "l2") if args.extra_level and args.extra_level != args.level else None
    small = side_level(args.small_level, None) if args.small_level and args.small_level != args.level else None

    out = {
        "metric": METRIC, "value": res["value"], "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle + f64 refinement", "data": "synthetic",
        "config": {"workload": f"unit cube, 6 Kuhn tetrahedra, level {args.level} ({dofs} free DoFs), manufactured "
                               "solution, V_var(3,3) from zero to 1e-8", "level": args.level, "free_dofs": dofs,
                   "mode": "FP32 V-cycle inside FP64 iterative refinement", "l2": "inputs larger than L2, and "
                   "flushed (256 MB write) between timed steps", "parallelism": "replicas" if world > 1 else
                   "single GPU"},
        "cycles": res["cycles"], "fp64": res["fp64"], "speedup_fp32ir_vs_fp64": res["speedup_fp32ir_vs_fp64"],
        "err_vs_oracle": err, "fmg": fmg, "roofline": roofline, "clocks": res["clocks"], "e2e": e2e,
        "gpu_launches": res["launches"],
    }
    if extra:
        out[f"level{args.extra_level}"] = extra
    if small:
        out[f"level{args.small_level}"] = small
    if channel:
        out[f"channel_level{args.channel_level}"] = channel
        out[f"slip_channel_level{args.channel_level}"] = slip_channel
    if dform:
        out[f"dform_level{args.dform_level}"] = dform
    if rank == 0:
        if not args.no_cpu:
            out["cpu_baseline"] = cpu
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def channel_solve(pkg, level, stream, reps=3, slip=False):
    """Obstacle channel (16 x 4 x 4 unit cubes, 6 seeded obstacles, inflow of
    peak 1, do-nothing outflow; the stand-in for the sphere bed of Sec. 6) at
    `level`, FP32+IR to 1e-8 from zero; coarsest level 1 with the
    tolerance-driven coarse MINRES (relative 5e-3, at most 300 iterations,
    Sec. 3.7).  slip: free-slip obstacle faces (Sec. 6.1) instead of no-slip.
    Best of `reps` device-timed set_rhs + solve steps."""
    import torch

    import workloads as W
    ch = W.slip_channel() if slip else W.obstacle_channel()
    mesh = pkg.Mesh(ch.vertices, ch.tets, ch.bc_flags, level, coarsest_level=1, coarse_minres_max=300,
                    coarse_minres_rtol=5e-3, stream=stream.cuda_stream)
    x = mesh.node_coords()
    ud = torch.from_numpy(W.channel_inflow(x)).cuda()
    del x
    dofs = mesh.free_dofs()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best, st = None, None
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        e0.record(stream)
        mesh.set_rhs(None, ud)
        _, _, st = mesh.solve(tol=TOL, max_cycles=60, mode=pkg.MODE_FP32_IR, want_solution=False)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    mesh.close()
    return {"free_dofs": dofs, "ms_per_step": best, "value": dofs / (best / 1e3), "unit": "DoF/s",
            "cycles": st.cycles, "rel_residual": st.rel_residual, "status": st.status,
            "config": "16x4x4 channel, 6 " + ("free-slip" if slip else "no-slip") +
                      " obstacle cubes, coarsest level 1, coarse MINRES 5e-3 / 300"}


def dform_solve(pkg, level, stream, reps=3):
    """The unit cube in the D-operator formulation (Sec. 2.1, a_2) beside the
    Laplace form, FP64 and FP32+IR to 1e-8, manufactured solution: best of
    `reps` device-timed set_rhs + solve steps each, and the D / Laplace time
    ratio (the paper's serial ratio for UMG is 2.10 at its level 5, Tab.
    "itertime_D_ser")."""
    import torch

    import workloads as W
    cube = W.unit_cube()
    out = {}
    for form in (0, 1):
        mesh = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, level, operator_form=form,
                        stream=stream.cuda_stream)
        f, ud = _inputs(mesh)
        f, ud = torch.from_numpy(f).cuda(), torch.from_numpy(ud).cuda()
        dofs = mesh.free_dofs()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for mode, key in ((pkg.MODE_FP64, "fp64"), (pkg.MODE_FP32_IR, "fp32ir")):
            best, st = None, None
            for _ in range(reps + 1):
                torch.cuda.synchronize()
                e0.record(stream)
                mesh.set_rhs(f, ud)
                _, _, st = mesh.solve(tol=TOL, max_cycles=60, mode=mode, want_solution=False)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[("laplace_" if form == 0 else "dform_") + key] = {
                "ms_per_step": best, "value": dofs / (best / 1e3), "unit": "DoF/s", "cycles": st.cycles}
        mesh.close()
    out["free_dofs"] = dofs
    out["time_ratio_d_over_laplace"] = {k: out["dform_" + k]["ms_per_step"] / out["laplace_" + k]["ms_per_step"]
                                        for k in ("fp64", "fp32ir")}
    return out


# ---- roofline of the dominant kernel ------------------------------------------------------------

def measure_roofline(mesh, lvl, stream, flush, bound="hbm"):
    """Roofline of the dominant kernel of the FP32 path: the velocity colour
    sweep with f - B^T p formed at each node (k_vel_colour_rhs<float>) on the
    finest level, timed with CUDA events on the mesh's stream (hhg_time_op).
    Algorithmic bytes of one forward sweep (four colour launches): u read and
    written (2 x 3 x 4 B), f (3 x 4 B), p (4 B) and the node flag (1 B) once per
    node; one colour launch carries a quarter of that."""
    import torch
    peak, peak_kind = _peaks()
    reps = 10
    with torch.cuda.stream(stream):
        flush.fill_(1.0)
    stream.synchronize()
    ms_sweep = mesh.time_op(lvl, "vel_forward_f", precision=1, reps=reps)  # 4 colour launches
    ms_launch = ms_sweep / 4.0
    nodes = mesh.num_nodes(lvl)
    alg_bytes = nodes * (2 * 3 * 4 + 3 * 4 + 4 + 1) / 4.0
    achieved = alg_bytes / (ms_launch / 1e3) / 1e9
    tb = TRAFFIC_BYTES_PER_NODE.get("k_vel_colour_rhs")
    return {"bound": bound, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None if tb is None else round(tb * nodes),
            "kernel": "k_vel_colour_rhs<float> (level %d)" % lvl, "peak_kind": peak_kind,
            "ms_per_launch": ms_launch, "alg_bytes_per_launch": alg_bytes}


def roofline_only(args):
    """Set up the workload of --level, run one FP32+IR solve and print the
    roofline measurement alone (the command the kernel profiles are taken with)."""
    import torch
    import paper_1511_02134_gb300 as pkg
    import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    cube = W.unit_cube()
    mesh = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, args.level, stream=stream.cuda_stream)
    x = mesh.node_coords()
    mesh.set_rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    del x
    mesh.solve(tol=TOL, max_cycles=50, mode=pkg.MODE_FP32_IR, want_solution=False)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    print(json.dumps(measure_roofline(mesh, args.level, stream, flush)))
    mesh.close()


def fused_pass_only(args):
    """Set up the cube of --level with the colour-fused FP32 passes on (levels
    of at least 2^20 nodes), set the manufactured right-hand side, run fused
    pass --fused-pass once and print its warm device time (the command the
    fused-pass profile is taken with)."""
    import torch
    import paper_1511_02134_gb300 as pkg
    import workloads as W
    torch.cuda.set_device(0)
    cube = W.unit_cube()
    mesh = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, args.level, fused_min_nodes=1 << 20)
    x = mesh.node_coords()
    mesh.set_rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    del x
    op = "fused_pass%d" % args.fused_pass
    mesh.level_op(args.level, op, precision=1)
    torch.cuda.synchronize()
    print(json.dumps({"kernel": "k_uzawa_pass<%d>" % args.fused_pass, "level": args.level,
                      "ms": mesh.time_op(args.level, op, precision=1, reps=3)}))
    mesh.close()


# ---- CPU oracle -----------------------------------------------------------------------------------

def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _oracle_problem(level: int):
    import workloads as W
    from oracle import multigrid as MG
    H = MG.build_hierarchy(W.unit_cube(), level)
    L = H.levels[level]
    x = L.mesh.xyz
    f, g = L.rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    return H, L, f, g


def _oracle_sample(level: int, seconds: float, problem=None):
    """Time the CPU oracle's FP64 solve (as it stands) on the cube at `level`
    until `seconds` of solve time have passed (at least one solve)."""
    from oracle import multigrid as MG
    H, L, f, g = problem or _oracle_problem(level)
    t_solve, runs, cycles = 0.0, 0, 0
    while t_solve < seconds or runs == 0:
        t0 = time.perf_counter()
        res = MG.solve(H, f, g, tol=TOL, max_cycles=50)
        t_solve += time.perf_counter() - t0
        runs += 1
        cycles = res.cycles
    return L.n_dofs * runs / t_solve, runs, cycles, L.n_dofs


def _oracle_worker(args):
    level, seconds = args
    return _oracle_sample(level, seconds)


def cpu_baseline(seconds: float, level: int = ORACLE_LEVEL):
    """The oracle on one core, and on all cores as independent solves (one
    spawned process per core, aggregate DoF/s)."""
    v, runs, cycles, dofs = _oracle_sample(level, seconds)
    cores = os.cpu_count() or 1
    v_all, procs = None, 1
    if cores > 1:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            outs = pool.map(_oracle_worker, [(level, seconds / 2)] * cores)
        v_all, procs = float(sum(o[0] for o in outs)), cores
    return {"value": v, "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": f"unit cube level {level} ({dofs} free DoFs), FP64 V_var(3,3) to 1e-8, {runs} solves "
                      f"x {cycles} cycles, numpy/scipy single thread; setup excluded",
            "all_cores": {"value": v_all, "unit": "DoF/s", "cores": procs,
                          "sample": "the same solve in one process per core, aggregate throughput"},
            "host": {"nproc": cores, "cpu_model": _cpu_model(), "machine": platform.machine()}}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    level = ORACLE_LEVEL
    problem = _oracle_problem(level)
    per = []
    for _ in range(args.warmup):
        _oracle_sample(level, 0.0, problem)
    for _ in range(args.steps):
        v, runs, cycles, dofs = _oracle_sample(level, 0.0, problem)
        per.append(v)
    value = float(np.mean(per))
    sample = (f"unit cube level {level} ({dofs} free DoFs) instead of level {args.level}: FP64 V_var(3,3) to 1e-8 "
              f"by the numpy/scipy oracle, one solve per step, single thread")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dofs / value * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"unit cube, 6 Kuhn tetrahedra, level {args.level}, manufactured solution "
                                  "(oracle on a bounded sample)", "level": level},
           "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle", "sample": sample,
                            "host": {"nproc": os.cpu_count(), "cpu_model": _cpu_model()}},
           "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=LEVEL)
    ap.add_argument("--extra-level", type=int, default=EXTRA_LEVEL,
                    help="second cube level reported beside the headline (0: none)")
    ap.add_argument("--small-level", type=int, default=4,
                    help="also time the small cube level (launch- and latency-bound); 0 = skip")
    ap.add_argument("--channel-level", type=int, default=6,
                    help="obstacle channel level reported beside the headline (0: none)")
    ap.add_argument("--dform-level", type=int, default=7,
                    help="cube level of the D-operator comparison (0: none)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--roofline-only", action="store_true",
                    help="print only the roofline measurement of the dominant kernel")
    ap.add_argument("--fused-pass", type=int, choices=[0, 1, 2], default=None,
                    help="run and time one colour-fused FP32 pass on the cube of --level and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import __graft_entry__ as g
    g.build()
    if args.fused_pass is not None:
        fused_pass_only(args)
        return
    if args.roofline_only:
        roofline_only(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
