#!/usr/bin/env python3
"""Benchmark of the surface multigrid hot path on GB300.

Workload (1M vertices): torus from a 2000 x 500 grid (R = 1, r = 0.3, 2% normal
noise), A = M + 1e-3 L, one right-hand side uniform in [-1, 1], paper-default
hierarchy (ratio 0.25, coarsest >= 500 vertices), V(2,2) multicolour
Gauss-Seidel, stop at relative residual 1e-9.

A step is one pass of the whole hot path on resident inputs: update (assembly
of A from the positions, the Galerkin hierarchy, the coarsest Cholesky) and a
solve from x = 0 to the tolerance.  value = V-cycles per second over the timed
steps (time per step = time to 1e-9 including the update).  L2 is flushed by a
256 MB write before every timed step.

The same line carries, under "configs", the other workloads of the method's
forms, each timed the same way on this GPU: the plain binary64 solve on a
perturbed icosphere split 4 times (2,562 vertices, 3 levels, to 1e-10), the
batched form (64 meshes of 10k-200k vertices x 3 right-hand sides), the mixed
precision form at 2.62M vertices (2 right-hand sides, to 1e-10), the
differentiable solve on a 400 x 400 Dirichlet disk (forward + adjoint) and
per-frame re-solves of a deforming 655k-vertex icosphere (p50 / p99), and a
3|V| system (block size 3) on a 200k-vertex torus.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--headline-only]

Under torchrun (N > 1) every rank solves its own replica of the workload (the
path of one mesh does not shard); the value adds all ranks' cycles over the
slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = dict(name="torus-2000x500-1M", nu=2000, nv=500, R=1.0, r=0.3, noise=0.02, mesh_seed=0,
                t=1e-3, rtol=1e-9, rhs_seed=1, nrhs=1)
SMALL = dict(name="torus-400x100-40k", nu=400, nv=100, R=1.0, r=0.3, noise=0.02, mesh_seed=0,
             t=1e-3, rtol=1e-9, rhs_seed=1, nrhs=1)
METRIC = "V-cycles/s at 1M verts (solve to rel. residual 1e-9, update included)"
L2_FLUSH_BYTES = 256 << 20


# DRAM traffic of the level-0 sweep from one ncu capture: dram__bytes_read.sum
# + dram__bytes_write.sum of the level-0 binary64 colour launches, per sweep
# (4 classes x 26.13 MB).  Valid only for the kernel source it was taken on;
# reported as null otherwise.
TRAFFIC_CAPTURE = dict(bytes_per_sweep=26133760 + 26132224 + 26132224 + 26131712, bytes_per_launch=26.13e6,
                       regions=(("paper_2104_13755_gb300/csrc/rowslice.cuh", "constexpr int kThreads = 256;",
                                 "}  // namespace kern"),
                                ("paper_2104_13755_gb300/csrc/kernels.cuh",
                                 "// ---------------------------------------------------------------------------\n"
                                 "// Multicolour Gauss-Seidel", "// Damped Jacobi update")),
                       sha256="35b591d3ff2b32291b12b0779e6ca50e24e0f94b60bcff874f275247a098eaa9")


def captured_traffic():
    """The captured per-sweep traffic while the source of the measured kernel
    (the sweep kernel and the row helpers it uses: fixed regions of two
    headers, hashed in order) is the one that was captured; None once it has
    changed."""
    import hashlib
    text = ""
    try:
        for path, first, last in TRAFFIC_CAPTURE["regions"]:
            with open(os.path.join(ROOT, path)) as f:
                src = f.read()
            a = src.index(first)
            text += src[a:src.index(last, a)]
    except (OSError, ValueError):
        return None
    if hashlib.sha256(text.encode()).hexdigest() != TRAFFIC_CAPTURE["sha256"]:
        return None
    return TRAFFIC_CAPTURE["bytes_per_sweep"]


# DRAM traffic of one binary64 V(2,2) cycle of the 1M-vertex torus from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum summed over every kernel
# of one plain cycle graph, caches kept warm between kernels as in a solve).
# Valid only while the kernel and layout sources are the ones captured (a hash
# over the CUDA and plan sources); null otherwise or before a capture exists.
CYCLE_TRAFFIC = dict(bytes_per_cycle=608224512 + 52605696,
                     sha256="8369f61993066303f38a6be9841634c8a90fc41adeffb43d68b59044c1c5ae8d")
CYCLE_SOURCES = ("kernels.cuh", "rowslice.cuh", "tail.cuh", "dense.cu", "device.cu", "device.hpp", "plan.hpp",
                 "plan.cpp")


def source_hash():
    """sha256 over the kernel and layout sources of the library, in name order."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2104_13755_gb300", "csrc")
    files = sorted({f for name in CYCLE_SOURCES for f in glob.glob(os.path.join(csrc, name))})
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_cycle_traffic():
    if CYCLE_TRAFFIC["bytes_per_cycle"] is None or CYCLE_TRAFFIC["sha256"] != source_hash():
        return None
    return CYCLE_TRAFFIC["bytes_per_cycle"]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_workload(w):
    V, F = synth.torus(w["nu"], w["nv"], R=w["R"], r=w["r"], noise=w["noise"], seed=w["mesh_seed"])
    b = synth.uniform_rhs(V.shape[0], nrhs=w["nrhs"], seed=w["rhs_seed"])
    return V, F, b


# ---------------------------------------------------------------------------
# algorithmic bytes (CSR figures: values + int32 column indices, row pointers)
def cycle_bytes(levels, s=8, k=1, mu=4):
    """Bytes one V(2,2) cycle must move: for every level l < H with n rows and z
    entries, A_l = z (s + 4) + 4 (n + 1); (mu_pre + mu_post) sweeps of A_l + 3 s k n,
    the residual and restriction A_l + 2 s k n + 3 (s + 4) n + s k n_c, the
    prolongation and correction 3 (s + 4) n + s k n_c + 2 s k n; the coarsest
    solve reads the two triangular inverse factors, n_H^2 binary64 values."""
    total = 0.0
    for l in range(len(levels) - 1):
        n, z = levels[l]
        nc = levels[l + 1][0]
        A = z * (s + 4) + 4 * (n + 1)
        total += mu * (A + 3 * s * k * n)
        total += A + 2 * s * k * n + 3 * (s + 4) * n + s * k * nc
        total += 3 * (s + 4) * n + s * k * nc + 2 * s * k * n
    nH = levels[-1][0]
    total += nH * nH * 8
    return total


def sweep_bytes(n, z, s=8, k=1):
    return z * (s + 4) + 4 * (n + 1) + 3 * s * k * n


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling during the timed region (200 ms period)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
def oracle_levels(V, F, t, plan, timings=None):
    """Oracle operators on the library's hierarchy; records update timings."""
    import oracle
    t0 = time.perf_counter()
    A = oracle.system_matrix(V, F, t)
    t1 = time.perf_counter()
    Ps = [plan.prolongation_csr(l) for l in range(1, plan.num_levels)]
    mats = [A]
    for P in Ps:
        mats.append(oracle.galerkin(mats[-1], P))
    t2 = time.perf_counter()
    L = oracle.cholesky(mats[-1].toarray())
    t3 = time.perf_counter()
    levels = []
    for l, P in enumerate(Ps):
        col = oracle.greedy_colouring(mats[l])
        levels.append(oracle.Level(A=mats[l], P=P, colour=col, fwd=oracle.colour_order(col),
                                   rev=oracle.colour_order(col, reverse=True)))
    levels.append(oracle.Level(A=mats[-1], L=L))
    if timings is not None:
        timings.update(assembly_s=t1 - t0, galerkin_s=t2 - t1, cholesky_s=t3 - t2, update_s=t3 - t0)
    return levels


def oracle_cycle_rate(V, F, b, w, plan, cycles_per_solve, sample_cycles):
    """Oracle V-cycles/s with the same definition as the GPU value."""
    import oracle
    tm = {}
    levels = oracle_levels(V, F, w["t"], plan, tm)
    x = np.zeros_like(b)
    t0 = time.perf_counter()
    for _ in range(sample_cycles):
        x = oracle.vcycle(levels, 0, np.ascontiguousarray(x), b, oracle.Options())
    tc = (time.perf_counter() - t0) / sample_cycles
    per_solve = tm["update_s"] + cycles_per_solve * tc
    return cycles_per_solve / per_solve, tm, tc, levels


def oracle_omp_cycle_rate(levels, b, update_s, cycles_per_solve, sample_cycles):
    """The oracle's cycle with its colour classes, residual and transfers run
    in parallel on all host cores (App. "Multi-Color Gauss Seidel"), timed on
    `sample_cycles` cycles; the update is the oracle's own (one thread)."""
    import oracle
    import oracle.omp as omp
    ol = omp.OmpLevels(levels)
    x = omp.vcycle(ol, 0, np.zeros_like(b), b, oracle.Options())  # first touch, thread start
    t0 = time.perf_counter()
    for _ in range(sample_cycles):
        x = omp.vcycle(ol, 0, x, b, oracle.Options())
    tc = (time.perf_counter() - t0) / sample_cycles
    per_solve = update_s + cycles_per_solve * tc
    return cycles_per_solve / per_solve, tc, omp.threads()


# ---------------------------------------------------------------------------
def aggregate_over_ranks(seconds, cycles, world, device=None):
    """Replicas (one independent solve per rank, no collective in the data path):
    the job's time is the slowest rank's, its cycles the sum over the ranks."""
    if world == 1:
        return seconds, cycles
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    c = torch.tensor([float(cycles)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(c.item()))


def run_ours(args, w, rank, world, local_rank):
    import torch
    import paper_2104_13755_gb300 as smg

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    V, F, b = make_workload(w)
    t0 = time.perf_counter()
    plan = smg.Plan(V, F)
    setup_s = time.perf_counter() - t0
    h = smg.Hierarchy(plan, rtol=w["rtol"], max_cycles=200)
    stream = torch.cuda.current_stream()
    Vd = torch.from_numpy(V).to(dev)
    bd = torch.from_numpy(np.ascontiguousarray(b)).to(dev)
    xd = torch.zeros_like(bd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    levels = [(plan.level_info(l)[0], plan.level_info(l)[1]) for l in range(plan.num_levels)]

    def step(precision=smg.FP64):
        xd.zero_()
        h.update_positions(Vd, w["t"])
        h.solve_async(bd, xd)

    def timed_steps(k, precision, solver=smg.VCYCLE):
        h.set_options(rtol=w["rtol"], max_cycles=200, precision=precision, solver=solver)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        cycles = []
        for i in range(k):
            flush.fill_(i)
            ev[i][0].record(stream)
            step(precision)
            ev[i][1].record(stream)
            torch.cuda.synchronize()
            info = h.solve_result()
            if info["return"] != 0:
                raise RuntimeError("solve failed: %s" % info)
            cycles.append(info["cycles"])
        return [a.elapsed_time(e) for a, e in ev], cycles

    # warm-up (graph instantiation happens here)
    for p in (smg.FP64, smg.MIXED):
        h.set_options(rtol=w["rtol"], max_cycles=200, precision=p)
        for _ in range(args.warmup):
            step(p)
            torch.cuda.synchronize()
            h.solve_result()

    if args.profile:  # one binary64 and one mixed step inside an NVTX range, then stop
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("smg_profile")
        for p in (smg.FP64, smg.MIXED):
            h.set_options(rtol=w["rtol"], max_cycles=200, precision=p)
            step(p)
            torch.cuda.synchronize()
            h.solve_result()
            # the solve graph's WHILE node hides its kernels from kernel profilers;
            # one plain cycle graph of each precision exposes them (own NVTX range each)
            torch.cuda.nvtx.range_push("smg_cycle_" + ("f64" if p == smg.FP64 else "mixed"))
            h.run_stage("cycle", precision=p)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        torch.cuda.nvtx.range_pop()
        h.close()
        return None

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    ms, cycles = timed_steps(args.steps, smg.FP64)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    total_s, cycles_total = aggregate_over_ranks(sum(ms) / 1e3, sum(cycles), world, dev)
    value = cycles_total / total_s

    # kernel launches of the timed binary64 steps, counted from the captured graphs
    h.set_options(rtol=w["rtol"], max_cycles=200, precision=smg.FP64)
    n_upd, n_solve, n_iter = h.launch_counts(w["nrhs"])
    gpu_launches = int(args.steps * (n_upd + n_solve) + sum(cycles) * n_iter)

    # mixed precision form, same steps
    ms_mx, cyc_mx = timed_steps(args.steps, smg.MIXED)
    # the cycle as a CG preconditioner (same steps; one cycle per CG iteration)
    pcg = {}
    for name, p in (("fp64", smg.FP64), ("mixed", smg.MIXED)):
        h.set_options(rtol=w["rtol"], max_cycles=200, precision=p, solver=smg.PCG)
        for _ in range(2):  # graph instantiation
            step(p)
            torch.cuda.synchronize()
            h.solve_result()
        ms_cg, it_cg = timed_steps(args.steps, p, smg.PCG)
        pcg[name] = {"time_to_tol_ms": sum(ms_cg) / len(ms_cg), "iterations_per_solve": it_cg[0],
                     "V-cycles/s": sum(it_cg) * world / (sum(ms_cg) / 1e3)}
    # App. "Ablation Study": relaxation method x mu (same hierarchy, binary64 solves)
    ablation = []
    for sm_name, sm in (("gauss-seidel", smg.GS), ("jacobi", smg.JACOBI)):
        for mu in (1, 2, 3):
            h.set_options(rtol=w["rtol"], max_cycles=400, precision=smg.FP64, mu_pre=mu, mu_post=mu, smoother=sm)
            for _ in range(2):  # graph instantiation
                step(smg.FP64)
                torch.cuda.synchronize()
                h.solve_result()
            ts, cs = [], []
            for i in range(2):
                flush.fill_(i)
                a0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                step(smg.FP64)
                e0.record(stream)
                torch.cuda.synchronize()
                info = h.solve_result()
                ts.append(a0.elapsed_time(e0))
                cs.append(info["cycles"])
            ablation.append({"smoother": sm_name, "mu": mu, "cycles": cs[0], "time_to_tol_ms": min(ts)})
    h.set_options(rtol=w["rtol"], max_cycles=200, precision=smg.FP64)

    # stage timings with CUDA events on this stream (L2 flushed before each)
    def stage_ms(stage, reps=10, count=1, **kw):
        out = []
        for i in range(reps):
            flush.fill_(i)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.run_stage(stage, count=count, **kw)
            e.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(e) / count)
        return statistics.median(out)

    n0, z0 = levels[0]
    sweep_ms = stage_ms("sweep", level=0)
    cyc64_ms = stage_ms("cycle", reps=5, count=5)
    cyc32_ms = stage_ms("cycle", reps=5, count=5, precision=smg.MIXED)
    upd_ms = stage_ms("update", reps=5)
    fac_ms = stage_ms("factor", reps=5)
    gal_ms = stage_ms("galerkin", level=0, reps=5)
    # fast parameter update (the split P^T M P + t P^T L P kept from the first call)
    h.update_t(w["t"])
    torch.cuda.synchronize()
    ut = []
    for i in range(5):
        flush.fill_(i)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.update_t(w["t"] * (1.0 + 0.1 * i), stream=stream)
        e.record(stream)
        torch.cuda.synchronize()
        ut.append(a.elapsed_time(e))
    upd_t_ms = statistics.median(ut)
    h.update_positions(Vd, w["t"])
    torch.cuda.synchronize()
    # warm per-level sweep cost (10 back-to-back forward sweeps, no flush):
    # per colour launch = time / (10 * colours)
    per_level = []
    for l in range(plan.num_levels - 1):
        ncol = plan.level_info(l)[2]
        row = {"level": l, "rows": levels[l][0], "colours": ncol}
        for name, p in (("f64", smg.FP64), ("f32", smg.MIXED)):
            h.run_stage("sweep", level=l, precision=p, count=2)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.run_stage("sweep", level=l, precision=p, count=10)
            e.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(e) / 10
            row["sweep_us_" + name] = t * 1e3
            row["per_colour_us_" + name] = t * 1e3 / max(ncol, 1)
        per_level.append(row)
    peak, peak_kind = load_peaks()
    sb = sweep_bytes(n0, z0)
    achieved = sb / (sweep_ms * 1e-3) / 1e9
    cb64 = cycle_bytes(levels, s=8)
    cb32 = cycle_bytes(levels, s=4)

    # end to end through the public API: pinned host inputs in, result out, every step
    Vh = torch.from_numpy(V).pin_memory()
    bh = torch.from_numpy(np.ascontiguousarray(b)).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    e2e_ms, e2e_cyc = [], []
    for i in range(args.steps):
        flush.fill_(i)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Vd.copy_(Vh, non_blocking=True)
        bd.copy_(bh, non_blocking=True)
        xd.zero_()
        h.update_positions(Vd, w["t"])
        h.solve_async(bd, xd)
        xh.copy_(xd, non_blocking=True)
        e.record(stream)
        torch.cuda.synchronize()
        e2e_cyc.append(h.solve_result()["cycles"])
        e2e_ms.append(a.elapsed_time(e))
    e2e_value = sum(e2e_cyc) / (sum(e2e_ms) / 1e3) * world

    res = {
        "metric": METRIC, "value": value, "unit": "V-cycles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "n_vertices": int(V.shape[0]), "faces": int(F.shape[0]),
                   "levels": [l[0] for l in levels], "nnz": [l[1] for l in levels],
                   "colours": [plan.level_info(l)[2] for l in range(plan.num_levels)],
                   "lanes_per_row_f64": [h.level_config(l)[0] for l in range(plan.num_levels - 1)],
                   "lanes_per_row_f32": [h.level_config(l)[1] for l in range(plan.num_levels - 1)],
                   "staged_sweep_f64": [h.level_staged(l)[0] for l in range(plan.num_levels - 1)],
                   "staged_sweep_f32": [h.level_staged(l)[1] for l in range(plan.num_levels - 1)],
                   "restriction": [dict(zip(("q_entries", "pt_entries", "slots", "lanes_f64", "lanes_f32"),
                                            h.level_restriction(l))) for l in range(plan.num_levels - 1)],
                   "cluster_tail_from_level": {"f64": h.cycle_config()[1], "f32": h.cycle_config()[2],
                                               "ctas": h.cycle_config()[3]},
                   "t": w["t"], "rtol": w["rtol"], "nrhs": w["nrhs"], "cycle": "V(2,2) multicolour GS",
                   "l2": "flushed by a 256 MB write before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "time_to_tol_ms": sum(ms) / len(ms),
        "cycles_per_solve": cycles[0],
        "setup_s": setup_s,
        "stages_ms": {"update": upd_ms, "update_t_fast": upd_t_ms, "galerkin_l0": gal_ms, "coarsest_factor": fac_ms,
                      "vcycle_fp64": cyc64_ms, "vcycle_mixed": cyc32_ms, "sweep_l0_fp64": sweep_ms},
        "per_level_sweeps": per_level,
        "mixed": {"value": sum(cyc_mx) * world / (sum(ms_mx) / 1e3), "ms_per_step": sum(ms_mx) / len(ms_mx),
                  "refinement_steps_per_solve": cyc_mx[0]},
        "pcg": pcg,
        "ablation": ablation,
        "roofline": {"kernel": "one binary64 V(2,2) cycle (graph of every kernel of Alg. 2 on every level, "
                               "the cluster tail and the coarsest solve)", "bound": "hbm",
                     "achieved": cb64 / (cyc64_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": cb64 / (cyc64_ms * 1e-3) / 1e9 / peak, "traffic": captured_cycle_traffic(),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum summed over the kernels "
                                       "of one plain cycle graph",
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                     "bytes_per_cycle": cb64, "cycle_us": cyc64_ms * 1e3},
        "roofline_sweep_l0": {"kernel": ("gs_colour_bulk<double,1,8> (entries staged by TMA)" if h.level_staged(0)[0]
                                         else "gs_colour<double,1,%d>" % h.level_config(0)[0])
                              + " level-0 sweep (all colour launches)", "bound": "hbm",
                              "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                              "traffic": captured_traffic(), "traffic_source": "ncu dram__bytes_read.sum + "
                              "dram__bytes_write.sum per sweep", "bytes_per_sweep": sb},
        "roofline_vcycle": {"fp64": {"bytes": cb64, "achieved": cb64 / (cyc64_ms * 1e-3) / 1e9,
                                     "frac": cb64 / (cyc64_ms * 1e-3) / 1e9 / peak},
                            "mixed_inner": {"bytes": cb32, "achieved": cb32 / (cyc32_ms * 1e-3) / 1e9,
                                            "frac": cb32 / (cyc32_ms * 1e-3) / 1e9 / peak}},
        "e2e": {"value": e2e_value, "unit": "V-cycles/s", "h2d_bytes_per_step": int(Vh.numel() * 8 + bh.numel() * 8),
                "d2h_bytes_per_step": int(xh.numel() * 8)},
        "clocks": clocks,
        "gpu_launches": gpu_launches,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, tm, tc, olev = oracle_cycle_rate(V, F, b, w, plan, cycles[0], sample_cycles=2)
        res["cpu_baseline"] = {"value": rate, "unit": "V-cycles/s", "cores": 1, "kind": "oracle",
                               "sample": "oracle update of the full workload (assembly %.1fs, Galerkin %.1fs, "
                                         "Cholesky %.1fs) + 2 V-cycles (%.2fs each), extrapolated to %d cycles"
                                         % (tm["assembly_s"], tm["galerkin_s"], tm["cholesky_s"], tc, cycles[0]),
                               "cycle_only_per_s": 1.0 / tc}
        orate, otc, nth = oracle_omp_cycle_rate(olev, b, tm["update_s"], cycles[0], sample_cycles=8)
        res["cpu_baseline_allcores"] = {
            "value": orate, "unit": "V-cycles/s", "cores": nth, "kind": "oracle, multicolour OpenMP cycle",
            "sample": "8 V-cycles of the full workload (%.1f ms each) on %d threads, plus the oracle's own update "
                      "(one thread, %.1f s), extrapolated to %d cycles" % (otc * 1e3, nth, tm["update_s"], cycles[0]),
            "cycle_only_per_s": 1.0 / otc}
    h.close()
    return res


def batch_meshes(count=64, seed=2, lo=1e4, hi=2e5):
    """Seeded batch: sizes log-uniform in [lo, hi]; even entries perturbed geodesic
    spheres (10 f^2 + 2 vertices), odd entries tori (R = 1, r = 0.3, 2% noise)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        if i % 2 == 0:
            f = max(2, int(round(np.sqrt((n - 2) / 10.0))))
            V, F = synth.perturbed_geodesic_sphere(f, seed=100 + i)
        else:
            u = max(8, int(round(np.sqrt(n * 1.0 / 0.3))))
            v = max(4, int(round(n / u)))
            V, F = synth.torus(u, v, seed=100 + i)
        out.append((V, F))
    return out


def _timed(stream, flush, fn, reps):
    """CUDA-event time (ms) of fn() on `stream` for each of `reps` runs, L2
    flushed before each."""
    import torch
    out = []
    for i in range(reps):
        flush.fill_(i)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        e.record(stream)
        torch.cuda.synchronize()
        out.append((a.elapsed_time(e), r))
    return out


def config_c1(args, dev, flush):
    """Plain binary64 solve: perturbed icosphere split 4 times (2,562 vertices,
    radius 1 + 0.1 x seeded spherical-harmonic noise), A = M + 1e-3 L, one RHS
    uniform in [-1, 1], 3 levels (ratio 0.25), V(2,2) to rel. residual 1e-10.
    Step = update + solve; the oracle solves the same system on one host thread."""
    import torch
    import oracle
    import paper_2104_13755_gb300 as smg
    V, F = synth.perturbed_icosphere(4, seed=0)
    t, rtol = 1e-3, 1e-10
    t0 = time.perf_counter()
    plan = smg.Plan(V, F, max_levels=3, min_coarse=0)
    h = smg.Hierarchy(plan, rtol=rtol, max_cycles=100, max_levels=3, min_coarse=0)
    setup_s = time.perf_counter() - t0
    n = plan.level_info(0)[0]
    b = synth.uniform_rhs(n, seed=1)
    Vd = torch.from_numpy(V).to(dev)
    bd = torch.from_numpy(b).to(dev)
    stream = torch.cuda.current_stream()

    def step():
        h.update_positions(Vd, t)
        return h.solve(bd)

    forms = {}
    for name, prec in (("f64", smg.FP64), ("mixed", smg.MIXED)):
        h.set_options(rtol=rtol, max_cycles=100, precision=prec)
        for _ in range(args.warmup):
            step()
        runs = _timed(stream, flush, step, args.steps)
        x, info = runs[-1][1]
        forms[name] = {"time_to_tol_ms": statistics.median([r[0] for r in runs]), "cycles": info["cycles"],
                       "rel_residual": info["rel_residual"], "x": x.cpu().numpy()}
    # the oracle on the same hierarchy (one host thread)
    t0 = time.perf_counter()
    A = oracle.system_matrix(V, F, t)
    levels = oracle.build_levels(A, [plan.prolongation_csr(l) for l in range(1, plan.num_levels)])
    ref = oracle.solve(levels, b, opt=oracle.Options(rtol=rtol))
    cpu_s = time.perf_counter() - t0
    for f in forms.values():
        xg = f.pop("x")
        f["max_rel_diff_vs_oracle"] = float(np.abs(xg - ref.x).max() / np.abs(ref.x).max())
    h.close()
    return {"metric": "time to rel. residual 1e-10, icosphere split 4 (2,562 vertices, update included)",
            "value": forms["f64"]["time_to_tol_ms"], "unit": "ms", "higher_is_better": False, "dtype": "f64",
            "config": {"workload": "icosphere4-2562-3levels", "n_vertices": int(V.shape[0]),
                       "levels": [plan.level_info(l)[0] for l in range(plan.num_levels)], "t": t, "rtol": rtol,
                       "l2": "flushed by a 256 MB write before every timed step"},
            "setup_s": setup_s, "forms": forms, "oracle_cycles": ref.cycles,
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": cpu_s * 1e3, "unit": "ms",
                             "sample": "the oracle's whole update (assembly, Galerkin, Cholesky) and solve to 1e-10"}}


def batch_meshes(count=64, seed=2, lo=1e4, hi=2e5):
    """Seeded batch: sizes log-uniform in [lo, hi]; even entries perturbed geodesic
    spheres (10 f^2 + 2 vertices), odd entries tori (R = 1, r = 0.3, 2% noise)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        if i % 2 == 0:
            f = max(2, int(round(np.sqrt((n - 2) / 10.0))))
            V, F = synth.perturbed_geodesic_sphere(f, seed=100 + i)
        else:
            u = max(8, int(round(np.sqrt(n * 1.0 / 0.3))))
            v = max(4, int(round(n / u)))
            V, F = synth.torus(u, v, seed=100 + i)
        out.append((V, F))
    return out


def config_c2(args, dev, flush):
    """Batched form: 64 meshes x 3 right-hand sides b = M X (implicit smoothing of the
    coordinates), A = M + 1e-2 L, coarsest <= 1000, rtol 1e-9; one graph launch
    updates all meshes and one solves them, against the same meshes one by one."""
    import concurrent.futures
    import torch
    import paper_2104_13755_gb300 as smg
    meshes = batch_meshes()
    t0 = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        plans = list(ex.map(lambda m: smg.Plan(m[0], m[1], max_coarse=1000), meshes))
    hs = [smg.Hierarchy(p, rtol=1e-9, max_cycles=200) for p in plans]
    setup_s = time.perf_counter() - t0
    Vcat = torch.from_numpy(np.concatenate([m[0] for m in meshes])).to(dev)
    batch = smg.Batch(hs)
    batch.update_positions(Vcat, 1e-2)
    bl = [h.apply_mass(torch.from_numpy(np.ascontiguousarray(m[0])).to(dev)) for h, m in zip(hs, meshes)]
    bcat = torch.cat(bl)
    stream = torch.cuda.current_stream()
    res = {}
    for name, prec in (("f64", smg.FP64), ("mixed", smg.MIXED)):
        for h in hs:
            h.set_options(rtol=1e-9, max_cycles=200, precision=prec)
        row = {}
        for mode in ("persistent", "graph"):
            batch.close()
            batch = smg.Batch(hs)
            batch.set_mode(mode)
            batch.update_positions(Vcat, 1e-2)
            for _ in range(args.warmup):
                batch.update_positions(Vcat, 1e-2)
                batch.solve(bcat)

            def bstep():
                batch.update_positions(Vcat, 1e-2)
                return batch.solve(bcat)[1]

            runs = _timed(stream, flush, bstep, args.steps)
            upd = _timed(stream, flush, lambda: batch.update_positions(Vcat, 1e-2), max(3, args.steps // 4))
            row[mode + "_ms"] = statistics.median([r[0] for r in runs])
            row[mode + "_update_ms"] = statistics.median([r[0] for r in upd])
            row[mode + "_cycles_total"] = sum(d["cycles"] for d in runs[-1][1])
        off = batch.vertex_offsets

        def sstep():
            for k, (h, b) in enumerate(zip(hs, bl)):
                h.update_positions(Vcat[off[k]:off[k + 1]], 1e-2)
                h.solve(b)

        seq = _timed(stream, flush, sstep, max(1, args.steps // 4))
        row["sequential_ms"] = statistics.median([r[0] for r in seq])
        row["batched_ms"] = row["persistent_ms"]
        row["speedup_vs_sequential"] = row["sequential_ms"] / row["persistent_ms"]
        res[name] = row
    batch.close()
    for h in hs:
        h.close()
    nv = int(sum(m[0].shape[0] for m in meshes))
    return {"metric": "batched time to rel. residual 1e-9 (64 meshes x 3 RHS, update included; one graph "
                      "launch updates all meshes, one persistent launch solves them)",
            "value": res["f64"]["batched_ms"], "unit": "ms", "higher_is_better": False, "dtype": "f64",
            "config": {"workload": "batch64-3rhs", "meshes": len(meshes), "n_vertices_total": nv,
                       "sizes": [int(m[0].shape[0]) for m in meshes], "t": 1e-2, "rtol": 1e-9,
                       "l2": "flushed by a 256 MB write before every timed step"},
            "setup_s": setup_s, "forms": res}


def config_c3(args, dev, flush):
    """Mixed-precision form at 2.62M vertices: perturbed icosphere split 9 times,
    A = M + 1e-4 L, 2 RHS uniform in [-1, 1], rtol 1e-10; each step = update +
    solve from zero, binary64 V-cycles, binary32 cycles in binary64 refinement,
    and both as CG preconditioners.  Also the level-0 binary64 sweep and the
    binary64 cycle against the measured HBM peak at a size where the level's
    matrix (~220 MB) cannot stay in L2 (L2 flushed before every timed run)."""
    import torch
    import paper_2104_13755_gb300 as smg
    V, F = synth.perturbed_icosphere(9, seed=3)
    t, rtol = 1e-4, 1e-10
    t0 = time.perf_counter()
    plan = smg.Plan(V, F)
    h = smg.Hierarchy(plan, rtol=rtol, max_cycles=300)
    setup_s = time.perf_counter() - t0
    Vd = torch.from_numpy(V).to(dev)
    bd = torch.from_numpy(synth.uniform_rhs(V.shape[0], nrhs=2, seed=7)).to(dev)
    h.update_positions(Vd, t)
    stream = torch.cuda.current_stream()
    forms, xs = {}, {}
    for name, prec, solver in (("f64", smg.FP64, smg.VCYCLE), ("mixed", smg.MIXED, smg.VCYCLE),
                               ("pcg_f64", smg.FP64, smg.PCG), ("pcg_mixed", smg.MIXED, smg.PCG)):
        h.set_options(rtol=rtol, max_cycles=300, precision=prec, solver=solver)
        for _ in range(args.warmup):
            h.update_positions(Vd, t)
            h.solve(bd)

        def step():
            h.update_positions(Vd, t)
            return h.solve(bd)

        runs = _timed(stream, flush, step, max(3, args.steps // 2))
        x, info = runs[-1][1]
        xs[name] = x.clone()
        forms[name] = {"time_to_tol_ms": statistics.median([r[0] for r in runs]), "cycles": info["cycles"],
                       "rel_residual": info["rel_residual"]}
    ref = xs["f64"]
    for name in forms:
        forms[name]["rel_diff_vs_f64"] = float((xs[name] - ref).norm() / ref.norm())
    h.set_options(rtol=rtol, max_cycles=300, precision=smg.FP64, solver=smg.VCYCLE)
    sw = [r[0] for r in _timed(stream, flush, lambda: h.run_stage("sweep", level=0, nrhs=2), 5)]
    cyc = [r[0] / 4 for r in _timed(stream, flush, lambda: h.run_stage("cycle", nrhs=2, count=4), 5)]
    n0, z0 = plan.level_info(0)[:2]
    levels = [(plan.level_info(l)[0], plan.level_info(l)[1]) for l in range(plan.num_levels)]
    peak, psrc = load_peaks()
    sweep_b = sweep_bytes(n0, z0, k=2)
    cyc_b = cycle_bytes(levels, s=8, k=2)
    achieved = sweep_b / (statistics.median(sw) / 1e3) / 1e9
    ach_c = cyc_b / (statistics.median(cyc) / 1e3) / 1e9
    h.close()
    return {"metric": "time to rel. residual 1e-10 at 2.62M verts, 2 RHS (mixed precision, update included)",
            "value": forms["mixed"]["time_to_tol_ms"], "unit": "ms", "higher_is_better": False,
            "dtype": "f32 inner / f64 outer",
            "config": {"workload": "icosphere9-2.62M-2rhs", "n_vertices": int(V.shape[0]),
                       "levels": [l[0] for l in levels], "t": t, "rtol": rtol,
                       "l2": "flushed by a 256 MB write before every timed step"},
            "setup_s": setup_s, "forms": forms,
            "roofline_sweep_l0": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak, "bytes_per_sweep": sweep_b,
                                  "sweep_us": statistics.median(sw) * 1e3, "peak_source": psrc},
            "roofline_vcycle_f64": {"bound": "hbm", "achieved": ach_c, "peak": peak, "unit": "GB/s",
                                    "frac": ach_c / peak, "bytes_per_cycle": cyc_b,
                                    "cycle_us": statistics.median(cyc) * 1e3}}


def config_c4(args, dev, flush):
    """Differentiable solve on a 400 x 400 grid mapped to the unit disk (160,000
    vertices, 1,596 Dirichlet boundary vertices), t = (mean edge length)^2:
    loss ||x||^2_M with (M + t L) x = M e_s; a step is the forward solve and
    the adjoint (a second solve and the per-face derivative kernels) giving
    the gradients in V, t and b, to rel. residual 1e-10."""
    import torch
    import paper_2104_13755_gb300 as smg
    V, F, bnd = synth.disk(400, seed=4)
    u = np.flatnonzero(~bnd)
    t = synth.mean_edge_length(V, F) ** 2
    s = int(np.random.default_rng(104).integers(u.size))
    t0 = time.perf_counter()
    plan = smg.Plan(V, F, dirichlet=bnd)
    h = smg.Hierarchy(plan, rtol=1e-10, max_cycles=200)
    setup_s = time.perf_counter() - t0
    e_s = torch.zeros(u.size, dtype=torch.float64, device=dev)
    e_s[s] = 1.0
    Vd = torch.from_numpy(V).to(dev)
    stream = torch.cuda.current_stream()

    def step():
        Vt = Vd.clone().requires_grad_(True)
        tt = torch.tensor(t, dtype=torch.float64, device=dev, requires_grad=True)
        m = smg.differentiable_mass(h, Vt)
        x = smg.differentiable_solve(h, Vt, tt, m * e_s)
        loss = (m * x * x).sum()
        loss.backward()
        return Vt.grad, tt.grad

    for _ in range(args.warmup):
        step()
    runs = _timed(stream, flush, step, max(3, args.steps // 2))
    gV, gt = runs[-1][1]
    h.close()
    return {"metric": "forward + adjoint time, 400 x 400 Dirichlet disk (gradients in V, t, b)",
            "value": statistics.median([r[0] for r in runs]), "unit": "ms", "higher_is_better": False,
            "dtype": "f64",
            "config": {"workload": "disk400-160k-dirichlet-adjoint", "n_vertices": int(V.shape[0]),
                       "unknowns": int(u.size), "t": t, "rtol": 1e-10,
                       "l2": "flushed by a 256 MB write before every timed step"},
            "setup_s": setup_s, "grad_t": float(gt.item()), "grad_V_norm": float(gV.norm().item())}


def config_c5(args, dev, flush):
    """Per-frame re-solve on a deforming mesh: perturbed icosphere split 8 times
    (655,362 vertices) moved each frame by a seeded sinusoidal displacement
    (amplitude 0.05); per frame: positions from pinned host memory to the GPU,
    assembly, Galerkin, coarsest factor, b = M(V_f) V_f (3 RHS) and a solve to
    rel. residual 1e-8 warm-started from the previous frame, in both forms.
    Latency per frame = host wall clock from the copy to the solve's status."""
    import torch
    import paper_2104_13755_gb300 as smg
    V0, F = synth.perturbed_icosphere(8, seed=5)
    t, rtol, nframes = 1e-3, 1e-8, 100
    t0 = time.perf_counter()
    plan = smg.Plan(V0, F)
    h = smg.Hierarchy(plan, rtol=rtol, max_cycles=200)
    setup_s = time.perf_counter() - t0
    Vh = torch.empty((V0.shape[0], 3), dtype=torch.float64).pin_memory()
    Vd = torch.empty((V0.shape[0], 3), dtype=torch.float64, device=dev)
    frames = [torch.from_numpy(synth.sinusoidal_displacement(V0, f, seed=11)) for f in range(nframes)]
    forms = {}
    for name, prec in (("f64", smg.FP64), ("mixed", smg.MIXED)):
        h.set_options(rtol=rtol, max_cycles=200, precision=prec)
        x = None
        lat, cyc = [], []
        for f in range(-args.warmup, nframes):
            Vh.copy_(frames[f % nframes])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Vd.copy_(Vh, non_blocking=True)
            h.update_positions(Vd, t)
            b = h.apply_mass(Vd)
            if x is None:
                x = torch.zeros_like(b)
            x, info = h.solve(b, x)
            dt = time.perf_counter() - t0
            if f >= 0:
                lat.append(dt * 1e3)
                cyc.append(info["cycles"])
        lat = np.array(lat)
        forms[name] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                       "mean_ms": float(lat.mean()), "cycles_p50": float(np.percentile(cyc, 50)),
                       "cycles_max": int(max(cyc))}
    h.close()
    return {"metric": "per-frame latency p50 (re-assembly, Galerkin, factor, warm solve to 1e-8, 3 RHS)",
            "value": forms["mixed"]["p50_ms"], "unit": "ms", "higher_is_better": False,
            "dtype": "f32 inner / f64 outer",
            "config": {"workload": "icosphere8-655k-100-frames", "n_vertices": int(V0.shape[0]), "t": t,
                       "rtol": rtol, "frames": nframes, "h2d_bytes_per_frame": int(V0.shape[0] * 24)},
            "setup_s": setup_s, "forms": forms}


def config_f3(args, dev, flush):
    """3|V| system (block size 3, Sec. 6): torus 800 x 250 (200k vertices, 600k
    unknowns), (M + 1e-3 L) (x) I_3 on the pattern of 3 x 3 blocks, one RHS
    uniform in [-1, 1], to rel. residual 1e-9, binary64 and mixed; the sweep
    runs in 3 x 3 blocks, one launch per vertex colour class.  Also the warm
    level-0 sweep."""
    import torch
    import paper_2104_13755_gb300 as smg
    V, F = synth.torus(800, 250, seed=7)
    t0 = time.perf_counter()
    plan = smg.Plan(V, F, block_size=3)
    h = smg.Hierarchy(plan, rtol=1e-9, max_cycles=200)
    setup_s = time.perf_counter() - t0
    Vd = torch.from_numpy(V).to(dev)
    n = plan.level_info(0)[0]
    bd = torch.from_numpy(synth.uniform_rhs(n, seed=3)).to(dev)
    stream = torch.cuda.current_stream()
    forms = {}
    for name, prec in (("f64", smg.FP64), ("mixed", smg.MIXED)):
        h.set_options(rtol=1e-9, max_cycles=200, precision=prec)
        for _ in range(args.warmup):
            h.update_positions(Vd, 1e-3)
            h.solve(bd)

        def step():
            h.update_positions(Vd, 1e-3)
            return h.solve(bd)

        runs = _timed(stream, flush, step, max(3, args.steps // 2))
        x, info = runs[-1][1]
        h.run_stage("sweep", level=0, precision=prec, count=2)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.run_stage("sweep", level=0, precision=prec, count=10)
        e.record(stream)
        torch.cuda.synchronize()
        forms[name] = {"time_to_tol_ms": statistics.median([r[0] for r in runs]), "cycles": info["cycles"],
                       "rel_residual": info["rel_residual"], "sweep_l0_us": a.elapsed_time(e) / 10 * 1e3}
    classes = [plan.level_info(l)[2] for l in range(plan.num_levels)]
    h.close()
    return {"metric": "time to rel. residual 1e-9, 3|V| system on a 200k-vertex torus (update included)",
            "value": forms["f64"]["time_to_tol_ms"], "unit": "ms", "higher_is_better": False, "dtype": "f64",
            "config": {"workload": "torus-800x250-block3", "n_vertices": int(V.shape[0]), "unknowns": int(n),
                       "launch_classes": classes, "t": 1e-3, "rtol": 1e-9,
                       "l2": "flushed by a 256 MB write before every timed step"},
            "setup_s": setup_s, "forms": forms}


CONFIGS = {"c1_icosphere4": config_c1, "c2_batch64": config_c2, "c3_icosphere9_mixed": config_c3,
           "c4_disk400_adjoint": config_c4, "c5_frames655": config_c5, "f3_block3_torus600k": config_f3}
WORKLOAD_FLAGS = {"ico2562": "c1_icosphere4", "batch64": "c2_batch64", "ico262": "c3_icosphere9_mixed",
                  "disk160": "c4_disk400_adjoint", "frames655": "c5_frames655", "block3": "f3_block3_torus600k"}


def run_configs(args, local_rank, names):
    import torch
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    out = {}
    for name in names:
        t0 = time.perf_counter()
        out[name] = CONFIGS[name](args, dev, flush)
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def run_reference(args, w, rank, world):
    """The oracle as it stands, on the host cores, same metric and workload."""
    if rank != 0:
        return None
    import paper_2104_13755_gb300 as smg
    import oracle
    V, F, b = make_workload(w)
    plan = smg.Plan(V, F)  # the hierarchy P_1..P_H (host setup, no GPU), which the oracle takes as data
    tm = {}
    levels = oracle_levels(V, F, w["t"], plan, tm)
    ref = oracle.solve(levels, b, opt=oracle.Options(rtol=w["rtol"], max_cycles=200))
    C = ref.cycles
    x = np.zeros_like(b)
    for _ in range(args.warmup):
        x = oracle.vcycle(levels, 0, np.ascontiguousarray(x), b, oracle.Options())
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        x = oracle.vcycle(levels, 0, np.ascontiguousarray(x), b, oracle.Options())
        times.append(time.perf_counter() - t0)
    tc = statistics.mean(times)
    per_solve = tm["update_s"] + C * tc
    value = C / per_solve
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "V-cycles/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_solve * 1e3 / C,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w["name"], "n_vertices": int(V.shape[0]), "t": w["t"], "rtol": w["rtol"],
                       "parallelism": "host, 1 thread"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": "V-cycles/s",
                             "sample": "each step one oracle V-cycle of the full workload; the oracle update "
                                       "(%.1f s) is measured once and amortised over the %d cycles of its own "
                                       "solve to 1e-9" % (tm["update_s"], C)},
            "e2e": {"value": value, "unit": "V-cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--small", action="store_true", help="40k-vertex torus (profiling captures)")
    ap.add_argument("--workload", default="torus1m", choices=["torus1m"] + sorted(WORKLOAD_FLAGS),
                    help="torus1m: the headline line (with every other workload under \"configs\"); "
                         "ico2562, batch64, ico262, disk160, frames655, block3: one of those workloads on its own line")
    ap.add_argument("--headline-only", action="store_true", help="the 1M-vertex torus line without \"configs\"")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="run one step of each precision inside the NVTX range smg_profile and exit")
    ap.add_argument("--lanes", default=None,
                    help="lanes per matrix row per level, e.g. 1,2,4,8,8 (skips the autotuner; for profiling)")
    ap.add_argument("--lanes-f32", default=None, help="the same for the binary32 kernels (with --lanes)")
    ap.add_argument("--rq-lanes", default=None, help="lanes per row of the fused restriction, per level (with --lanes)")
    ap.add_argument("--rq-lanes-f32", default=None, help="the same for binary32 (with --lanes)")
    ap.add_argument("--staged", default=None,
                    help="per level 1 = one lane per row with TMA-staged entries, e.g. 1,0,0,0,0 (with --lanes)")
    ap.add_argument("--staged-f32", default=None, help="the same for binary32 (with --lanes)")
    ap.add_argument("--tail", default=None, help="first level of the cluster tail (skips its tuning; for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    w = SMALL if args.small else WORKLOAD
    if args.lanes:
        os.environ["SMG_LANES_PER_ROW"] = args.lanes
        for flag, var in ((args.lanes_f32, "SMG_LANES_PER_ROW_F32"), (args.rq_lanes, "SMG_RQ_LANES"),
                          (args.rq_lanes_f32, "SMG_RQ_LANES_F32"), (args.staged, "SMG_STAGED_GS"),
                          (args.staged_f32, "SMG_STAGED_GS_F32")):
            if flag:
                os.environ[var] = flag
    if args.tail:
        os.environ["SMG_TAIL_LEVEL"] = args.tail
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, w, rank, world)
    elif args.workload != "torus1m":
        name = WORKLOAD_FLAGS[args.workload]
        res = dict(run_configs(args, local_rank, [name])[name], n_gpus=world, steps=args.steps,
                   warmup=args.warmup, scaling="weak", vs_baseline=None, data="synthetic")
        res["ms_per_step"] = res["value"]
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        res = run_ours(args, w, rank, world, local_rank)
        if res is not None and world == 1 and not args.headline_only and not args.small:
            # the other workloads, each on this rank's GPU (replicas under torchrun)
            res["configs"] = run_configs(args, local_rank, list(CONFIGS))
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if rank == 0 and res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
