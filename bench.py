#!/usr/bin/env python
"""Benchmark: DOF/s to 1e-10 relative residual for the ghost-FEM multigrid
solve on one GB300 (fp32 V-cycle inside fp64 iterative refinement, with the
plain fp64 V-cycle beside it), and the HBM roofline fraction of the dominant
kernel.

A step is one mg_solve of the flower problem (r - 0.3 - 0.1 sin 5 theta on
[-0.5, 0.5]^2, 4096^2 cells, u = sin 3x cos 2y) from u = 0 until
||F - A u||_inf / ||F||_inf <= 1e-10, with f, g, u resident in HBM.  L2 is
flushed (a 512 MB write) between steps, outside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The line's "batched" object times the batched workload: 256 seeded
geometries of uneven size solved together by one graph launch (the
persistent batch kernel), beside the same members solved one by one; its
"large" object the 8192^2 three-disc problem in both precisions.

Under torchrun with N > 1 every rank solves its own replica (no collective
on the data path); value = the DOFs all ranks solved / the slowest rank's
time.  ``--impl reference`` times the CPU oracle on a bounded sample of the
same workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF/s to 1e-10 rel. residual (mixed vs FP64 V-cycle, 1 GB300); % HBM roofline"
UNIT = "DOF/s"
TOL = 1e-10

# algorithmic bytes per fine-level DOF moved by one launch of each kernel:
# the method must read u, F and one byte of node class and write u (sweep);
# restriction writes a quarter-size coarse array, prolongation reads one.
ALGO_BYTES = {
    ("sweep", "f32"): 4 + 4 + 1 + 4,
    ("sweep", "f64"): 8 + 8 + 1 + 8,
    ("restrict", "f32"): 4 + 4 + 1 + 1,
    ("restrict", "f64"): 8 + 8 + 1 + 2,
    ("prolong", "f32"): 4 + 4 + 1 + 1,
    ("prolong", "f64"): 8 + 8 + 1 + 2,
    ("residual", "mixed"): 8 + 8 + 1 + 4,     # fp64 u, F in; fp32 scaled r out
    ("residual", "f64"): 8 + 8 + 1,
    ("update", "mixed"): 8 + 4 + 1 + 8,       # u64 in, e32 in, u64 out
}
# one extra-sweep launch per boundary node: u read and written, F, its row
BAND_BYTES = 4 + 4 + 4 + 4 * 10
# a mixed refinement cycle over all levels (fp32 V(2,1) ~ 80 B, fp64
# residual and update ~ 40 B per fine DOF)
SOLVE_BYTES_PER_DOF_CYCLE = 120


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--inner", type=int, default=0,
                    help="V-cycles between fp64 residual checks (0: adaptive)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="setup and one untimed mixed solve (for single-kernel profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched workload (256 seeded geometries)")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--no-small", action="store_true",
                    help="skip the 64^2 circle and the 512^2 adjoint workloads")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large workload (three discs, 8192^2 cells)")
    ap.add_argument("--large-N", type=int, default=8192)
    ap.add_argument("--profile-batch", action="store_true",
                    help="setup and two solves of the batched workload, untimed (for ncu)")
    ap.add_argument("--batch-shape", default="",
                    help="threads,first_group,cluster,coop_min_dof for --profile-batch")
    return ap.parse_args(argv)


def parse():
    return parse_args()


def workload_name(N):
    return f"flower r-0.3-0.1sin(5theta) on [-0.5,0.5]^2, {N}x{N} cells, u=sin3x cos2y"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic(kernel_tag, kind=None):
    """DRAM bytes per launch from the committed ncu summary
    profiles/<kernel_tag>.md, if every source file it lists still has the
    hash recorded there (a change to any of them voids the figure)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    try:
        txt = open(path).read()
        srcs = re.findall(r"source: `([^`]+)`\s*\n\s*source_sha256:\s*([0-9a-f]{64})", txt)
        t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
        if not srcs or not t:
            return None
        for rel, want in srcs:
            got = hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()
            if got != want:
                return None
        return float(t.group(1))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_hierarchy(N):
    """The oracle's system and hierarchy for the flower at N cells per side
    (assembly and Galerkin products in Python: setup, never timed)."""
    from oracle import ghostfem as gf
    from oracle import multigrid as mg
    from paper_2505_05105_gb300 import workloads as wl
    p = wl.flower(N)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s)
    return p, s, lev, s.rhs(p.f, p.g)


def cpu_vcycle(lev, F, threads, steps, warmup, tol=TOL):
    """Time the oracle's 4-colour V(2,1) (eta = 4) solve from u = 0 to tol in
    its plain-C OpenMP restatement (oracle/vcycle.c) with `threads` threads
    (0: all cores).  Returns (seconds per solve, cycles, threads used, u)."""
    from oracle import cvcycle
    C = cvcycle.CVCycle(lev)
    times, cyc, u = [], 0, None
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        u, hist, cyc = C.solve(F, tol=tol, threads=threads)
        dt = time.perf_counter() - t0
        if k >= warmup:
            times.append(dt)
    used = cvcycle.CVCycle.threads(threads)
    C.close()
    return statistics.mean(times), cyc, used, u


def host_info():
    """nproc and the CPU model of this host (/proc/cpuinfo: "model name" on
    x86, the implementer / part codes on Arm)."""
    import platform
    info = {"nproc": os.cpu_count(), "machine": platform.machine()}
    try:
        fields = {}
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = (x.strip() for x in line.split(":", 1))
                fields.setdefault(k, v)
        info["cpu_model"] = fields.get("model name") or " ".join(
            f"{k} {fields[k]}" for k in ("CPU implementer", "CPU part") if k in fields) or None
    except OSError:
        info["cpu_model"] = None
    return info


def sparse_direct_sample(N):
    """SciPy's sparse LU (SuperLU) solve of the flower system at N cells per
    side, assembly and factorisation of the oracle's matrix included (the
    direct alternative the paper sets against multigrid)."""
    from oracle import ghostfem as gf
    from paper_2505_05105_gb300 import workloads as wl
    p = wl.flower(N)
    s = gf.assemble_problem(p)
    F = s.rhs(p.f, p.g)
    t0 = time.perf_counter()
    gf.direct_solve(s, F, refine=0)
    dt = time.perf_counter() - t0
    ndof = int(s.dof.sum())
    return {"N": N, "value": ndof / dt, "unit": UNIT, "seconds": dt, "n_dof": ndof,
            "kind": "SciPy sparse LU of the oracle's matrix (factorisation and solve), 1 core"}


def max_over_ranks(x, dist, device):
    """The slowest rank's value of a time (all ranks get it); x itself on
    one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, ndof, steps, seconds):
    """Whole-job throughput: the DOFs all ranks solved over the slowest
    rank's time (each rank solves its own replica: weak scaling)."""
    return world * ndof * steps / seconds


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    N = args.N
    steps = max(1, args.steps)
    warm = max(0, args.warmup)
    p, s, lev, F = oracle_hierarchy(N)
    ndof = int(s.dof.sum())
    sec, cyc, cores, _ = cpu_vcycle(lev, F, 0, steps, warm)
    val = ndof / sec
    sample = (f"the whole {N}x{N} flower workload ({ndof} DOFs): full fp64 4-colour V(2,1) "
              f"solve from u = 0 to 1e-10 ({cyc} cycles) per step, by the oracle's V-cycle in "
              f"plain C with OpenMP (oracle/vcycle.c) on {cores} host threads; assembly and "
              f"hierarchy (Python) excluded")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
        "n_gpus": args.gpus, "steps": steps, "warmup": warm, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(N), "N": N, "n_dof": ndof, "tol": TOL},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample, "host": host_info()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_2505_05105_gb300 import ghostmg, workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ghostmg.load()

    N = args.N
    p = wl.flower(N)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(dev)
    psi, f, g = t(p.psi), t(p.f), t(p.g)
    stream = torch.cuda.current_stream(dev)
    solvers = {
        "mixed": ghostmg.Solver(psi, N, p.x0, p.y0, p.h, precision="mixed",
                                inner=args.inner, stream=stream.cuda_stream),
        "fp64": ghostmg.Solver(psi, N, p.x0, p.y0, p.h, precision="fp64",
                               stream=stream.cuda_stream),
    }
    n_levels, ndof, ncut, nbnd = solvers["mixed"].counts()
    u = torch.zeros_like(f)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(S, steps, warm, prof=False):
        for _ in range(warm):
            u.zero_()
            S.solve(f, g, u, tol=TOL)
        if prof:
            ghostmg.mg_set_profiling(S.handle, True)
        ms, cycles = [], []
        barrier()
        for k in range(steps):
            u.zero_()
            flush.fill_(float(k))               # evict L2 (512 MB write), untimed
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = S.solve(f, g, u, tol=TOL)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            cycles.append(info.cycles)
        barrier()
        prof_out = ghostmg.mg_get_profile(S.handle) if prof else None
        if prof:
            ghostmg.mg_set_profiling(S.handle, False)
        total = max_over_ranks(sum(ms), dist, dev)
        return total, ms, cycles, prof_out, info

    with ClockSampler(local) as clk:
        total_mx, ms_mx, cyc_mx, _, info_mx = timed(solvers["mixed"], args.steps, args.warmup)
        # per-launch CUDA events serialise the launches (no programmatic
        # overlap) and add their own cost, so the kernel breakdown and the
        # roofline come from a second pass of the same K solves, not from the
        # headline one
        _, _, _, prof, _ = timed(solvers["mixed"], args.steps, 0, prof=True)
        u_mixed = u.cpu().numpy().copy()
        total_64, ms_64, cyc_64, _, info_64 = timed(solvers["fp64"], args.steps, args.warmup)
        u_fp64 = u.cpu().numpy().copy()
        batched = None
        if not args.no_batched and world == 1:
            batched = run_batched(args, dev, flush)
        large = None
        if not args.no_large and world == 1:
            large = run_large(args, dev, flush, stream)
        small = adjoint = None
        if world == 1 and not args.no_small:
            small = run_small(args, dev, stream)
            adjoint = run_adjoint(args, dev, stream)
    clocks = clk.summary()

    value = job_value(world, ndof, args.steps, total_mx / 1e3)
    value64 = job_value(world, ndof, args.steps, total_64 / 1e3)

    # roofline: every kernel class timed live (CUDA events around each launch
    # on the solver's stream, second pass), its algorithmic bytes per launch,
    # and the dominant class (most device time) as the line's "roofline"
    launches, slots = prof
    peak, peak_src = measured_peaks()
    H = solvers["mixed"].handle
    lev_dofs = [ghostmg.mg_level_dofs(H, l) for l in range(n_levels)]
    inter = sum(lev_dofs[1:-1])          # the levels between the finest and the coarsest
    per_launch_bytes = {
        "sweep": ALGO_BYTES[("sweep", "f32")] * ndof,
        "band": BAND_BYTES * nbnd,
        "restrict": ALGO_BYTES[("restrict", "f32")] * ndof,
        "residual": ALGO_BYTES[("residual", "mixed")] * ndof,
        "update": ALGO_BYTES[("update", "mixed")] * ndof,
    }
    cycles_prof = sum(cyc_mx) / len(cyc_mx) * args.steps
    # the intermediate levels' kernels (separate, fused, tail) per V-cycle:
    # three sweeps and one residual + restriction of each level's DOFs
    per_step_bytes_coarse = (3 * ALGO_BYTES[("sweep", "f32")] + ALGO_BYTES[("restrict", "f32")]) \
        * inter * cycles_prof / args.steps
    kernel_roofline = {}
    total_ms = sum(v[1] for v in slots.values())
    for k, (n_l, ms) in slots.items():
        if n_l == 0 or ms <= 0:
            continue
        ent = {"launch_groups": n_l, "ms_per_step": ms / args.steps,
               "share": ms / total_ms, "avg_launch_us": ms / n_l * 1e3}
        if k in per_launch_bytes:
            gbs = per_launch_bytes[k] / (ms / n_l / 1e3) / 1e9
            ent.update({"algorithmic_bytes_per_launch": per_launch_bytes[k],
                        "achieved_gbs": gbs, "frac": gbs / peak})
        kernel_roofline[k] = ent
    coarse_cls = ("levels", "levels_band", "levels_restrict", "fused", "tail", "coarse")
    coarse_ms = sum(slots[k][1] for k in coarse_cls if k in slots)
    if coarse_ms > 0:
        gbs = per_step_bytes_coarse / (coarse_ms / args.steps / 1e3) / 1e9
        kernel_roofline["intermediate_levels_all"] = {
            "classes": list(coarse_cls),
            "algorithmic_bytes_per_step": per_step_bytes_coarse, "achieved_gbs": gbs,
            "frac": gbs / peak, "level_dofs": lev_dofs}
    # the dominant kernel: device time per kernel function over all the
    # levels it runs on; its roofline is that of its largest (fine-level)
    # launches, whose bytes are modelled and whose traffic ncu measured
    kernel_classes = {"k_gs_sweep_f32": ("sweep", "levels"),
                      "k_band<float>": ("band", "levels_band"),
                      "k_resid_restrict_f32": ("restrict", "levels_restrict"),
                      "k_smooth_step": ("fused",), "k_tail<float>": ("tail",),
                      "k_residual<double,float>": ("residual",), "k_update": ("update",),
                      "k_rhs, k_pack, k_unpack": ("io",), "k_prolong": ("prolong",),
                      "coarsest solve": ("coarse",)}
    kernel_ms = {kn: sum(slots[c][1] for c in cls if c in slots)
                 for kn, cls in kernel_classes.items()}
    dom_kernel = max(kernel_ms, key=kernel_ms.get)
    dom = next((c for c in kernel_classes[dom_kernel] if c in slots and slots[c][0] > 0),
               kernel_classes[dom_kernel][0])
    n_launch, dom_ms = slots[dom]
    per_launch_s = dom_ms / n_launch / 1e3
    names = {"sweep": "k_gs_sweep_f32 (fine level)", "band": "k_band<float> (fine level)",
             "restrict": "k_resid_restrict_f32 (fine level)",
             "residual": "k_residual<double,float> (fp64 refinement residual)",
             "update": "k_update", "levels": "k_gs_sweep_f32 (intermediate levels)",
             "levels_band": "k_band<float> (intermediate levels)",
             "levels_restrict": "k_resid_restrict_f32 (intermediate levels)",
             "fused": "k_smooth_step (fused smoothing steps)", "tail": "k_tail<float>",
             "coarse": "coarsest solve", "io": "right-hand side, pack, unpack",
             "prolong": "k_prolong"}
    if dom in per_launch_bytes:
        algo = per_launch_bytes[dom]
        bound = "hbm"
    else:
        # the intermediate levels' share of the algorithmic bytes over this class's time
        algo = per_step_bytes_coarse * (dom_ms / coarse_ms) / (n_launch / args.steps)
        bound = "hbm"
    achieved = algo / per_launch_s / 1e9
    traffic = profile_traffic(f"{dom}_f32_flower{N}", dom)
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": names.get(dom, dom),
                "class": dom, "dominant_kernel": dom_kernel,
                "dominant_kernel_share": kernel_ms[dom_kernel] / total_ms,
                "kernel_ms_per_step": {k: v / args.steps for k, v in kernel_ms.items() if v > 0},
                "algorithmic_bytes_per_launch": algo, "launches": n_launch,
                "avg_launch_us": per_launch_s * 1e6, "peak_source": f"{peak_src} hbm_gbs",
                "timing": f"CUDA events around each launch on the solver stream, over {args.steps} "
                          "profiled solves run after the timed ones"}
    # the whole solve against the HBM roofline: 120 B per fine DOF and mixed
    # refinement cycle (fp32 V(2,1) over all levels plus the fp64 residual
    # and update)
    solve_level = {"algorithmic_bytes_per_dof_cycle": SOLVE_BYTES_PER_DOF_CYCLE,
                   "cycles_per_solve": cyc_mx[-1],
                   "achieved_gbs": SOLVE_BYTES_PER_DOF_CYCLE * cyc_mx[-1] * ndof
                   / (total_mx / args.steps / 1e3) / 1e9}
    solve_level["frac"] = solve_level["achieved_gbs"] / peak
    breakdown = {k: {"launch_groups": v[0], "ms_per_step": v[1] / args.steps}
                 for k, v in slots.items()}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        fh = torch.from_numpy(np.ascontiguousarray(p.f, dtype=np.float64).ravel()).pin_memory()
        gh = torch.from_numpy(np.ascontiguousarray(p.g, dtype=np.float64).ravel()).pin_memory()
        uh = torch.zeros(fh.numel(), dtype=torch.float64).pin_memory()
        S = solvers["mixed"]
        for _ in range(max(1, args.warmup)):
            uh.zero_()
            S.solve(fh.data_ptr(), gh.data_ptr(), uh.data_ptr(), tol=TOL)
        barrier()
        tot = 0.0
        for k in range(args.steps):
            uh.zero_()
            flush.fill_(float(k))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            S.solve(fh.data_ptr(), gh.data_ptr(), uh.data_ptr(), tol=TOL)
            tot += time.perf_counter() - t0
        barrier()
        tot = max_over_ranks(tot, dist, dev)
        nb = fh.numel() * 8
        e2e = {"value": job_value(world, ndof, args.steps, tot), "unit": UNIT,
               "h2d_bytes_per_step": 3 * nb, "d2h_bytes_per_step": nb,
               "transfer": "pinned host f, g, u read and written in place by the kernels "
                           "(f at active-cell vertices, g at cut-cell vertices, u at DOFs; "
                           "all of u written); bytes above are the arrays' sizes"}

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the oracle's V-cycle in plain C (oracle/vcycle.c) on the same
        # workload, on one host thread and on all of them
        _, s_o, lev_o, F_o = oracle_hierarchy(N)
        sec_all, cyc_o, cores, _ = cpu_vcycle(lev_o, F_o, 0, steps=2, warmup=1)
        sec_one, _, _, _ = cpu_vcycle(lev_o, F_o, 1, steps=1, warmup=0)
        odof = int(s_o.dof.sum())
        cpu = {"value": odof / sec_all, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"the whole {N}x{N} flower workload ({odof} DOFs): full fp64 4-colour "
                         f"V(2,1) solve from u = 0 to 1e-10 ({cyc_o} cycles), the oracle's "
                         f"V-cycle in plain C with OpenMP (oracle/vcycle.c), {cores} threads; "
                         f"assembly and hierarchy (Python) excluded",
               "one_thread": {"value": odof / sec_one, "unit": UNIT, "seconds": sec_one},
               "all_threads": {"value": odof / sec_all, "unit": UNIT, "seconds": sec_all,
                               "threads": cores},
               "host": host_info(), "sparse_direct": sparse_direct_sample(1024)}
        # error of the GPU results against the fp64 oracle: its V-cycle
        # driven to the attainable residual (2e-15)
        _, _, _, u_ref = cpu_vcycle(lev_o, F_o, 0, steps=1, warmup=0, tol=2e-15)
        scale = float(np.abs(u_ref).max())
        accuracy = {"reference": "the oracle's fp64 4-colour V(2,1) solution of the same "
                                 "system driven to ||F - Au||_inf/||F||_inf <= 2e-15",
                    "mixed_max_rel_error": float(np.abs(u_mixed - u_ref).max()) / scale,
                    "fp64_max_rel_error": float(np.abs(u_fp64 - u_ref).max()) / scale,
                    "mixed_rel_res": info_mx.rel_res, "fp64_rel_res": info_64.rel_res}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_mx / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle in f64 refinement",
            "data": "synthetic",
            "config": {"workload": workload_name(N), "N": N, "n_dof": ndof, "n_cut": ncut,
                       "n_levels": n_levels, "tol": TOL, "precision": "mixed",
                       "cycles_per_solve": cyc_mx[-1], "V": "V(2,1), eta=4, gamma=2",
                       "cycles_between_fp64_checks": args.inner or "adaptive",
                       "fp64_checks_per_solve": info_mx.checks,
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{world}"},
            "fp64": {"value": value64, "unit": UNIT, "ms_per_step": total_64 / args.steps,
                     "cycles_per_solve": cyc_64[-1], "dtype": "f64"},
            "mixed_over_fp64": value / value64,
            "roofline": roofline,
            "kernel_roofline": kernel_roofline,
            "solve_roofline": solve_level,
            "kernel_breakdown_mixed": breakdown,
            "batched": batched,
            "large": large,
            "small_circle64": small,
            "adjoint_flower512": adjoint,
            "cpu_baseline": cpu,
            "accuracy": accuracy,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    for S in solvers.values():
        S.close()
    if dist is not None:
        dist.destroy_process_group()


def run_large(args, dev, flush, stream):
    """The large workload: the union of three seeded discs minus a small
    disc (several cut features), random Fourier f, g = 0, at 8192^2 cells;
    mixed precision and plain fp64 solves from u = 0 to 1e-10, timed as the
    headline (CUDA events on the solver's stream, L2 flushed between
    steps), and the fine fp32 sweep's share and bandwidth from a profiled
    pass."""
    import numpy as np
    import torch
    from paper_2505_05105_gb300 import ghostmg, workloads as wl
    N = args.large_N
    p = wl.three_discs(N, seed=0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(dev)
    psi, f, g = t(p.psi), t(p.f), t(p.g)
    u = torch.zeros_like(f)
    out = {"workload": f"three discs minus a disc (seed 0), random Fourier f, g=0, {N}^2 cells"}
    for prec in ("mixed", "fp64"):
        S = ghostmg.Solver(psi, N, p.x0, p.y0, p.h, precision=prec, stream=stream.cuda_stream)
        ndof = S.counts()[1]
        for _ in range(max(1, args.warmup)):
            u.zero_()
            S.solve(f, g, u, tol=TOL, allow_not_converged=True)
        steps = max(1, min(args.steps, 3))
        ms = []
        for k in range(steps):
            u.zero_()
            flush.fill_(float(k))
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = S.solve(f, g, u, tol=TOL, allow_not_converged=True)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        ent = {"value": ndof * steps / (sum(ms) / 1e3), "unit": UNIT,
               "ms_per_step": sum(ms) / steps, "cycles_per_solve": info.cycles,
               "rel_res": info.rel_res, "converged": info.rel_res <= TOL, "steps": steps}
        if prec == "mixed":
            ghostmg.mg_set_profiling(S.handle, True)
            u.zero_()
            S.solve(f, g, u, tol=TOL, allow_not_converged=True)
            _, slots = ghostmg.mg_get_profile(S.handle)
            ghostmg.mg_set_profiling(S.handle, False)
            n_l, sweep_ms = slots["sweep"]
            if n_l:
                algo = ALGO_BYTES[("sweep", "f32")] * ndof
                peak, src = measured_peaks()
                gbs = algo / (sweep_ms / n_l / 1e3) / 1e9
                ent["sweep_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak,
                                         "unit": "GB/s", "frac": gbs / peak,
                                         "avg_launch_us": sweep_ms / n_l * 1e3,
                                         "peak_source": f"{src} hbm_gbs"}
            out["n_dof"] = ndof
            out["n_cut"] = S.counts()[2]
        out[prec] = ent
        S.close()
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def run_small(args, dev, stream):
    """The circle at 64^2 (2157 DOFs; plain fp64 V(2,1), f = 0, g = u): a
    launch-latency-bound solve, by mg_solve (stream-ordered launches with a
    host residual check after each group of cycles: no graph) and as a
    one-member batch (mixed precision, the whole solve one CUDA graph)."""
    import numpy as np
    import torch
    from paper_2505_05105_gb300 import ghostmg, workloads as wl
    p = wl.circle64(64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(dev)
    psi, f, g = t(p.psi), t(p.f), t(p.g)
    u = torch.zeros_like(f)
    steps = max(5, args.steps)
    out = {"workload": "circle sqrt((x-.02)^2+(y-.01)^2)-.39, 64^2 cells, u=e^x sin y, f=0, g=u"}
    S = ghostmg.Solver(psi, 64, p.x0, p.y0, p.h, precision="fp64", stream=stream.cuda_stream)
    ndof = S.counts()[1]
    for _ in range(3):
        u.zero_()
        S.solve(f, g, u, tol=TOL)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        u.zero_()
        info = S.solve(f, g, u, tol=TOL)
    torch.cuda.synchronize(dev)
    sec = (time.perf_counter() - t0) / steps
    out["n_dof"] = ndof
    out["fp64_mg_solve"] = {"value": ndof / sec, "unit": UNIT, "ms_per_step": sec * 1e3,
                            "cycles_per_solve": info.cycles, "graph": False,
                            "timing": "wall clock around mg_solve, which returns with u written"}
    S.close()
    B = ghostmg.BatchSolver([p])
    f0, g0, u0 = B.buffers()
    f0.copy_(f)
    g0.copy_(g)
    for _ in range(3):
        B.solve(f0, g0, u0, tol=TOL)
    ms = []
    for _ in range(steps):
        info_b = B.solve(f0, g0, u0, tol=TOL)
        ms.append(B.timing()[1])
    out["mixed_one_graph"] = {"value": ndof / (statistics.mean(ms) / 1e3), "unit": UNIT,
                              "ms_per_step": statistics.mean(ms), "graph": True,
                              "cycles_per_solve": info_b[0].cycles,
                              "timing": "CUDA events around the graph launch"}
    B.close()
    return out


def run_adjoint(args, dev, stream):
    """The adjoint workload: flower 512^2, one forward fp64 solve to 1e-10,
    then 16 adjoints (L = 1/2 sum over internal nodes of (u - u_t)^2, u_t
    seeded) by mg_adjoint: transposed fp64 V-cycles to the solve's tolerance,
    then dL/df = M^T w and dL/dg = G^T w."""
    import numpy as np
    import torch
    from paper_2505_05105_gb300 import ghostmg, workloads as wl
    p = wl.flower(512)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(dev)
    f, g = t(p.f), t(p.g)
    S = ghostmg.Solver(t(p.psi), 512, p.x0, p.y0, p.h, precision="fp64",
                       stream=stream.cuda_stream)
    ndof = S.counts()[1]
    u = torch.zeros_like(f)
    S.solve(f, g, u, tol=TOL)
    inside = t((np.ravel(p.psi) < 0).astype(float))
    dLdu = [(u - t(wl.adjoint_target(p, seed))) * inside for seed in range(16)]
    dLdf, dLdg = torch.zeros_like(u), torch.zeros_like(u)
    S.adjoint(dLdu[0], dLdf, dLdg)                 # warm-up
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for d in dLdu:
        S.adjoint(d, dLdf, dLdg)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    S.close()
    return {"workload": "flower 512^2, 16 adjoints of L = 1/2 sum_internal (u - u_t)^2 "
                        "(seeded targets), fp64, to 1e-10",
            "n_dof": ndof, "members": 16, "value": 16 * ndof / (ms / 1e3), "unit": UNIT,
            "ms_per_adjoint": ms / 16,
            "timing": "CUDA events around the 16 mg_adjoint calls on the solver's stream"}


def batch_members(count):
    from paper_2505_05105_gb300 import workloads as wl
    return [wl.batch_geometry(i, seed=0) for i in range(count)]


def run_batched(args, dev, flush):
    """The batched workload: `count` seeded geometries (ellipses and flowers,
    N in {64, 128, 256, 512}, random Fourier f, g = 0) solved together to
    1e-10 by one graph launch per step (mg_batch_solve on the batch's own
    device buffers), the launch shape picked by the autotuner; beside it the
    same members solved one after another by mg_solve, mixed and plain fp64,
    and the batch end to end from pinned host buffers."""
    import numpy as np
    import torch
    from paper_2505_05105_gb300 import ghostmg
    ps = batch_members(args.batch_count)
    B = ghostmg.BatchSolver(ps)
    fh = torch.from_numpy(B.pack([p.f for p in ps])).pin_memory()
    gh = torch.from_numpy(B.pack([p.g for p in ps])).pin_memory()
    f0, g0, u0 = B.buffers()
    f0.copy_(fh.to(dev))
    g0.copy_(gh.to(dev))
    torch.cuda.synchronize(dev)
    shape, tune_ms = B.tune(f0, g0, tol=TOL, reps=2)
    info = B.solve(f0, g0, u0, tol=TOL)
    ndof = sum(i.n_dof for i in info)
    for _ in range(args.warmup):
        B.solve(f0, g0, u0, tol=TOL)
    ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        info = B.solve(f0, g0, u0, tol=TOL)
        ms.append(B.timing()[1])
    assert all(i.status == ghostmg.MG_OK for i in info)
    value = ndof * args.steps / (sum(ms) / 1e3)
    cyc = [i.cycles for i in info]
    # end to end: pinned host f, g in, u out, through mg_batch_solve
    uh = torch.zeros(B.total, dtype=torch.float64).pin_memory()
    B.solve(fh.data_ptr(), gh.data_ptr(), uh.data_ptr(), tol=TOL)
    tot = 0.0
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        B.solve(fh.data_ptr(), gh.data_ptr(), uh.data_ptr(), tol=TOL)
        tot += time.perf_counter() - t0
    e2e = {"value": ndof * args.steps / tot, "unit": UNIT,
           "h2d_bytes_per_step": 2 * B.total * 8, "d2h_bytes_per_step": B.total * 8,
           "transfer": "pinned host f, g read in place where they enter F, u written in "
                       "place; bytes above are the arrays' sizes"}
    setup_ms, _ = B.timing()
    B.close()
    # the same members one by one through mg_solve (one warm-up solve each)
    seq = {}
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(dev)
    for prec in ("mixed", "fp64"):
        tot_ms = 0.0
        for p in ps:
            S = ghostmg.Solver(t(p.psi), p.N, p.x0, p.y0, p.h, precision=prec)
            fd, gd = t(p.f), t(p.g)
            uu = torch.zeros_like(fd)
            S.solve(fd, gd, uu, tol=TOL)
            uu.zero_()
            tot_ms += S.solve(fd, gd, uu, tol=TOL).solve_ms
            S.close()
        seq[prec] = {"value": ndof / (tot_ms / 1e3), "unit": UNIT, "ms": tot_ms}
    sizes = sorted({p.N for p in ps})
    peak, peak_src = measured_peaks()
    traffic = profile_traffic("batch_k_batch_256members", "batch") if len(ps) == 256 else None
    per_step_s = sum(ms) / args.steps / 1e3
    return {
        "workload": f"batch of {len(ps)} seeded geometries (ellipses, flowers k=3..7), "
                    f"N in {sizes}, random Fourier f, g=0",
        "value": value, "unit": UNIT, "ms_per_step": sum(ms) / args.steps,
        "n_dof": ndof, "members": len(ps), "steps": args.steps,
        "cycles_per_member": {"min": min(cyc), "max": max(cyc),
                              "mean": float(np.mean(cyc))},
        "launch_shape": dict(zip(("threads", "first_group", "cluster", "coop_min_dof"), shape)),
        "tuned_ms": tune_ms, "setup_ms": setup_ms,
        "timing": "CUDA events around the graph launch on the batch's stream; L2 flushed "
                  "(512 MB write) between steps",
        "graph_kernels_per_step": 3,
        "roofline": {"bound": "latency", "kernel": "k_batch (persistent)",
                     "dram_traffic_per_step": traffic,
                     "dram_gbs": traffic / per_step_s / 1e9 if traffic else None,
                     "hbm_peak_gbs": peak,
                     "frac_of_hbm": traffic / per_step_s / 1e9 / peak if traffic else None,
                     "note": "DRAM bytes from the committed ncu summary "
                             "(profiles/batch_k_batch_256members.md) over this run's step time; "
                             f"{peak_src} HBM peak"},
        "sequential_mg_solve_mixed": seq["mixed"],
        "sequential_mg_solve_fp64": seq["fp64"],
        "batched_over_sequential_fp64": value / seq["fp64"]["value"],
        "e2e": e2e,
    }


def profile_batch(args):
    """Setup and two solves of the batched workload (default launch shape, or
    --batch-shape), untimed: the program batched-kernel profiler captures run."""
    import torch
    from paper_2505_05105_gb300 import ghostmg
    ghostmg.load()
    ps = batch_members(args.batch_count)
    B = ghostmg.BatchSolver(ps)
    if args.batch_shape:
        B.set_shape(*(int(x) for x in args.batch_shape.split(",")))
    f = torch.from_numpy(B.pack([p.f for p in ps])).cuda()
    g = torch.from_numpy(B.pack([p.g for p in ps])).cuda()
    u = torch.zeros(B.total, dtype=torch.float64, device="cuda")
    for _ in range(2):
        info = B.solve(f, g, u, tol=TOL)
    print(json.dumps({"profile_batch": len(ps), "shape": B.shape(),
                      "max_cycles": max(i.cycles for i in info)}))
    B.close()


def profile_solve(args):
    """Setup and one mixed solve of the flower workload, untimed: the program
    that single-kernel profiler captures run (no flush buffer, no oracle)."""
    import numpy as np
    import torch
    from paper_2505_05105_gb300 import ghostmg, workloads as wl
    ghostmg.load()
    p = wl.flower(args.N)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()
    S = ghostmg.Solver(t(p.psi), p.N, p.x0, p.y0, p.h, precision="mixed")
    u = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
    info = S.solve(t(p.f), t(p.g), u, tol=TOL)
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve": args.N, "cycles": info.cycles, "rel_res": info.rel_res}))
    S.close()


def main():
    args = parse()
    if args.profile_solve:
        profile_solve(args)
    elif args.profile_batch:
        profile_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
