"""Benchmark: reduced-Hessian CG to relative residual 1e-8 on one GB300.

Workload: the 1025^2 L-shaped P1 triangle mesh (784,385 states, 788,481
controls), 8x8 checkerboard kappa in {1, 1e4}, beta = 1e-4, 8 Gaussian-bump
desired state (seeded synthetic data).  One step = the whole hot path on that
input: device assembly, AMG setup of both hierarchies, right-hand side, outer
CG with the multilevel Hessian preconditioner to ||r||/||b|| <= 1e-8, and the
recomputed true residual.  Metric: fine-level Hessian applications per
second of step time (whole job over all ranks); the time to 1e-8 is
reported beside it.  Three precision forms are timed: "mixed" (FP64 CG for
every PDE solve preconditioned by FP32 V-cycles; the headline), "fp64", and
"refine" (FP32 CG and V-cycles inside FP64 iterative refinement).  Kernel
durations for the roofline (the level-0 Chebyshev smoother step) come from
an instrumented pass of the same step right after the timed region (CUDA
events per launch, which needs direct launches instead of CUDA graphs).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl amgh|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the batch runs one stream per solve slot: give them more hardware queues
# (read once, when CUDA is first initialised in this process)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

# kernel classes timed together in one instrumented pass (bit c = class c of
# amgh_kernel_class_stats): each level-0 class alone, then all the others
TIMING_GROUPS = [1 << 0, 1 << 2, 1 << 4, 1 << 6, 1 << 8, 1 << 10,
                 ((1 << 15) - 1) & ~((1 << 0) | (1 << 2) | (1 << 4) | (1 << 6) | (1 << 8) | (1 << 10))]
METRIC = "Hessian-CG time-to-1e-8 and Hessian matvecs/s, mixed vs FP64, same GB300"
PRECISION = {"fp64": 0, "refine": 1, "mixed": 2}
UNIT = "Hessian-matvecs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="amgh", choices=["amgh", "reference"])
    ap.add_argument("--workload", default="lshape", choices=["lshape", "cube"],
                    help="lshape: 1025^2 L-shape, checkerboard kappa (the headline workload); cube: 257^3 Kuhn "
                         "cube, 10 slabs of kappa in {1, 1e6}, beta 1e-6")
    ap.add_argument("--N", type=int, default=None, help="grid size (default 1025 for lshape, 257 for cube)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--coarse-max", type=int, default=1000,
                    help="AMG stops at or below this many rows (1000: 4 levels, 784k..847 on the L-shape)")
    ap.add_argument("--degree", type=int, default=2, help="Chebyshev smoother degree")
    ap.add_argument("--inner-tol", type=float, default=1e-10, help="state/adjoint solves of the outer H applies")
    ap.add_argument("--precond-tol", type=float, default=1e-8,
                    help="coarse-Hessian solves and mass solves inside the preconditioner (Sec. 5.2: 1e-8)")
    ap.add_argument("--hessian-levels", type=int, default=0,
                    help="levels of the Hessian preconditioner (0 = all AMG levels, as in Sec. 5.3)")
    ap.add_argument("--single-step", action="store_true",
                    help="run one untimed step of the first form (for profilers) and print its counters")
    ap.add_argument("--block-apply", action="store_true",
                    help="block solver against single-column solves on one 513^2 square with 8 desired "
                         "states (prints its own JSON line)")
    ap.add_argument("--no-slots", action="store_true",
                    help="with --block-apply: leave out the concurrent-slot batch solve (host threads)")
    ap.add_argument("--autotune", type=int, default=0,
                    help="time the SpMV layouts of every operator at setup (remembered per matrix shape)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched workload (16 squares, 128 desired states)")
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--forms", default="mixed,fp64,refine",
                    help="mixed = FP64 CG + FP32 V-cycles; fp64; refine = FP32 CG in FP64 refinement")
    ap.add_argument("--persistent-cg", type=int, default=1,
                    help="1 (default): mass CGs as one cooperative launch each (amg option persistent_cg; "
                         "the mixed form's single-column and block mass CGs), 0: graph-replayed kernels")
    ap.add_argument("--fuse-coarse", type=int, default=0,
                    help="0: V-cycle level by level; 2: levels of <= 262144 rows in one cooperative launch")
    ap.add_argument("--experiments", action="store_true",
                    help="run the paper's Tables 1-2 (a_j), 5 (two-grid, geometric vs AMG) and 7 (level "
                         "sweep, ball inclusion) on the GPU and print them as one JSON line")
    ap.add_argument("--no-cube", action="store_true",
                    help="skip the 257^3 slab-cube block (mixed and FP64, >= 6 AMG levels)")
    ap.add_argument("--cube-N", type=int, default=257)
    ap.add_argument("--cube-steps", type=int, default=1)
    ap.add_argument("--cube-warmup", type=int, default=1)
    ap.add_argument("--cube-coarse-max", type=int, default=16,
                    help="AMG coarsening of the cube block stops at or below this many rows")
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of oracle Hessian applies per CPU-baseline leg (one core, all cores)")
    return ap.parse_args()


def make_workload(args):
    """(workload, config name, kappa description, extra setup options, extra solve options)."""
    from paper_2001_11533_gb300 import workloads
    if args.workload == "cube":
        N = args.N or 257
        w = workloads.cube_slabs(N=N)
        # beta = 1e-6 with a 1e6 contrast: drop Hessian levels if the W-cycle turns indefinite,
        # and solve a coarsest Hessian level too large for the dense inverse by CG
        return (w, f"cube{N}_slabs", "10 jittered slabs {1,1e6}", dict(coarse_solve=2),
                dict(level_fallback=1))
    N = args.N or 1025
    return w_lshape(N), f"lshape{N}_checkerboard", "8x8 checkerboard {1,1e4}", {}, {}


def workload_names(args):
    if args.workload == "cube":
        return f"cube{args.N or 257}_slabs", "10 jittered slabs {1,1e6}"
    return f"lshape{args.N or 1025}_checkerboard", "8x8 checkerboard {1,1e4}"


def w_lshape(N):
    from paper_2001_11533_gb300 import workloads
    return workloads.lshape_checkerboard(N=N)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    def __init__(self, index):
        import tempfile
        self.index = index
        self.proc = None
        # raw samples go to a scratch file (BENCH_CLOCKS_DIR if set); the JSON line carries the summary
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ------------------------------------------------------------------------- amgh arm
def run_amgh(args, rank, world, local):
    import torch

    from paper_2001_11533_gb300 import _build, amgh, replicas, workloads
    _build.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w, _, _, xsetup, xsolve = make_workload(args)
    host = [np.ascontiguousarray(w.coords, np.float64), np.ascontiguousarray(w.elements, np.int32),
            np.ascontiguousarray(w.dirichlet, np.uint8), np.ascontiguousarray(w.kappa, np.float64),
            np.ascontiguousarray(w.y_d, np.float64)]
    dev = [torch.from_numpy(a).cuda() for a in host]
    pinned = [torch.from_numpy(a).pin_memory() for a in host]
    pinned_np = [t.numpy() for t in pinned]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def step(precision, e2e=False, timing=0):
        if e2e:
            prob = amgh.Problem(w.dim, *pinned_np[:4], w.beta, pinned_np[4], on_device=False)
        else:
            prob = amgh.Problem(w.dim, dev[0], dev[1], dev[2], dev[3], w.beta, dev[4], on_device=True)
        prob.amg_setup(precision=precision, hessian_levels=args.hessian_levels, coarse_max=args.coarse_max,
                       smooth_degree=args.degree, autotune=args.autotune, fuse_coarse=args.fuse_coarse,
                       persistent_cg=args.persistent_cg, **xsetup)
        if timing:
            prob.kernel_timing_mask(timing)
        tols = dict(tol=1e-8, inner_tol=args.inner_tol, mass_tol=args.precond_tol, precond_tol=args.precond_tol,
                    **xsolve)
        if e2e:
            u, y, info = prob.solve_host(**tols)
        else:
            u, y, info = prob.solve(**tols)
        ks = {"chebl0": prob.kernel_stats(), "classes": prob.kernel_class_stats()} if timing else None
        sizes = prob.sizes
        prob.close()
        return info, ks, sizes

    results = {}
    forms = [f for f in args.forms.split(",") if f]
    for form in forms:
        precision = PRECISION[form]
        for _ in range(args.warmup):
            step(precision)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        times, happ, infos = [], 0, []
        kstats = {"launches": 0, "ms": 0.0, "bytes": 0.0}
        classes = {}
        launches0 = amgh.launch_count()
        with ClockSampler(local) as clk:
            for k in range(args.steps):
                flush.zero_()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                info, _, sizes = step(precision)
                ev1.record(stream)
                ev1.synchronize()
                times.append(ev0.elapsed_time(ev1))
                happ += info["hessian_applies"]
                infos.append(info)
        torch.cuda.synchronize()
        barrier()
        launches = amgh.launch_count() - launches0
        # instrumented passes (not timed): CUDA events around the launches of
        # one group of kernel classes per pass (events keep a launch from
        # overlapping its neighbours, so each level-0 class is timed alone)
        for mask in TIMING_GROUPS:
            flush.zero_()
            _, ks, _ = step(precision, timing=mask)
            if mask & 1:
                for key in kstats:
                    kstats[key] += ks["chebl0"][key]
            for name, c in ks["classes"].items():
                acc = classes.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0})
                for key in acc:
                    acc[key] += c[key]
        t_total = sum(times) / 1000.0
        # max over ranks of the timed total, sum of work
        (t_total,), (happ_all,) = replicas.combine([t_total], [happ], device="cuda")
        results[form] = {
            "value": happ_all / t_total,
            "ms_per_step": 1000.0 * t_total / args.steps,
            "hessian_applies_per_step": happ / args.steps,
            "outer_iters": infos[-1]["outer_iters"],
            "final_relres": infos[-1]["final_relres"],
            "inner_iters_per_step": infos[-1]["inner_iters"],
            "setup_s": infos[-1]["t_setup_s"],
            "solve_s": infos[-1]["t_solve_s"],
            "refinements": infos[-1]["refinements"],
            "gpu_launches": launches,
            "kstats": kstats,
            "kernel_classes": classes,
            # algorithmic bytes of the solve phase (every kernel of the outer CG,
            # its Hessian applies and the preconditioner), from the last timed step
            "solve_phase": solve_phase(infos[-1]),
            "clocks": clk.summary(),
            "levels": {"state": sizes["state"], "control": sizes["control"], "ell": sizes["ell"]},
        }
    # end-to-end through the host-buffer entry points (H2D of the inputs from
    # pinned memory, D2H of u and y), timed as `value`: the same number of
    # steps, CUDA events on the launching stream, L2 flushed between steps
    head = forms[0]
    precision = PRECISION[head]
    for _ in range(args.warmup):
        step(precision, e2e=True)
    torch.cuda.synchronize()
    barrier()
    e_times, e_happ = [], 0
    for k in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        info, _, sizes = step(precision, e2e=True)
        ev1.record(stream)
        ev1.synchronize()
        e_times.append(ev0.elapsed_time(ev1))
        e_happ += info["hessian_applies"]
    torch.cuda.synchronize()
    barrier()
    e2e_t = sum(e_times) / 1000.0
    (e2e_t,), (e_happ,) = replicas.combine([e2e_t], [e_happ], device="cuda")
    h2d = sum(a.nbytes for a in host)
    d2h = 8 * (sizes["n"] + sizes["m"])
    e2e = {"value": e_happ / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": 1000.0 * e2e_t / args.steps,
           "timing": "CUDA events on the launching stream, same steps as value, 256 MB L2 flush between steps"}
    return w, results, e2e


def run_batch(args, rank, world, local):
    """The batching pattern: 16 jittered unit squares (65^2 .. 513^2, four
    of each), 8 desired states each, beta log-uniform in [1e-6, 1e-2]; every
    one of the 128 outer CGs to 1e-8.  Problems are dealt round-robin to the
    ranks.  Setup is timed apart; a step is one batched solve of all desired
    states (host clock around the synchronous call, after a warm-up solve
    that captures the CUDA graphs), once with one concurrent solve slot per
    desired state ("columns") and once with the block solver, all 8 desired
    states of a problem advanced together ("block")."""
    import torch

    from paper_2001_11533_gb300 import amgh, replicas, workloads
    every = workloads.batch_squares()
    tuned = "columns"
    ws = [every[i] for i in replicas.deal(len(every), rank, world)]
    yds = [torch.from_numpy(np.ascontiguousarray(w.y_d)).cuda() for w in ws]
    out = {}
    for form in ("mixed", "fp64"):
        probs = [amgh.Problem.from_workload(w) for w in ws]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch = amgh.Batch(probs).setup(coarse_max=1000, precision=PRECISION[form], coarse_solve=2,
                                        autotune=args.autotune)
        t_setup = time.perf_counter() - t0
        sopts = dict(tol=1e-8, inner_tol=args.inner_tol, mass_tol=args.precond_tol,
                     precond_tol=args.precond_tol, level_fallback=1)
        controls = {}
        for mode in ("columns", "block", "autotuned"):
            tuning = None
            if mode == "autotuned":
                # slot count and block width picked by timing the candidates on this
                # batch (mixed form, at a looser tolerance); the FP64 form reuses it
                if form == "mixed":
                    tuned_choice, tuning = batch.autotune(yds, **dict(sopts, tol=1e-6))
                    tuned = tuned_choice
                choice = tuned
                block, workers = {"columns": (0, 0), "block K=8": (1, 1), "block K=4 x 2 slots": (1, 2),
                                  "block K=2 x 4 slots": (1, 4)}[choice]
                batch.set_block(block)
                batch.set_workers(workers)
            else:
                batch.set_block(mode == "block")
                batch.set_workers(0)
            batch.solve(yds, **sopts)
            times, infos = [], None
            for _ in range(args.batch_steps):
                t0 = time.perf_counter()
                us, infos, st = batch.solve(yds, **sopts)
                times.append(time.perf_counter() - t0)
            controls[mode] = [u.cpu().numpy() for u in us]
            t = max(times)
            happ = sum(i["hessian_applies"] for i in infos)
            (t, ts), (happ,) = replicas.combine([t, t_setup], [happ], device="cuda")
            key = form if mode == "columns" else form + "_" + mode
            out[key] = {
                "time_to_1e-8_s": t, "hessian_matvecs_per_s": happ / t, "hessian_applies": happ,
                "setup_s": ts, "status": int(st),
                "outer_iters": sum(i["outer_iters"] for i in infos),
                "fallbacks": sum(i["fallbacks"] for i in infos),
                "max_final_relres": max(i["final_relres"] for i in infos),
                "hessian_levels": [i["hessian_levels"] for i in infos]}
            if mode == "autotuned":
                out[key]["choice"] = choice
                if tuning:
                    out[key]["tuning_s"] = {k: round(v, 3) for k, v in tuning.items()}
        # both modes run the same method per desired state: controls agree to the tolerance
        for mode in ("block", "autotuned"):
            out[form + "_" + mode]["max_rel_diff_vs_columns"] = max(
                float(np.linalg.norm(a[c] - b[c]) / max(np.linalg.norm(b[c]), 1e-300))
                for a, b in zip(controls[mode], controls["columns"]) for c in range(a.shape[0]))
        batch.close()
        for p in probs:
            p.close()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["time_to_1e-8_s"] / out["mixed"]["time_to_1e-8_s"]
    out["speedup_block_vs_columns_mixed"] = (out["mixed"]["time_to_1e-8_s"]
                                             / out["mixed_block"]["time_to_1e-8_s"])
    out["speedup_autotuned_vs_columns_mixed"] = (out["mixed"]["time_to_1e-8_s"]
                                                 / out["mixed_autotuned"]["time_to_1e-8_s"])
    out["workload"] = "16 squares 65^2..513^2, 8 desired states each (128 outer CGs to 1e-8)"
    out["timing"] = "host clock around the synchronous batched solve; max of steps"
    return out


def run_cube(args, rank, world, local):
    """The large 3D high-contrast case: 257^3 Kuhn cube (16.6M states), kappa in
    10 jittered slabs of {1, 1e6}, beta = 1e-6, 32 bumps, with the multilevel
    Hessian preconditioner over all AMG levels (coarsening to <= cube_coarse_max
    rows: >= 6 levels), the coarsest Hessian level dense up to 4096 dofs else by
    CG, and the level fallback on.  One step as in the headline (assembly +
    setup + rhs + outer CG to 1e-8 + true residual), in the mixed and the FP64
    form; CUDA events on the launching stream, L2 flushed before each step.
    Every rank runs its own replica."""
    import torch

    from paper_2001_11533_gb300 import amgh, replicas, workloads
    w = workloads.cube_slabs(N=args.cube_N)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
           for a in (w.coords, w.elements.astype(np.int32), w.dirichlet.astype(np.uint8), w.kappa, w.y_d)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    tols = dict(tol=1e-8, inner_tol=args.inner_tol, mass_tol=args.precond_tol, precond_tol=args.precond_tol,
                level_fallback=1)

    def step(precision, timing=0, mf=0):
        prob = amgh.Problem(w.dim, dev[0], dev[1], dev[2], dev[3], w.beta, dev[4], on_device=True)
        prob.amg_setup(precision=precision, coarse_max=args.cube_coarse_max, smooth_degree=args.degree,
                       coarse_solve=2, fuse_coarse=args.fuse_coarse, matrix_free=mf, persistent_cg=args.persistent_cg)
        if timing:
            prob.kernel_timing_mask(timing)
        u, y, info = prob.solve(want_y=False, **tols)
        ks = {"chebl0": prob.kernel_stats(), "classes": prob.kernel_class_stats()} if timing else None
        sizes = prob.sizes
        prob.close()
        return info, ks, sizes

    out = {"workload": f"cube{args.cube_N}_slabs", "m": w.n_interior, "n": w.n_vertices, "beta": w.beta,
           "kappa": "10 jittered slabs {1,1e6}", "coarse_max": args.cube_coarse_max,
           "steps": args.cube_steps, "warmup": args.cube_warmup,
           "timing": "CUDA events per step on the launching stream, 256 MB L2 flush before each step"}
    # "mixed_matrix_free": the mixed form with the level-0 smoother steps and
    # residual applied matrix-free from the element coefficients
    for form in ("mixed", "fp64", "mixed_matrix_free"):
        mf = 1 if form == "mixed_matrix_free" else 0
        precision = PRECISION[form.split("_")[0]]
        for _ in range(args.cube_warmup):
            step(precision, mf=mf)
        torch.cuda.synchronize()
        times, infos = [], []
        with ClockSampler(local) as clk:
            for _ in range(args.cube_steps):
                flush.zero_()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                info, _, sizes = step(precision, mf=mf)
                ev1.record(stream)
                ev1.synchronize()
                times.append(ev0.elapsed_time(ev1) / 1000.0)
                infos.append(info)
        t = sum(times)
        happ = sum(i["hessian_applies"] for i in infos)
        (t,), (happ_all,) = replicas.combine([t], [happ], device="cuda")
        last = infos[-1]
        res = {"time_to_1e-8_s": t / args.cube_steps, "hessian_matvecs_per_s": happ_all / t,
               "outer_iters": last["outer_iters"], "inner_iters": last["inner_iters"],
               "mass_iters": last["mass_iters"], "coarse_iters": last["coarse_iters"],
               "hessian_applies": last["hessian_applies"], "final_relres": last["final_relres"],
               "setup_s": last["t_setup_s"], "solve_s": last["t_solve_s"], "status": last["status"],
               "fallbacks": last["fallbacks"], "hessian_levels": last["hessian_levels"],
               "levels": {"state": sizes["state"], "control": sizes["control"], "ell": sizes["ell"]},
               "clocks": clk.summary()}
        if form in ("mixed", "mixed_matrix_free"):
            flush.zero_()
            # kernels of 10 us and more here: one pass times every class
            _, ks, _ = step(precision, timing=(1 << 15) - 1, mf=mf)
            res["roofline"] = roofline_from({"kstats": ks["chebl0"]}, args, kernel_note="level-0 Chebyshev "
                                            "smoother step on the 3D uniform-width SELL-32 matrix (int32 columns)",
                                            traffic=None)
            res["kernels"] = kernel_table(ks["classes"])
        res["solve_phase"] = solve_phase(last)
        out[form] = res
    out["speedup_mixed_vs_fp64"] = out["fp64"]["time_to_1e-8_s"] / out["mixed"]["time_to_1e-8_s"]
    out["speedup_matrix_free_vs_assembled_mixed"] = (out["mixed"]["time_to_1e-8_s"]
                                                     / out["mixed_matrix_free"]["time_to_1e-8_s"])
    out["mixed_matrix_free"]["note"] = ("level-0 smoother and residual of the FP32 V-cycles applied from the "
                                        "element coefficients (kappa, FP32) instead of the assembled matrix; "
                                        "its kernel bytes are on that basis")
    del dev
    torch.cuda.empty_cache()
    return out


def captured_traffic(args):
    """DRAM bytes per launch of the level-0 smoother step from the committed ncu
    summary, or None if the kernel source changed since that capture (or the
    workload is not the captured one)."""
    import hashlib
    if args.workload != "lshape" or (args.N or 1025) != 1025:
        return None
    try:
        txt = open(os.path.join(ROOT, "profiles", "k_cheb_step_level0_lshape1025.md")).read()
        want = txt.split("source_sha256:")[1].split()[0]
        traffic = float(txt.split("traffic_bytes_per_launch:")[1].split()[0])
        src = b"".join(open(os.path.join(ROOT, "paper_2001_11533_gb300", "csrc", f), "rb").read()
                       for f in ("sparse.cu", "spmv.cuh", "internal.cuh"))
        return traffic if hashlib.sha256(src).hexdigest() == want else None
    except Exception:
        return None


def hbm_peak():
    peaks = measured_peaks()
    if peaks and peaks.get("hbm_gbs"):
        return float(peaks["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def solve_phase(info):
    """Bytes per Hessian apply and the HBM fraction of the whole solve phase:
    the algorithmic bytes of every kernel the solve ran over its host-clock
    duration (outer CG, every Hessian apply and preconditioner application)."""
    peak, src = hbm_peak()
    b, t, happ = info.get("alg_bytes", 0.0), info["t_solve_s"], max(info["hessian_applies"], 1)
    if not b or t <= 0:
        return None
    return {"alg_bytes": b, "bytes_per_hessian_apply": b / happ, "solve_s": t,
            "achieved_GBs": round(b / t / 1e9, 1), "frac": round(b / t / 1e9 / peak, 4),
            "peak_GBs": peak, "peak_source": src,
            "note": "solve-phase bytes include preconditioner work and coarse levels that live in L2"}


def kernel_table(classes):
    """Per kernel class from the instrumented passes: launches, mean duration, achieved
    GB/s on algorithmic bytes, fraction of the measured HBM copy peak, and share of
    the timed kernel time.  A coarse class moving under 32 MB per launch works on
    operands that stay in the 129 MB L2: its bytes/s is labelled L2-resident."""
    peak, _ = hbm_peak()
    total = sum(c["ms"] for c in classes.values()) or 1.0
    out = {}
    for name, c in sorted(classes.items(), key=lambda kv: -kv[1]["ms"]):
        if c["launches"] == 0 or c["ms"] <= 0:
            continue
        gbs = c["bytes"] / (c["ms"] / 1000.0) / 1e9
        per = c["bytes"] / c["launches"]
        out[name] = {"launches": c["launches"], "avg_us": round(1000.0 * c["ms"] / c["launches"], 2),
                     "share": round(c["ms"] / total, 4), "achieved_GBs": round(gbs, 1),
                     "frac_of_hbm": round(gbs / peak, 4), "mb_per_launch": round(per / 1e6, 2),
                     "residency": "hbm" if (name.endswith("_l0") or per >= 32e6) else "l2-resident"}
    return out


def roofline_from(res, args, kernel_note=None, traffic="captured"):
    ks = res["kstats"]
    peak, src = hbm_peak()
    if ks["launches"] == 0 or ks["ms"] <= 0:
        return None
    achieved = ks["bytes"] / (ks["ms"] / 1000.0) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": captured_traffic(args) if traffic == "captured" else traffic, "peak_source": src,
            "kernel": kernel_note or "level-0 Chebyshev smoother step (k_cheb_step_ell: uniform-width SELL-32 "
                                     "staged into shared memory by bulk copies)",
            "launches": ks["launches"], "avg_us": round(1000.0 * ks["ms"] / ks["launches"], 2)}


# ------------------------------------------------------------------------- oracle (CPU)
def host_cpu():
    """The host's CPU as lscpu reports it (model, sockets, cores), read in this run."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        keep = ("Architecture", "Model name", "Vendor ID", "CPU(s)", "Thread(s) per core",
                "Core(s) per socket", "Socket(s)", "CPU max MHz")
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in keep and k.strip() not in info:
                info[k.strip()] = v.strip()
    except Exception as e:  # lscpu missing: keep nproc only
        info["lscpu"] = f"unavailable ({type(e).__name__})"
    return info


def oracle_for(w, args, omp=True):
    from oracle.oracle import Oracle
    return Oracle(w, hessian_levels=args.hessian_levels, coarse_max=args.coarse_max, degree=args.degree,
                  inner_tol=args.inner_tol, omp=omp)


def oracle_apply_rate(orc, budget_s, threads):
    """Time the FP64 oracle's Hessian apply on `threads` host threads (setup untimed):
    whole applies until the budget is spent.  Returns (applies, seconds, threads used)."""
    from oracle import oracle as orc_mod
    used = orc_mod.set_threads(threads)
    u = np.random.default_rng(0).standard_normal(orc.n)
    n, t = 0, 0.0
    while t < budget_s or n == 0:
        t0 = time.perf_counter()
        orc.hessian(u)
        t += time.perf_counter() - t0
        n += 1
    return n, t, used


def dense_fp64(n_coarse):
    """The FP64 rates the dense coarsest-level kernels are bound by (FMA pipe and
    mma.m8n8k4.f64, measured), and one dense SPD inverse at the coarsest size:
    Cholesky, L^-1 and W^T W are about n^3 / 3 flops each (n^3 in all), timed
    with CUDA events on the launching stream, median of 5."""
    import torch

    from paper_2001_11533_gb300 import amgh
    s = torch.cuda.current_stream()
    dfma = amgh.fp64_peak(0, s.cuda_stream)
    dmma = amgh.fp64_peak(1, s.cuda_stream)
    n = int(n_coarse)
    b = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    a = b @ b.T / n + 1e-3 * torch.eye(n, dtype=torch.float64, device="cuda")
    inv = torch.empty_like(a)
    times = []
    for k in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        st, info = amgh.dense_spd_inverse(a, inv, stream=s.cuda_stream)
        e1.record(s)
        e1.synchronize()
        if st != 0:
            return {"dfma_tflops": dfma, "dmma_tflops": dmma, "spd_inverse": {"n": n, "status": st}}
        if k:
            times.append(e0.elapsed_time(e1))
    ms = sorted(times)[len(times) // 2]
    tf = float(n) ** 3 / (ms * 1e-3) * 1e-12
    return {"dfma_tflops": round(dfma, 3), "dmma_tflops": round(dmma, 3),
            "spd_inverse": {"n": n, "ms": round(ms, 3), "tflops": round(tf, 3),
                            "frac_of_dfma": round(tf / dfma, 3),
                            "note": "fused panel Cholesky + L^-1 sweep with lookahead, then W^T W"}}


def cpu_baseline(w, args):
    """The oracle's Hessian apply on the same workload, on one host core and on
    every host core (the -fopenmp build: row loops split over threads, dot
    products sequential, results bit-identical)."""
    orc = oracle_for(w, args, omp=True)
    n1, t1, c1 = oracle_apply_rate(orc, args.cpu_budget, 1)
    nall = os.cpu_count() or 1
    n, t, c = oracle_apply_rate(orc, args.cpu_budget, nall)
    return {"value": n / t, "unit": UNIT, "cores": c, "kind": "oracle",
            "sample": f"{n} Hessian applies of the FP64 oracle on the same workload on {c} host threads "
                      f"({t:.1f} s, setup untimed; each apply = 2 AMG-CG solves to the inner tolerance)",
            "single_core": {"value": n1 / t1, "cores": c1, "sample": f"{n1} applies in {t1:.1f} s"},
            "host": host_cpu()}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as orc_mod
    orc_mod.build(omp=True)
    w, wname, _, _, _ = make_workload(args)
    orc = oracle_for(w, args, omp=True)
    cores = orc_mod.set_threads(os.cpu_count() or 1)
    u = np.random.default_rng(0).standard_normal(w.n_vertices)
    for _ in range(args.warmup):
        orc.hessian(u)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.hessian(u)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wname, "m": w.n_interior, "n": w.n_vertices,
                       "beta": w.beta, "step": "one fine-level Hessian apply of the FP64 CPU oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} Hessian applies (2 AMG-CG solves to 1e-10 each) on "
                                       f"{cores} host threads", "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------- main
def single_step(args):
    """One step of the first form, untimed, for profilers (ncu launch lists)."""
    import torch

    from paper_2001_11533_gb300 import _build, amgh, workloads
    _build.build()
    w, _, _, xsetup, xsolve = make_workload(args)
    prob = amgh.Problem.from_workload(w)
    prob.amg_setup(precision=PRECISION[args.forms.split(",")[0]], hessian_levels=args.hessian_levels,
                   coarse_max=args.coarse_max, smooth_degree=args.degree, autotune=args.autotune,
                   persistent_cg=args.persistent_cg, **xsetup)
    u, y, info = prob.solve(tol=1e-8, inner_tol=args.inner_tol, mass_tol=args.precond_tol,
                            precond_tol=args.precond_tol, **xsolve)
    torch.cuda.synchronize()
    print(json.dumps({"info": info, "levels": prob.level_counters(), "sizes": prob.sizes,
                      "launches": amgh.launch_count()}))


def block_apply(args):
    """The block solver against single-column work on one jittered 513^2 square
    with 8 desired states (mixed form, the batch's tolerances): one block
    Hessian apply of 8 columns against 8 single applies in a row, and one block
    solve of the 8 desired states against 8 concurrent single-column slots and
    against 8 single solves in a row.  Host clock around synchronous calls,
    best of 3 after a warm-up that captures the graphs."""
    import torch

    from paper_2001_11533_gb300 import _build, amgh, workloads
    _build.build()
    w = workloads.batch_squares(sizes=(513,), per_size=1, rhs=8)[0]
    Y = torch.from_numpy(np.ascontiguousarray(w.y_d)).cuda()
    amg = dict(coarse_max=1000, precision=PRECISION["mixed"], coarse_solve=2)
    sopts = dict(tol=1e-8, inner_tol=args.inner_tol, mass_tol=args.precond_tol,
                 precond_tol=args.precond_tol, level_fallback=1)
    prob = amgh.Problem.from_workload(w).amg_setup(**amg)

    def best(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return min(ts)

    U = torch.from_numpy(np.random.default_rng(1).standard_normal((8, prob.sizes["n"]))).cuda()
    prob.set_solve_opts(inner_tol=args.inner_tol, mass_tol=args.precond_tol, precond_tol=args.precond_tol)
    t_hb = best(lambda: prob.hessian_apply(U))
    t_hs = best(lambda: [prob.hessian_apply(U[c]) for c in range(8)])
    t_sb = best(lambda: prob.solve_block(Y, **sopts))
    prob_p = amgh.Problem.from_workload(w).amg_setup(persistent_cg=1, **amg)
    t_sbp = best(lambda: prob_p.solve_block(Y, **sopts))
    prob_p.close()

    def singles():
        for c in range(8):
            prob.set_yd(Y[c])
            prob.solve(want_y=False, **sopts)
    t_ss = best(singles)
    t_sc = None
    if not args.no_slots:
        batch = amgh.Batch([amgh.Problem.from_workload(w)]).setup(**amg)
        t_sc = best(lambda: batch.solve([Y], **sopts))
        batch.close()
    # one more block solve inside a profiler range, for
    # `ncu --profile-from-start off` launch lists of exactly one block solve
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    prob.solve_block(Y, **sopts)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"block_apply": {
        "workload": "jittered 513^2 square, 8 desired states, mixed form", "K": 8,
        "hessian_apply_block_s": t_hb, "hessian_apply_8_single_s": t_hs,
        "solve_block_s": t_sb, "solve_block_persistent_mass_cg_s": t_sbp,
        "solve_8_concurrent_slots_s": t_sc, "solve_8_single_s": t_ss,
        "timing": "host clock around synchronous calls, best of 3 after a warm-up"}}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.single_step:
        single_step(args)
        return
    if args.block_apply:
        block_apply(args)
        return
    if args.experiments:
        from paper_2001_11533_gb300 import _build, experiments
        _build.build()
        out = {}
        for name, fn in (("tables_1_2_a_numbers", experiments.a_numbers_table),
                         ("table_5_two_grid", experiments.two_grid_table),
                         ("table_7_level_sweep", experiments.level_sweep_table)):
            t0 = time.perf_counter()
            out[name] = fn()
            out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
            print(json.dumps({name: out[name]}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    w, results, e2e = run_amgh(args, rank, world, local)
    wname, kdesc = workload_names(args)
    batch = None if args.no_batch else run_batch(args, rank, world, local)
    cube = None if (args.no_cube or args.workload == "cube") else run_cube(args, rank, world, local)
    if rank != 0:
        return
    forms = list(results)
    head = results[forms[0]]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if forms[0] == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": wname, "m": w.n_interior, "n": w.n_vertices,
                   "beta": w.beta, "kappa": kdesc, "tol": 1e-8,
                   "hessian_levels": args.hessian_levels, "coarse_max": args.coarse_max,
                   "chebyshev_degree": args.degree, "inner_tol": args.inner_tol,
                   "autotune": args.autotune, "fuse_coarse": args.fuse_coarse,
                   "persistent_cg": args.persistent_cg,
                   "precond_and_mass_tol": args.precond_tol,
                   "precision": forms[0], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "256 MB buffer written between timed steps",
                   "step": "assembly + AMG setup + rhs + outer CG to 1e-8 + true residual"},
        "time_to_1e-8_s": head["ms_per_step"] / 1000.0,
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
        "roofline": roofline_from(head, args),
        "kernels": kernel_table(head["kernel_classes"]),
        "solve_phase": head["solve_phase"],
        "e2e": e2e,
        "forms": {f: {k: (kernel_table(v) if k == "kernel_classes" else v) for k, v in r.items()
                      if k not in ("kstats", "clocks")} for f, r in results.items()},
    }
    if batch is not None:
        line["batch"] = batch
    if "mixed" in results and "fp64" in results:
        line["speedup_mixed_vs_fp64"] = results["mixed"]["value"] / results["fp64"]["value"]
    if "refine" in results and "fp64" in results:
        line["speedup_refine_vs_fp64"] = results["refine"]["value"] / results["fp64"]["value"]
    if cube is not None:
        line["cube"] = cube
    if args.workload == "lshape":
        line["dense_fp64"] = dense_fp64(head["levels"]["state"][-1])
    if world == 1 and not args.no_cpu_baseline and args.workload == "lshape":
        line["cpu_baseline"] = cpu_baseline(w, args)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
