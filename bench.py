#!/usr/bin/env python
"""Benchmark: milliseconds per semi-implicit viscous solve to a 1e-6 true residual.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sphvisc|reference]

One step is the whole hot path on one particle set already resident in HBM:
neighbour build (cell sort + lists), coefficients of A(dt) with the Jacobi
diagonal, the start x0 (v^n on fluid rows, dummy-wall rows from Eq. dummyvel)
and the mixed-precision restructured BiCGSTAB with float64 refinement until
||b - A x|| / ||b|| <= 1e-6.  The workload is the lava-like box: a 100^3
jittered fluid lattice (dx = 5 mm) on a 3-layer dummy floor and walls
(1,157,308 particles), nu = 10 m^2/s, dt = 5e-4 s, v ~ N(0, 0.1^2), b = v.
Its matrix (1.5 GB of coefficients) is far larger than L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank solves its own
independently seeded box (weak scaling, no data-path collective); the time is the
max over ranks.  ``--impl reference`` times the FP64 CPU oracle instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ms per viscous solve to 1e-6 residual; matvec % HBM peak; learned vs plain"
UNIT = "ms/solve"
FALLBACK_HBM_GBS = 6800.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sphvisc", choices=["sphvisc", "reference"])
    ap.add_argument("--box-side", type=int, default=100, help="fluid lattice side of the box workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-gaussian", action="store_true")
    ap.add_argument("--no-poiseuille", action="store_true")
    ap.add_argument("--poiseuille-only", default=None,
                    help="comma-separated 1/dp list (e.g. 16,32,64): only the Poiseuille runs, one JSON line")
    ap.add_argument("--poiseuille-cases", default=None,
                    help="with --poiseuille-only: comma-separated configurations (default: all)")
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--no-shard", action="store_true")
    ap.add_argument("--ensemble-only", action="store_true")
    ap.add_argument("--ensemble-scenes", type=int, default=64, help="scenes of the ensemble leg (64: the workload)")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-sequence", action="store_true")
    ap.add_argument("--sequence-steps", type=int, default=200)
    ap.add_argument("--precision-only", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--learned-only", action="store_true")
    ap.add_argument("--weights", default=None, help="warm-start network (.npz); default: the committed weights")
    ap.add_argument("--merged", type=int, default=0)
    ap.add_argument("--eps-inner", type=float, default=2e-2)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--launch-mode", type=int, default=0, choices=[0, 1],
                    help="0: dependent launches in the solve loop (default); 1: plain stream order")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


def workload_name(n):
    return (f"lava box: {n}^3 jittered fluid lattice dx=5mm on 3-layer dummy floor+walls, Wendland h=1.3dx, "
            f"nu=10 m^2/s, dt=5e-4 s, v~N(0,0.1^2), b=v, x0=v with dummy-wall closure")


# ---------------------------------------------------------------- CPU oracle --
# The FP64 oracle runs in a separate one-thread process (fork + exec of this
# script), on the full workloads.  Jobs (jobs.json in a scratch folder):
#   box:           the bench workload itself; timed from the particle arrays to the
#                  accepted solution (k-d tree neighbours + assembled CSR A + the
#                  v^n start with the dummy-wall closure + textbook BiCGSTAB with
#                  Jacobi, restarted to a 1e-6 true residual): the CPU baseline.
#                  Untimed: a tighter solve (1e-11) as the reference solution, and,
#                  once the GPU's solution file exists, its oracle-computed true
#                  residual and its distance to that reference.
#   slope_subset:  the precision study's 57.5k subset (oracle mu pass + A), solved
#                  to 1e-11; the GPU's mixed and float64 solutions against it.

ORACLE_WAIT_S = 900.0
TIGHT_RTOL = 5e-8


def _wait_for(path, timeout):
    t0 = time.perf_counter()
    while not os.path.exists(path):
        if time.perf_counter() - t0 > timeout:
            return False
        time.sleep(0.5)
    time.sleep(0.2)
    return True


def _errors_against(A, b, x_ref, path, np, oop):
    x = np.load(path)
    res, per = oop.true_residual(A, x, b)
    return dict(oracle_true_rel_res=float(res), oracle_true_rel_res_c=[float(v) for v in per],
                rel_l2_vs_oracle=float(np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)))


def oracle_worker(folder):
    import numpy as np

    import scenes
    from oracle import neighbors as onb, operator as oop, rheology as orh, solvers as osv, warmstart as ows

    jobs = json.load(open(os.path.join(folder, "jobs.json")))
    out = []
    for job in jobs:
        if job["kind"] == "box":
            s = scenes.lava_box(job.get("seed", 0), n=job["n"])
            t0 = time.perf_counter()
            off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
            t1 = time.perf_counter()
            A = oop.assemble(s, off, idx)
            t2 = time.perf_counter()
            x0 = ows.start(A, s.b, s.vel, None, s.ptype, 1.0)
            stats = {}
            x = osv.reference_solution(A, s.b, x0, rtol=1e-6, stats=stats)
            t3 = time.perf_counter()
            res, _ = oop.true_residual(A, x, s.b)
            row = dict(kind="box", n=s.n, sec=t3 - t0, neighbours_s=t1 - t0, assemble_s=t2 - t1, solve_s=t3 - t2,
                       iterations=stats["iterations"], passes=stats["passes"], true_rel_res=float(res))
            if job.get("x_gpu"):
                x_ref = x if res <= 1e-11 else osv.reference_solution(A, s.b, x, rtol=1e-11)
                row["reference_true_rel_res"] = float(oop.true_residual(A, x_ref, s.b)[0])
                if _wait_for(job["x_gpu"], ORACLE_WAIT_S):
                    row.update(_errors_against(A, s.b, x_ref, job["x_gpu"], np, oop))
                if job.get("x_gpu_tight") and _wait_for(job["x_gpu_tight"], ORACLE_WAIT_S):
                    row["tight"] = _errors_against(A, s.b, x_ref, job["x_gpu_tight"], np, oop)
        else:
            s = scenes.slope_subset(0, mu0=job["mu0"], U=job["U"])
            off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
            mu = orh.mu_pass(s, off, idx)[0]
            A = oop.assemble(s, off, idx, mu=mu)
            x_ref = osv.reference_solution(A, s.b, s.x0, rtol=1e-11)
            row = dict(kind="slope_subset", mu0=job["mu0"], U=job["U"], n=s.n,
                       reference_true_rel_res=float(oop.true_residual(A, x_ref, s.b)[0]))
            for name, path in job["x_gpu"].items():
                if _wait_for(path, ORACLE_WAIT_S):
                    row[name] = _errors_against(A, s.b, x_ref, path, np, oop)
        out.append(row)
    print(json.dumps(out))


class OracleRun:
    """The oracle worker as a background process (one BLAS/OpenMP thread, no GPU)."""

    def __init__(self, jobs, folder):
        import tempfile

        self.folder = folder or tempfile.mkdtemp(prefix="sph_oracle_")
        json.dump(jobs, open(os.path.join(self.folder, "jobs.json"), "w"))
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                   CUDA_VISIBLE_DEVICES="")
        self.proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-worker", self.folder],
                                     stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)

    def result(self, timeout=1800):
        try:
            out, err = self.proc.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            return None, "oracle worker timed out"
        if self.proc.returncode != 0:
            return None, err[-2000:]
        return json.loads(out.strip().splitlines()[-1]), None


# ----------------------------------------------------------------- helpers ---

def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources of the operator apply kernel (k_apply_dot and what it includes)
TRAFFIC_SOURCES = ("apply.cuh", "solver.cu", "reduce.cuh", "bicgstab_scalars.cuh", "sph_internal.cuh")


def apply_traffic(alg_bytes):
    """DRAM bytes per apply launch: the ncu-measured ratio of DRAM traffic to algorithmic
    bytes (profiles/apply_traffic.txt) times this launch's algorithmic bytes, or None when
    the kernel sources changed since the counters were taken."""
    import hashlib

    try:
        kv = {}
        for line in open(os.path.join(ROOT, "profiles", "apply_traffic.txt")):
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                kv[k] = v
        src = b"".join(open(os.path.join(ROOT, "paper_2206_14780_gb300", "csrc", f), "rb").read()
                       for f in TRAFFIC_SOURCES)
        if hashlib.sha256(src).hexdigest()[:16] != kv["sources_sha256_16"]:
            return None, "kernel changed since the ncu capture"
        return float(kv["dram_bytes_per_algorithmic_byte"]) * alg_bytes, \
            "ncu dram bytes per algorithmic byte at 274k particles, scaled to this launch"
    except Exception as e:
        return None, f"unavailable ({type(e).__name__})"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if args.impl == "sphvisc" else "gloo"
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return world, rank, local


def max_over_ranks(value, world, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Seed of the box a rank solves: every replica draws its own particle set."""
    return rank


def whole_job_ms_per_solve(ms_max, steps, world):
    """Time-like whole-job value: the max-over-ranks time of K steps, each rank solving one
    box per step, divided by the K * N solves all ranks completed."""
    return ms_max / (steps * world)


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist

        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ------------------------------------------------------------------ GPU arm ---

def run_sphvisc(args):
    import numpy as np
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    binding.load()
    s = scenes.lava_box(replica_seed(rank), n=args.box_side)
    params = binding.visc_params(s.dt, s.boundary, s.mean)
    opts = binding.solve_opts(merged_reductions=args.merged, eps_inner=args.eps_inner, launch_mode=args.launch_mode,
                              precision=binding.SPH_PREC_FP64 if args.precision == "fp64" else binding.SPH_PREC_MIXED)
    t = binding.scene_tensors(s, dev)
    t["vel"] = torch.from_numpy(s.vel).to(dev)
    b = torch.from_numpy(s.b).to(dev)
    x0 = torch.from_numpy(s.x0).to(dev)
    x = torch.empty_like(x0)
    geo = (s.lo, s.hi, s.periodic, s.h)
    nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], *geo)
    stream = torch.cuda.current_stream(dev)

    def step():
        # x0 = v^n on fluid rows, dummy-wall rows from Eq. dummyvel (sph_warm_start, no network)
        nb.rebuild(t["pos"], t["rho"], t["mu"], t["ptype"], *geo)
        binding.warm_start(nb, params, None, t["vel"], t["ptype"], b, x)
        return nb.solve(params, opts, b, x)

    for _ in range(max(3, args.warmup)):
        rep = step()
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    nb.profile(True)
    nb.profile_read(reset=True)
    launches0 = binding.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    ev0.record(stream)
    reps = []
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        reps.append(step())
        marks[k].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - w0
    per_step = [ev0.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k]) for k in range(1, args.steps)]
    clk = clocks.stop()
    launches = binding.launch_count() - launches0
    prof = nb.profile_read(reset=True)
    nb.profile(False)
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world, dev)
    barrier(world, dev)
    x_last = x.cpu().numpy()           # the last timed solve, compared with the oracle below
    # the same K steps once more with the apply's CUDA events off: what the sampled events
    # themselves cost the timed loop (reported beside the line's value, not in it)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for k in range(args.steps):
        step()
        marks[k].record(stream)
    torch.cuda.synchronize(dev)
    # median per step: this pass runs while the CPU oracle starts up on the host
    ms_unprofiled = statistics.median([ev0.elapsed_time(marks[0])] +
                                      [marks[k - 1].elapsed_time(marks[k]) for k in range(1, args.steps)])
    # the same step to a true residual small enough for a solution within 1e-5 of the
    # oracle's (the box's error is ~150x its residual), timed alone, untimed in `value`
    tight = None
    if not args.no_cpu_baseline and world == 1:
        o_t = binding.solve_opts(rtol=TIGHT_RTOL, merged_reductions=args.merged, eps_inner=args.eps_inner,
                                 launch_mode=args.launch_mode)
        nb.rebuild(t["pos"], t["rho"], t["mu"], t["ptype"], *geo)
        binding.warm_start(nb, params, None, t["vel"], t["ptype"], b, x)
        nb.solve(params, o_t, b, x)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        nb.rebuild(t["pos"], t["rho"], t["mu"], t["ptype"], *geo)
        binding.warm_start(nb, params, None, t["vel"], t["ptype"], b, x)
        rep_t = nb.solve(params, o_t, b, x)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        tight = dict(rtol=TIGHT_RTOL, ms_per_solve=ev0.elapsed_time(ev1), iters=rep_t["iters"],
                     passes=rep_t["refinements"], true_rel_res=rep_t["true_rel_res"])
        x_tight = x.cpu().numpy()

    # end to end through the C-ABI's host-buffer call (sph_visc_solve_host): H2D of the
    # particle set (with v^n) and b from pinned host memory, neighbours, A(dt), x0, solve, D2H of x
    e2e = None
    if not args.no_e2e:
        host = {k: v.cpu().pin_memory() for k, v in t.items()}
        hb = b.cpu().pin_memory()
        hx = torch.empty_like(hb).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in host.values()) + hb.numel() * 8
        d2h = hx.numel() * 8
        e2e_nb = [None]

        def e2e_step():
            _, e2e_nb[0] = binding.solve_host(host["pos"], host["rho"], host["mu"], host["ptype"], *geo, params, opts,
                                              host["vel"], hb, hx, nb=e2e_nb[0])

        e2e_step()
        barrier(world, dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ems = max_over_ranks(e0.elapsed_time(e1), world, dev)
        e2e = dict(value=whole_job_ms_per_solve(ems, args.steps, world), unit=UNIT, h2d_bytes_per_step=int(h2d),
                   d2h_bytes_per_step=int(d2h), api="sph_visc_solve_host (pinned host buffers in and out)")
        e2e_nb[0].close()

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return
    # the FP64 oracle on the same box (and the slope subsets of the precision study),
    # in a background process while the remaining GPU legs run
    oracle = None
    if not args.no_cpu_baseline and world == 1:
        import tempfile

        import numpy as np

        folder = tempfile.mkdtemp(prefix="sph_oracle_")
        np.save(os.path.join(folder, "box_x.npy"), x_last)
        np.save(os.path.join(folder, "box_x_tight.npy"), x_tight)
        jobs = [dict(kind="box", n=args.box_side, seed=replica_seed(rank), x_gpu=os.path.join(folder, "box_x.npy"),
                     x_gpu_tight=os.path.join(folder, "box_x_tight.npy"))]
        if not args.no_precision:
            for tag, mu0, U in SUBSETS:
                jobs.append(dict(kind="slope_subset", mu0=mu0, U=U,
                                 x_gpu={k: os.path.join(folder, f"subset_{tag}_{k}.npy") for k in ("mixed", "fp64")}))
        oracle = OracleRun(jobs, folder)
    hbm, peak_kind = read_peaks()
    avg_apply_ms = prof["apply_ms"] / max(1, prof["apply_launches"])
    achieved = prof["apply_bytes"] / (avg_apply_ms * 1e-3) / 1e9 if prof["apply_launches"] else None
    traffic, traffic_src = apply_traffic(prof["apply_bytes"])
    roofline = dict(bound="hbm", achieved=achieved, peak=hbm, unit="GB/s",
                    frac=(achieved / hbm) if achieved else None, traffic=traffic, traffic_source=traffic_src,
                    kernel="k_apply_dot (operator apply + fused dots)", peak_source=peak_kind,
                    apply_launches=prof["apply_launches"], apply_avg_us=avg_apply_ms * 1e3,
                    apply_avg_us_Ap=1e3 * prof["phase_ms"][0] / max(1, prof["phase_launches"][0]),
                    apply_avg_us_Ars=1e3 * prof["phase_ms"][1] / max(1, prof["phase_launches"][1]),
                    apply_variant=prof["apply_variant"], apply_grid=prof["apply_grid"],
                    autotune_us=prof["tune_us"][:2],
                    algorithmic_bytes_per_launch=prof["apply_bytes"],
                    timing="CUDA events on the solve stream around both applies of every 8th BiCGSTAB "
                           "iteration inside the timed region (launches after convergence excluded)")
    apply_forms = None
    channel = None
    if world == 1:
        apply_forms = run_apply_forms(nb, params, s.n, dev)
        channel = run_channel(dev)
    gaussian = None
    if world == 1 and not args.no_gaussian:
        gaussian = run_gaussian(dev, n=args.box_side)
    poiseuille = None
    if world == 1 and not args.no_poiseuille:
        # the default run leaves out the h = 2.5 dp Wendland runs (about 500 neighbours on
        # a few thousand particles, 28 s); --poiseuille-only runs them too
        poiseuille = run_poiseuille(dev, cases=[c for c in POISEUILLE_PAPER if "wendland25" not in c])
    cg = shard = None
    if world == 1 and not args.no_cg:
        cg = run_cg(dev)
    if world == 1 and not args.no_shard:
        shard = run_shard(dev)
    sequence = None
    if not args.no_sequence and world == 1:
        sequence = run_sequence(nb, s, b, t, args.sequence_steps, dev)
        heads = _scale_heads()
        if "learned_scale" in heads:
            # the same sequence with the learned wall-row scale, computed once from v^0
            # (positions, and so the operator, stay frozen over the sequence)
            torch.cuda.synchronize(dev)
            w0_ = time.perf_counter()
            heads["learned_scale"](nb, binding.visc_params(s.dt, s.boundary, s.mean), t, None)
            torch.cuda.synchronize(dev)
            scale_ms = 1e3 * (time.perf_counter() - w0_)
            sequence["learned_scale"] = run_sequence(nb, s, b, t, args.sequence_steps, dev)
            sequence["learned_scale"]["scale_setup_ms"] = scale_ms
            nb.set_row_scale(None)
    ensemble = None
    if not args.no_ensemble and world == 1:
        nb.close()
        torch.cuda.empty_cache()
        ensemble = run_ensemble(0, dev, scenes_n=args.ensemble_scenes)
    precision = None
    if not args.no_precision and world == 1:
        torch.cuda.empty_cache()
        precision = run_precision(dev)
        torch.cuda.empty_cache()
        precision["low_plastic_viscosity"] = run_precision(dev, mu0=1.0, U=3.3)
        if oracle is not None:
            for tag, mu0, U in SUBSETS:
                torch.cuda.empty_cache()
                key = "subset" if tag == "default" else "low_plastic_viscosity_subset"
                precision[key] = run_subset(dev, mu0, U, oracle.folder, tag)
    learned = None
    if not args.no_learned and world == 1:
        torch.cuda.empty_cache()
        learned = run_learned(args.weights, dev)
        learned["mlp_forward"] = run_mlp_forward(dev)
        learned["mlp_grad"] = run_mlp_grad(dev)
        torch.cuda.empty_cache()
        learned["precond_scale"] = ps = run_precond_scale(dev, heads=_scale_heads())
        # the preconditioner-scale heads against Jacobi alone (same start, v^n + closure)
        if "learned_vs_plain" in learned:
            for case in ("box_1157k", "ensemble_64"):
                for k in ("learned_scale", "wall_p3", "wall_c0.125"):
                    if k in ps.get(case, {}):
                        learned["learned_vs_plain"].setdefault(case, {})[f"{k}/jacobi_vn_walls"] = ps[case][k]["vs_jacobi"]
                        if "vs_sequential_plain" in ps[case][k]:
                            learned["learned_vs_plain"][case][f"{k}_batched/sequential_plain"] = \
                                ps[case][k]["vs_sequential_plain"]
    cpu, oracle_error = None, None
    if oracle is not None:
        rows, err = oracle.result()
        if rows is None:
            cpu = dict(value=None, unit=UNIT, cores=1, kind="oracle", unavailable=err)
        else:
            box = rows[0]
            cpu = dict(value=box["sec"] * 1e3, unit=UNIT, cores=1, kind="oracle",
                       sample=(f"the full workload, one solve (N={box['n']}): k-d tree neighbours "
                               f"{box['neighbours_s']:.1f} s + scipy CSR A {box['assemble_s']:.1f} s + x0 and "
                               f"textbook BiCGSTAB with Jacobi restarted to a 1e-6 true residual "
                               f"{box['solve_s']:.1f} s, FP64, one thread, run while the later GPU legs ran"),
                       iterations=box["iterations"], passes=box["passes"], true_rel_res=box["true_rel_res"],
                       gpu_iterations=reps[-1]["iters"])
            oracle_error = {k: box.get(k) for k in ("oracle_true_rel_res", "oracle_true_rel_res_c",
                                                    "rel_l2_vs_oracle", "reference_true_rel_res")}
            oracle_error["solution"] = "the last timed GPU solve (rtol 1e-6) against the oracle's 1e-11 solve"
            if tight is not None:
                tight.update(box.get("tight", {}))
                oracle_error["tight_solve"] = tight
            for row in rows[1:]:
                key = "subset" if row["mu0"] == SUBSETS[0][1] else "low_plastic_viscosity_subset"
                if precision is not None and key in precision:
                    for name in ("mixed", "fp64"):
                        if name in row:
                            precision[key][name].update(row[name])
                    precision[key]["oracle_reference_true_rel_res"] = row["reference_true_rel_res"]
    its = [r["iters"] for r in reps]
    out = dict(metric=METRIC, value=whole_job_ms_per_solve(ms_max, args.steps, world), unit=UNIT, n_gpus=world, steps=args.steps,
               warmup=max(3, args.warmup), ms_per_step=ms_max / args.steps, higher_is_better=False,
               scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
               config=workload_config(args.box_side, s.n),
               solver=dict(precision="f32 operator+vectors, f64 dots/scalars, f64 true-residual refinement",
                           merged_reductions=args.merged, eps_inner=args.eps_inner,
                           launch_mode="dependent launches" if args.launch_mode == 0 else "stream order",
                           step="neighbour build + A(dt) coefficients + x0 (v^n, dummy-wall closure) + "
                                "restructured BiCGSTAB to 1e-6",
                           fused_into_apply="Jacobi scaling, the phase's dot products, their grid reduction "
                                            "and the scalar update (last block); the p update, r* = r - alpha Ap "
                                            "and the x/r update with its dots are separate row kernels",
                           iters=its, passes=[r["refinements"] for r in reps],
                           true_rel_res=[r["true_rel_res"] for r in reps], parallelism=f"replicas x{world}",
                           ms_per_step_median=statistics.median(per_step),
                           ms_per_step_min=min(per_step), ms_per_step_max=max(per_step),
                           ms_per_step_without_apply_events=ms_unprofiled),
               roofline=roofline, cpu_baseline=cpu, oracle_error=oracle_error, e2e=e2e, gpu_launches=int(launches), ensemble=ensemble,
               precision_study=precision, sequence=sequence, learned=learned, apply_forms=apply_forms,
               channel=channel, gaussian=gaussian, poiseuille=poiseuille, cg=cg, shard=shard,
               clocks=dict(sm_mhz=clk["sm_mhz"], sm_max_mhz=clk["sm_max_mhz"], reasons=clk["reasons"],
                           samples=clk["samples"]),
               wall_s=wall)
    print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ------------------------------------------------------------ channel ---------

def run_channel(dev, reps=10):
    """Plane Couette channel of 1,000,000 fluid particles (200 x 50 x 100, dx = 0.01 m, 3+3
    dummy wall layers, periodic x and z, top wall at 1 m/s, nu = 1, dt = 1e-4: the paper's
    mild stiffness, dt nu / dx^2 = 1): ms per step (neighbours + A(dt) + x0 + solve to 1e-6)."""
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    s = scenes.couette(0, nx=200, ny=50, nz=100)
    t = binding.scene_tensors(s, dev)
    t["vel"] = torch.from_numpy(s.vel).to(dev)
    p = binding.visc_params(s.dt, s.boundary, s.mean)
    geo = (s.lo, s.hi, s.periodic, s.h)
    nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], *geo)
    b = torch.from_numpy(s.b).to(dev)
    x = torch.empty_like(b)
    opts = binding.solve_opts()
    stream = torch.cuda.current_stream(dev)

    def step():
        nb.rebuild(t["pos"], t["rho"], t["mu"], t["ptype"], *geo)
        binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
        return nb.solve(p, opts, b, x)

    for _ in range(3):
        step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    reps_ = [step() for _ in range(reps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    # the wall-row scale on this mild system (D ~ 4): the fixed constant tuned for stiff
    # boxes against the learned scale, which reads the stiffness from its features
    scales = {}
    heads = _scale_heads()
    sc = torch.empty(s.n, dtype=torch.float32, device=dev)
    for name in ("jacobi", "wall_c0.125", "learned_scale"):
        if name == "jacobi":
            nb.set_row_scale(None)
        elif name == "wall_c0.125":
            nb.wall_row_scale(p, 0.125, 0.0, sc)
            nb.set_row_scale(sc)
        elif "learned_scale" in heads:
            heads["learned_scale"](nb, p, t, None)
        else:
            continue
        binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
        nb.solve(p, opts, b, x)
        binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        rep = nb.solve(p, opts, b, x)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        scales[name] = dict(iters=rep["iters"], solve_ms=e0.elapsed_time(e1), true_rel_res=rep["true_rel_res"])
    nb.set_row_scale(None)
    nb.close()
    return dict(workload="plane Couette channel 200x50x100 fluid (N=1,120,000), dx=0.01, nu=1, dt=1e-4, "
                         "top wall 1 m/s, v = linear profile + 1% noise", particles=s.n, ms_per_step=ms,
                iters=[r["iters"] for r in reps_][:3], passes=reps_[0]["refinements"],
                max_true_rel_res=max(r["true_rel_res"] for r in reps_), wall_scale=scales)


# ------------------------------------------------------- Gaussian kernel ------

def run_gaussian(dev, n=100, reps=3):
    """The lava box with the truncated Gaussian kernel of Sec. 5.2 (support 3h = 3.9 dx,
    ~250 neighbours, four dummy layers): ms per step (neighbours + A(dt) + x0 + solve
    to 1e-6), iterations, and the apply's algorithmic GB/s inside the solves."""
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    s = scenes.lava_box(0, n=n, layers=4, kernel=scenes.KERNEL_GAUSSIAN)
    t = binding.scene_tensors(s, dev)
    t["vel"] = torch.from_numpy(s.vel).to(dev)
    p = binding.visc_params(s.dt, s.boundary, s.mean)
    geo = (s.lo, s.hi, s.periodic, s.h)
    nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], *geo, max_neighbors=512, kernel=s.kernel)
    b = torch.from_numpy(s.b).to(dev)
    x = torch.empty_like(b)
    opts = binding.solve_opts()
    stream = torch.cuda.current_stream(dev)

    def step():
        nb.rebuild(t["pos"], t["rho"], t["mu"], t["ptype"], *geo, max_neighbors=512, kernel=s.kernel)
        binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
        return nb.solve(p, opts, b, x)

    for _ in range(2):
        step()
    nb.profile(True)
    nb.profile_read(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    reps_ = [step() for _ in range(reps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    step_ms = e0.elapsed_time(e1) / reps
    prof = nb.profile_read(reset=True)
    nb.profile(False)
    _, nnz, maxc = nb.info()
    # the same solve with the closed-form wall-row scale of the preconditioner (constant
    # 1/8 on the dummy-wall rows), from the same start
    sc = torch.empty(s.n, dtype=torch.float32, device=dev)
    nb.wall_row_scale(p, 0.125, 0.0, sc)
    nb.set_row_scale(sc)
    binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
    nb.solve(p, opts, b, x)
    binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    rep_sc = nb.solve(p, opts, b, x)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    wall_scaled = dict(iters=rep_sc["iters"], solve_ms=e0.elapsed_time(e1), true_rel_res=rep_sc["true_rel_res"])
    nb.set_row_scale(None)
    binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    rep_pl = nb.solve(p, opts, b, x)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    wall_scaled["jacobi_solve_ms"] = e0.elapsed_time(e1)
    wall_scaled["jacobi_iters"] = rep_pl["iters"]
    heads = _scale_heads()
    if "learned_scale" in heads:       # the learned scale (its features use this kernel's W)
        heads["learned_scale"](nb, p, t, None)
        binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
        nb.solve(p, opts, b, x)
        binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        rep_l = nb.solve(p, opts, b, x)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        wall_scaled["learned_iters"] = rep_l["iters"]
        wall_scaled["learned_solve_ms"] = e0.elapsed_time(e1)
        wall_scaled["learned_true_rel_res"] = rep_l["true_rel_res"]
        nb.set_row_scale(None)
    nb.close()
    us = 1e3 * prof["apply_ms"] / max(1, prof["apply_launches"])
    hbm, kind = read_peaks()
    gbs = prof["apply_bytes"] / (us * 1e-6) / 1e9 if prof["apply_launches"] else None
    return dict(workload=f"lava box {n}^3 fluid, truncated Gaussian (k = 3, h = 1.3 dx), 4 dummy layers "
                         f"(N={s.n})", particles=s.n, neighbour_pairs=int(nnz), max_neighbours=int(maxc),
                ms_per_step=step_ms, iters=[r["iters"] for r in reps_],
                passes=reps_[0]["refinements"], max_true_rel_res=max(r["true_rel_res"] for r in reps_),
                apply_us=us, apply_algorithmic_bytes=prof["apply_bytes"], apply_gbs=gbs,
                apply_frac_of_hbm=(gbs / hbm) if gbs else None, peak_source=kind,
                wall_scale_c0_125=wall_scaled)


# ------------------------------------------------- CG and sharded solve -------

def run_cg(dev, reps=3):
    """Rotated CG (Sec. 4.1) against BiCGSTAB on dynamic-wall systems, where the fluid
    block is symmetric: the 1.12M Couette channel (dt nu / dx^2 = 1) and the 1.16M lava
    box (200): ms per solve (CUDA events, after a warm-up solve) and iterations; CG
    applies the operator once per iteration, BiCGSTAB twice."""
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    out = {}
    for name, s in (("channel_1120k", scenes.couette(0, nx=200, ny=50, nz=100, boundary=scenes.BC_DYNAMIC)),
                    ("box_1157k", scenes.lava_box(0, n=100, boundary=scenes.BC_DYNAMIC))):
        t = binding.scene_tensors(s, dev)
        t["vel"] = torch.from_numpy(s.vel).to(dev)
        p = binding.visc_params(s.dt, s.boundary, s.mean)
        nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], s.lo, s.hi, s.periodic, s.h)
        b = torch.from_numpy(s.b).to(dev)
        x = torch.empty_like(b)
        stream = torch.cuda.current_stream(dev)
        row = {}
        for meth, key in ((binding.SPH_SOLVER_BICGSTAB, "bicgstab"), (binding.SPH_SOLVER_CG, "cg")):
            o = binding.solve_opts(method=meth)
            binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
            nb.solve(p, o, b, x)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms, its, res = [], [], []
            for _ in range(reps):
                binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
                torch.cuda.synchronize(dev)
                e0.record(stream)
                rep = nb.solve(p, o, b, x)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms.append(e0.elapsed_time(e1))
                its.append(rep["iters"])
                res.append(rep["true_rel_res"])
            row[key] = dict(ms_per_solve=statistics.median(ms), iters=its[0], passes=rep["refinements"],
                            true_rel_res=max(res))
        row["cg_over_bicgstab_ms"] = row["cg"]["ms_per_solve"] / row["bicgstab"]["ms_per_solve"]
        out[name] = dict(particles=s.n, **row)
        nb.close()
        torch.cuda.empty_cache()
    return out


def run_shard(dev, n=60, ranks=(1, 2, 4)):
    """One system over k emulated sub-domains (sph_shard_*, Sec. 7) on the 60^3 lava box
    (274k particles): ms per solve for each k, iterations, and whether x is the same bit
    for bit as with one sub-domain (it must be); the single-domain solver beside it."""
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    s = scenes.lava_box(0, n=n)
    t = binding.scene_tensors(s, dev)
    p = binding.visc_params(s.dt, s.boundary, s.mean)
    nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], s.lo, s.hi, s.periodic, s.h)
    b = torch.from_numpy(s.b).to(dev)
    x0 = torch.from_numpy(s.x0).to(dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = dict(workload=f"lava box {n}^3 fluid (N={s.n}), one system over k sub-domains on one GPU", particles=s.n)
    x_one = None
    for k in ranks:
        w0 = time.perf_counter()
        sh = binding.Shard(nb, p, k)
        create_s = time.perf_counter() - w0
        row = {}
        for striped in (False, True):               # striping: exchange overlapped with the interior slices
            sh.set_striping(striped)
            x = x0.clone()
            sh.solve(binding.solve_opts(), b, x)
            x = x0.clone()
            torch.cuda.synchronize(dev)
            e0.record(stream)
            rep = sh.solve(binding.solve_opts(), b, x)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if x_one is None:
                x_one = x.clone()
            key = "striped" if striped else "unstriped"
            row[f"ms_per_solve_{key}"] = e0.elapsed_time(e1)
            row[f"bit_identical_to_k1_{key}"] = bool(torch.equal(x, x_one))
        info = sh.info()
        sh.close()
        out[f"k{k}"] = dict(ms_per_solve=row["ms_per_solve_striped"], iters=rep["iters"],
                            true_rel_res=rep["true_rel_res"], halo_rows=info["halo"], layers=info["layers"],
                            create_s=create_s, bit_identical_to_k1=row["bit_identical_to_k1_striped"] and
                            row["bit_identical_to_k1_unstriped"], **row)
    x = x0.clone()
    nb.solve(p, binding.solve_opts(), b, x)
    x = x0.clone()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    rep = nb.solve(p, binding.solve_opts(), b, x)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    out["single_domain_solver"] = dict(ms_per_solve=e0.elapsed_time(e1), iters=rep["iters"])
    nb.close()
    return out


# ------------------------------------------------------ Poiseuille flow -------

# the paper's numbers (Sec. 5.3, Tables tab:newton-error and tab:newton-times; Sec. 5.4, Tables
# tab:papa-error and tab:papa-times) per configuration and 1/dp: the l1 and l2 errors of the
# steady profile (and, for Wendland Newtonian, against 102% of it) and the semi-implicit runtime
# in seconds of the whole run to t = 10 s on the paper's machine.  (The 1/64 Wendland dynamic
# l2 against 102% is printed as 1.204e-3, ten times its l1 and its rate: kept as printed.)
def _pp(l1, l2, rt, l1_102=None, l2_102=None):
    d = {"l1": l1, "l2": l2, "runtime_s": rt}
    if l1_102 is not None:
        d.update(l1_102=l1_102, l2_102=l2_102)
    return d


POISEUILLE_PAPER = {
    "newton_wendland_dummy": {16: _pp(1.227e-3, 1.282e-3, 33.0, 3.916e-4, 3.929e-4),
                              32: _pp(9.598e-4, 1.032e-3, 370.0, 1.260e-4, 1.294e-4),
                              64: _pp(8.792e-4, 9.585e-4, 5600.0, 4.573e-5, 5.435e-5)},
    "newton_wendland_dynamic": {16: _pp(1.210e-3, 1.325e-3, 24.0, 4.288e-4, 4.576e-4),
                                32: _pp(1.061e-3, 1.133e-3, 250.0, 2.283e-4, 2.338e-4),
                                64: _pp(9.490e-4, 1.024e-3, 4300.0, 1.158e-4, 1.204e-3)},
    "newton_gaussian_dummy": {16: _pp(3.615e-4, 3.713e-4, 68.0), 32: _pp(4.081e-5, 5.087e-5, 740.0),
                              64: _pp(2.010e-5, 2.096e-5, 13000.0)},
    "newton_gaussian_dynamic": {16: _pp(2.083e-3, 2.153e-3, 46.0), 32: _pp(1.033e-3, 1.050e-3, 430.0),
                                64: _pp(5.097e-4, 5.139e-4, 9700.0)},
    "papanastasiou_wendland_dummy": {16: _pp(4.724e-3, 4.815e-3, 95.0), 32: _pp(1.861e-3, 1.894e-3, 1400.0),
                                     64: _pp(7.339e-4, 7.631e-4, 27000.0)},
    "papanastasiou_wendland_dynamic": {16: _pp(3.009e-3, 3.232e-3, 74.0), 32: _pp(1.138e-3, 1.196e-3, 1000.0),
                                       64: _pp(3.715e-4, 6.833e-4, 20000.0)},
    # Wendland at h = 2.5 dp (Sec. 5.3, Table tab:newton-error-wendland-25; no runtimes printed)
    "newton_wendland25_dummy": {16: _pp(6.648e-4, 7.797e-4, None), 32: _pp(5.095e-5, 1.502e-4, None),
                                64: _pp(5.941e-5, 6.696e-5, None)},
    "newton_wendland25_dynamic": {16: _pp(5.436e-3, 5.625e-3, None), 32: _pp(2.588e-3, 2.673e-3, None),
                                  64: _pp(1.300e-3, 1.322e-3, None)},
    "papanastasiou_gaussian_dummy": {16: _pp(7.027e-3, 7.227e-3, 180.0), 32: _pp(2.928e-3, 2.982e-3, 2600.0),
                                     64: _pp(1.336e-3, 1.360e-3, 61000.0)},
    "papanastasiou_gaussian_dynamic": {16: _pp(4.569e-3, 4.769e-3, 130.0), 32: _pp(1.720e-3, 1.790e-3, 1700.0),
                                       64: _pp(7.245e-4, 7.635e-4, 43000.0)},
}


def run_poiseuille_case(dev, case, inv_dp=16, t_end=10.0):
    """One plane Poiseuille flow of Sec. 5 with the full semi-implicit step (sph_step),
    from rest to the viscous relaxation time t = 10 s: L = 1 m, g = 0.05 m/s^2,
    rho0 = 1 kg/m^3, c0 = 6.32 m/s, h = 1.3 dp, dp = 1/inv_dp, dt = 0.3 h / c0 (the
    sound-speed limit of Tables tab:newton-times and tab:papa-times), the wall layout of
    Sec. 5.2 for the boundary model; "wendland25": the Wendland kernel at h = 2.5 dp
    (Table tab:newton-error-wendland-25).  Newtonian: mu = 0.1 Pa s, profile
    u(z) = rho0 g / (2 mu) (L^2/4 - z^2).  Papanastasiou (Sec. 5.4): mu0 = 0.1 Pa s,
    tau0 = 0.0125 Pa, m = 1000 s, the viscosity recomputed from the velocities each
    step, compared with the non-regularised Bingham profile (plug |z| < tau0 / (rho0 g)).
    The l1 and l2 errors and the device time of the whole run, beside the paper's."""
    import numpy as np
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    rheo, kname, bname = case.split("_")
    kern = scenes.KERNEL_GAUSSIAN if kname == "gaussian" else scenes.KERNEL_WENDLAND
    h_factor = 2.5 if kname == "wendland25" else 1.3
    bc = scenes.BC_DYNAMIC if bname == "dynamic" else scenes.BC_DUMMY
    g, mu0, tau0, m, c0 = 0.05, 0.1, 0.0125, 1000.0, 6.32
    s = scenes.poiseuille(bc, kern, inv_dp=inv_dp, h_factor=h_factor)
    L = s.meta["L"]
    dt = 0.3 * s.h / c0
    steps = int(np.ceil(t_end / dt))
    t = {k: torch.from_numpy(getattr(s, k).copy()).to(dev) for k in ("pos", "vel", "rho", "mu", "ptype")}
    st = binding.Stepper(t["pos"], t["vel"], t["rho"], t["mu"], t["ptype"], s.lo, s.hi, s.periodic, s.h,
                         kernel=kern)
    prm = binding.step_params(dt, 1.0, c0, 7.0, (g, 0.0, 0.0), s.boundary, s.mean,
                              max_neighbors={"wendland": 128, "gaussian": 512}.get(kname, 640),
                              rheology=(tau0, mu0, m) if rheo == "papanastasiou" else None)
    opts = binding.solve_opts(rtol=1e-8)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    its = 0
    for _ in range(steps):
        rep = st.step(prm, opts)
        its += rep["half"]["iters"] + rep["full"]["iters"]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    st.close()
    fl = s.ptype == scenes.FLUID
    z = t["pos"].cpu().numpy()[fl, 1].astype(np.float64) - s.meta["centre"]
    u = t["vel"].cpu().numpy()[fl, 0].astype(np.float64)
    exact = 0.5 * g / mu0 * (0.25 * L * L - z * z)
    if rheo == "papanastasiou":
        zp = tau0 / g
        az = np.abs(z)
        u_plug = (0.5 * L - zp) * (g * 0.5 * L - tau0) / (2.0 * mu0)
        exact = np.where(az >= zp, exact - tau0 / mu0 * (0.5 * L - az), u_plug)
    paper = POISEUILLE_PAPER[case][inv_dp]
    out = dict(workload=f"{int(fl.sum())} fluid + {int((~fl).sum())} {bname} wall particles, {steps} steps of "
                        f"dt = {dt:.4g} s to t = {t_end} s", steps=steps, dt=dt,
               run_s=e0.elapsed_time(e1) / 1e3, ms_per_step=e0.elapsed_time(e1) / steps,
               iterations_per_step=its / steps, u_max=float(u.max()), u_max_exact=float(exact.max()), paper=paper)
    for f, k1, k2 in ((1.0, "l1", "l2"), (1.02, "l1_102", "l2_102")):
        if k1 not in paper:
            continue
        e = u - f * exact
        out[k1] = float(np.abs(e).mean())
        out[k2] = float(np.sqrt((e * e).mean()))
    return out


def run_poiseuille(dev, resolutions=(16,), cases=None):
    """Each configuration of POISEUILLE_PAPER (all of them unless `cases` names some) at
    each 1/dp in resolutions, one full run each; with more than one resolution, the
    convergence rates log2(e_coarse / e_fine) of l1 and l2 between consecutive ones (the
    paper prints its own rates beside its errors)."""
    import math

    out = {}
    for case in (cases or POISEUILLE_PAPER):
        runs = {r: run_poiseuille_case(dev, case, r) for r in resolutions}
        if len(resolutions) == 1:
            out[case] = runs[resolutions[0]]
            continue
        for r0, r1 in zip(resolutions, resolutions[1:]):
            for k in ("l1", "l2"):
                runs[r1][f"rate_{k}"] = math.log2(runs[r0][k] / runs[r1][k])
        out[case] = {str(r): v for r, v in runs.items()}
    return out


# --------------------------------------------------------- network forward ----

def run_mlp_forward(dev, m=1157308, reps=20):
    """The warm-start network's inference forward (tcgen05 kernel) on m particles of
    random bf16 features: device time per call, FLOP/s against the measured bf16 peak."""
    import numpy as np
    import torch

    from paper_2206_14780_gb300 import binding

    theta = np.random.default_rng(0).normal(scale=0.2, size=binding.MLP_NPARAMS).astype(np.float32)
    net = binding.Mlp(theta)
    feats = torch.randn((m, 16), device=dev).to(torch.bfloat16).view(torch.int16).contiguous()
    out = torch.empty((m, 4), dtype=torch.float32, device=dev)
    for _ in range(3):
        net.forward(feats, out)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        net.forward(feats, out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    us = 1e3 * e0.elapsed_time(e1) / reps
    flop = 2.0 * (16 * 64 + 64 * 64 + 64 * 64 + 64 * 3) * m        # algorithmic (N = 3 in the last layer)
    peak = None
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        pass
    tflops = flop / (us * 1e-6) / 1e12
    return dict(particles=m, us_per_forward=us, tflops=tflops, peak_tflops=peak,
                frac=(tflops / peak) if peak else None, bytes=48 * m, gbs=48 * m / (us * 1e-6) / 1e9,
                kernel="k_mlp_forward_tc (tcgen05.mma kind::f16, TMEM accumulators)")


def run_mlp_grad(dev, m=1157308, reps=20):
    """The warm-start network's training gradient (tcgen05 forward and backward, then the
    block-order sum of the per-CTA partial gradients) on m rows of random bf16 features
    and targets: device time per sph_mlp_grad call and FLOP/s (forward, data and weight
    gradients) against the measured bf16 peak."""
    import numpy as np
    import torch

    from paper_2206_14780_gb300 import binding

    theta = np.random.default_rng(0).normal(scale=0.2, size=binding.MLP_NPARAMS).astype(np.float32)
    net = binding.Mlp(theta)
    feats = torch.randn((m, 16), device=dev).to(torch.bfloat16).view(torch.int16).contiguous()
    tgt = torch.randn((m, 4), device=dev)
    mask = torch.ones(m, dtype=torch.uint8, device=dev)
    grad = torch.empty(binding.MLP_NPARAMS, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    for _ in range(3):
        net.grad(feats, tgt, mask, m, grad, loss)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        net.grad(feats, tgt, mask, m, grad, loss)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    us = 1e3 * e0.elapsed_time(e1) / reps
    net.close()
    fwd = 16 * 64 + 64 * 64 + 64 * 64 + 64 * 3
    flop = 2.0 * (fwd + (64 * 3 + 64 * 64 + 64 * 64) + fwd) * m   # forward, data gradients (not da_0), weight gradients
    peak = None
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        pass
    tflops = flop / (us * 1e-6) / 1e12
    return dict(rows=m, us_per_grad=us, tflops=tflops, peak_tflops=peak, frac=(tflops / peak) if peak else None,
                kernel="k_mlp_grad_tc (tcgen05.mma kind::f16, MN-major weight-gradient operands) + k_mlp_reduce")


# ----------------------------------------------------------- apply forms ------

def run_apply_forms(nb, params, n, dev, reps=20):
    """The two apply forms on the same operator: stored coefficients (the solver's) and
    coefficients recomputed per pair (the paper's GPU form); device time of the apply
    kernel alone (CUDA events around each launch), algorithmic bytes and GB/s."""
    import torch

    v = torch.randn((n, 4), dtype=torch.float32, device=dev)
    y = torch.empty_like(v)
    nb.apply(params, v, y)
    nb.apply_otf(params, v, y)                     # packs the per-particle geometry
    torch.cuda.synchronize(dev)
    nb.profile(True)
    nb.profile_read(reset=True)
    for _ in range(reps):
        nb.apply(params, v, y)
    for _ in range(reps):
        nb.apply_otf(params, v, y)
    torch.cuda.synchronize(dev)
    c = nb.profile_read(reset=True)
    nb.profile(False)
    out = {}
    for k, (name, nbytes) in enumerate((("stored", c["apply_bytes"] - 16 * n), ("on_the_fly", c["otf_bytes"]))):
        us = 1e3 * c["standalone_ms"][k] / max(1, c["standalone_launches"][k])
        out[name] = dict(us_per_apply=us, algorithmic_bytes=int(nbytes), gbs=nbytes / (us * 1e-6) / 1e9,
                         launches=c["standalone_launches"][k])
    out["note"] = ("y = A v alone (no fused dots); stored: 8 B per coefficient + 41 B per row; on the fly: "
                   "4 B per neighbour-list entry + 61 B per row, coefficients recomputed in float32")
    return out


# ------------------------------------------------------------- ensemble ------

def run_ensemble(seed=0, dev=None, scenes_n=64):
    """64 independent scenes (log-uniform 10k-500k particles, nu in 1-1e3, dt in 1e-4-5e-4):
    one batched solve (persistent kernel in a CUDA graph) vs 64 sequential plain solves."""
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    dev = dev or torch.device("cuda", 0)
    ens = scenes.ensemble(seed, S=scenes_n)
    nbs, bs, ts, params = [], [], [], []
    for s in ens:
        t = binding.scene_tensors(s, dev)
        t["vel"] = torch.from_numpy(s.vel).to(dev)
        ts.append(t)
        nbs.append(binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], s.lo, s.hi, s.periodic, s.h))
        bs.append(torch.from_numpy(s.b).to(dev))
        params.append(binding.visc_params(s.dt, s.boundary, s.mean))
    opts = binding.solve_opts()
    stream = torch.cuda.current_stream(dev)
    xs = [torch.empty_like(b) for b in bs]

    def starts():
        # x0 = v^n with the dummy-wall rows from Eq. dummyvel, per scene
        for nb, p, t, b, x in zip(nbs, params, ts, bs, xs):
            binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)

    def sequential():
        reps = []
        for nb, p, t, b, x in zip(nbs, params, ts, bs, xs):
            binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
            reps.append(nb.solve(p, opts, b, x))
        return reps

    sequential()                                   # warm-up: coefficients + per-handle autotune
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    seq = sequential()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    seq_ms = e0.elapsed_time(e1)
    batch = binding.Batch(nbs, params)
    starts()
    batch.solve(opts, bs, xs)                      # warm-up: autotune + graph capture
    launches0 = binding.launch_count()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    starts()
    st, bat = batch.solve(opts, bs, xs)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    bat_ms = e0.elapsed_time(e1)
    info = batch.info()
    out = dict(workload=f"{len(ens)} scenes (channel/box alternating), totals log-uniform 1e4-5e5 particles, "
                        "nu log-uniform 1-1e3 m^2/s, dt log-uniform 1e-4-5e-4 s; x0 = v^n with the dummy-wall "
                        "closure, inside the timed region of both forms",
               particles=int(sum(s.n for s in ens)), scenes=len(ens),
               sequential_ms=seq_ms, batched_ms=bat_ms, speedup=seq_ms / bat_ms,
               sequential_ms_per_solve=seq_ms / len(ens), batched_ms_per_solve=bat_ms / len(ens),
               sequential_iters=int(sum(r["iters"] for r in seq)), batched_iters=int(sum(r["iters"] for r in bat)),
               max_true_rel_res_sequential=max(r["true_rel_res"] for r in seq),
               max_true_rel_res_batched=max(r["true_rel_res"] for r in bat), batched_status=st,
               batched_launches=binding.launch_count() - launches0, persistent_variant=info["variant"],
               graph=info["graph"], graph_mode={2: "whole solve: conditional WHILE node over the passes",
                                                1: "one pass, replayed per pass",
                                                0: "direct launches"}[info["graph_mode"]],
               persistent_grid=info["grid"], autotune_ms=info["tune_ms"],
               tile_slices=info["tile_slices"], ntiles=info["ntiles"],
               tile_autotune_ms=dict(zip([str(c) for c in info["tile_candidates"]], info["tile_tune_ms"])))
    batch.close()
    for nb in nbs:
        nb.close()
    return out


# ------------------------------------------------------ learned warm start ----

def _starts(nb, p, net, t, b, x0_vn, fl, net_hp=None):
    """The initial guesses: name -> callable filling x (device) and returning nothing."""
    from paper_2206_14780_gb300 import binding

    def zero(x):
        x.copy_(b)
        x[fl] = 0.0

    def vn(x):
        x.copy_(x0_vn)

    def vn_walls(x):
        binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)

    def learned(x):
        binding.warm_start(nb, p, net, t["vel"], t["ptype"], b, x)

    out = dict(zero=zero, vn=vn, vn_walls=vn_walls, learned=learned)
    if net_hp is not None:
        def learned_highpass(x):
            binding.warm_start(nb, p, net_hp, t["vel"], t["ptype"], b, x)

        out["learned_highpass"] = learned_highpass
    return out


def run_learned(weights=None, dev=None, reps=3, mode=None):
    """Learned warm start against x0 = 0, x0 = v^n (walls b) and v^n with the
    dummy-wall closure, on scenes the network never saw: 1.16M-particle lava
    boxes (seeds 1-3) with single solves, and the 64-scene ensemble (seed 1,
    about 8.5M particles) through the batched solver.  Per start: iterations,
    true residual and ms, the warm start's own kernels included."""
    import numpy as np
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding
    from paper_2206_14780_gb300.train_warmstart import DEFAULT_WEIGHTS

    dev = dev or torch.device("cuda", 0)
    path = weights or DEFAULT_WEIGHTS
    if not os.path.exists(path):
        return dict(unavailable=f"no trained weights at {os.path.relpath(path, ROOT)}")
    z = np.load(path)
    net = binding.Mlp(z["params"])
    meta = json.loads(str(z["meta"])) if "meta" in z else {}
    if mode is None:
        mode = int(meta.get("mode", 0))
    net.set_mode(mode)
    net_hp = None
    if not mode & binding.MLP_HIGHPASS:        # the same weights with the high-passed correction
        net_hp = binding.Mlp(z["params"])
        net_hp.set_mode(mode | binding.MLP_HIGHPASS)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    opts = binding.solve_opts()
    out = dict(weights=os.path.relpath(path, ROOT), training=meta.get("train"), mode=mode,
               note="ms = warm start + solve, CUDA events; x0 = 0 and v^n cost a copy")

    # single 1.16M-particle boxes, three unseen seeds (iteration counts move by a few
    # percent with rounding, so one seed decides nothing)
    seeds = (1, 2, 3)
    names = ("zero", "vn", "vn_walls", "learned") + (("learned_highpass",) if net_hp is not None else ())
    per = {k: dict(iters=[], start_ms=[], solve_ms=[], r0_rel=[], true_rel_res=[]) for k in names}
    for sd in seeds:
        s = scenes.lava_box(sd, n=100)
        t = binding.scene_tensors(s, dev)
        t["vel"] = torch.from_numpy(s.vel).to(dev)
        p = binding.visc_params(s.dt, s.boundary, s.mean)
        nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], s.lo, s.hi, s.periodic, s.h)
        b = torch.from_numpy(s.b).to(dev)
        fl = torch.from_numpy(np.flatnonzero(s.ptype == scenes.FLUID)).to(dev)
        x0_vn = torch.from_numpy(s.x0).to(dev)
        x = torch.empty_like(b)
        for name, fill in _starts(nb, p, net, t, b, x0_vn, fl, net_hp).items():
            fill(x)
            nb.solve(p, opts, b, x)                    # warm-up (coefficients, autotune)
            st_ms, so_ms, its, rr = [], [], [], []
            for _ in range(reps):
                torch.cuda.synchronize(dev)
                ev[0].record(stream)
                fill(x)
                ev[1].record(stream)
                rep = nb.solve(p, opts, b, x)
                ev[2].record(stream)
                torch.cuda.synchronize(dev)
                st_ms.append(ev[0].elapsed_time(ev[1]))
                so_ms.append(ev[1].elapsed_time(ev[2]))
                its.append(rep["iters"])
                rr.append(rep["true_rel_res"])
            r = torch.empty_like(b)
            fill(x)
            nb.residual(p, x, b, r)
            d = per[name]
            d["iters"].append(int(np.median(its)))
            d["start_ms"].append(float(np.median(st_ms)))
            d["solve_ms"].append(float(np.median(so_ms)))
            d["r0_rel"].append(float(r.norm() / b.norm()))
            d["true_rel_res"].append(max(rr))
        nb.close()
        del t, b, x, x0_vn
        torch.cuda.empty_cache()
    res = {k: dict(iters=d["iters"], iters_mean=float(np.mean(d["iters"])),
                   start_ms_mean=float(np.mean(d["start_ms"])), solve_ms_mean=float(np.mean(d["solve_ms"])),
                   ms_mean=float(np.mean(d["start_ms"]) + np.mean(d["solve_ms"])), r0_rel=d["r0_rel"],
                   max_true_rel_res=max(d["true_rel_res"])) for k, d in per.items()}
    out["box_1157k"] = dict(workload="lava box 100^3 fluid (N=1,157,308), seeds 1-3, nu=10, dt=5e-4, v~N(0,0.1^2)",
                            **res)

    # 64-scene ensemble through the batched solver
    ens = scenes.ensemble(1)
    nbs, ts, bs, x0s, ps, fls = [], [], [], [], [], []
    for sc in ens:
        tt = binding.scene_tensors(sc, dev)
        tt["vel"] = torch.from_numpy(sc.vel).to(dev)
        ts.append(tt)
        nbs.append(binding.build_neighbors(tt["pos"], tt["rho"], tt["mu"], tt["ptype"], sc.lo, sc.hi, sc.periodic,
                                           sc.h))
        bs.append(torch.from_numpy(sc.b).to(dev))
        x0s.append(torch.from_numpy(sc.x0).to(dev))
        ps.append(binding.visc_params(sc.dt, sc.boundary, sc.mean))
        fls.append(torch.from_numpy(np.flatnonzero(sc.ptype == scenes.FLUID)).to(dev))
    xs = [torch.empty_like(bb) for bb in bs]
    batch = binding.Batch(nbs, ps)
    starts = [_starts(nbs[k], ps[k], net, ts[k], bs[k], x0s[k], fls[k], net_hp) for k in range(len(ens))]
    eres = {}
    for name in names:
        for k in range(len(ens)):
            starts[k][name](xs[k])
        batch.solve(opts, bs, xs)                      # warm-up
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for k in range(len(ens)):
            starts[k][name](xs[k])
        ev[1].record(stream)
        st, reps_ = batch.solve(opts, bs, xs)
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        eres[name] = dict(iters_sum=int(sum(r["iters"] for r in reps_)),
                          iters_max=int(max(r["iters"] for r in reps_)),
                          start_ms=ev[0].elapsed_time(ev[1]), solve_ms=ev[1].elapsed_time(ev[2]),
                          ms=ev[0].elapsed_time(ev[2]), max_true_rel_res=max(r["true_rel_res"] for r in reps_),
                          status=st)
    out["ensemble_64"] = dict(workload=f"64 scenes, seed 1, {sum(sc.n for sc in ens)} particles, batched solve",
                              **eres)
    out["learned_vs_plain"] = learned_vs_plain(out)
    batch.close()
    for nb_ in nbs:
        nb_.close()
    return out


def _scale_heads():
    """The learned wall-row scale (weights/scale_head_mlp.npz) as a head for
    run_precond_scale: features -> network -> exp(y_0) on wall rows."""
    import numpy as np

    from paper_2206_14780_gb300 import binding

    path = os.path.join(ROOT, "paper_2206_14780_gb300", "weights", "scale_head_mlp.npz")
    if not os.path.exists(path):
        return {}
    net = binding.Mlp(np.load(path)["params"])

    def learned_scale(nb, p, t, sc):
        binding.mlp_row_scale(nb, p, net, t["vel"], None)      # installed on the handle directly
        return "installed"

    learned_scale.net = net
    return {"learned_scale": learned_scale}


def run_precond_scale(dev=None, reps=3, fixed=((1.0, 3.0), (0.25, 0.0), (0.125, 0.0)), heads=None):
    """The diagonal preconditioner scale on top of Jacobi (S D^-1 from the left) against
    Jacobi alone, both from v^n with the dummy-wall closure, on the unseen 1.16M-particle
    boxes (seeds 1-3, single solves) and the unseen 64-scene ensemble (seed 1, batched
    solve).  Scales: the closed forms factor norm2^-power on the dummy-wall rows
    (sph_wall_row_scale) for each (factor, power) in fixed, and optional learned heads
    (name -> callable(nb, p, t, out) filling the scale).  ms = the scale's own kernels +
    the solve."""
    import numpy as np
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    dev = dev or torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev4 = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    opts = binding.solve_opts()
    heads = heads or {}

    def scalers():
        out = {"jacobi": None}
        for f, pw in fixed:
            key = f"wall_p{pw:g}" if f == 1.0 else (f"wall_c{f:g}" if pw == 0.0 else f"wall_c{f:g}_p{pw:g}")
            out[key] = (lambda f_, pw_: lambda nb, p, t, sc: nb.wall_row_scale(p, f_, pw_, sc))(f, pw)
        out.update(heads)
        return out

    names = list(scalers())
    per = {k: dict(iters=[], scale_ms=[], solve_ms=[], true_rel_res=[]) for k in names}
    for sd in (1, 2, 3):
        s = scenes.lava_box(sd, n=100)
        t = binding.scene_tensors(s, dev)
        t["vel"] = torch.from_numpy(s.vel).to(dev)
        p = binding.visc_params(s.dt, s.boundary, s.mean)
        nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], s.lo, s.hi, s.periodic, s.h)
        b = torch.from_numpy(s.b).to(dev)
        x = torch.empty_like(b)
        sc = torch.empty(s.n, dtype=torch.float32, device=dev)
        for name, fill_scale in scalers().items():
            sms, so_ms, its, rr = [], [], [], []
            for k in range(reps + 1):                     # the first is a warm-up
                torch.cuda.synchronize(dev)
                ev4[0].record(stream)
                if fill_scale is None:
                    nb.set_row_scale(None)
                elif fill_scale(nb, p, t, sc) != "installed":
                    nb.set_row_scale(sc)
                ev4[1].record(stream)
                binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
                ev4[2].record(stream)
                rep = nb.solve(p, opts, b, x)
                ev4[3].record(stream)
                torch.cuda.synchronize(dev)
                if k == 0:
                    continue
                sms.append(ev4[0].elapsed_time(ev4[1]))
                so_ms.append(ev4[2].elapsed_time(ev4[3]))
                its.append(rep["iters"])
                rr.append(rep["true_rel_res"])
            d = per[name]
            d["iters"].append(int(np.median(its)))
            d["scale_ms"].append(float(np.median(sms)))
            d["solve_ms"].append(float(np.median(so_ms)))
            d["true_rel_res"].append(max(rr))
        nb.set_row_scale(None)
        nb.close()
        del t, b, x, sc
        torch.cuda.empty_cache()
    box = {k: dict(iters=d["iters"], iters_mean=float(np.mean(d["iters"])), scale_ms_mean=float(np.mean(d["scale_ms"])),
                   solve_ms_mean=float(np.mean(d["solve_ms"])),
                   ms_mean=float(np.mean(d["scale_ms"]) + np.mean(d["solve_ms"])),
                   max_true_rel_res=max(d["true_rel_res"])) for k, d in per.items()}
    for k in names:
        box[k]["vs_jacobi"] = dict(iters=box[k]["iters_mean"] / box["jacobi"]["iters_mean"],
                                   ms=box[k]["ms_mean"] / box["jacobi"]["ms_mean"])
    out = dict(note=("x0 = v^n with the dummy-wall closure for every scale; ms = scale kernels (and, on the "
                     "ensemble, one synchronising validation per scene) + solve, CUDA events"),
               box_1157k=dict(workload="lava box 100^3 fluid (N=1,157,308), seeds 1-3", **box))

    ens = scenes.ensemble(1)
    nbs, ts, bs, ps = [], [], [], []
    for sc_ in ens:
        tt = binding.scene_tensors(sc_, dev)
        tt["vel"] = torch.from_numpy(sc_.vel).to(dev)
        ts.append(tt)
        nbs.append(binding.build_neighbors(tt["pos"], tt["rho"], tt["mu"], tt["ptype"], sc_.lo, sc_.hi, sc_.periodic,
                                           sc_.h))
        bs.append(torch.from_numpy(sc_.b).to(dev))
        ps.append(binding.visc_params(sc_.dt, sc_.boundary, sc_.mean))
    xs = [torch.empty_like(bb) for bb in bs]
    scs = [torch.empty(sc_.n, dtype=torch.float32, device=dev) for sc_ in ens]
    eres = {}
    for name, fill_scale in scalers().items():
        def set_all():
            for k in range(len(ens)):
                if fill_scale is None:
                    nbs[k].set_row_scale(None)
                elif fill_scale(nbs[k], ps[k], ts[k], scs[k]) != "installed":
                    nbs[k].set_row_scale(scs[k])

        set_all()                                          # warm-up (first-use buffers of each handle)
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        set_all()
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        scale_ms = ev[0].elapsed_time(ev[1])
        batch = binding.Batch(nbs, ps)
        for k in range(len(ens)):
            binding.warm_start(nbs[k], ps[k], None, ts[k]["vel"], ts[k]["ptype"], bs[k], xs[k])
        batch.solve(opts, bs, xs)                          # warm-up
        for k in range(len(ens)):
            binding.warm_start(nbs[k], ps[k], None, ts[k]["vel"], ts[k]["ptype"], bs[k], xs[k])
        torch.cuda.synchronize(dev)
        ev[1].record(stream)
        st, reps_ = batch.solve(opts, bs, xs)
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        batch.close()
        eres[name] = dict(iters_sum=int(sum(r["iters"] for r in reps_)), iters_max=int(max(r["iters"] for r in reps_)),
                          scale_ms=scale_ms, solve_ms=ev[1].elapsed_time(ev[2]),
                          ms=scale_ms + ev[1].elapsed_time(ev[2]),
                          max_true_rel_res=max(r["true_rel_res"] for r in reps_), status=st)
    for k in names:
        eres[k]["vs_jacobi"] = dict(iters=eres[k]["iters_sum"] / eres["jacobi"]["iters_sum"],
                                    ms=eres[k]["ms"] / eres["jacobi"]["ms"])
    # the plain GPU BiCGSTAB on the same scenes one by one (Jacobi, no batching): what the
    # learned and batched form is measured against
    for k in range(len(ens)):
        nbs[k].set_row_scale(None)
        binding.warm_start(nbs[k], ps[k], None, ts[k]["vel"], ts[k]["ptype"], bs[k], xs[k])
        nbs[k].solve(ps[k], opts, bs[k], xs[k])          # warm-up
    for k in range(len(ens)):
        binding.warm_start(nbs[k], ps[k], None, ts[k]["vel"], ts[k]["ptype"], bs[k], xs[k])
    seq_its, seq_res = 0, 0.0
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    for k in range(len(ens)):
        rep = nbs[k].solve(ps[k], opts, bs[k], xs[k])
        seq_its += rep["iters"]
        seq_res = max(seq_res, rep["true_rel_res"])
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    seq_ms = ev[0].elapsed_time(ev[1])
    eres["jacobi_sequential"] = dict(iters_sum=seq_its, ms=seq_ms, max_true_rel_res=seq_res,
                                     note="the 64 single-scene solves one after another (solves timed, as batched)")
    for k in names:
        eres[k]["vs_sequential_plain"] = dict(iters=eres[k]["iters_sum"] / seq_its, ms=eres[k]["ms"] / seq_ms)
    out["ensemble_64"] = dict(workload=f"64 scenes, seed 1, {sum(sc_.n for sc_ in ens)} particles, batched solve",
                              **eres)
    for nb_ in nbs:
        nb_.close()
    return out


def learned_vs_plain(out):
    """Iterations and ms of each learned start relative to the plain ones (the paper's
    previous-step start v^n, and v^n with the dummy-wall closure), on the unseen boxes
    (means over the seeds) and the unseen ensemble (sums): < 1 means the learned start
    needs fewer."""
    res = {}
    for case, it_key, ms_key in (("box_1157k", "iters_mean", "ms_mean"), ("ensemble_64", "iters_sum", "ms")):
        c = out.get(case, {})
        row = {}
        for learned in ("learned", "learned_highpass"):
            if learned not in c:
                continue
            for plain in ("vn", "vn_walls"):
                if plain in c:
                    row[f"{learned}/{plain}"] = dict(iters=c[learned][it_key] / c[plain][it_key],
                                                     ms=c[learned][ms_key] / c[plain][ms_key])
        res[case] = row
    return res


# ----------------------------------------------------- 200-step sequence ----

def run_sequence(nb, s, b, t, steps, dev):
    """Warm-started sequence on the same A(dt) (positions frozen): step k solves with
    b = v^k + dt g on fluid rows (g a fixed smooth stirring force) and x0 = the previous
    solution v^k (the first from v^0 with the dummy-wall closure), so the field settles
    to a steady stirred state."""
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    p = binding.visc_params(s.dt, s.boundary, s.mean)
    o = binding.solve_opts()
    fl3 = torch.from_numpy(s.ptype == 0).to(dev)[:, None].expand(-1, 3)
    dtg = torch.from_numpy(s.dt * scenes.stirring_force(s)).to(dev)
    bk = b.clone() + dtg
    x = torch.empty_like(b)
    binding.warm_start(nb, p, None, t["vel"], t["ptype"], bk, x)
    its = []
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    for k in range(steps):
        ev[k][0].record(stream)
        rep = nb.solve(p, o, bk, x)
        ev[k][1].record(stream)
        its.append(rep["iters"])
        torch.where(fl3, x + dtg, b, out=bk)       # fluid rows: v^{k+1} + dt g; walls keep b
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - w0
    solve_ms = [a.elapsed_time(c) for a, c in ev]
    return dict(steps=steps, total_solve_ms=sum(solve_ms), ms_per_solve=sum(solve_ms) / steps,
                ms_per_solve_max=max(solve_ms), wall_ms_per_step=1e3 * wall / steps, iters_first=its[0],
                iters_last=its[-1], iters_mean=sum(its) / len(its), last_true_rel_res=rep["true_rel_res"],
                last_status=rep["status"], rms_velocity_last=float(x[fl3[:, 0]].pow(2).mean().sqrt()),
                note="same A(dt) every step (positions frozen), b = previous solution + dt g on fluid rows "
                     "(g: fixed stirring force, 160 m/s^2 sine modes), x0 = previous solution; ms_per_solve "
                     "from CUDA events around each solve, wall_ms_per_step adds the right-hand-side update "
                     "in PyTorch between solves")


# ----------------------------------------------------- precision study ------

# the precision study's subset scenes (tag, plastic viscosity mu0, shear-profile speed U)
SUBSETS = (("default", 1e3, 0.1), ("low_mu0", 1.0, 3.3))


def run_subset(dev, mu0, U, folder, tag):
    """The 57.5k slope subset: GPU mu pass, then the mixed and the all-float64 solves to a
    1e-6 true residual; each solution is saved for the oracle's comparison."""
    import numpy as np
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    s = scenes.slope_subset(0, mu0=mu0, U=U)
    t = binding.scene_tensors(s, dev)
    nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], s.lo, s.hi, s.periodic, s.h)
    vel, wv = torch.from_numpy(s.vel).to(dev), torch.from_numpy(s.wall_vel).to(dev)
    mu = torch.empty(s.n, dtype=torch.float32, device=dev)
    nb.mu_papanastasiou(vel, wv, *s.rheology, mu, set_handle=True)
    p = binding.visc_params(s.dt, s.boundary, s.mean)
    b = torch.from_numpy(s.b).to(dev)
    out = dict(workload=f"slope subset 50x20x50 (N={s.n}), Papanastasiou tau0=100 Pa, mu0={mu0:g} Pa s, U={U:g} m/s",
               particles=s.n)
    for name, prec in (("mixed", binding.SPH_PREC_MIXED), ("fp64", binding.SPH_PREC_FP64)):
        x = torch.from_numpy(s.x0).to(dev)
        rep = nb.solve(p, binding.solve_opts(rtol=1e-6, precision=prec), b, x)
        out[name] = dict(iters=rep["iters"], true_rel_res=rep["true_rel_res"], status=rep["status"])
        np.save(os.path.join(folder, f"subset_{tag}_{name}.npy"), x.cpu().numpy())
    nb.close()
    return out


def run_precision(dev=None, full=True, mu0=1e3, U=0.1):
    """Papanastasiou slope (200x100x200 jittered fluid on a 3-layer floor, 4.12M particles): the mu
    pass, then the mixed (float32 operator, float64 dots and refinement) and all-float64 solves.
    mu0 is the plastic viscosity and U the speed of the seeded shear profile: the defaults give
    mu in 1e3..1e5 Pa s; mu0 = 1 Pa s with U = 3.3 m/s (shear rates up to ~90 1/s) spreads it
    over about 2..7e4 Pa s."""
    import torch

    import scenes
    from paper_2206_14780_gb300 import binding

    dev = dev or torch.device("cuda", 0)
    s = scenes.slope(0, mu0=mu0, U=U) if full else scenes.slope_subset(0, mu0=mu0, U=U)
    t = binding.scene_tensors(s, dev)
    nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], s.lo, s.hi, s.periodic, s.h)
    vel, wv = torch.from_numpy(s.vel).to(dev), torch.from_numpy(s.wall_vel).to(dev)
    mu = torch.empty(s.n, dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    nb.mu_papanastasiou(vel, wv, *s.rheology, mu, set_handle=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    nb.mu_papanastasiou(vel, wv, *s.rheology, mu, set_handle=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    mu_ms = e0.elapsed_time(e1)
    fl = torch.from_numpy(s.ptype == scenes.FLUID).to(dev)
    mu_f = mu[fl]
    p = binding.visc_params(s.dt, s.boundary, s.mean)
    b = torch.from_numpy(s.b).to(dev)
    x0 = torch.from_numpy(s.x0).to(dev)
    res = {}
    xs = {}
    for name, prec, rtol in (("mixed", binding.SPH_PREC_MIXED, 1e-6), ("fp64", binding.SPH_PREC_FP64, 1e-6),
                             ("fp64_tight", binding.SPH_PREC_FP64, 1e-10)):
        x = x0.clone()
        o = binding.solve_opts(rtol=rtol, precision=prec)
        if prec == binding.SPH_PREC_MIXED:
            nb.solve(p, o, b, x)                  # warm-up (coefficients, autotune)
            x = x0.clone()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        rep = nb.solve(p, o, b, x)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        res[name] = dict(ms=e0.elapsed_time(e1), iters=rep["iters"], passes=rep["refinements"],
                         true_rel_res=rep["true_rel_res"], status=rep["status"])
        xs[name] = x
    ref = xs["fp64_tight"]
    for name in ("mixed", "fp64"):
        res[name]["rel_l2_vs_fp64_tight"] = float(torch.linalg.norm(xs[name] - ref) / torch.linalg.norm(ref))
    nb.close()
    return dict(workload=("slope: %dx%dx%d jittered fluid on a 3-layer floor, periodic x/z, Papanastasiou "
                          "tau0=100 Pa, mu0=%g Pa s, m=1000 s, dt=5e-4 s, shear profile U=%g m/s"
                          % (200, 100, 200, mu0, U) if full else "slope subset 50x20x50, mu0=%g, U=%g" % (mu0, U)),
                particles=s.n, mu_pass_ms=mu_ms, mu_min=float(mu_f.min()), mu_max=float(mu_f.max()), **res)


# ------------------------------------------------------------ reference arm ---

def workload_config(n, n_particles):
    """The workload key of the JSON line, identical in both arms."""
    return dict(workload=workload_name(n), n_particles=n_particles, rtol=1e-6,
                l2="inputs larger than L2 (A(dt) coefficients ~1.5 GB), no flush between steps")


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the same workload, one full solve.

    The paper ships no code, so the oracle is the reference.  One step is one solve of
    the whole 1.16M-particle box (neighbours + A + x0 + solve), which takes minutes on
    one core: the arm runs one step whatever --steps asks (a bounded run) and says so;
    no warm-up (nothing to warm on the CPU).  Under torchrun only rank 0 runs it."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    run = OracleRun([dict(kind="box", n=args.box_side, seed=0, x_gpu=None)], None)
    rows, err = run.result()
    if rows is None:
        print(json.dumps(dict(impl="reference", unavailable=f"the oracle worker failed: {err[-300:]}")))
        return
    box = rows[0]
    val = box["sec"] * 1e3
    sample = (f"the full workload, one solve (N={box['n']}), FP64 oracle in one thread: k-d tree neighbours "
              f"{box['neighbours_s']:.1f} s, scipy CSR A {box['assemble_s']:.1f} s, x0 + textbook BiCGSTAB with "
              f"Jacobi restarted to a 1e-6 true residual {box['solve_s']:.1f} s")
    out = dict(metric=METRIC, value=val, unit=UNIT, n_gpus=world, steps=1, warmup=0, steps_requested=args.steps,
               warmup_requested=args.warmup, ms_per_step=val, higher_is_better=False, scaling="weak",
               vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
               config=workload_config(args.box_side, box["n"]),
               note="one full-size solve per run (minutes on one core), so steps = 1 and no warm-up",
               iterations=box["iterations"], passes=box["passes"], true_rel_res=box["true_rel_res"],
               cpu_baseline=dict(value=val, unit=UNIT, cores=1, kind="oracle", sample=sample),
               e2e=dict(value=val, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(out))


def _box_count(n, layers=3):
    m = n + 2 * layers
    return n ** 3 + m * m * layers + 2 * layers * m * n + 2 * layers * n * n


def main():
    args = parse()
    if args.oracle_worker:
        oracle_worker(args.oracle_worker)
        return
    if args.ensemble_only:
        print(json.dumps(run_ensemble(0, scenes_n=args.ensemble_scenes)))
        return
    if args.poiseuille_only:
        import torch

        res = tuple(int(r) for r in args.poiseuille_only.split(","))
        cases = args.poiseuille_cases.split(",") if args.poiseuille_cases else None
        print(json.dumps(run_poiseuille(torch.device("cuda", 0), res, cases)))
        return
    if args.precision_only:
        out = run_precision()
        out["low_plastic_viscosity"] = run_precision(mu0=1.0, U=3.3)
        print(json.dumps(out))
        return
    if args.learned_only:
        import torch

        out = run_learned(args.weights)
        out["mlp_forward"] = run_mlp_forward(torch.device("cuda", 0))
        out["mlp_grad"] = run_mlp_grad(torch.device("cuda", 0))
        out["precond_scale"] = run_precond_scale(torch.device("cuda", 0), heads=_scale_heads())
        print(json.dumps(out))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_sphvisc(args)


if __name__ == "__main__":
    main()
