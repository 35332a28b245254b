#!/usr/bin/env python
"""Benchmark of the GB300 MTF path (assembly + preconditioned GMRES solve).

Workload (one step = one pass of the whole hot path over one batch): the
unit cube partitioned 4 x 4 x 4 into 64 subcubes (65 blocks, eps_r ~
U[1.5, 6], k0 = 4, 12,000 skeleton triangles, 72,000 unknowns), 16 plane
waves (8 Fibonacci directions x 2 polarisations).  A step re-assembles the
MTF operator (regular + Sauter-Schwab pairs, transmission Grams, block-OSRC
T~ and the tensor-core operator copy), builds the right-hand sides, solves
with block flexible GMRES (all 16 waves in one Krylov space, tensor-core
matvec) inside FP64 iterative refinement to a relative residual that makes
the solution error <= 1e-5, and evaluates the far field on the z = 0 plane.

Metric: solved right-hand sides per second (plus assembly triangle pairs
per second).  ``value`` is device-timed (CUDA events on the launching
stream, inputs resident in HBM); ``e2e`` times the same work through the
C-ABI from host buffers.  The accuracy reference is the solution of the
FP64-assembled system (FP64 residuals of that operator, refined with mixed
solves to 1e-11).  A secondary line runs the split-sphere workload with the
plain FP64 block-OSRC GMRES and the learned correction beside it.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import mtf_inputs as mi  # noqa: E402

METRIC = "solved RHS/sec at 1e-5 rel. err vs FP64 oracle; assembly triangle-pairs/sec"
UNIT = "RHS/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12      # 152 SMs x 128 lanes x FMA x 2.07 GHz
FP64_PEAK_TFLOPS = 1.25                                # GB300 nominal dense FP64
# FP32 operations per kernel evaluation of the regular-pair kernel's
# moment-form inner loop (distance, G and grad G, the moment updates)
FLOPS_PER_EVAL = 57


# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture
# of the current streaming kernels (--set full, launches around Arnoldi column
# 100 of the split-sphere workload, n_total 13,068, 2 right-hand sides; both
# stream tiled operator copies, the block-OSRC one the FP16 T~ on the tensor
# cores, whose tiled rows carry up to 144 bytes of padding each); keyed by
# (kernel, n_total, nrhs), absent for other workloads
NCU_TRAFFIC = {("matvec32", 13068, 2): 232.30e6, ("osrc_apply", 13068, 2): 60.09e6}
# DRAM traffic over algorithmic bytes of the tensor-core Gram-Schmidt streams
# (ncu --set full, one launch each around block step 61 of the 25,920-unknown
# cube, 16 right-hand sides; both read the basis once, so their traffic grows
# with the basis vectors read and is scaled to the launch by this ratio).  The
# dots read the FP16 high part of the basis (1,088 vectors in the captured
# launch: 119.46 MB read and 2.75 MB of row sums written for 119.44 MB of
# algorithmic bytes).
NCU_TRAFFIC_RATIO = {("gmres_dots", 16): 122.21e6 / 119.44e6, ("gmres_axpy", 16): 216.31e6 / 215.65e6}


def _stream_bytes(name, Ns, n_total, nrhs):
    """Algorithmic bytes of one launch of an operator-apply kernel.
    matvec64: FP64 {T, K} entries (32 B per dense entry) + FP64 x reads and y
    writes + the exchange rows (6 entries of 24 B per row), for up to four
    right-hand sides.  matvec32 / osrc_apply (the streaming kernels, one
    launch per group of up to four right-hand sides): every stored entry once
    ({T, K}: 16 B; T~ in the default FP16 copy: 4 B on rows padded to a
    multiple of 4), the FP32 input of the group once (8 B per complex unknown
    and right-hand side) and the per-row piece sums (K floats per piece of
    256 {T, K} or 640 T~ entries, K = 4 or 8 values per right-hand side
    rounded up to a power of two)."""
    nl = min(nrhs, 4)
    if name == "matvec64":
        n_mat = sum(N * N for N in Ns)
        return n_mat * 32 + 2 * n_total * 16 * nl + (n_total // 2) * 6 * 24
    if name == "matvec32":
        mat = sum(N * N * 16 for N in Ns)
        L, raw = 256, 8 * nl
    else:
        mat = sum(N * ((N + 3) & ~3) * 4 for N in Ns)
        L, raw = 640, 4 * nl
    K = 4 if raw <= 4 else 8 if raw <= 8 else 16 if raw <= 16 else 32
    parts = sum(N * -(-N // L) for N in Ns) * K * 4
    return mat + n_total * 8 * nl + parts


def max_over_ranks(seconds, world, device="cuda"):
    """Longest per-rank duration of a phase that all ranks ran concurrently
    (replicas: each rank solves its own instance); the job's throughput is the
    units of all ranks over it.  A single rank returns its own value."""
    if world <= 1:
        return float(seconds)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds, world, device="cuda"):
    """Whole-job throughput of N replicas: world x units_per_rank over the
    slowest rank's time."""
    return world * units_per_rank / max_over_ranks(seconds, world, device)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


def workload(name):
    if name == "split_sphere":
        cfg = mi.config_split_sphere()
        desc = ("split sphere r=1 (equator disk, triple junction), eps_r 2/4, k0=2, 2178 skeleton "
                "triangles, 2 plane waves (x/y pol, +z)")
    elif name == "sphere":
        cfg = mi.config_sphere(2)
        desc = "dielectric sphere r=1 eps_r=2 k0=1, icosphere 320 triangles, 1 plane wave"
    elif name == "cube2":
        cfg = mi.config_cube2()
        desc = "unit cube 2x2x2 subcubes eps U[1.5,4] k0=3, 5832 triangles, 64 plane waves"
    elif name == "cube4":
        cfg = mi.config_cube4()
        desc = "unit cube 4x4x4 subcubes eps U[1.5,6] k0=4, 12000 triangles, 16 plane waves"
    else:
        raise ValueError(name)
    obs_t = np.linspace(0.0, np.pi, 181)
    cfg["obs"] = np.stack([np.cos(obs_t), np.sin(obs_t), 0 * obs_t], axis=1)
    cfg["desc"] = desc
    return cfg


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# oracle (CPU) baseline on a bounded sample
# ----------------------------------------------------------------------------
def oracle_sample(cfg, iters, budget_s=12.0):
    """Time the FP64 oracle on a bounded sample of the workload and
    extrapolate to one full step: assembly of a sample of block 0's triangle
    pairs (regular and singular timed separately), dense matvecs of the full
    block sizes for all right-hand sides at once, times the operator applies
    per right-hand side of the GPU solve (a lower bound for the oracle's own
    GMRES, which is not faster per apply)."""
    from oracle.skeleton import Skeleton
    from oracle.operators import classify_pairs, assemble_block
    from oracle.mtf import MTFSystem

    m = cfg["mesh"]
    sk = Skeleton(m.vertices, m.triangles, m.labels, m.n_domains)
    pr = classify_pairs(sk, 0)
    ntau = 8
    t0 = time.perf_counter()
    sel = np.isin(pr["regular"][0], np.arange(ntau))
    reg = {"regular": (pr["regular"][0][sel], pr["regular"][1][sel])}
    assemble_block(sk, 0, 2.0, pairs=reg)
    t_reg = time.perf_counter() - t0
    sing = {}
    for kind in ("coincident", "edge", "vertex"):
        s = np.isin(pr[kind][0], np.arange(ntau))
        sing[kind] = (pr[kind][0][s], pr[kind][1][s])
    t0 = time.perf_counter()
    assemble_block(sk, 0, 2.0, pairs=sing)
    t_sing = time.perf_counter() - t0
    n_reg = len(reg["regular"][0])
    n_sing = sum(len(v[0]) for v in sing.values())
    counts = np.zeros(3, dtype=np.int64)
    for i in range(sk.n_domains):
        prc = classify_pairs(sk, i)
        counts[0] += len(prc["regular"][0])
        counts[1] += sum(len(prc[k][0]) for k in ("coincident", "edge", "vertex"))
    t_asm = t_reg * counts[0] / max(1, n_reg) + t_sing * counts[1] / max(1, n_sing)
    # matvec cost with full-size dense blocks (random entries, same shapes)
    ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"], assemble=False)
    rng = np.random.default_rng(0)
    ref.T = [rng.standard_normal((n, n)) + 0j for n in sk.N]
    ref.K = [rng.standard_normal((n, n)) + 0j for n in sk.N]
    x = rng.standard_normal((sk.n_total, len(cfg["dirs"]))) + 0j
    t0 = time.perf_counter()
    nmv = 3
    for _ in range(nmv):
        ref.matvec(x)
    t_mv = (time.perf_counter() - t0) / nmv
    t_step = t_asm + (iters + 2) * t_mv
    return {
        "t_step": t_step, "t_assembly": t_asm, "t_matvec": t_mv,
        "sample": (f"measured: oracle assembly of {n_reg} regular + {n_sing} singular pairs of block 0 "
                   f"(test triangles 0..{ntau - 1}) and {nmv} FP64 matvecs with full-size dense blocks for all "
                   f"{x.shape[1]} right-hand sides; extrapolated: assembly to {counts[0]} + {counts[1]} pairs, "
                   f"solve to {iters + 2} operator applies"),
        "pairs_per_s": (n_reg + n_sing) / (t_reg + t_sing),
    }


# ----------------------------------------------------------------------------
# Operator applies per right-hand side of the GPU solve (block steps of the
# block FGMRES, or iterations of the single-vector solve for one wave), as
# the default bench run measured them on a GB300; the reference arm runs
# without the GPU and extrapolates the oracle's step with these counts
# (--ref-iters overrides).
MEASURED_APPLIES = {"cube4": 840, "split_sphere": 439, "sphere": 28, "cube2": 104}


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    iters = args.ref_iters if args.ref_iters > 0 else MEASURED_APPLIES.get(args.workload, 1000)
    vals = []
    res = None
    for _ in range(args.steps):
        res = oracle_sample(cfg, iters)
        vals.append(len(cfg["dirs"]) / res["t_step"])
    v = statistics.median(vals)
    cores = os.cpu_count()
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * res["t_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg["desc"], "nrhs": len(cfg["dirs"])},
            "measured": {"assembly_pairs_per_s": res["pairs_per_s"], "matvec_s": res["t_matvec"],
                         "assembly_s_extrapolated": res["t_assembly"]},
            "extrapolated": f"step = sampled assembly rate x all pairs + {iters + 2} operator applies "
                            f"(the GPU solve's applies per right-hand side) x the measured apply time",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_cuboid_study(args):
    """The concentric-cuboid workload of the paper's Sec. 5.4 (Table 3) on one
    GPU: for M = 1..args.study_m square rings on the grid of spacing
    args.study_h, one JSON line each with the sizes, GMRES iterations, the
    times of the paper's columns (one-time setup, assembly of M and P, solve,
    100 applies of M and of P) and the relative L2([0, pi]) error of RCS_z
    against M = 1 on the finer grid args.study_href (the first line)."""
    import torch
    from paper_2502_10907_gb300.build import build
    build()
    from paper_2502_10907_gb300 import api, _lib as L
    torch.cuda.set_device(0)
    th = np.linspace(0.0, np.pi, 181)
    obs = np.stack([np.cos(th), np.sin(th), 0 * th], axis=1)
    stream = torch.cuda.current_stream()

    def timed(fn, reps=1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0

    def rcs_z(s, x):
        f = s.farfield(x, obs).cpu().numpy()
        return np.abs(f[0, :, 2]) ** 2

    def run(M, h, tol):
        cfg = mi.config_concentric_cuboids(M, h=h)
        t0 = time.perf_counter()
        mesh = api.Mesh.from_inputs(cfg["mesh"])
        t_mesh = time.perf_counter() - t0
        sysg, _, t_setup = timed(lambda: api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1,
                                                     precond=L.MTF_PRECOND_OSRC, tol=tol, restart=args.study_restart,
                                                     max_iter=args.study_max_iter, osrc_np=args.osrc_np))
        _, t_asm, _ = timed(lambda: sysg.reassemble(cfg["k0"], cfg["eps_r"], cfg["mu_r"]))
        sysg.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)  # warm-up (scratch allocation)
        (x, st), t_solve, _ = timed(lambda: sysg.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False))
        xr = torch.randn(1, mesh.n_total, dtype=torch.complex64, device="cuda")
        _, t_mv, _ = timed(lambda: sysg.matvec_f32(xr), 100)
        _, t_pc, _ = timed(lambda: sysg.precond_f32(xr), 100)
        Ns = [int(v) for v in mesh.n_dofs]
        out = dict(M=M, h=h, triangles=int(cfg["mesh"].nt), N=int(mesh.n_total), n_gmres=int(st.iterations),
                   refinements=int(st.refinements), converged=bool(st.converged), rel_residual=float(st.rel_residual),
                   t_setup_s=round(t_setup, 4), t_assembly_s=round(t_asm, 4), t_solver_s=round(t_solve, 4),
                   t_matvec_M_100_s=round(t_mv, 4), t_matvec_P_100_s=round(t_pc, 4),
                   dense_entries_M=int(sum(n * n for n in Ns)), t_mesh_host_s=round(t_mesh, 3))
        rc = rcs_z(sysg, x)
        del sysg, mesh
        torch.cuda.empty_cache()
        return out, rc

    ref, rc_ref = run(1, args.study_href, 1e-7)
    ref["role"] = "reference (M = 1, fine grid)"
    print(json.dumps(ref), flush=True)
    for M in range(1, args.study_m + 1):
        out, rc = run(M, args.study_h, args.study_tol)
        out["rcs_z_rel_l2_err"] = float(np.linalg.norm(rc - rc_ref) / np.linalg.norm(rc_ref))
        print(json.dumps(out), flush=True)


def fp64_reference(api, L, mesh, cfg, restart, osrc_np, tol=1e-11, max_steps=8):
    """Solution of the FP64-assembled system for the workload's plane waves:
    x += (mixed solve of r), r = b - M64 x with the FP64 matvec of the FP64
    assembly (pinned to the oracle by sampled full rows at this size), until
    ||r|| / ||b|| <= tol for every right-hand side.  Returns x and a record."""
    import torch
    s64 = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    b = s64.rhs(cfg["dirs"], cfg["pols"])
    smx = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=L.MTF_PREC_MIXED,
                     precond=L.MTF_PRECOND_OSRC, tol=1e-8, restart=restart, max_iter=8 * restart, max_refine=8,
                     osrc_np=osrc_np)
    x = torch.zeros_like(b)
    bn = b.norm(dim=1)
    rel = 1.0
    steps = 0
    t0 = time.perf_counter()
    for steps in range(max_steps + 1):
        r = b - s64.matvec(x)
        rel = float((r.norm(dim=1) / bn).max())
        if rel <= tol or steps == max_steps:
            break
        d, _ = smx.solve_rhs(r, raise_on_noconv=False)
        x += d
    torch.cuda.synchronize()
    del s64, smx
    return x, {"fp64_rel_residual": rel, "refinement_steps": steps, "seconds": round(time.perf_counter() - t0, 2),
               "method": "FP64 residuals b - M x of the FP64-assembled operator, corrections by mixed solves"}


def run_steps(step, n, stream):
    """Time n calls of step() with CUDA events on the stream; returns
    (ms per step, last result)."""
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(n):
        out = step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n, out


def roofline_of(prof, counts, n_ss, hbm, src):
    """Roofline of the kernel with the largest device time: algorithmic bytes
    declared by the library's launch sites over the measured time (HBM), or
    ALU flops for the assembly kernels."""
    name, (nl, tms, byts) = max(prof.items(), key=lambda kv: kv[1][1])
    per_launch_s = tms / max(1, nl) / 1e3
    if name in ("regular64", "regular32"):
        peak = FP64_PEAK_TFLOPS if name == "regular64" else FP32_PEAK_TFLOPS
        ach = counts[3] * 36 * FLOPS_PER_EVAL / per_launch_s / 1e12
        roof = {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "peak_source": "derived from unit counts and max SM clock"}
    elif name == "singular64":
        npts, per = {0: 6, 1: 5, 2: 2}, {0: 1, 1: 2, 2: 2}
        evals = sum(int(counts[c]) // per[c] * npts[c] * n_ss ** 4 for c in range(3))
        ach = evals * 75 / per_launch_s / 1e12
        roof = {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "peak_source": "derived (FP64 1.25 TF/s)"}
    else:
        ach = byts / (tms / 1e3) / 1e9 if byts > 0 and tms > 0 else None
        roof = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm if ach else None, "traffic": None,
                "algorithmic_bytes_per_launch": byts / max(1, nl), "peak_source": src}
    roof["launches"] = nl
    roof["avg_launch_ms"] = per_launch_s * 1e3
    return roof


def kernel_table(prof):
    out = {}
    for k, (nl, ms, byts) in prof.items():
        if not nl:
            continue
        e = {"launches": nl, "ms": round(ms, 3)}
        if byts > 0 and ms > 0:
            e["GB_per_s"] = round(byts / (ms / 1e3) / 1e9, 1)
        out[k] = e
    return out


def batch_instances(api, L, args):
    """The batched workload: 32 uneven instances (spheres cut by 1..15
    parallel planes into slab subdomains, rotated, 500-5,000 skeleton
    triangles, k0 U[1, 4], eps_r U[1.5, 6]), 8 plane waves each, mixed path
    with block-OSRC at tol 1e-8 and FP64 refinement residuals (residual_fp64:
    on these thin-slab instances the FP32-stored operator alone leaves errors
    up to 1.8e-5 against the FP64 system, whatever the tolerance).  Every system is autotuned for 8
    right-hand sides once; then the batch (mtf_solve_batch, instances
    concurrent) is timed against a loop of mtf_solve over the same systems.
    Accuracy: the largest relative residual over all instances, and the
    solution error of the three largest instances against the FP64 solution
    of fp64_reference (FP64 residuals of the FP64 assembly, refined to
    1e-11; a plain FP64 GMRES stagnates on them at 3e-4 to 3e-2 after 6,000
    iterations)."""
    import torch
    cfgs = mi.config_batch_instances(n_inst=32, seed=0, tri_range=(500, 5000), nrhs=8)
    t0 = time.perf_counter()
    meshes = [api.Mesh.from_inputs(c["mesh"]) for c in cfgs]
    opts = dict(precision=L.MTF_PREC_MIXED, precond=L.MTF_PRECOND_OSRC, tol=1e-8, restart=500, max_iter=4000,
                osrc_np=args.osrc_np, residual_fp64=1)
    systems = [api.System(m, c["k0"], c["eps_r"], c["mu_r"], **opts) for m, c in zip(meshes, cfgs)]
    t_setup = time.perf_counter() - t0
    chosen = {}
    for s in systems:
        plan = s.autotune(8, reps=3)[-1].replace("chosen ", "")
        chosen[plan] = chosen.get(plan, 0) + 1
    dirs = [c["dirs"] for c in cfgs]
    pols = [c["pols"] for c in cfgs]
    nrhs_tot = sum(len(d) for d in dirs)
    api.solve_batch(systems, dirs, pols, raise_on_noconv=False)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xs, st = api.solve_batch(systems, dirs, pols, raise_on_noconv=False)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    for s, d, p in zip(systems, dirs, pols):
        s.solve(d, p, raise_on_noconv=False)
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    big = sorted(range(len(cfgs)), key=lambda i: -int(meshes[i].n_total))[:3]
    errs = []
    for i in big:
        xr, _ = fp64_reference(api, L, meshes[i], cfgs[i], 500, args.osrc_np)
        errs.append(float(((xs[i] - xr).norm(dim=1) / xr.norm(dim=1)).max()))
    n_tot = [int(m.n_total) for m in meshes]
    return {"workload": "32 cut spheres, 500-5000 skeleton triangles, 2-16 slab subdomains, 8 plane waves each",
            "instances": len(cfgs), "nrhs_total": nrhs_tot, "unknowns_min_max": [min(n_tot), max(n_tot)],
            "unknowns_total": sum(n_tot), "setup_seconds": round(t_setup, 2),
            "batch": {"value": nrhs_tot / t_batch, "unit": UNIT, "seconds": t_batch,
                      "how": "mtf_solve_batch: instances on their own streams, 4 host worker threads"},
            "loop": {"value": nrhs_tot / t_loop, "unit": UNIT, "seconds": t_loop, "how": "mtf_solve per instance"},
            "batch_over_loop": t_loop / t_batch,
            "autotune_choices": chosen,
            "converged": all(bool(x.converged) for x in st),
            "max_rel_residual": max(float(x.rel_residual) for x in st),
            "gmres_tol": 1e-8, "refinement_residuals": "FP64 blocks (residual_fp64)",
            "solution_rel_err_vs_fp64_three_largest": errs,
            "timing": "host wall clock around each synchronous call (the batch synchronises its streams)"}


def learned_on_workload(api, L, mesh, cfg, opts, x_ref, plain_iters):
    """The learned correction on the headline workload: a table-parametrised
    stencil fitted (2 rounds x 100 Adam steps, power loss K = 6) and
    validated on 16 other plane waves (one block Krylov space, as the solve),
    then the workload's 16 waves solved with the correction if the fit
    enabled it.  Iterations and error against the plain solve's."""
    sl = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], **opts)
    sl.learned_init("table")
    # 16 validation waves like the workload's (with fewer, restarted block
    # GMRES at restart 600 stalls on this cube: 4 waves reach 2.8e-5 in 4,000 steps)
    d_val = mi.fibonacci_directions(24)[8:16]
    dv = np.concatenate([d_val, d_val])
    pv = np.concatenate(list(mi.orthonormal_polarizations(d_val))).astype(np.complex128)
    t0 = time.perf_counter()
    rep = sl.learned_fit(dv, pv, rounds=2, steps_per_round=100, lr=3e-3, batch=16, K=6, seed=5)
    t_fit = time.perf_counter() - t0
    xl, stl = sl.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
    err = float(((xl - x_ref).norm(dim=1) / x_ref.norm(dim=1)).max()) if x_ref is not None else None
    del sl
    return {"fit": rep, "fit_seconds": round(t_fit, 2), "enabled": bool(rep["enabled"]),
            "gmres_iterations_plain": int(plain_iters), "gmres_iterations": int(stl.iterations),
            "solution_rel_err_vs_fp64": err,
            "note": "table-parametrised stencil on the 72,000 dofs; validation on 16 other waves in one block space; "
                    "enabled only if the validation solve beats plain block-OSRC"}


def osrc_type2_on_workload(api, L, mesh, cfg, opts, x_ref):
    """Block-OSRC Type 1 against Type 2 (T~2 = i R, R real symmetric; the
    wide applies stream R in FP16, 2 bytes per stored entry instead of 4) on
    the headline workload: one timed solve each (after a warm-up solve),
    block steps, error against the FP64 solution, and the device time of one
    16-column apply (CUDA events, 20 applies after 3 warm-ups)."""
    import torch
    n_entries = int(sum(int(n) ** 2 for n in mesh.n_dofs))
    out = {"streamed_bytes_per_apply": {"type1": 4 * n_entries, "type2": 2 * n_entries}}
    rng = torch.Generator(device="cuda")
    rng.manual_seed(7)
    r = torch.randn((16, mesh.n_total), dtype=torch.complex64, device="cuda", generator=rng)
    for t in (1, 2):
        s = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], **dict(opts, osrc_type=t))
        s.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, st = s.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        err = float(((x - x_ref).norm(dim=1) / x_ref.norm(dim=1)).max()) if x_ref is not None else None
        for _ in range(3):
            s.precond_f32(r)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            s.precond_f32(r)
        e1.record()
        torch.cuda.synchronize()
        out[f"type{t}"] = {"solve_seconds": round(secs, 3), "gmres_iterations": int(st.iterations),
                           "converged": bool(st.converged), "solution_rel_err_vs_fp64": err,
                           "apply_ms_16_columns": round(e0.elapsed_time(e1) / 20, 4)}
        del s
    out["note"] = ("Type 2 (reading of Sec. 5.4: symbols with the principal symbols' phase) changes the "
                   "preconditioner, not the solution")
    return out


def secondary_split_sphere(api, L, args, stream):
    """The split-sphere workload (3 blocks, 13,068 unknowns, 2 waves): the
    mixed path, the plain FP64 block-OSRC GMRES and the learned correction on
    the same GPU at equal accuracy (FP64 solve at tol 1e-11 as reference)."""
    cfg = workload("split_sphere")
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    kw = dict(tol=args.tol, restart=500, max_iter=2000, precond=L.MTF_PRECOND_OSRC, osrc_np=args.osrc_np)
    ref = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], tol=1e-11, restart=500, max_iter=4000,
                     precond=L.MTF_PRECOND_OSRC, osrc_np=args.osrc_np)
    x_ref, _ = ref.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
    del ref
    nrhs = len(cfg["dirs"])

    def err(x):
        return float(((x - x_ref).norm(dim=1) / x_ref.norm(dim=1)).max())

    out = {"workload": cfg["desc"], "nrhs": nrhs, "n_unknowns": int(mesh.n_total)}
    sm = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=L.MTF_PREC_MIXED, **kw)

    def step():
        sm.reassemble(cfg["k0"], cfg["eps_r"], cfg["mu_r"])
        x, st = sm.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
        sm.farfield(x, cfg["obs"])
        return x, st

    for _ in range(3):
        step()
    ms, (x, st) = run_steps(step, 5, stream)
    out["mixed"] = {"value": nrhs / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "gmres_iterations": int(st.iterations),
                    "solution_rel_err_vs_fp64": err(x), "converged": bool(st.converged)}
    del sm
    s64 = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], **kw)

    def step64():
        s64.reassemble(cfg["k0"], cfg["eps_r"], cfg["mu_r"])
        x6, st6 = s64.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
        s64.farfield(x6, cfg["obs"])
        return x6, st6

    step64()
    ms64, (x6, st6) = run_steps(step64, 2, stream)
    out["fp64_block_osrc"] = {"value": nrhs / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                              "gmres_iterations": int(st6.iterations), "converged": bool(st6.converged),
                              "solution_rel_err_vs_fp64": err(x6),
                              "path": "FP64 storage, matvec, Arnoldi; block-OSRC (same tolerance, restart, Pade order)"}
    del s64
    sl = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=L.MTF_PREC_MIXED, **kw)
    sl.learned_init("table")
    d_val = mi.fibonacci_directions(9)[0:2]
    p_val = mi.orthonormal_polarizations(d_val)[0].astype(np.complex128)
    t0 = time.perf_counter()
    rep = sl.learned_fit(d_val, p_val, rounds=4, steps_per_round=150, lr=3e-3, batch=16, K=6, seed=5)
    t_fit = time.perf_counter() - t0
    xl, stl = sl.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
    out["learned_correction"] = {"fit": rep, "fit_seconds": t_fit, "enabled": bool(rep["enabled"]),
                                 "gmres_iterations": int(stl.iterations), "solution_rel_err_vs_fp64": err(xl),
                                 "note": "table-parametrised stencil, power loss K = 6, validation on 2 other waves"}
    del sl
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube4")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--precond", default="osrc", choices=["none", "osrc"])
    ap.add_argument("--tol", type=float, default=1e-7)
    # block steps of the block FGMRES (each applies the operator to all
    # right-hand sides), or iterations of the single-vector solver
    ap.add_argument("--restart", type=int, default=600)
    # the Pade order of the OSRC square root is free (N_p >= 1); it only
    # changes the per-mode symbol formed at assembly, not the apply
    ap.add_argument("--osrc-np", type=int, default=16)
    ap.add_argument("--ref-iters", type=int, default=0,
                    help="operator applies per right-hand side for the reference arm's extrapolation "
                         "(0: the count the GPU arm measured for the workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparisons", action="store_true",
                    help="skip the secondary split-sphere line (FP64 path and learned correction)")
    ap.add_argument("--max-iter", type=int, default=4000)
    ap.add_argument("--no-accuracy-gate", action="store_true",
                    help="skip the FP64 reference solution (profiling runs)")
    ap.add_argument("--study", default="", choices=["", "cuboids"],
                    help="instead of the benchmark: the concentric-cuboid study (one JSON line per M)")
    ap.add_argument("--study-m", type=int, default=6)
    ap.add_argument("--study-h", type=float, default=0.18)
    ap.add_argument("--study-href", type=float, default=0.09)
    ap.add_argument("--study-tol", type=float, default=1e-5)
    ap.add_argument("--study-max-iter", type=int, default=12000)
    # restarted at 500 the M >= 4 solves stall; a 4,000-column FP32 basis
    # (2.8 GB at M = 6) lets them converge
    ap.add_argument("--study-restart", type=int, default=4000)
    args = ap.parse_args()
    if args.study == "cuboids":
        return run_cuboid_study(args)
    cfg = workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, cfg)

    import torch
    import torch.distributed as dist
    from paper_2502_10907_gb300.build import build
    build()
    from paper_2502_10907_gb300 import api, _lib as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    prec = L.MTF_PREC_FP64 if args.precision == "fp64" else L.MTF_PREC_MIXED
    pc = L.MTF_PRECOND_OSRC if args.precond == "osrc" else L.MTF_PRECOND_NONE
    m = cfg["mesh"]
    mesh = api.Mesh.from_inputs(m)
    counts = mesh.pair_counts()
    n_pairs = int(counts.sum())
    nrhs = len(cfg["dirs"])
    opts = dict(tol=args.tol, restart=args.restart, precision=prec, max_iter=args.max_iter, precond=pc,
                osrc_np=args.osrc_np)
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], **opts)
    stream = torch.cuda.current_stream()
    x_ref, ref_info = None, None
    if not args.no_accuracy_gate:
        x_ref, ref_info = fp64_reference(api, L, mesh, cfg, args.restart, args.osrc_np)

    def step():
        sysg.reassemble(cfg["k0"], cfg["eps_r"], cfg["mu_r"])
        x, st = sysg.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
        f = sysg.farfield(x, cfg["obs"])
        return x, st, f

    for _ in range(max(3, args.warmup)):
        x, st, f = step()
    torch.cuda.synchronize()
    L.mtf_profile_read_bytes()                # reset counters (launch counts are always kept)
    iters = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        host_split = []
        for _ in range(args.steps):
            x, st, f = step()
            iters.append(st.iterations)
            host_split.append((st.seconds, st.launch_seconds, st.lsq_seconds, st.wait_seconds))
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches_timed = L.mtf_profile_read_bytes()
    ms = ev0.elapsed_time(ev1) / args.steps
    # per-kernel device times: a second pass of the same steps with CUDA
    # events around every library launch (on the launching stream), kept out
    # of the timed region because the event pairs slow the solve down; the
    # per-kernel durations of this pass are upper bounds
    L.mtf_profile_enable(True)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    L.mtf_profile_enable(False)
    prof = L.mtf_profile_read_bytes()
    ms = 1e3 * max_over_ranks(ms / 1e3, world)
    value = world * nrhs / (ms / 1e3)
    err = float(((x - x_ref).norm(dim=1) / x_ref.norm(dim=1)).max()) if x_ref is not None else None
    # assembly alone (device-timed)
    t_asm_ms, _ = run_steps(lambda: sysg.reassemble(cfg["k0"], cfg["eps_r"], cfg["mu_r"]), 3, stream)
    t_asm = t_asm_ms / 1e3
    L.mtf_profile_read_bytes()
    hbm, bf16, src = _peaks()
    launches = sum(v[0] for v in launches_timed.values())
    roof = roofline_of(prof, counts, sysg.opt.n_ss, hbm, src)
    # ALU rooflines of the assembly kernels against the device's measured
    # FP32 / FP64 rates (the library's own FMA-chain probes)
    peaks = L.mtf_probe_peaks()
    asm_roof = []
    for name in ("regular32", "regular64", "singular64"):
        nl, tms, _ = prof.get(name, (0, 0.0, 0.0))
        if not nl or tms <= 0:
            continue
        per = tms / nl / 1e3
        if name.startswith("regular"):
            fl, pk = counts[3] * 36 * FLOPS_PER_EVAL, peaks[0 if name == "regular32" else 1]
        else:
            npts, per_pair = {0: 6, 1: 5, 2: 2}, {0: 1, 1: 2, 2: 2}
            fl = sum(int(counts[c]) // per_pair[c] * npts[c] * sysg.opt.n_ss ** 4 for c in range(3)) * 75
            pk = peaks[1]
        asm_roof.append({"kernel": name, "bound": "alu", "achieved": fl / per / 1e12, "peak": pk / 1e12,
                         "unit": "TFLOP/s", "frac": fl / per / pk, "ms_per_launch": per * 1e3,
                         "peak_source": "measured (mtf_probe_peaks: FP32 / FP64 FMA chains)"})
    roof["traffic"] = NCU_TRAFFIC.get((roof["kernel"], int(mesh.n_total), nrhs))
    ratio = NCU_TRAFFIC_RATIO.get((roof["kernel"], nrhs))
    if roof["traffic"] is None and ratio is not None and roof.get("algorithmic_bytes_per_launch"):
        roof["traffic"] = ratio * roof["algorithmic_bytes_per_launch"]
        roof["traffic_source"] = ("ncu DRAM bytes / algorithmic bytes of one launch of the 25,920-unknown cube "
                                  "(16 rhs), times this launch's algorithmic bytes")

    # ---- end to end through the C-ABI from host buffers ---------------------
    # The step of the timed region (materials re-assembled, plane waves
    # solved, far field) with its inputs taken from host arrays and its
    # results (surface currents and far field) read back to the host every
    # step.  The mesh and system handles are set up once, as long-lived state
    # (their one-time block-OSRC eigen-setup is reported separately below).
    d2h = nrhs * mesh.n_total * 16 + nrhs * len(cfg["obs"]) * 3 * 16
    h2d = 8 + 2 * 8 * m.n_domains + cfg["dirs"].nbytes + cfg["pols"].nbytes + cfg["obs"].nbytes
    mh = api.Mesh(m.vertices, m.triangles, m.labels, m.n_domains)
    sh = api.System(mh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], **opts)
    e2e_times = []
    for it in range(1 + max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sh.reassemble(cfg["k0"], np.asarray(cfg["eps_r"], dtype=np.float64), np.asarray(cfg["mu_r"], dtype=np.float64))
        xe, ste = sh.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
        fe = sh.farfield(xe, cfg["obs"])
        xh, fh = xe.cpu(), fe.cpu()
        torch.cuda.synchronize()
        if it > 0:                                   # the first pass is a warm-up
            e2e_times.append(time.perf_counter() - t0)
    del sh, mh
    e2e = job_throughput(nrhs, statistics.median(e2e_times), world)
    # the same with the mesh and system created from host arrays every step
    # (mesh tables, block-OSRC eigenpairs, assembly), for reference
    h2d_setup = h2d + m.vertices.nbytes + m.triangles.nbytes + m.labels.nbytes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mh = api.Mesh(m.vertices, m.triangles, m.labels, m.n_domains)
    sh = api.System(mh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], **opts)
    xe, ste = sh.solve(cfg["dirs"], cfg["pols"], raise_on_noconv=False)
    fe = sh.farfield(xe, cfg["obs"])
    xh, fh = xe.cpu(), fe.cpu()
    torch.cuda.synchronize()
    e2e_setup = job_throughput(nrhs, time.perf_counter() - t0, world)
    del sh, mh

    secondary = None
    batch = None
    learned = None
    type2 = None
    if rank == 0 and world == 1 and not args.no_comparisons and args.workload != "split_sphere":
        secondary = secondary_split_sphere(api, L, args, stream)
        batch = batch_instances(api, L, args)
        if prec == L.MTF_PREC_MIXED and pc == L.MTF_PRECOND_OSRC:
            learned = learned_on_workload(api, L, mesh, cfg, opts, x_ref, statistics.median(iters))
            type2 = osrc_type2_on_workload(api, L, mesh, cfg, opts, x_ref)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = oracle_sample(cfg, int(statistics.median(iters)))
        cpu = {"value": nrhs / res["t_step"], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": res["sample"], "assembly_pairs_per_s": res["pairs_per_s"], "matvec_s": res["t_matvec"]}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == L.MTF_PREC_FP64 else "f16x3+f32+f64",
            "data": "synthetic",
            "config": {"workload": cfg["desc"], "nrhs": nrhs, "n_unknowns": int(mesh.n_total),
                       "blocks": int(mesh.n_domains), "triangle_pairs": n_pairs, "precision": args.precision,
                       "preconditioner": args.precond, "osrc_pade_order": args.osrc_np, "gmres_tol": args.tol,
                       "krylov": "block FGMRES (one space for all right-hand sides)" if prec == L.MTF_PREC_MIXED
                       else "FGMRES per right-hand side", "restart": args.restart,
                       "matvec": "tcgen05, FP16 hi+lo split, FP32 accumulation" if prec == L.MTF_PREC_MIXED
                       else "FP64",
                       "l2": "inputs larger than L2 (dense blocks re-assembled each step)",
                       "parallelism": f"replicas x{world}"},
            "assembly": {"value": n_pairs / t_asm, "unit": "triangle-pairs/s", "ms": t_asm * 1e3,
                         "roofline": asm_roof},
            "alu_peaks_measured": {"fp32_tflops": peaks[0] / 1e12, "fp64_tflops": peaks[1] / 1e12,
                                   "sfu_gresults_per_s": peaks[2] / 1e9},
            "solution_rel_err_vs_fp64": err,
            "fp64_reference": ref_info,
            "gmres_iterations": int(statistics.median(iters)),
            "converged": bool(st.converged),
            "solve_host_split": {k: round(statistics.median(h[i] for h in host_split), 4) for i, k in
                                 enumerate(("solve_s", "launch_s", "lsq_s", "wait_s"))},
            "gpu_launches": int(launches),
            "kernels": kernel_table(prof),
            "kernel_times": "CUDA events around every library launch in a second pass of the same steps "
                            "(event pairs slow the solve, so that pass is not the timed one); GB/s from the "
                            "algorithmic bytes each launch declares",
            "roofline": roof,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "step": "mtf_reassemble (host eps_r, mu_r) + mtf_solve (host plane waves) + mtf_farfield, "
                            "x and far field read back; mesh and system handles created once"},
            "e2e_with_mesh_setup": {"value": e2e_setup, "unit": UNIT, "h2d_bytes_per_step": int(h2d_setup),
                                    "d2h_bytes_per_step": int(d2h),
                                    "step": "mtf_mesh_create + mtf_assemble (incl. block-OSRC eigenpairs) + "
                                            "mtf_solve + mtf_farfield from host arrays"},
            "cpu_baseline": cpu,
            "secondary": secondary,
            "batched_instances": batch,
            "learned_correction": learned,
            "block_osrc_type2": type2,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
