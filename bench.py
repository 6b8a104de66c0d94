#!/usr/bin/env python3
"""Benchmark: implicit time steps per second of the volume-penalized 2D Riesz
space-fractional diffusion scheme (Eq. 2.17), each step solved by flexible
GMRES with the sine-transform preconditioner (Eq. 4.6) to a true relative
residual of 1e-10, on the 2048 x 2048 convex 12-gon workload
(paper_2102_11576_gb300.workloads, recipe "polygon2048").

One "step" is one implicit time step: right side, initial guess, and the
whole FGMRES solve.  The headline value is the mixed form (preconditioner in
FP32, operator / residual / Arnoldi / Givens in FP64); the plain FP64 form is
measured beside it.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the single-instance solve does not shard (every column pass would
be an all-to-all); N ranks run N independent replicas, no collective on the
data path.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "implicit steps/s at 2048² grid, rel.res 1e-10: mixed vs FP64; % HBM roofline"
UNIT = "steps/s"
WORKLOAD = "polygon2048"
FORM_TEXT = {
    ("fp32", "df32"): "mixed: preconditioner FP32, Arnoldi operator and Krylov basis double-FP32",
    ("fp32", "fp32"): "mixed: preconditioner, Arnoldi operator and Krylov basis FP32",
    ("bf16x3", "fp32"): "mixed: preconditioner split-BF16 on tensor cores, Arnoldi operator and Krylov basis FP32",
    ("bf16", "fp32"): "mixed: preconditioner BF16 on tensor cores (FP32 accumulation), Arnoldi operator and "
                      "Krylov basis FP32",
}
RESID_TEXT = {"df32": "; true residual b - Mx double-FP32 (M x) and FP64 (b - Mx, norm); Hessenberg and Givens FP64",
              "fp64": "; true residual, Hessenberg and Givens FP64"}

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# the kernel classes, with the hash of the CUDA sources that define those
# kernels; reported as null once any of them changes.
TRAFFIC = {
    # profiles/dst_gemm_bf16_polygon2048.md: one preconditioner application
    # (four GEMM launches) 67.82 MB read, nothing written back within them
    "dst_gemm": {"bytes_per_launch": 67821824, "src": "ec2aabe5563973c1",
                 "files": ["common.cuh", "dst_gemm.cu", "dst_gemm.cuh", "umma.cuh"]},
}


def src_hash(files=None):
    """Hash of the CUDA sources `files` (default: every file of csrc/)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2102_11576_gb300", "csrc")
    for f in sorted(files or os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP64 FMA rate: 152 SMs x 2 DFMA per clock per SM x 2 flop x clock (a probe of
# dependent-chain-free DFMA streams measured 1.205 TFLOP/s at ~1.98 GHz).
def fp64_peak_gflops(sm_mhz):
    return 152 * 2 * 2 * sm_mhz / 1e3


def fp32_peak_gflops(sm_mhz):
    return 152 * 128 * 2 * sm_mhz / 1e3


# ---------------------------------------------------------------- clocks -----
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid_hint):
        self.uuid_hint = (uuid_hint or "").lower()
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(", ") for r in out.strip().splitlines() if r.strip()]
        mine = [r for r in rows if len(r) >= 10 and self.uuid_hint and self.uuid_hint in r[1].lower()]
        if not mine:
            idx0 = [r for r in rows if len(r) >= 10 and r[0] == rows[0][0]] if rows else []
            mine = idx0
        if not mine:
            return None
        sm = [float(r[2]) for r in mine if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in mine:
            for k, name in enumerate(names):
                if r[6 + k].strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(mine[0][3]) if mine[0][3].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(mine)}


# ------------------------------------------------------------ our arm ------
def algorithmic_bytes_per_iter(N, m, ez, ev=8):
    """Minimal HBM bytes of one FGMRES(m) iteration, averaged over a cycle:
    precond read v / write z, matvec read z / write w, CGS dots and update over
    the j+1 basis vectors (ev N (2j+4), ev = bytes per basis element), the
    mask, and the per-cycle x update and true residual spread over m
    iterations."""
    cgs = ev * N * (m - 1 + 4)          # mean over j = 0..m-1 of ev N (2j+4)
    pre = (ev + ez) * N
    mv = (ez + ev) * N
    mask = N / 8
    cyc = ((ez * m + 16) * N + (24 + ev) * N) / m
    return pre + mv + cgs + mask + cyc


def kernel_units(name, n1, n2, L1, L2):
    """Algorithmic work of one launch of a kernel class (flops, unit).

    Toeplitz passes: per vector two real FFTs of length L plus 3L pointwise
    flops, 5 L log2 L + 3 L.  Sine-transform passes: the flop count of a
    real DST-I of length n computed as a real FFT of length 2(n+1),
    2.5 * 2(n+1) log2(2(n+1)) per vector and transform."""
    import math
    def dst(n):
        m = 2 * (n + 1)
        return 2.5 * m * math.log2(m)
    if name == "toeplitz_rows":
        return n2 * (5 * L1 * math.log2(L1) + 3 * L1)
    if name == "toeplitz_cols":
        return n1 * (5 * L2 * math.log2(L2) + 3 * L2)
    if name == "dst_rows":
        return n2 * dst(n1)
    if name == "precond_cols":
        return n1 * 3 * dst(n2)
    if name == "precond_rows":
        return n2 * 2 * dst(n1)
    if name.startswith("dst_gemm"):  # one preconditioner apply: the six GEMM-equivalents of Eq. 4.6
        nt = 3 if name.endswith("bf16x3") else 1
        return nt * 2.0 * 3 * (n1 * n1 * n2 + n1 * n2 * n2)
    return None


def max_over_ranks(value, device=None):
    """Maximum of a per-rank float over all ranks (identity for one rank).
    The timed region's duration is the slowest rank's."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed per second of the slowest rank (replicas)."""
    return world * units_per_rank / seconds


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2102_11576_gb300 import Solver, workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workloads.make(args.workload)
    n1, n2, N = w["n1"], w["n2"], w["n1"] * w["n2"]
    mk = dict(restart=w["restart"], tol=w["tol"])
    solver_args = (n1, n2, w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
                   w["dt"], w["eta"])
    u0 = torch.as_tensor(w["u0"]).to(dev)
    peaks, peak_src = measured_peaks()
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    def march(solver, bufs, state, nsteps, stats):
        for _ in range(nsteps):
            prev, prevprev = state
            nxt = ({0, 1, 2} - {prev, prevprev}).pop()
            _, st = solver.step(bufs[prev], None if prevprev is None else bufs[prevprev],
                                out=bufs[nxt])
            stats.append(st)
            state = (nxt, prev)
        return state

    tiles = {}

    def timed_form(precond, matvec, steps, warmup, profile_steps, clocks=None, resid="fp64"):
        solver = Solver(*solver_args, precond=precond, matvec=matvec, use_graph=not args.no_graph, resid=resid,
                        **mk)
        if not args.no_autotune:  # tile shapes by measurement (setup, outside the timed region)
            tiles[f"{precond}+{matvec}"] = solver.autotune(reps=3)
        bufs = [u0.clone(), torch.empty_like(u0), torch.empty_like(u0)]
        state = (0, None)
        state = march(solver, bufs, state, warmup, [])
        barrier()
        l0 = solver.kernel_launches
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if clocks:
            clocks.start()
        e0.record(stream)
        stats = []
        state = march(solver, bufs, state, steps, stats)
        e1.record(stream)
        barrier()
        clk = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        launches = solver.kernel_launches - l0
        ms = max_over_ranks(ms, dev)
        # live per-kernel timing: the same march continued with every launch
        # bracketed by CUDA events on this stream
        prof = None
        if profile_steps:
            solver.profile(True)
            pstats = []
            march(solver, bufs, state, profile_steps, pstats)
            prof = solver.profile_read()
            solver.profile(False)
            prof = {"steps": profile_steps, "kernels": prof,
                    "iters": sum(s["iters"] for s in pstats),
                    "cycles": sum(s["restarts"] + 1 for s in pstats)}
        iters = [s["iters"] for s in stats]
        out = {"ms": ms, "steps": steps, "launches": launches, "clocks": clk, "prof": prof,
               "precond": precond, "matvec": matvec, "resid": resid,
               "iters_per_step": float(np.mean(iters)), "max_rel_res": max(s["rel_res"] for s in stats),
               "all_converged": all(s["converged"] for s in stats), "u": bufs[state[0]].clone()}
        solver.close()
        return out

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    # headline: the mixed form (FP32 preconditioner) with the double-FP32
    # Arnoldi operator; beside it the same with an FP64 operator and the plain
    # FP64 form, each marched from the same u0 over the same steps
    mixed = timed_form(args.precond, args.matvec, args.steps, args.warmup, args.profile_steps, clocks, args.resid)
    head = f"{args.precond}+{args.matvec}"
    others = {}
    if not args.only_headline:
        for pre, mv in (("bf16", args.matvec), ("bf16x3", args.matvec), ("fp32", args.matvec), ("fp32", "df32")):
            if f"{pre}+{mv}" != head and f"{pre}+{mv}" not in others:
                others[f"{pre}+{mv}"] = timed_form(pre, mv, args.steps, args.warmup, args.profile_steps,
                                                   resid=args.resid)
    if not args.no_fp64 and not args.only_headline:
        others["fp32_op64"] = timed_form("fp32", "fp64", args.steps, args.warmup, args.profile_steps)
        others["fp64"] = timed_form("fp64", "fp64", args.fp64_steps, args.warmup, args.profile_steps)
    plain = others.get("fp64")
    value = whole_job_rate(args.steps, world, mixed["ms"] / 1e3)

    # ---- roofline of the dominant kernel (mixed form) ----
    from paper_2102_11576_gb300 import Solver as _S  # noqa: F401
    L1 = 4
    while L1 < 2 * n1 - 1:
        L1 *= 2
    L2 = 4
    while L2 < 2 * n2 - 1:
        L2 *= 2
    roof = None
    kern = mixed["prof"]["kernels"] if mixed["prof"] else {}
    if kern:
        dom = max(kern, key=lambda k: kern[k][0])
        tot_ms, nl = kern[dom]
        iters_p, cycles_p = mixed["prof"]["iters"], mixed["prof"]["cycles"]
        # launches that did work: one per Arnoldi iteration, plus one per true
        # residual for the Toeplitz passes; gated no-op launches after
        # convergence are counted in the time (a few microseconds each)
        work = iters_p + (cycles_p + mixed["prof"]["steps"] if dom.startswith("toeplitz") else 0)
        avg_ms = tot_ms / max(work, 1)
        flops = kernel_units(dom if dom != "dst_gemm" else f"dst_gemm_{mixed['precond']}", n1, n2, L1, L2)
        sm_max = peaks.get("sm_max_mhz", 2070.0)
        bound = "alu"
        if dom == "dst_gemm":
            # tensor cores, timed inside a long step: the sustained measured BF16 rate
            bound, prec_name = "tensor", mixed["precond"]
            peak = 1e3 * peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
            kpeak_src = ("MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16 GEMM back to back)"
                         if "bf16_tflops_sustained" in peaks else "MEASURED_PEAKS.json bf16_tflops")
        elif dom.startswith("toeplitz") and mixed["matvec"] == "fp32":
            prec_name, peak = "fp32", fp32_peak_gflops(sm_max)
            kpeak_src = "152 SMs x 128 FFMA/clk x 2 x sm_max_mhz (derived)"
        elif dom.startswith("toeplitz") and mixed["matvec"] == "df32":
            # double-FP32: each algorithmic flop costs ~10 FP32 operations
            # (df.cuh: sloppy add 10, product 6, the FFT is mostly additions)
            prec_name, peak = "df32", fp32_peak_gflops(sm_max) / 10.0
            kpeak_src = "152 SMs x 128 FFMA/clk x 2 x sm_max_mhz / 10 FP32 ops per df flop (derived)"
        elif dom.startswith("toeplitz"):
            prec_name, peak = "fp64", fp64_peak_gflops(sm_max)
            kpeak_src = "152 SMs x 2 DFMA/clk x 2 x sm_max_mhz (derived)"
        else:
            prec_name, peak = "fp32", fp32_peak_gflops(sm_max)
            kpeak_src = "152 SMs x 128 FFMA/clk x 2 x sm_max_mhz (derived)"
        achieved = flops / (avg_ms / 1e3) / 1e9 if flops else None
        tr = TRAFFIC.get(dom)
        traffic = tr["bytes_per_launch"] if tr and tr.get("src") == src_hash(tr.get("files")) else None
        roof = {"kernel": dom, "bound": bound, "achieved": round(achieved / 1e3, 3) if achieved else None,
                "peak": round(peak / 1e3, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4) if achieved else None, "traffic": traffic,
                "precision": prec_name, "peak_source": kpeak_src,
                "avg_launch_ms": round(avg_ms, 4), "launches_with_work": work,
                "share_of_profiled_time": round(tot_ms / sum(v[0] for v in kern.values()), 4),
                "per_kernel_ms": {k: round(v[0], 3) for k, v in kern.items()},
                "per_kernel_launches": {k: v[1] for k, v in kern.items()}}
    # whole-step HBM roofline (the metric's "% HBM roofline")
    ez = 4 if mixed["precond"] != "fp64" else 8
    ev = {"fp32": 4, "df32": 8, "fp64": 8}[mixed["matvec"]]
    bpi = algorithmic_bytes_per_iter(N, w["restart"], ez, ev)
    bytes_step = mixed["iters_per_step"] * bpi + 40 * N
    ach_gbs = bytes_step / (mixed["ms"] / mixed["steps"] / 1e3) / 1e9
    hbm = {"algorithmic_bytes_per_step": bytes_step, "achieved_GBs": round(ach_gbs, 1),
           "peak_GBs": peaks["hbm_gbs"], "frac": round(ach_gbs / peaks["hbm_gbs"], 4),
           "peak_source": peak_src}

    # ---- end to end through the C ABI with host arrays ----
    e2e = None
    if not args.no_e2e:
        solver = Solver(*solver_args, precond=mixed["precond"], matvec=mixed["matvec"], resid=mixed["resid"], **mk)
        h = [torch.empty((n2, n1), dtype=torch.float64).pin_memory() for _ in range(3)]
        h[0].copy_(torch.as_tensor(w["u0"]))
        hn = [t.numpy() for t in h]
        prev, prevprev = 0, None
        for _ in range(args.warmup):
            nxt = ({0, 1, 2} - {prev, prevprev}).pop()
            solver.step_host(hn[prev], None if prevprev is None else hn[prevprev], out=hn[nxt])
            prevprev, prev = prev, nxt
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            nxt = ({0, 1, 2} - {prev, prevprev}).pop()
            solver.step_host(hn[prev], hn[prevprev], out=hn[nxt])
            prevprev, prev = prev, nxt
        barrier()
        el = max_over_ranks(time.perf_counter() - t0, dev)
        solver.close()
        e2e = {"value": round(whole_job_rate(args.steps, world, el), 4), "unit": UNIT,
               "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": N * 8}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        iters = plain["iters_per_step"] if plain else mixed["iters_per_step"]
        cpu = oracle_sample(w, iters, args.cpu_seconds)

    res = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(mixed["ms"] / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded 12-gon domain, bump initial field)",
        "config": {"workload": f"{WORKLOAD}: {n1}x{n2} grid, convex 12-gon, alpha=(1.3,1.6), k=(1,1), "
                               f"dt=0.02, eta=1e-8, FGMRES({w['restart']}), tol 1e-10",
                   "form": FORM_TEXT.get((args.precond, args.matvec), f"{args.precond}+{args.matvec}")
                   + RESID_TEXT[args.resid],
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"working set > L2 (Krylov basis {w['restart'] + 1} and preconditioned basis "
                         f"{w['restart']} vectors of {N / 1e6:.1f} M values)"},
        "iters_per_step": round(mixed["iters_per_step"], 2),
        "max_rel_res": mixed["max_rel_res"], "all_converged": mixed["all_converged"],
        "forms": {head: {"steps_per_s": round(value / world, 4),
                                "iters_per_step": round(mixed["iters_per_step"], 2),
                                "ms_per_step": round(mixed["ms"] / args.steps, 3)}},
        "hbm_roofline_step": hbm,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": mixed["launches"],
        "tile_shapes": tiles,
        "clocks": mixed["clocks"],
    }
    for name, f in others.items():
        res["forms"][name] = {"steps_per_s": round(f["steps"] / (f["ms"] / 1e3), 4),
                              "iters_per_step": round(f["iters_per_step"], 2),
                              "ms_per_step": round(f["ms"] / f["steps"], 3),
                              "max_rel_res": f["max_rel_res"], "all_converged": f["all_converged"],
                              "kernels_ms": ({k: round(v[0], 2) for k, v in f["prof"]["kernels"].items()}
                                             if f["prof"] else None)}
        if f["steps"] == args.steps:
            a, b = mixed["u"], f["u"]
            res["forms"][name]["headline_vs_this_rel_maxnorm_diff"] = float(
                (a - b).abs().max() / b.abs().max())
    if plain is not None:
        res["forms"]["speedup_headline_over_fp64"] = round(
            res["forms"][head]["steps_per_s"] / res["forms"]["fp64"]["steps_per_s"], 3)
    return res


# ------------------------------------------------------------ oracle -------
def oracle_sample(w, iters_per_step, budget_s):
    """The CPU oracle timed on a bounded sample of one FGMRES iteration of the
    workload, scaled to steps/s.  Sample: the operator M at P random grid
    points (or_apply_M_points) and R row and R column sine transforms of the
    oracle's table-driven routine; one iteration costs N point products plus
    3 x (n2 row + n1 column) transforms (Eq. 4.6 applies three 2D transforms).
    The Gram-Schmidt vector work (~4(j+1)N flops, < 1 % of the transforms)
    is left out."""
    import oracle
    n1, n2 = w["n1"], w["n2"]
    N = n1 * n2
    prob = oracle.Problem(n1, n2, w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"],
                          w["ky"], w["dt"], w["eta"])
    rng = np.random.default_rng(0)
    z = rng.standard_normal((n2, n1))
    share = budget_s / 3.0
    # calibrate sample sizes to the time budget
    P = 256
    t = time.perf_counter()
    prob.apply_M_points(z, rng.choice(N, P, replace=False))
    tp = (time.perf_counter() - t) / P
    P = int(min(N, max(256, share / max(tp, 1e-9))))
    t = time.perf_counter()
    prob.apply_M_points(z, rng.choice(N, P, replace=False))
    tp = (time.perf_counter() - t) / P
    R = 4
    t = time.perf_counter()
    prob.dst2_rows_sample(z, R)
    tr = (time.perf_counter() - t) / R
    R = int(min(n2, max(4, share / max(tr, 1e-9))))
    t = time.perf_counter()
    prob.dst2_rows_sample(z, R)
    tr = (time.perf_counter() - t) / R
    Rc = int(min(n1, max(4, share / max(tr, 1e-9))))
    t = time.perf_counter()
    prob.dst2_cols_sample(z, Rc)
    tc = (time.perf_counter() - t) / Rc
    t_iter = N * tp + 3 * (n2 * tr + n1 * tc)
    t_step = iters_per_step * t_iter
    return {"value": 1.0 / t_step, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"one FGMRES iteration at {n1}x{n2} from M at {P} sampled points and "
                       f"{R} row + {Rc} column sine transforms, scaled to the full grid "
                       f"({t_iter:.1f} s/iteration) x {iters_per_step:.2f} iterations/step"),
            "s_per_iteration": t_iter}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2102_11576_gb300 import workloads
    w = workloads.make(args.workload)
    iters = args.iters_per_step
    per_step = []
    for _ in range(args.warmup):
        oracle_sample(w, iters, args.cpu_seconds / 4)
    for _ in range(args.steps):
        per_step.append(oracle_sample(w, iters, args.cpu_seconds / 4))
    t_iter = statistics.median(p["s_per_iteration"] for p in per_step)
    value = 1.0 / (iters * t_iter)
    cpu = dict(per_step[-1])
    cpu["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded 12-gon domain, bump initial field)",
            "config": {"workload": f"{WORKLOAD}: {w['n1']}x{w['n2']} grid, convex 12-gon, "
                                   f"FGMRES({w['restart']}), tol 1e-10",
                       "iters_per_step": iters},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_op(args):
    """Times one operator-level entry point of the C ABI on the benchmark
    workload (a small, fixed command for ncu captures and per-operator
    timing)."""
    import torch
    from paper_2102_11576_gb300 import Solver, workloads
    w = workloads.make(args.workload)
    prec = args.op.split("_")[1] if args.op.startswith("precond_") else "fp64"
    matvec = args.op.split("_")[2] if args.op.startswith("apply_M_") else "fp64"
    s = Solver(w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
               w["dt"], w["eta"], restart=w["restart"], precond=prec, matvec=matvec)
    rng = np.random.default_rng(0)
    v = torch.as_tensor(rng.standard_normal((w["n2"], w["n1"]))).cuda()
    out = torch.empty_like(v)
    fn = s.dst2 if args.op == "dst2" else (s.apply_M if args.op.startswith("apply_M") else s.apply_precond)
    fn(v, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        fn(v, out)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"op": args.op, "workload": args.workload, "reps": args.reps,
                      "ms_per_call": e0.elapsed_time(e1) / args.reps}), flush=True)


def run_batched(args):
    """Times the batched workload: 256 independent instances (grid side
    uniform in 64..512, random alpha, k, ellipse or polygon domain), each
    advanced by one CUDA graph launch per time step (--batch-precond,
    --matvec, --resid select the precisions), residual to 1e-10."""
    import torch
    from paper_2102_11576_gb300 import Batch, workloads
    probs = workloads.make_batch(seed=0, count=args.batch_count)
    t0 = time.perf_counter()
    b = Batch(probs, precond=args.batch_precond, matvec=args.matvec, resid=args.resid)
    for i, p in enumerate(probs):
        b.set(i, p["u0"])
    if not args.no_autotune:
        b.autotune(reps=3)
    setup_s = time.perf_counter() - t0
    b.run(args.warmup)  # builds the graphs, first steps
    torch.cuda.synchronize()
    l0 = b.kernel_launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st = b.run(args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    unknowns = sum(p["n1"] * p["n2"] for p in probs)
    iters = [s["iters"] for s in st]
    print(json.dumps({"workload": f"batched: {len(probs)} instances, n in 64..512 (sum N = {unknowns}), "
                                  "random alpha/k/domain, FGMRES(20), tol 1e-10",
                      "form": f"{args.batch_precond} preconditioner, {args.matvec} Arnoldi operator and basis, "
                              f"{args.resid} true residual",
                      "steps": args.steps, "ms_per_batch_step": ms / args.steps,
                      "instance_steps_per_s": len(probs) * args.steps / (ms / 1e3),
                      "unknown_steps_per_s": unknowns * args.steps / (ms / 1e3),
                      "iters_last_step": {"mean": float(np.mean(iters)), "max": int(max(iters))},
                      "all_converged": all(s["converged"] for s in st),
                      "max_rel_res": max(s["rel_res"] for s in st),
                      "gpu_launches": b.kernel_launches - l0, "setup_s": setup_s}), flush=True)


def run_adjoint(args):
    """Times one differentiable march of the differentiation workload
    (disk1024: 1024^2, unit disk, alpha = 1.5, 200 steps, sqrt-m
    checkpointing): forward march, then the hand-written adjoint backward
    (gradients wrt u0, k_x, k_y and the per-cell source), after an untimed
    four-step warm-up march and backward."""
    import torch
    from paper_2102_11576_gb300 import Solver, workloads
    from paper_2102_11576_gb300.adjoint import march
    w = workloads.make("disk1024")
    steps = args.steps if args.steps != 10 else w["steps"]
    s = Solver(w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
               w["dt"], w["eta"], restart=w["restart"], tol=w["tol"], precond=args.precond, matvec=args.matvec,
               resid=args.resid)
    dev = torch.device("cuda")
    u0 = torch.as_tensor(w["u0"]).to(dev).requires_grad_(True)
    src = torch.zeros_like(u0).requires_grad_(True)
    kx = torch.tensor(w["kx"], dtype=torch.float64, requires_grad=True)
    ky = torch.tensor(w["ky"], dtype=torch.float64, requires_grad=True)
    target = torch.as_tensor(w["target"]).to(dev)
    # untimed warm-up: a short march and its backward (the first launches of a
    # process load the kernels and capture the graphs)
    leaf = [t.detach().clone().requires_grad_(True) for t in (u0, kx, ky, src)]
    ((march(s, leaf[0], leaf[1], leaf[2], leaf[3], steps=min(steps, 4)) - target) ** 2).sum().backward()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    uT = march(s, u0, kx, ky, src, steps=steps)
    loss = ((uT - target) ** 2).sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    print(json.dumps({"workload": f"disk1024: 1024x1024 unit disk, alpha=(1.5,1.5), {steps} steps, "
                                  f"checkpoint every {math.ceil(math.sqrt(steps))}",
                      "form": f"{args.precond} preconditioner, {args.matvec} Arnoldi operator and basis, "
                              f"{args.resid} true residual",
                      "loss": loss.item(), "forward_s": t1 - t0, "backward_s": t2 - t1,
                      "gradient_evals_per_s": 1.0 / (t2 - t0),
                      "forward_steps_per_s": steps / (t1 - t0),
                      "backward_steps_per_s": steps / (t2 - t1),
                      "dL_dkx": kx.grad.item(), "dL_dky": ky.grad.item(),
                      "grad_u0_norm": u0.grad.norm().item(), "grad_src_norm": src.grad.norm().item()}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batched", action="store_true",
                    help="time the batched workload (256 instances of uneven size)")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-precond", default="bf16")
    ap.add_argument("--adjoint", action="store_true",
                    help="time one differentiable march of the 1024^2 differentiation workload")
    ap.add_argument("--op", choices=["apply_M", "apply_M_df32", "apply_M_fp32", "precond_fp32", "precond_fp64",
                                     "precond_bf16x3", "precond_bf16", "dst2"],
                    default=None,
                    help="time one operator entry point instead of the time march")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--iters-per-step", type=float, default=None,
                    help="FGMRES iterations per step used to scale the oracle's per-iteration "
                         "time in --impl reference (default: the workload's recorded count)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the heuristic tile shapes")
    ap.add_argument("--only-headline", action="store_true", help="time the headline form only")
    ap.add_argument("--precond", choices=["fp32", "bf16", "bf16x3", "fp64"], default="bf16",
                    help="preconditioner precision of the headline form")
    ap.add_argument("--matvec", choices=["fp32", "df32", "fp64"], default="fp32",
                    help="Arnoldi operator (and Krylov basis) precision of the headline form")
    ap.add_argument("--resid", choices=["df32", "fp64"], default="df32",
                    help="arithmetic of the true residual in the mixed forms (the FP64 forms use FP64)")
    ap.add_argument("--no-graph", action="store_true",
                    help="direct kernel launches instead of the graph loop (ncu cannot profile "
                         "kernels inside graphs with conditional nodes)")
    args = ap.parse_args()
    if args.fp64_steps is None:
        args.fp64_steps = args.steps
    if args.op:
        run_op(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return
    if args.batched:
        run_batched(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.iters_per_step is None:
            from paper_2102_11576_gb300 import workloads
            args.iters_per_step = workloads.make(args.workload, n=8)["iters_per_step_recorded"]
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
