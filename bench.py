#!/usr/bin/env python3
"""Benchmark: implicit time steps per second of the volume-penalized 2D Riesz
space-fractional diffusion scheme (Eq. 2.17), each step solved by flexible
GMRES with the sine-transform preconditioner (Eq. 4.6) to a true relative
residual of 1e-10, on the 2048 x 2048 convex 12-gon workload
(paper_2102_11576_gb300.workloads, recipe "polygon2048").

One "step" is one implicit time step: right side, initial guess, and the
whole FGMRES solve.  The headline value is the mixed-precision form in which
only the preconditioner (split BF16 on the tensor cores) and the FFT
arithmetic of the Arnoldi operator (FP32, writing an FP64 basis) are reduced:
the Krylov basis, Gram-Schmidt, Hessenberg, Givens least squares, solution
and true residual are FP64 (the residual's Toeplitz products exact: integer
transforms and Chinese remaindering, rounded to FP64).  Beside it: the same
form with the FP64-FFT residual, the FP32 (FFT) preconditioner form, the
double-FP32 operator form, the plain FP64 form, and -- labelled as outside
that precision contract -- the fastest reduced form (BF16 preconditioner,
FP32 basis, double-FP32 residual).  Also timed: the other workloads (disk64,
ellipse512, the 256-instance batch, the disk1024 adjoint).
Prints one JSON line on rank 0.

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

# (preconditioner, operator arithmetic, Krylov basis + Gram-Schmidt, M x of the true residual)
HEADLINE = ("bf16x3", "fp32", "fp64", "exact")
RESID_TEXT = {"fp64": "FP64 (FFT)", "df32": "double-FP32 (FFT)",
              "exact": "exact (integer transforms mod four primes, Chinese remainder; rounded to FP64)"}
PREC_TEXT = {"fp64": "FP64 (FFT)", "fp32": "FP32 (FFT)", "bf16x3": "split BF16 on tensor cores (3 products, FP32 "
             "accumulation)", "bf16": "plain BF16 on tensor cores (FP32 accumulation)", "df32": "double-FP32"}

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per unit of
# work of a hot-path phase (one preconditioner application: its GEMM launches;
# one Gram-Schmidt iteration: multi-dot + update), with the hash of the CUDA
# sources that define those kernels; reported as null once any of them changes.
# gram_schmidt: profiles/gram_schmidt_fp64_polygon2048.md, the multi-dot and
# update of column j = 10 (FP64 basis): 813.5 MB of DRAM traffic against
# 805.3 MB of algorithmic bytes; the per-unit traffic reported is that ratio
# times the mean algorithmic bytes of the profiled iterations.
TRAFFIC = {
    "gram_schmidt": {"traffic_over_algorithmic": 813473280 / 805306368, "src": "310edcbdabee4098",
                     "files": ["common.cuh", "df.cuh", "internal.h", "krylov.cu"]},
}


def form_key(f):
    return "+".join(f)


def in_contract(f):
    """The precision contract: only the preconditioner (FP32 or split BF16)
    and the operator's FFT arithmetic reduced; basis, Gram-Schmidt, Givens and
    the true residual FP64."""
    pre, mv, ba, rs = f
    return pre in ("fp64", "fp32", "bf16x3") and ba == "fp64" and rs in ("fp64", "exact")


def form_text(f):
    pre, mv, ba, rs = f
    t = (f"preconditioner {PREC_TEXT[pre]}; Arnoldi operator arithmetic {PREC_TEXT.get(mv, mv).split(' (')[0]}; "
         f"Krylov basis and Gram-Schmidt {ba.upper() if ba != 'df32' else 'double-FP32'}; true residual M x "
         f"{RESID_TEXT[rs]}, b - M x and its norm FP64; Hessenberg, Givens and "
         f"solution FP64")
    return t + ("" if in_contract(f) else " [outside the FP64-Arnoldi/residual contract]")


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
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# FP64 FMA rate: 152 SMs x 2 DFMA per clock per SM x 2 flop x clock (a probe of
# dependency-free DFMA streams measured 1.205 TFLOP/s at ~1.98 GHz).
def fp64_peak_gflops(sm_mhz):
    return 152 * 2 * 2 * sm_mhz / 1e3


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


# ------------------------------------------------------- byte/flop model -----
def elem_bytes(f):
    """(e_v, e_z): bytes of a Krylov basis element and of a preconditioned vector."""
    pre, mv, ba, rs = f
    return (4 if ba == "fp32" else 8), (8 if pre == "fp64" else 4)


def sum_j(iters, restarts, m):
    """Sum of the Arnoldi column index j over a solve's iterations, with every
    cycle but the last run to m columns (a cycle otherwise ends only at
    convergence)."""
    cycles = restarts + 1
    last = max(0, min(m, iters - (cycles - 1) * m))
    return (cycles - 1) * m * (m - 1) // 2 + last * (last - 1) // 2


def phase_units(f, N, stats, m):
    """Algorithmic HBM bytes of each hot-path phase over a list of per-step
    stats: every grid vector the method must read or write once per use.
      preconditioner (a3), per application: read v (e_v N), write z (e_z N);
      operator (a2), per application: read z, write w, the mask bits;
      Gram-Schmidt (a4), per iteration j: e_v N (2j + 4) (the j+1 basis
        vectors and w read by the dots and again by the update, the new vector
        written);
      true residual (a6), per evaluation: read x and b, the mask bits, write r;
      solution update (a6), per cycle: read the cycle's z, read and write x.
    Returns {phase: (bytes, units)}."""
    ev, ez = elem_bytes(f)
    it = sum(s["iters"] for s in stats)
    cyc = sum(s["restarts"] + 1 for s in stats)
    sj = sum(sum_j(s["iters"], s["restarts"], m) for s in stats)
    return {
        "precond": ((ev + ez) * N * it, it),
        "operator": (((ez + ev) * N + N / 8) * it, it),
        "gram_schmidt": (ev * N * (2 * sj + 4 * it), it),
        "residual": (((16 + ev) * N + N / 8) * (cyc + len(stats)), cyc + len(stats)),
        "xupdate": ((ez * it + 16 * cyc) * N, cyc),
    }


# kernel classes of the library's profiler -> hot-path phase
PHASE_OF = {"toeplitz_rows": "operator", "toeplitz_cols": "operator", "dst_rows": "precond",
            "precond_cols": "precond", "precond_rows": "precond", "dst_gemm": "precond",
            "multidot": "gram_schmidt", "update": "gram_schmidt", "xupdate": "xupdate",
            "resid_rows": "residual", "resid_cols": "residual", "solve_y": "other", "other": "other"}


def gemm_issued_flops(n1, n2, nt):
    """Tensor-core flops issued by one preconditioner application of the GEMM
    form: four GEMMs of the symmetric form (each output pair i, n-1-i from one
    half-width product), n1^2 n2 + n1 n2^2 + 2 n1^2 n2 + 2 n1 n2^2 per BF16
    product, times nt products."""
    if n1 % 2 == 0 and n2 % 2 == 0:
        return nt * 3.0 * (n1 * n1 * n2 + n1 * n2 * n2)
    return nt * 6.0 * (n1 * n1 * n2 + n1 * n2 * n2)


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


def workload_config(w):
    """The workload as both arms name it."""
    return {"workload": f"{WORKLOAD}: {w['n1']}x{w['n2']} grid on [-1,1]^2, convex 12-gon (seed 0), "
                        f"alpha=({w['alpha1']},{w['alpha2']}), k=({w['kx']},{w['ky']}), dt={w['dt']}, "
                        f"eta={w['eta']}, FGMRES({w['restart']}), tol {w['tol']}, u0 masked bump"}


# ------------------------------------------------------------ our arm ------
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2102_11576_gb300 import Solver, workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workloads.make(args.workload)
    n1, n2, N = w["n1"], w["n2"], w["n1"] * w["n2"]
    m = w["restart"]
    mk = dict(restart=m, tol=w["tol"])
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
            _, st = solver.step(bufs[prev], None if prevprev is None else bufs[prevprev], out=bufs[nxt])
            stats.append(st)
            state = (nxt, prev)
        return state

    # FP64 context of the same problem: the oracle-free error bound of every
    # form (Lemma 3.1 with Lemma 2.3: ||M^-1||_inf <= 1, so the last step's
    # solution is within ||b - M u||_inf of the exact solution of its system)
    checker = Solver(*solver_args, **mk)

    def error_bound(bufs, state):
        u_k, u_km1 = bufs[state[0]], bufs[state[1]]
        u_km2 = bufs[({0, 1, 2} - {state[0], state[1]}).pop()]
        b, _ = checker.rhs(u_km1, u_km2)
        r = b - checker.apply_M(u_k)
        torch.cuda.synchronize()
        rinf = r.abs().max().item()
        return {"res_inf": rinf, "err_bound_inf": rinf, "err_bound_rel": rinf / u_k.abs().max().item(),
                "rel_res_fp64": (r.norm() / b.norm()).item()}

    tiles = {}

    def timed_form(f, steps, warmup, profile_steps, clocks=None):
        pre, mv, ba, rs = f
        solver = Solver(*solver_args, precond=pre, matvec=mv, basis=ba, resid=rs, use_graph=not args.no_graph,
                        **mk)
        if not args.no_autotune:  # tile shapes by measurement (setup, outside the timed region)
            tiles[form_key(f)] = solver.autotune(reps=3)
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
        ms = max_over_ranks(e0.elapsed_time(e1), dev)
        launches = solver.kernel_launches - l0
        err = error_bound(bufs, state) if steps >= 2 or warmup >= 1 else None
        u_last = bufs[state[0]].clone()
        # live per-kernel timing: the same march continued with every launch
        # bracketed by CUDA events on this stream
        prof = None
        if profile_steps:
            solver.profile(True)
            pstats = []
            march(solver, bufs, state, profile_steps, pstats)
            prof = {"steps": profile_steps, "kernels": solver.profile_read(), "stats": pstats}
            solver.profile(False)
        solver.close()
        return {"ms": ms, "steps": steps, "launches": launches, "clocks": clk, "prof": prof, "form": f,
                "stats": stats, "iters_per_step": float(np.mean([s["iters"] for s in stats])),
                "max_rel_res": max(s["rel_res"] for s in stats),
                "all_converged": all(s["converged"] for s in stats), "u": u_last, "err": err,
                "bytes_per_step": float(np.mean([s["bytes"] for s in stats]))}

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    head_form = (args.precond, args.matvec, args.basis, args.resid)
    head = timed_form(head_form, args.steps, args.warmup, args.profile_steps, clocks)
    others = {}
    if not args.only_headline:
        extra = [("bf16x3", "fp32", "fp64", "fp64"), ("fp32", "fp32", "fp64", "exact"),
                 ("bf16x3", "df32", "fp64", "exact"), ("bf16", "fp32", "fp32", "df32")]
        if not args.no_fp64:
            extra.append(("fp64", "fp64", "fp64", "fp64"))
        for f in extra:
            if f != head_form and form_key(f) not in others:
                st = args.fp64_steps if f == ("fp64", "fp64", "fp64", "fp64") else args.steps
                others[form_key(f)] = timed_form(f, st, args.warmup, args.profile_steps)
    plain = others.get(form_key(("fp64", "fp64", "fp64", "fp64")))
    value = whole_job_rate(args.steps, world, head["ms"] / 1e3)

    # ---- roofline of the dominant hot-path phase (headline form) ----
    roof, phases = None, None
    if head["prof"]:
        kern = head["prof"]["kernels"]
        pstats = head["prof"]["stats"]
        t_phase = {}
        for k, (ms_k, _) in kern.items():
            t_phase[PHASE_OF.get(k, "other")] = t_phase.get(PHASE_OF.get(k, "other"), 0.0) + ms_k
        units = phase_units(head_form, N, pstats, m)
        phases = {}
        for ph, (byts, nu) in units.items():
            t = t_phase.get(ph, 0.0)
            if t <= 0 or nu <= 0:
                continue
            gbs = byts / (t / 1e3) / 1e9
            phases[ph] = {"ms": round(t, 3), "units": nu, "us_per_unit": round(1e3 * t / nu, 2),
                          "algorithmic_bytes_per_unit": round(byts / nu), "achieved_GBs": round(gbs, 1),
                          "frac_of_hbm": round(gbs / peaks["hbm_gbs"], 4)}
        phases["other"] = {"ms": round(t_phase.get("other", 0.0), 3)}
        dom = max((p for p in phases if p != "other"), key=lambda p: phases[p]["ms"])
        d = phases[dom]
        tr = TRAFFIC.get(dom)
        traffic = None
        if tr and tr.get("src") == src_hash(tr.get("files")) and head_form[2] == "fp64":
            traffic = round(tr["traffic_over_algorithmic"] * d["algorithmic_bytes_per_unit"])
        roof = {"kernel": dom, "bound": "hbm", "achieved": d["achieved_GBs"], "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": d["frac_of_hbm"], "traffic": traffic,
                "traffic_over_algorithmic": (round(traffic / d["algorithmic_bytes_per_unit"], 3)
                                             if traffic else None),
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src}; of measured)",
                "unit_of_work": {"precond": "one preconditioner application",
                                 "operator": "one operator application (row + column pass)",
                                 "gram_schmidt": "one Arnoldi iteration (multi-dot + update)",
                                 "residual": "one true residual", "xupdate": "one solution update"}[dom],
                "us_per_unit": d["us_per_unit"], "algorithmic_bytes_per_unit": d["algorithmic_bytes_per_unit"]}
        if dom == "gram_schmidt" and head_form[2] == "fp64":
            # an FP64 basis makes Gram-Schmidt FP64-pipe bound (ncu: the multi-dot
            # and the update keep the FP64 pipe 86-93 % busy at under 50 % of
            # HBM): (2j + 3) FP64 multiply-adds per grid element at column j
            # (the j + 1 dots, the j + 1 subtractions, the norm), 2 flops each,
            # against 152 SMs x 2 FP64 FMA per clock x 2 flops x the SM clock
            sj = sum(sum_j(s["iters"], s["restarts"], m) for s in pstats)
            it = sum(s["iters"] for s in pstats)
            fl_unit = 2.0 * N * (2 * sj + 3 * it) / it
            gfs = fl_unit / (d["us_per_unit"] / 1e6) / 1e9
            pk = fp64_peak_gflops(peaks.get("sm_max_mhz", 2070.0))
            roof = {"kernel": dom, "bound": "alu", "achieved": round(gfs, 1), "peak": round(pk, 1),
                    "unit": "GFLOP/s (FP64)", "frac": round(gfs / pk, 4), "traffic": traffic,
                    "peak_source": "152 SMs x 2 FP64 FMA/clock x 2 flops x sm_max_mhz (GB300 unit counts)",
                    "unit_of_work": "one Arnoldi iteration (multi-dot + update)",
                    "us_per_unit": d["us_per_unit"], "fp64_flops_per_unit": round(fl_unit),
                    "algorithmic_bytes_per_unit": d["algorithmic_bytes_per_unit"],
                    "hbm": {"achieved": d["achieved_GBs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": d["frac_of_hbm"],
                            "traffic_over_algorithmic": (round(traffic / d["algorithmic_bytes_per_unit"], 3)
                                                         if traffic else None),
                            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src}; of measured)"}}
        if dom == "precond" and head_form[0] in ("bf16", "bf16x3"):
            nt = 3 if head_form[0] == "bf16x3" else 1
            fl = gemm_issued_flops(n1, n2, nt)
            gem_ms = kern["dst_gemm"][0] / d["units"]
            tfs = fl / (gem_ms / 1e3) / 1e12
            pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
            roof["tensor_pipe"] = {"issued_tflop_per_unit": round(fl / 1e12, 4), "achieved_TFLOPs": round(tfs, 1),
                                   "peak_TFLOPs": pk, "frac": round(tfs / pk, 4),
                                   "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"}
    if plain is not None and plain["prof"]:
        # the FP64 form's transforms are FP64-ALU bound: its flops over the FP64 peak
        kern = plain["prof"]["kernels"]
        L1 = 16
        while L1 < 2 * n1 - 1:
            L1 *= 2
        L2 = 16
        while L2 < 2 * n2 - 1:
            L2 *= 2
        pst = plain["prof"]["stats"]
        it = sum(s["iters"] for s in pst)
        nres = sum(s["restarts"] + 1 for s in pst) + len(pst)
        # per application: complex FFT pair of length L per two vectors and direction,
        # 5 L log2 L flops per transform; operator: rows + columns; preconditioner:
        # three 2D sine transforms, each a Bluestein convolution pair per vector
        fft = lambda L: 5.0 * L * math.log2(L)
        op_fl = (n2 / 2) * 2 * fft(L1) + (n1 / 2) * 2 * fft(L2)
        pre_fl = 3 * (n2 * 2 * fft(L1) + n1 * 2 * fft(L2))
        t_op = sum(kern[k][0] for k in ("toeplitz_rows", "toeplitz_cols", "resid_rows", "resid_cols"))
        t_pre = sum(kern[k][0] for k in ("dst_rows", "precond_cols", "precond_rows"))
        fl = op_fl * (it + nres) + pre_fl * it
        pk = fp64_peak_gflops(peaks.get("sm_max_mhz", 2070.0))
        plain["fp64_roofline"] = {"transform_gflop": round(fl / 1e9, 2), "transform_ms": round(t_op + t_pre, 2),
                                  "achieved_GFLOPs": round(fl / ((t_op + t_pre) / 1e3) / 1e9, 1),
                                  "peak_GFLOPs": round(pk, 1), "frac": round(fl / ((t_op + t_pre) / 1e3) / 1e9 / pk, 4),
                                  "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x sm_max_mhz (derived)"}
    # whole-step HBM roofline (the metric's "% HBM roofline"): the library's
    # algorithmic byte count of every step over the step time
    ach_gbs = head["bytes_per_step"] / (head["ms"] / head["steps"] / 1e3) / 1e9
    hbm = {"algorithmic_bytes_per_step": round(head["bytes_per_step"]), "achieved_GBs": round(ach_gbs, 1),
           "peak_GBs": peaks["hbm_gbs"], "frac": round(ach_gbs / peaks["hbm_gbs"], 4),
           "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        pre, mv, ba, rs = head_form
        solver = Solver(*solver_args, precond=pre, matvec=mv, basis=ba, resid=rs, **mk)
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
    checker.close()

    # ---- the other workloads (each a separate, short timed region) ----
    configs = {}
    if not args.no_configs and not args.only_headline:
        for name, fn in (("disk64", run_plain_workload), ("ellipse512", run_plain_workload)):
            configs[name] = fn(name, peaks, dev)
        configs["batched256"] = run_batched_config(args, peaks)
        if args.batch_precond != "bf16x3":  # the headline's form (split-BF16 P-hat, exact residual), labelled extra
            configs["batched256_bf16x3"] = run_batched_config(args, peaks, precond="bf16x3", resid="exact")
        configs["disk1024_adjoint"] = run_adjoint_config(args, head_form)

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        iters = plain["iters_per_step"] if plain else None
        src = "the FP64 GPU form's mean over this run's timed steps" if plain else None
        if iters is None:
            iters = w["iters_per_step_recorded"]
            src = "the FP64 form's recorded mean (workloads.py)"
        cpu = oracle_sample(w, iters, args.cpu_seconds, src)

    config = workload_config(w)
    config.update({"form": form_text(head_form), "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"inputs larger than L2 (Krylov basis {m + 1} and preconditioned basis {m} vectors of "
                         f"{N / 1e6:.1f} M values, 1.2 GB)"})
    res = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(head["ms"] / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+bf16x3+f32+u32",
        "data": "synthetic (seeded 12-gon domain, bump initial field)",
        "config": config,
        "iters_per_step": round(head["iters_per_step"], 2),
        "max_rel_res": head["max_rel_res"], "all_converged": head["all_converged"],
        "error_bound": head["err"],
        "forms": {},
        "hbm_roofline_step": hbm,
        "roofline": roof,
        "phases": phases,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": head["launches"],
        "tile_shapes": tiles,
        "clocks": head["clocks"],
        "configs": configs,
    }
    for name, f in [(form_key(head_form), head)] + list(others.items()):
        fm = {"in_contract": in_contract(f["form"]), "steps_per_s": round(f["steps"] / (f["ms"] / 1e3), 4),
              "iters_per_step": round(f["iters_per_step"], 2), "ms_per_step": round(f["ms"] / f["steps"], 3),
              "max_rel_res": f["max_rel_res"], "all_converged": f["all_converged"], "error_bound": f["err"],
              "hbm_frac_step": round(f["bytes_per_step"] / (f["ms"] / f["steps"] / 1e3) / 1e9 / peaks["hbm_gbs"], 4),
              "kernels_ms": ({k: round(v[0], 2) for k, v in f["prof"]["kernels"].items() if v[1]}
                             if f["prof"] else None)}
        if "fp64_roofline" in f:
            fm["fp64_roofline"] = f["fp64_roofline"]
        if f is not head and f["steps"] == args.steps:
            a, b = head["u"], f["u"]
            fm["headline_vs_this_rel_maxnorm_diff"] = float((a - b).abs().max() / b.abs().max())
        res["forms"][name] = fm
    if plain is not None:
        sp = res["forms"][form_key(head_form)]["steps_per_s"] / res["forms"][form_key(plain["form"])]["steps_per_s"]
        res["speedup_headline_over_fp64"] = round(sp, 3)
    return res


def run_plain_workload(name, peaks, dev):
    """disk64 (64 steps) or ellipse512 (100 steps, FGMRES(30), Gaussian
    source): the plain FP64 method, whole march timed after a 3-step warm-up
    march."""
    import torch
    from paper_2102_11576_gb300 import Solver, workloads
    w = workloads.make(name)
    s = Solver(w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"], w["dt"],
               w["eta"], restart=w["restart"], tol=w["tol"])
    u0 = torch.as_tensor(w["u0"]).to(dev)
    src = None if w["src"] is None else torch.as_tensor(w["src"]).to(dev)
    s.march(u0, 3, src)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, st = s.march(u0, w["steps"], src)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s.close()
    byts = sum(x["bytes"] for x in st)
    return {"workload": f"{name}: {w['n1']}x{w['n2']}, {w['steps']} steps, FGMRES({w['restart']}), FP64",
            "steps_per_s": round(w["steps"] / (ms / 1e3), 2), "iters_per_step": round(np.mean([x["iters"] for x in st]), 2),
            "max_rel_res": max(x["rel_res"] for x in st), "all_converged": all(x["converged"] for x in st),
            "hbm_frac": round(byts / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], 4),
            "l2_note": "working set fits in L2" if w["n1"] * w["n2"] * 8 * (2 * w["restart"] + 8) < 120e6 else None}


def run_batched_config(args, peaks, steps=None, count=None, precond=None, resid=None):
    """The 256-instance batch (grid side uniform in 64..512, random alpha, k,
    ellipse or polygon domain) in its own precisions: FP32 (FFT)
    preconditioner, FP32 operator arithmetic, FP64 basis and FP64 true
    residual; one CUDA graph launch per batch step.  precond="bf16x3": the
    split-BF16 tensor-core preconditioner instead (grouped GEMMs)."""
    import torch
    from paper_2102_11576_gb300 import Batch, workloads
    precond = precond or args.batch_precond
    resid = resid or args.batch_resid
    probs = workloads.make_batch(seed=0, count=count or args.batch_count)
    t0 = time.perf_counter()
    b = Batch(probs, precond=precond, matvec="fp32", basis="fp64", resid=resid,
              use_graph=not args.no_graph)
    for i, p in enumerate(probs):
        b.set(i, p["u0"])
    if not args.no_autotune:
        b.autotune(reps=2)
    setup_s = time.perf_counter() - t0
    b.run(max(args.warmup, 1))
    torch.cuda.synchronize()
    steps = steps or args.batch_steps
    l0 = b.kernel_launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st = b.run(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = b.kernel_launches - l0
    unknowns = sum(p["n1"] * p["n2"] for p in probs)
    b.close()
    iters = [s["iters"] for s in st]
    return {"workload": f"batched: {len(probs)} instances, n in 64..512 (sum N = {unknowns}), random alpha/k/domain, "
                        "FGMRES(20), tol 1e-10",
            "form": f"{precond} preconditioner, FP32 operator arithmetic, FP64 basis, "
                    f"{RESID_TEXT[resid] if resid != 'fp64' else 'FP64'} residual",
            "steps": steps, "ms_per_batch_step": round(ms / steps, 3),
            "instance_steps_per_s": round(len(probs) * steps / (ms / 1e3), 1),
            "unknown_steps_per_s": unknowns * steps / (ms / 1e3),
            "iters_last_step": {"mean": float(np.mean(iters)), "max": int(max(iters))},
            "all_converged": all(s["converged"] for s in st), "max_rel_res": max(s["rel_res"] for s in st),
            "gpu_launches_per_instance_step": round(launches / (len(probs) * steps), 1), "setup_s": round(setup_s, 1)}


def run_adjoint_config(args, form, steps=None):
    """One differentiable march of disk1024 (1024^2, unit disk, alpha 1.5,
    200 steps, sqrt-m checkpointing) and its hand-written adjoint backward
    (gradients wrt u0, k_x, k_y and the per-cell source), after an untimed
    four-step warm-up march and backward."""
    import torch
    from paper_2102_11576_gb300 import Solver, workloads
    from paper_2102_11576_gb300.adjoint import march
    w = workloads.make("disk1024")
    steps = steps or w["steps"]
    pre, mv, ba, rs = form
    s = Solver(w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
               w["dt"], w["eta"], restart=w["restart"], tol=w["tol"], precond=pre, matvec=mv, basis=ba, resid=rs)
    dev = torch.device("cuda")
    u0 = torch.as_tensor(w["u0"]).to(dev).requires_grad_(True)
    src = torch.zeros_like(u0).requires_grad_(True)
    kx = torch.tensor(w["kx"], dtype=torch.float64, requires_grad=True)
    ky = torch.tensor(w["ky"], dtype=torch.float64, requires_grad=True)
    target = torch.as_tensor(w["target"]).to(dev)
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
    s.close()
    return {"workload": f"disk1024: 1024x1024 unit disk, alpha=(1.5,1.5), {steps} steps, checkpoint every "
                        f"{math.ceil(math.sqrt(steps))}", "form": form_key(form),
            "loss": loss.item(), "forward_s": round(t1 - t0, 3), "backward_s": round(t2 - t1, 3),
            "gradient_evals_per_s": round(1.0 / (t2 - t0), 4),
            "forward_steps_per_s": round(steps / (t1 - t0), 2), "backward_steps_per_s": round(steps / (t2 - t1), 2),
            "dL_dkx": kx.grad.item(), "dL_dky": ky.grad.item()}


# ------------------------------------------------------------ oracle -------
def oracle_sample(w, iters_per_step, budget_s, iters_source):
    """The CPU oracle timed on a bounded sample of one FGMRES iteration of the
    workload, scaled to steps/s.  Sample: the operator M at P random grid
    points (or_apply_M_points) and R row and R column sine transforms of the
    oracle's table-driven routine; one iteration costs N point products plus
    3 x (n2 row + n1 column) transforms (Eq. 4.6 applies three 2D transforms).
    The Gram-Schmidt vector work (~4(j+1)N flops, < 1 % of the transforms)
    is left out.  A whole oracle step at 2048^2 takes hours, so the oracle's
    own iteration count there is out of reach: the count comes from the FP64
    form of the same method (the oracle's FGMRES and the GPU's differ only in
    the Gram-Schmidt variant, and agree within one iteration per step
    wherever both run)."""
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
                       f"({t_iter:.1f} s/iteration) x {iters_per_step:.2f} iterations/step ({iters_source})"),
            "s_per_iteration": t_iter}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2102_11576_gb300 import workloads
    w = workloads.make(args.workload)
    iters = args.iters_per_step
    src = "given on the command line" if args.iters_per_step_given else "the FP64 form's recorded mean (workloads.py)"
    per_step = []
    for _ in range(args.warmup):
        oracle_sample(w, iters, args.cpu_seconds / 4, src)
    for _ in range(args.steps):
        per_step.append(oracle_sample(w, iters, args.cpu_seconds / 4, src))
    t_iter = statistics.median(p["s_per_iteration"] for p in per_step)
    value = 1.0 / (iters * t_iter)
    cpu = dict(per_step[-1])
    cpu["value"] = value
    config = workload_config(w)
    config.update({"form": "oracle: plain FP64 C, explicit Toeplitz sums and naive O(n^2) sine transforms",
                   "parallelism": "one host core"})
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded 12-gon domain, bump initial field)",
            "config": config, "iters_per_step": iters,
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batched", action="store_true",
                    help="time only the batched workload (256 instances of uneven size)")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--batch-precond", default="fp32")
    ap.add_argument("--batch-resid", choices=["fp64", "exact"], default="fp64")
    ap.add_argument("--adjoint", action="store_true",
                    help="time only one differentiable march of the 1024^2 differentiation workload")
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
                         "time in --impl reference (default: the workload's recorded FP64-form count)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-autotune", action="store_true", help="keep the heuristic tile shapes")
    ap.add_argument("--only-headline", action="store_true", help="time the headline form only")
    ap.add_argument("--precond", choices=["fp32", "bf16", "bf16x3", "fp64"], default=HEADLINE[0],
                    help="preconditioner precision of the headline form")
    ap.add_argument("--matvec", choices=["fp32", "df32", "fp64"], default=HEADLINE[1],
                    help="Arnoldi operator arithmetic of the headline form")
    ap.add_argument("--basis", choices=["fp32", "df32", "fp64"], default=HEADLINE[2],
                    help="Krylov basis and Gram-Schmidt precision of the headline form")
    ap.add_argument("--resid", choices=["df32", "fp64", "exact"], default=HEADLINE[3],
                    help="arithmetic of M x in the true residual of the headline form")
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
        print(json.dumps(run_adjoint_config(args, (args.precond, args.matvec, args.basis, args.resid),
                                            steps=None if args.steps == 10 else args.steps)), flush=True)
        return
    if args.batched:
        peaks, _ = measured_peaks()
        print(json.dumps(run_batched_config(args, peaks, steps=args.steps)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        args.iters_per_step_given = args.iters_per_step is not None
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
