#!/usr/bin/env python
"""Benchmark: MDoF/s per V-cycle and time to 1e-10 relative residual, mixed
precision (FP32 V-cycle inside FP64 flexible CG) vs plain FP64, on one GB300.

Workload: 3D SIPG Poisson on the unit cube, 64^3 cells, 6 levels, Q3
(16,777,216 DoFs), penalty 2 k(k+1)/h, source f = 3 pi^2 prod sin(pi x_e) at
the nodes plus seeded U[-1,1] noise per DoF (seed 2), b = M_h f, solved from
x = 0 to ||r||/||b|| <= 1e-10.

One step = one complete mixed-precision solve (every kernel of the hot path:
operator apply, colour-pass smoother, restriction, prolongation, coarse solve,
FP64 Krylov vector kernels).  value = DoFs x V-cycles / time, summed over
ranks (each rank solves its own replica: the path is not sharded, so N > 1
runs independent replicas, weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm) on a bounded
sample of the same workload.
"""
import os

# the oracle legs run single-threaded; set before numpy is first imported
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import argparse
import json
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MDoF/s per V-cycle & time to 1e-10 rel. residual, mixed vs FP64 on 1 GB300"
DIM, K, LOG2N, NLEV = 3, 3, 6, 6
RTOL = 1e-10
NOISE_SEED = 2
WORKLOAD = ("3D SIPG Poisson, unit cube, 64^3 cells, 6 levels, Q3 GLL (16.8M DoFs), "
            "gamma = 2k(k+1)/h, f = manufactured 3pi^2 prod sin + U[-1,1] noise (seed 2), "
            "FP32 V-cycle (1+1 vertex-patch smoothing) inside FP64 flexible CG to 1e-10; "
            "plain FP64 solve timed beside it")
# DRAM bytes (read + write) of one launch of a kernel, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum; summaries under profiles/)
# of the library built from sources whose digest is recorded here; reported
# as null once any of those sources has changed since the capture
TRAFFIC = {
    # smooth_int3_kernel<4, float, interior, tile 4>: 126,980,096 read + 11,745,536 written
    "colour_pass": {"bytes": 138725632, "sha": "08f4bc710c210ab4", "tiles": (0, 2, 3, 4),
                    "sources": ["smooth_i_d3_f32_a.cu", "smoother_impl.cuh", "smooth_int3.cuh", "tensor_ops.cuh",
                                "sipg_internal.cuh"]},
    # apply_kernel<3, 4, double>: 134,308,864 read + 98,416,640 written
    "fp64_apply": {"bytes": 232725504, "sha": "9b6eb1bcf65a7765",
                   "sources": ["apply.cu", "apply3.cuh", "tensor_ops.cuh", "sipg_internal.cuh"]},
}
TRAFFIC_SOURCE = "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"


def source_digest(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2405_18982_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(name, tile=None):
    """The recorded DRAM bytes, or None when the kernel's sources changed
    since the capture or (colour pass) the benched tile tiles the patches
    differently from the captured one (tiles 0, 2, 3 share the patch tiling
    and access pattern; the capture ran tile 3)."""
    t = TRAFFIC[name]
    if t["bytes"] is None or t["sha"] != source_digest(t["sources"]):
        return None
    if tile is not None and tile not in t.get("tiles", (tile,)):
        return None
    return t["bytes"]


# peaks (MEASURED_PEAKS.json for HBM; ALU peaks from unit counts x max SM clock)
SMS, FP32_LANES, FP64_UNITS, SM_MAX_MHZ = 152, 128, 2, 2070.0


def fp32_peak_tflops(mhz=SM_MAX_MHZ):
    return SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12


def fp64_peak_tflops(mhz=SM_MAX_MHZ):
    return SMS * FP64_UNITS * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
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
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- algorithmic counts
def _lr_nz(nn, a, c):
    """Structural nonzero (a, c) of the 1D patch SIPG matrix on the two patch
    cells (2nn nodes): the own cell is dense; across the vertex the coupling
    is rank two (the vertex node's row sees the whole other cell, every other
    row only the other cell's node next to the vertex)."""
    return (a // nn == c // nn) or ((a == nn - 1 or c == nn) if a < nn else (a == nn or c == nn - 1))


def colour_pass_schedule_flops(dim, k, packed=True):
    """Flops per interior patch of the colour-pass kernels' sum-factorised
    schedule (Algorithm 1, Eqs. inverse2d / inverse3d): the local residual by
    line sweeps of the 1D patch mass (diagonal plus rank one per cell) and
    SIPG rows (structural zeros skipped; FP32 pairs two rows per packed FMA
    over the union of their nonzeros), then the six (four in 2D) p x p
    eigenvector sweeps and the eigenvalue scaling.  An FMA counts 2."""
    nn, P, p, off = k + 1, 2 * (k + 1), 2 * k, 1

    def mass(acc):
        return 2 * (2 * nn - 1) + p * (4 if acc else 3)

    def sipg():
        f = 0
        if packed:
            for q in range(p // 2):
                a0 = 2 * q + off
                nz = sum(1 for c in range(P) if _lr_nz(nn, a0, c) or _lr_nz(nn, a0 + 1, c))
                f += 2 + 4 * nz
        else:
            for r in range(p):
                f += 1 + 2 * sum(1 for c in range(P) if _lr_nz(nn, r + off, c))
        return f

    st = p * (2 * p - 1)
    if dim == 3:
        x = P * P * (mass(False) + sipg()) + 4 * P * mass(False)
        y = p * P * (mass(False) + sipg() + mass(True)) + 2 * p * mass(False)
        z = p * p * (sipg() + mass(True) + p)
        return x + y + z + 6 * p * p * st + p ** 3
    x = P * (mass(False) + sipg()) + 2 * mass(False)
    y = p * (sipg() + mass(True) + 1)
    return x + y + 4 * p * st + p ** 2


def smoother_counts(dim, k, N, colour, s_bytes):
    """One colour pass over its interior patches.  Returns (survey flops,
    schedule flops, bytes, patches): survey = the reference count with dense
    1D operators, residual 4pP^3 + 6p^2P^2 + 4p^3P (2D 4pP^2 + 4p^2P) plus FD
    4d p^(d+1) + p^d per patch (P = 2(k+1), p = 2k); schedule =
    colour_pass_schedule_flops (the work the kernels do); bytes = the
    colour-pass model (P^d + 2p^d) s per patch: x read on the patch cells,
    b read and x written on V_j."""
    n = k + 1
    P, p = 2 * n, 2 * k
    npatch = 1
    for e in range(dim):
        npatch *= N // 2 if (colour >> e) & 1 else N // 2 - 1
    if dim == 3:
        fl = 4 * p * P ** 3 + 6 * p * p * P * P + 4 * p ** 3 * P + 4 * dim * p ** (dim + 1) + p ** dim
    else:
        fl = 4 * p * P * P + 4 * p * p * P + 4 * dim * p ** (dim + 1) + p ** dim
    by = (P ** dim + 2 * p ** dim) * s_bytes
    sched = colour_pass_schedule_flops(dim, k, packed=(s_bytes == 4))
    return npatch * fl, npatch * sched, npatch * by, npatch


def apply_counts(dim, k, N, s_bytes):
    """Operator apply y = A x (Sec. 2.2, sum-factorised): flops of the
    kernel's schedule per DoF -- d normal sweeps with the n x n 1D blocks
    (2n each), the rank-two neighbour couplings along each direction where a
    neighbour exists ((8n + 2)/n per DoF), and the mass sweeps as diagonal
    plus rank one (3D: 3 plain (5 - 1/n) + 2 accumulating (6 - 1/n); 2D: one
    of each); bytes = read x + write y.  3D interior: 6n + 51 + 1/n."""
    n = k + 1
    nd = N ** dim * n ** dim
    nb = dim * (8 * n + 2) / n * (N - 1) / N
    if dim == 3:
        per = 6 * n + nb + 3 * (5 - 1 / n) + 2 * (6 - 1 / n)
    else:
        per = 4 * n + nb + (5 - 1 / n) + (6 - 1 / n)
    return nd * per, nd * 2 * s_bytes


# ----------------------------------------------------------------- our arm
def reduce_over_ranks(dist, v, op, device):
    """One float reduced over all ranks ("max" or "sum"); v itself on one rank."""
    import torch
    if dist is None:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_mdofs(dist, device, ndofs, vcycles, seconds):
    """Whole-job MDoF/s per V-cycle: every rank solves its own replica of the
    problem (ndofs DoFs, `vcycles` V-cycles in `seconds` on this rank); the
    units of all ranks divided by the slowest rank's time.  Returns (value,
    slowest time)."""
    t_max = reduce_over_ranks(dist, seconds, "max", device)
    total = reduce_over_ranks(dist, float(vcycles), "sum", device)
    return ndofs * total / t_max / 1e6, t_max


C3 = (3, 7, 5, 5)   # dim, k, log2 N, levels: Q7 on 32^3 cells (16.8M DoFs)
C3_SEED = 3


def c3_record(torch, dev, reps=3):
    """3D Q7 on 32^3 cells, f ~ N(0,1) per DoF (seed 3), b = M f: FP64 outer
    flexible CG to 1e-10 preconditioned by the FP32 V-cycle and by the TF32
    one (tensor-core fast-diagonalisation sweeps in the interior colour
    passes), each solution's error against the FP64-V-cycle solve, and the
    finest interior colour pass of each (colour 0, CUDA events)."""
    from paper_2405_18982_gb300 import SIPG, SIPG_FP32, SIPG_FP64, SIPG_TF32, Params, inputs
    dim, k, l2, nl = C3
    out = {"workload": "3D SIPG Poisson, 32^3 cells, Q7 (16.8M DoFs), 5 levels, f ~ N(0,1) seed 3, "
                       "FP64 flexible CG to 1e-10"}
    sol = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    b = None
    for tag, prec in (("fp64", SIPG_FP64), ("fp32", SIPG_FP32), ("tf32", SIPG_TF32)):
        s = SIPG(Params(dim=dim, degree=k, log2_cells=l2, n_levels=nl, vcycle_precision=prec, use_graphs=1),
                 device=dev)
        if b is None:
            f = torch.from_numpy(inputs.normal(C3_SEED, s.ndofs())).to(dev).view(1, -1)
            b = torch.zeros_like(f)
            s.rhs(f, b)
        x = torch.zeros_like(b)
        s.solve(b, x, rtol=1e-10, maxit=100, zero_start=True)   # warm-up (graph capture)
        torch.cuda.synchronize()
        n_rep = 1 if prec == SIPG_FP64 else reps
        e0.record(stream)
        for _ in range(n_rep):
            info = s.solve(b, x, rtol=1e-10, maxit=100, zero_start=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / n_rep
        rec = {"time_to_1e-10_s": round(t, 5), "iterations": info.iterations, "rel_residual": info.rel_residual,
               "mdofs_per_vcycle": round(s.ndofs() * info.iterations / t / 1e6, 1)}
        if prec != SIPG_FP64:
            bf = b.float()
            xf = torch.zeros_like(bf)
            L = nl - 1
            for _ in range(3):
                s.smooth_colour(L, 0, bf, xf)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(10):
                s.smooth_colour(L, 0, bf, xf)
            e1.record(stream)
            torch.cuda.synchronize()
            rec["colour_pass_us"] = round(e0.elapsed_time(e1) / 10 * 1e3, 2)
        sol[tag] = x
        out[tag] = rec
        s.close()
        del s
    for tag in ("fp32", "tf32"):
        out[tag]["solution_rel_l2_vs_fp64"] = float(((sol[tag] - sol["fp64"]).norm() / sol["fp64"].norm()).item())
    del sol
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2405_18982_gb300 as pkg
    from paper_2405_18982_gb300 import SIPG, SIPG_FP32, SIPG_FP64, Params, inputs
    pkg.load(pkg.build())

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        return reduce_over_ranks(dist, v, "max", dev)

    def sum_over_ranks(v):
        return reduce_over_ranks(dist, v, "sum", dev)

    mk = lambda prec: SIPG(Params(dim=DIM, degree=K, log2_cells=LOG2N, n_levels=NLEV,
                                  vcycle_precision=prec, use_graphs=1), device=dev)
    s_mix = mk(SIPG_FP32)
    s_64 = mk(SIPG_FP64)
    n = s_mix.ndofs()
    f = torch.zeros(1, n, dtype=torch.float64, device=dev)
    s_mix.manufactured_source(f)
    f += torch.from_numpy(inputs.uniform(NOISE_SEED, n)).to(dev).view(1, n)
    b = torch.zeros_like(f)
    s_mix.rhs(f, b)
    x = torch.zeros_like(f)
    stream = torch.cuda.current_stream(dev)

    # ---- warm-up (also captures the CUDA graphs)
    for _ in range(args.warmup):
        s_mix.solve(b, x, rtol=RTOL, maxit=200, zero_start=True)
    torch.cuda.synchronize()

    # ---- timed region: K mixed-precision solves
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = s_mix.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    # (an NVTX range around the timed solves, so that a profiler's launch
    # list can be restricted to them)
    torch.cuda.nvtx.range_push("timed_mixed_solves")
    ev0.record(stream)
    for _ in range(args.steps):
        info = s_mix.solve(b, x, rtol=RTOL, maxit=200, zero_start=True)
        iters.append(info.iterations)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    t_mix = ev0.elapsed_time(ev1) / 1e3
    launches = s_mix.launch_count() - l0
    value, t_mix_max = whole_job_mdofs(dist, dev, n, sum(iters), t_mix)
    rel_res_mix = info.rel_residual

    # solution error of the mixed solve against the FP64 solve (reported)
    x64 = torch.zeros_like(f)
    for _ in range(max(1, min(2, args.warmup))):
        s_64.solve(b, x64, rtol=RTOL, maxit=200, zero_start=True)
    torch.cuda.synchronize()
    k64 = max(1, (args.steps + 1) // 2)
    ev0.record(stream)
    it64 = []
    for _ in range(k64):
        i64 = s_64.solve(b, x64, rtol=RTOL, maxit=200, zero_start=True)
        it64.append(i64.iterations)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_64 = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
    err_mix = float(((x - x64).norm() / x64.norm()).item())

    # ---- V-cycle-only throughput (mixed and FP64)
    bf = b.float()
    xf = torch.zeros_like(bf)
    xd = torch.zeros_like(b)
    for _ in range(2):
        s_mix.vcycle(bf, xf)
        s_64.vcycle(b, xd)
    torch.cuda.synchronize()
    nv = 10
    ev0.record(stream)
    for _ in range(nv):
        s_mix.vcycle(bf, xf)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_vc32 = ev0.elapsed_time(ev1) / 1e3 / nv
    ev0.record(stream)
    for _ in range(3):
        s_64.vcycle(b, xd)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_vc64 = ev0.elapsed_time(ev1) / 1e3 / 3

    # ---- dominant kernels.  (1) The finest-level FP32 interior colour pass:
    # colour 0 (all vertex indices even) has no patch on the domain boundary,
    # so sipg_smooth_colour launches exactly one kernel
    # (smooth_int3_kernel<4, float, interior>) on the calling stream; CUDA
    # events around repeated launches give its average duration.  (2) The
    # FP64 operator apply of the outer CG (apply_kernel<3, 4, double>), one
    # launch per sipg_apply on the finest level in FP64.
    L = NLEV - 1
    N = 1 << LOG2N
    hbm, hbm_src = measured_peaks()
    peak32, peak64 = fp32_peak_tflops(), fp64_peak_tflops()

    def launch_time(fn, nrep=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(nrep):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / nrep

    def roofline(kernel, flops, nbytes, t, peak_tf, alu_name, traffic, extra):
        t_alu = flops / (peak_tf * 1e12)
        t_hbm = nbytes / (hbm * 1e9)
        ach_tf, ach_gb = flops / t / 1e12, nbytes / t / 1e9
        if t_alu >= t_hbm:
            r = {"bound": "alu", "achieved": round(ach_tf, 3), "peak": round(peak_tf, 3), "unit": "TFLOP/s",
                 "frac": round(ach_tf / peak_tf, 4),
                 "peak_source": f"{alu_name}: 152 SMs x unit count x 2 x 2070 MHz (derived)"}
        else:
            r = {"bound": "hbm", "achieved": round(ach_gb, 1), "peak": hbm, "unit": "GB/s",
                 "frac": round(ach_gb / hbm, 4), "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({hbm_src})"}
        r.update({"kernel": kernel, "traffic": traffic,
                  "traffic_source": TRAFFIC_SOURCE if traffic is not None else
                  "null: the kernel's sources changed since the last ncu capture",
                  "avg_launch_us": round(t * 1e6, 2), "algorithmic_flops_per_launch": int(flops),
                  "algorithmic_bytes_per_launch": int(nbytes),
                  "hbm_frac": round(ach_gb / hbm, 4), "alu_frac": round(ach_tf / peak_tf, 4)})
        if traffic is not None:
            r["traffic_over_algorithmic"] = round(traffic / nbytes, 3)
        r.update(extra)
        return r

    t_col = launch_time(lambda: s_mix.smooth_colour(L, 0, bf, xf))
    fl_survey, fl_sched, by_col, npatch0 = smoother_counts(DIM, K, N, 0, 4)
    _, tile = s_mix.tuning(L)
    roof = roofline("smooth_int3_kernel<4,float,interior,tile %d> (finest level, colour 0, %d patches; the "
                    "autotuner's tile)" % (tile, npatch0),
                    fl_sched, by_col, t_col, peak32, "FP32", measured_traffic("colour_pass", tile),
                    {"survey_flops_per_launch": int(fl_survey),
                     "survey_alu_frac": round(fl_survey / t_col / 1e12 / peak32, 4),
                     "counts": "flops = kernel schedule (sum-factorised, rank-one mass, structural zeros "
                               "skipped); bytes = (P^3 + 2p^3) x 4 B per patch"})
    y64 = torch.zeros_like(b)
    t_app = launch_time(lambda: s_64.apply(L, b, y64))
    fl_app, by_app = apply_counts(DIM, K, N, 8)
    roof_apply = roofline("apply_kernel<3,4,double> (outer CG operator apply, finest level)", fl_app, by_app,
                          t_app, peak64, "FP64", measured_traffic("fp64_apply"),
                          {"launches_per_solve": "iterations + 1 (q = A p per iteration, final true residual)",
                           "counts": "flops per DoF = 6n + 51 + 1/n (3D interior; neighbour terms only where a "
                                     "neighbour exists); bytes = 2 x 8 B per DoF"})

    # ---- per-operation throughput on this workload (finest level), with the
    # fraction of each operation's roofline: apply and smoothing step against
    # max(flop time, byte time) at the peaks above; the V-cycle and the solve
    # as MDoF/s
    yf = torch.zeros_like(bf)
    t_a32 = launch_time(lambda: s_mix.apply(L, bf, yf), 10)
    t_step = launch_time(lambda: s_mix.smooth(L, bf, xf), 5)
    fl_a32, by_a32 = apply_counts(DIM, K, N, 4)
    st_fl, st_by = 0, 0
    for c in range(2 ** DIM):
        _, f_c, b_c, _ = smoother_counts(DIM, K, N, c, 4)
        st_fl, st_by = st_fl + f_c, st_by + b_c

    def op(t, flops=None, nbytes=None, peak_tf=None):
        o = {"mdofs": round(n / t / 1e6, 1), "us": round(t * 1e6, 2)}
        if flops is not None:
            floor = max(flops / (peak_tf * 1e12), nbytes / (hbm * 1e9))
            o["roofline_frac"] = round(floor / t, 4)
            o["bound"] = "alu" if flops / (peak_tf * 1e12) >= nbytes / (hbm * 1e9) else "hbm"
        return o

    per_op = {"apply_fp32": op(t_a32, fl_a32, by_a32, peak32),
              "apply_fp64": op(t_app, fl_app, by_app, peak64),
              "smoothing_step_fp32": op(t_step, st_fl, st_by, peak32),
              "vcycle_fp32": op(t_vc32), "vcycle_fp64": op(t_vc64),
              "solve_mixed_per_vcycle": op(t_mix_max / sum(iters)),
              "note": "finest level of this workload; roofline_frac = max(flops / FP peak, bytes / HBM peak) / "
                      "time with the counts of the roofline objects (smoothing step: interior-patch model for "
                      "every patch of the 2^d colours)"}

    # ---- C3: the degree-7 configuration with the FP32 and the TF32 V-cycle
    c3 = c3_record(torch, dev) if not args.no_c3 else None
    c4a, c4b = c4_records(torch) if not args.no_c3 else (None, None)

    # ---- end to end through the public host-buffer call
    fh = f.detach().cpu().pin_memory()
    uh = torch.zeros_like(fh).pin_memory()
    s_mix.solve_host(fh, uh, rtol=RTOL)
    torch.cuda.synchronize()
    ke = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    it_e = 0
    for _ in range(ke):
        ie = s_mix.solve_host(fh, uh, rtol=RTOL)
        it_e += ie.iterations
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    e2e_value = n * sum_over_ranks(float(it_e)) / t_e2e / 1e6

    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 2), "unit": "MDoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_mix_max / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dim": DIM, "degree": K, "cells_per_dir": N,
                       "levels": NLEV, "dofs_per_gpu": n, "rtol": RTOL,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (each FP64 vector 134 MB > 129 MB L2)"},
            "extra": {
                "time_to_rtol_s": {"mixed": round(t_mix_max / args.steps, 4), "fp64": round(t_64 / k64, 4)},
                "speedup_mixed_vs_fp64": round((t_64 / k64) / (t_mix_max / args.steps), 3),
                "iterations": {"mixed": iters, "fp64": it64},
                "rel_residual": {"mixed": rel_res_mix, "fp64": i64.rel_residual},
                "nu": {"mixed": info.nu, "fp64": i64.nu},
                "mixed_vs_fp64_solution_rel_l2": err_mix,
                "vcycle_only_mdofs": {"fp32": round(n / t_vc32 / 1e6, 1), "fp64": round(n / t_vc64 / 1e6, 1)},
                "vcycle_ms": {"fp32": round(t_vc32 * 1e3, 3), "fp64": round(t_vc64 * 1e3, 3)},
                "fp64_mdofs_per_vcycle_in_solve": round(n * sum(it64) / t_64 / 1e6, 2),
            },
            "roofline": roof,
            "roofline_fp64_apply": roof_apply,
            "per_op": per_op,
            "c3_q7": c3,
            "c4a_multirhs": c4a,
            "c4b_ragged": c4b,
            "e2e": {"value": round(e2e_value, 2), "unit": "MDoF/s", "h2d_bytes_per_step": n * 8,
                    "d2h_bytes_per_step": n * 8,
                    "note": "sipg_solve_host: pinned f in, b = M f, solve from 0, u out"},
            "clocks": clk,
            "gpu_launches": int(launches),
        }
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------- kernel-only runs
def run_kernel_only(args):
    """Small-footprint run of one kernel family on the benchmark workload (for
    profiler captures): --mode smooth (FP32/FP64 finest-level colour passes),
    apply (FP64/FP32 finest-level operator apply) or vcycle."""
    import torch
    import paper_2405_18982_gb300 as pkg
    from paper_2405_18982_gb300 import SIPG, SIPG_FP32, SIPG_FP64, Params, inputs
    pkg.load(pkg.build())
    from paper_2405_18982_gb300 import SIPG_TF32
    prec = {"fp64": SIPG_FP64, "fp32": SIPG_FP32, "tf32": SIPG_TF32}[args.precision]
    dt = torch.float64 if prec == SIPG_FP64 else torch.float32
    dim, k, l2 = args.dim, args.degree, args.log2n
    nlev = args.levels or l2
    from paper_2405_18982_gb300 import (SIPG_SMOOTHER_CLAMPED, SIPG_SMOOTHER_CONSISTENT, SIPG_SMOOTHER_FULL,
                                        SIPG_SMOOTHER_PAPER)
    sm = {"consistent": SIPG_SMOOTHER_CONSISTENT, "paper": SIPG_SMOOTHER_PAPER, "full": SIPG_SMOOTHER_FULL,
          "clamped": SIPG_SMOOTHER_CLAMPED}[args.smoother]
    s = SIPG(Params(dim=dim, degree=k, log2_cells=l2, n_levels=nlev, vcycle_precision=prec, smoother=sm))
    n = s.ndofs()
    b = torch.from_numpy(inputs.uniform(NOISE_SEED, n)).to("cuda").view(1, n).to(dt)
    x = torch.zeros_like(b)
    L = nlev - 1

    if args.mode == "levels":
        # per-level cost of the V-cycle pieces (smoothing step, residual,
        # transfer) on this workload, CUDA events around each call
        out = {}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for lev in range(nlev - 1, 0, -1):
            nl = s.ndofs(lev)
            bl = torch.from_numpy(inputs.uniform(NOISE_SEED + lev, nl)).to("cuda").view(1, nl).to(dt)
            xl = torch.zeros_like(bl)
            rl = torch.zeros_like(bl)
            bc = torch.zeros(1, s.ndofs(lev - 1), dtype=dt, device="cuda")
            row = {}
            for name, fn in (("smooth_step", lambda: s.smooth(lev, bl, xl)),
                             ("residual", lambda: s.residual(lev, bl, xl, rl)),
                             ("restrict", lambda: s.restrict(lev, rl, bc)),
                             ("prolongate", lambda: s.prolongate_add(lev, bc, xl))):
                for _ in range(2):
                    fn()
                torch.cuda.synchronize()
                e0.record()
                for _ in range(args.steps):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                row[name] = round(e0.elapsed_time(e1) / args.steps * 1e3, 2)
            out[f"N={1 << (l2 - (nlev - 1 - lev))}"] = row
        print(json.dumps({"mode": "levels", "precision": args.precision, "us_per_call": out}))
        return

    def one():
        if args.mode == "smooth":
            for c in (range(2 ** dim) if args.colour < 0 else (args.colour,)):
                s.smooth_colour(L, c, b, x)
        elif args.mode == "apply":
            s.apply(L, b, x)
        else:
            s.vcycle(b, x)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"mode": args.mode, "precision": args.precision, "smoother": args.smoother, "dim": dim, "degree": k,
                      "cells_per_dir": 1 << l2, "levels": nlev, "dofs": n, "colour": args.colour,
                      "ms_per_rep": round(ms, 4)}))


# ----------------------------------------------------------------- batched runs
def c4_records(torch, reps=2):
    """C4a: 3D Q4 on 32^3 cells with 32 N(0,1) right-hand sides (seeds
    100..131) in one mixed solve to 1e-10, next to one right-hand side alone.
    C4b: the ragged batch of 64 independent 2D problems (2^L x 2^L cells, L
    uniform in 5..9, degree uniform in 2..6, seed 4; f ~ N(0,1), seeds
    1000 + i, b = M f), one batched mixed solve to 1e-10 (members on their own
    streams with CUDA-graph iteration bodies), next to the members one after
    another.  CUDA events around `reps` solves after one warm-up."""
    from paper_2405_18982_gb300 import SIPG, SIPG_FP32, Params, SIPGBatch, inputs
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    nrhs = 32
    s = SIPG(Params(dim=3, degree=4, log2_cells=5, n_levels=5, vcycle_precision=SIPG_FP32, nrhs=nrhs, use_graphs=1))
    one = SIPG(Params(dim=3, degree=4, log2_cells=5, n_levels=5, vcycle_precision=SIPG_FP32, use_graphs=1))
    nd = s.ndofs()
    b = torch.from_numpy(inputs.normal_columns(list(range(100, 100 + nrhs)), nd)).to("cuda")
    x = torch.zeros_like(b)
    b1 = b[:1].contiguous()
    x1 = torch.zeros_like(b1)
    ms_m, inf = timed(lambda: s.solve(b, x, rtol=1e-10, maxit=100, zero_start=True))
    ms_1, inf1 = timed(lambda: one.solve(b1, x1, rtol=1e-10, maxit=100, zero_start=True))
    c4a = {"workload": "3D Q4 32^3 (4.1M DoFs) x 32 RHS, mixed FCG to 1e-10", "ms_per_solve": round(ms_m, 3),
           "MDoF_per_s": round(nd * nrhs / ms_m / 1e3, 1), "iterations": inf.iterations,
           "rel_residual": inf.rel_residual, "single_rhs_ms_per_solve": round(ms_1, 3),
           "single_MDoF_per_s": round(nd / ms_1 / 1e3, 1)}
    s.close()
    one.close()
    del s, one, b, x
    torch.cuda.empty_cache()

    shapes = inputs.ragged_problems(4)
    mk = lambda: SIPGBatch([Params(dim=2, degree=k, log2_cells=L, n_levels=L, vcycle_precision=SIPG_FP32,
                                   use_graphs=1) for L, k in shapes])
    bt = mk()
    old = os.environ.get("SIPG_BATCH_FUSED")
    os.environ["SIPG_BATCH_FUSED"] = "1"
    bf = mk()      # the fused path: one cooperative launch per smoothing stage across members
    if old is None:
        del os.environ["SIPG_BATCH_FUSED"]
    else:
        os.environ["SIPG_BATCH_FUSED"] = old
    bs, xs = [], []
    for i, m in enumerate(bt.members):
        f = torch.from_numpy(inputs.normal(1000 + i, m.ndofs())).to("cuda").view(1, -1)
        bb = torch.zeros_like(f)
        m.rhs(f, bb)
        bs.append(bb)
        xs.append(torch.zeros_like(bb))
    total = sum(m.ndofs() for m in bt.members)

    def batched(b_=bt):
        for xx in xs:
            xx.zero_()
        return b_.solve(bs, xs, rtol=1e-10, maxit=100)

    def sequential():
        return [m.solve(bb, xx, rtol=1e-10, maxit=100, zero_start=True) for m, bb, xx in zip(bt.members, bs, xs)]

    ms_b, infos = timed(batched)
    ms_f, infos_f = timed(lambda: batched(bf))
    ms_s, _ = timed(sequential)
    bf.close()
    its = [i.iterations for i in infos]
    c4b = {"workload": "64 ragged 2D problems, L in 5..9, k in 2..6 (seed 4), mixed FCG to 1e-10",
           "total_dofs": total, "batched_ms_per_solve": round(ms_b, 3),
           "fused_stages_ms_per_solve": round(ms_f, 3),
           "fused_worst_rel_residual": max(i.rel_residual for i in infos_f),
           "sequential_ms_per_solve": round(ms_s, 3), "batched_MDoF_per_s": round(total / ms_b / 1e3, 1),
           "iterations_min_max": [min(its), max(its)], "worst_rel_residual": max(i.rel_residual for i in infos)}
    bt.close()
    del bt, bs, xs
    torch.cuda.empty_cache()
    return c4a, c4b


def run_batched(args):
    """--mode ragged / multirhs: the C4b / C4a records of c4_records (with
    --steps timed solves after one warm-up)."""
    import torch
    import paper_2405_18982_gb300 as pkg
    pkg.load(pkg.build())
    c4a, c4b = c4_records(torch, reps=max(1, args.steps))
    print(json.dumps({"mode": args.mode, **(c4b if args.mode == "ragged" else c4a)}))


# ----------------------------------------------------------------- throughput sweep
def run_sweep(args):
    """--mode sweep: MDoF/s of the finest-level apply, one smoothing step, one
    V-cycle (FP32) and one mixed solve to 1e-10, over 3D k = 2..7 with
    N = 16, 32, 64 and 2D k = 2..7 with N = 512, 1024, 2048 (coarsest level 2
    cells per direction; f ~ N(0,1), seed 3), with the roofline fraction of
    the apply and the smoothing step (max(flop time, byte time) at the peaks
    over the measured time, the counts of apply_counts and smoother_counts).
    One JSON line per configuration."""
    import torch
    import paper_2405_18982_gb300 as pkg
    from paper_2405_18982_gb300 import SIPG, SIPG_FP32, Params, inputs
    pkg.load(pkg.build())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hbm, _ = measured_peaks()
    peak32 = fp32_peak_tflops()

    def frac(t, flops, nbytes):
        floor = max(flops / (peak32 * 1e12), nbytes / (hbm * 1e9))
        return round(floor / t, 4), ("alu" if flops / (peak32 * 1e12) >= nbytes / (hbm * 1e9) else "hbm")

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    cases = [(3, k, l2) for l2 in (4, 5, 6) for k in range(2, 8)] + \
            [(2, k, l2) for l2 in (9, 10, 11) for k in range(2, 8)]
    for dim, k, l2 in cases:
        nd = (1 << l2) ** dim * (k + 1) ** dim
        if nd > 140_000_000:
            continue
        s = SIPG(Params(dim=dim, degree=k, log2_cells=l2, n_levels=l2, vcycle_precision=SIPG_FP32, use_graphs=1))
        n = s.ndofs()
        f = torch.from_numpy(inputs.normal(3, n)).to("cuda").view(1, n)
        b = torch.zeros_like(f)
        s.rhs(f, b)
        bf = b.float()
        xf = torch.zeros_like(bf)
        yf = torch.zeros_like(bf)
        x = torch.zeros_like(b)
        t_apply = timed(lambda: s.apply(l2 - 1, bf, yf), 10)
        t_smooth = timed(lambda: s.smooth(l2 - 1, bf, xf), 5)
        t_vc = timed(lambda: s.vcycle(bf, xf), 5)

        def solve():
            x.zero_()
            return s.solve(b, x, rtol=1e-10, maxit=200)

        info = solve()
        t_solve = timed(solve, 2)
        N = 1 << l2
        fa, ba = apply_counts(dim, k, N, 4)
        fs, bs = 0, 0
        for c in range(2 ** dim):
            _, f_c, b_c, _ = smoother_counts(dim, k, N, c, 4)
            fs, bs = fs + f_c, bs + b_c
        fr_a, bd_a = frac(t_apply, fa, ba)
        fr_s, bd_s = frac(t_smooth, fs, bs)
        print(json.dumps({"mode": "sweep", "dim": dim, "degree": k, "cells_per_dir": 1 << l2, "dofs": n,
                          "apply_fp32_mdofs": round(n / t_apply / 1e6, 1),
                          "apply_roofline_frac": fr_a, "apply_bound": bd_a,
                          "smooth_step_fp32_mdofs": round(n / t_smooth / 1e6, 1),
                          "smooth_step_roofline_frac": fr_s, "smooth_step_bound": bd_s,
                          "vcycle_fp32_mdofs": round(n / t_vc / 1e6, 1),
                          "solve_mixed_ms": round(t_solve * 1e3, 2), "iterations": info.iterations,
                          "solve_mdofs_per_vcycle": round(n * info.iterations / t_solve / 1e6, 1)}), flush=True)
        s.close()
        del s
        torch.cuda.empty_cache()


def run_table2(args):
    """--mode table2: the setting of the paper's Table 2 (Dirichlet kernel) on
    the device: 3D unit cube, f = 1, 2^L cells per direction down to 2^3 on
    the coarsest level, GMRES to 1e-8 preconditioned from the right by one
    V-cycle whose smoother uses the Dirichlet-kernel residual; nu (Sec. 3.3),
    steps and time to solution with the FP64 and the FP32 V-cycle (each
    restart cycle one graph launch on the device, and step by step from the
    host), the
    consistent residual, the full kernel (Table 1's setting) and the clamped
    kernel (Table 2 right; also with GMRES preconditioned from the left, the
    reading that reproduces that column) beside it, and the values printed
    in Tables 1 and 2.  Cases
    k = 3..7, L = 2..7 up to --max-dofs DoFs.  One JSON line per case."""
    import time

    import numpy as np
    import torch
    import paper_2405_18982_gb300 as pkg
    from paper_2405_18982_gb300 import (SIPG, SIPG_FP32, SIPG_FP64, SIPG_SMOOTHER_CLAMPED, SIPG_SMOOTHER_CONSISTENT,
                                        SIPG_SMOOTHER_FULL, SIPG_SMOOTHER_PAPER, Params)
    pkg.load(pkg.build())
    printed = np.loadtxt(os.path.join(ROOT, "tests", "golden", "table2_dirichlet_nu.txt"))
    printed1 = np.loadtxt(os.path.join(ROOT, "tests", "golden", "table1_full_nu.txt"))
    printed_c = np.loadtxt(os.path.join(ROOT, "tests", "golden", "table2_clamped_nu.txt"))
    for L in range(2, 8):
        for k in range(3, 8):
            n = (1 << L) ** 3 * (k + 1) ** 3
            if n > args.max_dofs:
                continue
            row = {"mode": "table2", "degree": k, "L": L, "dofs": n,
                   "nu_table2": None if np.isnan(printed[L - 2, k - 2]) else float(printed[L - 2, k - 2])}
            row["nu_table1"] = None if np.isnan(printed1[L - 2, k - 2]) else float(printed1[L - 2, k - 2])
            row["nu_table2_clamped"] = None if np.isnan(printed_c[L - 2, k - 2]) else float(printed_c[L - 2, k - 2])
            # graphs = 1: every GMRES restart cycle is one graph launch on the
            # device; the *_hoststeps rows drive each step from the host
            for tag, prec, sm, left, graphs in (
                    ("fp64", SIPG_FP64, SIPG_SMOOTHER_PAPER, False, 1),
                    ("mixed", SIPG_FP32, SIPG_SMOOTHER_PAPER, False, 1),
                    ("fp64_hoststeps", SIPG_FP64, SIPG_SMOOTHER_PAPER, False, 0),
                    ("mixed_hoststeps", SIPG_FP32, SIPG_SMOOTHER_PAPER, False, 0),
                    ("consistent_mixed", SIPG_FP32, SIPG_SMOOTHER_CONSISTENT, False, 1),
                    ("full_mixed", SIPG_FP32, SIPG_SMOOTHER_FULL, False, 1),
                    ("clamped_mixed", SIPG_FP32, SIPG_SMOOTHER_CLAMPED, False, 1),
                    # left preconditioning needs a fixed linear V-cycle: FP64
                    ("clamped_fp64_left", SIPG_FP64, SIPG_SMOOTHER_CLAMPED, True, 1)):
                s = SIPG(Params(dim=3, degree=k, log2_cells=L, n_levels=L, vcycle_precision=prec, smoother=sm,
                                use_graphs=graphs))
                f = torch.ones(1, s.ndofs(), dtype=torch.float64, device="cuda")
                b = torch.zeros_like(f)
                s.rhs(f, b)
                x = torch.zeros_like(b)
                work = torch.empty(s.gmres_workspace_bytes(30) + 256, dtype=torch.uint8, device="cuda")
                s.gmres_solve(b, x, rtol=1e-8, maxit=200, restart=30, work=work, left=left)   # warm-up
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = s.gmres_solve(b, x, rtol=1e-8, maxit=200, restart=30, work=work, left=left)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                row[f"nu_{tag}"] = round(info.nu, 2)
                row[f"steps_{tag}"] = info.iterations
                row[f"time_to_1e-8_{tag}_ms"] = round(dt * 1e3, 2)
                s.close()
                del s, work, f, b, x
                torch.cuda.empty_cache()
            print(json.dumps(row), flush=True)


# ----------------------------------------------------------------- oracle arm
SAMPLE = (3, 3, 8, 3)   # dim, k, N, levels: the same discretisation on 8^3 cells


def _oracle_sample():
    import numpy as np
    from oracle.assembly import rhs_from_nodal
    from oracle.mg import Hierarchy
    from paper_2405_18982_gb300 import inputs
    dim, k, N, nl = SAMPLE
    H = Hierarchy(dim, k, N, nl)
    nd = H.A.shape[0]
    from oracle.layout import node_coordinates
    from oracle.basis import gauss_lobatto
    X = node_coordinates(dim, N, gauss_lobatto(k)[0])
    f = dim * np.pi ** 2 * np.prod(np.sin(np.pi * X), axis=1) + inputs.uniform(NOISE_SEED, nd)
    b = rhs_from_nodal(dim, k, N, f)
    return H, b


def _oracle_iteration(H, r):
    """One FCG iteration's preconditioner + operator work in the oracle."""
    z = H.vcycle(r)
    q = H.A @ z
    return z, q


SINGLE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def _oracle_workers(seconds, count):
    """`count` fresh single-threaded interpreters, started together, each
    timing oracle FCG iterations on its own copy of the sample for about
    `seconds`; returns their JSON results (None on failure)."""
    env = dict(os.environ, **SINGLE_THREAD_ENV)
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._cpu_baseline_here(%r)))" % (ROOT, float(seconds)))
    procs = [subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT, stdout=subprocess.PIPE,
                              stderr=subprocess.DEVNULL, text=True) for _ in range(count)]
    out = []
    for p in procs:
        try:
            so, _ = p.communicate(timeout=seconds * 10 + 300)
            out.append(json.loads(so.strip().splitlines()[-1]) if p.returncode == 0 else None)
        except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
            p.kill()
            out.append(None)
    return out


def cpu_baseline(seconds=12.0):
    """The oracle timed on the host cores: one single-threaded interpreter
    alone (the single-core figure), then one per core at the same time (the
    all-cores figure: independent copies of the sample, the oracle's
    iteration being sequential NumPy/SciPy code).  BLAS and OpenMP pools are
    limited to one thread before NumPy loads in each."""
    one = _oracle_workers(seconds, 1)[0]
    cores = os.cpu_count() or 1
    many = _oracle_workers(seconds, cores)
    ok = [m for m in many if m is not None]
    if one is None or not ok:
        out = _cpu_baseline_here(seconds)  # threads not pinned in this process
        out["sample"] += " (in-process: BLAS threads not pinned)"
        out["cores"] = None
        return out
    total = sum(m["value"] for m in ok)
    return {"value": round(total, 5), "unit": "MDoF/s", "cores": len(ok), "kind": "oracle",
            "single_core_value": one["value"],
            "sample": f"oracle V-cycle + CSR apply (one FCG iteration) on the same discretisation at 8^3 cells, "
                      f"one single-threaded copy per host core ({len(ok)} of {cores} ran), ~{seconds:.0f} s each; "
                      f"single core alone: {one['sample']}"}


def _cpu_baseline_here(seconds):
    H, b = _oracle_sample()
    nd = H.A.shape[0]
    r = b.copy()
    _oracle_iteration(H, r)
    t0 = time.perf_counter()
    cnt = 0
    while time.perf_counter() - t0 < seconds:
        z, _ = _oracle_iteration(H, r)
        cnt += 1
    dt = time.perf_counter() - t0
    return {"value": round(nd * cnt / dt / 1e6, 5), "unit": "MDoF/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle V-cycle + CSR apply (one FCG iteration) on the same discretisation at 8^3 cells "
                      f"({nd} DoFs, 3 levels), {cnt} iterations in {dt:.1f} s, single thread"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    os.environ.update(SINGLE_THREAD_ENV)  # one core: set before NumPy loads
    H, b = _oracle_sample()
    nd = H.A.shape[0]
    r = b.copy()
    for _ in range(args.warmup):
        _oracle_iteration(H, r)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_iteration(H, r)
    dt = time.perf_counter() - t0
    value = nd * args.steps / dt / 1e6
    out = {"metric": METRIC, "value": round(value, 5), "unit": "MDoF/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "sample": "8^3 cells, 3 levels (same k, d, penalty, source)"},
           "cpu_baseline": {"value": round(value, 5), "unit": "MDoF/s", "cores": 1, "kind": "oracle",
                            "sample": f"one oracle FCG iteration (V-cycle + CSR apply) per step on 8^3 cells ({nd} DoFs)"},
           "e2e": {"value": round(value, 5), "unit": "MDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c3", action="store_true", help="skip the C3 (degree 7) and C4 (batched) records")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "smooth", "apply", "vcycle", "levels", "ragged", "multirhs", "sweep", "table2",
                             "c3"])
    ap.add_argument("--max-dofs", type=float, default=2e7, help="largest case of --mode table2")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "tf32"])
    # workload of the kernel-only modes (default: the benchmark's 3D Q3 64^3, 6 levels)
    ap.add_argument("--dim", type=int, default=DIM)
    ap.add_argument("--degree", type=int, default=K)
    ap.add_argument("--log2n", type=int, default=LOG2N)
    ap.add_argument("--levels", type=int, default=NLEV)
    ap.add_argument("--colour", type=int, default=-1, help="--mode smooth: one colour (default all)")
    ap.add_argument("--smoother", default="consistent", choices=["consistent", "paper", "full", "clamped"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode in ("ragged", "multirhs"):
        run_batched(args)
    elif args.mode == "sweep":
        run_sweep(args)
    elif args.mode == "table2":
        run_table2(args)
    elif args.mode == "c3":
        import torch
        import paper_2405_18982_gb300 as pkg
        pkg.load(pkg.build())
        print(json.dumps({"mode": "c3", **c3_record(torch, torch.device("cuda", 0))}))
    elif args.mode != "solve":
        run_kernel_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
