#!/usr/bin/env python
"""Benchmark: time-to-solution of the Stokes solve phase on GB300.

Default workload (one "step" = one full solve to relative residual 1e-8):
3D finite-difference Stokes, N=64 (262,144 nodes, 1,048,576 unknowns),
lognormal viscosity sigma=0.5, K stored as 4x4 BSR FP64, monolithic
block smoothed-aggregation AMG (damped Jacobi 1+1) + BiCGStab, FP64.
Inputs are resident in HBM when the timed region starts; each solve
iteration streams K and two V-cycles' hierarchy (about 1.2 GB), far more
than L2 (129 MB).  Kernels timed alone (the roofline objects) follow a
256 MB buffer write each launch.

The line also carries the metric's "FP64 vs mixed" comparison ("mixed"):
C2 and the largest config C3 (N=128, Schur + GMRES(30)) solved with FP64,
FP32 and BF16 hierarchies, with C3's errors against the oracle's stored
full-size solve, and the measured FP64 FMA rate ("fp64_peak") that the
FP64 kernels' roofline uses.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2|c1|c3-fp64|c3-fp32|c3-bf16]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the same workload

Multi-GPU: the solve does not shard in this build (replicas only): under
torchrun every rank solves its own copy; value = max-over-ranks time per
step divided by the number of ranks (aggregate time per solve).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "time-to-solution at rel. residual 1e-8 (solve phase)"
L2_FLUSH_BYTES = 256 << 20   # twice GB300's 129 MB L2
UNIT = "ms"

WORKLOADS = {
    "c2": dict(system="c2", precision=0, desc=(
        "3D FD Stokes N=64 (1,048,576 unknowns), lognormal mu sigma=0.5, 4x4 BSR FP64, "
        "monolithic block SA-AMG (damped Jacobi 1+1) + BiCGStab, tol 1e-8")),
    "c2-fp32": dict(system="c2", precision=1, desc=(
        "same as c2 with an FP32 hierarchy (FP64 outer BiCGStab, dots and residual "
        "replacement)")),
    "c2-bf16": dict(system="c2", precision=2, desc=(
        "same as c2 with a BF16 hierarchy (FP32 accumulation; FP64 outer BiCGStab, dots and "
        "residual replacement)")),
    "c1": dict(system="c1", precision=0, desc=(
        "3D FD Stokes N=16 (16,384 unknowns), mu=1, scalar CSR FP64, SA-AMG (SPAI0 1+1) + "
        "BiCGStab, tol 1e-8")),
    "c3-fp64": dict(system="c3", precision=0, desc=(
        "3D FD Stokes N=128 (8,388,608 unknowns), lognormal mu sigma=1, Schur pressure "
        "correction (3x3 velocity SA-AMG + scalar SA-AMG on S_hat, SPAI0) + GMRES(30) FP64, "
        "hierarchy FP64")),
    "c3-fp32": dict(system="c3", precision=1, desc="same as c3-fp64 with an FP32 hierarchy"),
    "c3-bf16": dict(system="c3", precision=2, desc=(
        "same as c3-fp64 with a BF16 hierarchy (FP32 accumulation)")),
}


def solver_params(gb, wl, **kw):
    name = WORKLOADS[wl]["system"]
    prec = WORKLOADS[wl]["precision"]
    if name == "c3":
        kw.setdefault("krylov", gb.GBS_GMRES)
        return gb.params_default(precond=gb.GBS_PC_SCHUR, precision=prec, enable_adjoint=0, **kw)
    relax = kw.pop("relax", gb.GBS_SPAI0 if name == "c1" else gb.GBS_JACOBI)
    return gb.params_default(relax=relax, precision=prec, enable_adjoint=0, **kw)


def kernel_source_sha1():
    """Hash of the sources of the outer SpMV kernels (kernels.cuh, sell.cuh,
    outer.cuh)."""
    import hashlib
    h = hashlib.sha1()
    for f in ("kernels.cuh", "sell.cuh", "outer.cuh"):
        with open(os.path.join(ROOT, "paper_2006_06052_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    profiles/<kernel>_<workload>.txt, or None when the kernel sources have
    changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "%s_%s.txt" % (kernel, workload))
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_sha1") != kernel_source_sha1():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def level1_relax_roofline(gb, H, B, precision, timed, peak, peak_kind, fp64):
    """Roofline of one level-1 relaxation sweep y = x + M (f - A_1 x) (block
    form when the level's blocks are more than half nonzero): FP64 is bound
    by the FP64 pipe (B*B FMAs a stored block; peak: the measured DFMA rate
    of gbs_fp64_peak), the FP32/BF16 forms by HBM."""
    import torch
    info = gb.hierarchy_info(H)
    if info["nlevels"] < 3:
        return None
    nbr, nnzb = info["n_brows"][1], info["nnzb"][1]
    vals = gb.export_level(H, 0, 1, 0)[2]
    nnz = int(np.count_nonzero(vals))
    block = nnz > 0.5 * vals.size
    n = nbr * B
    sv, sx = {0: (8, 8), 1: (4, 4), 2: (2, 4)}[precision]
    dt = torch.float64 if precision == 0 else torch.float32
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(n, dtype=dt, device="cuda", generator=g)
    f = torch.randn(n, dtype=dt, device="cuda", generator=g)
    y = torch.empty_like(x)
    ms = timed(lambda: gb.level_apply(H, 0, 1, 1, x, f, y))
    a_bytes = nnzb * (B * B * sv + 4) + 4 * (nbr + 1) if block else nnz * (sv + 4) + 4 * (n + 1)
    nbytes = a_bytes + nbr * B * B * sv + 3 * n * sx
    flops = 2.0 * (nnzb * B * B if block else nnz) + 2.0 * n * B + n
    gbs = nbytes / (ms * 1e-3) / 1e9
    tflops = flops / (ms * 1e-3) / 1e12
    layout, _ = gb.level_format(H, 0, 1)
    kname = {"block slices": "k_bsell_relax (%dx%d blocks in block-row slices)" % (B, B),
             "block": "k_relax (%dx%d blocks)" % (B, B),
             "csr": "k_csr_relax (scalar CSR)",
             "sliced": "k_sell_relax (scalar slices)"}[layout]
    desc = ("%s: level-1 relaxation sweep y = x + M (f - A_1 x), %d block rows, %d stored blocks"
            % (kname, nbr, nnzb))
    traffic = profiled_traffic("k_relax_level1", "c2") if precision == 0 else None
    hbm = {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
           "algorithmic_bytes": nbytes, "peak_kind": peak_kind}
    if precision == 0:
        return {"bound": "alu", "achieved": tflops, "peak": fp64["tflops"], "unit": "TFLOP/s",
                "frac": tflops / fp64["tflops"], "traffic": traffic, "kernel": desc,
                "ms": ms, "algorithmic_flops": flops, "peak_kind": fp64["kind"], "hbm": hbm}
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "traffic": traffic, "kernel": desc, "ms": ms, "algorithmic_bytes": nbytes,
            "peak_kind": peak_kind}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
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
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_spmv_bytes(nbr, nnzb, B, sv=8, sx=8):
    """x read once, y written once, int32 indices, values of every stored block."""
    return nnzb * (B * B * sv + 4) + 4 * (nbr + 1) + nbr * B * (sx + sx)


def exported(gb, H, which):
    """Every level of hierarchy `which` of a handle (the FP64 setup values),
    in import_hierarchy's layout."""
    nl = gb.hierarchy_info(H, which)["nlevels"]
    As, Ps, Rs, Ms = [], [], [], []
    for l in range(nl):
        As.append(gb.export_level(H, which, l, 0))
        if l + 1 < nl:
            Ps.append(gb.export_level(H, which, l, 1))
            Rs.append(gb.export_level(H, which, l, 2))
            Ms.append(gb.export_level(H, which, l, 3))
    return As, Ps, Rs, Ms, gb.export_level(H, which, nl - 1, 5)


def load_c3_oracle():
    """The oracle's full-size C3 solve (written by tests/golden/make_c3_oracle.py)."""
    path = os.path.join(ROOT, "tests", "golden", "c3_oracle_solution.txt")
    if not os.path.exists(path):
        return None
    g = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or ":" not in line:
                continue
            k, v = line.split(":", 1)
            g[k.strip()] = [float(t) for t in v.split()]
    return g


def time_solves(gb, H, b, steps, warmup):
    """Mean device time of `steps` solves from x = 0 (CUDA events around the
    whole loop, after `warmup` untimed solves); the last x and Info."""
    import torch
    stream = torch.cuda.current_stream()
    x = torch.zeros_like(b)
    for _ in range(warmup):
        x.zero_()
        gb.solve(H, b, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        x.zero_()
        _, info = gb.solve(H, b, x)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, x, info


def mixed_forms(gb, si, args, s_main, H_main, spec_main):
    """FP64 vs the mixed forms (FP32 and BF16 hierarchies; outer Krylov,
    dots, norms and residual replacement FP64) on C2 and on the largest
    config, C3 (N=128, Schur + GMRES(30)).  Each system's host setup runs
    once, for the FP64 handle; the mixed forms import its exported
    hierarchy (gbs_import_hierarchy / gbs_import_schur), so all three forms
    run the same setup values.  Errors: against the oracle's stored C3 solve
    (sampled estimate) and against this run's FP64 solution."""
    import torch
    out = {}
    kw = {} if args.gmres_reorth is None else {"gmres_reorth": args.gmres_reorth}
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    for name in ("c2", "c3"):
        wl = "c2" if name == "c2" else "c3-fp64"
        if name == "c2" and spec_main["system"] == "c2" and spec_main["precision"] == 0:
            s, H64, setup_s = s_main, H_main, None
        else:
            s = si.make_system(name)
            t0 = time.perf_counter()
            H64 = gb.build_hierarchy(s.indptr, s.indices, s.data, s.bdim,
                                     solver_params(gb, wl, use_graph=1, **kw))
            torch.cuda.synchronize()
            setup_s = time.perf_counter() - t0
        b = torch.as_tensor(s.b, device="cuda")
        forms = {}
        x64 = None
        for prec, tag in ((0, "fp64"), (1, "fp32"), (2, "bf16")):
            if prec == 0:
                H = H64
            else:
                p = solver_params(gb, wl, use_graph=1, **kw)
                p.precision = prec
                if name == "c3":
                    H = gb.import_schur(s.indptr, s.indices, s.data, exported(gb, H64, 0),
                                        exported(gb, H64, 1), None, p)
                else:
                    As, Ps, Rs, Ms, Ai = exported(gb, H64, 0)
                    H = gb.import_hierarchy(As, Ps, Rs, Ms, Ai, s.bdim, p)
            ms, x, info = time_solves(gb, H, b, args.steps, args.warmup)
            xh = x.cpu().numpy()
            if prec == 0:
                x64 = xh
            f = {"ms": ms, "iterations": info.iters, "rel_res": info.rel_res,
                 "converged": bool(info.converged),
                 "err_vs_fp64": float(np.linalg.norm(xh - x64) / np.linalg.norm(x64)),
                 "precond_bytes": gb.precond_bytes(H)}
            if name == "c3":
                g = load_c3_oracle()
                if g is not None and int(g["n"][0]) == s.n:
                    idx = np.array(g["sample_idx"], dtype=np.int64)
                    f["err_vs_oracle"] = float(
                        np.sqrt(s.n / len(idx) * np.sum((xh[idx] - np.array(g["sample_x"])) ** 2))
                        / g["x_norm"][0])
            forms[tag] = f
            if prec != 0:
                H.destroy()
        entry = {"workload": WORKLOADS[wl]["desc"],
                 "setup_s": setup_s, "forms": forms,
                 "speedup": {t: forms["fp64"]["ms"] / forms[t]["ms"] for t in ("fp32", "bf16")}}
        if name == "c3":
            g = load_c3_oracle()
            if g is not None:
                entry["oracle"] = {"iterations": int(g["iterations"][0]),
                                   "true_rel_res": g["true_rel_res"][0],
                                   "err_estimate": "sqrt(n/m sum_sample (x - x_oracle)^2) / "
                                                   "||x_oracle|| over the %d stored entries of "
                                                   "tests/golden/c3_oracle_solution.txt"
                                                   % len(g["sample_idx"])}
        out[name] = entry
        if H64 is not H_main:
            H64.destroy()
    out["clocks"] = sampler.stop()
    return out


def time_cpu_oracle(system, wl, iters_to_scale, sample_iters=3, calibrate=False):
    """The FP64 oracle on the host: setup (untimed), `sample_iters` Krylov
    iterations timed, scaled to a full solve by `iters_to_scale` (or by the
    oracle's own iteration count when calibrate=True)."""
    from oracle import amg, bsr, krylov, schur
    s = system
    K = bsr.from_arrays(s.indptr, s.indices, s.data, s.bdim)
    Ks = K.scipy().tocsr()
    if s.method == "amg_bicgstab":
        relax = "spai0" if s.name == "c1" else "jacobi"
        Ho = amg.build_hierarchy(K, amg.AmgParams(relax=relax))

        def run(maxiter):
            return krylov.bicgstab(lambda v: Ks @ v, lambda v: amg.vcycle(Ho, v), s.b, tol=1e-8,
                                   maxiter=maxiter)
    else:
        pc = schur.build(K, 3)

        def run(maxiter):
            return krylov.gmres(lambda v: Ks @ v, pc.apply, s.b, m=30, tol=1e-8, maxiter=maxiter)
    full_iters = None
    full_s = None
    if calibrate:
        t0 = time.perf_counter()
        _, info = run(10000)
        full_s = time.perf_counter() - t0
        full_iters = info.iters
        iters_to_scale = full_iters
    return run, iters_to_scale, full_iters, sample_iters, full_s


def cpu_oracle_sample(run, sample_iters):
    t0 = time.perf_counter()
    run(sample_iters)
    return (time.perf_counter() - t0) / sample_iters


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    """--impl reference: the FP64 CPU oracle on the same workload."""
    if rank != 0:
        return 0
    import stokes_inputs as si
    wl = args.workload
    s = si.make_system(WORKLOADS[wl]["system"])
    run, iters, full_iters, k, full_s = time_cpu_oracle(s, wl, None, sample_iters=args.sample_iters,
                                                        calibrate=True)
    for _ in range(args.warmup):
        cpu_oracle_sample(run, 1)
    per = []
    for _ in range(args.steps):
        per.append(cpu_oracle_sample(run, k))
    per_it = float(np.mean(per))
    value = per_it * full_iters * 1e3
    sample = ("oracle setup untimed; per step %d Krylov iterations of the full-size workload "
              "timed, scaled by the oracle's own iteration count (%d) to one solve; one "
              "complete oracle solve, timed once as a check of that scaling, took %.1f s"
              % (k, full_iters, full_s))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": value,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOADS[wl]["desc"]},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "iterations": full_iters, "full_solve_ms": full_s * 1e3}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbstokes", choices=["gbstokes", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--sample-iters", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the FP64-vs-mixed comparison (C2 and C3 forms)")
    ap.add_argument("--schur-order", type=int, default=0,
                    help="c3 workloads: 0 full Eq. SchurPC, 1 lower factorisation")
    ap.add_argument("--schur-p", type=int, default=0,
                    help="c3 workloads: 0 pressure AMG V-cycle, 1 one SPAI0 application on S_hat")
    ap.add_argument("--krylov", default=None, choices=["bicgstab", "gmres", "idrs"],
                    help="outer solver (default: the workload's: BiCGStab for c1/c2, GMRES(30) for c3)")
    ap.add_argument("--gmres-reorth", type=int, default=None, choices=[0, 1, 2],
                    help="GMRES second Gram-Schmidt pass: 0 never, 1 DGKS test, 2 always")
    ap.add_argument("--level-format", type=int, default=0,
                    help="0 scalar CSR for mostly-zero block levels, 1 block form everywhere")
    ap.add_argument("--plain-aggregation", action="store_true",
                    help="unsmoothed aggregation (P = P_tent), the paper's velocity AMG")
    ap.add_argument("--relax", default=None, choices=["spai0", "jacobi", "ilut"],
                    help="smoother of the monolithic / velocity AMG (default: the workload's; "
                         "ilut = the velocity smoother of the paper's Listings V2-V4)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import paper_2006_06052_gb300 as gb
    import stokes_inputs as si

    torch.cuda.set_device(local)
    if rank == 0:
        gb.build()
    barrier(world)
    gb.load_library()
    wl = args.workload
    spec = WORKLOADS[wl]
    s = si.make_system(spec["system"])
    extra = {"level_format": args.level_format}
    if args.krylov:
        extra["krylov"] = {"bicgstab": gb.GBS_BICGSTAB, "gmres": gb.GBS_GMRES,
                           "idrs": gb.GBS_IDRS}[args.krylov]
    if spec["system"] == "c3":
        extra.update(schur_order=args.schur_order, schur_p=args.schur_p)
    if args.gmres_reorth is not None:
        extra["gmres_reorth"] = args.gmres_reorth
    if args.relax:
        extra["relax"] = {"spai0": gb.GBS_SPAI0, "jacobi": gb.GBS_JACOBI,
                          "ilut": gb.GBS_ILUT}[args.relax]
    if args.plain_aggregation:
        extra["smooth_P"] = 0
    prm = solver_params(gb, wl, use_graph=0 if args.no_graph else 1, **extra)
    t0 = time.perf_counter()
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, s.bdim, prm)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    b = torch.as_tensor(s.b, device="cuda")
    x = torch.zeros_like(b)

    for _ in range(args.warmup):
        x.zero_()
        _, info = gb.solve(H, b, x)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    l0 = gb.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        x.zero_()
        _, info = gb.solve(H, b, x)
        iters.append(info.iters)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = gb.kernel_launches() - l0
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, world)
    rel_res = info.rel_res
    converged = bool(info.converged)

    # end-to-end: pinned host b -> device, solve, device x -> pinned host, every step
    bh = torch.as_tensor(s.b).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    for _ in range(2):
        b.copy_(bh, non_blocking=True)
        x.zero_()
        gb.solve(H, b, x)
        xh.copy_(x, non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for _ in range(args.steps):
        b.copy_(bh, non_blocking=True)
        x.zero_()
        gb.solve(H, b, x)
        xh.copy_(x, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)

    # Kernels timed alone: each launch is preceded by a write of a buffer
    # twice the size of L2, with CUDA events around the launch only, so no
    # launch finds the previous one's data in L2.
    peak, peak_kind = load_peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device="cuda")

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        for a, z in evs:
            flush.zero_()
            a.record(stream)
            fn()
            z.record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(z) for a, z in evs]))

    ft, nsm = gb.fp64_peak()
    fp64 = {"tflops": ft, "kind": "measured: gbs_fp64_peak (independent DFMA chains on all %d SMs, "
                                  "CUDA events)" % nsm}
    B = s.bdim
    nbr = len(s.indptr) - 1
    nnzb = len(s.indices)
    nnz_true = int(np.count_nonzero(s.data))
    y = torch.empty_like(b)

    spmv_ms = timed(lambda: gb.spmv(H, x, y))
    csr_bytes = nnz_true * 12 + 4 * (nbr * B + 1) + nbr * B * 16
    csr_gbs = csr_bytes / (spmv_ms * 1e-3) / 1e9
    # the BSR kernel on K's block arrays (the allocation-free entry point
    # launches the same one-lane-per-row block kernel), dots allocated once
    rp = torch.as_tensor(s.indptr, device="cuda")
    ci = torch.as_tensor(s.indices, device="cuda")
    va = torch.as_tensor(s.data.reshape(-1), device="cuda")
    wv = torch.ones_like(b)
    dots = torch.zeros(2, dtype=torch.float64, device="cuda")
    bsr_ms = timed(lambda: gb.spmv_dots_noalloc(rp, ci, va, B, x, y, w=wv, dots=dots))
    spmv_bytes = algorithmic_spmv_bytes(nbr, nnzb, B)
    achieved = spmv_bytes / (bsr_ms * 1e-3) / 1e9
    # FP64 block SpMV does B*B FMAs per stored block; on GB300 the FP64 pipe
    # (not HBM) is the tighter roofline for the block kernel
    flops = 2.0 * nnzb * B * B
    tflops = flops / (bsr_ms * 1e-3) / 1e12
    bsr_spmv = {"kernel": "k_outer_n (BSR %dx%d FP64 SpMV of K, with two fused dots)" % (B, B),
                "ms": bsr_ms, "bound": "alu", "achieved_tflops": tflops,
                "peak_tflops": fp64["tflops"], "frac": tflops / fp64["tflops"],
                "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "algorithmic_bytes": spmv_bytes, "peak_kind": peak_kind},
                "traffic": profiled_traffic("k_outer_n", spec["system"])}
    # the outer SpMV of K as the solve runs it
    kform, kstored = gb.outer_format(H)
    kname = {"block": "k_outer_n", "csr": "k_outer_csr", "sliced": "k_outer_sell"}[kform]
    kdesc = {"block": "as %dx%d blocks" % (B, B),
             "csr": "as scalar CSR of its %d nonzeros" % nnz_true,
             "sliced": "as its %d nonzeros in uniform 32-node component slices (%d stored "
                       "entries, no column indices)" % (nnz_true, kstored)}[kform]
    k_run_bytes = {"block": nnzb * (B * B * 8 + 4) + 4 * (nbr + 1),
                   "csr": nnz_true * 12 + 4 * (nbr * B + 1),
                   "sliced": kstored * 8}[kform]
    traffic = profiled_traffic(kname, spec["system"])
    outer_spmv = {"bound": "hbm", "achieved": csr_gbs, "peak": peak, "unit": "GB/s",
                  "frac": csr_gbs / peak, "traffic": traffic,
                  # DRAM bytes actually moved (ncu) over the same time: below the
                  # algorithmic figure when the format needs no column indices
                  "traffic_gbs": traffic / (spmv_ms * 1e-3) / 1e9 if traffic else None,
                  "kernel": "%s (FP64 SpMV of K %s)" % (kname, kdesc),
                  "algorithmic_bytes": csr_bytes, "ms": spmv_ms, "peak_kind": peak_kind,
                  "fp64": {"achieved_tflops": 2.0 * nnz_true / (spmv_ms * 1e-3) / 1e12,
                           "peak_tflops": fp64["tflops"]}}
    roofline = outer_spmv
    # the dominant kernel of the C2 solve by ncu launch-list share: the
    # level-1 relaxation sweep, timed through gbs_level_apply exactly as the
    # V-cycle launches it
    if spec["system"] == "c2":
        roofline = level1_relax_roofline(gb, H, B, spec["precision"], timed, peak, peak_kind,
                                         fp64) or outer_spmv
    # the V-cycle as a whole (monolithic AMG only)
    vcycle = None
    if spec["system"] != "c3":
        vms = timed(lambda: gb.apply_precond(H, b, y))
        vb = gb.precond_bytes(H)
        vcycle = {"ms": vms, "algorithmic_bytes": vb, "achieved_gbs": vb / (vms * 1e-3) / 1e9,
                  "frac": vb / (vms * 1e-3) / 1e9 / peak}

    mixed = None
    if not args.no_mixed and world == 1:
        mixed = mixed_forms(gb, si, args, s, H, spec)

    out = {
        "metric": METRIC, "value": ms_max / world, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if spec["precision"] == 0 else ("f64+f32" if spec["precision"] == 1
                                                        else "f64+bf16"),
        "data": "synthetic",
        "config": {"workload": spec["desc"],
                   "l2": ("inputs larger than L2: one solve streams K (%.0f MB as run) and the "
                          "hierarchy (%.0f MB per preconditioner application) each iteration; "
                          "kernels timed alone follow a %d MB buffer write"
                          % (k_run_bytes / 1e6, gb.precond_bytes(H) / 1e6,
                             L2_FLUSH_BYTES >> 20)),
                   "parallelism": "replicas" if world > 1 else "1gpu",
                   "iterations": iters[-1], "rel_res": rel_res, "converged": converged,
                   "setup_s": setup_s, "graph": not args.no_graph,
                   **{k: (args.relax if k == "relax" else v) for k, v in extra.items()}},
        "e2e": {"value": e2e_ms / world, "unit": UNIT, "h2d_bytes_per_step": int(b.numel() * 8),
                "d2h_bytes_per_step": int(x.numel() * 8)},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "fp64_peak": fp64,
        "outer_spmv": outer_spmv,
        "bsr_spmv": bsr_spmv,
        "vcycle": vcycle,
        "mixed": mixed,
        "clocks": clocks,
        "hierarchy_bytes": gb.hierarchy_info(H)["bytes"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        run, it_scale, _, k, _ = time_cpu_oracle(s, wl, iters[-1], sample_iters=args.sample_iters)
        per_it = cpu_oracle_sample(run, k)
        out["cpu_baseline"] = {
            "value": per_it * it_scale * 1e3, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": ("FP64 NumPy/SciPy oracle, 1 thread; setup untimed; %d Krylov iterations "
                       "of the full-size workload timed and scaled to the GPU solve's %d "
                       "iterations" % (k, it_scale))}
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
