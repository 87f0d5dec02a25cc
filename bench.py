#!/usr/bin/env python3
"""Benchmark: GIAMG-PCG time to a 1e-8 relative residual on one GB300.

Workload (default): Helmholtz -lap u + 10 u = f on the unit cube, 16^3 hexahedra with interior
vertices jittered by +-0.2 h (seed 1), nodal GLL order 6: 912,673 dofs, 410,227,705 nonzeros
(FP64 CSR, 4.9 GB), manufactured right-hand side, Chebyshev degree 3, rtol 1e-8.  One step is one
full solve (all V-cycle levels, the outer CG) with inputs resident in HBM.  The headline is the
FP32 V-cycle inside FP64 flexible CG; the FP64 V-cycle in PCG is timed the same way beside it.

  python bench.py [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

`--impl reference` times the CPU oracle (plain FP64 C, OpenMP row loops) on the host cores with
the same metric and config: each step is one full oracle solve to the tolerance (the FP32 V-cycle
in FP64 flexible CG, as the headline).  Under torchrun every rank solves its own copy (replicas;
no collective on the data path) and rank 0 prints the line with the max over ranks.

Besides the headline workload the line carries every other configuration of the workload set
(`configs`): the 4^3 p = 4 latency case, the 24^3 p = 4 Poisson case with 32 right-hand sides
(batched FP32 V-cycle against single FP64 solves), the 12^3 graded p = 8 case with its own
roofline, and the served request stream; and for each solve the distance of the GPU's mixed-
precision solution from the oracle's FP64 solution.
"""
from __future__ import annotations

import argparse
import collections
import csv
import hashlib
import io
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

METRIC = "PCG time-to-1e-8 relres & V-cycle HBM GB/s, FP32-in-FP64 vs FP64; p50/p99 ms"
WORKLOAD_TEXT = {
    "helmholtz_16cube_jitter_p6": "Helmholtz lambda=10, unit cube, 16^3 hex jittered +-0.2h (seed 1), GLL p=6",
    "helmholtz_4cube_p4": "Helmholtz lambda=1, unit cube, 4^3 hex, GLL p=4",
    "helmholtz_8cube_jitter_p6": "Helmholtz lambda=10, unit cube, 8^3 hex jittered +-0.2h (seed 1), GLL p=6",
    "helmholtz_12cube_jitter_p6": "Helmholtz lambda=10, unit cube, 12^3 hex jittered +-0.2h (seed 1), GLL p=6",
    "poisson_24cube_jitter_p4": "Poisson lambda=0, unit cube, 24^3 hex jittered (seed 2), GLL p=4",
    "helmholtz_12cube_graded_p8": "Helmholtz lambda=1000, kappa=1+0.5sin(2pi x), 12^3 hex graded to z=0, GLL p=8",
}


def config_of(workload, prob, k, rtol, levels):
    """The `config` object of the JSON line, the same for both arms."""
    return {"workload": workload, "description": WORKLOAD_TEXT.get(workload, ""), "dofs": prob.n, "nnz": prob.nnz,
            "rtol": rtol, "cheb_degree": k, "levels": [[L["n"], L["nnz"], L["order"]] for L in levels],
            "l2": f"inputs larger than L2 (finest matrix {12 * prob.nnz / 1e9:.2f} GB), no flush",
            "parallelism": "replicas"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="helmholtz_16cube_jitter_p6")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the multi-RHS and serving measurements")
    ap.add_argument("--schedules", action="store_true",
                    help="compare the p schedules (halving, by one, by two) on two 16^3 operators and print them")
    ap.add_argument("--block", action="store_true",
                    help="compare block CG with independent columns (32 RHS) on the Poisson workload and the modal operator")
    ap.add_argument("--serving-full", action="store_true",
                    help="run only the 512-request serving stream and print it")
    ap.add_argument("--serving-meshes", default="4,8,12,16", help="mesh sizes of the served stream")
    ap.add_argument("--no-serving", action="store_true", help="skip the served stream")
    ap.add_argument("--case", metavar="SPEC",
                    help="run one case for a profiler and exit: setup, then --solves solves (or --rhs-columns "
                         "multi-RHS solves); SPEC is a workload name or n,p,mesh,lambda,cheb_degree")
    ap.add_argument("--precision", type=int, default=1, help="with --case: 0 FP64, 1 FP32 V-cycle")
    ap.add_argument("--solves", type=int, default=1, help="with --case: number of solves")
    ap.add_argument("--rhs-columns", type=int, default=1, help="with --case: right-hand sides per solve")
    ap.add_argument("--summarize-launches", metavar="CSV",
                    help="print a per-kernel summary of an ncu launch list and exit (no GPU work)")
    ap.add_argument("--split-at", metavar="KERNEL",
                    help="with --summarize-launches: also a table per segment starting at this kernel")
    return ap.parse_args()


_T0 = time.perf_counter()


def phase(msg):
    """Progress of the run on stderr (the JSON line goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def pct(v, q):
    v = sorted(v)
    if not v:
        return None
    k = (len(v) - 1) * q
    lo = int(k)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.path = tempfile.mktemp(suffix=".csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 8:
                    continue
                try:
                    sm.append(float(p[0]))
                    mx.append(float(p[1]))
                except ValueError:
                    continue
                for name, v in zip(names, p[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2512_15121_gb300", "csrc", "solve_kernels.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def _launch_table(launches):
    agg = collections.OrderedDict()
    for name, ns in launches:
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += ns
    tot = sum(a[1] for a in agg.values()) or 1.0
    out = [f"{'launches':>8} {'total_ms':>10} {'share':>7}  kernel", "-" * 70]
    for k, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append(f"{c:8d} {t / 1e6:10.3f} {100 * t / tot:6.2f}%  {k}")
    out.append(f"{sum(a[0] for a in agg.values()):8d} {tot / 1e6:10.3f} 100.00%  (all)")
    return "\n".join(out)


def summarize_launches(path, split=None):
    """Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) by kernel: launches,
    total device time and share.  With `split`, also one table per segment of the list, a new
    segment starting at every launch whose kernel name contains `split`."""
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    launches = []
    for r in csv.DictReader(io.StringIO("".join(lines))):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        raw = r["Kernel Name"].replace("(anonymous namespace)::", "").replace("<unnamed>::", "")
        raw = re.sub(r"^void\s+", "", raw.replace("unnamed>::", ""))
        name = re.sub(r"\(.*", "", raw)
        m = re.search(r"csr_rows<(\d+), (\w+), (\d)>", r["Kernel Name"])
        if m:
            name = f"csr_rows<{m.group(1)},{m.group(2)},{['spmv','residual','cheb','add'][int(m.group(3))]}>"
        v = float(r["Metric Value"])
        if r["Metric Unit"] in ("usecond", "us"):
            v *= 1e3
        elif r["Metric Unit"] in ("msecond", "ms"):
            v *= 1e6
        launches.append((name, v))
    out = ["all launches", _launch_table(launches)]
    if split:
        segs = []
        for name, v in launches:
            if split in name or not segs:
                segs.append([])
            segs[-1].append((name, v))
        for i, seg in enumerate(segs):
            out += ["", f"segment {i} (from launch {sum(len(s) for s in segs[:i])})", _launch_table(seg)]
    return "\n".join(out)


def ncu_traffic(workload, mode):
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary, if it was taken
    on the current kernel source; otherwise None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload][mode]
        if e.get("solve_kernels_sha") != kernel_source_hash():
            return None
        return e["dram_bytes_per_launch"]
    except Exception:
        return None


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as td
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    td.init_process_group(backend)
    return rank, ws, local, td


def max_over_ranks(td, v):
    if td is None:
        return v
    import torch
    t = torch.tensor([float(v)], device="cuda" if torch.cuda.is_available() else "cpu")
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------ reference arm
def run_reference(args):
    """The CPU oracle as it stands on the host cores: every step one full solve of the workload to
    the tolerance (FP32 V-cycle in FP64 flexible CG, the headline's method), wall-clock timed."""
    rank, ws, local, td = dist()
    if rank != 0:
        return
    import fegen
    import oracle
    k = fegen.WORKLOADS[args.workload]["k"]
    prob = fegen.workload(args.workload)
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
    levels = [H.level_info(l) for l in range(H.num_levels)]
    times, iters = [], 0
    t_all = time.perf_counter()
    for s in range(args.warmup + args.steps):
        if s == args.warmup:
            t_all = time.perf_counter()
        t0 = time.perf_counter()
        _, iters, rr, _, st = H.solve(prob.b, rtol=args.rtol, precision=1)
        dt = (time.perf_counter() - t0) * 1e3
        if s >= args.warmup:
            times.append(dt)
    wall = (time.perf_counter() - t_all) * 1e3
    cores = oracle.num_threads()
    p50 = pct(times, 0.5)
    line = {"metric": METRIC, "value": round(p50, 3), "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(wall / args.steps, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle in f64 FCG (CPU oracle)",
            "data": "synthetic", "impl": "reference", "p99_ms": round(pct(times, 0.99), 3), "iters": iters,
            "relres": rr, "config": config_of(args.workload, prob, k, args.rtol, levels),
            "cpu_baseline": {"value": round(p50, 3), "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": f"each step: one full oracle solve to rtol {args.rtol:g} ({iters} iterations, "
                                       f"FP32 V-cycle in FP64 flexible CG) on the full workload"},
            "e2e": {"value": round(p50, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    H.close()
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ our arm
def timed_solves(S, b, x, stream, rtol, precision, steps, warmup, profiled, td=None):
    """K timed solves after W warm-ups.  profiled=False: the default path (the whole PCG loop as one
    CUDA graph).  profiled=True: per-kernel CUDA events by category, which need the host-driven
    loop (event records cannot sit inside the graph's conditional bodies): same kernels, same
    launch shapes; this pass gives the roofline's kernel times."""
    import torch
    import paper_2512_15121_gb300 as g
    S.profile(False)
    for _ in range(warmup):
        S.solve(b, rtol=rtol, precision=precision, x=x)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if td:
        td.barrier()
    torch.cuda.synchronize()
    if profiled:
        S.profile(True)
    torch.cuda.profiler.start()  # marks the timed region for an external profiler (no effect otherwise)
    c0 = g.launch_count()
    t_start = time.perf_counter()
    its = []
    for e0, e1 in ev:
        e0.record(stream)
        _, it, rr = S.solve(b, rtol=rtol, precision=precision, x=x)
        e1.record(stream)
        its.append(it)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t_start) * 1e3
    torch.cuda.profiler.stop()
    if td:
        td.barrier()
    launches = g.launch_count() - c0
    ms = [a.elapsed_time(b_) for a, b_ in ev]
    prof = [S.profile_read(c) for c in range(6)] if profiled else None
    S.profile(False)
    _, true_rr = S.stats(0)
    return dict(p50=pct(ms, 0.5), p99=pct(ms, 0.99), total=sum(ms), wall=wall, iters=its[-1],
                iters_all=sorted(set(its)), launches=launches, prof=prof, true_relres=true_rr)


def roofline(res, S, prob, workload, mode, peak, peak_kind):
    """The finest level's row kernels inside the V-cycle (category 0: smoother steps and residual):
    algorithmic bytes of their launches / their CUDA-event time, against the measured copy
    bandwidth."""
    ms, cnt, by = res["prof"][0]
    if cnt == 0 or ms <= 0:
        return None
    tpr, form = S.kernel(0, 1 if mode == "mixed" else 0)
    achieved = by / cnt / (ms / cnt * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": ncu_traffic(workload, mode),
            "kernel": f"finest-level row kernels ({'FP32' if mode == 'mixed' else 'FP64'} Chebyshev step and "
                      f"residual): {form} form, {tpr} threads per row",
            "launches": cnt, "avg_launch_ms": round(ms / cnt, 4), "algorithmic_bytes_per_launch": round(by / cnt),
            "peak_kind": peak_kind,
            "timed_region": "a second timed region of the same K solves with per-kernel CUDA events "
                            "(host-driven loop, same kernels and launch shapes)"}


def roofline_fp64(res, S, prob, workload, peak, peak_kind):
    """The FP64 row kernels are bound by GB300's FP64 pipe (1/64 of the FP32 rate), not by HBM:
    2 flops per nonzero against the nominal 1.25 TFLOP/s FP64 peak (152 SMs x 2070 MHz x 2 flops x
    2 FP64 FMA per SM per clock; a probe kernel measured 1.204 TFLOP/s)."""
    hbm = roofline(res, S, prob, workload, "fp64", peak, peak_kind)
    if hbm is None:
        return None
    ms, cnt, _ = res["prof"][0]
    flops = 2.0 * prob.nnz  # one FMA per nonzero of the finest matrix per launch
    achieved = flops * cnt / (ms * 1e-3) / 1e12
    out = dict(hbm)
    out.update({"bound": "alu", "achieved": round(achieved, 4), "peak": 1.25, "unit": "TFLOP/s",
                "frac": round(achieved / 1.25, 4), "peak_kind": "nominal FP64 rate (derived)",
                "algorithmic_flops_per_launch": flops,
                "hbm": {"achieved": hbm["achieved"], "peak": peak, "unit": "GB/s", "frac": hbm["frac"]}})
    return out


def vcycle_gbs(res):
    """V-cycle bytes and time: every profiler category except the outer CG product (5)."""
    ms = sum(res["prof"][c][0] for c in range(5))
    by = sum(res["prof"][c][2] for c in range(5))
    return round(by / (ms * 1e-3) / 1e9, 1) if ms > 0 else None


def gpu_uuid(dev):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None


def timed_setup(prob, **opts):
    """The library's setup on input arrays already in device memory, and the upload of those arrays
    from host memory before it, timed apart: (Solver, setup_ms, upload_ms)."""
    import torch
    import paper_2512_15121_gb300 as g
    dev = torch.device("cuda", torch.cuda.current_device())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    arrs = [torch.from_numpy(a).to(dev) for a in (prob.row_ptr, prob.col, prob.val, prob.elem_dof)]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    S = g.Solver(prob.n, *arrs, prob.p, None, device_ptrs=1, **opts)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del arrs
    return S, (t2 - t1) * 1e3, (t1 - t0) * 1e3


def measure_autotuned(prob, k, b, steps, warmup, rtol, default_mixed, default_fp64):
    """The same operator set up with autotune = 1 (the finest level's row kernels chosen by timing
    forced-iteration solves inside setup): setup time, what it picked, and the solve times against
    the defaults'."""
    import torch
    import paper_2512_15121_gb300 as g
    S, setup_ms, _ = timed_setup(prob, cheb_degree=k, autotune=1)
    x = torch.empty_like(b)
    stream = torch.cuda.current_stream()
    mixed = timed_solves(S, b, x, stream, rtol, 1, steps, warmup, False)
    fp64 = timed_solves(S, b, x, stream, rtol, 0, steps, warmup, False)
    out = {"setup_ms": round(setup_ms, 1),
           "picked": {"fp64": list(S.kernel(0, 0)), "fp32": list(S.kernel(0, 1))},
           "mixed_p50_ms": round(mixed["p50"], 3), "fp64_p50_ms": round(fp64["p50"], 3),
           "mixed_vs_default": round(mixed["p50"] / default_mixed, 3),
           "fp64_vs_default": round(fp64["p50"] / default_fp64, 3)}
    S.close()
    return out


def measure_config(name, steps, warmup, profiled, peak, peak_kind, rtol=1e-8, autotune=False):
    """One workload of the set with the default options: setup time, the FP32-V-cycle and FP64 solves
    (CUDA-event p50/p99 of the captured graph), with profiled=True the roofline of the finest row
    kernels, and the two solutions (host copies) for the comparison with the oracle."""
    import torch
    import fegen
    import paper_2512_15121_gb300 as g
    k = fegen.WORKLOADS[name]["k"]
    prob = fegen.workload(name)
    dev = torch.device("cuda", torch.cuda.current_device())
    S, setup_ms, upload_ms = timed_setup(prob, cheb_degree=k)
    b = torch.from_numpy(prob.b).to(dev)
    x = torch.empty_like(b)
    stream = torch.cuda.current_stream(dev)
    clocks = Clocks(gpu_uuid(dev))
    mixed = timed_solves(S, b, x, stream, rtol, 1, steps, warmup, False)
    fp64 = timed_solves(S, b, x, stream, rtol, 0, steps, warmup, False)
    if profiled:
        mixed["prof"] = timed_solves(S, b, x, stream, rtol, 1, steps, warmup, True)["prof"]
        fp64["prof"] = timed_solves(S, b, x, stream, rtol, 0, steps, warmup, True)["prof"]
    clk = clocks.stop()
    xm = S.solve(b, rtol=rtol, precision=1)[0].cpu().numpy()
    xd = S.solve(b, rtol=rtol, precision=0)[0].cpu().numpy()
    out = {"workload": name, "description": WORKLOAD_TEXT.get(name, ""), "dofs": prob.n, "nnz": prob.nnz,
           "cheb_degree": k, "levels": [[L["n"], L["nnz"], L["order"]] for L in
                                        (S.level_info(l) for l in range(S.num_levels))],
           "setup_ms": round(setup_ms, 1), "upload_ms": round(upload_ms, 1),
           "mixed": {"p50_ms": round(mixed["p50"], 3), "p99_ms": round(mixed["p99"], 3), "iters": mixed["iters"],
                     "true_relres": mixed["true_relres"], "launches_per_solve": mixed["launches"] // steps},
           "fp64": {"p50_ms": round(fp64["p50"], 3), "p99_ms": round(fp64["p99"], 3), "iters": fp64["iters"],
                    "true_relres": fp64["true_relres"]},
           "speedup_mixed_vs_fp64": round(fp64["p50"] / mixed["p50"], 3), "steps": steps, "warmup": warmup,
           "clocks": clk}
    if profiled:
        out["roofline"] = roofline(mixed, S, prob, name, "mixed", peak, peak_kind)
        out["fp64"]["roofline"] = roofline_fp64(fp64, S, prob, name, peak, peak_kind)
        out["vcycle_gbs"] = vcycle_gbs(mixed)
        out["fp64"]["vcycle_gbs"] = vcycle_gbs(fp64)
    out["row_kernels"] = {"fp64": list(S.kernel(0, 0)), "fp32": list(S.kernel(0, 1))}
    S.close()
    if autotune:
        out["autotune"] = measure_autotuned(prob, k, b, steps, warmup, rtol, mixed["p50"], fp64["p50"])
    return out, (prob, k, prob.b, {"mixed": xm, "fp64": xd})


def oracle_errors(prob, k, b, sols, rtol=1e-8, H=None):
    """The oracle's FP64 PCG on the same system (stopping freely at rtol) and the relative distance
    of each GPU solution from it."""
    import numpy as np
    import oracle
    own = H is None
    if own:
        H = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
    t0 = time.perf_counter()
    xo, ito, rro, _, st = H.solve(b, rtol=rtol)
    ms = (time.perf_counter() - t0) * 1e3
    if own:
        H.close()
    nx = np.linalg.norm(xo)
    out = {f"{key}_vs_oracle_fp64": float(np.linalg.norm(x - xo) / nx) for key, x in sols.items()}
    out.update({"oracle_iters": ito, "oracle_relres": rro, "oracle_status": st, "oracle_solve_ms": round(ms, 1)})
    return out


def run_ours(args):
    import numpy as np
    import torch

    import fegen
    import paper_2512_15121_gb300 as g

    rank, ws, local, td = dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    k = fegen.WORKLOADS[args.workload]["k"]
    prob = fegen.workload(args.workload)
    stream = torch.cuda.current_stream(dev)

    S, setup_ms, upload_ms = timed_setup(prob, cheb_degree=k)
    levels = [S.level_info(l) for l in range(S.num_levels)]
    b = torch.from_numpy(prob.b).to(dev)
    x = torch.empty_like(b)
    peak, peak_kind = measured_peaks()

    phase(f"setup {args.workload}: {setup_ms:.0f} ms")
    clocks = Clocks(gpu_uuid(dev))
    steps, warmup = args.steps, args.warmup
    mixed = timed_solves(S, b, x, stream, args.rtol, 1, steps, warmup, False, td)
    fp64 = timed_solves(S, b, x, stream, args.rtol, 0, steps, warmup, False, td)
    mixed_prof = timed_solves(S, b, x, stream, args.rtol, 1, steps, warmup, True, td)
    fp64_prof = timed_solves(S, b, x, stream, args.rtol, 0, steps, warmup, True, td)
    clk = clocks.stop()
    mixed["prof"], fp64["prof"] = mixed_prof["prof"], fp64_prof["prof"]
    sols = {"mixed": S.solve(b, rtol=args.rtol, precision=1)[0].cpu().numpy(),
            "fp64": S.solve(b, rtol=args.rtol, precision=0)[0].cpu().numpy()}

    # end to end through the C ABI with host buffers (pinned): H2D of b and D2H of x inside
    S.set_device_ptrs(False)
    bh = torch.from_numpy(prob.b).pin_memory()
    xh = torch.empty(prob.n, dtype=torch.float64).pin_memory()
    bh_np, xh_np = bh.numpy(), xh.numpy()
    e2e = []
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        S.solve(bh_np, rtol=args.rtol, precision=1, x=xh_np)
        dt = (time.perf_counter() - t0) * 1e3
        if s >= warmup:
            e2e.append(dt)
    S.set_device_ptrs(True)
    phase("headline timed regions and e2e done")

    extras, later = {}, {}
    if not args.no_extras:
        from paper_2512_15121_gb300 import tune
        best_k, tk = tune.tune_cheb_degree(S, b, degrees=(1, 2, 3, 4, 5), precision=1, rtol=args.rtol)
        extras["cheb_degree_tuning"] = {"best": best_k, "paper_default": k,
                                        "ms": {t.degree: round(t.ms, 3) for t in tk},
                                        "iters": {t.degree: t.iterations for t in tk}}
        S.set_cheb_degree(k)
    roof_mixed = roofline(mixed, S, prob, args.workload, "mixed", peak, peak_kind)
    roof_fp64 = roofline_fp64(fp64, S, prob, args.workload, peak, peak_kind)
    S.close()
    if not args.no_extras:
        configs = {}
        # the latency case and the graded p = 8 case (with its own roofline)
        for name, profiled in (("helmholtz_4cube_p4", False), ("helmholtz_12cube_graded_p8", True)):
            configs[name], later[name] = measure_config(name, steps, warmup, profiled, peak, peak_kind, args.rtol,
                                                        autotune=profiled)
            phase(f"config {name} done")
        # 32 right-hand sides against single solves in both precisions
        configs["poisson_24cube_jitter_p4"], later["poisson_24cube_jitter_p4"] = measure_batch(g, torch)
        phase("config poisson_24cube_jitter_p4 done")
        extras["grouped_solve"] = measure_grouped()
        phase("grouped solve done")
        extras["configs"] = configs

    value = max_over_ranks(td, mixed["p50"])
    ms_per_step = max_over_ranks(td, mixed["wall"] / steps)
    cpu, err = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, err = cpu_baseline(prob, k, args.rtol, sols)
        phase("cpu baseline and oracle error of the headline done")
        for name, (p2, k2, b2, sols2) in later.items():
            extras["configs"][name]["error"] = oracle_errors(p2, k2, b2, sols2, args.rtol)
            phase(f"oracle error of {name} done")
    config = config_of(args.workload, prob, k, args.rtol, levels)
    n_dofs = prob.n
    # the served stream holds its operators on the host: free the other workloads' first
    for p2, _, _, _ in later.values():
        p2.close()
    later.clear()
    prob.close()
    del prob
    if not args.no_extras and not args.no_serving:
        extras["configs"]["served_stream"] = measure_serving_full(
            meshes=tuple(int(m) for m in args.serving_meshes.split(",")))
        phase("served stream done")
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": ws, "steps": steps,
        "warmup": warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle in f64 FCG",
        "data": "synthetic (seeded jittered-hex GLL assembly; stands in for the paper's Nektar++ matrices)",
        "config": config,
        "p50_ms": round(mixed["p50"], 3), "p99_ms": round(mixed["p99"], 3), "iters": mixed["iters"],
        "true_relres": mixed["true_relres"],
        "fp64": {"p50_ms": round(fp64["p50"], 3), "p99_ms": round(fp64["p99"], 3), "iters": fp64["iters"],
                 "true_relres": fp64["true_relres"], "roofline": roof_fp64, "vcycle_gbs": vcycle_gbs(fp64)},
        "speedup_mixed_vs_fp64": round(fp64["p50"] / mixed["p50"], 3),
        "error": err,
        "profiled_p50_ms": {"mixed": round(mixed_prof["p50"], 3), "fp64": round(fp64_prof["p50"], 3)},
        "vcycle_gbs": vcycle_gbs(mixed),
        "setup_ms": round(setup_ms, 1),
        "setup_note": "giamg_setup on the input arrays already in device memory; their upload from "
                      f"host memory before it: {upload_ms:.1f} ms",
        "roofline": roof_mixed,
        "cpu_baseline": cpu,
        "e2e": {"value": round(pct(e2e, 0.5), 3), "unit": "ms", "h2d_bytes_per_step": 8 * n_dofs,
                "d2h_bytes_per_step": 8 * n_dofs},
        "gpu_launches": mixed["launches"],
        "clocks": clk,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)


def measure_batch(g, torch, m=32, reps=5):
    """32 right-hand sides of the 24^3 Poisson workload as one multi-RHS solve (FP32 V-cycle in
    flexible CG) and as one block in block CG, against single-RHS solves of the first column with
    the FP32 V-cycle and with the plain FP64 V-cycle (the throughput the batched mixed form is
    compared with)."""
    import numpy as np
    import fegen
    name = "poisson_24cube_jitter_p4"
    k = fegen.WORKLOADS[name]["k"]
    prob = fegen.workload(name, rhs="none")
    B = np.stack([prob.rhs("fourier", 1000 + j) for j in range(m)], axis=1)
    S, setup_ms, upload_ms = timed_setup(prob, cheb_degree=k)
    Bd = torch.from_numpy(B).cuda()
    b0 = Bd[:, 0].contiguous()
    for _ in range(2):
        S.solve_batch(Bd, rtol=1e-8, precision=1)
        S.solve(b0, rtol=1e-8, precision=1)
        S.solve(b0, rtol=1e-8, precision=0)
    for _ in range(2):
        S.solve_batch(Bd, rtol=1e-8, precision=1, block=True)
    st = torch.cuda.current_stream()
    clocks = Clocks(gpu_uuid(torch.device("cuda", torch.cuda.current_device())))
    tb, ts, t64, tk = [], [], [], []

    def timed(fn, out):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r = fn()
        e1.record(st)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
        return r

    for _ in range(reps):
        X, it, rr = timed(lambda: S.solve_batch(Bd, rtol=1e-8, precision=1), tb)
        _, it1, _ = timed(lambda: S.solve(b0, rtol=1e-8, precision=1), ts)
        x64, it64, _ = timed(lambda: S.solve(b0, rtol=1e-8, precision=0), t64)
        _, itk, rrk = timed(lambda: S.solve_batch(Bd, rtol=1e-8, precision=1, block=True), tk)
    clk = clocks.stop()
    sols = {"mixed_batched_column0": X[:, 0].cpu().numpy(), "fp64": x64.cpu().numpy()}
    S.close()
    pb, ps, p64, pk = pct(tb, 0.5), pct(ts, 0.5), pct(t64, 0.5), pct(tk, 0.5)
    out = {"workload": name, "description": WORKLOAD_TEXT[name], "dofs": prob.n, "nnz": prob.nnz, "cheb_degree": k,
           "setup_ms": round(setup_ms, 1), "upload_ms": round(upload_ms, 1), "m": m, "reps": reps,
           "batch_mixed": {"p50_ms": round(pb, 3), "per_solve_ms": round(pb / m, 3),
                           "iters": [int(it.min()), int(it.max())], "max_relres": float(rr.max())},
           "single_mixed": {"p50_ms": round(ps, 3), "iters": int(it1)},
           "single_fp64": {"p50_ms": round(p64, 3), "iters": int(it64)},
           "throughput_batch_mixed_vs_single_fp64": round(p64 * m / pb, 2),
           "throughput_batch_mixed_vs_single_mixed": round(ps * m / pb, 2),
           "block_cg": {"p50_ms": round(pk, 3), "iters": int(itk.max()), "max_relres": float(rrk.max())},
           "clocks": clk}
    return out, (prob, k, np.ascontiguousarray(B[:, 0]), sols)


def measure_serving(n_requests=128, rate=150.0):
    """A stream of solve requests (jittered 4^3..8^3 meshes, p in {2,4,6}, lambda in {0,1,1000},
    1..8 right-hand sides, Poisson arrivals) through the continuous-batching server."""
    from paper_2512_15121_gb300 import serve
    # warm-up stream on a throwaway server (loads the kernels' modules; its hierarchies are dropped)
    warm, _ = serve.synthetic_stream(16, seed=99, rate_per_s=rate)
    w = serve.Server(slots=4)
    serve.run_stream(w, warm)
    w.close()
    reqs, ops = serve.synthetic_stream(n_requests, seed=7, rate_per_s=rate)
    srv = serve.Server(slots=4)
    stats = serve.run_stream(srv, reqs)
    srv.close()
    stats.update({k: int(v) for k, v in srv.stats.items()})
    stats.update({"rate_per_s": rate, "operators": len(ops), "errors": sum(r.error is not None for r in reqs),
                  "mix": "jittered 4^3/6^3/8^3, p in {2,4,6}, lambda in {0,1,1000}, 1-8 RHS, FP32 V-cycle"})
    return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in stats.items()}


def measure_grouped(reps=10, warmup=3):
    """The grouped solve against separate ones: eight small operators of the served stream's
    kind (jittered 4^3 and 8^3 meshes, p 2 and 4, lambda 1 and 1000), 4 right-hand sides each,
    FP32 V-cycle: one giamg_solve_grouped call against the eight giamg_solve_batch calls one after
    the other (CUDA-event medians), and the results compared bit for bit."""
    import numpy as np
    import torch
    import fegen
    import paper_2512_15121_gb300 as g
    probs, solvers, Bs = [], [], []
    for mesh in (4, 8):
        for p in (2, 4):
            for lam in (1.0, 1000.0):
                prob = fegen.make(mesh, p, mesh="jitter", mesh_seed=mesh, lam=lam, rhs="none")
                S = g.Solver.from_problem(prob, device=True, cheb_degree=3, row_form=2)
                Bs.append(torch.from_numpy(np.stack([prob.rhs("fourier", 500 + j) for j in range(4)], axis=1)).cuda())
                probs.append(prob)
                solvers.append(S)

    def separate():
        return [S.solve_batch(B, rtol=1e-8, precision=1) for S, B in zip(solvers, Bs)]

    def grouped():
        return g.solve_grouped(solvers, Bs, rtol=1e-8)

    out = {}
    for name, fn in (("separate", separate), ("grouped", grouped)):
        for _ in range(warmup):
            fn()
        ts = []
        launches = g.launch_count()
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            res = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[name] = {"p50_ms": round(pct(ts, 0.5), 3), "launches_per_call": (g.launch_count() - launches) // reps}
        out[name + "_x"] = [r[0] for r in res]
    same = all(torch.equal(a, b) for a, b in zip(out.pop("separate_x"), out.pop("grouped_x")))
    for S, pr in zip(solvers, probs):
        S.close()
        pr.close()
    return {"operators": [[pr.n, pr.nnz, pr.p] for pr in probs], "rhs_per_operator": 4, **out,
            "speedup": round(out["separate"]["p50_ms"] / out["grouped"]["p50_ms"], 2), "bitwise_equal": same}


def measure_serving_full(n_requests=512, load=0.8, meshes=(4, 8, 12, 16)):
    """The served request stream: 512 requests on jittered 4^3 / 8^3 / 12^3 / 16^3 meshes, p in
    {2, 4, 6, 8}, lambda in {0, 1, 1000} (up to 48 operators, the largest 2,146,689 dofs and 1.94e9
    nonzeros), 1..8 right-hand sides each (the seeded Fourier fields at the nodes), FP32 V-cycle.
    First the capacity: every request submitted at once to a fresh server; then the same stream
    with Poisson arrivals at `load` times that capacity, again on a fresh server (setups included
    in both).  Latency is arrival to result on the host."""
    import dataclasses
    import torch
    from paper_2512_15121_gb300 import serve
    warm, _ = serve.synthetic_stream(16, seed=99, rate_per_s=1e6, meshes=(4,), orders=(2, 4, 8))
    w = serve.Server(slots=4)
    serve.run_stream(w, warm)
    w.close()
    t0 = time.perf_counter()
    # arrival offsets for rate 1/s; run_stream scales them by time_scale = 1 / rate
    reqs, ops = serve.synthetic_stream(n_requests, seed=7, rate_per_s=1.0, meshes=meshes, orders=(2, 4, 6, 8),
                                       lambdas=(0.0, 1.0, 1000.0), rhs_kind="nodal")
    gen_s = time.perf_counter() - t0
    offsets = [r.arrival for r in reqs]
    cols = sum(r.columns for r in reqs)
    largest = max(ops.values(), key=lambda pr: pr.nnz)

    def run(time_scale, label):
        rs = [dataclasses.replace(r, arrival=off) for r, off in zip(reqs, offsets)]
        clocks = Clocks(gpu_uuid(torch.device("cuda", torch.cuda.current_device())))
        t = time.perf_counter()
        srv = serve.Server(slots=4)
        try:
            st = serve.run_stream(srv, rs, time_scale=time_scale, drain_timeout=300.0)
        except TimeoutError:  # report what finished; the line says the pass did not drain
            st = serve.latency_summary(rs)
            st["did_not_drain_s"] = 300.0
            with srv.cv:
                srv.pending.clear()
        srv.close()
        st.update({k: int(v) for k, v in srv.stats.items()})
        st["errors"] = sum(r.error is not None for r in rs)
        st["first_error"] = next((r.error for r in rs if r.error is not None), None)
        st["wall_s"] = time.perf_counter() - t
        st["clocks"] = clocks.stop()
        out = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()}
        phase(f"served stream, {label}: {json.dumps(out)}")
        return out

    phase(f"served stream generated: {len(ops)} operators, {cols} solves, {gen_s:.1f} s")
    cap = run(0.0, "capacity")
    capacity = cap.get("solves_per_s") or 1.0
    rate = load * capacity * n_requests / cols  # requests per second
    loaded = run(1.0 / rate, f"{load}x capacity")
    loaded["rate_per_s"] = round(rate, 2)
    out = {"requests": n_requests, "solves": cols, "operators": len(ops), "generation_s": round(gen_s, 1),
           "largest_operator": {"dofs": largest.n, "nnz": largest.nnz, "order": largest.p},
           "mix": f"jittered {'/'.join(f'{m}^3' for m in meshes)}, p in {{2,4,6,8}}, lambda in {{0,1,1000}}, "
                  f"1-8 nodal Fourier RHS, FP32 V-cycle, Poisson arrivals (seed 7)",
           "capacity": cap, f"at_{load}x_capacity": loaded}
    for pr in ops.values():
        pr.close()
    return out


def measure_schedules(steps=10, warmup=3):
    """The p schedules compared (the paper compares coarsening by one and by two): halving, by one
    and by two on the 16^3 p = 6 benchmark operator, on a 16^3 p = 5 one, and on the benchmark
    operator in the modal basis (injection P); levels, iterations, solve time (FP32 V-cycle in
    FP64 FCG and FP64 PCG, CUDA-event medians) and setup time."""
    import statistics
    import torch
    import fegen
    import paper_2512_15121_gb300 as g
    out = {}
    for name, cfg, k in (("helmholtz_16cube_jitter_p6", fegen.WORKLOADS["helmholtz_16cube_jitter_p6"], 3),
                         ("helmholtz_16cube_jitter_p5", dict(n=16, p=5, mesh="jitter", mesh_seed=1, lam=10.0,
                                                             rhs="manufactured"), 3),
                         ("helmholtz_16cube_jitter_p6_modal", dict(fegen.WORKLOADS["helmholtz_16cube_jitter_p6"],
                                                                   basis="modal"), 3)):
        cfg = {key: v for key, v in cfg.items() if key != "k"}
        basis = 1 if cfg.get("basis") == "modal" else 0
        prob = fegen.make(**cfg)
        b = torch.from_numpy(prob.b).cuda()
        res = {}
        for sched, label in ((0, "halving"), (1, "by_one"), (2, "by_two")):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            S = g.Solver.from_problem(prob, device=True, cheb_degree=k, p_schedule=sched, basis=basis)
            torch.cuda.synchronize()
            setup_ms = (time.perf_counter() - t0) * 1e3
            row = {"levels": [[S.level_info(l)["n"], S.level_info(l)["order"]] for l in range(S.num_levels)],
                   "setup_ms": round(setup_ms, 1)}
            for prec, key in ((1, "mixed"), (0, "fp64")):
                for _ in range(warmup):
                    S.solve(b, rtol=1e-8, precision=prec)
                ts = []
                for _ in range(steps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    _, it, rr = S.solve(b, rtol=1e-8, precision=prec)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                row[key] = {"iters": int(it), "relres": rr, "ms": round(statistics.median(ts), 3),
                            "ms_per_iter": round(statistics.median(ts) / it, 3)}
            S.close()
            res[label] = row
        out[name] = res
        prob.close()
    return out


def measure_block(m=32, steps=3, warmup=1):
    """32 right-hand sides solved as independent CG recurrences (giamg_solve_batch) and as one
    block in block CG (giamg_solve_block), FP32 and FP64 V-cycle, CUDA-event medians: the 24^3
    p = 4 Poisson workload and the 16^3 p = 6 operator in the modal basis."""
    import statistics
    import numpy as np
    import torch
    import fegen
    import paper_2512_15121_gb300 as g
    out = {}
    for name, cfg, k in (("poisson_24cube_jitter_p4", fegen.WORKLOADS["poisson_24cube_jitter_p4"], 2),
                         ("helmholtz_16cube_jitter_p6_modal", dict(fegen.WORKLOADS["helmholtz_16cube_jitter_p6"],
                                                                   basis="modal"), 3)):
        cfg = {key: v for key, v in cfg.items() if key != "k"}
        cfg["rhs"] = "none"
        prob = fegen.make(**cfg)
        B = torch.from_numpy(np.stack([prob.rhs("fourier", 1000 + j) for j in range(m)], axis=1)).cuda()
        S = g.Solver.from_problem(prob, device=True, cheb_degree=k, basis=1 if cfg.get("basis") == "modal" else 0)
        res = {}
        for prec, pkey in ((1, "mixed"), (0, "fp64")):
            for block, bkey in ((False, "independent"), (True, "block")):
                for _ in range(warmup):
                    S.solve_batch(B, rtol=1e-8, precision=prec, block=block)
                ts = []
                for _ in range(steps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    _, it, rr = S.solve_batch(B, rtol=1e-8, precision=prec, block=block)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                med = statistics.median(ts)
                res[f"{pkey}_{bkey}"] = {"ms": round(med, 2), "iters": int(it.max()),
                                         "ms_per_iter": round(med / max(int(it.max()), 1), 3),
                                         "max_relres": float(rr.max()), "status": S.last_status}
        S.close()
        out[name] = {"dofs": prob.n, "m": m, **res}
        prob.close()
    return out


def cpu_baseline(prob, k, rtol, sols, reps=3):
    """The oracle as it stands, on the host cores: full solves of the workload to rtol with the
    headline's method (FP32 V-cycle in FP64 flexible CG), the median of `reps` on all cores, then
    one on a single thread ("plain"; the fixed-block reductions make it bitwise equal); and the
    oracle's FP64 PCG, the reference the GPU solutions are compared with."""
    import oracle
    t0 = time.perf_counter()
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
    setup_ms = (time.perf_counter() - t0) * 1e3
    cores = oracle.num_threads()
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        x_all, iters, rr, _, st = H.solve(prob.b, rtol=rtol, precision=1)
        times.append((time.perf_counter() - t0) * 1e3)
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        x_one, iters_one, _, _, _ = H.solve(prob.b, rtol=rtol, precision=1)
        one = (time.perf_counter() - t0) * 1e3
    finally:
        oracle.set_num_threads(cores)
    err = oracle_errors(prob, k, prob.b, sols, rtol, H=H)
    H.close()
    cpu = {"value": round(pct(times, 0.5), 1), "unit": "ms", "cores": cores, "kind": "oracle",
           "sample": f"full oracle solves of the workload to rtol {rtol:g} ({iters} iterations, FP32 V-cycle in FP64 "
                     f"flexible CG): median of {reps} on all cores",
           "setup_ms": round(setup_ms, 1), "iters": iters,
           "plain": {"value": round(one, 1), "cores": 1, "sample": "one full solve on one thread",
                     "bitwise_equal_to_all_cores": x_all.tobytes() == x_one.tobytes() and iters == iters_one}}
    return cpu, err


def run_case(args):
    """Setup and a few solves of one case, nothing timed: the command a profiler wraps."""
    import numpy as np
    import torch
    import fegen
    import paper_2512_15121_gb300 as g
    if args.case in fegen.WORKLOADS:
        k = fegen.WORKLOADS[args.case]["k"]
        prob = fegen.workload(args.case)
    else:
        n, p, mesh, lam, k = args.case.split(",")
        prob = fegen.make(int(n), int(p), mesh=mesh, mesh_seed=1, lam=float(lam), rhs="fourier")
        k = int(k)
    S = g.Solver.from_problem(prob, device=True, cheb_degree=k)
    if args.rhs_columns == 1:
        b = torch.from_numpy(prob.b).cuda()
        for _ in range(args.solves):
            _, it, rr = S.solve(b, rtol=args.rtol, precision=args.precision)
    else:
        B = np.stack([prob.rhs("fourier", 1000 + j) for j in range(args.rhs_columns)], axis=1)
        Bd = torch.from_numpy(B).cuda()
        for _ in range(args.solves):
            _, its, rrs = S.solve_batch(Bd, rtol=args.rtol, precision=args.precision)
        it, rr = int(its.max()), float(rrs.max())
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "dofs": prob.n, "nnz": prob.nnz, "precision": args.precision,
                      "rhs_columns": args.rhs_columns, "iters": int(it), "relres": float(rr),
                      "kernels": {"fp64": S.kernel(0, 0), "fp32": S.kernel(0, 1)}}), flush=True)
    S.close()


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    if args.summarize_launches:
        print(summarize_launches(args.summarize_launches, args.split_at))
        return
    if args.block:
        print(json.dumps({"block": measure_block()}))
        return
    if args.schedules:
        print(json.dumps({"schedules": measure_schedules()}))
        return
    if args.serving_full:
        print(json.dumps({"serving_full": measure_serving_full(meshes=tuple(int(m) for m in args.serving_meshes.split(",")))}))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
