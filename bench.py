#!/usr/bin/env python3
"""Benchmark: GIAMG-PCG time to a 1e-8 relative residual on one GB300.

Workload (default): Helmholtz -lap u + 10 u = f on the unit cube, 16^3 hexahedra with interior
vertices jittered by +-0.2 h (seed 1), nodal GLL order 6: 912,673 dofs, 410,227,705 nonzeros
(FP64 CSR, 4.9 GB), manufactured right-hand side, Chebyshev degree 3, rtol 1e-8.  One step is one
full solve (all V-cycle levels, the outer CG) with inputs resident in HBM.  The headline is the
FP32 V-cycle inside FP64 flexible CG; the FP64 V-cycle in PCG is timed the same way beside it.

  python bench.py [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

`--impl reference` times the CPU oracle (plain FP64 C, OpenMP row loops) on the host cores with
the same metric: each step is one oracle CG iteration (one V-cycle and one product) scaled to the
oracle's iteration count.  Under torchrun every rank solves its own copy (replicas; no
collective on the data path) and rank 0 prints the line with the max over ranks.
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
                    help="run only the 512-request serving stream (36 operators up to 12^3, p = 8) and print it")
    ap.add_argument("--summarize-launches", metavar="CSV",
                    help="print a per-kernel summary of an ncu launch list and exit (no GPU work)")
    ap.add_argument("--split-at", metavar="KERNEL",
                    help="with --summarize-launches: also a table per segment starting at this kernel")
    return ap.parse_args()


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
    rank, ws, local, td = dist()
    if rank != 0:
        return
    import fegen
    import oracle
    k = fegen.WORKLOADS[args.workload]["k"]
    prob = fegen.workload(args.workload)
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
    # iterations to the tolerance (untimed), then bounded steps of one iteration each
    _, iters, _, _, st = H.solve(prob.b, rtol=args.rtol, precision=1)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        H.solve(prob.b, force_iters=1, precision=1)
        dt = (time.perf_counter() - t0) * 1e3
        if s >= args.warmup:
            times.append(dt * iters)
    cores = oracle.num_threads()
    p50 = pct(times, 0.5)
    line = {"metric": METRIC, "value": p50, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(times) / len(times), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle in f64 FCG (CPU oracle)",
            "data": "synthetic", "impl": "reference", "p99_ms": pct(times, 0.99), "iters": iters,
            "config": {"workload": args.workload, "description": WORKLOAD_TEXT.get(args.workload, ""),
                       "dofs": prob.n, "nnz": prob.nnz, "rtol": args.rtol, "cheb_degree": k},
            "cpu_baseline": {"value": p50, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": f"each step: one oracle CG iteration (1 V-cycle + 1 SpMV) on the full "
                                       f"workload, scaled by the oracle's {iters} iterations to rtol"},
            "e2e": {"value": p50, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ our arm
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

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = g.Solver.from_problem(prob, device=True, cheb_degree=k)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    levels = [S.level_info(l) for l in range(S.num_levels)]
    b = torch.from_numpy(prob.b).to(dev)
    x = torch.empty_like(b)

    def timed(precision, profiled):
        """K timed solves after W warm-ups.  profiled=False: the default path (the whole PCG loop as
        one CUDA graph).  profiled=True: per-kernel CUDA events by category, which need the
        host-driven loop (event records cannot sit inside the graph's conditional bodies): same
        kernels, same launch shapes; this pass gives the roofline's kernel times."""
        S.profile(False)
        for _ in range(args.warmup):
            S.solve(b, rtol=args.rtol, precision=precision, x=x)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
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
            _, it, rr = S.solve(b, rtol=args.rtol, precision=precision, x=x)
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

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = Clocks(uuid)
    mixed = timed(1, False)
    fp64 = timed(0, False)
    mixed_prof = timed(1, True)
    fp64_prof = timed(0, True)
    clk = clocks.stop()
    mixed["prof"], fp64["prof"] = mixed_prof["prof"], fp64_prof["prof"]

    # end to end through the C ABI with host buffers (pinned): H2D of b and D2H of x inside
    S.set_device_ptrs(False)
    bh = torch.from_numpy(prob.b).pin_memory()
    xh = torch.empty(prob.n, dtype=torch.float64).pin_memory()
    bh_np, xh_np = bh.numpy(), xh.numpy()
    e2e = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        S.solve(bh_np, rtol=args.rtol, precision=1, x=xh_np)
        dt = (time.perf_counter() - t0) * 1e3
        if s >= args.warmup:
            e2e.append(dt)
    S.set_device_ptrs(True)

    peak, peak_kind = measured_peaks()
    variant = {}
    for mode, prec in (("fp64", 0), ("mixed", 1)):
        tpr, form = S.kernel(0, prec)
        variant[mode] = f"{form} form, {tpr} threads per row"

    def roof(res, mode):
        ms, cnt, by = res["prof"][0]
        if cnt == 0 or ms <= 0:
            return None
        achieved = by / cnt / (ms / cnt * 1e-3) / 1e9
        tr = ncu_traffic(args.workload, mode)
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": tr,
                "kernel": f"finest-level row kernels ({'FP32' if mode == 'mixed' else 'FP64'} Chebyshev step and "
                          f"residual): {variant[mode]}",
                "launches": cnt, "avg_launch_ms": round(ms / cnt, 4),
                "algorithmic_bytes_per_launch": round(by / cnt), "peak_kind": peak_kind,
                "timed_region": "a second timed region of the same K solves with per-kernel CUDA events "
                                "(host-driven loop, same kernels and launch shapes)"}

    def roof_fp64(res):
        """The FP64 row kernels are bound by GB300's FP64 pipe (1/64 of the FP32 rate), not by HBM:
        2 flops per nonzero against the nominal 1.25 TFLOP/s FP64 peak (152 SMs x 2070 MHz x
        2 flops x 2 FP64 FMA per SM per clock; a probe kernel measured 1.204 TFLOP/s)."""
        hbm = roof(res, "fp64")
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
        # V-cycle bytes and time: every category except the outer CG product (5)
        ms = sum(res["prof"][c][0] for c in range(5))
        by = sum(res["prof"][c][2] for c in range(5))
        return round(by / (ms * 1e-3) / 1e9, 1) if ms > 0 else None

    extras = {}
    if not args.no_extras:
        from paper_2512_15121_gb300 import tune
        best_k, tk = tune.tune_cheb_degree(S, b, degrees=(1, 2, 3, 4, 5), precision=1, rtol=args.rtol)
        extras["cheb_degree_tuning"] = {"best": best_k, "paper_default": k,
                                        "ms": {t.degree: round(t.ms, 3) for t in tk},
                                        "iters": {t.degree: t.iterations for t in tk}}
        S.set_cheb_degree(k)
        extras.update({"batch": measure_batch(g, torch), "serving": measure_serving()})

    value = max_over_ranks(td, mixed["p50"])
    ms_per_step = max_over_ranks(td, mixed["wall"] / args.steps)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, k, args.rtol, mixed["iters"])
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle in f64 FCG",
        "data": "synthetic (seeded jittered-hex GLL assembly; stands in for the paper's Nektar++ matrices)",
        "config": {"workload": args.workload, "description": WORKLOAD_TEXT.get(args.workload, ""),
                   "dofs": prob.n, "nnz": prob.nnz, "rtol": args.rtol, "cheb_degree": k,
                   "levels": [(L["n"], L["nnz"], L["order"]) for L in levels],
                   "l2": f"inputs larger than L2 (finest matrix {12 * prob.nnz / 1e9:.2f} GB), no flush",
                   "parallelism": "replicas"},
        "p50_ms": round(mixed["p50"], 3), "p99_ms": round(mixed["p99"], 3), "iters": mixed["iters"],
        "true_relres": mixed["true_relres"],
        "fp64": {"p50_ms": round(fp64["p50"], 3), "p99_ms": round(fp64["p99"], 3), "iters": fp64["iters"],
                 "true_relres": fp64["true_relres"], "roofline": roof_fp64(fp64), "vcycle_gbs": vcycle_gbs(fp64)},
        "speedup_mixed_vs_fp64": round(fp64["p50"] / mixed["p50"], 3),
        "profiled_p50_ms": {"mixed": round(mixed_prof["p50"], 3), "fp64": round(fp64_prof["p50"], 3)},
        "vcycle_gbs": vcycle_gbs(mixed),
        "setup_ms": round(setup_ms, 1),
        "roofline": roof(mixed, "mixed"),
        "cpu_baseline": cpu,
        "e2e": {"value": round(pct(e2e, 0.5), 3), "unit": "ms", "h2d_bytes_per_step": 8 * prob.n,
                "d2h_bytes_per_step": 8 * prob.n},
        "gpu_launches": mixed["launches"],
        "clocks": clk,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    S.close()


def measure_batch(g, torch, m=32, reps=5):
    """32 right-hand sides of the 24^3 Poisson workload as one multi-RHS solve (FP32 V-cycle in
    flexible CG), against one single-RHS solve of the first column, and as one block in block
    CG."""
    import numpy as np
    import fegen
    name = "poisson_24cube_jitter_p4"
    prob = fegen.workload(name, rhs="none")
    B = np.stack([prob.rhs("fourier", 1000 + j) for j in range(m)], axis=1)
    S = g.Solver.from_problem(prob, device=True, cheb_degree=fegen.WORKLOADS[name]["k"])
    Bd = torch.from_numpy(B).cuda()
    b0 = Bd[:, 0].contiguous()
    for _ in range(2):
        S.solve_batch(Bd, rtol=1e-8, precision=1)
        S.solve(b0, rtol=1e-8, precision=1)
    for _ in range(2):
        S.solve_batch(Bd, rtol=1e-8, precision=1, block=True)
    st = torch.cuda.current_stream()
    tb, ts, tk = [], [], []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        X, it, rr = S.solve_batch(Bd, rtol=1e-8, precision=1)
        e1.record(st)
        torch.cuda.synchronize()
        tb.append(e0.elapsed_time(e1))
        e0.record(st)
        S.solve(b0, rtol=1e-8, precision=1)
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        e0.record(st)
        _, itk, rrk = S.solve_batch(Bd, rtol=1e-8, precision=1, block=True)
        e1.record(st)
        torch.cuda.synchronize()
        tk.append(e0.elapsed_time(e1))
    S.close()
    pb, ps, pk = pct(tb, 0.5), pct(ts, 0.5), pct(tk, 0.5)
    return {"workload": name, "dofs": prob.n, "nnz": prob.nnz, "m": m, "p50_ms": round(pb, 3),
            "per_solve_ms": round(pb / m, 3), "single_rhs_p50_ms": round(ps, 3),
            "throughput_vs_single": round(ps * m / pb, 2), "iters": [int(it.min()), int(it.max())],
            "max_relres": float(rr.max()), "dtype": "f32 V-cycle in f64 FCG",
            "block_cg": {"p50_ms": round(pk, 3), "iters": int(itk.max()), "max_relres": float(rrk.max())}}


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


def measure_serving_full(n_requests=512, load=0.8):
    """The larger serving stream: 512 requests on jittered 4^3 / 8^3 / 12^3 meshes, p in
    {2, 4, 6, 8}, lambda in {0, 1, 1000} (36 operators, up to 912,673 dofs and 7.97e8 nonzeros),
    1..8 right-hand sides (the seeded Fourier fields at the nodes).  First the capacity: every
    request submitted at once to a fresh server; then the same stream with Poisson arrivals at
    `load` times that capacity, again on a fresh server (setups included in both)."""
    import dataclasses
    from paper_2512_15121_gb300 import serve
    warm, _ = serve.synthetic_stream(16, seed=99, rate_per_s=1e6, meshes=(4,), orders=(2, 4, 8))
    w = serve.Server(slots=4)
    serve.run_stream(w, warm)
    w.close()
    t0 = time.perf_counter()
    # arrival offsets for rate 1/s; run_stream scales them by time_scale = 1 / rate
    reqs, ops = serve.synthetic_stream(n_requests, seed=7, rate_per_s=1.0, meshes=(4, 8, 12), orders=(2, 4, 6, 8),
                                       lambdas=(0.0, 1.0, 1000.0), rhs_kind="nodal")
    gen_s = time.perf_counter() - t0
    offsets = [r.arrival for r in reqs]
    cols = sum(r.columns for r in reqs)

    def run(time_scale):
        rs = [dataclasses.replace(r, arrival=off) for r, off in zip(reqs, offsets)]
        srv = serve.Server(slots=4)
        st = serve.run_stream(srv, rs, time_scale=time_scale)
        srv.close()
        st.update({k: int(v) for k, v in srv.stats.items()})
        st["errors"] = sum(r.error is not None for r in rs)
        return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()}

    cap = run(0.0)
    capacity = cap["solves_per_s"]
    rate = load * capacity * n_requests / cols  # requests per second
    loaded = run(1.0 / rate)
    loaded["rate_per_s"] = round(rate, 2)
    return {"requests": n_requests, "solves": cols, "operators": len(ops), "generation_s": round(gen_s, 1),
            "mix": "jittered 4^3/8^3/12^3, p in {2,4,6,8}, lambda in {0,1,1000}, 1-8 nodal Fourier RHS, FP32 V-cycle",
            "capacity": cap, f"at_{load}x_capacity": loaded}


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


def cpu_baseline(prob, k, rtol, iters):
    """The oracle as it stands, on the host cores: two CG iterations (FP32 V-cycle, flexible CG)
    on the full workload, scaled to the GPU's iteration count; then the same two iterations on
    one thread ("plain"), which the fixed-block reductions make bitwise equal."""
    import oracle
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    x_all = H.solve(prob.b, force_iters=2, precision=1)[0]
    per_iter = (time.perf_counter() - t0) * 1e3 / 2
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        x_one = H.solve(prob.b, force_iters=2, precision=1)[0]
        per_iter_one = (time.perf_counter() - t0) * 1e3 / 2
    finally:
        oracle.set_num_threads(cores)
    H.close()
    return {"value": round(per_iter * iters, 1), "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": f"2 oracle CG iterations (FP32 V-cycle in FP64 flexible CG) on the full workload, "
                      f"scaled to {iters} iterations",
            "plain": {"value": round(per_iter_one * iters, 1), "cores": 1,
                      "bitwise_equal_to_all_cores": x_all.tobytes() == x_one.tobytes()}}


def main():
    args = parse()
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
        print(json.dumps({"serving_full": measure_serving_full()}))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
