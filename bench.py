"""Benchmark of the triangular tensor Sylvester solver on one GB300 (or N replicas).

Workload (default): d = 3, n = 256^3, FP64, coefficients and right-hand side
drawn by synthetic.py (seed 0): one step = one FP64 solve of the Laplace form
(Eq. (2.2)) and one FP64 solve of the d-term generalized form, both through the
C ABI on device-resident inputs; plus, when the library provides them, the
mixed-precision refined solves of the same two problems to
||B - A(X)|| / (||A|| ||X||) <= 1e-12.

Prints one JSON line (rank 0).  `value` = unknowns solved per second over the
whole step (all ranks).  `--impl reference` times the CPU oracle on a bounded
sample of the same workload instead.

Under torchrun (N > 1) every rank solves its own replica (the solve of one
equation does not shard; there is no collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak measured on this machine's GB300 (DMMA m8n8k4 loop, 152 SMs; DFMA
# 1.06, cuBLAS DGEMM 1.10): see profiles/fp64_peak_probe.txt
FP64_PEAK_TFLOPS = 1.10


def algorithmic_flops(A, C=None):
    """Flops of one solve counted on the operator's off-diagonal structure.

    Laplace form: every off-diagonal nonzero of the assembled Kronecker-sum
    operator is used exactly once (2 flops) plus one division per unknown:
    F = 2 sum_mu (N / n_mu) offnnz(A_mu) + N.
    Generalized d-term form: the Horner recurrence over the modes (level d: one
    C and one A product; levels d-1..2: two C and one A product; level 1: one C
    and one A product), each product using the strictly-upper structure of its
    factor once per fiber, plus one division per unknown.
    """
    shape = [a.shape[0] for a in A]
    N = float(np.prod(shape))

    def off(M, quasi):
        n = M.shape[0]
        nnz = n * (n - 1) / 2
        if quasi:
            nnz += int(np.count_nonzero(np.diag(M, -1)))
        return nnz

    d = len(shape)
    if C is None:
        return sum(2 * N / shape[mu] * off(A[mu], True) for mu in range(d)) + N
    f = 0.0
    for mu in range(d):
        nC = 1 if mu in (0, d - 1) else 2
        f += 2 * N / shape[mu] * (nC * off(C[mu], False) + off(A[mu], True))
    return f + N


class ClockSampler:
    """nvidia-smi samples of SM clock / throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        loaded = sorted(sm)[len(sm) // 4:] if len(sm) > 4 else sm
        return {"sm_mhz": float(np.median(loaded)) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons), "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(v, ws, device):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, ws, device):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------- CPU oracle

def oracle_sample(shape_lap, shape_gen, full_shape, seed=0):
    """Time the oracle (O-B recursion, single thread) on bounded samples and
    scale to the full workload by the algorithmic-flop ratio."""
    import oracle
    import synthetic
    out = {}
    t_full = 0.0
    for gen, shape in ((False, shape_lap), (True, shape_gen)):
        p = synthetic.problem(seed, shape, generalized=gen)
        t0 = time.perf_counter()
        oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=8)
        dt = time.perf_counter() - t0
        # flop ratio with the full-size counts (structure-independent leading terms)
        fs = algorithmic_flops(p["A"], p["C"])
        Nf = float(np.prod(full_shape))
        if gen:
            ff = sum(2 * Nf / n * (((1 if mu in (0, len(full_shape) - 1) else 2) * n * (n - 1) / 2) +
                                   n * (n - 1) / 2) for mu, n in enumerate(full_shape)) + Nf
        else:
            ff = sum(2 * Nf / n * n * (n - 1) / 2 for n in full_shape) + Nf
        t_full += dt * ff / fs
        out["gen" if gen else "laplace"] = {"shape": list(shape), "seconds": dt}
    return t_full, out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    full = (256, 256, 256)
    N = float(np.prod(full))
    times = []
    for it in range(args.warmup + args.steps):
        t_full, parts = oracle_sample((96, 96, 96), (64, 64, 64), full, seed=it % 3)
        if it >= args.warmup:
            times.append(t_full)
    # the oracle solves each of the four parts of a step (FP64 and refined,
    # Laplace and generalized) in FP64: two Laplace and two generalized solves
    step = 2 * float(np.mean(times))
    value = 4 * N / step
    line = {
        "impl": "reference",
        "metric": "unknowns/s (d=3 256^3, Laplace + generalized, FP64 and FP32-refined to rel. residual <= 1e-12); "
                  "% of FP64 peak; mixed-precision vs FP64 speed-up",
        "value": value, "unit": "unknowns/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (synthetic.py, seed 0..2)",
        "config": {"workload": "d=3 n=256^3: FP64 solve and FP32-refined solve, Laplace + generalized form",
                   "form": ["laplace", "generalized"],
                   "sample": "oracle O-B on 96^3 (Laplace) + 64^3 (generalized), scaled by algorithmic flops"},
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                         "sample": "O-B recursion, 96^3 Laplace + 64^3 generalized per step (each solved twice: the "
                                   "FP64 and the refined part), time scaled to 256^3 by the algorithmic-flop ratio"},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU path

def run_ours(args, ws, rank, local):
    import torch
    import paper_1905_09539_gb300 as ts
    import synthetic
    from paper_1905_09539_gb300 import _lib
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ts.load()
    shape = (args.n, args.n, args.n)
    N = float(np.prod(shape))

    def to_dev(a):
        a = np.asfortranarray(a)
        t = torch.from_numpy(a)
        out = torch.empty_strided(t.shape, t.stride(), dtype=torch.float64, device=dev)
        out.copy_(t)
        return out

    probs = {}
    for gen in (False, True):
        p = synthetic.problem(args.seed + rank, shape, generalized=gen)
        probs[gen] = {
            "np": p,
            "A": [to_dev(a) for a in p["A"]],
            "C": [to_dev(c) for c in p["C"]] if gen else None,
            "B": to_dev(p["B"]),
            "X": ts.empty_fortran(shape, dev),
            "flops": algorithmic_flops(p["A"], p["C"]),
        }
    stream = torch.cuda.current_stream(dev)
    PARTS = [("fp64_laplace", False, _lib.TSYLV_FP64), ("fp64_generalized", True, _lib.TSYLV_FP64),
             ("fp32r_laplace", False, _lib.TSYLV_FP32_REFINED), ("fp32r_generalized", True, _lib.TSYLV_FP32_REFINED)]
    infos = {name: _lib.Info() for name, _, _ in PARTS}
    for gen in (False, True):
        probs[gen]["Xr"] = ts.empty_fortran(shape, dev)

    def solve(name, gen, prec, timing=0):
        pr = probs[gen]
        X = pr["X"] if prec == _lib.TSYLV_FP64 else pr["Xr"]
        if gen:
            ts.gtsylv_solve(pr["A"], pr["C"], pr["B"], X=X, info=infos[name], timing=timing, precision=prec)
        else:
            ts.tsylv_solve(pr["A"], pr["B"], X=X, info=infos[name], timing=timing, precision=prec)

    def step(timing=0):
        for name, gen, prec in PARTS:
            solve(name, gen, prec, timing)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # ---- device-resident timed region
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            step()
            launches += sum(infos[name].launches for name, _, _ in PARTS)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(ws)
    clocks = clk.summary()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, ws, dev)
    units = sum_over_ranks(len(PARTS) * N, ws, dev)
    value = units / (ms * 1e-3)

    # ---- per-solve timing (CUDA events recorded on the launching stream inside
    # the captured graphs: whole call, wavefront launches, residual launches)
    tim = {name: {"tot": [], "wave": [], "res": []} for name, _, _ in PARTS}
    for _ in range(max(3, args.steps)):
        for name, gen, prec in PARTS:
            solve(name, gen, prec, timing=1)
            tim[name]["tot"].append(infos[name].t_total_ms)
            tim[name]["wave"].append(infos[name].t_waves_ms)
            tim[name]["res"].append(infos[name].t_resid_ms)
    # residual of every result, measured independently of the solve with the
    # library's FP64-pipe residual
    parts = {}
    for name, gen, prec in PARTS:
        pr = probs[gen]
        X = pr["X"] if prec == _lib.TSYLV_FP64 else pr["Xr"]
        _, rho, _ = ts.tsylv_residual(pr["A"], pr["B"], X, pr["C"], residual=_lib.TSYLV_RESID_FP64)
        f = pr["flops"]
        tm = float(np.median(tim[name]["tot"]))
        parts[name] = {
            "ms": tm, "wave_ms": float(np.median(tim[name]["wave"])), "resid_ms": float(np.median(tim[name]["res"])),
            "iterations": infos[name].iterations, "rel_residual_fp64": rho, "waves": infos[name].waves,
            "tiles": infos[name].tiles, "unknowns_per_s": N / (tm * 1e-3),
        }
        if prec == _lib.TSYLV_FP64:
            parts[name].update({"algorithmic_gflop": f / 1e9, "executed_gflop": infos[name].flops / 1e9,
                                "tflops_algorithmic": f / (tm * 1e-3) / 1e12,
                                "frac_fp64_peak": f / (tm * 1e-3) / 1e12 / FP64_PEAK_TFLOPS})
    mixed_vs_fp64 = {"laplace": parts["fp64_laplace"]["ms"] / parts["fp32r_laplace"]["ms"],
                     "generalized": parts["fp64_generalized"]["ms"] / parts["fp32r_generalized"]["ms"]}
    dom = "fp64_generalized"  # the generalized FP64 wavefront kernel carries most of the step
    f_dom = probs[True]["flops"]
    w_dom = parts[dom]["wave_ms"]
    nwaves = parts[dom]["waves"]
    achieved = (f_dom / nwaves) / (w_dom * 1e-3 / nwaves) / 1e12
    roofline = {"bound": "alu", "kernel": "k_wave<double,3,generalized>", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": None,
                "peak_source": "measured FP64 DMMA/DFMA probe on this GB300 (MEASURED_PEAKS.json has no FP64 "
                               "entry; bf16 1956.8 x 1.25/2250 nominal ratio gives 1.09)",
                "per_launch_gflop": f_dom / nwaves / 1e9, "per_launch_ms": w_dom / nwaves}

    # ---- end to end: pinned host buffers, H2D + solve + D2H inside the timed region
    host = {}
    h2d = d2h = 0
    for gen in (False, True):
        pr = probs[gen]
        hb = torch.empty(pr["B"].shape[::-1], dtype=torch.float64).pin_memory().permute(2, 1, 0)
        hb.copy_(pr["B"])
        hA = [a.cpu().pin_memory() for a in pr["A"]]
        hC = [c.cpu().pin_memory() for c in pr["C"]] if gen else None
        hx = torch.empty(pr["B"].shape[::-1], dtype=torch.float64).pin_memory().permute(2, 1, 0)
        host[gen] = (hb, hA, hC, hx)
    for name, gen, prec in PARTS:
        hb, hA, hC, hx = host[gen]
        h2d += hb.numel() * 8 + sum(a.numel() * 8 for a in hA) + (sum(c.numel() * 8 for c in hC) if gen else 0)
        d2h += hx.numel() * 8
    barrier(ws)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.steps):
        for name, gen, prec in PARTS:
            pr = probs[gen]
            hb, hA, hC, hx = host[gen]
            pr["B"].copy_(hb, non_blocking=True)
            for a, h in zip(pr["A"], hA):
                a.copy_(h, non_blocking=True)
            if gen:
                for c, h in zip(pr["C"], hC):
                    c.copy_(h, non_blocking=True)
            solve(name, gen, prec)
            hx.copy_(pr["X"] if prec == _lib.TSYLV_FP64 else pr["Xr"], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws, dev)

    line = {
        "metric": "unknowns/s (d=3 256^3, Laplace + generalized, FP64 and FP32-refined to rel. residual <= 1e-12); "
                  "% of FP64 peak; mixed-precision vs FP64 speed-up",
        "value": value, "unit": "unknowns/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (synthetic.py, seed %d)" % args.seed,
        "config": {"workload": "d=3 n=%d^3: FP64 solve and FP32-refined solve, Laplace + generalized form" % args.n,
                   "form": ["laplace", "generalized"], "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (%.0f MB per tensor)" % (N * 8 / 1e6)},
        "parts": parts,
        "mixed_vs_fp64": mixed_vs_fp64,
        "roofline": roofline,
        "e2e": {"value": sum_over_ranks(len(PARTS) * N, ws, dev) / (e2e_ms * 1e-3), "unit": "unknowns/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu:
        t_full, samp = oracle_sample((128, 128, 128), (96, 96, 96), shape, seed=args.seed)
        line["cpu_baseline"] = {"value": 4 * N / (2 * t_full), "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                                "sample": "O-B recursion on 128^3 (Laplace, %.1f s) + 96^3 (generalized, %.1f s), "
                                          "time scaled to %d^3 by the algorithmic-flop ratio" %
                                          (samp["laplace"]["seconds"], samp["gen"]["seconds"], args.n)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
