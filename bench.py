"""Benchmark of the triangular tensor Sylvester solver on one GB300 (or N replicas).

One step is one pass of the whole hot path on synthetic inputs (synthetic.py,
seed 0), every call through the C ABI on device-resident inputs:
  * d = 3, n = 256^3: FP64 solve and FP32-refined solve (to
    ||B - A(X)|| / (||A|| ||X||) <= 1e-12) of the Laplace form (Eq. (2.2)) and
    of the d-term generalized form;
  * d = 3, n = (200, 160, 120), Laplace form: forward solve + adjoint (transposed
    solve, masked dA) of L = 0.5 ||X - X*||^2, FP64 and FP32-refined;
  * 512 independent d = 3 Laplace equations, n_mu ~ U{8..48}: one batched
    persistent solve (FP64).
Prints one JSON line (rank 0).  `value` = unknowns solved per second over the
whole step (all ranks; a forward + adjoint pass counts two solves).
`--impl reference` times the CPU oracle on bounded samples of the same step;
`--fp64-peak` builds and runs the FP64 throughput probe (bench_fp64_peak.cu).

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
# FP64 peak measured on this GB300 model (DMMA m8n8k4 loop over 152 SMs;
# DFMA 1.06, cuBLAS DGEMM 1.10): `python bench.py --fp64-peak`
FP64_PEAK_TFLOPS = 1.10
# DRAM bytes (read + write) per launch of the dominant kernel (one FP64 solve of
# the 256^3 generalized form) from an ncu capture of the current kernel:
# 10.531 GB read + 0.842 GB written (the capture is summarised under profiles/)
TRAFFIC_PER_LAUNCH_BYTES = 11.373e9


def bf16_peak_measured():
    """Dense bf16 burst TFLOP/s of MEASURED_PEAKS.json (the fallback figure when absent)."""
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        return 1900.0


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


# ----------------------------------------------------------------- workload

SOLVE_PARTS = [("fp64_laplace", False, 0), ("fp64_generalized", True, 0),
               ("fp32r_laplace", False, 1), ("fp32r_generalized", True, 1)]
ADJ_SHAPE = (200, 160, 120)
D4_SHAPES = ((64, 64, 64, 64), (128, 96, 64, 32))
BATCH = dict(count=512, lo=8, hi=48)


def laplace_flops_dense(shape):
    """Leading-term algorithmic flops of one Laplace solve (no 2x2 blocks)."""
    N = float(np.prod(shape))
    return sum(2 * N / n * n * (n - 1) / 2 for n in shape) + N


def gen_flops_dense(shape):
    N = float(np.prod(shape))
    d = len(shape)
    return sum(2 * N / n * ((1 if mu in (0, d - 1) else 2) * n * (n - 1) / 2 + n * (n - 1) / 2)
               for mu, n in enumerate(shape)) + N


def grad_flops(shape):
    """Flops of the masked contractions dA_mu (Laplace form): 2 n_mu N each (upper half used)."""
    N = float(np.prod(shape))
    return sum(N * n for n in shape)


# ----------------------------------------------------------------- CPU oracle

def _batch_worker(args):
    """One batch equation solved by the oracle in a worker process ('spawn'; one thread)."""
    import oracle
    import synthetic
    seed, e, shape = args
    q = synthetic.problem([seed, 1 + e], shape)
    t0 = time.perf_counter()
    oracle.solve_recursive(q["A"], q["B"], None, nmin=8)
    return time.perf_counter() - t0


# The sampling rule of the CPU oracle, one rule for the reference arm and for
# the cpu_baseline object of the GPU arm.  A 256^3 generalized solve takes the
# oracle about three minutes, so the two 256^3 parts are timed on a 128^3
# sample of the same distributions and scaled by the ratio of algorithmic
# flops (every off-diagonal entry of the update blocks once): checked against
# full 256^3 runs on an x86 host, 1.07 s -> 17.2 s predicted vs 17.6 s run
# (Laplace), 10.5 s -> 171 s vs 180 s (generalized).  The adjoint workload
# (200,160,120) and the 512-equation batch run in full.  The oracle is serial
# C: a single solve uses one core (its recursion is a chain of dependent
# steps); with more than one core the batch's independent equations are
# spread over worker processes, one core each.
ORACLE_PARTS = ("laplace", "generalized", "adjoint", "batched")
ORACLE_SAMPLE = (128, 128, 128)
_FULL_FLOPS = {}


def oracle_part_seconds(part, threads, seed=0):
    """Oracle seconds of one part of the bench step (FP64 and refined parts
    counted), by the rule above, on `threads` host cores."""
    import multiprocessing
    import oracle
    import synthetic
    used = threads if threads > 0 else (os.cpu_count() or 1)
    if part in ("laplace", "generalized"):
        gen = part == "generalized"
        if gen not in _FULL_FLOPS:
            q = synthetic.problem(seed, (256, 256, 256), generalized=gen)
            _FULL_FLOPS[gen] = algorithmic_flops(q["A"], q["C"])
        p = synthetic.problem(seed, ORACLE_SAMPLE, generalized=gen)
        t0 = time.perf_counter()
        oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=8)
        dt = time.perf_counter() - t0
        pred = dt * _FULL_FLOPS[gen] / algorithmic_flops(p["A"], p["C"])
        return 2 * pred, {"sample": list(ORACLE_SAMPLE), "sample_s": dt, "predicted_256_s": pred, "cores": 1}
    if part == "adjoint":
        p = synthetic.problem(seed, ADJ_SHAPE)
        t0 = time.perf_counter()
        X = oracle.solve_recursive(p["A"], p["B"], None, nmin=8)
        t_fwd = time.perf_counter() - t0
        Lam = oracle.solve_recursive(p["A"], X - p["Xstar"], None, nmin=8, transpose=True)
        oracle.grad(p["A"], X, Lam)
        dt = time.perf_counter() - t0
        return 2 * dt, {"shape": list(ADJ_SHAPE), "seconds": dt, "forward_s": t_fwd, "cores": 1}
    shapes = synthetic.batch_shapes(seed, BATCH["count"], BATCH["lo"], BATCH["hi"])
    jobs = [(seed, e, s) for e, s in enumerate(shapes)]
    t0 = time.perf_counter()
    if used <= 1:
        for j in jobs:
            _batch_worker(j)
    else:  # the equations spread over the threads, one thread each
        with multiprocessing.get_context("spawn").Pool(used) as pool:
            pool.map(_batch_worker, jobs, chunksize=8)
    dt = time.perf_counter() - t0
    return dt, {"equations": len(jobs), "seconds": dt, "processes": used}


def oracle_step_seconds(threads, seed=0):
    """Oracle seconds of one whole bench step (every part), and the details."""
    total, det = 0.0, {}
    for part in ORACLE_PARTS:
        t, det[part] = oracle_part_seconds(part, threads, seed)
        total += t
    det["threads"] = threads if threads > 0 else (os.cpu_count() or 1)
    return total, det


ORACLE_RULE = ("oracle O-B (serial C, -O3, FP64) on the host: the 256^3 Laplace and generalized solves timed on "
               "128^3 samples and scaled by the algorithmic-flop ratio, each counted for the FP64 and the refined "
               "part; the (200,160,120) forward solve + transposed solve + gradient run in full (counted for both "
               "adjoint parts); the 512 batch equations run in full, spread over worker processes (one core each)")


def step_units():
    """Unknowns solved per step (a forward + adjoint pass counts two solves)."""
    import synthetic
    N = 256.0 ** 3
    Na = float(np.prod(ADJ_SHAPE))
    Nb = float(sum(np.prod(s) for s in synthetic.batch_shapes(0, BATCH["count"], BATCH["lo"], BATCH["hi"])))
    return {"solves_256": 4 * N, "adjoint": 2 * 2 * Na, "batched": Nb}


METRIC = ("unknowns/s (one step: d=3 256^3 Laplace + generalized, FP64 and FP32-refined to rel. residual <= 1e-12; "
          "(200,160,120) forward + adjoint, FP64 and FP32-refined; 512-equation batch FP64); % of FP64 peak; "
          "mixed-precision vs FP64 speed-up")
WORKLOAD = ("d=3: 256^3 FP64 and FP32-refined solves (Laplace + generalized); (200,160,120) Laplace forward + "
            "adjoint (FP64, FP32-refined); 512 Laplace equations n_mu~U{8..48} batched (FP64)")


def run_reference(args, ws, rank):
    """The oracle under the sampling rule above, on all host cores.  Each
    iteration times one part of the step, the parts in rotation, so that an
    iteration is a bounded sample; a step's time is the sum of the parts'
    mean timed samples (parts without a timed sample, when there are fewer
    timed iterations than parts, are timed once more after the loop)."""
    if rank != 0:
        return
    units = sum(step_units().values())
    timed = {p: [] for p in ORACLE_PARTS}
    det = {}
    threads = os.cpu_count() or 1
    for it in range(args.warmup + args.steps):
        part = ORACLE_PARTS[it % len(ORACLE_PARTS)]
        t, det[part] = oracle_part_seconds(part, 0, seed=0)
        if it >= args.warmup:
            timed[part].append(t)
    for part in ORACLE_PARTS:
        if not timed[part]:
            t, det[part] = oracle_part_seconds(part, 0, seed=0)
            timed[part].append(t)
    step = float(sum(np.mean(v) for v in timed.values()))
    value = units / step
    sample = ORACLE_RULE + "; %d host cores; one part per iteration, in rotation" % threads
    line = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "unknowns/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (synthetic.py, seed 0)",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": threads, "kind": "oracle",
                         "sample": sample, "detail": det},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_fp64_peak():
    """Build and run the FP64 throughput probe; print its JSON lines."""
    import shutil
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out_dir = os.path.join(ROOT, "paper_1905_09539_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "fp64_peak")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(ROOT, "bench_fp64_peak.cu")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    sys.stdout.write(r.stdout)
    try:
        import torch
        a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
        b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        best = 1e30
        for _ in range(3):
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        print(json.dumps({"kernel": "cublas_dgemm_4096", "tflops": 2 * 4096 ** 3 / (best * 1e-3) / 1e12}))
    except Exception as ex:  # the probe above is the measurement; the DGEMM line is context
        print(json.dumps({"kernel": "cublas_dgemm_4096", "error": str(ex)}))
    sys.exit(r.returncode)


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
    PREC = {0: _lib.TSYLV_FP64, 1: _lib.TSYLV_FP32_REFINED, 2: _lib.TSYLV_TF32_REFINED, 3: _lib.TSYLV_BF16_REFINED,
            4: _lib.TSYLV_DF64}
    PNAME = {0: "fp64", 1: "fp32r", 2: "tf32r", 3: "bf16r", 4: "df64"}

    def to_dev(a):
        a = np.asfortranarray(a)
        t = torch.from_numpy(a)
        out = torch.empty_strided(t.shape, t.stride(), dtype=torch.float64, device=dev)
        out.copy_(t)
        return out

    # ---- inputs (device resident)
    probs = {}
    for gen in (False, True):
        p = synthetic.problem(args.seed + rank, shape, generalized=gen)
        probs[gen] = {
            "A": [to_dev(a) for a in p["A"]],
            "C": [to_dev(c) for c in p["C"]] if gen else None,
            "B": to_dev(p["B"]),
            "X": {0: ts.empty_fortran(shape, dev), 1: ts.empty_fortran(shape, dev)},
            "flops": algorithmic_flops(p["A"], p["C"]),
        }
    pa = synthetic.problem(args.seed + rank, ADJ_SHAPE)
    adj = {"A": [to_dev(a) for a in pa["A"]], "B": to_dev(pa["B"]), "Xs": to_dev(pa["Xstar"]),
           "X": {0: ts.empty_fortran(ADJ_SHAPE, dev), 1: ts.empty_fortran(ADJ_SHAPE, dev)}, "out": {}}
    bps = synthetic.batch(args.seed + rank, **BATCH)
    pools = ts.BatchPools([([to_dev(a) for a in q["A"]], to_dev(q["B"])) for q in bps])
    stream = torch.cuda.current_stream(dev)
    infos = {name: _lib.Info() for name, _, _ in SOLVE_PARTS}
    infos.update({"adjoint_fp64_fwd": _lib.Info(), "adjoint_fp64_bwd": _lib.Info(),
                  "adjoint_fp32r_fwd": _lib.Info(), "adjoint_fp32r_bwd": _lib.Info(), "batched_fp64": _lib.Info()})

    def solve(name, gen, prec, timing=0):
        pr = probs[gen]
        if gen:
            ts.gtsylv_solve(pr["A"], pr["C"], pr["B"], X=pr["X"][prec], info=infos[name], timing=timing,
                            precision=PREC[prec])
        else:
            ts.tsylv_solve(pr["A"], pr["B"], X=pr["X"][prec], info=infos[name], timing=timing, precision=PREC[prec])

    def adjoint(prec):
        tag = "adjoint_fp64" if prec == 0 else "adjoint_fp32r"
        X = adj["X"][prec]
        ts.tsylv_solve(adj["A"], adj["B"], X=X, info=infos[tag + "_fwd"], precision=PREC[prec])
        # dL/dX of L = 0.5 ||X - X*||^2 (one elementwise torch op: marshalling of the loss, not the path)
        dX = X - adj["Xs"]
        adj["out"][prec] = ts.tsylv_backward(adj["A"], X, dX, want_dB=True, want_dA=True,
                                             info=infos[tag + "_bwd"], precision=PREC[prec])

    def batched():
        pools.solve(info=infos["batched_fp64"])

    def step():
        for name, gen, prec in SOLVE_PARTS:
            solve(name, gen, prec)
        adjoint(0)
        adjoint(1)
        batched()

    def launches_of_step():
        return sum(i.launches for i in infos.values())

    if args.only:
        table = {name: (lambda name=name, gen=gen, prec=prec: solve(name, gen, prec)) for name, gen, prec in SOLVE_PARTS}
        table.update({"adjoint_fp64": lambda: adjoint(0), "adjoint_fp32r": lambda: adjoint(1), "batched_fp64": batched})
        for prec in (2, 3, 4):
            for gen in (False, True):
                pr = probs[gen]
                pr["X"][prec] = ts.empty_fortran(shape, dev)
                name = "%s_%s" % (PNAME[prec], "generalized" if gen else "laplace")
                infos[name] = _lib.Info()
                table[name] = (lambda gen=gen, prec=prec, name=name: solve(name, gen, prec))
        if args.only.startswith("complex_"):
            # the complex-triangular variant at the bench's size (FP64)
            zgen = args.only == "complex_dterm"
            zq = synthetic.complex_problem(args.seed + rank, shape, generalized=zgen)
            zt = lambda a: torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to(dev).T
            zA = [zt(a) for a in zq["A"]]
            zC = [zt(c) for c in zq["C"]] if zgen else None
            zB = torch.from_numpy(np.ascontiguousarray(zq["B"].transpose(2, 1, 0))).to(dev).permute(2, 1, 0)
            zX = ts.empty_fortran(shape, dev, torch.complex128)
            table[args.only] = lambda: ts.ztsylv_solve(zA, zB, zC, X=zX)
        fn = table[args.only]
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"only": args.only, "ms": e0.elapsed_time(e1) / max(1, args.steps)}), flush=True)
        return

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
            launches += launches_of_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(ws)
    clocks = clk.summary()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, ws, dev)
    units_rank = step_units()
    units = sum_over_ranks(sum(units_rank.values()), ws, dev)
    value = units / (ms * 1e-3)

    # ---- per-part timing: solves with the calls' own CUDA events (recorded on
    # the launching stream inside the captured graphs); adjoint and batch with
    # events around the calls
    tim = {name: {"tot": [], "wave": [], "res": []} for name, _, _ in SOLVE_PARTS}
    for _ in range(max(3, args.steps)):
        for name, gen, prec in SOLVE_PARTS:
            solve(name, gen, prec, timing=1)
            tim[name]["tot"].append(infos[name].t_total_ms)
            tim[name]["wave"].append(infos[name].t_waves_ms)
            tim[name]["res"].append(infos[name].t_resid_ms)

    def event_ms(fn, reps):
        out = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))

    parts = {}
    for name, gen, prec in SOLVE_PARTS:
        pr = probs[gen]
        _, rho, _ = ts.tsylv_residual(pr["A"], pr["B"], pr["X"][prec], pr["C"], residual=_lib.TSYLV_RESID_FP64)
        f = pr["flops"]
        tm = float(np.median(tim[name]["tot"]))
        parts[name] = {
            "ms": tm, "wave_ms": float(np.median(tim[name]["wave"])), "resid_ms": float(np.median(tim[name]["res"])),
            "iterations": infos[name].iterations, "rel_residual_fp64": rho, "waves": infos[name].waves,
            "tiles": infos[name].tiles, "unknowns_per_s": N / (tm * 1e-3),
        }
        if prec == 0:
            parts[name].update({"algorithmic_gflop": f / 1e9, "executed_gflop": infos[name].flops / 1e9,
                                "tflops_algorithmic": f / (tm * 1e-3) / 1e12,
                                "frac_fp64_peak": f / (tm * 1e-3) / 1e12 / FP64_PEAK_TFLOPS})
    Na = float(np.prod(ADJ_SHAPE))
    fa = 2 * algorithmic_flops([a.cpu().numpy() for a in adj["A"]]) + grad_flops(ADJ_SHAPE)
    for prec in (0, 1):
        tag = "adjoint_fp64" if prec == 0 else "adjoint_fp32r"
        tm = event_ms(lambda: adjoint(prec), max(3, args.steps))
        dB, dA, _ = adj["out"][prec]
        dB0, dA0, _ = adj["out"][0]
        parts[tag] = {"ms": tm, "unknowns_per_s": 2 * Na / (tm * 1e-3), "algorithmic_gflop": fa / 1e9,
                      "tflops_algorithmic": fa / (tm * 1e-3) / 1e12,
                      "iterations_fwd_bwd": [infos[tag + "_fwd"].iterations, infos[tag + "_bwd"].iterations]}
        if prec == 1:
            parts[tag]["rel_diff_vs_fp64"] = {
                "dB": float(torch.linalg.vector_norm(dB - dB0) / torch.linalg.vector_norm(dB0)),
                "dA": max(float(torch.linalg.matrix_norm(a - b) / torch.linalg.matrix_norm(b)) for a, b in zip(dA, dA0))}
    tb = event_ms(batched, max(3, args.steps))
    ib = infos["batched_fp64"]
    parts["batched_fp64"] = {"ms": tb, "unknowns_per_s": units_rank["batched"] / (tb * 1e-3), "equations": pools.count,
                             "unknowns": pools.unknowns, "tiles": ib.tiles, "max_waves": ib.waves,
                             "queue_order": ib.batch_order, "ctas_per_sm": ib.batch_ctas_per_sm,
                             "tile_shape": list(ib.leaf[:3])}
    mixed_vs_fp64 = {"laplace": parts["fp64_laplace"]["ms"] / parts["fp32r_laplace"]["ms"],
                     "generalized": parts["fp64_generalized"]["ms"] / parts["fp32r_generalized"]["ms"]}

    # the dominant kernel: the persistent FP64 solve of the generalized form,
    # one launch per solve; its duration is taken with CUDA events recorded on
    # the launching stream around the launch inside the captured graph
    dom = "fp64_generalized"
    f_dom = probs[True]["flops"]
    w_dom = parts[dom]["wave_ms"]
    achieved = f_dom / (w_dom * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_batched<double,3,generalized> (persistent FP64 solve, 1 launch/solve)",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": TRAFFIC_PER_LAUNCH_BYTES,
                "peak_source": "of measured: FP64 DMMA/DFMA probe on this GB300 (bench_fp64_peak.cu); "
                               "MEASURED_PEAKS.json has no FP64 entry (its bf16 burst x 1.25/2250 gives %.2f)"
                               % (bf16_peak_measured() * 1.25 / 2250),
                "per_launch_gflop": f_dom / 1e9, "per_launch_ms": w_dom,
                "dram_gbs_from_traffic": (TRAFFIC_PER_LAUNCH_BYTES / 1e9 / (w_dom * 1e-3)
                                          if TRAFFIC_PER_LAUNCH_BYTES else None)}

    # ---- end to end through the public API: pinned host buffers, H2D of every
    # input and D2H of every result inside the timed region.  The copies run on
    # a copy stream, overlapped with the solves of the other parts (every part
    # has its own device inputs and outputs; events order each copy against
    # the solve that produces or consumes its buffer)
    rev = lambda t: t.permute(*range(t.dim() - 1, -1, -1))

    def pinned_like(t):
        if t.dim() >= 2:
            h = rev(torch.empty(t.shape[::-1], dtype=t.dtype).pin_memory())
        else:
            h = torch.empty(t.shape, dtype=t.dtype).pin_memory()
        h.copy_(t)
        return h

    def dev_like(t):
        return torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=dev)

    jobs = []  # (inputs [(host, device)], run(), outputs() -> [device tensors], host outputs)
    plans, plan_inputs = {}, {}
    plan_status = {}
    for name, gen, prec in SOLVE_PARTS:
        pr = probs[gen]
        dA = [dev_like(a) for a in pr["A"]]
        dC = [dev_like(c) for c in pr["C"]] if gen else None
        dB = dev_like(pr["B"])
        dXo = ts.empty_fortran(tuple(pr["B"].shape), dev)
        ins = [(pinned_like(pr["B"]), dB)] + [(pinned_like(a), d) for a, d in zip(pr["A"], dA)]
        if gen:
            ins += [(pinned_like(c), d) for c, d in zip(pr["C"], dC)]

        def run(gen=gen, prec=prec, dA=dA, dC=dC, dB=dB, dXo=dXo, name=name):
            if name in plans:
                # FP64: the solve plan of these coefficient buffers (created
                # once, outside the timed region): no host synchronisation
                plans[name].solve(dB, X=dXo, status=plan_status[name])
            elif gen:
                ts.gtsylv_solve(dA, dC, dB, X=dXo, info=infos[name], precision=PREC[prec])
            else:
                ts.tsylv_solve(dA, dB, X=dXo, info=infos[name], precision=PREC[prec])
            return [dXo]
        if prec == 0:
            plan_inputs[name] = (dA, dC)
        jobs.append((ins, run, [pinned_like(dXo)]))
    for prec in (0, 1):
        tag = "adjoint_fp64" if prec == 0 else "adjoint_fp32r"
        dA = [dev_like(a) for a in adj["A"]]
        dB = dev_like(adj["B"])
        dXs = dev_like(adj["Xs"])
        Xa = ts.empty_fortran(ADJ_SHAPE, dev)
        ins = [(pinned_like(adj["B"]), dB), (pinned_like(adj["Xs"]), dXs)] + \
              [(pinned_like(a), d) for a, d in zip(adj["A"], dA)]

        gX = ts.empty_fortran(ADJ_SHAPE, dev)
        gB = ts.empty_fortran(ADJ_SHAPE, dev)
        gA = [ts.empty_fortran((m, m), dev) for m in ADJ_SHAPE]

        def run(prec=prec, tag=tag, dA=dA, dB=dB, dXs=dXs, Xa=Xa, gX=gX, gB=gB, gA=gA):
            ts.tsylv_solve(dA, dB, X=Xa, info=infos[tag + "_fwd"], precision=PREC[prec])
            torch.sub(Xa, dXs, out=gX)
            ts.tsylv_backward(dA, Xa, gX, want_dB=True, want_dA=True, info=infos[tag + "_bwd"],
                              precision=PREC[prec], out=(gB, gA, None))
            return [gB] + gA
        outs_h = [pinned_like(adj["out"][prec][0])] + [pinned_like(g) for g in adj["out"][prec][1]]
        jobs.append((ins, run, outs_h))
    ins = [(pinned_like(pools.B), pools.B), (pinned_like(pools.A), pools.A)]

    def run_batch():
        batched()
        return [pools.X]
    jobs.append((ins, run_batch, [pinned_like(pools.X)]))
    h2d = sum(h.numel() * h.element_size() for ins, _, _ in jobs for h, _ in ins)
    d2h = sum(h.numel() * h.element_size() for _, _, outs in jobs for h in outs)

    cs = torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in jobs]     # inputs of job k on the device
    ev_run = [torch.cuda.Event() for _ in jobs]    # job k's solve done
    ev_out = [torch.cuda.Event() for _ in jobs]    # job k's results on the host
    ev_done = torch.cuda.Event()

    def copy_in(k):
        with torch.cuda.stream(cs):
            for h, d in jobs[k][0]:
                d.copy_(h, non_blocking=True)
            ev_in[k].record(cs)

    def e2e_step(first):
        # every step copies its own inputs in and its results out
        if not first:
            cs.wait_event(ev_run[0])  # the previous step's job 0 is done with its inputs
        copy_in(0)
        for k, (ins, run, outs_h) in enumerate(jobs):
            if k + 1 < len(jobs):
                if not first:
                    cs.wait_event(ev_run[k + 1])
                copy_in(k + 1)  # prefetched while job k runs
            stream.wait_event(ev_in[k])
            if not first:
                stream.wait_event(ev_out[k])  # the previous step's results of job k are on the host
            outs_d = run()
            ev_run[k].record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(ev_run[k])
                for h, d in zip(outs_h, outs_d):
                    h.copy_(d, non_blocking=True)
                ev_out[k].record(cs)

    # one untimed pass (first=True) so that the graphs for the new buffers exist;
    # then the FP64 parts' solve plans on the copied-in coefficients (the plan
    # reads their 2x2 structure once; every execution re-packs the values and
    # checks the structure on the device), and a second untimed pass for their graphs
    e2e_step(True)
    torch.cuda.synchronize(dev)
    for name, (pA, pC) in plan_inputs.items():
        plans[name] = ts.SolvePlan(pA, pC)
        plan_status[name] = torch.full((1,), -99, dtype=torch.int32, device=dev)
    e2e_step(False)
    torch.cuda.synchronize(dev)
    barrier(ws)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    cs.wait_event(e0)
    for _ in range(args.steps):
        e2e_step(False)
    ev_done.record(cs)
    stream.wait_event(ev_done)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws, dev)
    for name, st in plan_status.items():
        if int(st.item()) != 0:
            raise RuntimeError("end-to-end leg: plan execution of %s returned status %d" % (name, int(st.item())))
    for pl in plans.values():
        pl.close()

    # ---- the other configurations, measured beside the step (not part of
    # `value`; after the end-to-end leg, whose captured schedules a larger
    # workspace would invalidate): the d = 4 generalized form in FP64 and every
    # refined precision (FP32 solves; TF32 / BF16 tensor-core block updates),
    # the tensor-core precisions at 256^3 and in the adjoint, and the
    # 512-equation batch FP32-refined against its FP64 solutions
    other = {}

    def precision_sweep(qA, qC, qB, shp, precs):
        res = {}
        for prec in precs:
            qX = ts.empty_fortran(shp, dev)
            qi = _lib.Info()
            if qC is not None:
                fn = lambda: ts.gtsylv_solve(qA, qC, qB, X=qX, info=qi, precision=PREC[prec], max_refine=40)
            else:
                fn = lambda: ts.tsylv_solve(qA, qB, X=qX, info=qi, precision=PREC[prec], max_refine=40)
            fn()
            tm = event_ms(fn, 3)
            _, rho, _ = ts.tsylv_residual(qA, qB, qX, qC, residual=_lib.TSYLV_RESID_FP64)
            res[PNAME[prec]] = {"ms": tm, "iterations": qi.iterations, "rel_residual_fp64": rho}
            del qX
        if 0 in precs:
            for prec in precs:
                if prec:
                    res[PNAME[prec]]["vs_fp64"] = res["fp64"]["ms"] / res[PNAME[prec]]["ms"]
        return res

    if not args.no_other:
        for shp in D4_SHAPES:
            q = synthetic.problem(args.seed + rank, shp, generalized=True)
            qA = [to_dev(a) for a in q["A"]]
            qC = [to_dev(c) for c in q["C"]]
            qB = to_dev(q["B"])
            res = precision_sweep(qA, qC, qB, shp, (0, 1, 2, 3, 4))
            res["mixed_vs_fp64"] = res["fp64"]["ms"] / res["fp32r"]["ms"]
            other["d4_generalized_" + "x".join(str(v) for v in shp)] = res
            del qA, qC, qB
        for gen in (False, True):
            pr = probs[gen]
            other["tensorcore_256_" + ("generalized" if gen else "laplace")] = precision_sweep(
                pr["A"], pr["C"], pr["B"], shape, (2, 3))
        for tag, prc in (("adjoint_tf32r", 2), ("adjoint_df64", 4)):
            infos[tag + "_fwd"] = _lib.Info()
            infos[tag + "_bwd"] = _lib.Info()
            Xt = ts.empty_fortran(ADJ_SHAPE, dev)

            def adjoint_tc(tag=tag, prc=prc, Xt=Xt):
                ts.tsylv_solve(adj["A"], adj["B"], X=Xt, info=infos[tag + "_fwd"], precision=PREC[prc])
                adj["out"][prc] = ts.tsylv_backward(adj["A"], Xt, Xt - adj["Xs"], want_dB=True, want_dA=True,
                                                    info=infos[tag + "_bwd"], precision=PREC[prc])
            adjoint_tc()
            tm = event_ms(adjoint_tc, max(3, args.steps))
            dB, dA, _ = adj["out"][prc]
            dB0, dA0, _ = adj["out"][0]
            other[tag] = {"ms": tm, "unknowns_per_s": 2 * Na / (tm * 1e-3),
                          "iterations_fwd_bwd": [infos[tag + "_fwd"].iterations, infos[tag + "_bwd"].iterations],
                          "vs_fp64": parts["adjoint_fp64"]["ms"] / tm,
                          "rel_diff_vs_fp64": {
                              "dB": float(torch.linalg.vector_norm(dB - dB0) / torch.linalg.vector_norm(dB0)),
                              "dA": max(float(torch.linalg.matrix_norm(a - b) / torch.linalg.matrix_norm(b))
                                        for a, b in zip(dA, dA0))}}
        del Xt
        # general (dense) coefficients, Alg. 1: host Schur reduction, GPU
        # change-of-basis transforms (dense FP64 mode products) and the FP64
        # triangular solve, 256^3 Laplace form
        from paper_1905_09539_gb300.general import reduce_coefficients, solve_general, transform
        rg = np.random.default_rng(args.seed + rank + 1000)
        Ag = [to_dev(np.asfortranarray(rg.standard_normal((n, n)) / np.sqrt(n) + 2.5 * np.eye(n))) for n in shape]
        Bg = probs[False]["B"]
        th = time.perf_counter()
        red = reduce_coefficients([a.cpu().numpy() for a in Ag], device=dev)
        th = time.perf_counter() - th
        Xg = ts.empty_fortran(shape, dev)
        fn = lambda: solve_general(Ag, Bg, X=Xg, reduced=red)
        fn()
        tg = event_ms(fn, 3)
        Ug = [u for _, u in red]
        Tb = ts.empty_fortran(shape, dev)
        tt = event_ms(lambda: transform(Bg, Ug, trans=[True] * 3, Y=Tb), 3)
        ftr = 2.0 * N * sum(shape)  # one transform: a dense mode product per mode
        other["general_laplace_256"] = {
            "ms_gpu": tg, "host_reduction_s": th, "transform_ms": tt,
            "transform_tflops": ftr / (tt * 1e-3) / 1e12,
            "transform_frac_fp64_peak": ftr / (tt * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
            "note": "two transforms (B x U^T, X x U) + FP64 triangular solve on the GPU; real Schur forms on the host"}
        del Ag, Ug, Tb, Xg
        # the batch with the tile shape fixed at the default (8, 8, 8): what the
        # shape search of the autotuner gains
        X64 = pools.X.clone()
        iff = _lib.Info()
        fnf = lambda: pools.solve(info=iff, leaf=(8, 8, 8))
        fnf()
        tf = event_ms(fnf, max(3, args.steps))
        other["batched_fp64_fixed_shape_8x8x8"] = {
            "ms": tf, "tuned_ms": parts["batched_fp64"]["ms"], "tuned_shape": parts["batched_fp64"]["tile_shape"],
            "tuned_vs_fixed": tf / parts["batched_fp64"]["ms"], "queue_order": iff.batch_order,
            "ctas_per_sm": iff.batch_ctas_per_sm,
            "rel_diff_vs_tuned": float(torch.linalg.vector_norm(pools.X - X64) / torch.linalg.vector_norm(X64))}
        # single solves with the autotuned tile shape (opts.nmin = -1; the first
        # call tunes, the timed calls reuse the choice)
        tuned = {}
        for name, gen, prec in SOLVE_PARTS:
            pr = probs[gen]
            Xt = ts.empty_fortran(shape, dev)
            it_ = _lib.Info()
            if gen:
                fnt = lambda: ts.gtsylv_solve(pr["A"], pr["C"], pr["B"], X=Xt, info=it_, precision=PREC[prec], nmin=-1)
            else:
                fnt = lambda: ts.tsylv_solve(pr["A"], pr["B"], X=Xt, info=it_, precision=PREC[prec], nmin=-1)
            fnt()
            tt = event_ms(fnt, 3)
            tuned[name] = {"ms": tt, "tile_shape": list(it_.leaf[:3]), "default_ms": parts[name]["ms"],
                           "tuned_vs_default": parts[name]["ms"] / tt}
            del Xt
        other["autotuned_256"] = tuned
        # the 64^3 workload (Laplace FP64, and the generalized form): default
        # tile shape against the autotuned one
        small = {}
        for gen in (False, True):
            q = synthetic.problem(args.seed + rank, (64, 64, 64), generalized=gen)
            qA = [to_dev(a) for a in q["A"]]
            qC = [to_dev(c) for c in q["C"]] if gen else None
            qB = to_dev(q["B"])
            qX = ts.empty_fortran((64, 64, 64), dev)
            row = {}
            for tag, nm in (("default", 0), ("tuned", -1)):
                qi = _lib.Info()
                if gen:
                    fq = lambda: ts.gtsylv_solve(qA, qC, qB, X=qX, info=qi, nmin=nm)
                else:
                    fq = lambda: ts.tsylv_solve(qA, qB, X=qX, info=qi, nmin=nm)
                fq()
                row[tag] = {"ms": event_ms(fq, 5), "tile_shape": list(qi.leaf[:3])}
            row["tuned_vs_default"] = row["default"]["ms"] / row["tuned"]["ms"]
            small["generalized" if gen else "laplace"] = row
        other["autotuned_64"] = small
        # the paper's n_min sweep shapes (Sec. 2.4: n = 80 for d = 3, n = 25 for
        # d = 4; the merged-mode sweep also covers d = 5, here n = 14): the FP64
        # Laplace solve at every recursion cutoff the block tiles allow, and a
        # d = 5 workload (20^5) in every precision
        sweep = {}
        for dd, nn_ in ((3, 80), (4, 25), (5, 14)):
            shp = (nn_,) * dd
            q = synthetic.problem(args.seed + rank, shp)
            qA = [to_dev(a) for a in q["A"]]
            qB = to_dev(q["B"])
            qX = ts.empty_fortran(shp, dev)
            te = {3: 8, 4: 4, 5: 4}[dd]
            row = {}
            for nm in range(2, te + 1):
                fq = lambda: ts.tsylv_solve(qA, qB, X=qX, nmin=nm)
                fq()
                row[str(nm)] = event_ms(fq, 5)
            sweep["d%d_n%d_laplace_fp64_ms_by_nmin" % (dd, nn_)] = row
        other["paper_nmin_sweeps"] = sweep
        # the paper's own two-term form Eq. (3.1) at 256^3 (FP64): time, and
        # the FP64 residual of the result, evaluated with the library's
        # change-of-basis (dense mode product) kernel
        from paper_1905_09539_gb300.general import transform
        q = synthetic.problem(args.seed + rank, shape, generalized=True)
        qA = [to_dev(a) for a in q["A"]]
        qC = to_dev(q["C"][0])
        qB = probs[True]["B"]
        qX = ts.empty_fortran(shape, dev)
        qi = _lib.Info()
        fq = lambda: ts.gsylvten_solve(qA, qC, qB, X=qX, info=qi)
        fq()
        tq = event_ms(fq, 3)
        T1 = transform(qX, [qA[0], None, None])
        T2 = transform(qX, [qC] + qA[1:])
        Rq = qB - T1 - T2
        nrm = lambda a: float(np.linalg.norm(a, 2))
        opn = nrm(q["A"][0]) + nrm(q["C"][0]) * nrm(q["A"][1]) * nrm(q["A"][2])
        other["two_term_256_fp64"] = {
            "ms": tq, "unknowns_per_s": N / (tq * 1e-3), "executed_gflop": qi.flops / 1e9,
            "rel_residual_fp64": float(torch.linalg.vector_norm(Rq) / (opn * torch.linalg.vector_norm(qX))),
            "note": "gsylvten_solve, Eq. (3.1): X x_1 A_1 + X x_1 C x_2 A_2 x_3 A_3 = B; residual by the DMMA "
                    "mode-product kernel"}
        fqd = lambda: ts.gsylvten_solve(qA, qC, qB, X=qX, precision=_lib.TSYLV_DF64)
        fqd()
        tqd = event_ms(fqd, 3)
        T1 = transform(qX, [qA[0], None, None])
        T2 = transform(qX, [qC] + qA[1:])
        Rq = qB - T1 - T2
        other["two_term_256_df64"] = {
            "ms": tqd, "unknowns_per_s": N / (tqd * 1e-3), "vs_fp64": tq / tqd,
            "rel_residual_fp64": float(torch.linalg.vector_norm(Rq) / (opn * torch.linalg.vector_norm(qX))),
            "note": "gsylvten_solve with precision TSYLV_DF64 (double-float arithmetic on the FP32 pipes)"}
        del qA, qC, qX, T1, T2, Rq
        # the double-float solve at 256^3 (pairs of floats on the FP32 pipes),
        # both forms, against the FP64 solve of the step; FP64 residual of the result
        for dgen in (False, True):
            pr = probs[dgen]
            pr["X"][4] = ts.empty_fortran(shape, dev)
            nm = "df64_" + ("generalized" if dgen else "laplace")
            infos[nm] = _lib.Info()
            fd = lambda: solve(nm, dgen, 4)
            fd()
            td = event_ms(fd, 3)
            _, rho_d, _ = ts.tsylv_residual(pr["A"], pr["B"], pr["X"][4], pr["C"], residual=_lib.TSYLV_RESID_FP64)
            fp = parts["fp64_generalized" if dgen else "fp64_laplace"]["ms"]
            other["df64_256_" + ("generalized" if dgen else "laplace")] = {
                "ms": td, "unknowns_per_s": N / (td * 1e-3), "rel_residual_fp64": rho_d, "vs_fp64": fp / td,
                "note": "precision TSYLV_DF64: one solve in double-float arithmetic (float pairs) on the FP32 pipes"}
            del pr["X"][4]
        # the complex-triangular variant at 256^3 (coefficients in complex
        # Schur form, as in the paper's experiments), both forms; the residual
        # is a check computed by torch mode products, outside the timed calls
        for zgen in (False, True):
            zq = synthetic.complex_problem(args.seed + rank, shape, generalized=zgen)
            zt = lambda a: torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to(dev).T
            zA = [zt(a) for a in zq["A"]]
            zC = [zt(c) for c in zq["C"]] if zgen else None
            zB = torch.from_numpy(np.ascontiguousarray(zq["B"].transpose(2, 1, 0))).to(dev).permute(2, 1, 0)
            zX = ts.empty_fortran(shape, dev, torch.complex128)
            zi = _lib.Info()
            fz = lambda: ts.ztsylv_solve(zA, zB, zC, X=zX, info=zi)
            fz()
            tz = event_ms(fz, 3)
            zR = zB.clone()
            for mu in range(3):
                Y = torch.movedim(torch.tensordot(zA[mu], torch.movedim(zX, mu, 0), dims=1), 0, mu)
                if zgen:
                    for eta in range(3):
                        if eta != mu:
                            Y = torch.movedim(torch.tensordot(zC[eta], torch.movedim(Y, eta, 0), dims=1), 0, eta)
                zR -= Y
            nrm = lambda a: float(np.linalg.norm(a, 2))
            opn = sum(nrm(zq["A"][mu]) * (np.prod([nrm(zq["C"][e]) for e in range(3) if e != mu]) if zgen else 1.0)
                      for mu in range(3))
            other["complex_256_" + ("dterm" if zgen else "laplace") + "_fp64"] = {
                "ms": tz, "unknowns_per_s": N / (tz * 1e-3), "executed_gflop": zi.flops / 1e9,
                "tflops": zi.flops / (tz * 1e-3) / 1e12,
                "frac_fp64_peak": zi.flops / (tz * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                "rel_residual_fp64": float(torch.linalg.vector_norm(zR) / (opn * torch.linalg.vector_norm(zX))),
                "note": "ztsylv_solve / zgtsylv_solve: complex upper triangular A_mu (C_mu), complex128 B and X; "
                        "a complex multiply-add counted as 4 real FP64 multiply-adds (8 flops)"}
            del zA, zC, zB, zX, zR, Y
        q = synthetic.problem(args.seed + rank, (20,) * 5)
        qA = [to_dev(a) for a in q["A"]]
        qB = to_dev(q["B"])
        other["d5_laplace_20"] = precision_sweep(qA, None, qB, (20,) * 5, (0, 1, 2, 3))
        del qA, qB
        ir = _lib.Info()
        fnr = lambda: pools.solve(info=ir, precision=_lib.TSYLV_FP32_REFINED)
        fnr()
        tr = event_ms(fnr, max(3, args.steps))
        other["batched_fp32r"] = {
            "ms": tr, "unknowns_per_s": units_rank["batched"] / (tr * 1e-3), "iterations": ir.iterations,
            "mixed_vs_fp64": parts["batched_fp64"]["ms"] / tr,
            "rel_diff_vs_fp64": float(torch.linalg.vector_norm(pools.X - X64) / torch.linalg.vector_norm(X64))}
        idf = _lib.Info()
        fdf = lambda: pools.solve(info=idf, precision=_lib.TSYLV_DF64)
        fdf()
        tdf = event_ms(fdf, max(3, args.steps))
        other["batched_df64"] = {
            "ms": tdf, "unknowns_per_s": units_rank["batched"] / (tdf * 1e-3),
            "vs_fp64": parts["batched_fp64"]["ms"] / tdf,
            "rel_diff_vs_fp64": float(torch.linalg.vector_norm(pools.X - X64) / torch.linalg.vector_norm(X64)),
            "note": "precision TSYLV_DF64: the double-float solve of every equation in one persistent launch"}
        pools.solve(info=infos["batched_fp64"])  # leave the FP64 solutions in place
        del X64

    line = {
        "metric": METRIC,
        "value": value, "unit": "unknowns/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (synthetic.py, seed %d)" % args.seed,
        "config": {"workload": WORKLOAD.replace("256^3", "%d^3" % args.n),
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (%.0f MB per 256^3 tensor); no flush" % (N * 8 / 1e6),
                   "units_per_step": units_rank},
        "parts": parts,
        "mixed_vs_fp64": mixed_vs_fp64,
        "other_configs": other,
        "roofline": roofline,
        "e2e": {"value": units / (e2e_ms * 1e-3), "unit": "unknowns/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "note": "FP64 256^3 parts through solve plans (tsylv_plan_execute; each plan created once "
                        "before the timed region on the device coefficient buffers, which every step "
                        "refills from the host); refined, adjoint and batch parts through their solve calls"},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu:
        # all host cores (the single solves take one core each, the batch all),
        # and one core: the single-solve parts are the same runs, the batch is
        # timed again on one core
        t_all, det_all = oracle_step_seconds(0, seed=args.seed)
        t_b1, det_b1 = oracle_part_seconds("batched", 1, seed=args.seed)
        t_one = t_all - det_all["batched"]["seconds"] + t_b1
        units_step = sum(units_rank.values())
        line["cpu_baseline"] = {
            "value": units_step / t_all, "unit": "unknowns/s", "cores": det_all["threads"], "kind": "oracle",
            "sample": ORACLE_RULE + "; %d host cores" % det_all["threads"],
            "value_1core": units_step / t_one, "batched_1core_s": t_b1, "detail": det_all}
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
    ap.add_argument("--no-other", action="store_true",
                    help="skip the measurements of the d = 4 and batched FP32-refined configurations")
    ap.add_argument("--fp64-peak", action="store_true", help="build and run the FP64 throughput probe")
    ap.add_argument("--only", default=None,
                    help="profiling aid: run just this part of the step (e.g. fp64_generalized; also "
                         "complex_laplace, complex_dterm) for the warm-up and timed steps, print its time and exit")
    args = ap.parse_args()
    if args.fp64_peak:
        run_fp64_peak()
        return
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
