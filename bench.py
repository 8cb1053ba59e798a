"""Benchmark: seconds per eigenproblem and Chebyshev-filter TFLOP/s of the
GB300 ChFSI on a correlated sequence of dense complex Hermitian problems.

Workload (default): 10 correlated complex128 problems, n = 4096, nev = 256,
nex = 64, spectrum with 300 low eigenvalues in [-3, -1] and the bulk in
[0, 20], H_{l+1} = U H_l U^H + 1e-4 diag(d), U = exp(1e-3 i A); problem 1
starts from a random block, problem l+1 from problem l's Ritz vectors;
tolerance 1e-10.  One step = solving the whole sequence.  Every H is
268 MB (larger than the 129 MB L2), so no L2 flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own
replica of the sequence (independent problems shard with no exchange).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filter TFLOP/s and s per eigenproblem at resid≤1e-10: mixed+learned vs FP64"
UNIT = "s/eigenproblem"
SEQ_SEED_OFFSET = 2000
# ncu capture of one tc_filter_kernel launch of the fixed-shape probe
# (bench.py --filter-probe --probe-k 320 --probe-deg 8: n 4096, 8 steps on 320
# columns, BF16x3, 160-wide column blocks in groups of 4).
# The bench's own filter launches mix shapes (k_act, degrees, 3 or 6 products),
# so their per-launch traffic is not captured; this is the kernel's measured
# traffic against its algorithmic bytes (8 n^2 + 56 n k per step).
TC_FILTER_PROBE_TRAFFIC = {"shape": "n 4096, k 320, degree 8, BF16x3, 160-wide blocks, group 4",
                           "dram_bytes": 1.602e9, "algorithmic_bytes": 1.661e9,
                           "ratio": 0.96, "ncu_duration_ms": 0.917,
                           "executed_tflops_ncu": 1124.0}
TC_FILTER_TRAFFIC_NOTE = ("per-launch traffic of the bench's mixed launches not captured; "
                          "see probe_traffic (one captured launch of the filter probe)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["tc", "mixed", "fp64"], default="tc")
    ap.add_argument("--n", type=int, default=None, help="override n (smaller test runs)")
    ap.add_argument("--length", type=int, default=None)
    ap.add_argument("--fp64-compare", type=int, default=-1,
                    help="also time the plain FP64 GPU path on this many problems of the same "
                         "sequence (-1: all of them, 0: skip)")
    ap.add_argument("--cpu-budget", type=float, default=90.0,
                    help="seconds of oracle work on the host cores: the CPU baseline solves "
                         "the sequence's problems in order until this is spent")
    ap.add_argument("--no-certify", action="store_true",
                    help="skip the untimed per-problem residual and eigenvalue checks")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--degrees", choices=["learned", "analytic"], default="learned")
    ap.add_argument("--deg-warm", type=int, default=None,
                    help="filter degree of the first loop on a warm start (library default 8)")
    ap.add_argument("--warm-rr", action="store_true",
                    help="Rayleigh-Ritz on each warm start before the first filter")
    ap.add_argument("--warm-resid", type=int, choices=[0, 1], default=0,
                    help="warm starts: residuals of the starting block on the new H, per-vector "
                         "first-loop degrees (1) or the uniform deg_warm (0, the library default); "
                         "the FP64 comparison always uses 1, its faster setting")
    ap.add_argument("--f64-gemm", choices=["ozaki", "fp64"], default="ozaki",
                    help="engine of the FP64 products in the tc/mixed modes")
    ap.add_argument("--batched-scale", type=float, default=0.25,
                    help="n range of the 64-problem batched measurement, as a fraction of "
                         "[1500, 6000] (0 skips it)")
    ap.add_argument("--batched-full", type=int, default=0,
                    help="also run the 64-sequence workload at its stated size (n 1500-6000, "
                         "10 steps; several minutes)")
    ap.add_argument("--learned-protocol", type=int, default=1,
                    help="run the learned-degree protocol at n = 8192 (30 problems)")
    ap.add_argument("--train-length", type=int, default=None,
                    help="problems in the (separate) training sequence of the degree MLP "
                         "(default: the sequence length, so training covers every step index)")
    ap.add_argument("--filter-probe", action="store_true",
                    help="time the tensor-core filter alone on one fixed shape (uniform "
                         "degree, so the work per launch is exact) and print its own JSON "
                         "line; the sequence benchmark is not run")
    ap.add_argument("--probe-k", type=int, default=320)
    ap.add_argument("--probe-deg", type=int, default=8)
    ap.add_argument("--probe-split", choices=["x3", "x6"], default="x3")
    ap.add_argument("--probe-reps", type=int, default=5)
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace('.', '').isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace('.', '').isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def sizes(cfg, n):
    if n == cfg.n:
        return cfg.nev, cfg.nex
    return max(1, cfg.nev * n // cfg.n), max(1, cfg.nex * n // cfg.n)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The oracle (plain FP64 NumPy ChFSI) on the host cores: each step
    solves problem 1 (random start) and problem 2 (warm start) of the same
    sequence; the value extrapolates to the 10-problem sequence as
    (t1 + 9 t2) / 10."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import torch
    import oracle
    from workloads.synthetic import WORKLOADS, random_block
    cfg = WORKLOADS["seq10_n4096"]
    n = args.n or cfg.n
    nev, nex = sizes(cfg, n)
    length = args.length or cfg.length
    dev = torch.device("cuda:0") if torch.cuda.is_available() else None
    from workloads.synthetic import config_sequence
    Hs, lam = config_sequence(cfg, 14044161 + 2000, length=2, n=n, device=dev)
    Hs = [h.cpu().numpy() if dev is not None else h for h in Hs]
    X0 = random_block(n, nev + nex, 14044161 + 2500)
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r1 = oracle.chfsi(Hs[0], nev, nex, X0, cfg.tol)
        t1 = time.perf_counter()
        r2 = oracle.chfsi(Hs[1], nev, nex, r1["X"], cfg.tol,
                          warm=(r1["evals"][0], r1["evals"][-1]))
        t2 = time.perf_counter()
        if it >= args.warmup:
            times.append((t1 - t0, t2 - t1))
    t1m = float(np.mean([a for a, _ in times]))
    t2m = float(np.mean([b for _, b in times]))
    val = (t1m + (length - 1) * t2m) / length
    cores = os.cpu_count()
    sample = (f"problems 1 (random start) and 2 (warm start) of the n={n} sequence per step; "
              f"value = (t1 + {length - 1} t2)/{length}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * (t1m + t2m),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"correlated sequence of {length} complex128 Hermitian problems, "
                               f"n={n}, nev={nev}, nex={nex}, tol 1e-10",
                   "l2": ("inputs larger than L2" if 16 * n * n > 129e6 else
                          "inputs smaller than L2 (reduced-size run)")},
        "cpu_baseline": {"kind": "oracle", "value": val, "unit": UNIT, "cores": cores,
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "loops": [int(r1["loops"]), int(r2["loops"])],
    }))


def cpu_baseline_sample(Hs_host, nev, nex, tol, X0, budget_s):
    """Oracle on the host cores over the same sequence: problems in order
    (problem 1 from the random block, each later one warm from its
    predecessor's Ritz vectors), until the budget is spent; the value is the
    mean over the problems solved."""
    import oracle
    times, X, warm = [], X0, None
    t_start = time.perf_counter()
    for l, H in enumerate(Hs_host):
        t0 = time.perf_counter()
        r = oracle.chfsi(H, nev, nex, X, tol, warm=warm)
        times.append(time.perf_counter() - t0)
        X, warm = r["X"], (r["evals"][0], r["evals"][-1])
        if time.perf_counter() - t_start > budget_s:
            break
    done = len(times)
    return {"value": float(np.mean(times)), "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": (f"problems 1..{done} of the {len(Hs_host)}-problem sequence "
                       f"(problem 1 from the random block), value = their mean; per problem "
                       + ", ".join(f"{t:.2f}" for t in times) + " s")}


def measure_batched(scale, dev, stream, prec):
    """64 independent sequences (k-point style): n uniform in scale x [1500,
    6000], nev = n/16, nex = nev/4, 2 steps each; lockstep batched solve
    (one batched filter launch per loop) against the same problems solved
    one at a time."""
    import torch
    from paper_1404_4161_gb300 import _lib as L
    from paper_1404_4161_gb300.solver import Chfsi, colmajor
    from workloads.synthetic import WORKLOADS, config_sequence, random_block
    cfg = WORKLOADS["batched64"]
    rng = np.random.Generator(np.random.PCG64(14044161 + 4000))
    lo, hi = int(1500 * scale), int(6000 * scale)
    seqs, steps = [], 2
    for p in range(64):
        n = int(rng.integers(lo, hi + 1))
        nev = max(1, n // 16)
        nex = max(1, nev // 4)
        Hs, _ = config_sequence(cfg, 14044161 + 4100 + p, length=steps, n=n)
        X0 = random_block(n, nev + nex, 14044161 + 4300 + p)
        seqs.append(([colmajor(torch.from_numpy(h).to(dev)) for h in Hs], nev, nex,
                     colmajor(torch.from_numpy(X0).to(dev))))
    s = Chfsi(precision=prec if prec != L.PREC_FP64 else L.PREC_TC, profile=1)
    work = [(H, nev, nex, X.clone()) for H, nev, nex, X in seqs]
    s.solve_batched(work, 1e-10)  # warm-up
    work = [(H, nev, nex, X.clone()) for H, nev, nex, X in seqs]
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    evs, stats, rc, _ = s.solve_batched(work, 1e-10)
    b.record(stream)
    torch.cuda.synchronize()
    t_batch = a.elapsed_time(b) / 1e3
    filt_ms = sum(st[0]["k_tc_ms"] for st in stats)
    filt_fl = sum(st[0]["k_tc_flops"] for st in stats)
    a.record(stream)
    for H, nev, nex, X in seqs:
        s.solve_sequence(H, nev, nex, X.clone(), 1e-10)
    b.record(stream)
    torch.cuda.synchronize()
    t_seq = a.elapsed_time(b) / 1e3
    s.close()
    return {"problems": 64 * steps, "n_range": [lo, hi], "steps": steps, "rc": rc,
            "s_per_problem_batched": t_batch / (64 * steps),
            "s_per_problem_one_at_a_time": t_seq / (64 * steps),
            "batched_filter_useful_tflops": filt_fl / (filt_ms / 1e3) / 1e12 if filt_ms else None,
            "batched_filter_executed_tflops": 3 * filt_fl / (filt_ms / 1e3) / 1e12 if filt_ms else None,
            "max_loops": max(st["loops"] for row in stats for st in row)}


def measure_learned_protocol(dev, stream, n=8192, nev=512, nex=128, length=30, train=10):
    """The learned-degree protocol at the size of the n = 8192 workload: a
    correlated sequence of `length` problems (circulant construction: exact
    spectrum, eigenvectors turned by ~eps per step), problems 1..train
    solved with the analytic rule while the solver records its traces, the
    degree MLP trained on them (library kernels), the learned degree's
    margin chosen on training problems train/2+1 .. train, then problems
    train+1 .. length solved twice from problem train's Ritz vectors:
    analytic rule vs learned degrees.  Loops, filter column-degrees and seconds per problem
    for both; eigenvalues checked against the exact spectrum."""
    import torch
    from paper_1404_4161_gb300 import _lib as L
    from paper_1404_4161_gb300 import learned
    from paper_1404_4161_gb300.solver import Chfsi, colmajor
    from workloads.synthetic import WORKLOADS, BASE_SEED, circulant_sequence, random_block
    cfg = WORKLOADS["seq30_n8192"]
    import dataclasses
    cfg = dataclasses.replace(cfg, n=n, nev=nev, nex=nex, n_low=nev + nex // 2)
    hs, lam = circulant_sequence(cfg, BASE_SEED + 9000, length=length, device=dev)
    Hc = [colmajor(h) for h in hs]
    del hs
    normH = float(np.abs(lam).max())
    s = Chfsi(precision=L.PREC_TC, f64_gemm=L.GEMM_OZAKI)
    s.trace_enable(1 << 21)
    X = colmajor(torch.from_numpy(random_block(n, nev + nex, BASE_SEED + 9500)).to(dev))
    half = train // 2
    ev, sts, rc = s.solve_sequence(Hc[:half], nev, nex, X, cfg.tol)
    X_half = X.clone()  # Ritz vectors of training problem `half`
    s.set_opts(step0=half)
    ev, sts2, rc2 = s.solve_sequence(Hc[half:train], nev, nex, X, cfg.tol)
    s.set_opts(step0=0)
    if rc != L.OK or rc2 != L.OK:
        raise RuntimeError(f"learned protocol: training sequence rc {rc}, {rc2}")
    xs, ys = learned.dataset(s)
    losses = learned.train(s, xs, ys, steps=3000, lr=2e-3)
    s.trace_enable(0)
    # Model selection on the training problems only: the learned degree's
    # margin (opts.mlp_extra) that solves problems half+1..train (from the
    # Ritz vectors of problem half) fastest is kept for the evaluation.
    sel = {}
    for extra in (0, 1, 2):
        s.set_opts(degree_model=L.DEG_MLP, mlp_extra=extra, step0=half)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, stv, rcv = s.solve_sequence(Hc[half:train], nev, nex, X_half.clone(), cfg.tol)
        b.record(stream)
        torch.cuda.synchronize()
        if rcv == L.OK:
            sel[extra] = {"s": a.elapsed_time(b) / 1e3, "loops": sum(x["loops"] for x in stv),
                          "col_degrees": sum(x["col_degrees"] for x in stv)}
    best_extra = min(sel, key=lambda e: sel[e]["s"]) if sel else 2
    out = {"workload": f"circulant correlated sequence, n={n}, nev={nev}, nex={nex}, "
                       f"{length} problems; trained on problems 1..{train}, evaluated on "
                       f"{train + 1}..{length}",
           "train_rows": int(xs.shape[0]), "loss0": losses[0], "loss": losses[-1],
           "mlp_extra_selected_on_training": best_extra,
           "mlp_extra_validation": {str(e): v for e, v in sel.items()}}
    for name, model in (("analytic", L.DEG_ANALYTIC), ("learned", L.DEG_MLP)):
        s.set_opts(degree_model=model, step0=train, mlp_extra=best_extra)
        Xe = X.clone()
        s.solve_sequence(Hc[train:train + 1], nev, nex, Xe.clone(), cfg.tol)  # warm-up
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ev, sts, rc = s.solve_sequence(Hc[train:], nev, nex, Xe, cfg.tol)
        b.record(stream)
        torch.cuda.synchronize()
        if rc != L.OK:
            raise RuntimeError(f"learned protocol: {name} evaluation rc {rc}")
        err = float(np.abs(ev.cpu().numpy()[:, :nev] - lam[None, :nev]).max()) / normH
        if err > 1e-12:
            raise RuntimeError(f"learned protocol: {name} eigenvalue error {err:.2e}")
        out[name] = {"s_per_problem": a.elapsed_time(b) / 1e3 / (length - train),
                     "loops": sum(x["loops"] for x in sts),
                     "col_degrees": sum(x["col_degrees"] for x in sts),
                     "loops_mlp": sum(x["loops_mlp"] for x in sts),
                     "mlp_fallbacks": sum(x["mlp_fallback"] for x in sts),
                     "max_eig_err_rel_normH": err}
    s.close()
    del Hc
    torch.cuda.empty_cache()
    out["time_ratio_learned_over_analytic"] = (out["learned"]["s_per_problem"] /
                                               out["analytic"]["s_per_problem"])
    return out


def measure_batched_full(dev, stream, problems=64, steps=10, window=2, oracle_sample=2):
    """The k-point-style workload at its stated size: `problems` independent
    correlated sequences (circulant construction, see
    workloads.synthetic.circulant_window), n uniform in [1500, 6000]
    (seeded), nev = n/16, nex = nev/4, `steps` steps each, tol 1e-10.  The
    steps run in windows of `window` (the matrices of one window are made
    on the device, untimed; the next window starts warm from the last Ritz
    blocks).  Timed: the lockstep batched solve (one batched filter launch
    per outer loop) and the same problems solved one at a time.  Checked:
    every status, the eigenvalues of every problem and step against the
    exact spectrum, residuals of the last step.  The oracle (host cores)
    solves the first two steps of the `oracle_sample` smallest problems."""
    import torch
    from paper_1404_4161_gb300 import _lib as L
    from paper_1404_4161_gb300.solver import Chfsi
    from workloads.synthetic import WORKLOADS, BASE_SEED, circulant_window, random_block
    cfg = WORKLOADS["batched64"]
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 4000))
    ns = [int(x) for x in rng.integers(1500, 6001, problems)]
    dims = [(n, n // 16, (n // 16) // 4) for n in ns]
    seeds = [BASE_SEED + 4100 + p for p in range(problems)]
    X0 = [random_block(n, nev + nex, BASE_SEED + 4300 + p) for p, (n, nev, nex) in enumerate(dims)]
    out = {"workload": f"{problems} correlated sequences (circulant), n uniform in [1500, 6000] "
                       f"(min {min(ns)}, max {max(ns)}), nev = n/16, nex = nev/4, {steps} steps, "
                       f"tol 1e-10, windows of {window} steps",
           "problem_steps": problems * steps}
    for mode in ("batched", "one_at_a_time"):
        s = Chfsi(precision=L.PREC_TC, f64_gemm=L.GEMM_OZAKI, profile=1)
        Xs = [torch.from_numpy(x).to(dev).t().contiguous() for x in X0]
        warm = None
        t_solve, loops, filt_ms, filt_fl, eig_err, resid = 0.0, 0, 0.0, 0.0, 0.0, 0.0
        for w0 in range(0, steps, window):
            cnt = min(window, steps - w0)
            hs, lams = [], []
            for p, (n, nev, nex) in enumerate(dims):
                h, lam = circulant_window(cfg, seeds[p], w0, cnt, n, device=dev)
                hs.append([x.t().contiguous() for x in h])
                lams.append(lam)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if mode == "batched":
                seqs = [(hs[p], nev, nex, Xs[p]) for p, (n, nev, nex) in enumerate(dims)]
                evs, stats, rc, warm = s.solve_batched(seqs, cfg.tol, warm=warm)
                if rc != L.OK:
                    raise RuntimeError(f"batched64: rc {rc} at steps {w0}..{w0 + cnt - 1}")
                flat = [st for row in stats for st in row]
                filt_ms += sum(row[0]["k_tc_ms"] for row in stats)
                filt_fl += sum(row[0]["k_tc_flops"] for row in stats)
                evs = [e.cpu().numpy() for e in evs]
            else:
                warm = warm or [None] * problems
                evs, flat = [], []
                for p, (n, nev, nex) in enumerate(dims):
                    rows = []
                    for l in range(cnt):
                        s.set_opts(step0=w0 + l)
                        ev, st, rc = s.solve(hs[p][l], nev, nex, Xs[p], cfg.tol, warm=warm[p])
                        if rc != L.OK:
                            raise RuntimeError(f"batched64 one-at-a-time: rc {rc}")
                        warm[p] = (float(ev[0]), float(ev[-1]))
                        rows.append(ev.cpu().numpy())
                        flat.append(st)
                    evs.append(np.vstack(rows))
            b.record(stream)
            torch.cuda.synchronize()
            t_solve += a.elapsed_time(b) / 1e3
            loops += sum(st["loops"] for st in flat)
            for p, (n, nev, nex) in enumerate(dims):
                normH = float(np.abs(lams[p]).max())
                eig_err = max(eig_err, float(np.abs(evs[p][:, :nev] - lams[p][None, :nev]).max())
                              / normH)
                if w0 + cnt == steps:
                    H = hs[p][-1].t()
                    X = Xs[p].t()[:, :nev]
                    ev_last = torch.from_numpy(evs[p][-1, :nev]).to(dev)
                    R = torch.linalg.vector_norm(H @ X - X * ev_last.to(X.dtype), dim=0)
                    resid = max(resid, float(R.max()) / normH)
            del hs
            torch.cuda.empty_cache()
        s.close()
        if eig_err > 1e-12 or resid > cfg.tol:
            raise RuntimeError(f"batched64 {mode}: eigenvalue error {eig_err:.2e}, "
                               f"residual {resid:.2e}")
        out[mode] = {"s_per_problem": t_solve / (problems * steps), "loops": loops,
                     "max_eig_err_rel_normH": eig_err, "max_resid_last_step": resid}
        if mode == "batched" and filt_ms > 0:
            out[mode]["filter_useful_tflops"] = filt_fl / (filt_ms / 1e3) / 1e12
    if oracle_sample:
        import oracle
        order = np.argsort(ns)[:oracle_sample]
        t, cnt = 0.0, 0
        for p in order:
            n, nev, nex = dims[p]
            hs, lam = circulant_window(cfg, seeds[p], 0, 2, n)
            X, wv = X0[p], None
            for h in hs:
                t0 = time.perf_counter()
                r = oracle.chfsi(h.numpy(), nev, nex, X, cfg.tol, warm=wv)
                t += time.perf_counter() - t0
                cnt += 1
                X, wv = r["X"], (r["evals"][0], r["evals"][-1])
        out["cpu_oracle"] = {"s_per_problem": t / cnt, "cores": os.cpu_count(),
                             "sample": f"steps 1-2 of the {oracle_sample} smallest problems "
                                       f"(n = {[ns[p] for p in order]})"}
    return out


def filter_probe(args):
    """One filter shape, chfsi_filter with the tensor-core split product: a
    random Hermitian H (n x n), a random block Y0 (n x k), every column of
    degree m.  Per launch the method's complex work is 8 n^2 k m flops (m
    products H Y of k columns); the tensor cores execute 3x (BF16x3) or 6x
    (BF16x6) that in BF16 products.  The timed call also repacks H into its
    bf16 pieces and splits Y0; the kernel's own share comes from the
    library's kernel timer (filter launches only)."""
    import torch
    from paper_1404_4161_gb300.build import build
    build()
    from paper_1404_4161_gb300 import _lib as L
    from paper_1404_4161_gb300.solver import Chfsi, colmajor
    from workloads.synthetic import random_block
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, k, m = args.n or 4096, args.probe_k, args.probe_deg
    g = torch.Generator(device=dev).manual_seed(14044161 + 77)
    A = torch.randn(n, n, dtype=torch.complex128, device=dev, generator=g)
    H = (A + A.conj().t()) / (2.0 * n ** 0.5)  # spectrum within about [-2, 2]
    del A
    Hc = colmajor(H)
    del H
    Y0c = colmajor(torch.from_numpy(random_block(n, k, 14044161 + 78)).to(dev))
    split = L.SPLIT_BF16X3 if args.probe_split == "x3" else L.SPLIT_BF16X6
    s = Chfsi(precision=L.PREC_MIXED, split=split, profile=1)
    lz = s.lanczos(Hc, 20, 14044161 + 79)
    lo, hi = lz["theta_min"], lz["beta"]
    cut = lo + 0.1 * (hi - lo)  # filter interval [cut, hi], lam1 = lo
    c, e = 0.5 * (cut + hi), 0.5 * (hi - cut)
    deg = [m] * k
    stream = torch.cuda.current_stream()
    for _ in range(3):  # the first call also tunes the tiling of this shape
        out = s.filter(Hc, Y0c, deg, lo, c, e, precision=L.PREC_MIXED)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.probe_reps):
        out = s.filter(Hc, Y0c, deg, lo, c, e, precision=L.PREC_MIXED)
    b.record(stream)
    torch.cuda.synchronize()
    call_ms = a.elapsed_time(b) / args.probe_reps
    if not bool(torch.isfinite(torch.view_as_real(out)).all()):
        raise RuntimeError("filter probe: non-finite output")
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    pk = peaks.get("bf16_tflops", 1900.0)
    useful = 8.0 * n * n * k * m
    mult = 3.0 if split == L.SPLIT_BF16X3 else 6.0
    ex = useful * mult / (call_ms / 1e3) / 1e12
    print(json.dumps({"probe": "tc_filter_kernel via chfsi_filter", "n": n, "k": k, "degree": m,
                      "split": args.probe_split, "reps": args.probe_reps,
                      "ms_per_call": call_ms, "useful_tflops": useful / (call_ms / 1e3) / 1e12,
                      "executed_tflops": ex, "peak_bf16_burst": pk, "frac_of_burst": ex / pk,
                      "note": "call time includes the repack of H and the split of Y0",
                      "tiling": s.autotune_table()}))
    s.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.filter_probe:
        return filter_probe(args)
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1404_4161_gb300.build import build
    if rank == 0:
        build()
    if ws > 1:
        dist.barrier()
    from paper_1404_4161_gb300 import _lib as L
    from paper_1404_4161_gb300.solver import Chfsi, colmajor
    from workloads.synthetic import WORKLOADS, random_block

    cfg = WORKLOADS["seq10_n4096"]
    n = args.n or cfg.n
    nev, nex = sizes(cfg, n)
    k = nev + nex
    length = args.length or cfg.length
    from workloads.synthetic import config_sequence
    Hs, lam = config_sequence(cfg, 14044161 + 2000, length=length, n=n, device=dev)
    Hcs = [colmajor(h) for h in Hs]  # H Hermitian: column-major copy of H
    del Hs
    X0 = random_block(n, k, 14044161 + 2500)
    X0c = colmajor(torch.from_numpy(X0).to(dev))
    torch.cuda.synchronize()

    prec = {"tc": L.PREC_TC, "mixed": L.PREC_MIXED, "fp64": L.PREC_FP64}[args.precision]
    f64g = L.GEMM_OZAKI if (args.f64_gemm == "ozaki" and prec != L.PREC_FP64) else L.GEMM_FP64
    warm_rr = 1 if (prec == L.PREC_TC and args.warm_rr) else 0
    extra = {"deg_warm": args.deg_warm} if args.deg_warm else {}
    s = Chfsi(precision=prec, profile=1, f64_gemm=f64g, warm_rr=warm_rr,
              warm_resid=args.warm_resid, **extra)
    stream = torch.cuda.current_stream()
    train_info = None
    if args.degrees == "learned":
        # The degree MLP learns from traces the method itself generates, on a
        # separate training sequence (same generator, other seed); untimed.
        from paper_1404_4161_gb300 import learned
        train_len = args.train_length or length
        Ht, _ = config_sequence(cfg, 14044161 + 2700, length=train_len, n=n, device=dev)
        Htc = [colmajor(h) for h in Ht]
        del Ht
        s.trace_enable(1 << 20)
        Xt = colmajor(torch.from_numpy(random_block(n, k, 14044161 + 2750)).to(dev))
        s.solve_sequence(Htc, nev, nex, Xt, cfg.tol)
        xs, ys = learned.dataset(s)
        losses = learned.train(s, xs, ys, steps=3000, lr=2e-3)
        s.trace_enable(0)
        del Htc, Xt
        torch.cuda.empty_cache()
        train_info = {"rows": int(xs.shape[0]), "steps": 3000, "loss0": losses[0],
                      "loss": losses[-1], "train_problems": train_len}
        s.set_opts(degree_model=L.DEG_MLP)

    def step():
        Xc = X0c.clone()
        ev, sts, rc = s.solve_sequence(Hcs, nev, nex, Xc, cfg.tol)
        return ev, sts, rc, Xc

    def require_ok(rc, sts, what):
        bad = [l for l, x in enumerate(sts) if x["status"] != L.OK]
        if rc != L.OK or bad:
            raise RuntimeError(f"{what}: rc {rc}, problems not converged: {bad}")

    for _ in range(args.warmup):
        _, sts, rc, _ = step()
        require_ok(rc, sts, "warm-up step")
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stats_all, rcs = [], []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ev, sts, rc, Xc = step()
        stats_all.append(sts)
        rcs.append(rc)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    for rc, sts in zip(rcs, stats_all):
        require_ok(rc, sts, "timed step")
    from paper_1404_4161_gb300 import dist as D
    # every rank solved its own replica of the sequence: all ranks' problems
    # over the slowest rank's time
    sec_per_problem, t_max, _ = D.whole_job_seconds_per_unit(
        length, e0.elapsed_time(e1) / args.steps / 1e3, dev)
    ms = 1e3 * t_max
    ev_timed = ev.clone()

    # Certificate of the timed result, untimed: the same sequence problem by
    # problem through chfsi_solve (same arithmetic: warm start from the
    # previous problem's lam_1, lam_k, step index set), and for every
    # problem the residuals ||H x - lam x|| / ||H|| of the nev wanted pairs
    # in FP64 (torch on the device); the eigenvalues of the first and the
    # last problem against numpy's eigvalsh (LAPACK, host).
    cert = None
    if not args.no_certify:
        normH = max(abs(float(lam[0])), abs(float(lam[-1])))
        Xc = X0c.clone()
        warm, resid, same, statuses = None, [], 0.0, []
        for l in range(length):
            s.set_opts(step0=l)
            evl, stl, rcl = s.solve(Hcs[l], nev, nex, Xc, cfg.tol, warm=warm)
            statuses.append(int(stl["status"]))
            Xl = Xc.t()[:, :nev]
            Hl = Hcs[l].t()
            R = torch.linalg.vector_norm(Hl @ Xl - Xl * evl[:nev].to(Xl.dtype), dim=0)
            resid.append(float(R.max()) / normH)
            same = max(same, float((evl - ev_timed[l]).abs().max()))
            warm = (float(evl[0]), float(evl[-1]))
        s.set_opts(step0=0)
        eig_err = {}
        for l in sorted({0, length - 1}):
            w = np.linalg.eigvalsh(Hcs[l].t().cpu().numpy())
            eig_err[l] = float(np.abs(ev_timed[l, :nev].cpu().numpy() - w[:nev]).max() / normH)
        cert = {"status_per_problem": statuses, "max_resid_per_problem": resid,
                "max_resid_all": max(resid),
                "eigvalsh_err_rel_normH": {str(k): v for k, v in eig_err.items()},
                "max_abs_diff_vs_timed_evals": same}
        if max(statuses) != L.OK or max(resid) > cfg.tol or max(eig_err.values()) > 1e-12:
            raise RuntimeError(f"certificate failed: {cert}")

    last = stats_all[-1]
    filt_ms = sum(x["ms_filter"] for x in last)
    filt_flops = sum(x["filter_flops"] for x in last)
    filt_launch = sum(x["filter_launches"] for x in last)
    launches = sum(sum(x["launches"] for x in sts) for sts in stats_all)
    lowp_flops = sum(8.0 * n * n * x["col_degrees_lowp"] for x in last)
    filter_tflops = filt_flops / (filt_ms / 1e3) / 1e12 if filt_ms > 0 else 0.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    tot = lambda key: sum(x[key] for x in last)
    k64_ms, k64_fl, k64_fx, k64_n = (tot("k_f64_ms"), tot("k_f64_flops"),
                                     tot("k_f64_exec_flops"), tot("k_f64_launches"))
    ktc_ms, ktc_fl, ktc_n = tot("k_tc_ms"), tot("k_tc_flops"), tot("k_tc_launches")
    ktc_fx = tot("k_tc_exec_flops")
    FP64_PEAK = 1.10  # TFLOP/s, cuBLAS FP64 GEMM on this GB300 (python -m paper_1404_4161_gb300.peaks)
    bf16_peak = peaks.get("bf16_tflops_sustained", 1700.0)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    f64_roof = None
    if k64_ms > 0:
        a = k64_fl / (k64_ms / 1e3) / 1e12
        oz = f64g == L.GEMM_OZAKI
        ax = k64_fx / (k64_ms / 1e3) / 1e12  # executed: S(S+1)/2 BF16 slice products
        f64_roof = {"bound": "tensor" if oz else "alu",
                    "achieved": ax if oz else a,
                    "peak": bf16_peak if oz else FP64_PEAK, "unit": "TFLOP/s",
                    "frac": (ax / bf16_peak) if oz else a / FP64_PEAK, "traffic": None,
                    "fp64_equivalent_tflops": a,
                    "kernel": ("oz_gemm_kernel (FP64-accurate complex GEMM, S(S+1)/2 BF16 "
                               "slice products per product: 28 at S = 7, 36 at S = 8)") if oz else
                              "zgemm_nn_kernel + zgemm_cn_part_kernel (FP64 complex GEMMs)",
                    "launches": int(k64_n), "avg_launch_ms": k64_ms / max(k64_n, 1),
                    "peak_source": ("bf16_tflops_sustained of measured" if oz else
                                    "measured FP64 GEMM rate on this GB300 (no FP64 entry in "
                                    "MEASURED_PEAKS.json)")}
    tc_roof = None
    if ktc_ms > 0:
        a = ktc_fx / (ktc_ms / 1e3) / 1e12  # 3 or 6 BF16 products per complex product
        tc_roof = {"bound": "tensor", "achieved": a, "peak": bf16_peak, "unit": "TFLOP/s",
                   "frac": a / bf16_peak, "traffic": None,
                   "traffic_note": TC_FILTER_TRAFFIC_NOTE,
                   "probe_traffic": TC_FILTER_PROBE_TRAFFIC,
                   "useful_tflops": ktc_fl / (ktc_ms / 1e3) / 1e12,
                   "kernel": "tc_filter_kernel (persistent, all steps of a filter call in "
                             "one launch; BF16x3 / BF16x6 tcgen05, fused recurrence)",
                   "launches": int(ktc_n), "avg_launch_ms": ktc_ms / max(ktc_n, 1),
                   "peak_source": "bf16_tflops_sustained of measured"}
    lz_ms = tot("k_lanczos_ms")
    lz_roof = None
    if lz_ms > 0:
        # 20 Lanczos steps read the FP32 split of H (16 n^2 B) once each
        lz_bytes = length * 20 * 16.0 * n * n
        a = lz_bytes / (lz_ms / 1e3) / 1e9
        lz_roof = {"bound": "hbm", "achieved": a, "peak": hbm_peak, "unit": "GB/s",
                   "frac": a / hbm_peak, "traffic": None,
                   "kernel": "lanczos_persistent_kernel (20 steps, FP32 hi/lo split of H)",
                   "launches": length, "avg_launch_ms": lz_ms / length,
                   "peak_source": "hbm_gbs of measured"}
    # every timed kernel family, library or not; the roofline object is the
    # family with the most device time among those with a roofline
    kernel_ms = {"ozaki_gemm" if f64g == L.GEMM_OZAKI else "fp64_gemm": k64_ms,
                 "tc_filter": ktc_ms, "fp32_eig_start": tot("k_solver_ms"),
                 "cholinv": tot("k_cholinv_ms"), "lanczos": lz_ms,
                 "ozaki_slicers": tot("k_slice_ms"), "eig_control": tot("k_eigctl_ms")}
    kernel_ms["other (phases minus the above)"] = max(0.0, sum(
        x["ms_" + p] for x in last for p in ["lanczos", "filter", "qr", "rr", "resid", "lock"])
        - sum(kernel_ms.values()))
    cands = [r for r in (f64_roof, tc_roof, lz_roof) if r is not None]
    roof = max(cands, key=lambda r: r["avg_launch_ms"] * r["launches"]) if cands else None
    dominant = max(kernel_ms, key=kernel_ms.get)

    filter_tuning = s.autotune_table()

    # end to end: same solve through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        Hh = [h.cpu().pin_memory() for h in Hcs]
        X0h = X0c.cpu().pin_memory()
        Xh = X0h.clone().pin_memory()
        torch.cuda.synchronize()
        reps = max(1, min(args.steps, 2))
        t0 = time.perf_counter()
        for _ in range(reps):
            Xh.copy_(X0h)
            _, sts_h, rc_h = s.solve_sequence_host(Hh, nev, nex, Xh, cfg.tol)
            require_ok(rc_h, sts_h, "end-to-end step")
        t1 = time.perf_counter()
        e2e = {"value": (t1 - t0) / reps / (length * ws), "unit": UNIT,
               "h2d_bytes_per_step": int(length * 16 * n * n + 16 * n * k),
               "d2h_bytes_per_step": int(16 * n * k + 8 * length * k)}
        del Hh

    def timed_sequence(solver):
        Xc = X0c.clone()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, sts_x, rc_x = solver.solve_sequence(Hcs, nev, nex, Xc, cfg.tol)
        b.record(stream)
        torch.cuda.synchronize()
        require_ok(rc_x, sts_x, "comparison run")
        return a.elapsed_time(b) / 1e3, sts_x

    analytic_cmp = None
    if args.degrees == "learned":
        s.set_opts(degree_model=L.DEG_ANALYTIC)
        t_a, sts_a = timed_sequence(s)
        analytic_cmp = {"s_per_problem": t_a / length, "loops": [x["loops"] for x in sts_a],
                        "col_degrees": [x["col_degrees"] for x in sts_a]}
        s.set_opts(degree_model=L.DEG_MLP)

    fp64_cmp = None
    m64 = length if args.fp64_compare < 0 else min(args.fp64_compare, length)
    if m64 and prec != L.PREC_FP64:
        s64 = Chfsi(precision=L.PREC_FP64, warm_resid=1)
        Xw = X0c.clone()
        s64.solve(Hcs[0], nev, nex, Xw, cfg.tol)  # warm-up (kernels, workspaces)
        torch.cuda.synchronize()
        Xc = X0c.clone()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, sts64, rc64 = s64.solve_sequence(Hcs[:m64], nev, nex, Xc, cfg.tol)
        b.record(stream)
        torch.cuda.synchronize()
        require_ok(rc64, sts64, "FP64 comparison")
        fp64_cmp = {"s_per_problem": a.elapsed_time(b) / 1e3 / m64, "problems": m64,
                    "loops": [x["loops"] for x in sts64],
                    "same_sequence_as_headline": m64 == length,
                    "config": "FP64 filter, FP64 products, analytic degrees, warm starts with "
                              "residual-based first-loop degrees (opts.warm_resid = 1: one loop "
                              "per warm problem instead of two)"}
        s64.close()

    learned_protocol = None
    if args.learned_protocol and prec == L.PREC_TC:
        learned_protocol = measure_learned_protocol(dev, stream)

    batched = None
    if args.batched_scale > 0:
        batched = measure_batched(args.batched_scale, dev, stream, prec)
    batched_full = None
    if args.batched_full and prec == L.PREC_TC:
        batched_full = measure_batched_full(dev, stream)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        Hh_np = [h.t().cpu().numpy() for h in Hcs]
        cpu = cpu_baseline_sample(Hh_np, nev, nex, cfg.tol, X0, args.cpu_budget)

    if rank == 0:
        out = {
            "metric": METRIC, "value": sec_per_problem, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == L.PREC_FP64 else "bf16x3 (filter) + f64",
            "data": "synthetic",
            "config": {"workload": f"correlated sequence of {length} complex128 Hermitian "
                                   f"problems, n={n}, nev={nev}, nex={nex}, eps=1e-3, "
                                   f"delta=1e-4, tol 1e-10",
                       "precision": args.precision, "degree_model": args.degrees,
                       "f64_products": "ozaki (tensor cores)" if f64g == L.GEMM_OZAKI else "fp64 pipe",
                       "warm_rayleigh_ritz": bool(warm_rr),
                       "warm_residual_start": bool(args.warm_resid),
                       "l2": (f"inputs larger than L2 (each H is 16 n^2 = {16 * n * n / 1e6:.0f} MB)"
                              if 16 * n * n > 129e6 else
                              "inputs smaller than L2 (reduced-size run; not a bench value)"),
                       "parallelism": f"replicas x{ws}"},
            "status_per_problem": [int(x["status"]) for x in last],
            "filter_tflops": filter_tflops,
            "filter_tflops_lowp_share": lowp_flops / filt_flops if filt_flops else 0.0,
            "max_resid": cert["max_resid_all"] if cert else None,
            "certificate": cert,
            "loops": [x["loops"] for x in last],
            "col_degrees": [x["col_degrees"] for x in last],
            "phase_ms": {p: sum(x["ms_" + p] for x in last)
                         for p in ["lanczos", "filter", "qr", "rr", "resid", "lock"]},
            "kernel_ms": kernel_ms,
            "dominant_kernel_bucket": dominant,
            "roofline": roof,
            "filter_roofline": tc_roof,
            "fp64_gemm_roofline": f64_roof,
            "lanczos_roofline": lz_roof,
            "gpu_launches": int(launches),
            "filter_launches_per_step": int(filt_launch),
            "clocks": ck,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "fp64_gpu": fp64_cmp,
            "analytic_degrees_gpu": analytic_cmp,
            "mlp_training": train_info,
            "batched": batched,
            "batched64_full": batched_full,
            "loops_mlp": [x["loops_mlp"] for x in last],
            "filter_autotune": filter_tuning,
            "learned_protocol_n8192": learned_protocol,
        }
        print(json.dumps(out))
    s.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
