#!/usr/bin/env python
"""Benchmark of the GB300 blocked Jacobi library.

Default workload (the metric's own comparison, mixed + batched vs plain
FP64 at the same error): the mixed-precision two-sided blocked Jacobi EVD of a
dense symmetric n = 8192 matrix, b = 128 -- bf16 hi/lo x3 tensor-core updates
in the early sweeps, FP64 pivot solves, FP64 refinement and closing sweeps
with FP64-accurate tensor-core products -- eigenvalues plus the full
eigenvector matrix, gated at the FP64 tolerances.  Input: A = Q diag(lam) Q^T,
lam ~ U[-1, 1], Q Haar (Householder QR of a seeded Gaussian), seed 6.  Beside
it in the same line: the plain FP64 solve of the same matrix (`plain_fp64`,
one timed call, its accuracy at the same gates, and the ratio), and the three
batched forms (20000 symmetric matrices, n ~ U{8..512}, FP64 and FP32; 4096
tall 1024 x 64 FP32 SVDs), each next to the per-matrix plain FP64 path
(`batched`).  `--no-compare` leaves those out.  Other workloads
(--workload): the n = 256 and n = 4096 FP64 cases, the graded spectrum, the
one-sided SVD (direct, QR-preconditioned, emulated products), the other
mixed forms, and each batched form alone.

One step = one complete call (every sweep to convergence plus the
finalisation) on the resident input: jacobi_syev / jacobi_gesvd for a single
matrix, one plan execution over the whole batch for the batched forms.
Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on the same workload
  python bench.py --ncu-case             # a few single steps, for ncu captures

Under torchrun (N > 1) every rank solves its own replica of the workload
(the single-matrix path has no data-parallel split: replicas only; a batch
is independent problems, so each rank takes a full batch of its own: weak
scaling with no collective on the data path); the value is the matrices
solved by all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Jacobi matrices/s & eff. TFLOP/s: mixed+batched vs plain FP64, same error"
U64 = 2.0 ** -53

# FP64 pipe of GB300: 2 DFMA per clock per SM, 152 SMs, 2070 MHz maximum
# clock (nominal 1.25 TFLOP/s); a DFMA counts 2 flops.  FP32 pipe: 128 FFMA
# per clock per SM.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_BASIS = ("derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 pipe; "
              "measured DFMA loop 1.197 TFLOP/s on a GB300)")
FP32_BASIS = "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz (FP32 pipe)"


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}

WORKLOADS = {
    "evd4096": dict(kind="evd", n=4096, b=64, spectrum="uniform", seed=2, ref_sweeps=14,
                    desc="plain FP64 two-sided block Jacobi EVD, n=4096, b=64, round-robin, "
                         "eigenvalues + full Q, off(A) <= 1e-14 ||A||_F"),
    "evd4096emu": dict(kind="evd", n=4096, b=64, spectrum="uniform", seed=2, precision=5, ref_sweeps=14, compare_plain=True,
                       desc="two-sided block Jacobi EVD with FP64-accurate update products on the bf16 "
                            "tensor cores (eight 7-bit slices per operand), FP64 pivots and off-norm, "
                            "n=4096, b=64, round-robin, eigenvalues + full Q, off(A) <= 1e-14 ||A||_F"),
    "evd4096qrcp": dict(kind="evd", n=4096, b=64, spectrum="uniform", seed=2, ref_sweeps=14, pivot_order=2,
                        desc="plain FP64 two-sided block Jacobi EVD with the pivoting step of Sec. 2.1 (QRCP "
                             "of the leading rows of each pivot's eigenvectors), n=4096, b=64, round-robin, "
                             "eigenvalues + full Q, off(A) <= 1e-14 ||A||_F"),
    "evd256": dict(kind="evd", n=256, b=16, spectrum="uniform", seed=1, ref_sweeps=10,
                   desc="plain FP64 two-sided block Jacobi EVD, n=256, b=16, round-robin, "
                        "eigenvalues + full Q, off(A) <= 1e-14 ||A||_F"),
    "evd4096g": dict(kind="evd", n=4096, b=64, spectrum="graded", seed=3, ref_sweeps=29,
                     desc="plain FP64 two-sided block Jacobi EVD, n=4096, b=64, round-robin, "
                          "graded lam_i = +-10^(-12 i/(n-1)), eigenvalues + full Q, "
                          "off(A) <= 1e-14 ||A||_F"),
    "svd16384x2048": dict(kind="svd", m=16384, n=2048, b=64, seed=5, ref_sweeps=28,
                          desc="plain FP64 one-sided block Jacobi SVD, 16384 x 2048, b=64, "
                               "sigma_i = 10^(-10 i/(n-1)), U, sigma, V"),
    "svd16384x2048qr": dict(kind="svd", m=16384, n=2048, b=64, seed=5, svd_qr=1, ref_sweeps=10,
                            desc="one-sided block Jacobi SVD preconditioned by a reduced QR factorisation "
                                 "(blocked Householder QR in FP64, the one-sided method on R^T, U = Q W), "
                                 "16384 x 2048, b=64, sigma_i = 10^(-10 i/(n-1)), U, sigma, V"),
    "svd16384x2048qremu": dict(kind="svd", m=16384, n=2048, b=64, seed=5, svd_qr=1, precision=5, ref_sweeps=10,
                               desc="one-sided block Jacobi SVD preconditioned by a reduced QR factorisation "
                                    "(blocked Householder QR in FP64), the sweeps on R^T with the Gram and "
                                    "column products FP64-accurate on the bf16 tensor cores, FP64 pivots, "
                                    "16384 x 2048, b=64, sigma_i = 10^(-10 i/(n-1)), U, sigma, V"),
    "svd16384x2048emu": dict(kind="svd", m=16384, n=2048, b=64, seed=5, precision=5, ref_sweeps=28,
                             desc="one-sided block Jacobi SVD with the Gram and column products FP64-accurate "
                                  "on the bf16 tensor cores, FP64 pivots, 16384 x 2048, b=64, "
                                  "sigma_i = 10^(-10 i/(n-1)), U, sigma, V"),
    "mixed4096": dict(kind="evd", n=4096, b=64, spectrum="uniform", seed=2, precision=2, ref_sweeps=14, compare_plain=True,
                      refine_steps=2,
                      desc="mixed-precision two-sided block Jacobi EVD (bf16 hi/lo x3 tensor-core "
                           "updates, FP64 pivots, FP64 refinement + closing sweeps), n=4096, "
                           "b=64, lam ~ U[-1,1], eigenvalues + full Q, off <= 1e-14 ||A||_F"),
    "mixed8192": dict(kind="evd", n=8192, b=128, spectrum="uniform", seed=6, precision=2, ref_sweeps=14, compare_plain=True,
                      refine_steps=1,
                      desc="mixed-precision two-sided block Jacobi EVD (bf16 hi/lo x3 tensor-core "
                           "updates, FP64 pivots, FP64 refinement + closing sweeps), n=8192, "
                           "b=128, lam ~ U[-1,1], eigenvalues + full Q, off <= 1e-14 ||A||_F"),
    "mixed4096f16": dict(kind="evd", n=4096, b=64, spectrum="uniform", seed=2, precision=3,
                         refine_steps=2, ref_sweeps=14,
                         desc="mixed-precision two-sided block Jacobi EVD (fp16 hi/lo x3 tensor-core "
                              "updates with power-of-two scaling, FP64 pivots, FP64 refinement + closing "
                              "sweeps), n=4096, b=64, lam ~ U[-1,1], eigenvalues + full Q"),
    "mixed4096tf32": dict(kind="evd", n=4096, b=64, spectrum="uniform", seed=2, precision=4,
                          refine_steps=2, ref_sweeps=14,
                          desc="mixed-precision two-sided block Jacobi EVD (tf32 big/small x3 tensor-core "
                               "updates, FP64 pivots, FP64 refinement + closing sweeps), n=4096, b=64, "
                               "lam ~ U[-1,1], eigenvalues + full Q"),
    "mixed8192f16": dict(kind="evd", n=8192, b=128, spectrum="uniform", seed=6, precision=3,
                         refine_steps=1, ref_sweeps=14,
                         desc="mixed-precision two-sided block Jacobi EVD (fp16 hi/lo x3 tensor-core "
                              "updates with power-of-two scaling, FP64 pivots, FP64 refinement + closing "
                              "sweeps), n=8192, b=128, lam ~ U[-1,1], eigenvalues + full Q"),
    "mixed8192tf32": dict(kind="evd", n=8192, b=128, spectrum="uniform", seed=6, precision=4,
                          refine_steps=1, ref_sweeps=14,
                          desc="mixed-precision two-sided block Jacobi EVD (tf32 big/small x3 tensor-core "
                               "updates, FP64 pivots, FP64 refinement + closing sweeps), n=8192, b=128, "
                               "lam ~ U[-1,1], eigenvalues + full Q"),
    "mixed4096emu": dict(kind="evd", n=4096, b=64, spectrum="uniform", seed=2, precision=2, ref_sweeps=14, compare_plain=True,
                         refine_steps=2, fp64_products=1,
                         desc="mixed-precision two-sided block Jacobi EVD (bf16 hi/lo x3 tensor-core "
                              "updates, FP64 pivots, refinement and closing-sweep products FP64-accurate "
                              "on the bf16 tensor cores), n=4096, b=64, lam ~ U[-1,1], eigenvalues + full Q"),
    "mixed8192emu": dict(kind="evd", n=8192, b=128, spectrum="uniform", seed=6, precision=2, ref_sweeps=14,
                         refine_steps=2, switch_tol=1e-5, fp64_products=1, compare_plain=True, compare_batched=True,
                         desc="mixed-precision two-sided block Jacobi EVD (bf16 hi/lo x3 tensor-core "
                              "updates, FP64 pivots, refinement and closing-sweep products FP64-accurate "
                              "on the bf16 tensor cores), n=8192, b=128, lam ~ U[-1,1], eigenvalues + full Q"),
    "evd8192": dict(kind="evd", n=8192, b=128, spectrum="uniform", seed=6, ref_sweeps=14,
                    desc="plain FP64 two-sided block Jacobi EVD, n=8192, b=128, round-robin, "
                         "lam ~ U[-1,1], eigenvalues + full Q, off(A) <= 1e-14 ||A||_F"),
    "batched_f32": dict(kind="batched_evd", count=20000, lo=8, hi=512, seed=7, f32=True,
                        desc="batched FP32 EVD: 20000 symmetric (M+M^T)/2, M_ij ~ N(0,1), "
                             "n ~ U{8..512}, eigenvalues + Q, one plan execution per batch"),
    "batched_f64": dict(kind="batched_evd", count=20000, lo=8, hi=512, seed=7, f32=False,
                        desc="batched FP64 EVD: 20000 symmetric (M+M^T)/2, M_ij ~ N(0,1), "
                             "n ~ U{8..512}, eigenvalues + Q, one plan execution per batch"),
    "batched_svd_f32": dict(kind="batched_svd", count=4096, m=1024, n=64, seed=7, f32=True,
                            desc="batched FP32 one-sided Jacobi SVD: 4096 tall 1024 x 64, "
                                 "G_ij ~ N(0,1), U, sigma, V, one plan execution per batch"),
}


# ----------------------------------------------------------------------------- helpers
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate_max(value: float, world: int, device=None) -> float:
    """Max of a float over all ranks (identity at world size 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_sum(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def profile_traffic(name: str) -> tuple[float | None, str | None]:
    """DRAM bytes per launch recorded under profiles/<name>.md by an ncu
    capture, if the kernel's sources are unchanged since: the summary lists
    them (`source_files:`, names under the package's csrc/) with their hash
    (`source_sha256:`); without a list the hash covers every source."""
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None, None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    f = re.search(r"source_files:\s*([^\n]+)", txt)
    files = f.group(1).split() if f else None
    if not m or not h or h.group(1) != source_hash(files):
        return None, path
    return float(m.group(1)), path


def source_hash(files: list[str] | None = None) -> str:
    d = os.path.join(ROOT, "paper_2608_28952_gb300", "csrc")
    names = sorted(files) if files else sorted(f for f in os.listdir(d) if f.endswith((".cu", ".cpp", ".h", ".cuh")))
    hsh = hashlib.sha256()
    for f in names:
        p = os.path.join(d, f)
        hsh.update(open(p, "rb").read() if os.path.exists(p) else b"missing:" + f.encode())
    return hsh.hexdigest()[:16]


# ----------------------------------------------------------------------------- inputs
def make_input(wl):
    import jacobi_inputs as gen
    if wl["kind"] == "evd":
        A, lam = gen.sym_known(wl["n"], wl["spectrum"], seed=wl["seed"])
        return A, lam
    G, sig = gen.svd_known(wl["m"], wl["n"], seed=wl["seed"], decades=10.0)
    return G, sig


def evd_update_flops(np_, b):
    """Algorithmic flops of one update launch (one step) of the symmetric
    two-sided formulation: A'_{P1P2} = V1^T A_{P1P2} V2 over the P(P-1)/2
    off-diagonal pair-blocks (2 GEMMs of 2k^3 each, k = 2b, P = np/(2b)) plus
    Q'(:,P) = Q(:,P) V_P (2 np k^2 per pair)."""
    k = 2 * b
    P = np_ // k
    return P * (P - 1) // 2 * 4 * k ** 3 + P * 2 * np_ * k * k


# ----------------------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(wl, sweeps: int, budget_s: float = 10.0, start_step: int = 0,
                      max_steps: int | None = None):
    """Time the CPU oracle on consecutive steps of the workload's first sweep
    (with vectors) until budget_s has passed; return seconds per step, the
    number of steps per sweep and the once-per-matrix seconds (the QR
    factorisation and U = Q W of the QR form, else 0)."""
    import numpy as np
    import oracle
    A, _ = make_input(wl)
    extra = 0.0
    b = wl["b"]
    if wl["kind"] == "evd":
        n = wl["n"]
        N = oracle.padded_blocks(n, b)
        tab = oracle.ordering(oracle.ORDER_ROUND_ROBIN, N)
        Ak = np.zeros((N * b, N * b), order="F")
        Ak[:n, :n] = A
        Qk = np.eye(N * b)
        run = lambda s, X, Y: oracle.syev_step(X, Y, b, tab[s])[:2]
    else:
        m, n = wl["m"], wl["n"]
        N = oracle.padded_blocks(n, b)
        tab = oracle.ordering(oracle.ORDER_ROUND_ROBIN, N)
        if wl.get("svd_qr"):
            # the oracle's QR form: LAPACK QR through numpy, the one-sided
            # steps on R^T, and U = Q W (timed once on a stand-in W)
            t1 = time.perf_counter()
            Qf, R = np.linalg.qr(A, mode="reduced")
            t2 = time.perf_counter()
            _ = Qf @ np.eye(n)
            extra = (t2 - t1) + (time.perf_counter() - t2)
            A = np.asfortranarray(np.triu(R).T)
            m = n
        Ak = np.zeros((m, N * b), order="F")
        Ak[:, :n] = A
        Qk = np.eye(N * b)
        tol = oracle.svd_tol(m)
        cap = 2 if wl.get("svd_qr") else 30   # the library's automatic inner-sweep caps
        run = lambda s, X, Y: oracle.gesvd_step(X, Y, b, tab[s], tol_rel=tol, inner_max=cap)[:2]
    S = len(tab)
    done, t0 = 0, time.perf_counter()
    times = []
    while True:
        s = (start_step + done) % S
        t1 = time.perf_counter()
        Ak, Qk = run(s, Ak, Qk)
        times.append(time.perf_counter() - t1)
        done += 1
        if time.perf_counter() - t0 >= budget_s or (max_steps and done >= max_steps):
            break
    return times, S, extra


def cpu_baseline(wl, sweeps: int, budget_s: float = 12.0):
    times, S, extra = cpu_oracle_sample(wl, sweeps, budget_s)
    t_step = sum(times) / len(times)
    t_matrix = t_step * S * sweeps + extra
    cores = len(os.sched_getaffinity(0))
    qr = (f" on R^T, plus {extra:.1f} s for the QR factorisation and U = Q W (LAPACK/BLAS "
          f"through numpy)") if extra else ""
    return {"value": 1.0 / t_matrix, "unit": "matrices/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} consecutive parallel steps from the start of sweep 1 "
                      f"({S} per sweep, with vectors){qr}, "
                      f"{sum(times):.1f} s, extrapolated x{S} steps x{sweeps} sweeps "
                      f"(the GPU run's sweep count); OpenMP over the pairs of a step",
            "seconds_per_step": t_step, "measured_s": sum(times), "steps_sampled": len(times),
            "extrapolated": True, "extrapolation_factor": S * sweeps}


# ----------------------------------------------------------------------------- reference arm
def run_reference_batched(args, wl):
    shapes = batch_shapes(wl)
    B = len(shapes)
    mats = batched_host_sample(wl, shapes, 256)
    rates = []
    cores = len(os.sched_getaffinity(0))
    secs_all = []
    for i in range(args.warmup + args.steps):
        secs, done, frac = batched_cpu_sample(wl, shapes, mats, budget_s=6.0, threads=cores)
        mats = mats[done:] + mats[:done]  # the next step starts where this one ended
        rates.append(secs / frac)
        secs_all.append(secs)
    t_batch = sum(rates[args.warmup:]) / args.steps
    value = B / t_batch
    evd = wl["kind"] == "batched_evd"
    sample = (f"each step = the FP64 oracle (scalar parallel-ordered Jacobi per matrix, one "
              f"matrix per thread on {cores} threads) on consecutive matrices of the batch for 6 s, "
              f"extrapolated by {'n^3' if evd else 'm n^2'} work to all {B} matrices")
    ms_sample = 1e3 * sum(secs_all[args.warmup:]) / args.steps
    return value, ms_sample, sample, t_batch / (ms_sample / 1e3)


def workload_config(wl, world: int) -> dict:
    """The `config` object of a workload's bench line: what is solved, with
    its sizes and seed (the same object in the GPU arm and the reference
    arm, so the two lines name the same configuration)."""
    if wl["kind"] in ("batched_evd", "batched_svd"):
        evd = wl["kind"] == "batched_evd"
        return {"workload": wl["desc"], "count": wl["count"], "seed": wl["seed"],
                **({"n_range": [wl["lo"], wl["hi"]]} if evd else {"m": wl["m"], "n": wl["n"]}),
                "parallelism": f"one batch per rank x{world}",
                "l2": "inputs larger than L2 (the whole batch, GBs)"}
    prec = wl.get("precision", 0)
    return {"workload": wl["desc"], "b": wl["b"], "n": wl["n"],
            **({"m": wl["m"]} if "m" in wl else {}),
            "seed": wl["seed"], "parallelism": f"replicas x{world}",
            **({"svd_qr": True} if wl.get("svd_qr") else {}),
            **({"pivot_order": wl["pivot_order"]} if "pivot_order" in wl else {}),
            **({"precision": {2: "mixed bf16x3", 3: "mixed fp16x3", 4: "mixed tf32x3",
                              5: "fp64 emulated products"}[prec],
                "refine_steps": wl.get("refine_steps")} if prec else {}),
            **({"switch_tol": wl["switch_tol"]} if "switch_tol" in wl else {}),
            **({"fp64_products": True} if wl.get("fp64_products") else {}),
            "l2": "inputs larger than L2 (working A, Q double-buffered: 4 x n^2 x 8 B)"}


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    if wl["kind"] in ("batched_evd", "batched_svd"):
        value, ms_step, sample, factor = run_reference_batched(args, wl)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matrices/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(wl, args.gpus),
                "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": cores,
                                 "kind": "oracle", "sample": sample, "extrapolated": True,
                                 "extrapolation_factor": factor},
                "ms_per_step_basis": "measured wall time of one sampled step (6 s of oracle work)",
                "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    sweeps = wl["ref_sweeps"]   # the oracle's own sweep count on this input (one full solve)
    times, S, extra = cpu_oracle_sample(wl, sweeps, budget_s=1e9, max_steps=args.warmup + args.steps)
    timed = times[args.warmup:]
    t_step = sum(timed) / len(timed)
    value = 1.0 / (t_step * S * sweeps + extra)
    sample = (f"each step = one parallel step (of {S} per sweep, with vectors) of the FP64 oracle on "
              f"the workload's matrix, OpenMP over the pairs of the step on {cores} cores; the rate is "
              f"extrapolated x{S} steps x{sweeps} sweeps (the oracle's own sweep count on this input, "
              f"from a full solve); first-sweep steps cost more than later ones, so this overstates "
              f"the full solve's time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matrices/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, args.gpus),
            "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": cores,
                             "kind": "oracle", "sample": sample, "extrapolated": True,
                             "extrapolation_factor": S * sweeps, "seconds_per_step": t_step},
            "ms_per_step_basis": "measured wall time of one sampled oracle step (one parallel "
                                 "step of the sweep); value = 1 / (that time x steps x sweeps)",
            "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def padded_np(n, b):
    N = (n + b - 1) // b
    N += N & 1
    return N * b


def evd_kernel_classes(stats, wl, peaks):
    """Device time, launches and issued flops per kernel class of the
    two-sided solve (summed over the timed steps), each with its roofline."""
    b = wl["b"]
    npd = padded_np(wl["n"], b)
    S = npd // b - 1
    lowp_steps = sum(st.sweeps_lowp for st in stats) * S
    tot = lambda f: sum(getattr(st, f) for st in stats)
    bf16 = peaks.get("bf16_tflops_sustained")
    emu = wl.get("precision", 0) == 5 or wl.get("fp64_products", 0) == 1
    # an emulated FP64 product issues 36 bf16 slice products per FP64 product
    emu_slice = 36 * tot("flops_update") if emu else 0
    cls = {
        "pivot": dict(kernel="k_pivot / k_pivot_cluster", ms=tot("ms_pivot"),
                      launches=tot("pivot_launches"),
                      flops=tot("flops_fp64") - (0 if emu else tot("flops_update")) - tot("flops_refine"),
                      bound="alu", peak=FP64_PEAK_TFLOPS, peak_basis=FP64_BASIS),
    }
    if emu:
        # FP64-accurate products from bf16 slices: the roofline is the bf16
        # tensor pipe on the issued slice products; the FP64-equivalent rate
        # is reported beside it
        ms_emu = tot("ms_update") - tot("ms_update_lowp")
        cls["update_emu"] = dict(kernel="k_emu_upd1 + k_emu_upd2 (tcgen05, FP64-accurate)",
                                 ms=ms_emu, launches=tot("update_launches") - 3 * lowp_steps,
                                 flops=emu_slice, bound="tensor", peak=bf16,
                                 peak_basis="measured bf16 dense, sustained (MEASURED_PEAKS.json); "
                                            "flops = the 36 bf16 slice products issued",
                                 fp64_equiv_tflops=(tot("flops_update") / (ms_emu / 1e3) / 1e12
                                                    if ms_emu > 0 else None))
    else:
        cls["update_fp64"] = dict(kernel="k_update_evd", ms=tot("ms_update") - tot("ms_update_lowp"),
                                  launches=tot("update_launches") - 3 * lowp_steps,
                                  flops=tot("flops_update"), bound="alu", peak=FP64_PEAK_TFLOPS,
                                  peak_basis=FP64_BASIS)
    if tot("sweeps_lowp") > 0:
        cls["update_lowp"] = dict(kernel="k_tc_split_v + k_tc_upd1 + k_tc_upd2 (tcgen05)",
                                  ms=tot("ms_update_lowp"), launches=3 * lowp_steps,
                                  flops=tot("flops_lowp") - emu_slice, bound="tensor",
                                  peak=bf16, peak_basis="measured bf16 dense, sustained "
                                  "(MEASURED_PEAKS.json); flops = the three bf16 products issued")
        if emu:
            cls["refine"] = dict(kernel="k_emu_gemm_big (tcgen05, FP64-accurate; + elementwise)",
                                 ms=tot("ms_refine"), launches=None, flops=36 * tot("flops_refine"),
                                 bound="tensor", peak=bf16,
                                 peak_basis="measured bf16 dense, sustained (MEASURED_PEAKS.json); "
                                            "flops = the 36 bf16 slice products issued",
                                 fp64_equiv_tflops=(tot("flops_refine") / (tot("ms_refine") / 1e3) / 1e12
                                                    if tot("ms_refine") > 0 else None))
        else:
            cls["refine"] = dict(kernel="k_gemm64 (+ elementwise)", ms=tot("ms_refine"),
                                 launches=None, flops=tot("flops_refine"), bound="alu",
                                 peak=FP64_PEAK_TFLOPS, peak_basis=FP64_BASIS)
    for c in cls.values():
        c["achieved"] = c["flops"] / (c["ms"] / 1e3) / 1e12 if c["ms"] > 0 else None
        c["frac"] = c["achieved"] / c["peak"] if c["achieved"] and c["peak"] else None
        c["unit"] = "TFLOP/s"
    if "update_lowp" in cls:
        # HBM view of the tensor-core update: per step A, Q (FP32) read and
        # written once, the stage-1 products T written and read once
        k = 2 * b
        P = npd // k
        per_step = 4 * (4 * npd * npd) + 2 * 4 * (P * (P - 1) // 2) * k * k
        c = cls["update_lowp"]
        c["hbm_bytes_per_step"] = per_step
        c["hbm_gbs"] = per_step * lowp_steps / (c["ms"] / 1e3) / 1e9 if c["ms"] > 0 else None
        c["hbm_peak_gbs"] = peaks.get("hbm_gbs")
    return cls


def qr_precond_flops(m, n, nb=32):
    """FP64-equivalent flops of the QR preconditioning as the library counts
    them, split into the panel work (reflectors, T, Y T: always FP64) and the
    blocked products (W = Y^T X and X -= (Y T) W for the trailing matrix
    and for U = Q W), which run on the emulated tensor-core products when
    those are on.  Leading terms: products 6 m n^2 - 8 n^3 / 3."""
    panel = prod = 0.0
    for j0 in range(0, n, nb):
        nbp, rows = min(nb, n - j0), m - j0
        nc = n - j0 - nbp
        panel += 5.0 * rows * nbp * nbp + 2.0 * rows * nbp * nbp
        prod += 4.0 * rows * nbp * nc + 4.0 * rows * nbp * n
    return panel, prod


def svd_kernel_classes(stats, wl, peaks):
    """Device time, issued flops and roofline of the one-sided solve's kernel
    classes (summed over the timed steps): Gram + column update, the Gram
    pivots and, for the QR form, the QR preconditioning."""
    tot = lambda f: sum(getattr(st, f) for st in stats)
    qr = bool(wl.get("svd_qr"))
    emu = wl.get("precision", 0) == 5 or wl.get("fp64_products", 0) == 1
    kernels = {"update": dict(kernel="k_gram + k_update_cols", ms=tot("ms_update"),
                              launches=tot("update_launches"), flops=tot("flops_update")),
               "pivot": dict(kernel="k_pivot / k_pivot_cluster (Gram pivots)", ms=tot("ms_pivot"),
                             launches=tot("pivot_launches"),
                             flops=tot("flops_fp64") - (0 if emu else tot("flops_update"))
                             - tot("flops_precond"))}
    if qr:
        kernels["precond"] = dict(kernel="k_house_vec + k_house_apply + k_qr_ytx + k_gemm64 "
                                         "(Householder QR and U = Q W, FP64)",
                                  ms=tot("ms_precond"), launches=None, flops=tot("flops_precond"))
    for c in kernels.values():
        c.update(bound="alu", peak=FP64_PEAK_TFLOPS, peak_basis=FP64_BASIS, unit="TFLOP/s")
    if emu:
        # FP64-accurate products from bf16 slices: the tensor pipe on the
        # issued slice products, the FP64-equivalent rate beside it
        u = kernels["update"]
        u.update(kernel="k_emu_gram + k_emu_cols (tcgen05, FP64-accurate)", flops=36 * tot("flops_update"),
                 bound="tensor", peak=peaks.get("bf16_tflops_sustained"),
                 peak_basis="measured bf16 dense, sustained (MEASURED_PEAKS.json); "
                            "flops = the 36 bf16 slice products issued",
                 fp64_equiv_tflops=(tot("flops_update") / (u["ms"] / 1e3) / 1e12 if u["ms"] > 0 else None))
        if qr:
            # the blocked products of the QR and of U = Q W are emulated, the
            # panels stay FP64: the tensor pipe on the issued slice products
            # over the whole class time (panel kernels included: a lower bound)
            c = kernels["precond"]
            panel, prod = qr_precond_flops(wl["m"], wl["n"])
            c.update(kernel="k_house_vec + k_house_apply + k_gemm64 (FP64 panels) + k_emu_line_exps + k_emu_gemm_big + "
                            "k_emu_sum_t (trailing, Q and Q W products, tcgen05, FP64-accurate)",
                     flops=36 * prod * len(stats), flops_fp64_panels=panel * len(stats),
                     bound="tensor", peak=peaks.get("bf16_tflops_sustained"),
                     peak_basis="measured bf16 dense, sustained (MEASURED_PEAKS.json); flops = the 36 bf16 "
                                "slice products issued, time = the whole class (FP64 panels included)",
                     fp64_equiv_tflops=(tot("flops_precond") / (c["ms"] / 1e3) / 1e12 if c["ms"] > 0 else None))
    for c in kernels.values():
        c["achieved"] = c["flops"] / (c["ms"] / 1e3) / 1e12 if c["ms"] > 0 else None
        c["frac"] = c["achieved"] / c["peak"] if c["achieved"] and c["peak"] else None
    return kernels


def evd_accuracy(X, lam_true, w, V, dev) -> dict:
    """Eigenvalue errors against the constructed spectrum, residual and
    orthogonality of a solve (FP64 products on the GPU)."""
    import numpy as np
    import torch
    n = X.shape[0]
    wv = w.cpu().numpy()
    lam = np.sort(lam_true)
    big = np.abs(lam) >= 1e-3 * np.abs(lam).max()
    acc = {"max_abs_eig_err_over_norm2": float(np.abs(wv - lam).max() / np.abs(lam).max()),
           "max_rel_eig_err_abs_ge_1e-3": float((np.abs(wv - lam)[big] / np.abs(lam[big])).max())}
    A64 = torch.from_numpy(np.asarray(X)).to(dev)
    R = A64 @ V - V * w[None, :]
    acc["residual_fro_over_normA"] = float(torch.linalg.norm(R) / torch.linalg.norm(A64))
    del R
    acc["orth_fro_over_n"] = float(torch.linalg.norm(V.t() @ V - torch.eye(n, device=dev,
                                                                           dtype=torch.float64)) / n)
    del A64
    return acc


def evd_gates(acc: dict) -> dict:
    """The FP64 gates of the two-sided solve (the stated target for plain
    FP64; the mixed forms are held to the same gates here)."""
    g = {"eig_le_1e-13": acc["max_abs_eig_err_over_norm2"] <= 1e-13,
         "residual_le_1e-12": acc["residual_fro_over_normA"] <= 1e-12,
         "orth_le_1e-13_n": acc["orth_fro_over_n"] <= 1e-13}
    g["all"] = all(g.values())
    return g


def plain_fp64_solve(wl, X, lam, dev, stream) -> dict:
    """The plain FP64 solve (DFMA products, the library's defaults) of the
    workload's matrix at the same block size: one jacobi_syev call on the
    resident input, timed with CUDA events on the stream."""
    import torch

    import paper_2608_28952_gb300 as jg
    n = X.shape[0]
    p = jg.params(b=wl["b"])
    Xd = jg.colmajor(X, device=dev, dtype=torch.float64)
    w = torch.empty(n, dtype=torch.float64, device=dev)
    V = jg.colmajor_empty(n, n, torch.float64, dev)
    sampler = ClockSampler(gpu_uuid(torch, dev))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    rc, st = jg.jacobi_syev(Xd, w, V, p, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    if rc != 0:
        raise RuntimeError(f"plain FP64 solve: status {rc}")
    ms = e0.elapsed_time(e1)
    del Xd
    acc = evd_accuracy(X, lam, w, V, dev)
    del w, V
    return {"value": 1e3 / ms, "unit": "matrices/s", "ms": ms, "sweeps": st.sweeps,
            "steps": 1, "warmup": 0, "precision": "fp64 (DFMA products)", "b": wl["b"],
            "timing": "CUDA events around one jacobi_syev call on the resident input, after the "
                      "timed steps (context and modules loaded)",
            "phases_ms": {"pivot": st.ms_pivot, "update": st.ms_update, "total": st.ms_total},
            "eff_tflops_issued": st.flops_fp64 / (st.ms_total / 1e3) / 1e12,
            "accuracy": acc, "accuracy_gates": evd_gates(acc), "clocks": clocks}


def run_gpu(args, wl):
    if wl["kind"] in ("batched_evd", "batched_svd"):
        return run_batched(args, wl)
    import numpy as np
    import torch

    import paper_2608_28952_gb300 as jg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    jg.lib()
    peaks = measured_peaks()
    stream = torch.cuda.current_stream(dev)
    X, ref = make_input(wl)
    b = wl["b"]
    prec = wl.get("precision", 0)
    extra = {k: wl[k] for k in ("refine_steps", "switch_tol", "fp64_products", "svd_qr", "pivot_order") if k in wl}
    p = jg.params(b=b, inner_max_sweeps=args.inner_max_sweeps, precision=prec, **extra)
    Xd = jg.colmajor(X, device=dev, dtype=torch.float64)
    Wd = torch.empty_like(Xd.t()).t()  # column-major work copy
    if wl["kind"] == "evd":
        n = wl["n"]
        out = torch.empty(n, dtype=torch.float64, device=dev)
        V = jg.colmajor_empty(n, n, torch.float64, dev)
        call = lambda: jg.jacobi_syev(Wd, out, V, p, stream)
    else:
        m, n = wl["m"], wl["n"]
        out = torch.empty(n, dtype=torch.float64, device=dev)
        V = jg.colmajor_empty(n, n, torch.float64, dev)
        call = lambda: jg.jacobi_gesvd(Wd, out, V, p, stream)

    def step():
        Wd.copy_(Xd)
        rc, st = call()
        if rc != 0:
            raise RuntimeError(f"status {rc} ({jg.status_string(rc)})")
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier(world)
    sampler = ClockSampler(gpu_uuid(torch, dev))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    stats = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms_max = aggregate_max(ms, world, dev)
    total = aggregate_sum(float(args.steps), world, dev)
    value = total / (ms_max / 1e3)

    # accuracy of the last step (outside the timed region)
    if wl["kind"] == "evd":
        acc = evd_accuracy(X, ref, out, V, dev)
    else:
        acc = {}
        s = out.cpu().numpy()
        acc["max_abs_sigma_err_over_sigma_max"] = float(np.abs(s - ref).max() / ref[0])
        big = ref >= 1e-3 * ref[0]
        acc["max_rel_sigma_err_sigma_ge_1e-3"] = float((np.abs(s - ref)[big] / ref[big]).max())

    sweeps = stats[-1].sweeps
    flops_issued = sum(st.flops_fp64 for st in stats)
    launches = int(sum(st.launches for st in stats))

    # roofline of the dominant kernel class
    if wl["kind"] == "evd":
        kernels = evd_kernel_classes(stats, wl, peaks)
        dom = max(kernels, key=lambda c: kernels[c]["ms"])
        kc = kernels[dom]
        if dom in ("update_fp64", "update_emu", "pivot") and kc["launches"]:
            avg_ms = kc["ms"] / kc["launches"]
            per_launch = kc["flops"] / kc["launches"]
        else:
            avg_ms, per_launch = kc["ms"], kc["flops"]
        npd = padded_np(wl["n"], b)
        prof_name = {"update_fp64": f"update_evd_n{wl['n']}_b{b}",
                     "update_emu": f"emu_update_n{wl['n']}_b{b}",
                     "pivot": f"pivot_n{wl['n']}_b{b}",
                     "refine": f"gemm64_n{wl['n']}",
                     "update_lowp": f"tc_update_n{wl['n']}_b{b}"}[dom]
        traffic, prof = profile_traffic(prof_name)
        roofline = {"kernel": kc["kernel"], "class": dom, "bound": kc["bound"],
                    "achieved": kc["achieved"], "peak": kc["peak"], "unit": "TFLOP/s",
                    "frac": kc["frac"], "traffic": traffic, "peak_basis": kc["peak_basis"],
                    "flops_per_launch_issued": per_launch, "avg_launch_ms": avg_ms,
                    "alg_update_flops_per_step_full": evd_update_flops(npd, b),
                    "share_of_step": kc["ms"] / ms if ms else None,
                    "profile": os.path.relpath(prof, ROOT) if prof else None}
    else:
        m, n_ = wl["m"], wl["n"]
        m_eff = n_ if wl.get("svd_qr") else m   # with QR preconditioning the sweeps run on R^T
        emu = prec == 5 or wl.get("fp64_products", 0) == 1
        kernels = svd_kernel_classes(stats, wl, peaks)
        dom = max(kernels, key=lambda c: kernels[c]["ms"])
        kc = kernels[dom]
        k = 2 * b
        P = ((n_ + b - 1) // b + 1) // 2
        npd = 2 * P * b
        # Gram (lower triangle, split-K) + column update of G and V, per step
        alg = P * (m_eff * k * k + 2 * m_eff * k * k + 2 * npd * k * k)
        if kc["launches"]:
            # the update class counts two launches per step (Gram, columns)
            per = kc["launches"] // 2 if dom == "update" else kc["launches"]
            avg_ms, per_launch = kc["ms"] / max(per, 1), kc["flops"] / max(per, 1)
        else:
            avg_ms, per_launch = kc["ms"], kc["flops"]
        prof_name = {"update": f"svd_update_m{m_eff}_n{n_}_b{b}", "pivot": f"pivot_svd_n{n_}_b{b}",
                     "precond": f"qr_m{m}_n{n_}"}[dom]
        traffic, prof = profile_traffic(prof_name)
        if emu and dom == "update":
            prof_name = f"emu_svd_update_m{m_eff}_n{n_}_b{b}"
            traffic, prof = profile_traffic(prof_name)
        roofline = {"kernel": kc["kernel"], "class": dom, "bound": kc["bound"], "achieved": kc["achieved"],
                    "peak": kc["peak"], "unit": "TFLOP/s", "frac": kc["frac"], "traffic": traffic,
                    "peak_basis": kc["peak_basis"], "alg_update_flops_per_step_full": alg,
                    "flops_per_launch_issued": per_launch, "avg_launch_ms": avg_ms,
                    "share_of_step": kc["ms"] / ms if ms else None,
                    "profile": os.path.relpath(prof, ROOT) if prof else None}

    # end to end: the same calls with host buffers, copies inside the timing
    e2e = None
    if args.e2e_steps > 0:
        Xh = jg.colmajor(X, dtype=torch.float64).pin_memory()
        Wh = jg.colmajor_empty(X.shape[0], X.shape[1], torch.float64, "cpu").pin_memory()
        oh = torch.empty(out.shape[0], dtype=torch.float64).pin_memory()
        Vh = jg.colmajor_empty(V.shape[0], V.shape[1], torch.float64, "cpu").pin_memory()
        fh = jg.jacobi_syev_h if wl["kind"] == "evd" else jg.jacobi_gesvd_h
        tt = 0.0
        for i in range(args.e2e_steps + 1):
            Wh.copy_(Xh)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            rc, _ = fh(Wh, oh, Vh, p, stream)
            t1 = time.perf_counter()
            if rc != 0:
                raise RuntimeError(f"e2e status {rc}")
            if i > 0:  # the first call warms the host-buffer path
                tt += t1 - t0
        tt_max = aggregate_max(tt, world, dev)
        e_total = aggregate_sum(float(args.e2e_steps), world, dev)
        h2d = X.shape[0] * X.shape[1] * 8
        d2h = (X.shape[0] * X.shape[1] + out.shape[0] + V.shape[0] * V.shape[1]) * 8
        e2e = {"value": e_total / tt_max, "unit": "matrices/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "timing": "wall clock around each jacobi_*_h call (pinned host buffers)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, sweeps)

    # the metric's comparisons (one GPU, rank 0 alone): the plain FP64 solve of
    # the same matrix, and the batched forms next to the per-matrix FP64 path
    plain = batched = None
    if world == 1 and not args.no_compare and wl.get("compare_plain"):
        del Wd, V, out
        torch.cuda.empty_cache()
        plain = plain_fp64_solve(wl, X, ref, dev, stream)
    if world == 1 and not args.no_compare and wl.get("compare_batched"):
        batched = {}
        for name in ("batched_f64", "batched_f32", "batched_svd_f32"):
            torch.cuda.empty_cache()
            bl = measure_batched(WORKLOADS[name], 1, 1, 0, not args.no_cpu_baseline, 1, dev, stream,
                                 plain_loop_s=6.0)
            batched[name] = {k: bl.get(k) for k in (
                "value", "unit", "dtype", "ms_per_step", "steps", "warmup", "config", "plan",
                "accuracy", "roofline", "cpu_baseline", "plain_fp64_loop", "vs_plain_fp64_loop",
                "gpu_launches", "clocks")}

    if rank == 0:
        st = stats[-1]
        line = {"metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == 0 else ("f64 (products from bf16 slices)" if prec == 5 else
                                                  {2: "bf16x3", 3: "fp16x3", 4: "tf32x3"}[prec] + "+f32+f64"),
                "data": "synthetic (seeded; see config)",
                "config": workload_config(wl, world),
                "eff_tflops_issued": (sum(st_.flops_fp64 + st_.flops_lowp for st_ in stats)
                                      / (sum(st_.ms_total for st_ in stats) / 1e3) / 1e12),
                "sweeps": sweeps, "sweeps_lowp": st.sweeps_lowp,
                "inner_max_sweeps": args.inner_max_sweeps,
                "phases_ms_last_step": {"lowp": st.ms_lowp, "refine": st.ms_refine,
                                        "pivot": st.ms_pivot, "update": st.ms_update,
                                        "total": st.ms_total},
                "pivot_stats": {"pair_solves": st.pair_solves,
                                "inner_sweeps_per_solve": st.inner_sweeps / max(1, st.pair_solves),
                                "rotations": st.rotations},
                "accuracy": acc, "kernels": kernels,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "source_sha256": source_hash()}
        if wl["kind"] == "evd":
            line["accuracy_gates"] = evd_gates(acc)
        if plain is not None:
            line["plain_fp64"] = plain
            line["vs_plain_fp64"] = value / plain["value"]
            line["same_error"] = {"this": evd_gates(acc), "plain_fp64": plain["accuracy_gates"],
                                  "gates": "|lambda - lambda_true| <= 1e-13 ||A||_2, "
                                           "||AQ - QD||_F <= 1e-12 ||A||_F, ||Q^T Q - I||_F <= 1e-13 n"}
        if batched is not None:
            line["batched"] = batched
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ----------------------------------------------------------------------------- batched forms
def batch_shapes(wl):
    import jacobi_inputs as gen
    if wl["kind"] == "batched_evd":
        return [(int(n), int(n)) for n in gen.batch_sizes(wl["count"], wl["lo"], wl["hi"], wl["seed"])]
    return [(wl["m"], wl["n"])] * wl["count"]


def batched_cpu_sample(wl, shapes, mats_host, budget_s: float, max_items: int | None = None,
                       threads: int = 1):
    """The oracle on consecutive matrices of the batch (LPT order is not
    used: matrices are taken as listed) until budget_s has passed, one
    matrix per thread at a time on `threads` threads (the ctypes calls
    release the interpreter lock; each oracle call runs on one core).
    Returns (wall seconds, matrices done, work done / work of the whole
    batch)."""
    import threading

    import numpy as np
    import oracle
    evd = wl["kind"] == "batched_evd"
    work = lambda mn: mn[1] ** 3 if evd else mn[0] * mn[1] ** 2
    total_work = sum(work(x) for x in shapes)
    lim = len(mats_host) if not max_items else min(max_items, len(mats_host))
    lock = threading.Lock()
    state = {"next": 0, "done": 0, "work": 0}
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                i = state["next"]
                if i >= lim or time.perf_counter() - t0 >= budget_s:
                    return
                state["next"] = i + 1
            A = mats_host[i]
            if evd:
                n = A.shape[0]
                k = n + (n & 1)
                Ap = np.zeros((k, k))
                Ap[:n, :n] = A
                oracle.pivot_solve(Ap)
            else:
                n = A.shape[1]
                oracle.gesvd(A, b=max(1, n // 2), threads=1)
            with lock:
                state["done"] += 1
                state["work"] += work(shapes[i])

    ts = [threading.Thread(target=worker) for _ in range(max(1, threads))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return time.perf_counter() - t0, state["done"], state["work"] / total_work


def batched_host_sample(wl, shapes, count: int):
    """The first `count` matrices of the batch as float64 numpy arrays.  They
    are drawn on the CUDA device when there is one, which reproduces the GPU
    run's matrices exactly (same seeded generator, same draws); without a
    GPU, torch's CPU generator gives other draws of the same distribution."""
    import torch
    import jacobi_inputs as gen
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    flat, views, _ = gen.batch_flat_torch(shapes[:count], wl["seed"], dev, torch.float64,
                                          symmetric=wl["kind"] == "batched_evd")
    out = [v.cpu().numpy() for v in views]
    del flat, views
    return out


def run_batched(args, wl):
    import torch

    import paper_2608_28952_gb300 as jg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    jg.lib()
    stream = torch.cuda.current_stream(dev)
    line = measure_batched(wl, args.steps, args.warmup, args.e2e_steps,
                           rank == 0 and world == 1 and not args.no_cpu_baseline, world, dev, stream)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def measure_batched(wl, steps, warmup, e2e_steps, want_cpu, world, dev, stream,
                    plain_loop_s: float = 0.0):
    """One batched workload: `warmup` untimed plan executions, `steps` timed
    ones (CUDA events on the stream), accuracy on a spread sample, roofline,
    end-to-end executions from pinned host memory, the CPU oracle and, when
    plain_loop_s > 0, the per-matrix plain FP64 path (jacobi_syev /
    jacobi_gesvd called matrix by matrix) sampled for that many seconds.
    Returns the bench line (a dict)."""
    import numpy as np
    import torch

    import jacobi_inputs as gen
    import paper_2608_28952_gb300 as jg

    evd = wl["kind"] == "batched_evd"
    dtype = torch.float32 if wl["f32"] else torch.float64
    shapes = batch_shapes(wl)
    B = len(shapes)
    flat0, views0, offs = gen.batch_flat_torch(shapes, wl["seed"], dev, dtype, symmetric=evd)
    flat = flat0.clone()
    X = [flat[o:o + m * n].view(n, m).t() for (m, n), o in zip(shapes, offs)]
    ncols = [n for _, n in shapes]
    y_off = np.concatenate([[0], np.cumsum(ncols)]).astype(np.int64)
    z_off = np.concatenate([[0], np.cumsum([n * n for n in ncols])]).astype(np.int64)
    yflat = torch.empty(int(y_off[-1]), dtype=dtype, device=dev)
    zflat = torch.empty(int(z_off[-1]), dtype=dtype, device=dev)
    Y = [yflat[int(y_off[i]):int(y_off[i + 1])] for i in range(B)]
    Z = [zflat[int(z_off[i]):int(z_off[i + 1])].view(n, n).t() for i, n in enumerate(ncols)]
    info = torch.full((B,), -7, dtype=torch.int32, device=dev)
    prec = jg.PREC_FP32 if wl["f32"] else jg.PREC_FP64
    plan = jg.Plan(0 if evd else 1, prec, ncols, m=None if evd else [m for m, _ in shapes],
                   p=jg.params(), stream=stream)
    t0 = time.perf_counter()
    if evd:
        plan.autotune(X, Y, Z, info, stream)
    tune_s = time.perf_counter() - t0
    shape = plan.shape()
    blocking = plan.blocking()

    def step():
        flat.copy_(flat0)
        rc, st = plan.execute(X, Y, Z, info, stream)
        if rc != 0:
            raise RuntimeError(f"status {rc} ({jg.status_string(rc)})")
        return st

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    if int((info != 0).sum()) != 0:
        raise RuntimeError(f"{int((info != 0).sum())} matrices did not converge")
    barrier(world)
    sampler = ClockSampler(gpu_uuid(torch, dev))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    stats = [step() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms_max = aggregate_max(ms, world, dev)
    total = aggregate_sum(float(steps * B), world, dev)
    value = total / (ms_max / 1e3)
    bad = int((info != 0).sum())

    # accuracy on a spread sample (LAPACK on the host as the witness)
    acc = {"matrices_not_converged": bad}
    idx = list(range(0, B, max(1, B // 16)))[:16]
    e_eig = e_res = e_orth = 0.0
    for i in idx:
        A = views0[i].double().cpu().numpy()
        y = Y[i].double().cpu().numpy()
        Zi = Z[i].double().cpu().numpy()
        n = A.shape[1]
        if evd:
            ref = np.linalg.eigvalsh(A)
            e_eig = max(e_eig, float(np.abs(y - ref).max() / max(np.abs(ref).max(), 1e-300)))
            e_res = max(e_res, float(np.linalg.norm(A @ Zi - Zi * y[None, :]) / np.linalg.norm(A)))
        else:
            ref = np.linalg.svd(A, compute_uv=False)
            e_eig = max(e_eig, float(np.abs(y - ref).max() / ref[0]))
            U = X[i].double().cpu().numpy()
            e_res = max(e_res, float(np.linalg.norm(A @ Zi - U * y[None, :]) / np.linalg.norm(A)))
        e_orth = max(e_orth, float(np.linalg.norm(Zi.T @ Zi - np.eye(n)) / n))
    acc.update({"sample": len(idx), "max_abs_err_over_norm2": e_eig,
                "max_residual_fro_over_normA": e_res, "max_orth_fro_over_n": e_orth,
                "witness": "numpy.linalg (LAPACK) on the sampled matrices"})

    st = stats[-1]
    f_issued = (st.flops_fp32 if wl["f32"] else st.flops_fp64)
    peak = FP32_PEAK_TFLOPS if wl["f32"] else FP64_PEAK_TFLOPS
    achieved = f_issued / (st.ms_total / 1e3) / 1e12
    kname = "k_batched_evd" if evd else (
        "k_batched_svd" if os.environ.get("JACOBI_BATCHED_SVD") == "rowwise" else "k_batched_svd_tiled")
    traffic, prof = profile_traffic(f"{kname}_{'f32' if wl['f32'] else 'f64'}_{B}")
    roofline = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "peak_basis": FP32_BASIS if wl["f32"] else FP64_BASIS,
                "flops_per_launch_issued": f_issued, "avg_launch_ms": st.ms_total,
                "launches_per_step": st.launches,
                "profile": os.path.relpath(prof, ROOT) if prof else None}

    e2e = None
    if e2e_steps > 0:
        hx = flat0.cpu().pin_memory()
        hy = torch.empty_like(yflat, device="cpu").pin_memory()
        hz = torch.empty_like(zflat, device="cpu").pin_memory()
        hu = torch.empty_like(flat, device="cpu").pin_memory() if not evd else None
        tt = 0.0
        for i in range(e2e_steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            flat.copy_(hx, non_blocking=True)
            rc, _ = plan.execute(X, Y, Z, info, stream)
            hy.copy_(yflat, non_blocking=True)
            hz.copy_(zflat, non_blocking=True)
            if hu is not None:
                hu.copy_(flat, non_blocking=True)
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            if rc != 0:
                raise RuntimeError(f"e2e status {rc}")
            if i > 0:
                tt += t1 - t0
        tt_max = aggregate_max(tt, world, dev)
        e_total = aggregate_sum(float(e2e_steps * B), world, dev)
        esz = flat.element_size()
        e2e = {"value": e_total / tt_max, "unit": "matrices/s",
               "h2d_bytes_per_step": flat.numel() * esz,
               "d2h_bytes_per_step": (yflat.numel() + zflat.numel()
                                      + (flat.numel() if hu is not None else 0)) * esz,
               "steps": e2e_steps,
               "timing": "wall clock: pinned host -> device copy of the batch, plan "
                         "execution, device -> pinned host copy of the results"}
        del hx, hy, hz, hu
    plan.close()
    del flat, yflat, zflat, X, Y, Z

    cpu = None
    if want_cpu:
        mats = batched_host_sample(wl, shapes, 512)
        cores = len(os.sched_getaffinity(0))
        secs, done, frac = batched_cpu_sample(wl, shapes, mats, budget_s=8.0, threads=cores)
        cpu = {"value": B / (secs / frac), "unit": "matrices/s", "cores": cores, "kind": "oracle",
               "sample": f"the first {done} matrices of the batch ({frac:.2e} of its "
                         f"{'n^3' if evd else 'm n^2'} work), {secs:.1f} s wall on {cores} threads "
                         f"(one matrix per thread at a time), extrapolated by work to all {B}; "
                         f"FP64 oracle (scalar parallel-ordered Jacobi per matrix)",
               "extrapolated": True, "extrapolation_factor": 1.0 / frac, "measured_s": secs}

    plain = None
    if plain_loop_s > 0:
        plain = plain_loop_sample(wl, shapes, views0, plain_loop_s, dev, stream)
    del flat0, views0

    line = {"metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": ms_max / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if wl["f32"] else "f64", "data": "synthetic (seeded; see config)",
            "config": workload_config(wl, world),
            "plan": {"shape": {"threads": shape[0], "smem_kmax": shape[1], "grid": shape[2]},
                     "blocking": {"b": blocking[0], "unblocked_up_to_order": blocking[1]},
                     "autotune_s": tune_s,
                     "batch_gb": sum(m * n for m, n in shapes) * (4 if wl["f32"] else 8) / 1e9},
            "eff_tflops_issued": achieved, "accuracy": acc,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(sum(s_.launches for s_ in stats)), "clocks": clocks,
            "source_sha256": source_hash()}
    if plain is not None:
        line["plain_fp64_loop"] = plain
        line["vs_plain_fp64_loop"] = value / plain["value"] if plain["value"] else None
    return line


def plain_loop_sample(wl, shapes, views, budget_s, dev, stream):
    """The per-matrix plain FP64 path on the batch: jacobi_syev (jacobi_gesvd
    for the tall batch) called matrix by matrix on FP64 copies of the first
    matrices, b = 16, until budget_s has passed; the rate is extrapolated to
    the whole batch by n^3 (m n^2) work."""
    import torch

    import paper_2608_28952_gb300 as jg
    evd = wl["kind"] == "batched_evd"
    work = lambda mn: mn[1] ** 3 if evd else mn[0] * mn[1] ** 2
    total_work = sum(work(x) for x in shapes)
    secs, done, w = 0.0, 0, 0
    p = jg.params(b=16)
    for i, (m, n) in enumerate(shapes):
        X = views[i].double().t().contiguous().t()
        out = torch.empty(n, dtype=torch.float64, device=dev)
        V = jg.colmajor_empty(n, n, torch.float64, dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rc, _ = (jg.jacobi_syev if evd else jg.jacobi_gesvd)(X, out, V, p, stream)
        secs += time.perf_counter() - t0
        if rc != 0:
            raise RuntimeError(f"plain FP64 path: status {rc}")
        done += 1
        w += work((m, n))
        if secs >= budget_s:
            break
    frac = w / total_work
    return {"value": len(shapes) / (secs / frac), "unit": "matrices/s",
            "sample": f"{'jacobi_syev' if evd else 'jacobi_gesvd'} (FP64, b=16) on the first {done} "
                      f"matrices ({frac:.2e} of the batch's {'n^3' if evd else 'm n^2'} work), "
                      f"{secs:.1f} s wall clock around the calls, extrapolated by work",
            "extrapolated": True, "extrapolation_factor": 1.0 / frac, "measured_s": secs}


def run_ncu_case(args, wl):
    """A handful of single steps of the workload (for ncu captures): FP64
    steps, or low-precision steps for the mixed workloads; for a batch, one
    plan execution over its 32 largest matrices."""
    import torch

    import paper_2608_28952_gb300 as jg
    if wl["kind"] in ("batched_evd", "batched_svd"):
        import jacobi_inputs as gen
        dev = torch.device("cuda", 0)
        evd = wl["kind"] == "batched_evd"
        shapes = sorted(batch_shapes(wl), key=lambda mn: -mn[0] * mn[1] * mn[1])[:32]
        dtype = torch.float32 if wl["f32"] else torch.float64
        flat, X, _ = gen.batch_flat_torch(shapes, wl["seed"], dev, dtype, symmetric=evd)
        Y = [torch.empty(n, dtype=dtype, device=dev) for _, n in shapes]
        Z = [jg.colmajor_empty(n, n, dtype, dev) for _, n in shapes]
        info = torch.zeros(len(shapes), dtype=torch.int32, device=dev)
        plan = jg.Plan(0 if evd else 1, jg.PREC_FP32 if wl["f32"] else jg.PREC_FP64, [n for _, n in shapes],
                       m=None if evd else [m for m, _ in shapes], p=jg.params())
        rc, _ = plan.execute(X, Y, Z, info)
        torch.cuda.synchronize()
        assert rc == 0 and int((info != 0).sum()) == 0
        plan.close()
        print(json.dumps({"ncu_case": wl["desc"], "matrices": len(shapes)}))
        return 0
    X, _ = make_input(wl)
    if wl.get("svd_qr"):
        # the sweeps of the QR form run on R^T (n x n): the same step kernels
        import numpy as np
        X = np.asfortranarray(np.triu(np.linalg.qr(X, mode="r")).T)
    dev = torch.device("cuda", 0)
    mixed = wl.get("precision", 0) in (2, 3, 4)
    dt = torch.float32 if mixed else torch.float64
    Xd = jg.colmajor(X, device=dev, dtype=dt)
    Qd = jg.colmajor(torch.eye(X.shape[0], dtype=dt), device=dev)
    p = jg.params(b=wl["b"], precision=wl.get("precision", 0))
    for s in range(args.warmup + args.steps):
        if wl["kind"] == "evd":
            f = jg.jacobi_syev_step_lowp if mixed else jg.jacobi_syev_step
            rc = f(Xd, Qd, s % (X.shape[0] // wl["b"] - 1), p)
        else:
            rc, _ = jg.jacobi_gesvd_step(Xd, None, s % (X.shape[1] // wl["b"] - 1), p)
        assert rc == 0, rc
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": wl["desc"], "steps": args.warmup + args.steps}))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="mixed8192emu", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--inner-max-sweeps", type=int, default=0,
                    help="cap on the sweeps of one pivot solve (0 = the library's automatic choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the plain FP64 solve and the batched forms beside the default line")
    ap.add_argument("--ncu-case", action="store_true")
    args = ap.parse_args(argv)
    if args.warmup < 3 and not args.ncu_case:
        ap.error("--warmup must be >= 3")
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.ncu_case:
        return run_ncu_case(args, wl)
    return run_gpu(args, wl)


if __name__ == "__main__":
    sys.exit(main())
