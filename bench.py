#!/usr/bin/env python
"""Benchmark of the GB300 blocked Jacobi library.

Default workload: plain FP64 two-sided blocked Jacobi EVD of a dense
symmetric n = 4096 matrix, b = 64, round-robin ordering, eigenvalues plus the
full eigenvector matrix, stop at off(A) <= 1e-14 ||A||_F.  Input: A = Q diag(lam)
Q^T, lam ~ U[-1, 1], Q Haar (Householder QR of a seeded Gaussian), seed 2.

One step = one complete jacobi_syev call (every sweep to convergence plus
the finalisation) on the resident input.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on the same workload
  python bench.py --ncu-case             # a few single steps, for ncu captures

Under torchrun (N > 1) every rank solves its own replica of the workload
(the single-matrix path has no data-parallel split: replicas only); the
value is the matrices solved by all ranks over the slowest rank's time.
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
# clock (nominal 1.25 TFLOP/s); a DFMA counts 2 flops.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

WORKLOADS = {
    "evd4096": dict(kind="evd", n=4096, b=64, spectrum="uniform", seed=2,
                    desc="plain FP64 two-sided block Jacobi EVD, n=4096, b=64, round-robin, "
                         "eigenvalues + full Q, off(A) <= 1e-14 ||A||_F"),
    "evd256": dict(kind="evd", n=256, b=16, spectrum="uniform", seed=1,
                   desc="plain FP64 two-sided block Jacobi EVD, n=256, b=16, round-robin, "
                        "eigenvalues + full Q, off(A) <= 1e-14 ||A||_F"),
    "svd16384x2048": dict(kind="svd", m=16384, n=2048, b=64, seed=5,
                          desc="plain FP64 one-sided block Jacobi SVD, 16384 x 2048, b=64, "
                               "sigma_i = 10^(-10 i/(n-1)), U, sigma, V"),
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
    capture, if the kernel sources are unchanged since (same source hash)."""
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None, None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != source_hash():
        return None, path
    return float(m.group(1)), path


def source_hash() -> str:
    d = os.path.join(ROOT, "paper_2608_28952_gb300", "csrc")
    hsh = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cpp", ".h", ".cuh")):
            hsh.update(open(os.path.join(d, f), "rb").read())
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
    (with vectors) until budget_s has passed; return seconds per step and the
    number of steps timed."""
    import numpy as np
    import oracle
    A, _ = make_input(wl)
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
        Ak = np.zeros((m, N * b), order="F")
        Ak[:, :n] = A
        Qk = np.eye(N * b)
        tol = oracle.svd_tol(m)
        run = lambda s, X, Y: oracle.gesvd_step(X, Y, b, tab[s], tol_rel=tol)[:2]
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
    return times, S


def cpu_baseline(wl, sweeps: int, budget_s: float = 12.0):
    times, S = cpu_oracle_sample(wl, sweeps, budget_s)
    t_step = sum(times) / len(times)
    t_matrix = t_step * S * sweeps
    cores = len(os.sched_getaffinity(0))
    return {"value": 1.0 / t_matrix, "unit": "matrices/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} of the {S} parallel steps of sweep 1 (with vectors), "
                      f"{sum(times):.1f} s, extrapolated x{S} steps x{sweeps} sweeps "
                      f"(the GPU run's sweep count); OpenMP over the pairs of a step",
            "seconds_per_step": t_step}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    sweeps = wl.get("ref_sweeps", 9)
    times, S = cpu_oracle_sample(wl, sweeps, budget_s=1e9, max_steps=args.warmup + args.steps)
    timed = times[args.warmup:]
    t_step = sum(timed) / len(timed)
    value = 1.0 / (t_step * S * sweeps)
    cores = len(os.sched_getaffinity(0))
    sample = (f"each step = one parallel step (of {S} per sweep) of the oracle on the workload, "
              f"extrapolated x{S} x{sweeps} sweeps")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matrices/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step * S * sweeps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"]},
            "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args, wl):
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
    stream = torch.cuda.current_stream(dev)
    X, ref = make_input(wl)
    b = wl["b"]
    p = jg.params(b=b, inner_max_sweeps=args.inner_max_sweeps)
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
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
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
    acc = {}
    if wl["kind"] == "evd":
        w = out.cpu().numpy()
        lam = np.sort(ref)
        acc["max_abs_eig_err_over_norm2"] = float(np.abs(w - lam).max() / np.abs(lam).max())
        A64 = torch.from_numpy(np.asarray(X)).to(dev)
        R = A64 @ V - V * out[None, :]
        acc["residual_fro_over_normA"] = float(torch.linalg.norm(R) / torch.linalg.norm(A64))
        acc["orth_fro_over_n"] = float(torch.linalg.norm(V.t() @ V - torch.eye(n, device=dev,
                                                           dtype=torch.float64)) / n)
        del A64, R
    else:
        s = out.cpu().numpy()
        acc["max_abs_sigma_err_over_sigma_max"] = float(np.abs(s - ref).max() / ref[0])
        big = ref >= 1e-3 * ref[0]
        acc["max_rel_sigma_err_sigma_ge_1e-3"] = float((np.abs(s - ref)[big] / ref[big]).max())

    sweeps = stats[-1].sweeps
    flops_issued = sum(st.flops_fp64 for st in stats)
    ms_update = sum(st.ms_update for st in stats)
    ms_pivot = sum(st.ms_pivot for st in stats)
    n_upd = sum(st.update_launches for st in stats)
    n_piv = sum(st.pivot_launches for st in stats)
    launches = int(sum(st.launches for st in stats))

    # roofline of the dominant kernel (FP64 pipe: plain ALU arithmetic)
    kernels = {"update": {"ms": ms_update, "launches": n_upd},
               "pivot": {"ms": ms_pivot, "launches": n_piv}}
    upd_flops = sum(st.flops_update for st in stats)
    if wl["kind"] == "evd":
        npd = ((wl["n"] + b - 1) // b + 1) // 2 * 2 * b
        alg = evd_update_flops(npd, b)
        avg_ms = ms_update / max(n_upd, 1)
        # issued work: pair-blocks whose two pivots did not rotate are copies
        alg_issued = upd_flops / max(n_upd, 1)
        achieved = alg_issued / (avg_ms / 1e3) / 1e12
        traffic, prof = profile_traffic("update_evd_n4096_b64") if wl["n"] == 4096 else (None, None)
        kname = "k_update_evd"
    else:
        m, n_ = wl["m"], wl["n"]
        k = 2 * b
        P = ((n_ + b - 1) // b + 1) // 2
        npd = 2 * P * b
        # Gram (lower triangle, split-K) + column update of G and V, per step
        alg = P * (m * k * k + 2 * m * k * k + 2 * npd * k * k)
        avg_ms = ms_update / max(n_upd // 2, 1)
        alg_issued = upd_flops / max(n_upd // 2, 1)
        achieved = alg_issued / (avg_ms / 1e3) / 1e12
        traffic, prof = (None, None)
        kname = "k_gram + k_update_cols"
    sm_mhz = clocks.get("sm_mhz")
    roofline = {"kernel": kname, "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": traffic,
                "peak_basis": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 pipe; "
                              "measured DFMA loop 1.197 TFLOP/s on this pool)",
                "alg_flops_per_launch_full": alg, "flops_per_launch_issued": alg_issued,
                "avg_launch_ms": avg_ms,
                "share_of_step": ms_update / ms if ms else None}

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

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded; see config)",
                "config": {"workload": wl["desc"], "b": b,
                           "n": wl["n"], **({"m": wl["m"]} if "m" in wl else {}),
                           "seed": wl["seed"], "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (working A, Q double-buffered: "
                                 "4 x n^2 x 8 B)"},
                "eff_tflops_issued": flops_issued / (sum(st.ms_total for st in stats) / 1e3) / 1e12,
                "sweeps": sweeps, "inner_max_sweeps": args.inner_max_sweeps,
                "pivot_stats": {"pair_solves": stats[-1].pair_solves,
                                "inner_sweeps_per_solve": stats[-1].inner_sweeps / max(1, stats[-1].pair_solves),
                                "rotations": stats[-1].rotations},
                "accuracy": acc, "kernels": kernels,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "source_sha256": source_hash()}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_ncu_case(args, wl):
    """A handful of single steps of the workload (for ncu captures)."""
    import torch

    import paper_2608_28952_gb300 as jg
    X, _ = make_input(wl)
    dev = torch.device("cuda", 0)
    Xd = jg.colmajor(X, device=dev, dtype=torch.float64)
    Qd = jg.colmajor(torch.eye(X.shape[0], dtype=torch.float64), device=dev)
    p = jg.params(b=wl["b"])
    for s in range(args.warmup + args.steps):
        if wl["kind"] == "evd":
            rc = jg.jacobi_syev_step(Xd, Qd, s % (X.shape[0] // wl["b"] - 1), p)
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
    ap.add_argument("--workload", default="evd4096", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--inner-max-sweeps", type=int, default=0,
                    help="cap on the sweeps of one pivot solve (0 = the library's automatic choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
