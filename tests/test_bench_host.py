"""Host-side logic of bench.py: the cross-rank aggregation of the N-GPU
launch (run here as two gloo ranks on the CPU), the workload table, the
algorithmic work counts and the kernel-class roofline bookkeeping."""
from __future__ import annotations

import os
import socket
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank measured its own replica: time differs, matrices add up
    t = bench.aggregate_max(10.0 + rank, world)
    n = bench.aggregate_sum(3.0, world)
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, t, n))


def test_aggregation_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time and the total work
    assert out == [(0, 11.0, 6.0), (1, 11.0, 6.0)]


def test_single_rank_aggregation_is_identity():
    assert bench.aggregate_max(2.5, 1) == 2.5
    assert bench.aggregate_sum(4.0, 1) == 4.0


def test_workloads_are_complete():
    for name, wl in bench.WORKLOADS.items():
        assert wl["kind"] in ("evd", "svd", "batched_evd", "batched_svd"), name
        assert "desc" in wl and "seed" in wl
    # the five configurations of the workload description are all present
    assert bench.WORKLOADS["evd256"]["n"] == 256 and bench.WORKLOADS["evd256"]["b"] == 16
    assert bench.WORKLOADS["evd4096"]["n"] == 4096 and bench.WORKLOADS["evd4096"]["b"] == 64
    assert bench.WORKLOADS["svd16384x2048"]["m"] == 16384
    assert bench.WORKLOADS["mixed8192"]["n"] == 8192 and bench.WORKLOADS["mixed8192"]["b"] == 128
    assert bench.WORKLOADS["batched_f64"]["count"] == 20000
    assert bench.WORKLOADS["batched_svd_f32"]["count"] == 4096
    # the reference arm extrapolates by the oracle's own sweep count on each input
    for name, wl in bench.WORKLOADS.items():
        if wl["kind"] in ("evd", "svd"):
            assert isinstance(wl.get("ref_sweeps"), int) and wl["ref_sweeps"] >= 1, name


def test_padding_and_update_flops():
    assert bench.padded_np(4096, 64) == 4096
    assert bench.padded_np(100, 16) == 128       # 7 blocks -> 8
    assert bench.padded_np(96, 16) == 96
    # one step at np = 4096, b = 64: 32 pairs, 496 pair-blocks of 4 k^3 plus Q
    k = 128
    assert bench.evd_update_flops(4096, 64) == 496 * 4 * k ** 3 + 32 * 2 * 4096 * k * k


def _stats(**kw):
    """A stand-in for the library's Stats with every field the accounting reads."""
    base = dict(ms_update=0.0, update_launches=0, flops_update=0.0, ms_pivot=0.0, pivot_launches=0,
                flops_fp64=0.0, flops_precond=0.0, ms_precond=0.0, flops_lowp=0.0, ms_update_lowp=0.0,
                sweeps_lowp=0, ms_refine=0.0, flops_refine=0.0)
    base.update(kw)
    return SimpleNamespace(**base)


def test_kernel_classes_plain_fp64():
    wl = dict(n=4096, b=64)
    st = _stats(ms_pivot=1000.0, pivot_launches=819, flops_fp64=8e12, flops_update=7e12,
                ms_update=5500.0, update_launches=819)
    cls = bench.evd_kernel_classes([st], wl, {})
    assert set(cls) == {"pivot", "update_fp64"}
    assert cls["update_fp64"]["launches"] == 819
    assert cls["update_fp64"]["achieved"] == pytest.approx(7e12 / 5.5 / 1e12)
    assert cls["pivot"]["flops"] == pytest.approx(1e12)


def test_kernel_classes_mixed_split_the_phases():
    wl = dict(n=4096, b=64)
    S = 63
    st = _stats(sweeps_lowp=11, ms_pivot=1100.0, pivot_launches=13 * S, flops_fp64=2.5e12,
                flops_update=1.0e12, flops_refine=1.2e12, ms_update=1300.0, ms_update_lowp=500.0,
                update_launches=3 * 11 * S + 2 * S, flops_lowp=1.75e13, ms_refine=1000.0)
    cls = bench.evd_kernel_classes([st], wl, {"bf16_tflops_sustained": 1688.5, "hbm_gbs": 6777.0})
    assert cls["update_lowp"]["launches"] == 3 * 11 * S
    assert cls["update_fp64"]["launches"] == 2 * S
    assert cls["update_fp64"]["ms"] == pytest.approx(800.0)
    assert cls["update_lowp"]["bound"] == "tensor" and cls["update_lowp"]["peak"] == 1688.5
    assert cls["pivot"]["flops"] == pytest.approx(2.5e12 - 1.0e12 - 1.2e12)
    assert cls["update_lowp"]["hbm_gbs"] > 0


def test_batch_shapes_follow_the_recipe():
    wl = bench.WORKLOADS["batched_f32"]
    sh = bench.batch_shapes(wl)
    assert len(sh) == 20000 and all(m == n and 8 <= n <= 512 for m, n in sh)
    sv = bench.batch_shapes(bench.WORKLOADS["batched_svd_f32"])
    assert sv == [(1024, 64)] * 4096


def test_cpu_sample_of_the_qr_form_runs_the_oracle_on_r_transpose():
    """The CPU baseline of the QR-preconditioned SVD: numpy's QR once, then
    the oracle's one-sided steps on the n x n R^T (small case)."""
    wl = dict(kind="svd", m=120, n=24, b=4, seed=5, svd_qr=1, desc="small QR form")
    times, S, extra = bench.cpu_oracle_sample(wl, sweeps=3, budget_s=0.01, max_steps=2)
    assert S == 5 and len(times) >= 1 and extra > 0.0
    wl_direct = dict(kind="svd", m=120, n=24, b=4, seed=5, desc="small direct form")
    times2, S2, extra2 = bench.cpu_oracle_sample(wl_direct, sweeps=3, budget_s=0.01, max_steps=2)
    assert S2 == 5 and extra2 == 0.0


def test_new_workloads_carry_their_options():
    assert bench.WORKLOADS["svd16384x2048qr"]["svd_qr"] == 1
    assert bench.WORKLOADS["svd16384x2048qremu"]["precision"] == 5
    assert bench.WORKLOADS["mixed8192emu"]["fp64_products"] == 1


def test_svd_kernel_classes_direct_qr_and_emulated():
    peaks = {"bf16_tflops_sustained": 1688.5}
    st = _stats(ms_update=1000.0, update_launches=620, flops_update=1e12, ms_pivot=500.0, pivot_launches=310,
                flops_fp64=1.2e12 + 5e11, flops_precond=5e11, ms_precond=400.0)
    # direct FP64: update flops are FP64 flops, pivot = the rest of flops_fp64
    k = bench.svd_kernel_classes([st], dict(m=16384, n=2048, b=64), peaks)
    assert set(k) == {"update", "pivot"} and k["update"]["bound"] == "alu"
    assert abs(k["update"]["achieved"] - 1.0) < 1e-12          # 1e12 flops in 1 s
    assert abs(k["pivot"]["flops"] - (1.7e12 - 1e12 - 5e11)) < 1.0
    # QR form: the preconditioning is its own class
    k = bench.svd_kernel_classes([st], dict(m=16384, n=2048, b=64, svd_qr=1), peaks)
    assert set(k) == {"update", "pivot", "precond"} and k["precond"]["ms"] == 400.0
    # emulated products: the update class counts the 36 slice products against bf16
    k = bench.svd_kernel_classes([st], dict(m=16384, n=2048, b=64, svd_qr=1, precision=5), peaks)
    assert k["update"]["bound"] == "tensor" and k["update"]["flops"] == 36e12
    assert abs(k["update"]["fp64_equiv_tflops"] - 1.0) < 1e-12
    assert abs(k["pivot"]["flops"] - (1.7e12 - 5e11)) < 1.0     # emulated updates add no FP64 flops
    # ... and the QR's blocked products: tensor-bound on their issued slice products
    panel, prod = bench.qr_precond_flops(16384, 2048)
    assert k["precond"]["bound"] == "tensor" and k["precond"]["flops"] == 36 * prod
    assert k["precond"]["flops_fp64_panels"] == panel
    assert abs(k["precond"]["fp64_equiv_tflops"] - 5e11 / 0.4 / 1e12) < 1e-12
    k = bench.svd_kernel_classes([st], dict(m=16384, n=2048, b=64, svd_qr=1), peaks)
    assert k["precond"]["bound"] == "alu" and k["precond"]["flops"] == 5e11


@pytest.mark.parametrize("m,n", [(16384, 2048), (4096, 4096), (3000, 1000), (100, 37)])
def test_qr_precond_flops_leading_terms(m, n):
    """Householder QR with a blocked (compact WY) update plus U = Q W:
    products 2 m n^2 - 2 n^3/3 (the factorisation) + 4 m n^2 - 2 n^3 (the
    back-application), up to the panels' lower-order terms; panels
    7 nb (m n - n^2 / 2) to leading order."""
    nb = 32
    panel, prod = bench.qr_precond_flops(m, n, nb)
    lead = 6.0 * m * n * n - 8.0 * n ** 3 / 3.0
    assert abs(prod - lead) <= 4.0 * nb * m * n + 4.0 * nb * n * n     # O(nb m n) correction
    assert abs(panel - 7.0 * nb * (m * n - n * n / 2.0)) <= 7.0 * nb * nb * m
    # exact count for one panel (n <= nb): no trailing matrix, back-application only
    p1, q1 = bench.qr_precond_flops(m, min(n, nb), nb)
    k = min(n, nb)
    assert p1 == 7.0 * m * k * k and q1 == 4.0 * m * k * k


def test_evd_kernel_classes_emulated_and_mixed():
    peaks = {"bf16_tflops_sustained": 1688.5}
    st = _stats(ms_update=2000.0, update_launches=1764, flops_update=2e12, ms_pivot=900.0,
                pivot_launches=882, flops_fp64=4e11, flops_lowp=72e12)
    k = bench.evd_kernel_classes([st], dict(n=4096, b=64, precision=5), peaks)
    assert "update_emu" in k and k["update_emu"]["flops"] == 36 * 2e12
    assert abs(k["update_emu"]["fp64_equiv_tflops"] - 1.0) < 1e-12
    assert abs(k["pivot"]["flops"] - 4e11) < 1.0
    k = bench.evd_kernel_classes([st], dict(n=4096, b=64), peaks)
    assert "update_fp64" in k and k["update_fp64"]["bound"] == "alu"


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` runs the oracle on the host (no GPU) and
    prints one JSON line with the contract's keys, the oracle described in
    cpu_baseline and an e2e entry without copies."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "evd256", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("plain FP64") and "n=256" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the same configuration object as the GPU arm's line, the sample's real
    # duration as ms_per_step and the extrapolation stated
    assert d["config"] == bench.workload_config(bench.WORKLOADS["evd256"], 1)
    assert d["config"]["n"] == 256 and d["config"]["b"] == 16 and d["config"]["seed"] == 1
    assert cb["extrapolated"] is True and cb["extrapolation_factor"] == 15 * 10
    assert abs(d["ms_per_step"] / 1e3 - cb["seconds_per_step"]) <= 1e-9 * d["ms_per_step"]
    assert d["ms_per_step"] < 1e3 / d["value"]        # one sampled step, not the extrapolated solve


def test_default_workload_is_the_metrics_comparison():
    """The default line is the mixed form at n = 8192, b = 128 with the plain
    FP64 solve of the same matrix and the three batched forms beside it."""
    import argparse
    wl = bench.WORKLOADS["mixed8192emu"]
    assert wl["compare_plain"] and wl["compare_batched"]
    assert wl["n"] == 8192 and wl["b"] == 128 and wl["seed"] == 6 and wl["precision"] == 2
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert 'ap.add_argument("--workload", default="mixed8192emu"' in src
    cfg = bench.workload_config(wl, 1)
    assert cfg["precision"] == "mixed bf16x3" and cfg["fp64_products"] is True
    assert bench.workload_config(bench.WORKLOADS["batched_f64"], 1)["count"] == 20000


def test_evd_gates():
    ok = dict(max_abs_eig_err_over_norm2=5e-15, residual_fro_over_normA=6e-14, orth_fro_over_n=1e-15)
    assert bench.evd_gates(ok)["all"] is True
    bad = dict(ok, residual_fro_over_normA=2e-12)
    g = bench.evd_gates(bad)
    assert g["all"] is False and g["residual_le_1e-12"] is False and g["eig_le_1e-13"] is True


def test_batched_cpu_sample_uses_threads_and_counts_work():
    """The batched CPU baseline: the oracle on consecutive matrices, one per
    thread at a time; the work fraction is the n^3 share of the batch done."""
    import numpy as np
    import jacobi_inputs as gen
    wl = dict(kind="batched_evd")
    shapes = [(n, n) for n in (8, 12, 16, 20, 24, 9)]
    mats = [gen.sym_gaussian(n, 60 + n) for _, n in shapes]
    secs, done, frac = bench.batched_cpu_sample(wl, shapes, mats, budget_s=30.0, threads=3)
    assert done == len(shapes) and abs(frac - 1.0) < 1e-12 and secs > 0
    secs, done, frac = bench.batched_cpu_sample(wl, shapes, mats, budget_s=30.0, max_items=2, threads=2)
    tot = sum(n ** 3 for _, n in shapes)
    assert done == 2 and abs(frac - (8 ** 3 + 12 ** 3) / tot) < 1e-12
    wl_svd = dict(kind="batched_svd")
    sh = [(64, 8)] * 4
    G = [gen.tall_gaussian(64, 8, 70 + i, dtype=np.float64) for i in range(4)]
    secs, done, frac = bench.batched_cpu_sample(wl_svd, sh, G, budget_s=30.0, threads=4)
    assert done == 4 and abs(frac - 1.0) < 1e-12
