#!/usr/bin/env python
"""Benchmark: thick-restarted GKL on a GWAS-shaped packed genotype matrix.

Workload (N = 1): 200,000 samples x 1,000,000 SNPs, 20-population admixture,
Beta(0.5, 2) base frequencies, 1% missing, 2-bit packed: 50 GB resident in
HBM (far larger than L2, so no flush is needed between steps).  The matrix is
drawn on the GPU by the seeded generator (byte for byte the C generator's).

One step = one complete top-k solve (time-to-top-k at the stated residual):
FP32 Lanczos vectors, reorthogonalisation with the adaptive second pass
(DGKS), k = 20, subspace 50, tol 1e-6 -- plus the per-SNP weight gradient
of sum_i sigma_i^2 from the solve's triplets.  The metric is matrix-vector
pairs (A.v and A^T.u) per second over the whole job; ms_per_step is the time
to top-k plus the gradient.  The true residuals of the timed solve are checked
against tol with the library's 8-digit tensor-core block products.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica on its own GPU (the
path does not shard: replicas only, weak scaling); rank 0 prints one JSON line.
--impl reference times the plain FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import csv
import ctypes
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "large_200k_x_1m"
METRIC = "GKL matvec-pairs/s and time-to-top-k at stated residual; HBM GB/s fraction"
# oracle samples: the first SLAB_SNPS SNP rows of the workload (all samples),
# drawn by the host generator (the same rows, byte for byte)
SLAB_SNPS = 4000


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def reduce_over_ranks(x: float, dist, device, op: str) -> float:
    """x combined over all ranks ("max" or "sum") through a collective of the
    process group (NCCL on the GPU machine, gloo in the CPU tests)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_local: float, ms_local: float, dist=None, device="cpu") -> tuple[float, float]:
    """Whole-job throughput of independent replicas: the units of all ranks
    over the slowest rank's time.  Returns (units per second, max ms)."""
    if dist is None:
        return units_local / (ms_local / 1e3), ms_local
    ms = reduce_over_ranks(ms_local, dist, device, "max")
    units = reduce_over_ranks(units_local, dist, device, "sum")
    return units / (ms / 1e3), ms


def measured_peaks():
    """(HBM GB/s, source): the measured copy bandwidth, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_e4m3_peak():
    """Dense e4m3 tensor peak (TFLOP/s): the measured bf16 burst peak x 2 (the
    nominal fp8/bf16 ratio), else the fallback 1.9 PFLOP/s bf16 x 2."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return 2.0 * float(d["bf16_tflops"]), "measured bf16 burst x 2"
    return 3800.0, "fallback bf16 x 2"


def source_digest(fn: str) -> str:
    """sha256 (16 hex) of one kernel source file under csrc/."""
    with open(os.path.join(ROOT, "paper_1808_03374_gb300", "csrc", fn), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.json),
    if the kernel's source file is unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(kernel)
    if not e:
        return None
    try:
        if source_digest(e["source"]) != e.get("source_sha"):
            return None
    except OSError:
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.file.read())) if len(r) >= 9]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name as lscpu reports it ("" if unavailable)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return ""
    for line in out.splitlines():
        if line.startswith("Model name:"):
            return line.split(":", 1)[1].strip()
    return ""


# ---- CPU oracle samples ------------------------------------------------------------

def oracle_slab(w, snps: int = SLAB_SNPS):
    """The first `snps` SNP rows of the workload (all samples), drawn by the
    host generator -- the same bytes as those rows of the full matrix -- and
    the oracle's operator over them."""
    import dataclasses

    import oracle
    import synth
    spec = dataclasses.replace(w.geno, m=min(snps, w.geno.m))
    g = synth.genotypes(spec)
    return g, oracle.Matrix.from_packed(g.packed, g.n)


def time_oracle_pairs(M, m_full: int, budget_s: float, max_pairs: int, seed: int = 77):
    """Oracle A.v + A^T.u pairs on the slab until the budget is spent.
    Returns (pairs, seconds, full-matrix pairs per second): a pair over the
    slab reads M.m / m_full of the full matrix's entries."""
    import numpy as np

    import synth
    v = synth.normal_vec(seed, 0, M.m)
    pairs, t0 = 0, time.perf_counter()
    while pairs < max_pairs:
        u = M.matvec(v)
        u /= np.linalg.norm(u)
        v = M.rmatvec(u)
        v /= np.linalg.norm(v)
        pairs += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return pairs, dt, pairs / dt * (M.m / m_full)


def cpu_baseline_sample(w, budget_s=15.0, max_pairs=200):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload."""
    g, M = oracle_slab(w)
    pairs, dt, rate = time_oracle_pairs(M, w.geno.m, budget_s, max_pairs)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{pairs} A.v + A^T.u pairs of the FP64 CPU oracle over the first {M.m} of the {w.geno.m} "
                      f"SNP rows (all {g.n} samples; {dt:.1f} s), scaled to the full matrix by {M.m}/{w.geno.m}"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores.  One step =
    one oracle pair over the first SLAB_SNPS SNP rows; the value is scaled to
    full-matrix pairs per second."""
    import synth
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    w = synth.CONFIGS[WORKLOAD]
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    if world > 1:
        # the launcher gives every rank OMP_NUM_THREADS=1; rank 0 alone runs the
        # oracle here, on all host cores as at one GPU
        cores = os.cpu_count() or 1
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(cores)
    g, M = oracle_slab(w)
    time_oracle_pairs(M, w.geno.m, 1e9, max(0, args.warmup))
    pairs, dt, rate = time_oracle_pairs(M, w.geno.m, 1e9, args.steps)
    # a step is one pair over the slab; its measured time is the step time, and the
    # value counts the full-matrix pairs that the slab's share of the entries makes up
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, pairs),
            "ms_per_full_matrix_pair": 1e3 / rate, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": w.geno.n, "m": w.geno.m,
                       "step": f"one A.v + A^T.u pair of the FP64 oracle over the first {M.m} SNP rows; "
                               f"value in full-matrix pairs ({w.geno.m} SNPs) per second"},
            "cpu_baseline": {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"{pairs} oracle pairs over {M.m} of {w.geno.m} SNP rows ({dt:.1f} s)"},
            "e2e": {"value": rate, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- the GPU arm -------------------------------------------------------------------

def true_resid(h, res):
    """max_i max(||A^T u_i - s_i v_i||, ||A v_i - s_i u_i||) / s_1 from the
    library's 8-digit tensor-core block products (16 vectors per pass)."""
    import torch
    worst = 0.0
    for c0 in range(0, res.U.shape[1], 16):
        Ut = res.U[:, c0:c0 + 16].T.contiguous().float()
        Vt = res.V[:, c0:c0 + 16].T.contiguous().float()
        Z, Y = h.matmat(Ut, transpose=True), h.matmat(Vt)
        sg = torch.tensor(res.sigma[c0:c0 + 16], device="cuda", dtype=torch.float32)[:, None]
        worst = max(worst, torch.linalg.norm((Z - sg * Vt).double(), dim=1).max().item(),
                    torch.linalg.norm((Y - sg * Ut).double(), dim=1).max().item())
    return worst / res.sigma[0]


def true_resid64(h, res):
    """The same residual from the library's FP64 products, one vector at a time
    (for FP64 solves, whose residuals lie below FP32 rounding)."""
    import torch
    worst = 0.0
    for i in range(res.U.shape[1]):
        u = res.U[:, i].double().contiguous()
        v = res.V[:, i].double().contiguous()
        s = float(res.sigma[i])
        worst = max(worst, torch.linalg.norm(h.rmatvec(u) - s * v).item(), torch.linalg.norm(h.matvec(v) - s * u).item())
    return worst / res.sigma[0]


def solve_kw(w, **extra):
    return dict(k=w.k, ell=w.ell, reorth=w.reorth, precision=w.precision, tol=w.tol, maxit=3000, seed=7, **extra)


def step_once(h, w, profile=False):
    """One benchmark step: the top-k solve, then dL/dw for L = sum_i sigma_i^2
    (the sigma part of the gradient, one A^T u per triplet).  Returns the
    solve's result, the gradient and the pairs applied (an A^T u alone counts
    as half a pair)."""
    r = h.svd(profile=profile, **solve_kw(w))
    _, gw = h.grad(sigma_bar=2.0 * r.sigma, want_s=False)
    return r, gw, r.info["matvec_pairs"] + 0.5 * w.k


def run_ours(args):
    import numpy as np
    import torch
    import synth
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_1808_03374_gb300 import build, gkl
    build()
    w = synth.CONFIGS[WORKLOAD]
    n, m = w.geno.n, w.geno.m
    t0 = time.time()
    packed, _, _ = synth.genotypes_device(w.geno)
    gen_s = time.time() - t0
    h = gkl.GKL(packed, n)
    stream = torch.cuda.current_stream()

    for _ in range(max(3, args.warmup)):
        step_once(h, w)
    torch.cuda.synchronize()
    infos, pairs = [], 0.0
    with ClockSampler(local) as clk:
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            r, gw, p = step_once(h, w, profile=True)
            infos.append(r.info)
            pairs += p
        e1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
    value, ms = job_throughput(pairs, e0.elapsed_time(e1), pg, "cuda")
    clocks = clk.summary()
    resid_true = true_resid(h, r)

    # roofline of the dominant kernel, from the CUDA events the library records
    # around each main product kernel of the timed solves
    peak, peak_kind = measured_peaks()
    packed_bytes = m * ((n + 3) // 4)
    kb = packed_bytes + 4 * m + 4 * n  # algorithmic bytes per launch: the packed matrix once + the two vectors
    mv_ms = sum(i["ms_mv"] for i in infos) / max(1, sum(i["n_mv"] for i in infos))
    rmv_ms = sum(i["ms_rmv"] for i in infos) / max(1, sum(i["n_rmv"] for i in infos))
    tot_mv, tot_rmv = sum(i["ms_mv"] for i in infos), sum(i["ms_rmv"] for i in infos)
    kern = {"k_mv_pair": {"file": "packed_ops.cu", "avg_launch_ms": mv_ms, "achieved_gbs": kb / mv_ms / 1e6,
                          "frac": kb / mv_ms / 1e6 / peak, "total_ms_per_step": tot_mv / args.steps,
                          "traffic": ncu_traffic("k_mv_pair", WORKLOAD)},
            "k_rmv_tc": {"file": "packed_tc.cu", "avg_launch_ms": rmv_ms, "achieved_gbs": kb / rmv_ms / 1e6,
                         "frac": kb / rmv_ms / 1e6 / peak, "total_ms_per_step": tot_rmv / args.steps,
                         "traffic": ncu_traffic("k_rmv_tc", WORKLOAD)}}
    dom = "k_mv_pair" if tot_mv >= tot_rmv else "k_rmv_tc"
    oth = "k_rmv_tc" if dom == "k_mv_pair" else "k_mv_pair"
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["achieved_gbs"], "peak": peak, "unit": "GB/s",
                "frac": kern[dom]["frac"], "peak_source": peak_kind, "traffic": kern[dom]["traffic"],
                "algorithmic_bytes_per_launch": kb, "avg_launch_ms": kern[dom]["avg_launch_ms"],
                "other_kernel": {oth: kern[oth]}, "share_of_step": (tot_mv + tot_rmv) / ms}

    # end to end through the public API with host buffers: the packed matrix
    # from pinned host memory to the device, gkl_init (statistics, TMA views,
    # missing-code lists), the solve with U and V copied to host memory, the
    # gradient copied back
    e2e = None
    if not args.no_e2e:
        host = torch.empty((m, packed.shape[1]), dtype=torch.uint8, pin_memory=True)
        host.copy_(packed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_pairs, d2h = 0.0, 0
        for _ in range(args.e2e_steps):
            dev = host.to("cuda", non_blocking=True)
            hh = gkl.GKL(dev, n)
            rr = hh.svd(out_host=True, **solve_kw(w))
            _, gwe = hh.grad(sigma_bar=2.0 * rr.sigma, want_s=False)
            gwh = gwe.cpu()
            hh.close()
            del dev
            e2e_pairs += rr.info["matvec_pairs"] + 0.5 * w.k
            d2h = (rr.U.numel() * rr.U.element_size() + rr.V.numel() * rr.V.element_size()
                   + gwh.numel() * gwh.element_size() + 16 * w.k)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": job_throughput(e2e_pairs, dt * 1e3, pg, "cuda")[0], "unit": "pairs/s",
               "h2d_bytes_per_step": int(host.numel()), "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps}
        del host

    # block form (tensor-core block products, b = 16, subspace 128) beside the
    # timed solve: time to the converged top-k and its true residual
    block_form = None
    if not args.no_block:
        bkw = dict(k=w.k, ell=w.extra["block_ell"], precision="block", block=w.extra["block"],
                   k_keep=w.extra["k_keep"], tol=w.tol, maxit=500, seed=7, profile=True)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        rb = h.svd(**bkw)
        b1.record(stream)
        torch.cuda.synchronize()
        tpeak, tsrc = measured_e4m3_peak()
        stride = packed.shape[1]
        mmas = 16 * ((m + 127) // 128) * ((stride + 127) // 128)  # MMAs of one 16-vector product
        issued = 2.0 * 128 * 256 * 32 * mmas
        bt = {}
        for key, kn in (("rmv", "k_bt_rmv"), ("mv", "k_bt_mv")):
            nl = rb.info["n_" + key]
            kms = rb.info["ms_" + key] / max(1, nl)
            bt[kn] = {"avg_launch_ms": kms, "launches": nl,
                      "achieved_gbs": kb / kms / 1e6 if kms > 0 else None,
                      "achieved_issued_tflops": issued / (kms / 1e3) / 1e12 if kms > 0 else None,
                      "algorithmic_tflops_16_vectors": 2.0 * n * m * 16 / (kms / 1e3) / 1e12 if kms > 0 else None}
        block_form = {"config": {"block": w.extra["block"], "ell": w.extra["block_ell"], "k_keep": w.extra["k_keep"],
                                 "tol": w.tol, "digits": 8, "products": "tcgen05 kind::f8f6f4 (k_bt_rmv, k_bt_mv)"},
                      "time_to_topk_ms": b0.elapsed_time(b1), "vector_pairs": rb.info["matvec_pairs"],
                      "restarts": rb.info["restarts"], "converged": bool(rb.info["converged"]),
                      "true_max_rel_resid": true_resid(h, rb),
                      "sigma_max_rel_diff_vs_fp32": float(np.max(np.abs(rb.sigma - r.sigma) / r.sigma)),
                      "peak_e4m3_tflops": tpeak, "peak_source": tsrc, "kernels": bt}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(w)

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0
    ms_step = ms / args.steps
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "m": m, "k": w.k, "ell": w.ell, "reorth": w.reorth,
                       "tol": w.tol, "precision": w.precision, "packed_bytes": int(packed.numel()),
                       "step": "top-k solve + per-SNP weight gradient of sum sigma_i^2",
                       "l2": "inputs larger than L2 (50 GB packed vs 129 MB L2); no flush",
                       "generated_on_device_s": gen_s, "parallelism": f"replicas x{world}"},
            "time_to_topk_ms": sum(i["ms_total"] for i in infos) / args.steps,
            "pairs_per_step": pairs / args.steps, "true_max_rel_resid": resid_true,
            "reported_max_rel_resid": infos[-1]["max_rel_resid"], "restarts": infos[-1]["restarts"],
            "reorth": {"u": infos[-1]["reorth_u"], "v": infos[-1]["reorth_v"], "second_u": infos[-1]["second_u"],
                       "second_v": infos[-1]["second_v"]},
            "breakdown_ms_per_step": {
                "A.v_main": tot_mv / args.steps, "A^T.u_main": tot_rmv / args.steps,
                "projected_svd": sum(i["ms_svd"] for i in infos) / args.steps,
                "reorth": sum(i["ms_cgs"] for i in infos) / args.steps},
            "sigma_top4": [float(x) for x in r.sigma[:4]],
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "block_form": block_form,
            "gpu_launches": sum(i["launches"] for i in infos) + args.steps * 7 * w.k, "clocks": clocks}
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def run_profile(args):
    """Setup, then exactly one benchmark step (solve + gradient) on the
    benchmark workload -- for profiler launch lists; prints one line."""
    import torch
    import synth
    from paper_1808_03374_gb300 import build, gkl
    build()
    w = synth.CONFIGS[args.profile_workload]
    packed, _, _ = synth.genotypes_device(w.geno)
    h = gkl.GKL(packed, w.geno.n)
    torch.cuda.synchronize()
    r, _, pairs = step_once(h, w)
    torch.cuda.synchronize()
    print(json.dumps({"profile_step": args.profile_workload, "launches_solve": r.info["launches"],
                      "ms_solve": r.info["ms_total"], "pairs": pairs}), flush=True)
    return 0


PROFILE_SLAB = "slab_200k_x_38912"


def run_profile_products(args):
    """Products only, for ncu captures: args.reps FP32 A.v and A^T u (and with
    --block-vectors q, the 8-digit tensor-core block products of q vectors) on
    a workload of synth.CONFIGS, or on the slab of large_200k_x_1m with all
    200,000 samples and its first 38,912 SNP rows (152 tiles of 256 SNPs: one
    A^T u work item per SM; 1.95 GB packed)."""
    from dataclasses import replace
    import torch
    import synth
    from paper_1808_03374_gb300 import build, gkl
    build()
    name = args.profile_products
    geno = (replace(synth.CONFIGS["large_200k_x_1m"].geno, m=38_912) if name == PROFILE_SLAB
            else synth.CONFIGS[name].geno)
    packed, _, _ = synth.genotypes_device(geno)
    h = gkl.GKL(packed, geno.n)
    v = torch.tensor(synth.normal_vec(31, 0, geno.m), dtype=torch.float32, device="cuda")
    u = torch.tensor(synth.normal_vec(31, 1, geno.n), dtype=torch.float32, device="cuda")
    q = args.block_vectors
    if q:
        V = torch.tensor(synth.normal_vec(31, 2, q * geno.m).reshape(q, geno.m), dtype=torch.float32, device="cuda")
        U = torch.tensor(synth.normal_vec(31, 3, q * geno.n).reshape(q, geno.n), dtype=torch.float32, device="cuda")
    for _ in range(args.reps):
        h.matvec(v)
        h.rmatvec(u)
        if q:
            h.matmat(V)
            h.matmat(U, transpose=True)
    torch.cuda.synchronize()
    h.sync()
    print(json.dumps({"profile_products": name, "n": geno.n, "m": geno.m, "reps": args.reps, "block_vectors": q}))
    return 0


def run_paper_model(args):
    """The paper's own workload: its synthetic genotype model (section 2,
    Algorithm 1) at 41,505 markers x 81,700 patients, top 10 singular triplets
    as in Table 3.  Each solver's matrix-vector pair count (mvps), time,
    ||Delta theta||_1 (sum of the reported residuals) and the relative error of
    sigma_10 against a tight FP64 solve.  One JSON line."""
    import numpy as np
    import torch
    import synth
    from paper_1808_03374_gb300 import build, gkl
    build()
    t0 = time.time()
    g = synth.paper_model(synth.PAPER_MODEL)
    gen_s = time.time() - t0
    h = gkl.GKL(torch.from_numpy(g.packed).cuda(), g.n)
    k = 10

    def run(**kw):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = h.svd(k=k, maxit=3000, seed=7, **kw)
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    _, ref = run(ell=40, reorth="full", precision="fp64", tol=1e-12)
    runs = []
    for name, kw in (("GKL (FRO, TR) FP64, restart after 20", dict(ell=20, reorth="full", precision="fp64", tol=1e-8)),
                     ("GKL (PRO) FP64, l=128", dict(ell=128, reorth="partial", precision="fp64", tol=1e-8)),
                     ("GKL (FRO, TR) FP32, restart after 20", dict(ell=20, reorth="full", precision="fp32", tol=1e-6)),
                     ("GKL (PRO, TR) FP32, l=50", dict(ell=50, reorth="partial", precision="fp32", tol=1e-6)),
                     ("GKL (DGKS, TR) FP32, l=50", dict(ell=50, reorth="dgks", precision="fp32", tol=1e-6)),
                     ("block b=16 l=128, tensor-core products", dict(ell=128, precision="block", block=16, k_keep=48,
                                                                     tol=1e-6))):
        run(**kw)  # warm-up
        t, r = run(**kw)
        runs.append({"solver": name, "mvps": int(r.info["matvec_pairs"]), "restarts": int(r.info["restarts"]),
                     "time_s": t, "dtheta1": float(r.info["dtheta1"]),
                     "rel_err_sigma10": float(abs(r.sigma[k - 1] - ref.sigma[k - 1]) / ref.sigma[k - 1]),
                     "converged": bool(r.info["converged"])})
    print(json.dumps({"paper_model": {"markers": g.m, "patients": g.n, "r": synth.PAPER_MODEL.r,
                                      "nsignal": "m n", "rkins": synth.PAPER_MODEL.rkins,
                                      "packed_bytes": int(g.packed.nbytes), "generated_s": gen_s},
                      "sigma_top10": [float(x) for x in ref.sigma[:k]], "runs": runs}), flush=True)
    return 0



def run_cpu_pairs(args):
    """Seconds per A.v + A^T.u pair of the FP64 CPU oracle on one workload (a
    bounded sample on --cpu-threads OpenMP threads; the matrix is generated on
    all cores first); with --cpu-solve also one full oracle solve with the
    workload's settings."""
    import numpy as np
    import oracle
    import synth
    w = synth.CONFIGS[args.cpu_pairs]
    t0 = time.perf_counter()
    g = synth.genotypes(w.geno)
    gen_s = time.perf_counter() - t0
    M = oracle.Matrix.from_packed(g.packed, g.n)
    v = synth.normal_vec(77, 0, g.m)
    # the oracle and the generator share one OpenMP runtime in this process
    ctypes.CDLL("libgomp.so.1").omp_set_num_threads(args.cpu_threads)
    pairs, t0 = 0, time.perf_counter()
    while pairs < args.max_pairs:
        u = M.matvec(v)
        u /= np.linalg.norm(u)
        v = M.rmatvec(u)
        v /= np.linalg.norm(v)
        pairs += 1
        if time.perf_counter() - t0 > args.budget:
            break
    per_pair = (time.perf_counter() - t0) / pairs
    out = {"workload": args.cpu_pairs, "n": g.n, "m": g.m, "threads": args.cpu_threads,
           "generated_s": gen_s, "pairs_timed": pairs, "s_per_pair": per_pair}
    if args.cpu_solve:
        t0 = time.perf_counter()
        r = oracle.gkl(M, k=w.k, ell=w.ell, tol=w.tol, v0=synth.normal_vec(5, 0, g.m), maxit=2000)
        out["full_solve"] = {"s": time.perf_counter() - t0, "pairs": int(getattr(r, "pairs", -1)),
                             "converged": bool(r.converged)}
    print(json.dumps({"cpu_pairs": out}), flush=True)
    return 0


TABLE_WORKLOADS = ("fp64_full_1k_x_10k", "fp32_pro_10k_x_100k", "grad_20k_x_200k", "block_50k_x_500k")


def run_solver_table(args):
    """Every solver form on the smaller workloads (the 200,000 x 1,000,000
    one is the benchmark itself): time to the top-k, vector pairs, restarts,
    and the true residual max_i max(||A^T u_i - s_i v_i||, ||A v_i - s_i u_i||) / s_1
    from the 8-digit tensor-core block products.  One JSON line."""
    import torch
    import synth
    from paper_1808_03374_gb300 import build, gkl
    build()
    solvers = [
        ("fp64 dgks", dict(precision="fp64", reorth="dgks", tol=1e-10, ell=None)),
        ("fp32 dgks", dict(precision="fp32", reorth="dgks", tol=1e-6, ell=None)),
        ("fp32 full", dict(precision="fp32", reorth="full", tol=1e-6, ell=None)),
        ("fp32 partial", dict(precision="fp32", reorth="partial", tol=1e-6, ell=None)),
        ("fp32 onesided", dict(precision="fp32", reorth="onesided", tol=1e-6, ell=None)),
        ("block b16", dict(precision="block", block=16, k_keep=48, tol=1e-6, ell=128)),
        ("block16 b32", dict(precision="block16", block=32, k_keep=64, tol=1e-6, ell=128)),
    ]
    out = {"solver_table": []}
    for name in TABLE_WORKLOADS:
        w = synth.CONFIGS[name]
        packed, _, _ = synth.genotypes_device(w.geno)
        h = gkl.GKL(packed, w.geno.n)
        row = {"workload": name, "n": w.geno.n, "m": w.geno.m, "k": w.k, "solvers": {}}
        for label, kw in solvers:
            kw = dict(kw)
            ell = kw.pop("ell") or w.ell
            if kw["precision"].startswith("block") and w.k >= ell:
                continue
            h.svd(k=w.k, ell=ell, maxit=3000, seed=7, raise_on_fail=False, **kw)  # warm-up (allocations)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = h.svd(k=w.k, ell=ell, maxit=3000, seed=7, raise_on_fail=False, **kw)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            row["solvers"][label] = {"ms": dt * 1e3, "pairs": int(r.info["matvec_pairs"]),
                                     "restarts": int(r.info["restarts"]), "converged": bool(r.converged),
                                     "tol": kw["tol"],
                                     "true_max_rel_resid": (true_resid64(h, r) if kw["precision"] == "fp64"
                                                            else true_resid(h, r)),
                                     "reported_max_rel_resid": float(r.info["max_rel_resid"]),
                                     "sigma_1": float(r.sigma[0])}
        out["solver_table"].append(row)
        del h, packed
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def run_cpu_table(args):
    """The FP64 CPU oracle per pair on all host cores and on one core, full
    oracle solves (FULL reorthogonalisation, each workload's k, l and tol) of
    the 1,000 x 10,000, 10,000 x 100,000 and 20,000 x 200,000 workloads on all
    cores, and pairs of the 50,000 x 500,000 one (the 200,000 x 1,000,000 one
    is the benchmark line's cpu_baseline); each measurement in its own process.
    About ten minutes on 16 cores."""
    cores = os.cpu_count() or 1
    plan = [("fp64_full_1k_x_10k", cores, True), ("fp64_full_1k_x_10k", 1, False),
            ("fp32_pro_10k_x_100k", cores, True), ("fp32_pro_10k_x_100k", 1, False),
            ("grad_20k_x_200k", cores, True), ("grad_20k_x_200k", 1, False),
            ("block_50k_x_500k", cores, False)]
    rows = []
    for name, threads, solve in plan:
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-pairs", name, "--cpu-threads", str(threads),
               "--max-pairs", "3", "--budget", "10"] + (["--cpu-solve"] if solve else [])
        env = {k: v for k, v in os.environ.items() if k != "OMP_NUM_THREADS"}
        res = subprocess.run(cmd, env=env, capture_output=True, text=True, cwd=ROOT)
        line = [x for x in res.stdout.splitlines() if x.startswith("{")]
        rows.append(json.loads(line[-1])["cpu_pairs"] if line else {"workload": name, "threads": threads,
                                                                      "error": res.stderr[-300:]})
    print(json.dumps({"cpu_table": {"host_cores": cores, "cpu": cpu_model(), "rows": rows}}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-block", action="store_true", help="skip the block-form solve")
    ap.add_argument("--profile", action="store_true",
                    help="only set up and run one benchmark step (for profiler launch lists)")
    ap.add_argument("--profile-workload", default=WORKLOAD, help=argparse.SUPPRESS)
    ap.add_argument("--profile-products", default=None, metavar="WORKLOAD",
                    help="only run --reps FP32 A.v + A^T u products on WORKLOAD (for ncu captures)")
    ap.add_argument("--reps", type=int, default=3, help=argparse.SUPPRESS)
    ap.add_argument("--block-vectors", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--paper-model", action="store_true",
                    help="the paper's synthetic model at its Table 3 size: solvers side by side (one JSON line)")
    ap.add_argument("--solver-table", action="store_true",
                    help="every solver form on the smaller workloads: time, pairs, true residual (one JSON line)")
    ap.add_argument("--cpu-table", action="store_true",
                    help="the FP64 CPU oracle per pair at several workloads, all cores and one core (one JSON line)")
    ap.add_argument("--cpu-pairs", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-solve", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-threads", type=int, default=os.cpu_count() or 1, help=argparse.SUPPRESS)
    ap.add_argument("--max-pairs", type=int, default=3, help=argparse.SUPPRESS)
    ap.add_argument("--budget", type=float, default=20.0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_table:
        return run_cpu_table(args)
    if args.solver_table:
        return run_solver_table(args)
    if args.cpu_pairs:
        return run_cpu_pairs(args)
    if args.profile:
        return run_profile(args)
    if args.profile_products:
        return run_profile_products(args)
    if args.paper_model:
        return run_paper_model(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
