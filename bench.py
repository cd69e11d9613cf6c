#!/usr/bin/env python
"""Benchmark: thick-restarted GKL on a GWAS-shaped packed genotype matrix.

One step = one complete top-k solve (time-to-top-k at the stated residual) on
the 10,000 samples x 100,000 SNPs workload (5-population admixture, 2%
missing, 2-bit packed, 251 MB resident in HBM -- larger than L2, so no flush is
needed between steps): FP32, partial reorthogonalisation, k=20, subspace 50,
tol 1e-6.  The metric is matrix-vector pairs (A.v and A^T.u) per second over
the whole job; ms_per_step is the time to top-k.

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

WORKLOAD = "fp32_pro_10k_x_100k"
METRIC = "GKL matvec-pairs/s and time-to-top-k at stated residual; HBM GB/s fraction"


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


def make_inputs():
    import synth
    w = synth.CONFIGS[WORKLOAD]
    g = synth.genotypes(w.geno)
    return w, g


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


def cpu_baseline_sample(w, g, budget_s=15.0, max_pairs=40):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload:
    repeated A.v / A^T.u pairs over the full matrix (the per-step cost of GKL)."""
    import numpy as np
    import oracle
    import synth
    M = oracle.Matrix.from_packed(g.packed, g.n)
    v = synth.normal_vec(77, 0, g.m)
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
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": pairs / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{pairs} A.v + A^T.u pairs of the FP64 CPU oracle on the full {g.n} x {g.m} packed matrix "
                      f"({dt:.1f} s)"}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    w, g = make_inputs()
    import numpy as np
    import oracle
    import synth
    M = oracle.Matrix.from_packed(g.packed, g.n)
    v = synth.normal_vec(77, 0, g.m)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    if world > 1:
        # the launcher gives every rank OMP_NUM_THREADS=1; rank 0 alone runs the
        # oracle here, on all host cores as at one GPU
        cores = os.cpu_count() or 1
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(cores)

    def step():
        nonlocal v
        u = M.matvec(v)
        u /= np.linalg.norm(u)
        v = M.rmatvec(u)
        v /= np.linalg.norm(v)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    val = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": g.n, "m": g.m, "step": "one A.v + A^T.u pair of the FP64 oracle"},
            "cpu_baseline": {"value": val, "unit": "pairs/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"{args.steps} oracle pairs on the full matrix"},
            "e2e": {"value": val, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_1808_03374_gb300 import build, gkl
    build()
    w, g = make_inputs()
    packed_host = torch.from_numpy(g.packed).pin_memory()
    packed = packed_host.to("cuda", non_blocking=False)
    h = gkl.GKL(packed, g.n)
    solve_kw = dict(k=w.k, ell=w.ell, reorth=w.reorth, precision=w.precision, tol=w.tol, maxit=2000, seed=7)

    for _ in range(max(3, args.warmup)):
        r = h.svd(**solve_kw)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    infos = []
    with ClockSampler(local) as clk:
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            r = h.svd(profile=True, **solve_kw)
            infos.append(r.info)
        e1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
    pairs = sum(i["matvec_pairs"] for i in infos)
    value, ms = job_throughput(pairs, e0.elapsed_time(e1), pg, "cuda")
    clocks = clk.summary()

    # roofline of the dominant kernel, from the CUDA events recorded around each
    # main product kernel during the timed solves
    peak, peak_kind = measured_peaks()
    n, m = g.n, g.m
    packed_bytes = m * ((n + 3) // 4)
    mv_ms = sum(i["ms_mv"] for i in infos) / max(1, sum(i["n_mv"] for i in infos))
    rmv_ms = sum(i["ms_rmv"] for i in infos) / max(1, sum(i["n_rmv"] for i in infos))
    tot_mv = sum(i["ms_mv"] for i in infos)
    tot_rmv = sum(i["ms_rmv"] for i in infos)
    # the FP32 path runs k_mv_pair (packed_ops.cu) and k_rmv_tc (packed_tc.cu; k_rmv_n256 with
    # GKL_RMV_KERNEL=n256, k_rmv_mma in packed_mma.cu with GKL_RMV_KERNEL=mma); algorithmic bytes
    # per launch = packed G once + the FP32 input and output vectors
    rk = {"mma": ("k_rmv_mma", "packed_mma.cu"), "n256": ("k_rmv_n256", "packed_tc.cu")}.get(
        os.environ.get("GKL_RMV_KERNEL", ""), ("k_rmv_tc", "packed_tc.cu"))
    mv = ("k_mv_pair", "packed_ops.cu", mv_ms, packed_bytes + 4 * m + 4 * n)
    rmv = (rk[0], rk[1], rmv_ms, packed_bytes + 4 * n + 4 * m)
    dom, oth = (mv, rmv) if tot_mv >= tot_rmv else (rmv, mv)
    kname, _, kms, kbytes = dom
    achieved = kbytes / (kms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": ncu_traffic(kname, WORKLOAD),
                "algorithmic_bytes_per_launch": kbytes, "avg_launch_ms": kms,
                "other_kernel": {oth[0]: {"avg_launch_ms": oth[2],
                                          "achieved_gbs": oth[3] / (oth[2] / 1e3) / 1e9,
                                          "traffic": ncu_traffic(oth[0], WORKLOAD)}},
                "share_of_step": (tot_mv + tot_rmv) / ms}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_pairs = 0
        for _ in range(e2e_steps):
            dev = packed_host.to("cuda", non_blocking=True)
            hh = gkl.GKL(dev, n)
            rr = hh.svd(**solve_kw)
            Uh = rr.U.cpu()
            Vh = rr.V.cpu()
            hh.close()
            e2e_pairs += rr.info["matvec_pairs"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": job_throughput(e2e_pairs, dt * 1e3, pg, "cuda")[0], "unit": "pairs/s", "h2d_bytes_per_step": int(packed_host.numel()),
               "d2h_bytes_per_step": int(Uh.numel() * Uh.element_size() + Vh.numel() * Vh.element_size() + 16 * w.k),
               "steps": e2e_steps}

    # block form (tensor-core block products) beside the FP32 solves (the timed
    # PARTIAL one and one with FULL reorthogonalisation), timed separately: time
    # to the converged top-k and the true residuals
    # max_i max(||A^T u_i - s_i v_i||, ||A v_i - s_i u_i||) / s_1 from the
    # library's own 8-digit block products
    block_form = None
    if not args.no_block:
        def true_resid(res):
            Ut, Vt = res.U.T.contiguous(), res.V.T.contiguous()
            Z, Y = h.matmat(Ut, transpose=True), h.matmat(Vt)
            sgm = torch.tensor(res.sigma, device="cuda", dtype=torch.float32)[:, None]
            ra = torch.linalg.norm((Z - sgm * Vt).double(), dim=1).max().item()
            rb = torch.linalg.norm((Y - sgm * Ut).double(), dim=1).max().item()
            return max(ra, rb) / res.sigma[0]
        bkw = dict(k=w.k, ell=128, precision="block", block=16, k_keep=48, tol=w.tol, maxit=500, seed=7)
        for _ in range(2):
            rb_ = h.svd(**bkw)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nb = 3
        b0.record(stream)
        binfos = []
        for _ in range(nb):
            rb_ = h.svd(profile=True, **bkw)
            binfos.append(rb_.info)
        b1.record(stream)
        torch.cuda.synchronize()
        bms = b0.elapsed_time(b1) / nb
        # tensor roofline of the block products: per launch 16 ceil(m/128) ceil(stride/128)
        # MMAs of M=128, N=256, K=32 (e4m3); algorithmic FLOP 2 n m q with q = 16 vectors
        stride = (g.n + 3) // 4
        stride = (stride + 15) // 16 * 16
        mmas = 16 * ((g.m + 127) // 128) * ((stride + 127) // 128)
        issued = 2.0 * 128 * 256 * 32 * mmas
        algo = 2.0 * g.n * g.m * 16
        tpeak, tsrc = measured_e4m3_peak()
        bt = {}
        for key, kn in (("rmv", "k_bt_rmv"), ("mv", "k_bt_mv")):
            nl = sum(i["n_" + key] for i in binfos)
            kms = sum(i["ms_" + key] for i in binfos) / max(1, nl)
            bt[kn] = {"avg_launch_ms": kms, "launches": nl,
                      "achieved_issued_tflops": issued / (kms / 1e3) / 1e12 if kms > 0 else None,
                      "achieved_algorithmic_tflops": algo / (kms / 1e3) / 1e12 if kms > 0 else None,
                      "traffic": ncu_traffic(kn, WORKLOAD)}
        dom_bt = max(bt, key=lambda x: bt[x]["avg_launch_ms"] * bt[x]["launches"])
        a_ = bt[dom_bt]["achieved_issued_tflops"]
        block_roofline = {"bound": "tensor", "kernel": dom_bt, "achieved": a_, "peak": tpeak, "unit": "TFLOP/s",
                          "frac": a_ / tpeak if a_ else None, "peak_source": tsrc,
                          "traffic": bt[dom_bt]["traffic"], "issued_flop_per_launch": issued,
                          "algorithmic_flop_per_launch": algo, "kernels": bt}
        # the FP32 single-vector solve with full reorthogonalisation: orthonormal
        # bases, so its true residual follows its reported one
        fkw = dict(solve_kw, reorth="full")
        rf = h.svd(**fkw)
        torch.cuda.synchronize()
        b0.record(stream)
        for _ in range(nb):
            rf = h.svd(**fkw)
        b1.record(stream)
        torch.cuda.synchronize()
        fms = b0.elapsed_time(b1) / nb
        block_form = {"config": {"block": 16, "ell": 128, "k_keep": 48, "tol": w.tol, "digits": 8,
                                 "products": "tcgen05 kind::f8f6f4 (k_bt_rmv, k_bt_mv)"},
                      "time_to_topk_ms": bms, "vector_pairs": rb_.info["matvec_pairs"],
                      "restarts": rb_.info["restarts"], "converged": bool(rb_.info["converged"]),
                      "true_max_rel_resid": true_resid(rb_),
                      "fp32_path": {"time_to_topk_ms": ms / args.steps, "true_max_rel_resid": true_resid(r),
                                    "reported_max_rel_resid": infos[-1]["max_rel_resid"]},
                      "fp32_full_reorth": {"time_to_topk_ms": fms, "vector_pairs": rf.info["matvec_pairs"],
                                           "true_max_rel_resid": true_resid(rf),
                                           "reported_max_rel_resid": rf.info["max_rel_resid"]},
                      "sigma_max_rel_diff_vs_fp32": float(np.max(np.abs(rb_.sigma - r.sigma)) / r.sigma[0]),
                      "roofline": block_roofline}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(w, g)

    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "m": m, "k": w.k, "ell": w.ell, "reorth": w.reorth,
                       "tol": w.tol, "precision": w.precision, "packed_bytes": int(g.packed.nbytes),
                       "l2": "inputs larger than L2 (251 MB packed vs 129 MB L2); no flush",
                       "parallelism": f"replicas x{world}"},
            "time_to_topk_ms": ms / args.steps, "pairs_per_step": pairs / args.steps,
            "max_rel_resid": infos[-1]["max_rel_resid"], "restarts": infos[-1]["restarts"],
            "jacobi_sweeps": infos[-1]["jacobi_sweeps"], "svd_fallbacks": infos[-1]["svd_fallbacks"],
            "svd_clusters": infos[-1]["svd_clusters"], "reorth_u": infos[-1]["reorth_u"],
            "breakdown_ms_per_step": {
                "A.v_main": sum(i["ms_mv"] for i in infos) / args.steps,
                "A^T.u_main": sum(i["ms_rmv"] for i in infos) / args.steps,
                "projected_svd": sum(i["ms_svd"] for i in infos) / args.steps,
                "reorth": sum(i["ms_cgs"] for i in infos) / args.steps},
            "reorth_v": infos[-1]["reorth_v"],
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "block_form": block_form,
            "gpu_launches": sum(i["launches"] for i in infos), "clocks": clocks}
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def run_block_profile(args):
    """Two warm-up solves and one timed block-form solve at the benchmark
    workload (for launch lists and kernel captures); prints one line."""
    import torch
    from paper_1808_03374_gb300 import build, gkl
    build()
    w, g = make_inputs()
    h = gkl.GKL(torch.from_numpy(g.packed).cuda(), g.n)
    bkw = dict(k=w.k, ell=128, precision="block", block=16, k_keep=48, tol=w.tol, maxit=500, seed=7)
    for _ in range(2):
        r = h.svd(**bkw)
    r = h.svd(**bkw)
    torch.cuda.synchronize()
    print(json.dumps({"block_profile": WORKLOAD, "launches_per_solve": r.info["launches"],
                      "ms": r.info["ms_total"], "vector_pairs": r.info["matvec_pairs"],
                      "converged": r.info["converged"]}), flush=True)
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


def run_compare(args):
    """One workload of synth.CONFIGS: the FP32 single-vector solve (PARTIAL) and
    the block form (b=16, l=128, k_keep=48), each once after the matrix is on
    the device; times, pair counts, true residuals from the 8-digit block
    products, singular-value agreement, and the sigma-part gradient
    (d sum_i sigma_i^2 / dw) after the FP32 solve.  One JSON line."""
    import numpy as np
    import torch
    import synth
    from paper_1808_03374_gb300 import build, gkl
    build()
    w = synth.CONFIGS[args.compare]
    t0 = time.time()
    g = synth.genotypes(w.geno)
    gen_s = time.time() - t0
    t0 = time.time()
    h = gkl.GKL(torch.from_numpy(g.packed).cuda(), g.n)
    torch.cuda.synchronize()
    init_s = time.time() - t0

    def true_resid(res):
        worst = 0.0
        for c0 in range(0, res.U.shape[1], 16):  # 16 vectors per 8-digit pass
            Ut = res.U[:, c0:c0 + 16].T.contiguous().float()
            Vt = res.V[:, c0:c0 + 16].T.contiguous().float()
            Z, Y = h.matmat(Ut, transpose=True), h.matmat(Vt)
            sg = torch.tensor(res.sigma[c0:c0 + 16], device="cuda", dtype=torch.float32)[:, None]
            worst = max(worst, torch.linalg.norm((Z - sg * Vt).double(), dim=1).max().item(),
                        torch.linalg.norm((Y - sg * Ut).double(), dim=1).max().item())
        return worst / res.sigma[0]

    def timed(**kw):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = h.svd(**kw)
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    out = {"workload": args.compare, "n": g.n, "m": g.m, "packed_bytes": int(g.packed.nbytes),
           "generated_s": gen_s, "to_device_and_init_s": init_s}
    tb, rb = timed(k=w.k, ell=128, precision="block", block=16, k_keep=48, tol=1e-6, maxit=500, seed=7)
    out["block"] = {"time_s": tb, "vector_pairs": int(rb.info["matvec_pairs"]), "restarts": int(rb.info["restarts"]),
                    "converged": bool(rb.info["converged"]), "true_max_rel_resid": true_resid(rb)}
    tf, rf = timed(k=w.k, ell=50, reorth="partial", precision="fp32", tol=1e-6, maxit=3000, seed=7)
    out["fp32_partial"] = {"time_s": tf, "pairs": int(rf.info["matvec_pairs"]), "restarts": int(rf.info["restarts"]),
                           "converged": bool(rf.info["converged"]), "reported_max_rel_resid": rf.info["max_rel_resid"],
                           "true_max_rel_resid": true_resid(rf)}
    out["sigma_max_rel_diff"] = float(np.max(np.abs(rb.sigma - rf.sigma)) / rf.sigma[0])
    out["sigma_top5"] = [float(x) for x in rf.sigma[:5]]
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, gw = h.grad(sigma_bar=2.0 * rf.sigma, want_s=False, dtype=torch.float32)
    torch.cuda.synchronize()
    out["grad_w_sigma_part"] = {"time_s": time.perf_counter() - t, "norm": float(gw.double().norm().item())}
    print(json.dumps({"compare": out}), flush=True)
    return 0


def run_fp32_profile(args):
    """One FP32 solve of the benchmark step at the benchmark workload, right
    after the handle is set up (for launch lists; no warm-up solves, so the
    profiler skips only the set-up kernels); prints one line."""
    import torch
    from paper_1808_03374_gb300 import build, gkl
    build()
    w, g = make_inputs()
    h = gkl.GKL(torch.from_numpy(g.packed).cuda(), g.n)
    torch.cuda.synchronize()
    r = h.svd(k=w.k, ell=w.ell, reorth=w.reorth, precision=w.precision, tol=w.tol, maxit=2000, seed=7)
    torch.cuda.synchronize()
    print(json.dumps({"fp32_profile": WORKLOAD, "launches_per_solve": r.info["launches"],
                      "ms": r.info["ms_total"], "pairs": r.info["matvec_pairs"]}), flush=True)
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


def run_cpu_table(args):
    """The FP64 CPU oracle per pair at the workloads whose generation and
    timing fit about half a minute each, on all host cores and on one core,
    and one full oracle solve of the small workload; each measurement in its
    own process."""
    cores = os.cpu_count() or 1
    plan = [("fp64_full_1k_x_10k", cores, True), ("fp64_full_1k_x_10k", 1, False),
            ("fp32_pro_10k_x_100k", cores, False), ("fp32_pro_10k_x_100k", 1, False),
            ("grad_20k_x_200k", cores, False), ("grad_20k_x_200k", 1, False)]
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
    ap.add_argument("--no-block", action="store_true", help="skip the block-form comparison")
    ap.add_argument("--profile-block", action="store_true",
                    help="only warm up and run one block-form solve (for profiler launch lists)")
    ap.add_argument("--profile-fp32", action="store_true",
                    help="only set up and run one FP32 solve of the benchmark step (for profiler launch lists)")
    ap.add_argument("--paper-model", action="store_true",
                    help="the paper's synthetic model at its Table 3 size: solvers side by side (one JSON line)")
    ap.add_argument("--cpu-table", action="store_true",
                    help="the FP64 CPU oracle per pair at several workloads, all cores and one core (one JSON line)")
    ap.add_argument("--cpu-pairs", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-solve", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-threads", type=int, default=os.cpu_count() or 1, help=argparse.SUPPRESS)
    ap.add_argument("--max-pairs", type=int, default=3, help=argparse.SUPPRESS)
    ap.add_argument("--budget", type=float, default=20.0, help=argparse.SUPPRESS)
    ap.add_argument("--compare", default=None,
                    help="a workload of synth.CONFIGS: FP32 solve and block form side by side (one JSON line)")
    args = ap.parse_args()
    if args.compare:
        return run_compare(args)
    if args.cpu_table:
        return run_cpu_table(args)
    if args.cpu_pairs:
        return run_cpu_pairs(args)
    if args.profile_block:
        return run_block_profile(args)
    if args.profile_fp32:
        return run_fp32_profile(args)
    if args.paper_model:
        return run_paper_model(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
