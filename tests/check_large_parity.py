"""Parity of the GPU solver at the large GWAS-shaped workloads, against the
FP64 CPU oracle and against what the mathematics fixes.

Run on a GPU machine from the repository root:

    python tests/check_large_parity.py null_10k_x_100k paths_50k_x_500k gradient_20k_x_200k \
        benchmark_200k_x_1m --out large_parity

Each check prints one JSON line and the run writes a Markdown summary
(``--out`` + ``.md``) and the JSON lines (``--out`` + ``.jsonl``).  The
checks, with the pins they rest on:

* ``null_10k_x_100k`` -- 10,000 x 100,000, no population structure, 2% missing: the
  largest singular value of the standardised matrix sits at the
  Marchenko-Pastur bulk edge sqrt(1 - f) (sqrt(n) + sqrt(m)) (section 2,
  Eqs. 4-5; f the missing fraction, whose entries are 0 after centring), to
  within 2%.
* ``paths_50k_x_500k`` -- 50,000 x 500,000, 10-population admixture, 1% missing: the
  FP64, FP32 and both block forms solve for k = 20; every triplet's residuals
  ||A v_i - sigma_i u_i|| and ||A^T u_i - sigma_i v_i|| are recomputed with the
  oracle's own products (section 3's convergence criterion, applied a
  posteriori).  A converged FP64 triplet with residual r_i has a singular
  value within r_i of sigma_i (Weyl), so the FP64 values serve as the
  reference for the other paths' per-value relative errors and subspace
  angles.
* ``gradient_20k_x_200k`` -- 20,000 x 200,000 with per-sample and per-SNP weights
  U(0.5, 1.5): the gradient of L = sum_{i<=10} c_i sigma_i^2 + ||S r||^2
  (S the PC scores, r on the well-separated population components) from
  gkl_grad against central differences of FP64 solves at 64 seeded
  coordinates of w and of s, with h = 1e-6 and h = 1e-4, and the sigma part
  against its closed form sigma_i v_ij^2 / w_j.
* ``benchmark_200k_x_1m`` -- 200,000 x 1,000,000, 20-population admixture, 1% missing: the
  FP32 solve and the 8-digit block form, residuals from the oracle's
  products (the oracle reads the 50 GB packed matrix in host memory).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def _lib():
    import torch  # noqa: F401
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl


def device_matrix(spec):
    """The packed matrix generated on the GPU (bit-identical to the host
    generator) and a host copy for the oracle."""
    P, _, _ = synth.genotypes_device(spec)
    return P, P.cpu().numpy()


def oracle_residuals(M, sigma, U, V):
    """Per triplet max(||A v - s u||, ||A^T u - s v||), with the oracle's FP64
    products of the GPU's vectors (as FP64)."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    Y = M.matmat(V) - U * sigma
    Z = M.rmatmat(U) - V * sigma
    return np.maximum(np.linalg.norm(Y, axis=0), np.linalg.norm(Z, axis=0))


def angles(X, Y):
    """Angle between column i of X and column i of Y (unit vectors)."""
    c = np.abs(np.sum(X * Y, axis=0)) / (np.linalg.norm(X, axis=0) * np.linalg.norm(Y, axis=0))
    return np.arccos(np.clip(c, 0.0, 1.0))


def solve(h, **kw):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = h.svd(raise_on_fail=False, **kw)
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def host(t):
    return t.double().cpu().numpy()


# ---------------------------------------------------------------- null model

def check_null_10k_x_100k(gk):
    w = synth.CONFIGS["fp32_pro_10k_x_100k"]
    spec = synth.null_variant(w.geno)
    P, _, _ = synth.genotypes_device(spec)
    h = gk.GKL(P, spec.n)
    r, dt = solve(h, k=5, ell=30, reorth="dgks", precision="fp32", tol=1e-6, maxit=500, seed=3)
    edge = np.sqrt(1.0 - spec.miss_rate) * (np.sqrt(spec.n) + np.sqrt(spec.m))
    rel = float(r.sigma[0] / edge - 1.0)
    return {"check": "null_10k_x_100k", "n": spec.n, "m": spec.m, "converged": bool(r.converged),
            "sigma": [float(x) for x in r.sigma], "mp_edge": float(edge), "sigma1_rel_to_edge": rel,
            "solve_s": dt, "pass": bool(r.converged and abs(rel) <= 0.02)}


# ---------------------------------------------------------------- 50,000 x 500,000

def check_paths_50k_x_500k(gk):
    w = synth.CONFIGS["block_50k_x_500k"]
    spec = w.geno
    P, packed = device_matrix(spec)
    h = gk.GKL(P, spec.n)
    k = w.k
    runs = {
        "fp64": dict(k=k, ell=50, reorth="dgks", precision="fp64", tol=1e-10, maxit=3000, seed=7),
        "fp32": dict(k=k, ell=50, reorth="dgks", precision="fp32", tol=1e-6, maxit=3000, seed=7),
        "block": dict(k=k, ell=128, precision="block", block=16, k_keep=48, tol=1e-6, maxit=500, seed=7),
        "block16": dict(k=k, ell=128, precision="block16", block=32, k_keep=64, tol=1e-6, maxit=500, seed=7),
    }
    res = {}
    for name, kw in runs.items():
        r, dt = solve(h, **kw)
        res[name] = (r, dt)
    del h, P
    M = oracle.Matrix.from_packed(packed, spec.n)
    ref = res["fp64"][0]
    Vr = host(ref.V)
    out = {"check": "paths_50k_x_500k", "n": spec.n, "m": spec.m, "k": k, "paths": {}}
    ok = True
    for name, (r, dt) in res.items():
        t0 = time.perf_counter()
        rr = oracle_residuals(M, r.sigma, host(r.U), host(r.V))
        tor = time.perf_counter() - t0
        rel_res = rr / r.sigma[0]
        tol = runs[name]["tol"]
        e = {"converged": bool(r.converged), "solve_s": dt, "pairs": int(r.info["matvec_pairs"]),
             "oracle_max_rel_resid": float(rel_res.max()), "lib_max_rel_resid": float(r.info["max_rel_resid"]),
             "oracle_products_s": tor}
        if name != "fp64":
            rel = np.abs(r.sigma - ref.sigma) / ref.sigma
            e["sigma_max_rel_err_vs_fp64"] = float(rel.max())
            e["sigma_rel_err_vs_fp64"] = [float(x) for x in rel]
            e["max_angle_vs_fp64"] = float(angles(host(r.V), Vr).max())
            bar = 1e-5 if name == "fp32" else 1e-6
            e["sigma_bar"] = bar
            e["pass"] = bool(r.converged and rel.max() <= bar and rel_res.max() <= 2 * tol)
        else:
            # Weyl: each sigma_i is within r_i of a singular value of A
            e["sigma_within_resid"] = True
            e["pass"] = bool(r.converged and rel_res.max() <= 2 * tol)
        ok = ok and e["pass"]
        out["paths"][name] = e
    out["fp64_sigma"] = [float(x) for x in ref.sigma]
    out["pass"] = ok
    return out


# ---------------------------------------------------------------- 20,000 x 200,000, gradient

def loss_and_grad(gk, h, s, w, c, r, v0=None, tol=1e-13, want_grad=True, seed=5):
    """L = sum c_i sigma_i^2 + ||S r||^2 from an FP64 solve with weights s, w
    (FP32 device tensors); with want_grad also (dL/ds, dL/dw) from gkl_grad."""
    import torch
    h.set_weights(s, w)
    kw = dict(k=len(c), ell=40, reorth="dgks", precision="fp64", tol=tol, maxit=3000, seed=seed)
    if v0 is not None:
        kw["v0"] = v0
    res = h.svd(**kw)
    S = h.scores()
    rt = torch.tensor(r, dtype=torch.float64, device="cuda")
    Sr = S @ rt
    L = float(np.sum(c * res.sigma ** 2) + torch.dot(Sr, Sr).item())
    if not want_grad:
        return L, res
    Sbar = 2.0 * torch.outer(Sr, rt)
    gs, gw = h.grad(sigma_bar=2.0 * c * res.sigma, scores_bar=Sbar, dtype=torch.float64)
    return L, res, host(gs), host(gw)


def check_gradient_20k_x_200k(gk, ncoords=64):
    import torch
    wl = synth.CONFIGS["grad_20k_x_200k"]
    spec = wl.geno
    P, _, _ = synth.genotypes_device(spec)
    h = gk.GKL(P, spec.n)
    k = wl.k
    lo, hi = wl.extra["weights"]
    s = synth.uniform_vec(spec.seed, 20, spec.n, lo, hi).astype(np.float32)
    w = synth.uniform_vec(spec.seed, 21, spec.m, lo, hi).astype(np.float32)
    c = synth.normal_vec(spec.seed, 22, k)
    r = np.zeros(k)
    r[:spec.n_pops - 1] = synth.normal_vec(spec.seed, 23, spec.n_pops - 1)  # the well-separated components
    sd = torch.tensor(s, device="cuda")
    wd = torch.tensor(w, device="cuda")
    t0 = time.perf_counter()
    L0, base, gs, gw = loss_and_grad(gk, h, sd, wd, c, r)
    t_base = time.perf_counter() - t0
    # the sigma part alone against its closed form at converged triplets
    _, gw_sig = h.grad(sigma_bar=2.0 * c * base.sigma, want_s=False, dtype=torch.float64)
    V = host(base.V)
    closed = (2.0 * c * base.sigma) @ (base.sigma[:, None] * V.T ** 2) / w.astype(np.float64)
    closed_err = float(np.abs(host(gw_sig) - closed).max() / np.abs(closed).max())
    # noise of one loss evaluation: a second solve from another start vector
    L0b, _ = loss_and_grad(gk, h, sd, wd, c, r, want_grad=False, seed=11)
    dL = abs(L0b - L0) + 1e-16 * abs(L0)
    v0 = base.V.sum(dim=1)
    v0 = (v0 / torch.linalg.norm(v0)).contiguous()
    rng = np.random.default_rng(spec.seed)
    cw = np.sort(rng.choice(spec.m, ncoords, replace=False))
    cs = np.sort(rng.choice(spec.n, ncoords, replace=False))
    rows = []
    t1 = time.perf_counter()
    pairs = 0
    for side, coords, base_vec, g in (("w", cw, w, gw), ("s", cs, s, gs)):
        for j in coords:
            fd = {}
            for hstep in (1e-6, 1e-4):
                vals = []
                steps = []
                for sign in (1.0, -1.0):
                    pert = base_vec.copy()
                    pert[j] = np.float32(np.float64(base_vec[j]) + sign * hstep)
                    steps.append(np.float64(pert[j]))
                    pt = torch.tensor(pert, device="cuda")
                    if side == "w":
                        Lp, rp = loss_and_grad(gk, h, sd, pt, c, r, v0=v0, want_grad=False)
                    else:
                        Lp, rp = loss_and_grad(gk, h, pt, wd, c, r, v0=v0, want_grad=False)
                    pairs += int(rp.info["matvec_pairs"])
                    vals.append(Lp)
                fd[hstep] = (vals[0] - vals[1]) / (steps[0] - steps[1])
                if hstep == 1e-6:
                    floor = 3.0 * dL / (steps[0] - steps[1])
            gj = float(g[j])
            err6 = abs(fd[1e-6] - gj)
            err4 = abs(fd[1e-4] - gj)
            rows.append({"side": side, "coord": int(j), "grad": gj, "fd_h1e-6": float(fd[1e-6]),
                         "fd_h1e-4": float(fd[1e-4]), "floor": float(floor),
                         "pass_h1e-6": bool(err6 <= 1e-4 * abs(gj) + floor),
                         "rel_err_h1e-4": float(err4 / max(abs(gj), 1e-300))})
    t_fd = time.perf_counter() - t1
    h.set_weights(sd, wd)
    gmax_w, gmax_s = float(np.abs(gw).max()), float(np.abs(gs).max())
    worst6 = max(abs(x["fd_h1e-6"] - x["grad"]) / (1e-4 * abs(x["grad"]) + x["floor"]) for x in rows)
    worst4 = max(x["rel_err_h1e-4"] for x in rows)
    ok = all(x["pass_h1e-6"] for x in rows) and closed_err <= 1e-8
    return {"check": "gradient_20k_x_200k", "n": spec.n, "m": spec.m, "k": k, "L": L0, "loss_noise": dL,
            "base_solve_s": t_base, "fd_solves": 4 * len(rows), "fd_pairs": pairs, "fd_s": t_fd,
            "closed_form_sigma_part_max_rel_err": closed_err, "grad_max_abs_w": gmax_w, "grad_max_abs_s": gmax_s,
            "coords_per_side": ncoords, "worst_err_over_bar_h1e-6": float(worst6),
            "worst_rel_err_h1e-4": float(worst4), "rows": rows, "pass": bool(ok)}


# ---------------------------------------------------------------- 200,000 x 1,000,000

def check_benchmark_200k_x_1m(gk):
    w = synth.CONFIGS["large_200k_x_1m"]
    spec = w.geno
    P, packed = device_matrix(spec)
    h = gk.GKL(P, spec.n)
    runs = {
        "fp32": dict(k=w.k, ell=w.ell, reorth=w.reorth, precision="fp32", tol=w.tol, maxit=3000, seed=7),
        "block": dict(k=w.k, ell=w.extra["block_ell"], precision="block", block=w.extra["block"],
                      k_keep=w.extra["k_keep"], tol=w.tol, maxit=500, seed=7),
    }
    res = {name: solve(h, **kw) for name, kw in runs.items()}
    vecs = {name: (r.sigma.copy(), host(r.U), host(r.V)) for name, (r, _) in res.items()}
    del h, P
    M = oracle.Matrix.from_packed(packed, spec.n)
    # one pass of the oracle's products over both paths' vectors
    sig = np.concatenate([vecs[nm][0] for nm in runs])
    U = np.concatenate([vecs[nm][1] for nm in runs], axis=1)
    V = np.concatenate([vecs[nm][2] for nm in runs], axis=1)
    t0 = time.perf_counter()
    rr = oracle_residuals(M, sig, U, V)
    tor = time.perf_counter() - t0
    out = {"check": "benchmark_200k_x_1m", "n": spec.n, "m": spec.m, "k": w.k, "oracle_products_s": tor, "paths": {}}
    ok = True
    for q, name in enumerate(runs):
        r, dt = res[name]
        rel = rr[q * w.k:(q + 1) * w.k] / r.sigma[0]
        e = {"converged": bool(r.converged), "solve_s": dt, "pairs": int(r.info["matvec_pairs"]),
             "oracle_max_rel_resid": float(rel.max()), "lib_max_rel_resid": float(r.info["max_rel_resid"]),
             "pass": bool(r.converged and rel.max() <= 2 * w.tol)}
        ok = ok and e["pass"]
        out["paths"][name] = e
    f, b = vecs["fp32"][0], vecs["block"][0]
    # both paths' values lie within their residuals of singular values of A
    out["sigma_max_rel_diff_fp32_vs_block"] = float(np.max(np.abs(f - b) / f))
    out["pass"] = ok
    return out


CHECKS = {"null_10k_x_100k": check_null_10k_x_100k, "paths_50k_x_500k": check_paths_50k_x_500k, "gradient_20k_x_200k": check_gradient_20k_x_200k, "benchmark_200k_x_1m": check_benchmark_200k_x_1m}


def markdown(results):
    lines = ["# Parity at the large workloads", "",
             "Written by `python tests/check_large_parity.py " + " ".join(r["check"] for r in results) +
             " --out <path>` on one GB300; the oracle is the FP64 CPU oracle (`oracle/`).", ""]
    for r in results:
        lines.append(f"## {r['check']}: n = {r['n']:,}, m = {r['m']:,} -- {'PASS' if r['pass'] else 'FAIL'}")
        lines.append("")
        if r["check"] == "null_10k_x_100k":
            lines.append(f"sigma_1 = {r['sigma'][0]:.4f}, Marchenko-Pastur edge sqrt(1-f)(sqrt n + sqrt m) = "
                         f"{r['mp_edge']:.4f}, relative {r['sigma1_rel_to_edge']:+.4%} (bar 2%).")
        elif r["check"] in ("paths_50k_x_500k", "benchmark_200k_x_1m"):
            lines.append("| path | converged | solve s | pairs | oracle max r_i/sigma_1 | library's | "
                         "max sigma rel err vs FP64 | max angle vs FP64 |")
            lines.append("|---|---|---|---|---|---|---|---|")
            for name, e in r["paths"].items():
                lines.append(f"| {name} | {e['converged']} | {e['solve_s']:.2f} | {e['pairs']} | "
                             f"{e['oracle_max_rel_resid']:.3e} | {e['lib_max_rel_resid']:.3e} | "
                             f"{e.get('sigma_max_rel_err_vs_fp64', float('nan')):.2e} | "
                             f"{e.get('max_angle_vs_fp64', float('nan')):.2e} |")
            if "sigma_max_rel_diff_fp32_vs_block" in r:
                lines.append("")
                lines.append(f"max |sigma_fp32 - sigma_block| / sigma_fp32 = "
                             f"{r['sigma_max_rel_diff_fp32_vs_block']:.2e}")
        elif r["check"] == "gradient_20k_x_200k":
            lines.append(f"{r['coords_per_side']} coordinates of w and of s; {r['fd_solves']} FP64 solves "
                         f"({r['fd_pairs']} pairs, {r['fd_s']:.1f} s).  Loss L = {r['L']:.6e}, evaluation noise "
                         f"{r['loss_noise']:.2e}.")
            lines.append("")
            lines.append(f"* h = 1e-6: worst |g - FD| / (1e-4 |g| + 3 noise / (2h)) = "
                         f"{r['worst_err_over_bar_h1e-6']:.3f} (pass below 1)")
            lines.append(f"* h = 1e-4: worst |g - FD| / |g| = {r['worst_rel_err_h1e-4']:.2e}")
            lines.append(f"* sigma part vs closed form sigma_i v_ij^2 / w_j: max rel err "
                         f"{r['closed_form_sigma_part_max_rel_err']:.2e}")
        lines.append("")
    return "\n".join(lines) + "\n"


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("checks", nargs="+", choices=sorted(CHECKS))
    ap.add_argument("--out", default="large_parity", help="path prefix of the .md and .jsonl records")
    ap.add_argument("--coords", type=int, default=64, help="gradient_20k_x_200k: coordinates per weight vector")
    args = ap.parse_args()
    oracle.build()
    gk = _lib()
    results = []
    os.makedirs(os.path.dirname(args.out) or ".", exist_ok=True)
    for name in args.checks:
        r = CHECKS[name](gk, args.coords) if name == "gradient_20k_x_200k" else CHECKS[name](gk)
        results.append(r)
        print(json.dumps({k: v for k, v in r.items() if k != "rows"}), flush=True)
        with open(args.out + ".jsonl", "a") as f:
            f.write(json.dumps(r) + "\n")
    with open(args.out + ".md", "w") as f:
        f.write(markdown(results))
    sys.exit(0 if all(r["pass"] for r in results) else 1)


if __name__ == "__main__":
    main()
