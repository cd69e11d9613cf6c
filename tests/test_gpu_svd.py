"""GPU parity of the thick-restarted GKL solver against the FP64 CPU oracle.

Bars: FP64 path, every singular value to 1e-10 of itself (relative); FP32
path, 1e-5 relative.  Singular vectors are compared through
the angle to the oracle's vector, bounded by (residual + rounding)/gap, since
a vector's error is its residual divided by the gap to the rest of the
spectrum (section 3, refined bounds).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import oracle_matrix, small_geno, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gk():
    import torch  # noqa: F401
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl


def angles(X, Y):
    """Angle between matching columns, up to sign, from the chord length
    (accurate down to rounding level, unlike sqrt(1 - cos^2))."""
    Xn = X / np.linalg.norm(X, axis=0)
    Yn = Y / np.linalg.norm(Y, axis=0)
    d = np.minimum(np.linalg.norm(Xn - Yn, axis=0), np.linalg.norm(Xn + Yn, axis=0))
    return 2.0 * np.arcsin(np.minimum(d / 2.0, 1.0))


def gaps(sig):
    s = np.asarray(sig)
    g = np.full(len(s), np.inf)
    d = np.abs(np.diff(s))
    g[:-1] = np.minimum(g[:-1], d)
    g[1:] = np.minimum(g[1:], d)
    return g


def run_pair(gk, g, k, ell, tol, precision, reorth, seed_v0=3, maxit=500, oracle_tol=None, **kw):
    import torch
    M = oracle_matrix(g)
    v0 = synth.normal_vec(seed_v0, 0, g.m)
    ref = oracle.gkl(M, k=k + 2, ell=max(ell, k + 12), tol=oracle_tol or 1e-13, v0=v0, maxit=2000)
    assert ref.converged
    h = gk.GKL(to_dev(g.packed), g.n)
    dt = torch.float64 if precision == "fp64" else torch.float32
    r = h.svd(k=k, ell=ell, reorth=reorth, precision=precision, tol=tol, maxit=maxit,
              v0=torch.tensor(v0, dtype=dt), **kw)
    return M, ref, r


def check_against_oracle(M, ref, r, k, sig_rel, vec_eps, omega=0.0):
    """omega: orthogonality level kept by partial reorthogonalisation; the
    Ritz residual estimate ignores the basis's departure from orthogonality,
    so the true residual may exceed it by up to omega * sigma_1."""
    assert r.converged, r.info
    assert np.all(np.diff(r.sigma) <= 0)
    rel = np.abs(r.sigma - ref.sigma[:k]) / ref.sigma[:k]
    assert rel.max() < sig_rel, (rel.max(), r.sigma[:3], ref.sigma[:3])
    U = r.U.double().cpu().numpy()
    V = r.V.double().cpu().numpy()
    g = gaps(ref.sigma)[:k]
    bound = 10 * (np.maximum(r.resid, 0) + vec_eps * ref.sigma[0]) / g + 1e-12
    assert np.all(angles(V, ref.V[:, :k]) <= bound)
    assert np.all(angles(U, ref.U[:, :k]) <= bound)
    # sign rule: largest-|.| entry of each v is positive
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(k)] > 0)
    # centring (1^T A = 0): 1^T u_i = -1^T r_i / sigma_i for the residual r_i of A v_i = sigma_i u_i
    n = U.shape[0]
    csum = np.abs(U.sum(axis=0))
    cbar = np.sqrt(n) * (2 * np.maximum(r.resid, 0) + (50 * vec_eps + omega) * ref.sigma[0]) / ref.sigma[:k] + 1e-5
    assert np.all(csum <= cbar), (csum, cbar)
    # reported residuals bound the true ones (a-posteriori, computed by the oracle)
    for i in range(k):
        t = np.linalg.norm(M.rmatvec(U[:, i]) - r.sigma[i] * V[:, i])
        assert t <= max(2 * r.resid[i], 0) + (50 * vec_eps + omega) * ref.sigma[0]


def test_fp64_full_two_population_workload(gk):
    w = synth.CONFIGS["fp64_full_1k_x_10k"]
    g = synth.genotypes(w.geno)
    M, ref, r = run_pair(gk, g, w.k, w.ell, w.tol, "fp64", "full")
    check_against_oracle(M, ref, r, w.k, 1e-10, 1e-13)
    assert r.info["restarts"] > 0
    assert r.info["max_rel_resid"] <= w.tol


@pytest.mark.parametrize("reorth", ["full", "partial", "dgks", "onesided"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_admixture_small(gk, precision, reorth):
    g = small_geno(2003, 15_007, pops=5, miss=0.02, seed=41)
    tol = 1e-10 if precision == "fp64" else 1e-6
    M, ref, r = run_pair(gk, g, 10, 28, tol, precision, reorth)
    sig_rel = 1e-10 if precision == "fp64" else 1e-5
    vec_eps = 1e-13 if precision == "fp64" else 3e-6
    omega = 0.0 if reorth in ("full", "dgks") else min(1e-8 if precision == "fp64" else 2.0 ** -12, 10 * tol)
    check_against_oracle(M, ref, r, 10, sig_rel, vec_eps, omega)
    i = r.info
    # one-sided runs recompute the other side's k vectors at the end: half a pair each
    pairs = i["matvec_pairs"] - ((10 + 1) // 2 if reorth == "onesided" else 0)
    if reorth == "partial":
        assert i["reorth_u"] < pairs
    if reorth in ("full", "partial"):
        assert i["second_u"] == 0 and i["second_v"] == 0  # both passes always run, uncounted
    if reorth == "dgks":
        # every step reorthogonalises, and the first pass almost always suffices
        assert i["reorth_v"] == i["matvec_pairs"]
        assert i["second_u"] < i["reorth_u"] // 2 and i["second_v"] < i["reorth_v"] // 2
    if reorth == "onesided":
        # n < m: u (the shorter side) every step, v only when its estimate asks
        assert i["reorth_u"] >= pairs - i["cycles"]
        assert i["reorth_v"] < pairs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_onesided_tall(gk, precision):
    """One-sided reorthogonalisation with more samples than SNPs: the v side
    (the shorter) is reorthogonalised at every step, the u side by its
    estimate, and the k output u vectors are recomputed as A v_i."""
    g = small_geno(6007, 1503, pops=5, miss=0.02, seed=43)
    tol = 1e-10 if precision == "fp64" else 1e-6
    M, ref, r = run_pair(gk, g, 10, 28, tol, precision, "onesided")
    vec_eps = 1e-13 if precision == "fp64" else 3e-6
    omega = min(1e-8 if precision == "fp64" else 2.0 ** -12, 10 * tol)
    check_against_oracle(M, ref, r, 10, 1e-10 if precision == "fp64" else 1e-5, vec_eps, omega)
    i = r.info
    pairs = i["matvec_pairs"] - (10 + 1) // 2
    assert i["reorth_v"] >= pairs - i["cycles"]
    assert i["reorth_u"] < pairs
    # the recomputed u vectors are orthonormal and satisfy A v_i = sigma_i u_i to the residual
    U = r.U.double().cpu().numpy()
    V = r.V.double().cpu().numpy()
    assert np.abs(U.T @ U - np.eye(10)).max() < (1e-12 if precision == "fp64" else 1e-5)
    for j in range(10):
        t = np.linalg.norm(M.matvec(V[:, j]) - r.sigma[j] * U[:, j])
        assert t <= 2 * max(r.resid[j], 0) + (50 * vec_eps + omega) * ref.sigma[0]


def test_tiny_ragged_and_k1(gk):
    g = small_geno(37, 301, pops=2, miss=0.1, seed=5)
    M, ref, r = run_pair(gk, g, 1, 4, 1e-12, "fp64", "full")
    check_against_oracle(M, ref, r, 1, 1e-10, 1e-13)
    M, ref, r = run_pair(gk, g, 6, 20, 1e-12, "fp64", "partial")
    check_against_oracle(M, ref, r, 6, 1e-10, 1e-13, 1e-8)


def test_breakdown_on_duplicated_samples(gk):
    import torch
    from tests.test_oracle_core import pack_codes
    n0, m = 40, 300
    g = synth.genotypes(synth.GenoSpec(n=n0, m=m, n_pops=2, miss_rate=0.0, seed=23))
    codes = np.stack([(g.packed >> (2 * t)) & 3 for t in range(4)], -1).reshape(m, -1)[:, :n0]
    packed = pack_codes(np.concatenate([codes, codes[:, :10]], axis=1))
    M = oracle.Matrix.from_packed(packed, 50)
    sd = np.linalg.svd(M.dense(), compute_uv=False)
    h = gk.GKL(to_dev(packed), 50)
    r = h.svd(k=8, ell=45, tol=1e-12, precision="fp64", v0=torch.tensor(synth.normal_vec(2, 0, m)))
    assert r.converged and r.info["breakdowns"] > 0
    assert np.allclose(r.sigma, sd[:8], rtol=1e-10)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rank_deficient_status(gk, precision):
    """8 distinct samples, each twice: centred, the rank is at most 7.  Asking
    for k = 10 returns GKL_RANK_DEFICIENT with the 7 nonzero values of the
    dense SVD and exact zeros after them."""
    import torch
    from tests.test_oracle_core import pack_codes
    n0, m = 8, 400
    g = synth.genotypes(synth.GenoSpec(n=n0, m=m, n_pops=2, miss_rate=0.0, seed=31))
    codes = np.stack([(g.packed >> (2 * t)) & 3 for t in range(4)], -1).reshape(m, -1)[:, :n0]
    packed = pack_codes(np.concatenate([codes, codes], axis=1))
    M = oracle.Matrix.from_packed(packed, 2 * n0)
    sd = np.linalg.svd(M.dense(), compute_uv=False)
    rank = int(np.sum(sd > 1e-10 * sd[0]))
    assert rank <= 7
    h = gk.GKL(to_dev(packed), 2 * n0)
    tol = 1e-12 if precision == "fp64" else 1e-6
    r = h.svd(k=10, ell=14, tol=tol, precision=precision, maxit=200)
    assert r.status == gk.RANK_DEFICIENT and r.converged
    assert r.info["rank"] == rank
    assert np.all(r.sigma[rank:] == 0.0)
    rel = np.abs(r.sigma[:rank] - sd[:rank]) / sd[:rank]
    assert rel.max() < (1e-10 if precision == "fp64" else 1e-5)


def test_host_outputs_scores_and_sync(gk):
    """out_host=True copies U and V into host memory (same values as the
    device outputs); gkl_scores gives U diag(sigma); gkl_sync reports no
    pending error; a host pointer without out_host is rejected."""
    import torch
    g = small_geno(900, 5000, pops=3, seed=12)
    h = gk.GKL(to_dev(g.packed), g.n)
    for prec in ("fp64", "fp32", "block"):
        kw = dict(k=5, ell=24 if prec != "block" else 48, precision=prec, tol=1e-6, seed=4)
        if prec == "block":
            kw["block"] = 8
        rd = h.svd(**kw)
        rh = h.svd(out_host=True, **kw)
        assert not rh.U.is_cuda and not rh.V.is_cuda
        assert np.array_equal(rd.sigma, rh.sigma)
        assert bool((rd.U.cpu() == rh.U).all()) and bool((rd.V.cpu() == rh.V).all())
        S = h.scores()
        expect = rh.U.double() * torch.tensor(rh.sigma)[None, :]
        assert torch.allclose(S.double().cpu(), expect, rtol=1e-6 if prec != "fp64" else 1e-15, atol=0)
        Sh = h.scores(out_host=True)
        assert bool((Sh == S.cpu()).all())
    h.sync()
    with pytest.raises(gk.GKLError) as e:
        bad = torch.empty(5, g.n, dtype=torch.float64)  # host memory without out_host
        h.svd(k=5, ell=24, precision="fp64", U=bad)
    assert e.value.code == gk.ERR_ARG


def test_not_converged_and_argument_errors(gk):
    g = small_geno(300, 2000, seed=8)
    h = gk.GKL(to_dev(g.packed), 300)
    r = h.svd(k=10, ell=12, tol=1e-14, maxit=1, precision="fp64")
    assert r.status == gk.NOT_CONVERGED and not r.converged
    assert r.info["cycles"] == 1 and np.all(r.sigma > 0)
    with pytest.raises(gk.GKLError) as e:
        h.svd(k=12, ell=12)
    assert e.value.code == gk.ERR_ARG
    with pytest.raises(gk.GKLError):
        h.svd(k=5, ell=301)  # ell > n
    # the C entry points reject vectors that are not device memory of the handle's GPU, before any launch
    import ctypes
    import torch
    lib, vp = gk.lib(), ctypes.c_void_p
    host_m, host_n = np.zeros(2000), np.zeros(300)
    dev_m = torch.zeros(2000, dtype=torch.float64, device="cuda")
    dev_n = torch.zeros(300, dtype=torch.float64, device="cuda")
    hp = lambda a: a.ctypes.data_as(vp)  # noqa: E731
    dp = lambda t: vp(t.data_ptr())  # noqa: E731
    assert lib.gkl_matvec(h._h, gk.FP64, hp(host_m), dp(dev_n)) == gk.ERR_ARG
    assert lib.gkl_matvec(h._h, gk.FP64, dp(dev_m), hp(host_n)) == gk.ERR_ARG
    assert lib.gkl_rmatvec(h._h, gk.FP64, hp(host_n), dp(dev_m)) == gk.ERR_ARG
    assert lib.gkl_rmatvec(h._h, gk.FP64, dp(dev_n), hp(host_m)) == gk.ERR_ARG
    assert b"device memory" in lib.gkl_last_error(h._h)
    X = np.zeros((2, 2000), dtype=np.float32)
    Y = torch.zeros((2, 300), dtype=torch.float32, device="cuda")
    assert lib.gkl_matmat(h._h, 0, 2, 8, hp(X), 2000, dp(Y), 300) == gk.ERR_ARG
    h.sync()
    torch.testing.assert_close(h.matvec(dev_m), dev_n)  # the handle is still usable: A 0 = 0


def test_solver_deterministic(gk):
    g = small_geno(1500, 8000, seed=9)
    h = gk.GKL(to_dev(g.packed), 1500)
    a = h.svd(k=8, ell=24, precision="fp32", reorth="partial", tol=1e-6)
    b = h.svd(k=8, ell=24, precision="fp32", reorth="partial", tol=1e-6)
    assert np.array_equal(a.sigma, b.sigma)
    assert bool((a.U == b.U).all()) and bool((a.V == b.V).all())


def test_full_size_fp32_partial_residuals():
    """10,000 x 100,000, 5-population admixture, 2% missing: k=20, ell=50,
    tol 1e-6, FP32 with partial reorthogonalisation.  Checked a posteriori with
    the oracle's FP64 products: ||A v - sigma u|| and ||A^T u - sigma v||
    relative to sigma_1, orthonormality, and the planted S-1 outliers."""
    import torch
    from paper_1808_03374_gb300 import build, gkl
    build()
    w = synth.CONFIGS["fp32_pro_10k_x_100k"]
    g = synth.genotypes(w.geno)
    M = oracle_matrix(g)
    h = gkl.GKL(to_dev(g.packed), g.n)
    r = h.svd(k=w.k, ell=w.ell, reorth="partial", precision="fp32", tol=w.tol, maxit=2000)
    assert r.converged, r.info
    U = r.U.double().cpu().numpy()
    V = r.V.double().cpu().numpy()
    s1 = r.sigma[0]
    assert np.abs(U.T @ U - np.eye(w.k)).max() < 1e-4
    assert np.abs(V.T @ V - np.eye(w.k)).max() < 1e-4
    for i in range(w.k):
        ra = np.linalg.norm(M.matvec(V[:, i]) - r.sigma[i] * U[:, i]) / s1
        rb = np.linalg.norm(M.rmatvec(U[:, i]) - r.sigma[i] * V[:, i]) / s1
        assert ra < 2 * w.tol and rb < 2 * w.tol  # omega = 10 tol keeps the true residual within tol
    edge = np.sqrt(1 - w.geno.miss_rate) * (np.sqrt(g.n) + np.sqrt(g.m))
    assert (r.sigma[:4] > 1.1 * edge).all() and r.sigma[4] < 1.05 * edge
