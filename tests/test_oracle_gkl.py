"""Oracle GKL pins: brute force, Lanczos invariants, residual bound, planted
structure and the Marchenko-Pastur null (section 2 Eq. 5; section 3)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import mp


def small_matrix(n=120, m=700, pops=3, miss=0.02, seed=21, **kw):
    g = synth.genotypes(synth.GenoSpec(n=n, m=m, n_pops=pops, admixture=True, miss_rate=miss, seed=seed, **kw))
    return g, oracle.Matrix.from_packed(g.packed, n)


def principal_cosines(X, Y):
    qx, _ = np.linalg.qr(X)
    qy, _ = np.linalg.qr(Y)
    return np.linalg.svd(qx.T @ qy, compute_uv=False)


@pytest.mark.parametrize("ell,k", [(30, 6), (14, 6)])
def test_gkl_matches_lapack_svd(ell, k):
    g, M = small_matrix()
    A = M.dense()
    Ud, sd, Vdt = np.linalg.svd(A, full_matrices=False)
    r = oracle.gkl(M, k=k, ell=ell, tol=1e-13, v0=synth.normal_vec(9, 0, M.m), maxit=500)
    assert r.converged
    if ell == 14:
        assert r.restarts > 0
    assert np.allclose(r.sigma, sd[:k], rtol=1e-12, atol=0)
    gaps = np.minimum(np.abs(np.diff(sd[:k + 1])), np.r_[np.inf, np.abs(np.diff(sd[:k]))])
    for i in range(k):
        # singular vectors agree up to sign; error bounded by resid/gap
        cu = abs(r.U[:, i] @ Ud[:, i])
        cv = abs(r.V[:, i] @ Vdt[i])
        tolv = 1e-10 * sd[0] / gaps[i]
        assert 1 - cv < tolv and 1 - cu < tolv
    # reported residuals are the true residuals of the returned triplets
    for i in range(k):
        ru = np.linalg.norm(A.T @ r.U[:, i] - r.sigma[i] * r.V[:, i])
        rv = np.linalg.norm(A @ r.V[:, i] - r.sigma[i] * r.U[:, i])
        assert rv < 1e-12 * sd[0]
        assert abs(ru - r.resid[i]) < 1e-11 * sd[0]
    # sign rule
    for i in range(k):
        j = np.argmax(np.abs(r.V[:, i]))
        assert r.V[j, i] > 0


def test_lanczos_invariants_after_restart():
    g, M = small_matrix(n=150, m=900, seed=22)
    A = M.dense()
    ell, k = 16, 5
    r = oracle.gkl(M, k=k, ell=ell, tol=1e-30, v0=synth.normal_vec(9, 1, M.m), maxit=3, bases=True)
    assert r.restarts == 2 and not r.converged
    Ub, Vb, B = r.Ub, r.Vb, r.B
    nA = np.linalg.norm(A, 2)
    # A V_ell = U_ell B_ell (B upper triangular: diagonal, spike column k', bidiagonal)
    assert np.linalg.norm(A @ Vb[:, :ell] - Ub @ B) / nA < 1e-12
    assert np.abs(Ub.T @ Ub - np.eye(ell)).max() < 1e-12
    assert np.abs(Vb.T @ Vb - np.eye(ell + 1)).max() < 1e-12
    kk = k + (ell - k) // 2
    # structure of B after a thick restart
    assert np.allclose(np.triu(B), B)
    assert np.allclose(B[:kk, :kk], np.diag(np.diag(B[:kk, :kk])))
    # the spike equals U_k'^T A v_k'
    assert np.allclose(Ub[:, :kk].T @ (A @ Vb[:, kk]), B[:kk, kk], atol=1e-12 * nA)
    # A^T U_ell = V_ell B^T + beta v_{ell+1} e_ell^T: the residual sits only in the last column
    R = A.T @ Ub - Vb[:, :ell] @ B.T
    assert np.linalg.norm(R[:, :-1]) / nA < 1e-12
    assert np.abs(Vb[:, :ell].T @ R[:, -1]).max() / nA < 1e-12


def test_rank_deficient_duplicates_breakdown():
    # kinship: duplicated samples produce exact zero singular values (section 1)
    n0, m = 40, 300
    g = synth.genotypes(synth.GenoSpec(n=n0, m=m, n_pops=2, miss_rate=0.0, seed=23))
    codes = np.stack([(g.packed >> (2 * t)) & 3 for t in range(4)], -1).reshape(m, -1)[:, :n0]
    dup = np.concatenate([codes, codes[:, :10]], axis=1)  # 50 samples, rank <= 40
    from tests.test_oracle_core import pack_codes
    packed = pack_codes(dup)
    M = oracle.Matrix.from_packed(packed, 50)
    A = M.dense()
    sd = np.linalg.svd(A, compute_uv=False)
    assert sd[40:].max() < 1e-10 * sd[0]
    # ask for all 39 informative values plus 1 zero -> the recurrence meets breakdown
    r = oracle.gkl(M, k=8, ell=45, tol=1e-12, v0=synth.normal_vec(2, 0, m), maxit=50)
    assert r.converged and r.breakdowns > 0
    assert np.allclose(r.sigma, sd[:8], rtol=1e-11)


def test_planted_two_population_outlier():
    w = synth.CONFIGS["fp64_full_1k_x_10k"]
    g = synth.genotypes(w.geno)
    M = oracle.Matrix.from_packed(g.packed, w.geno.n)
    r = oracle.gkl(M, k=w.k, ell=w.ell, tol=w.tol, v0=synth.normal_vec(11, 0, M.m), maxit=300)
    assert r.converged and r.max_rel_resid <= w.tol
    f = w.geno.miss_rate
    edge = np.sqrt(1 - f) * (np.sqrt(w.geno.n) + np.sqrt(w.geno.m))
    assert r.sigma[0] > 1.2 * edge
    assert r.sigma[1] < 1.05 * edge
    pop = g.q[:, 1] > 0.5
    s = np.sign(r.U[:, 0])
    agree = max(np.mean(s[pop] > 0) + np.mean(s[~pop] < 0), np.mean(s[pop] < 0) + np.mean(s[~pop] > 0)) / 2
    assert agree >= 0.99
    # ||Delta theta||_1 (Table 3) is the sum of the reported residuals
    from numpy.testing import assert_allclose
    assert_allclose(r.dtheta1, r.resid.sum(), rtol=1e-14)


def test_admixture_outliers_span_ancestry():
    S = 5
    g = synth.genotypes(synth.GenoSpec(n=2000, m=20_000, n_pops=S, admixture=True, miss_rate=0.02, seed=24))
    M = oracle.Matrix.from_packed(g.packed, 2000)
    r = oracle.gkl(M, k=8, ell=24, tol=1e-8, v0=synth.normal_vec(12, 0, M.m), maxit=300)
    assert r.converged
    edge = np.sqrt(0.98) * (np.sqrt(2000) + np.sqrt(20000))
    assert (r.sigma[:S - 1] > 1.1 * edge).all()
    assert r.sigma[S - 1] < 1.05 * edge
    Qc = g.q - g.q.mean(0)
    cos = principal_cosines(r.U[:, :S - 1], Qc[:, :S - 1])
    assert cos.min() >= 0.95


def test_null_model_bulk_follows_marchenko_pastur():
    n, m, f = 1000, 10_000, 0.02
    spec = synth.null_variant(synth.GenoSpec(n=n, m=m, miss_rate=f, seed=25))
    g = synth.genotypes(spec)
    M = oracle.Matrix.from_packed(g.packed, n)
    A = M.dense()
    s = np.linalg.svd(A, compute_uv=False)
    _, _, nobs = oracle.colstats(g.packed, n)
    sigma2 = nobs[M.d > 0].sum() / (n * m)  # mean entry variance, ~1 - f
    # Frobenius closed form: sum sigma^2 = ||A||_F^2 = sum_j n_obs,j over non-monomorphic SNPs
    assert np.isclose((s ** 2).sum(), nobs[M.d > 0].sum(), rtol=1e-10)
    ks = mp.ks_distance(s / np.sqrt(m), y=n / m, sigma=np.sqrt(sigma2))
    assert ks <= 0.03
    edge = np.sqrt(sigma2) * (np.sqrt(n) + np.sqrt(m))
    assert abs(s[0] / edge - 1) < 0.02
