"""Block form (GKL_BLOCK: blocks of b vectors, FP32 bases, tensor-core block
products, FP64 projected matrix, final Rayleigh-Ritz step) against the FP64
oracle.

Bars: singular values 1e-6 relative to sigma_1 (the Rayleigh-Ritz values are
accurate to the square of the subspace angle); vector angles within
10 (residual + 3e-6 sigma_1) / gap; the reported residuals are the true ones,
||A^T u_i - sigma_i v_i|| from the library's own products: they agree with the
oracle's to 1e-6 sigma_1 (FP32 rounding of the vectors)."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import oracle_matrix, small_geno, to_dev
from tests.test_gpu_svd import angles, gaps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gk():
    import torch  # noqa: F401
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl


def check(M, ref, r, k):
    assert r.converged, r.info
    assert np.all(np.diff(r.sigma) <= 0)
    rel = np.abs(r.sigma - ref.sigma[:k]) / ref.sigma[:k]
    assert rel.max() < 1e-6, (rel.max(), r.sigma[:4], ref.sigma[:4])
    U = r.U.double().cpu().numpy()
    V = r.V.double().cpu().numpy()
    g = gaps(ref.sigma)[:k]
    bound = 10 * (np.maximum(r.resid, 0) + 3e-6 * ref.sigma[0]) / g + 1e-12
    assert np.all(angles(V, ref.V[:, :k]) <= bound)
    assert np.all(angles(U, ref.U[:, :k]) <= bound)
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(k)] > 0)
    for i in range(k):
        t = np.linalg.norm(M.rmatvec(U[:, i]) - r.sigma[i] * V[:, i])
        assert abs(t - r.resid[i]) <= 1e-6 * ref.sigma[0], (i, t, r.resid[i])


@pytest.mark.parametrize("b,ell", [(8, 48), (32, 128)])
def test_block_admixture(gk, b, ell):
    g = small_geno(1503, 9_001, pops=5, miss=0.02, seed=61)
    M = oracle_matrix(g)
    k = 10
    ref = oracle.gkl(M, k=k + 2, ell=40, tol=1e-13, v0=synth.normal_vec(4, 0, g.m), maxit=2000)
    assert ref.converged
    h = gk.GKL(to_dev(g.packed), g.n)
    r = h.svd(k=k, ell=ell, precision="block", block=b, tol=1e-6, maxit=200, seed=9)
    check(M, ref, r, k)
    # blocks of b, plus k per Rayleigh-Ritz step (one, and one more per refinement)
    assert (r.info["matvec_pairs"] - k * (1 + r.info["refine_cycles"])) % b == 0
    assert r.info["converged"] and r.info["max_rel_resid"] <= 1e-6


def test_block_ragged_sizes(gk):
    g = small_geno(301, 2_003, pops=3, miss=0.05, seed=62)
    M = oracle_matrix(g)
    ref = oracle.gkl(M, k=7, ell=30, tol=1e-13, v0=synth.normal_vec(5, 0, g.m), maxit=2000)
    h = gk.GKL(to_dev(g.packed), g.n)
    r = h.svd(k=5, ell=60, precision="block", block=12, tol=1e-6, maxit=200, seed=3)
    check(M, ref, r, 5)


def test_block_rank_deficient_replaces_directions(gk):
    """Duplicated samples make A rank-deficient (rank <= 40): the block Krylov
    space exhausts the range and the dependent directions are replaced by random
    vectors; the top singular values are still found."""
    from tests.test_oracle_core import pack_codes
    n0, m = 40, 400
    g = synth.genotypes(synth.GenoSpec(n=n0, m=m, n_pops=2, miss_rate=0.0, seed=29))
    codes = np.stack([(g.packed >> (2 * t)) & 3 for t in range(4)], -1).reshape(m, -1)[:, :n0]
    packed = pack_codes(np.concatenate([codes, codes[:, :24]], axis=1))
    M = oracle.Matrix.from_packed(packed, 64)
    sd = np.linalg.svd(M.dense(), compute_uv=False)
    h = gk.GKL(to_dev(packed), 64)
    r = h.svd(k=6, ell=48, precision="block", block=8, tol=1e-6, maxit=100, seed=4)
    assert r.converged and r.info["breakdowns"] > 0
    assert np.allclose(r.sigma, sd[:6], rtol=1e-5)


def test_block_argument_errors(gk):
    g = small_geno(200, 500, seed=63)
    h = gk.GKL(to_dev(g.packed), g.n)
    for kw in (dict(k=5, ell=40, block=33), dict(k=5, ell=40, block=24), dict(k=40, ell=40, block=8),
               dict(k=5, ell=40, block=8, k_keep=7)):
        with pytest.raises(gk.GKLError) as e:
            h.svd(precision="block", tol=1e-6, **kw)
        assert e.value.code == gk.ERR_ARG


def test_block_two_pass_and_large_k(gk):
    """reorth="full" (two block Gram-Schmidt passes always) gives the same
    solution as the default adaptive second pass; k > 32 skips the
    Rayleigh-Ritz step (Ritz values from the projected SVD, FP32-level
    accuracy)."""
    g = small_geno(700, 3_001, pops=3, miss=0.02, seed=64)
    M = oracle_matrix(g)
    ref = oracle.gkl(M, k=42, ell=90, tol=1e-12, v0=synth.normal_vec(6, 0, g.m), maxit=3000)
    h = gk.GKL(to_dev(g.packed), g.n)
    r2 = h.svd(k=6, ell=48, precision="block", block=8, tol=1e-6, maxit=200, seed=5, reorth="full")
    check(M, ref, r2, 6)
    r1 = h.svd(k=6, ell=48, precision="block", block=8, tol=1e-6, maxit=200, seed=5)
    check(M, ref, r1, 6)
    assert r2.info["second_v"] >= r1.info["second_v"]
    r = h.svd(k=40, ell=96, precision="block", block=8, tol=1e-6, maxit=400, seed=5)
    assert r.converged
    rel = np.abs(r.sigma - ref.sigma[:40]) / ref.sigma[:40]
    assert rel.max() < 1e-5, rel.max()


def test_block16_split_precision_refined(gk):
    """GKL_BLOCK16: the iteration runs on 16-bit fixed-point products (32
    vectors per tensor-core pass); the final Rayleigh-Ritz step with 8-digit
    products brings the singular values to 1e-6 of the FP64 oracle."""
    g = small_geno(1503, 9_001, pops=5, miss=0.02, seed=61)
    M = oracle_matrix(g)
    k = 10
    ref = oracle.gkl(M, k=k + 2, ell=40, tol=1e-13, v0=synth.normal_vec(4, 0, g.m), maxit=2000)
    h = gk.GKL(to_dev(g.packed), g.n)
    r = h.svd(k=k, ell=128, precision="block16", block=32, tol=1e-5, maxit=200, seed=9)
    check(M, ref, r, k)
