"""The oracle's two thick-restart options (section 3: ordinary and harmonic
Ritz values) against LAPACK: both reach the top singular values to FP64
rounding with true residuals at the reported ones, and the ordinary restart
takes exactly the pairs of the C oracle's solver."""
import numpy as np
import pytest

import oracle
import synth
from oracle.restarts import gkl_restarted


@pytest.fixture(scope="module")
def problem():
    g = synth.genotypes(synth.GenoSpec(n=600, m=3000, n_pops=5, admixture=True, miss_rate=0.02, seed=3))
    M = oracle.Matrix.from_packed(g.packed, g.n)
    return M, M.dense(), synth.normal_vec(4, 0, g.m)


@pytest.mark.parametrize("variant", ["ritz", "harmonic"])
def test_restart_variants_against_lapack(problem, variant):
    M, A, v0 = problem
    k = 10
    sv = np.linalg.svd(A, compute_uv=False)
    r = gkl_restarted(A, k=k, ell=30, tol=1e-10, v0=v0, variant=variant)
    assert r.converged and r.restarts > 0
    assert np.max(np.abs(r.sigma - sv[:k]) / sv[:k]) < 1e-13
    true = [max(np.linalg.norm(A @ r.V[:, i] - r.sigma[i] * r.U[:, i]),
                np.linalg.norm(A.T @ r.U[:, i] - r.sigma[i] * r.V[:, i])) for i in range(k)]
    assert np.allclose(true, r.resid, rtol=1e-6, atol=1e-13 * sv[0])
    assert np.max(r.resid) <= 1e-10 * r.sigma[0]
    if variant == "ritz":
        ref = oracle.gkl(M, k=k, ell=30, tol=1e-10, v0=v0, maxit=2000)
        assert (r.pairs, r.restarts) == (ref.pairs, ref.restarts)


@pytest.mark.parametrize("variant", ["ritz", "harmonic"])
def test_matrix_free_equals_dense(problem, variant):
    """The packed operator (the C oracle's products) and its dense copy give
    the same run: pairs, restarts and values to rounding."""
    M, A, v0 = problem
    a = gkl_restarted(A, k=10, ell=30, tol=1e-10, v0=v0, variant=variant)
    b = gkl_restarted(M, k=10, ell=30, tol=1e-10, v0=v0, variant=variant)
    assert (a.pairs, a.restarts) == (b.pairs, b.restarts)
    assert np.max(np.abs(a.sigma - b.sigma) / a.sigma) < 1e-13
