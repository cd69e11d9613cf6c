"""Oracle gradient pins: the adjoint formula against the closed form for the
singular-value part and against central finite differences for the full loss
(values + PC scores), on small weighted genotype matrices."""
import numpy as np
import pytest

import synth
from oracle import grad


def setup(n=40, m=90, seed=3, k=4):
    g = synth.genotypes(synth.GenoSpec(n=n, m=m, n_pops=3, admixture=True, miss_rate=0.03, seed=seed))
    s = synth.uniform_vec(seed, 10, n, 0.5, 1.5)
    w = synth.uniform_vec(seed, 11, m, 0.5, 1.5)
    A, A0 = grad.weighted_dense(g.packed, n, s, w)
    c = synth.normal_vec(seed, 12, k)
    r = synth.normal_vec(seed, 13, k)
    return A, A0, s, w, c, r


def test_sigma_part_matches_closed_form():
    A, A0, s, w, c, r = setup()
    k = len(c)
    L, gs, gw = grad.loss_grad(A, A0, s, w, k, c, np.zeros(k))
    gs2, gw2 = grad.sigma_grad_closed_form(A, s, w, k, c)
    assert np.allclose(gw, gw2, rtol=1e-10, atol=1e-12 * np.abs(gw2).max())
    assert np.allclose(gs, gs2, rtol=1e-10, atol=1e-12 * np.abs(gs2).max())


@pytest.mark.parametrize("seed", [3, 4])
def test_full_loss_matches_finite_differences(seed):
    A, A0, s, w, c, r = setup(seed=seed)
    k = len(c)
    L, gs, gw = grad.loss_grad(A, A0, s, w, k, c, r)
    assert np.isclose(L, grad.loss(A, k, c, r), rtol=1e-13)
    rng = np.random.default_rng(seed)
    # 64 random coordinates per weight vector (every one where it has fewer)
    cw = rng.choice(A.shape[1], min(64, A.shape[1]), replace=False)
    cs = rng.choice(A.shape[0], min(64, A.shape[0]), replace=False)
    fs, fw = grad.finite_difference(A0, s, w, k, c, r, cw, cs, h=1e-6)
    scale = max(np.abs(gw).max(), np.abs(gs).max())
    assert np.abs(fw - gw[cw]).max() <= 1e-5 * scale
    assert np.abs(fs - gs[cs]).max() <= 1e-5 * scale


def test_weights_one_reduces_to_unweighted():
    A, A0, s, w, c, r = setup()
    k = len(c)
    one_s, one_w = np.ones_like(s), np.ones_like(w)
    L1, gs1, gw1 = grad.loss_grad(A0, A0, one_s, one_w, k, c, r)
    # with unit weights dL/dw_j = sum_r Abar_rj A0_rj: scaling column j by (1 + t) changes L by t * gw1_j
    t = 1e-6
    j = 5
    Ap = A0.copy()
    Ap[:, j] *= 1 + t
    Am = A0.copy()
    Am[:, j] *= 1 - t
    fd = (grad.loss(Ap, k, c, r) - grad.loss(Am, k, c, r)) / (2 * t)
    assert abs(fd - gw1[j]) <= 1e-5 * np.abs(gw1).max()


def test_cg_form_matches_dense_adjoint():
    # the matrix-free form (own GKL triplets + CG on the complement) equals the
    # dense full-SVD adjoint, for score adjoints on well-separated components
    import oracle
    n, m, k = 60, 150, 4
    g = synth.genotypes(synth.GenoSpec(n=n, m=m, n_pops=3, admixture=True, miss_rate=0.03, seed=7))
    s = synth.uniform_vec(7, 10, n, 0.5, 1.5)
    w = synth.uniform_vec(7, 11, m, 0.5, 1.5)
    A, A0 = grad.weighted_dense(g.packed, n, s, w)
    c = synth.normal_vec(7, 12, k)
    r = np.array([0.7, -1.2, 0.0, 0.0])
    L, gs, gw = grad.loss_grad(A, A0, s, w, k, c, r)
    M0 = oracle.Matrix.from_packed(g.packed, n)
    M = oracle.Matrix(g.packed, n, M0.mu, M0.d, s=s, w=w)
    L2, gs2, gw2, _ = grad.loss_grad_cg(M, k, c, r, ell=30, v0=synth.normal_vec(7, 14, m))
    assert np.isclose(L, L2, rtol=1e-11)
    assert np.abs(gw2 - gw).max() <= 1e-8 * np.abs(gw).max()
    assert np.abs(gs2 - gs).max() <= 1e-8 * np.abs(gs).max()
