"""GPU gradients (gkl_grad behind GKLFunction) against the FP64 oracle and
central finite differences.

Loss: L = sum_i c_i sigma_i^2 + || S r ||^2, S = U diag(sigma) the PC scores.
Score adjoints are taken on well-separated components (the population
outliers), as the gradient of a singular vector needs a gap.  Bar: 1e-7
relative (FP64 path), 1e-4 relative (FP32 path)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import grad
from tests.helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gk():
    import torch  # noqa: F401
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl


def problem(n, m, pops, seed, k):
    g = synth.genotypes(synth.GenoSpec(n=n, m=m, n_pops=pops, admixture=True, miss_rate=0.02, seed=seed))
    s = synth.uniform_vec(seed, 10, n, 0.5, 1.5).astype(np.float32).astype(np.float64)
    w = synth.uniform_vec(seed, 11, m, 0.5, 1.5).astype(np.float32).astype(np.float64)
    c = synth.normal_vec(seed, 12, k)
    r = np.zeros(k)
    r[:pops - 1] = synth.normal_vec(seed, 13, pops - 1)
    return g, s, w, c, r


def gpu_loss_grad(gk, g, s, w, c, r, k, ell, precision, tol):
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    h = gk.GKL(to_dev(g.packed), g.n)
    st = torch.tensor(s, dtype=torch.float32, device="cuda", requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float32, device="cuda", requires_grad=True)
    kw = dict(k=k, ell=ell, precision=precision, tol=tol, maxit=3000, seed=5)
    sigma, scores = gk.GKLFunction.apply(st, wt, h, kw, 1e-3)
    L = (torch.tensor(c, device="cuda") * sigma ** 2).sum() + ((scores.double() @ torch.tensor(r, device="cuda")) ** 2).sum()
    L.backward()
    gpu_loss_grad.sigma = sigma.detach().cpu().numpy()
    return float(L.detach()), st.grad.double().cpu().numpy(), wt.grad.double().cpu().numpy(), h


def test_fp64_tiny_matches_dense_adjoint_and_fd(gk):
    n, m, k = 120, 700, 4
    g, s, w, c, r = problem(n, m, 3, 31, k)
    L, gs, gw, h = gpu_loss_grad(gk, g, s, w, c, r, k, 24, "fp64", 1e-13)
    A, A0 = grad.weighted_dense(g.packed, n, s, w)
    Lo, gso, gwo = grad.loss_grad(A, A0, s, w, k, c, r)
    assert np.isclose(L, Lo, rtol=1e-9)
    assert np.abs(gw - gwo).max() <= 1e-7 * np.abs(gwo).max()
    assert np.abs(gs - gso).max() <= 1e-7 * np.abs(gso).max()
    # central differences of the oracle loss at a few coordinates
    rng = np.random.default_rng(0)
    cw, cs = rng.choice(m, 6, replace=False), rng.choice(n, 6, replace=False)
    fs, fw = grad.finite_difference(A0, s, w, k, c, r, cw, cs, h=1e-6)
    sc = max(np.abs(gwo).max(), np.abs(gso).max())
    assert np.abs(fw - gw[cw]).max() <= 1e-5 * sc
    assert np.abs(fs - gs[cs]).max() <= 1e-5 * sc


def test_sigma_only_matches_closed_form(gk):
    # at exact triplets dsigma_i/dw_j = sigma_i v_ij^2 / w_j; computed vectors
    # are accurate to residual / gap, so the 1e-8 bar is applied to the
    # well-separated components (the population outliers)
    n, m, k = 200, 1500, 5
    g, s, w, c, r = problem(n, m, 3, 32, k)
    c[2:] = 0.0
    L, gs, gw, h = gpu_loss_grad(gk, g, s, w, c, np.zeros(k), k, 24, "fp64", 1e-13)
    A, A0 = grad.weighted_dense(g.packed, n, s, w)
    gs2, gw2 = grad.sigma_grad_closed_form(A, s, w, k, c)
    # through autograd the gradients come back in the weights' dtype (float32)
    assert np.abs(gw - gw2).max() <= 1e-7 * np.abs(gw2).max()
    # the FP64 gradient itself, straight from the handle
    gs, gw = h.grad(2 * c * gpu_loss_grad.sigma)
    gs, gw = gs.cpu().numpy(), gw.cpu().numpy()
    assert np.abs(gw - gw2).max() <= 1e-8 * np.abs(gw2).max()
    assert np.abs(gs - gs2).max() <= 1e-8 * np.abs(gs2).max()


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-7), ("fp32", 1e-4)])
def test_moderate_size_matches_matrix_free_oracle(gk, precision, bar):
    n, m, k = 2000, 20_000, 6
    g, s, w, c, r = problem(n, m, 5, 33, k)
    L, gs, gw, h = gpu_loss_grad(gk, g, s, w, c, r, k, 30, precision, 1e-12 if precision == "fp64" else 1e-6)
    M0 = oracle.Matrix.from_packed(g.packed, n)
    M = oracle.Matrix(g.packed, n, M0.mu, M0.d, s=s, w=w)
    Lo, gso, gwo, res = grad.loss_grad_cg(M, k, c, r, ell=30, v0=synth.normal_vec(33, 14, m))
    assert np.isclose(L, Lo, rtol=bar)
    assert np.linalg.norm(gw - gwo) <= bar * np.linalg.norm(gwo)
    assert np.linalg.norm(gs - gso) <= bar * np.linalg.norm(gso)


def test_gap_and_state_errors(gk):
    import torch
    g, s, w, c, r = problem(150, 900, 3, 34, 6)
    h = gk.GKL(to_dev(g.packed), 150)
    with pytest.raises(gk.GKLError) as e:
        h.grad(np.ones(6))
    assert e.value.code == gk.ERR_STATE
    res = h.svd(k=6, ell=24, precision="fp64", tol=1e-12)
    assert res.converged
    # a score adjoint on a bulk component with a tiny gap is refused
    Sbar = torch.zeros(150, 6, dtype=torch.float64)
    Sbar[:, 4] = 1.0
    with pytest.raises(gk.GKLError) as e:
        h.grad(None, Sbar, min_relgap=0.5)
    assert e.value.code == gk.ERR_GAP


def test_weight_change_and_resolve_invalidate_triplets(gk):
    """gkl_set_weights changes the operator: the stored triplets no longer
    serve gkl_grad (GKL_ERR_STATE) until the next solve; an autograd backward
    whose handle was solved again after its forward pass refuses too."""
    import torch
    g, s, w, c, r = problem(150, 900, 3, 35, 6)
    h = gk.GKL(to_dev(g.packed), 150)
    res = h.svd(k=6, ell=24, precision="fp64", tol=1e-12)
    assert res.converged
    h.grad(np.ones(6), want_s=False)
    h.set_weights(torch.tensor(s, dtype=torch.float32), torch.tensor(w, dtype=torch.float32))
    with pytest.raises(gk.GKLError) as e:
        h.grad(np.ones(6), want_s=False)
    assert e.value.code == gk.ERR_STATE
    with pytest.raises(gk.GKLError) as e:
        h.scores()
    assert e.value.code == gk.ERR_STATE
    st = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    kw = dict(k=6, ell=24, precision="fp64", tol=1e-12)
    sigma, scores = gk.GKLFunction.apply(st, wt, h, kw, 1e-3)
    h.svd(**kw)  # the handle now holds another solve's triplets
    with pytest.raises(gk.GKLError) as e:
        (sigma ** 2).sum().backward()
    assert e.value.code == gk.ERR_STATE


def test_sigma_gradient_after_block_solve(gk):
    """The block form leaves its (FP32) triplets in the handle: the sigma part
    of the gradient equals its closed form 2 sum_i sigma_i^2 v_ij^2 / w_j."""
    import torch
    g, s, w, c, r = problem(700, 4000, 3, 36, 6)
    h = gk.GKL(to_dev(g.packed), 700)
    h.set_weights(None, torch.tensor(w, dtype=torch.float32))
    res = h.svd(k=6, ell=48, precision="block", block=8, tol=1e-6, seed=2)
    assert res.converged
    _, gw = h.grad(2.0 * res.sigma, want_s=False)
    assert gw.dtype == torch.float32
    V = res.V.double().cpu().numpy()
    closed = 2.0 * (V ** 2) @ (res.sigma ** 2) / w.astype(np.float32).astype(np.float64)
    err = np.abs(gw.double().cpu().numpy() - closed).max() / np.abs(closed).max()
    assert err < 1e-4, err
