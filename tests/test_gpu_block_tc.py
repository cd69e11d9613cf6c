"""Tensor-core block products (gkl_matmat) against the FP64 oracle, elementwise.

With D digits per vector the kernel holds each input vector in fixed point,
x' = S sum_{p<D} delta_p 16^-(p+1) with S = 2^e >= max|x~| (|x~ - x'| <= 2^-(4D+1) S),
where x~ is the FP32 input block as the kernel forms it (s_i u_i, or d_j w_j v_j
and -mu_j d_j w_j v_j: one to three FP32 roundings, <= 5 2^-24 relative), sums
the products exactly and rounds once to FP32.  With |g - mu| <= 2 per entry:
    A^T U:  |x_j - xo_j| <= 2^-23 |xo_j| + 2 d_j w_j (2^-24 ||s o u||_1 + n 2^-(4D+1) S)
    A V:    |y_i - yo_i| <= 2^-23 |yo_i| + s_i (2^-20 ||d o w o v||_1 + 3 m 2^-(4D+1) S)
"""
import numpy as np
import pytest

import synth
from tests.helpers import oracle_matrix, small_geno, to_dev

pytestmark = pytest.mark.gpu

# ragged in every direction; (600, 40_000) splits the SNPs of A V into several
# chunks, (70_000, 300) spans many sample stages
SHAPES = [(1, 1, 1), (5, 3, 2), (300, 200, 5), (513, 130, 16), (1000, 2000, 32), (4099, 777, 17),
          (600, 40_000, 4), (70_000, 300, 3)]


@pytest.fixture(scope="module")
def gk():
    import torch  # noqa: F401
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl


def pow2_at_least(x):
    mx = np.max(np.abs(x))
    return np.ldexp(1.0, int(np.frexp(mx)[1])) if mx > 0 else 1.0


@pytest.mark.parametrize("n,m,q", SHAPES)
@pytest.mark.parametrize("digits", [8, 4])
@pytest.mark.parametrize("weights", [False, True])
def test_matmat_elementwise(gk, n, m, q, digits, weights):
    import torch
    g = small_geno(n, m, miss=0.03, seed=7 * n + m + q)
    s = synth.uniform_vec(23, 0, n, 0.5, 1.5).astype(np.float32).astype(np.float64) if weights else None
    w = synth.uniform_vec(23, 1, m, 0.5, 1.5).astype(np.float32).astype(np.float64) if weights else None
    M = oracle_matrix(g, s, w)
    h = gk.GKL(to_dev(g.packed), g.n)
    if weights:
        h.set_weights(torch.tensor(s, dtype=torch.float32), torch.tensor(w, dtype=torch.float32))
    sv = s if weights else np.ones(n)
    wv = w if weights else np.ones(m)
    dw = M.d * wv
    # A^T U
    U = np.stack([synth.normal_vec(29, c, n) for c in range(q)]).astype(np.float32)
    X = h.matmat(torch.tensor(U, device="cuda"), transpose=True, digits=digits).double().cpu().numpy()
    for c in range(q):
        u = U[c].astype(np.float64)
        xo = M.rmatvec(u)
        ut = sv * u
        b = 2.0 ** -23 * np.abs(xo) + 2 * dw * (2.0 ** -24 * np.abs(ut).sum() +
                                                n * 2.0 ** -(4 * digits + 1) * pow2_at_least(ut * (1 + 2.0 ** -20))) + 1e-300
        err = np.abs(X[c] - xo)
        assert np.all(err <= b), (c, np.max(err / b))
    # A V
    V = np.stack([synth.normal_vec(31, c, m) for c in range(q)]).astype(np.float32)
    Y = h.matmat(torch.tensor(V, device="cuda"), transpose=False, digits=digits).double().cpu().numpy()
    for c in range(q):
        v = V[c].astype(np.float64)
        yo = M.matvec(v)
        vt = dw * v
        S = pow2_at_least(np.maximum(np.abs(vt), np.abs(M.mu * vt)) * (1 + 2.0 ** -20))
        b = 2.0 ** -23 * np.abs(yo) + sv * (2.0 ** -20 * np.abs(vt).sum() +
                                            3 * m * 2.0 ** -(4 * digits + 1) * S) + 1e-300
        err = np.abs(Y[c] - yo)
        assert np.all(err <= b), (c, np.max(err / b))


def test_matmat_digits8_near_fp32(gk):
    """8 digits: the products agree with the FP64 oracle to FP32 rounding level
    (relative to the row's |A||x| scale) on a 10-vector block."""
    import torch
    n, m, q = 2000, 5000, 10
    g = small_geno(n, m, miss=0.02, seed=91)
    M = oracle_matrix(g)
    h = gk.GKL(to_dev(g.packed), g.n)
    V = np.stack([synth.normal_vec(37, c, m) for c in range(q)]).astype(np.float32)
    Y = h.matmat(torch.tensor(V, device="cuda")).double().cpu().numpy()
    for c in range(q):
        yo = M.matvec(V[c].astype(np.float64))
        assert np.max(np.abs(Y[c] - yo)) <= 1e-6 * np.max(np.abs(yo))


def test_matmat_arguments(gk):
    import torch
    g = small_geno(100, 50, seed=3)
    h = gk.GKL(to_dev(g.packed), g.n)
    X = torch.zeros((4, 50), device="cuda")
    with pytest.raises(gk.GKLError):
        h.matmat(X, digits=5)
    with pytest.raises(gk.GKLError):
        h.matmat(torch.zeros((33, 50), device="cuda"))


def test_full_size_block_products_sampled(gk):
    """10,000 x 100,000 workload (2% missing, 5-population admixture), 16
    vectors in 8 digits (the block solver's launch configuration) and 32 in 4:
    sampled outputs of both products against the oracle's one-by-one rows and
    columns, within the elementwise bound of the header."""
    import torch
    w = synth.CONFIGS["fp32_pro_10k_x_100k"]
    g = synth.genotypes(w.geno)
    M = oracle_matrix(g)
    h = gk.GKL(to_dev(g.packed), g.n)
    rng = np.random.default_rng(1)
    rows = np.unique(np.r_[0, g.n - 1, rng.integers(0, g.n, 24)])
    cols = np.unique(np.r_[0, g.m - 1, rng.integers(0, g.m, 24)])
    dw = M.d
    for q, digits in ((16, 8), (32, 4)):
        U = np.stack([synth.normal_vec(41, c, g.n) for c in range(q)]).astype(np.float32)
        V = np.stack([synth.normal_vec(43, c, g.m) for c in range(q)]).astype(np.float32)
        X = h.matmat(torch.tensor(U, device="cuda"), transpose=True, digits=digits).double().cpu().numpy()
        Y = h.matmat(torch.tensor(V, device="cuda"), digits=digits).double().cpu().numpy()
        for c in range(q):
            u = U[c].astype(np.float64)
            v = V[c].astype(np.float64)
            xo = M.rmatvec_cols(u, cols)
            yo = M.matvec_rows(v, rows)
            bx = 2.0 ** -23 * np.abs(xo) + 2 * dw[cols] * (2.0 ** -24 * np.abs(u).sum() +
                                                        g.n * 2.0 ** -(4 * digits + 1) * pow2_at_least(u * (1 + 2.0 ** -20)))
            vt = dw * v
            S = pow2_at_least(np.maximum(np.abs(vt), np.abs(M.mu * vt)) * (1 + 2.0 ** -20))
            by = 2.0 ** -23 * np.abs(yo) + (2.0 ** -20 * np.abs(vt).sum() + 3 * g.m * 2.0 ** -(4 * digits + 1) * S)
            assert np.all(np.abs(X[c][cols] - xo) <= bx), (q, digits, c)
            assert np.all(np.abs(Y[c][rows] - yo) <= by), (q, digits, c)
