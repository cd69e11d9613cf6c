"""Oracle pins: decode, standardisation, products and the Jacobi SVD.

Each check ties the oracle to something outside itself: a hand-worked example,
NumPy/LAPACK on small dense matrices, or a closed form of the standardised
matrix (zero column sums, column norms equal to the observed counts).
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def pack_codes(codes, stride=None):
    """Pure-Python packing of an int matrix [m, n] of codes 0..3 (3 = missing)."""
    codes = np.asarray(codes, dtype=np.int64)
    m, n = codes.shape
    stride = stride or synth.padded_stride(n)
    out = np.full((m, stride), 0xFF, dtype=np.uint8)
    for j in range(m):
        for i in range(n):
            b = int(out[j, i >> 2])
            sh = 2 * (i & 3)
            out[j, i >> 2] = (b & ~(3 << sh) & 0xFF) | (int(codes[j, i]) << sh)
    return out


def read_hand():
    sec, data = None, {}
    for line in open(os.path.join(GOLDEN, "hand_decode.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.isalpha():
            sec = line
            data[sec] = []
            continue
        data[sec].append([float(x) for x in line.split()])
    return data


def test_hand_worked_decode():
    h = read_hand()
    codes = np.array(h["codes"], dtype=np.int64)
    packed = pack_codes(codes)
    n = codes.shape[1]
    mu, d, nobs = oracle.colstats(packed, n)
    assert np.array_equal(nobs, np.array(h["nobs"][0], dtype=np.int64))
    assert np.array_equal(mu, np.array(h["mu"][0]))
    assert np.allclose(d, np.array(h["d"][0]), rtol=2e-16, atol=0)
    A = oracle.Matrix(packed, n, mu, d).dense()
    expect = np.where(codes.T < 3, (codes.T - mu) * d, 0.0)
    assert np.array_equal(A, expect)
    # SNP 0: (0-1)*sqrt2, (1-1)*sqrt2, (2-1)*sqrt2, missing, 0
    assert A[0, 0] == -d[0] and A[2, 0] == d[0] and A[3, 0] == 0.0


def _random_case(n, m, seed, miss=0.05):
    g = synth.genotypes(synth.GenoSpec(n=n, m=m, n_pops=3, admixture=True, miss_rate=miss, seed=seed))
    return g, oracle.Matrix.from_packed(g.packed, n)


def test_colstats_match_numpy_nan_statistics():
    g, M = _random_case(203, 150, 11)
    codes = np.stack([(g.packed >> (2 * t)) & 3 for t in range(4)], -1).reshape(150, -1)[:, :203].astype(float)
    codes[codes == 3] = np.nan
    assert np.allclose(M.mu, np.nanmean(codes, axis=1), rtol=1e-15, atol=0)
    sd = np.nanstd(codes, axis=1)
    assert np.allclose(M.d, np.where(sd > 0, 1 / sd, 0), rtol=1e-13)


def test_standardised_closed_forms():
    # every column sums to zero (centring) and has squared norm n_obs (population SD)
    g, M = _random_case(301, 97, 12)
    A = M.dense()
    _, _, nobs = oracle.colstats(g.packed, 301)
    assert np.abs(A.sum(0)).max() < 1e-11
    nz = M.d > 0
    assert np.allclose((A ** 2).sum(0)[nz], nobs[nz], rtol=1e-12)
    assert np.allclose((A ** 2).sum(), nobs[nz].sum(), rtol=1e-12)


@pytest.mark.parametrize("weights", [False, True])
def test_products_match_dense(weights):
    n, m = 157, 211
    g, M = _random_case(n, m, 13)
    if weights:
        M = oracle.Matrix(g.packed, n, M.mu, M.d, s=synth.uniform_vec(5, 0, n, 0.5, 1.5),
                          w=synth.uniform_vec(5, 1, m, 0.5, 1.5))
        A0 = oracle.Matrix(g.packed, n, M.mu, M.d).dense()
        assert np.allclose(M.dense(), M.s[:, None] * A0 * M.w[None, :], rtol=1e-15, atol=1e-15)
    A = M.dense()
    v, u = synth.normal_vec(3, 0, m), synth.normal_vec(3, 1, n)
    assert np.allclose(M.matvec(v), A @ v, rtol=1e-12, atol=1e-12)
    assert np.allclose(M.rmatvec(u), A.T @ u, rtol=1e-12, atol=1e-12)
    rows, cols = np.array([0, 5, n - 1]), np.array([1, m - 1, 77])
    assert np.allclose(M.matvec_rows(v, rows), (A @ v)[rows], rtol=1e-12)
    assert np.allclose(M.rmatvec_cols(u, cols), (A.T @ u)[cols], rtol=1e-12)


@pytest.mark.parametrize("n,m,k", [(157, 211, 3), (1030, 97, 5), (1, 3, 1)])
def test_block_products_match_dense(n, m, k):
    """A X and A^T U for k vectors against NumPy's dense products (a library
    routine), across more than one 512-sample tile and a ragged tail; and each
    column equal, bit for bit, to the single-vector product (same sums in the
    same order)."""
    g, M = _random_case(n, m, 21 + k)
    M = oracle.Matrix(g.packed, n, M.mu, M.d, s=synth.uniform_vec(7, 0, n, 0.5, 1.5),
                      w=synth.uniform_vec(7, 1, m, 0.5, 1.5))
    A = M.dense()
    X = np.stack([synth.normal_vec(9, c, m) for c in range(k)], axis=1)
    U = np.stack([synth.normal_vec(10, c, n) for c in range(k)], axis=1)
    Y, Z = M.matmat(X), M.rmatmat(U)
    assert np.allclose(Y, A @ X, rtol=1e-12, atol=1e-12)
    assert np.allclose(Z, A.T @ U, rtol=1e-12, atol=1e-12)
    for c in range(k):
        assert np.array_equal(Y[:, c], M.matvec(X[:, c]))
        assert np.array_equal(Z[:, c], M.rmatvec(U[:, c]))


def test_unit_vector_products_are_single_rounded_entries():
    # A e_j is column j exactly: ((double)c - mu_j) * d_j with no other rounding
    n, m = 90, 40
    g, M = _random_case(n, m, 14)
    A = M.dense()
    for j in (0, 7, m - 1):
        e = np.zeros(m)
        e[j] = 1.0
        assert np.array_equal(M.matvec(e), A[:, j])
    for i in (0, 45, n - 1):
        e = np.zeros(n)
        e[i] = 1.0
        assert np.array_equal(M.rmatvec(e), A[i, :])


@pytest.mark.parametrize("shape", [(40, 25), (30, 30), (200, 7)])
def test_jacobi_matches_lapack(shape):
    rng = np.random.default_rng(1)
    A = rng.standard_normal(shape)
    U, s, V, sweeps = oracle.jacobi_svd(A)
    assert sweeps > 0
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, ref, rtol=1e-13, atol=0)
    assert np.abs(U.T @ U - np.eye(shape[1])).max() < 1e-13
    assert np.abs(V.T @ V - np.eye(shape[1])).max() < 1e-13
    assert np.abs(U * s @ V.T - A).max() < 1e-13 * np.abs(A).max() * shape[1]


def test_jacobi_closed_forms():
    # 2x2 upper triangular [[a, b], [0, c]]: sigma1*sigma2 = |ac|, s1^2 + s2^2 = a^2 + b^2 + c^2
    a, b, c = 3.0, 4.0, 0.5
    _, s, _, _ = oracle.jacobi_svd(np.array([[a, b], [0.0, c]]))
    assert np.isclose(s[0] * s[1], abs(a * c), rtol=1e-15)
    assert np.isclose((s ** 2).sum(), a * a + b * b + c * c, rtol=1e-15)
    # diagonal input: singular values are the sorted |entries|
    _, s, _, _ = oracle.jacobi_svd(np.diag([1.0, -5.0, 2.0]))
    assert np.array_equal(s, [5.0, 2.0, 1.0])
    # duplicated column: rank deficiency shows as an exact-ish zero
    rng = np.random.default_rng(2)
    X = rng.standard_normal((20, 4))
    X[:, 3] = X[:, 1]
    U, s, V, _ = oracle.jacobi_svd(X)
    assert s[3] < 1e-14 * s[0]
    assert np.all(U[:, 3] == 0) or np.linalg.norm(U[:, 3]) < 1.5


def test_sign_rule():
    U = np.array([[1.0, 2.0], [3.0, -4.0]])
    V = np.array([[-0.6, 0.5], [0.8, -0.5], [0.0, 0.1]])
    U2, V2 = oracle.sign_fix(U, V)
    # column 0: largest |v| is 0.8 (positive) -> unchanged
    assert np.array_equal(V2[:, 0], V[:, 0]) and np.array_equal(U2[:, 0], U[:, 0])
    # column 1: tie |0.5| = |-0.5| -> first wins, positive -> unchanged
    assert np.array_equal(V2[:, 1], V[:, 1])
    U3, V3 = oracle.sign_fix(U, -V)
    assert np.array_equal(V3[:, 0], V[:, 0]) and np.array_equal(U3[:, 0], -U[:, 0])
