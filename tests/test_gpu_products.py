"""GPU parity of the packed products and per-SNP statistics against the CPU oracle.

Bar: integer counts and FP64 unit-vector products bit-exact; FP64 products to
1e-13 relative (norm-wise); FP32 products to 2e-5 relative (FP32 rounding of
sums over up to 10^5 terms).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import oracle_matrix, rel_err, small_geno, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (3, 5), (17, 33), (64, 100), (257, 1031), (1000, 2000), (4099, 777)]


@pytest.fixture(scope="module")
def gk():
    import torch  # noqa: F401
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl


@pytest.mark.parametrize("n,m", SHAPES)
def test_colstats_bit_exact(gk, n, m):
    g = small_geno(n, m, miss=0.05, seed=n + m)
    mu, sc, nobs = gk.colstats(to_dev(g.packed), n)
    omu, od, onobs = oracle.colstats(g.packed, n)
    assert np.array_equal(nobs.cpu().numpy(), onobs)
    assert np.array_equal(mu.cpu().numpy(), omu)
    assert np.array_equal(sc.cpu().numpy(), od)


def test_colstats_degenerate_rows(gk):
    from tests.test_oracle_core import pack_codes
    codes = np.array([[0, 1, 2, 3, 1], [2, 2, 2, 2, 2], [3, 3, 3, 3, 3], [0, 0, 0, 0, 2]])
    packed = pack_codes(codes)
    mu, sc, nobs = gk.colstats(to_dev(packed), 5)
    assert nobs.tolist() == [4, 5, 0, 5]
    assert mu.tolist() == [1.0, 2.0, 0.0, 0.4]
    assert sc.cpu().numpy()[1:3].tolist() == [0.0, 0.0]


@pytest.mark.parametrize("n,m", [(17, 33), (257, 1031), (1000, 2000)])
def test_fp64_unit_vector_products_bit_exact(gk, n, m):
    import torch
    g = small_geno(n, m, seed=7 * n + m)
    M = oracle_matrix(g)
    A = M.dense()
    h = gk.GKL(to_dev(g.packed), n)
    for j in sorted({0, m // 2, m - 1}):
        e = torch.zeros(m, dtype=torch.float64, device="cuda")
        e[j] = 1.0
        assert np.array_equal(h.matvec(e).cpu().numpy(), A[:, j])
    for i in sorted({0, n // 2, n - 1}):
        e = torch.zeros(n, dtype=torch.float64, device="cuda")
        e[i] = 1.0
        assert np.array_equal(h.rmatvec(e).cpu().numpy(), A[i, :])


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("weights", [False, True])
def test_products_match_oracle(gk, n, m, weights):
    import torch
    g = small_geno(n, m, seed=3 * n + m)
    s = synth.uniform_vec(11, 0, n, 0.5, 1.5).astype(np.float32).astype(np.float64) if weights else None
    w = synth.uniform_vec(11, 1, m, 0.5, 1.5).astype(np.float32).astype(np.float64) if weights else None
    M = oracle_matrix(g, s, w)
    h = gk.GKL(to_dev(g.packed), n)
    if weights:
        h.set_weights(torch.tensor(s, dtype=torch.float32), torch.tensor(w, dtype=torch.float32))
    v = synth.normal_vec(5, 0, m)
    u = synth.normal_vec(5, 1, n)
    yo, xo = M.matvec(v), M.rmatvec(u)
    y64 = h.matvec(torch.tensor(v, device="cuda")).cpu().numpy()
    x64 = h.rmatvec(torch.tensor(u, device="cuda")).cpu().numpy()
    assert rel_err(y64, yo) < 1e-13
    assert rel_err(x64, xo) < 1e-13
    v32, u32 = v.astype(np.float32), u.astype(np.float32)
    y32 = h.matvec(torch.tensor(v32, device="cuda")).cpu().numpy()
    x32 = h.rmatvec(torch.tensor(u32, device="cuda")).cpu().numpy()
    assert rel_err(y32, M.matvec(v32.astype(np.float64))) < 2e-5
    assert rel_err(x32, M.rmatvec(u32.astype(np.float64))) < 2e-5


def test_products_deterministic(gk):
    import torch
    g = small_geno(3000, 5000, seed=99)
    h = gk.GKL(to_dev(g.packed), 3000)
    v = torch.randn(5000, device="cuda", dtype=torch.float32)
    a, b = h.matvec(v), h.matvec(v)
    assert torch.equal(a, b)
    u = torch.randn(3000, device="cuda", dtype=torch.float32)
    assert torch.equal(h.rmatvec(u), h.rmatvec(u))


def test_full_size_products_sampled(gk):
    """10,000 x 100,000 workload (2% missing, 5-population admixture): sampled
    outputs of both products against the oracle's one-by-one rows/columns."""
    import torch
    w = synth.CONFIGS["fp32_pro_10k_x_100k"]
    g = synth.genotypes(w.geno)
    M = oracle_matrix(g)
    h = gk.GKL(to_dev(g.packed), g.n)
    rng = np.random.default_rng(0)
    v = synth.normal_vec(21, 0, g.m)
    u = synth.normal_vec(21, 1, g.n)
    rows = np.unique(np.r_[0, g.n - 1, rng.integers(0, g.n, 48)])
    cols = np.unique(np.r_[0, g.m - 1, rng.integers(0, g.m, 48)])
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
        y = h.matvec(torch.tensor(v, dtype=dt, device="cuda")).double().cpu().numpy()
        x = h.rmatvec(torch.tensor(u, dtype=dt, device="cuda")).double().cpu().numpy()
        vv = v.astype(np.float32).astype(np.float64) if dt == torch.float32 else v
        uu = u.astype(np.float32).astype(np.float64) if dt == torch.float32 else u
        yo = M.matvec_rows(vv, rows)
        xo = M.rmatvec_cols(uu, cols)
        scale_y = np.linalg.norm(y) / np.sqrt(g.n)
        scale_x = np.linalg.norm(x) / np.sqrt(g.m)
        assert np.max(np.abs(y[rows] - yo)) < tol * 10 * scale_y
        assert np.max(np.abs(x[cols] - xo)) < tol * 10 * scale_x
