"""tcgen05 A^T u (FP32 path) against the FP64 oracle, elementwise.

The kernel computes sum_i g_ij u~'_i exactly, where u~' is u~ = s o u
written in fixed point relative to S = 2^e >= max|u~| (max|u~| = f 2^e, f in
[1/2, 1)) with |u~ - u~'| <= 2^-29 S, and rounds once to FP32 at the end.
Bound per entry:
    |x_j - xo_j| <= 2^-23 |xo_j| + 2^-28 n S d_j w_j
(the second term covers the truncation: |g - mu| <= 2 per entry).
"""
import numpy as np
import pytest

import synth
from tests.helpers import oracle_matrix, small_geno, to_dev

pytestmark = pytest.mark.gpu

# ragged tails in both directions; n = 70,000 spans several K-ranges of the kernel (the plan splits rows
# of few SNP tiles into ranges to fill the SMs)
SHAPES = [(1, 1), (5, 3), (255, 129), (256, 128), (257, 300), (1000, 2000), (4099, 777), (70_000, 300)]


@pytest.fixture(scope="module")
def gk():
    import torch  # noqa: F401
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl


def handle(gk, g):
    return gk.GKL(to_dev(g.packed), g.n)


def bound(M, ut, xo):
    S = np.ldexp(1.0, int(np.frexp(np.max(np.abs(ut)))[1])) if np.any(ut) else 1.0  # 2^e >= max|u~|
    dw = M.d * (M.w if M.w is not None else 1.0)
    return 2.0 ** -23 * np.abs(xo) + 2.0 ** -28 * M.n * S * dw + 1e-300


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("weights", [False, True])
def test_tc_rmatvec_elementwise(gk, n, m, weights):
    import torch
    g = small_geno(n, m, miss=0.03, seed=5 * n + m)
    s = synth.uniform_vec(13, 0, n, 0.5, 1.5).astype(np.float32).astype(np.float64) if weights else None
    w = synth.uniform_vec(13, 1, m, 0.5, 1.5).astype(np.float32).astype(np.float64) if weights else None
    M = oracle_matrix(g, s, w)
    h = handle(gk, g)
    if weights:
        h.set_weights(torch.tensor(s, dtype=torch.float32), torch.tensor(w, dtype=torch.float32))
    u = synth.normal_vec(17, n, n).astype(np.float32)
    x = h.rmatvec(torch.tensor(u, device="cuda")).double().cpu().numpy()
    u64 = u.astype(np.float64)
    xo = M.rmatvec(u64)
    ut = u64 * (s if weights else 1.0)
    assert np.all(np.abs(x - xo) <= bound(M, ut, xo))


def test_tc_all_missing_and_monomorphic_rows(gk):
    """Rows that are entirely missing, entirely one code, or one observed entry:
    the centring and the missing-code terms must cancel exactly to 0 where the
    oracle gives 0."""
    import torch
    n, m = 2051, 260
    g = small_geno(n, m, miss=0.02, seed=41)
    packed = g.packed.copy()
    packed[0, :] = 0xFF                       # all missing (and padding)
    packed[1, : (n + 3) // 4] = 0x55          # all code 1: monomorphic, d = 0
    packed[2, :] = 0xFF
    packed[2, 0] = 0xFC                       # one observed entry (sample 0, code 0)
    packed[3, : (n + 3) // 4] = 0xAA          # all code 2
    for r in (1, 3):                          # padding entries of the last byte hold code 3
        tail = n % 4
        if tail:
            packed[r, n // 4] = (packed[r, n // 4] & ((1 << (2 * tail)) - 1)) | (0xFF << (2 * tail) & 0xFF)
    h = gk.GKL(to_dev(packed), n)
    from oracle import Matrix
    M = Matrix.from_packed(packed, n)
    u = synth.normal_vec(29, 0, n).astype(np.float32)
    x = h.rmatvec(torch.tensor(u, device="cuda")).double().cpu().numpy()
    xo = M.rmatvec(u.astype(np.float64))
    assert np.all(x[:4] == 0.0) and np.all(xo[:4] == 0.0)
    assert np.all(np.abs(x - xo) <= bound(M, u.astype(np.float64), xo))


def test_tc_special_vectors(gk):
    """Zero vector, a single nonzero sample, all-equal entries (centring makes
    A^T 1 = 0 up to the truncation), and a vector spanning 2^40 in magnitude."""
    import torch
    n, m = 1500, 700
    g = small_geno(n, m, miss=0.02, seed=3)
    M = oracle_matrix(g)
    h = handle(gk, g)
    zero = torch.zeros(n, device="cuda")
    assert torch.count_nonzero(h.rmatvec(zero)).item() == 0
    e = np.zeros(n, dtype=np.float32)
    e[777] = 3.0
    x = h.rmatvec(torch.tensor(e, device="cuda")).double().cpu().numpy()
    xo = M.rmatvec(e.astype(np.float64))
    assert np.all(np.abs(x - xo) <= bound(M, e.astype(np.float64), xo))
    wide = (synth.normal_vec(23, 0, n) * 2.0 ** np.linspace(-20, 20, n)).astype(np.float32)
    x = h.rmatvec(torch.tensor(wide, device="cuda")).double().cpu().numpy()
    xo = M.rmatvec(wide.astype(np.float64))
    assert np.all(np.abs(x - xo) <= bound(M, wide.astype(np.float64), xo))


def test_products_after_solves_that_grow_the_outputs(gk):
    """Solves with growing k reallocate the handle's output buffers; the FP32
    A^T u afterwards (which reads the handle's list of missing codes) still
    matches the oracle."""
    import torch
    n, m = 2003, 3001
    g = small_geno(n, m, miss=0.02, seed=83)
    M = oracle_matrix(g)
    h = handle(gk, g)
    for k in (3, 6, 9):
        assert h.svd(k=k, ell=24, precision="fp32", tol=1e-5, seed=1).converged
    u = synth.normal_vec(31, 0, n).astype(np.float32)
    for _ in range(2):
        x = h.rmatvec(torch.tensor(u, device="cuda")).double().cpu().numpy()
        xo = M.rmatvec(u.astype(np.float64))
        assert np.all(np.abs(x - xo) <= bound(M, u.astype(np.float64), xo))
    h.sync()


# The missing-code list is cut into sample blocks of 24,576 with 16-bit offsets;
# its gather takes the first 256 entries of a segment in one batch and walks the
# rest.  Sizes at and around the block edges (a last block of one sample), and
# missing rates whose segments run past the batch (30%: about 7,400 entries a
# segment), in both precisions.
@pytest.mark.parametrize("n,m,miss", [(24_576, 97, 0.05), (24_577, 96, 0.3), (49_153, 40, 0.01),
                                      (73_729, 33, 0.3), (300, 1_001, 0.9)])
def test_missing_list_block_edges(gk, n, m, miss):
    import torch
    g = small_geno(n, m, miss=miss, seed=n + m)
    M = oracle_matrix(g)
    h = handle(gk, g)
    u64 = synth.normal_vec(19, 2, n)
    xo = M.rmatvec(u64)
    x64 = h.rmatvec(torch.tensor(u64, device="cuda")).cpu().numpy()
    assert np.abs(x64 - xo).max() <= 1e-12 * np.abs(xo).max()
    u = u64.astype(np.float32)
    x = h.rmatvec(torch.tensor(u, device="cuda")).double().cpu().numpy()
    xo32 = M.rmatvec(u.astype(np.float64))
    assert np.all(np.abs(x - xo32) <= bound(M, u.astype(np.float64), xo32))
