"""tcgen05 A^T u (FP32 path) against the FP64 oracle, elementwise.

Two kernels: the default one with N = 16 (k_rmv_tc) and the one with 256
SNPs on the MMA's N side (k_rmv_n256, GKL_RMV_KERNEL=n256).  Both compute
sum_i g_ij u~'_i exactly, where u~' is u~ = s o u truncated
to 28 fractional bits of S = 2^e >= max|u~| (max|u~| = f 2^e, f in [1/2, 1)) (|u~ - u~'| <= 2^-29 S), and
rounds once to FP32 at the end.  Bound per entry:
    |x_j - xo_j| <= 2^-23 |xo_j| + 2^-28 n S d_j w_j
(the second term covers the truncation: |g - mu| <= 2 per entry).
"""
import os

import numpy as np
import pytest

import synth
from tests.helpers import oracle_matrix, small_geno, to_dev

pytestmark = pytest.mark.gpu

# ragged tails in both directions; n = 70,000 spans two K-ranges of the N = 16
# kernel, n = 600,000 two of the N = 256 kernel (1023 stages of 512 samples each)
SHAPES = [(1, 1), (5, 3), (255, 129), (256, 128), (257, 300), (1000, 2000), (4099, 777), (70_000, 300),
          (600_000, 130)]


@pytest.fixture(scope="module")
def gk():
    import torch  # noqa: F401
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl


def handle(gk, g, kernel="tc"):
    old = os.environ.get("GKL_RMV_KERNEL")
    if kernel:
        os.environ["GKL_RMV_KERNEL"] = kernel
    try:
        return gk.GKL(to_dev(g.packed), g.n)
    finally:
        if kernel:
            if old is None:
                del os.environ["GKL_RMV_KERNEL"]
            else:
                os.environ["GKL_RMV_KERNEL"] = old


def bound(M, ut, xo):
    S = np.ldexp(1.0, int(np.frexp(np.max(np.abs(ut)))[1])) if np.any(ut) else 1.0  # 2^e >= max|u~|
    dw = M.d * (M.w if M.w is not None else 1.0)
    return 2.0 ** -23 * np.abs(xo) + 2.0 ** -28 * M.n * S * dw + 1e-300


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("weights", [False, True])
@pytest.mark.parametrize("kernel", ["tc", "n256"])
def test_tc_rmatvec_elementwise(gk, n, m, weights, kernel):
    import torch
    if n == 600_000 and (weights or kernel == "tc"):
        pytest.skip("one large case: the N = 256 kernel's second K-range")
    g = small_geno(n, m, miss=0.03, seed=5 * n + m)
    s = synth.uniform_vec(13, 0, n, 0.5, 1.5).astype(np.float32).astype(np.float64) if weights else None
    w = synth.uniform_vec(13, 1, m, 0.5, 1.5).astype(np.float32).astype(np.float64) if weights else None
    M = oracle_matrix(g, s, w)
    h = handle(gk, g, kernel)
    if weights:
        h.set_weights(torch.tensor(s, dtype=torch.float32), torch.tensor(w, dtype=torch.float32))
    u = synth.normal_vec(17, n, n).astype(np.float32)
    x = h.rmatvec(torch.tensor(u, device="cuda")).double().cpu().numpy()
    u64 = u.astype(np.float64)
    xo = M.rmatvec(u64)
    ut = u64 * (s if weights else 1.0)
    assert np.all(np.abs(x - xo) <= bound(M, ut, xo))


def test_tc_agrees_with_mma_kernel(gk):
    import torch
    n, m = 3001, 2049
    g = small_geno(n, m, miss=0.02, seed=77)
    M = oracle_matrix(g)
    u = torch.tensor(synth.normal_vec(19, 0, n).astype(np.float32), device="cuda")
    x_tc = handle(gk, g).rmatvec(u).double().cpu().numpy()
    x_256 = handle(gk, g, "n256").rmatvec(u).double().cpu().numpy()
    x_mma = handle(gk, g, "mma").rmatvec(u).double().cpu().numpy()
    xo = M.rmatvec(u.double().cpu().numpy())
    b = bound(M, u.double().cpu().numpy(), xo)
    assert np.all(np.abs(x_tc - xo) <= b)
    assert np.all(np.abs(x_256 - xo) <= b)
    assert np.all(np.abs(x_mma - xo) <= 2 * b)


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
