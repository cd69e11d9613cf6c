"""Input generator: Philox known answers, layout, determinism and model moments."""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def unpack_codes(packed, n):
    """Pure-numpy decode of the 2-bit SNP-major layout -> int8 [m, n]."""
    b = np.asarray(packed, dtype=np.uint8)
    c = np.stack([(b >> (2 * t)) & 3 for t in range(4)], axis=-1).reshape(b.shape[0], -1)
    return c[:, :n].astype(np.int8), c[:, n:]


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert synth.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_padded_stride():
    assert synth.padded_stride(1) == 16
    assert synth.padded_stride(64) == 16
    assert synth.padded_stride(65) == 32
    assert synth.padded_stride(10_000) == 2512
    assert synth.padded_stride(200_000) == 50_000


def test_generator_deterministic_and_padded():
    spec = synth.GenoSpec(n=333, m=257, n_pops=3, admixture=True, miss_rate=0.05, seed=42)
    a = synth.genotypes(spec)
    b = synth.genotypes(spec)
    assert np.array_equal(a.packed, b.packed)
    c = synth.genotypes(synth.GenoSpec(n=333, m=257, n_pops=3, admixture=True, miss_rate=0.05, seed=43))
    assert not np.array_equal(a.packed, c.packed)
    codes, pad = unpack_codes(a.packed, spec.n)
    assert (pad == 3).all()
    assert a.packed.shape == (257, spec.stride)


def test_generator_moments():
    spec = synth.GenoSpec(n=4000, m=800, n_pops=4, admixture=True, miss_rate=0.02, seed=7)
    g = synth.genotypes(spec)
    codes, _ = unpack_codes(g.packed, spec.n)
    miss = codes == 3
    # MCAR missingness at the stated rate (binomial 6-sigma band)
    N = codes.size
    assert abs(miss.mean() - 0.02) < 6 * np.sqrt(0.02 * 0.98 / N)
    # E[g_ij] = 2 p_ij with p_ij = sum_k q_ik f_kj
    p = g.q @ g.f  # n x m
    obs = ~miss
    gsum = np.where(obs, codes, 0).astype(np.float64)
    expected = (2 * p.T * obs).sum()
    var = (2 * p.T * (1 - p.T) * obs).sum()
    assert abs(gsum.sum() - expected) < 6 * np.sqrt(var)
    # ancestry rows are probability vectors
    assert np.allclose(g.q.sum(1), 1.0) and (g.q >= 0).all()
    assert (g.f >= 0.01).all() and (g.f <= 0.99).all()


def test_discrete_pm_delta_populations():
    w = synth.CONFIGS["fp64_full_1k_x_10k"]
    spec = w.geno
    g = synth.genotypes(synth.GenoSpec(**{**spec.__dict__, "m": 500}))
    # first half of the samples in population 0, second half in population 1
    assert (g.q[:500, 0] == 1).all() and (g.q[500:, 1] == 1).all()
    # f_0j and f_1j straddle a common p_j symmetrically unless clipped
    mid = 0.5 * (g.f[0] + g.f[1])
    unclipped = (g.f > 0.01).all(0) & (g.f < 0.99).all(0)
    assert ((mid >= 0.05 - 1e-12) & (mid <= 0.5 + 1e-12))[unclipped].all()


def test_beta_base_frequencies():
    spec = synth.GenoSpec(n=16, m=20000, base=("beta", 0.5, 2.0, 0.01, 0.5), delta_sd=0.0, seed=3)
    g = synth.genotypes(spec)
    p = g.f[0]
    assert (p >= 0.01).all() and (p <= 0.5).all()
    # Beta(0.5, 2) has mean 0.2; clipping to [0.01, 0.5] moves it only slightly
    assert 0.17 < p.mean() < 0.23


def test_vectors():
    a = synth.normal_vec(1, 0, 100_000)
    assert abs(a.mean()) < 0.02 and abs(a.std() - 1) < 0.02
    b = synth.normal_vec(1, 1, 100_000)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.02
    u = synth.uniform_vec(1, 2, 100_000, 0.5, 1.5)
    assert u.min() >= 0.5 and u.max() < 1.5 and abs(u.mean() - 1.0) < 0.01


# ---- the paper's synthetic model (section 2, Algorithm 1) --------------------

def _model_draw(seed, a, b, st, d):
    return synth.philox4x32_10((a, b, st, d), (seed & 0xFFFFFFFF, seed >> 32))


def _below(x, bound):
    return (x * bound) >> 32


def _codes(g):
    return np.stack([(g.packed >> (2 * t)) & 3 for t in range(4)], -1).reshape(g.m, -1)


def test_paper_model_blocks_and_kinship_exact():
    """With no signal draws the matrix is the admixture sub-blocks (later ones on
    top) followed by the ordered row copies: rebuilt here from the same
    counter-based draws, entry for entry."""
    spec = synth.ModelSpec(n=203, m=97, r=6, nsignal_frac=0.0, rkins=0.08, seed=0x1234_5678_9ABC)
    g = synth.paper_model(spec)
    n, m = spec.n, spec.m
    A = np.zeros((m, n), dtype=np.int64)
    for b in range(spec.r):
        x = _model_draw(spec.seed, b, 0, 6, 0)
        y = _model_draw(spec.seed, b, 0, 6, 1)
        k = _below(x[0], 3)
        j1, j2 = sorted((_below(x[1], m), _below(x[2], m)))
        i1, i2 = sorted((_below(x[3], n), _below(y[0], n)))
        A[j1:j2 + 1, i1:i2 + 1] = k
    for c in range(round(spec.rkins * m)):
        x = _model_draw(spec.seed, c, 0, 8, 0)
        A[_below(x[0], m)] = A[_below(x[1], m)].copy()
    codes = _codes(g)
    assert np.array_equal(codes[:, :n], A)
    assert np.all(codes[:, n:] == 3)


def test_paper_model_signal_distribution():
    """Each entry is hit by the signal draws with probability 1 - (1 - 1/mn)^nsignal
    and then holds a uniform value in {0, 1, 2}: with no sub-blocks the share of
    zeros is (1 - p) + p/3 and of ones and twos p/3 each."""
    spec = synth.ModelSpec(n=400, m=300, r=0, nsignal_frac=1.0, rkins=0.0, seed=77)
    codes = _codes(synth.paper_model(spec))[:, :spec.n]
    mn = spec.n * spec.m
    p = 1.0 - (1.0 - 1.0 / mn) ** mn
    share = np.bincount(codes.ravel(), minlength=3) / mn
    sd = np.sqrt(p / 3 * (1 - p / 3) / mn)
    assert abs(share[1] - p / 3) < 6 * sd and abs(share[2] - p / 3) < 6 * sd
    assert abs(share[0] - (1 - p + p / 3)) < 12 * sd
