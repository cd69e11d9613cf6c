"""Shared helpers of the GPU parity tests."""
import numpy as np

import oracle
import synth


def small_geno(n, m, pops=3, miss=0.02, seed=1, admixture=True, **kw):
    return synth.genotypes(synth.GenoSpec(n=n, m=m, n_pops=pops, admixture=admixture, miss_rate=miss, seed=seed,
                                          **kw))


def to_dev(packed):
    import torch
    return torch.from_numpy(np.ascontiguousarray(packed)).cuda()


def rel_err(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def align_signs(X, Y):
    """Flip columns of X to best match Y (singular vectors are defined up to sign)."""
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1
    return X * s


def oracle_matrix(g, s=None, w=None):
    M = oracle.Matrix.from_packed(g.packed, g.n)
    if s is not None or w is not None:
        M = oracle.Matrix(g.packed, g.n, M.mu, M.d, s=s, w=w)
    return M
