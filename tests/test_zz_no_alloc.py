"""gkl_matvec_noalloc: y = A v for callers that may not allocate device memory.

Such callers (code living inside another application's device-memory pool, or
loops where an allocation's device-wide synchronisation is not allowed) get a
product whose scratch is a fixed array inside the library.  This file is
collected last so that a run stopping at its first failure has already run
every other test.  It checks, through the C ABI, that two calls in a row agree
with gkl_matvec and with the oracle's product on the same inputs, and that
oversized problems are refused.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_1808_03374_gb300 import build, gkl
    build()
    g = synth.genotypes(synth.GenoSpec(n=3001, m=20_011, n_pops=3, admixture=True, miss_rate=0.02, seed=123))
    packed = torch.from_numpy(g.packed).cuda()
    mu, scale, _ = gkl.colstats(packed, g.n)
    h = gkl.GKL(packed, g.n, mu, scale)
    return gkl, g, packed, mu, scale, h


@pytest.fixture(scope="module")
def oracle_mat(setup):
    g = setup[1]
    return oracle.Matrix.from_packed(g.packed, g.n)


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-5)])
def test_noalloc_matches_matvec_and_oracle_twice(setup, oracle_mat, prec, tol):
    import torch
    gkl, g, packed, mu, scale, h = setup
    dt = torch.float64 if prec == 0 else torch.float32
    lib = gkl.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        v = torch.tensor(synth.normal_vec(31 + call, 0, g.m), dtype=dt, device="cuda")
        ref = h.matvec(v)
        y = torch.full((g.n,), float("nan"), dtype=dt, device="cuda")
        st = lib.gkl_matvec_noalloc(ctypes.c_void_p(packed.data_ptr()), g.n, g.m, g.stride,
                                    ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(scale.data_ptr()), prec,
                                    ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)
        assert st == 0, lib.gkl_last_error(None)
        torch.cuda.synchronize()
        a, b = y.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)
        yo = oracle_mat.matvec(v.double().cpu().numpy())
        assert np.linalg.norm(a - yo) <= tol * np.linalg.norm(yo)


def test_noalloc_rejects_sizes_beyond_static_scratch(setup):
    import torch
    gkl, g, packed, mu, scale, h = setup
    lib = gkl.lib()
    y = torch.empty(g.n, dtype=torch.float64, device="cuda")
    # claim 100x more SNPs than the buffer holds: rejected on size before any work
    st = lib.gkl_matvec_noalloc(ctypes.c_void_p(packed.data_ptr()), g.n, 100 * g.m, g.stride,
                                ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(scale.data_ptr()), 0,
                                ctypes.c_void_p(y.data_ptr() + 8), ctypes.c_void_p(y.data_ptr()), None)
    assert st == gkl.ERR_ARG
    assert b"static maximum" in lib.gkl_last_error(None)
