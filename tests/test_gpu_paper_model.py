"""The paper's own synthetic workload (section 2, Algorithm 1: r admixture
sub-blocks, signal entries drawn nsignal = m n times, duplicated marker rows
at rate rkins), scaled down to a size the oracle solves in seconds, through
every solver form against the FP64 oracle.

Bars as for the other workloads: FP64 singular values to 1e-10 of
themselves, FP32 to 1e-5, the block forms to 1e-6 (Rayleigh-Ritz values);
vectors through their angles, bounded by (residual + rounding) / gap; and
||Delta theta||_1 (Table 3's error measure, the sum of the reported
residuals) within the solve's tolerance."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import to_dev
from tests.test_gpu_svd import angles, gaps

pytestmark = pytest.mark.gpu

SPEC = synth.ModelSpec(n=4_000, m=2_500, r=10, nsignal_frac=1.0, rkins=0.017, seed=0x5EED0106)
K = 10


@pytest.fixture(scope="module")
def gk():
    import torch  # noqa: F401
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl


@pytest.fixture(scope="module")
def model():
    g = synth.paper_model(SPEC)
    M = oracle.Matrix.from_packed(g.packed, SPEC.n)
    ref = oracle.gkl(M, k=K + 4, ell=40, tol=1e-13, v0=synth.normal_vec(8, 0, SPEC.m), maxit=2000)
    assert ref.converged
    return g, M, ref


@pytest.mark.parametrize("kw,sig_rel,vec_eps", [
    (dict(precision="fp64", reorth="full", ell=30, tol=1e-10), 1e-10, 1e-13),
    (dict(precision="fp64", reorth="partial", ell=40, tol=1e-10), 1e-10, 1e-8),
    (dict(precision="fp32", reorth="dgks", ell=30, tol=1e-6), 1e-5, 3e-6),
    (dict(precision="block", block=8, ell=48, tol=1e-6), 1e-6, 3e-6),
    (dict(precision="block16", block=16, ell=64, k_keep=32, tol=1e-6), 1e-6, 3e-6),
])
def test_paper_model_against_oracle(gk, model, kw, sig_rel, vec_eps):
    g, M, ref = model
    h = gk.GKL(to_dev(g.packed), SPEC.n)
    r = h.svd(k=K, maxit=500, seed=4, **kw)
    assert r.converged, r.info
    rel = np.abs(r.sigma - ref.sigma[:K]) / ref.sigma[:K]
    assert rel.max() < sig_rel, (rel.max(), r.sigma[:3], ref.sigma[:3])
    U = r.U.double().cpu().numpy()
    V = r.V.double().cpu().numpy()
    bound = 10 * (np.maximum(r.resid, 0) + vec_eps * ref.sigma[0]) / gaps(ref.sigma)[:K] + 1e-12
    assert np.all(angles(V, ref.V[:, :K]) <= bound)
    assert np.all(angles(U, ref.U[:, :K]) <= bound)
    # Table 3's error measure: ||Delta theta||_1 = sum of the residuals, each within tol sigma_1
    assert r.info["dtheta1"] <= K * kw["tol"] * r.sigma[0] * (1 + 1e-9)
