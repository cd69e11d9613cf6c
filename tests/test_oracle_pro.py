"""Pins of the partial-reorthogonalisation estimates (the omega recurrence)
after a thick restart, oracle/pro.py, against the computed inner products
themselves (section 3: reorthogonalise only when the estimated loss of
orthogonality exceeds a threshold).

One cycle after a restart runs with no reorthogonalisation, so that U^T U and
V^T V lose orthogonality step by step.  Two properties are checked:

- the recurrence is an identity: evaluated on the true inner products and the
  cycle's B (kept values, spike column, new bidiagonal part) it reproduces
  the next step's true inner products to within rounding (measured at most
  33 eps sigma_1; a dropped, sign-flipped, mis-indexed or transposed term,
  the spike's included, leaves 700 to 10^16 eps sigma_1 in at least one of the
  cases below);
- the estimates with their rounding term bound the true loss while it grows
  (never below half of it, never more than 10^3 above it), and cross a
  threshold omega = 1e-8 no later than the true loss does, and at most 8
  steps earlier.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.pro import cycle_after_restart, mu_row, nu_row

EPS = 2.0 ** -53
CASES = [  # n, m, populations, kept vectors, l, seed
    (600, 3000, 5, 15, 60, 3),
    (1000, 4000, 3, 10, 80, 5),
    (800, 2000, 8, 20, 70, 7),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"{c[0]}x{c[1]}_k{c[3]}_l{c[4]}")
def trace(request):
    n, m, pops, kk, ell, seed = request.param
    g = synth.genotypes(synth.GenoSpec(n=n, m=m, n_pops=pops, admixture=True, miss_rate=0.02, seed=seed))
    A = oracle.Matrix.from_packed(g.packed, n).dense()
    return cycle_after_restart(A, kk, ell, synth.normal_vec(4, 0, m))


def test_orthogonality_is_lost_without_reorthogonalisation(trace):
    """The setting the estimates are for: without reorthogonalisation the new
    vectors lose orthogonality to the kept ones far beyond rounding."""
    kk, ell = trace.kk, trace.ell
    off = np.abs(trace.mu_true - np.eye(ell))[kk:, :]  # the new u's against every earlier one
    assert off.max() > 1e-5  # about 1e11 unit roundoffs
    assert np.abs(trace.mu_true[:kk, :kk] - np.eye(kk)).max() < 1e-13  # the kept vectors start orthonormal


def test_recurrence_is_an_identity_on_true_inner_products(trace):
    sigma1 = trace.B[0, 0]
    for j in range(trace.kk, trace.ell):
        alpha, beta = trace.B[j, j], trace.B[j, j + 1]
        du = mu_row(trace.B, trace.mu_true, trace.nu_true, j, alpha) - trace.mu_true[j, :j]
        dv = nu_row(trace.B, trace.mu_true, trace.nu_true, j, beta) - trace.nu_true[j + 1, :j + 1]
        assert np.abs(du).max() * alpha <= 150 * EPS * sigma1, (j, np.abs(du).max())
        assert np.abs(dv).max() * beta <= 150 * EPS * sigma1, (j, np.abs(dv).max())


def test_estimates_bound_and_track_the_loss(trace, omega=1e-8):
    cross_est = cross_true = None
    for j in range(trace.kk, trace.ell):
        est_u, true_u = np.abs(trace.mu_est[j, :j]).max(), np.abs(trace.mu_true[j, :j]).max()
        est_v, true_v = np.abs(trace.nu_est[j + 1, :j + 1]).max(), np.abs(trace.nu_true[j + 1, :j + 1]).max()
        if max(true_u, true_v) > 1e-4:  # growth phase over: orthogonality is gone
            break
        for est, true in ((est_u, true_u), (est_v, true_v)):
            assert 0.5 * true <= est <= 1e3 * max(true, 1e-15), (j, est, true)
        if cross_est is None and max(est_u, est_v) > omega:
            cross_est = j
        if cross_true is None and max(true_u, true_v) > omega:
            cross_true = j
    assert cross_true is not None and cross_est is not None
    assert cross_true - 8 <= cross_est <= cross_true, (cross_est, cross_true)
