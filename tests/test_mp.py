"""Marchenko-Pastur law (section 2, Eqs. 4-5): normalisation, edges and the
paper's Fig. mplaw setting (1000 x 667 iid Gaussian, rho = 1.5)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import mp


@pytest.mark.parametrize("y", [0.1, 0.5, 1.5, 3.0])
def test_densities_integrate_to_one(y):
    lo, hi = mp.edges(y)
    tot_s = integrate.quad(lambda x: mp.sv_density(np.array([x]), y)[0], lo, hi, limit=200)[0]
    tot_e = integrate.quad(lambda x: mp.ev_density(np.array([x]), y)[0], lo ** 2, hi ** 2, limit=200)[0]
    assert abs(tot_s - 1) < 1e-6 and abs(tot_e - 1) < 1e-6


def test_edges_and_first_moment():
    # sigma_+- = sigma |1 +- sqrt(rho)|; the eigenvalue mean of (1/N) X X^T over
    # nonzero eigenvalues is sigma^2 max(1, y)
    lo, hi = mp.edges(0.25, sigma=2.0)
    assert np.isclose(lo, 1.0) and np.isclose(hi, 3.0)
    for y in (0.3, 2.0):
        l2, h2 = (e ** 2 for e in mp.edges(y))
        mean = integrate.quad(lambda x: x * mp.ev_density(np.array([x]), y)[0], l2, h2, limit=200)[0]
        assert np.isclose(mean, max(1.0, y), rtol=1e-6)


def test_gaussian_1000_x_667_matches_law():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((1000, 667))
    s = np.linalg.svd(X, compute_uv=False) / np.sqrt(667)
    assert mp.ks_distance(s, y=1000 / 667) <= 0.03
    lo, hi = mp.edges(1000 / 667)
    assert abs(s.max() / hi - 1) < 0.02 and abs(s.min() / lo - 1) < 0.1


def test_wrong_reading_is_rejected():
    # the law with rho taken as columns/rows (the other reading of section 2) must not fit
    rng = np.random.default_rng(1)
    X = rng.standard_normal((1000, 667))
    s = np.linalg.svd(X, compute_uv=False) / np.sqrt(667)
    assert mp.ks_distance(s, y=667 / 1000) > 0.1
