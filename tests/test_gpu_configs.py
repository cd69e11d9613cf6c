"""Parity at the full-size workloads that fit a test run: the 10,000 x
100,000 null model against the Marchenko-Pastur edge (section 2, Eqs. 4-5)
and the 20,000 x 200,000 gradient against central differences of FP64
solves.  The
50,000 x 500,000 and 200,000 x 1,000,000 checks against the oracle's own
products take minutes of CPU time and run as ``tests/check_large_parity.py``
(its summary is committed beside it)."""
import pytest

from tests import check_large_parity as clp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gk():
    return clp._lib()


def test_null_model_sigma1_at_marchenko_pastur_edge(gk):
    r = clp.check_null_10k_x_100k(gk)
    assert r["converged"]
    assert abs(r["sigma1_rel_to_edge"]) <= 0.02, r


def test_config4_gradient_against_central_differences(gk):
    r = clp.check_gradient_20k_x_200k(gk, ncoords=3)
    assert r["closed_form_sigma_part_max_rel_err"] <= 1e-8, r["closed_form_sigma_part_max_rel_err"]
    for row in r["rows"]:
        assert row["pass_h1e-6"], row
        assert row["rel_err_h1e-4"] <= 1e-4, row
