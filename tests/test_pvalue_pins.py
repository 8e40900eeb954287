"""The oracle's Gumbel P-value (the per-sequence P-value the filters record,
Alg. 2 / Alg. 7) against a library routine and closed forms."""
import math

import numpy as np
import pytest

import oracle


def test_matches_scipy_gumbel_survival():
    stats = pytest.importorskip("scipy.stats")
    x = np.linspace(-20, 40, 601)
    for mu, lam in ((-4.2, math.log(2)), (0.0, 1.0), (3.5, 0.5)):
        want = stats.gumbel_r.sf(x, loc=mu, scale=1.0 / lam)
        got = oracle.gumbel_pvalue(x, mu, lam)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)


def test_closed_forms():
    mu, lam = 1.25, 0.7
    assert oracle.gumbel_pvalue(mu, mu, lam) == pytest.approx(1 - math.exp(-1), rel=1e-15)
    big = mu + 60.0
    assert oracle.gumbel_pvalue(big, mu, lam) == pytest.approx(math.exp(-lam * 60.0), rel=1e-12)
    assert oracle.gumbel_pvalue(mu - 30.0, mu, lam) == pytest.approx(1.0, abs=1e-12)
    x = np.linspace(-10, 10, 200)
    p = oracle.gumbel_pvalue(x, mu, lam)
    assert np.all(np.diff(p) <= 0)
    inner = p < 1 - 1e-12                      # below the float64 saturation at 1
    assert np.all(np.diff(p[inner]) < 0)
    assert oracle.gumbel_pvalue(np.inf, mu, lam) == 0.0
    assert np.isnan(oracle.gumbel_pvalue(np.nan, mu, lam))
