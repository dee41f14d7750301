"""Oracle pre-processing upstream of C: the EWMA-weighted
Pearson correlation and the market-mode removal, pinned against library
routines (NumPy's weighted covariance, LAPACK eigenvectors) and closed forms."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth


def test_ewma_lambda_one_is_pearson(orc):
    R = synth.n100().R[:500]
    assert np.max(np.abs(orc.pearson_ewma(R, 1.0) - orc.pearson(R))) < 1e-14


@pytest.mark.parametrize("lam", [0.98, 0.9, 0.5])
def test_ewma_matches_numpy_weighted_cov(orc, lam):
    R = synth.n100().R[:400]
    T = R.shape[0]
    w = lam ** np.arange(T - 1, -1, -1, dtype=np.float64)
    S = np.cov(R, rowvar=False, aweights=w, ddof=0)
    d = np.sqrt(np.diag(S))
    ref = np.clip(S / np.outer(d, d), -1, 1)
    np.fill_diagonal(ref, 1.0)
    assert np.max(np.abs(orc.pearson_ewma(R, lam) - ref)) < 1e-12


def test_ewma_weights_only_the_recent_past(orc):
    """With a small lambda the estimate follows the newest rows: two halves
    with opposite correlation, the EWMA sees the second."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal(600)
    y = np.concatenate([x[:300], -x[300:]]) + 0.1 * rng.standard_normal(600)
    R = np.stack([x, y], axis=1)
    assert orc.pearson_ewma(R, 0.9)[0, 1] < -0.9
    assert abs(orc.pearson(R)[0, 1]) < 0.2


def test_market_removal_closed_form(orc):
    """A one-factor (market) correlation C = (1 - b) I + b J: its top
    eigenvector is uniform, lambda_1 = 1 + (N - 1) b, and the cleaned matrix
    is the identity."""
    N, b = 20, 0.3
    C = (1 - b) * np.eye(N) + b * np.ones((N, N))
    out, lam = orc.remove_market(C)
    assert lam == pytest.approx(1 + (N - 1) * b, rel=1e-12)
    # the cleaned off-diagonal entries are -1/(N-1)-scaled residuals of the
    # uniform mode: C' = (1 - b)(I - J/N), renormalised
    ref = (np.eye(N) - np.ones((N, N)) / N) / (1 - 1 / N)
    np.fill_diagonal(ref, 1.0)
    assert np.max(np.abs(out - ref)) < 1e-12


def test_market_removal_invariants(orc):
    pl = synth.n100()
    C = orc.pearson(pl.R)
    out, lam = orc.remove_market(C)
    assert np.allclose(np.diag(out), 1.0) and np.allclose(out, out.T)
    w, V = np.linalg.eigh(C)
    v = V[:, -1]
    # the removed direction: (C - lam v v^T) v = 0 before the renormalisation
    assert np.max(np.abs((C - lam * np.outer(v, v)) @ v)) < 1e-10
    # the market mode dominated the planted structure; once removed the mean
    # off-diagonal correlation drops
    off = ~np.eye(100, dtype=bool)
    assert out[off].mean() < C[off].mean() - 0.05
