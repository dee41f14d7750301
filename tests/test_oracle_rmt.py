"""Oracle random-matrix cleaning of C (Sec. 4.2: the eigenvalues in the Wishart
range are removed in a trace-preserving way), pinned against closed forms that
do not call an eigensolver: matrices built from a known spectrum and a random
orthogonal basis, two-block correlation matrices whose eigenvectors are block
indicators, the identity, and spectra with nothing in the range."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth


def _orthogonal(rng, n):
    # QR of a Gaussian matrix, signs fixed: a random orthogonal basis
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))


def test_wishart_range_edges(orc):
    """Marchenko-Pastur edges of the correlation of independent series."""
    assert orc.wishart_range(25, 100) == pytest.approx((0.25, 2.25), abs=1e-15)
    assert orc.wishart_range(50, 50) == pytest.approx((0.0, 4.0), abs=1e-15)
    lo, hi = orc.wishart_range(18, 1800)
    assert lo == pytest.approx(0.81, abs=1e-15) and hi == pytest.approx(1.21, abs=1e-15)


# q = 6 / 24 = 0.25: range [0.25, 2.25]. 0.1 lies below it, 2.5 and 5.0 above;
# 0.3, 1.0 and 2.0 are noise, mean 1.1. The usual slips move the edges to
# (1 + q)^2 = 1.5625, 1 + sqrt q = 1.5, (1 - q)^2 = 0.5625 or 1 - sqrt q = 0.5,
# and each of those changes the noise set.
SPECTRUM = np.array([0.1, 0.3, 1.0, 2.0, 2.5, 5.0])


def test_known_spectrum_discriminates_edge_slips():
    lo, hi = 0.25, 2.25
    right = (SPECTRUM >= lo) & (SPECTRUM <= hi)
    q = 0.25
    for a, b in [(lo, (1 + q) ** 2), (lo, 1 + np.sqrt(q)), ((1 - q) ** 2, hi), (1 - np.sqrt(q), hi)]:
        assert not np.array_equal((SPECTRUM >= a) & (SPECTRUM <= b), right)


def test_clip_known_spectrum(orc):
    rng = np.random.default_rng(11)
    Q = _orthogonal(rng, 6)
    C = (Q * SPECTRUM) @ Q.T
    C = 0.5 * (C + C.T)
    Cp, w, noise, m = orc.rmt_clip(C, 24)
    assert np.allclose(w, SPECTRUM, atol=1e-13)
    assert noise.tolist() == [False, True, True, True, False, False]
    assert m == pytest.approx(1.1, abs=1e-13)
    want = (Q * np.array([0.1, 1.1, 1.1, 1.1, 2.5, 5.0])) @ Q.T
    assert np.max(np.abs(Cp - want)) < 1e-12
    assert np.trace(Cp) == pytest.approx(np.trace(C), abs=1e-12)


def _two_blocks(n1, r1, n2, r2):
    N = n1 + n2
    C = np.zeros((N, N))
    C[:n1, :n1] = r1
    C[n1:, n1:] = r2
    np.fill_diagonal(C, 1.0)
    return C


def test_clean_two_blocks_closed_form(orc):
    """Blocks of sizes n_b with inner correlation r_b: eigenvalues
    1 + (n_b - 1) r_b (block indicator vectors) and 1 - r_b (n_b - 1 times).
    At T = 100 (q = 0.5, range [0.0858, 2.914]) the 48 within-block modes are
    noise with mean m; C' keeps the two block modes, so inside block b
    C'_ij = (lambda_b - m) / n_b (+ m on the diagonal), 0 across blocks."""
    n1, r1, n2, r2 = 30, 0.6, 20, 0.3
    C = _two_blocks(n1, r1, n2, r2)
    out, w, n_noise = orc.clean_rmt(C, 100)
    assert n_noise == (n1 - 1) + (n2 - 1)
    m = ((n1 - 1) * (1 - r1) + (n2 - 1) * (1 - r2)) / (n1 + n2 - 2)
    want = np.zeros_like(C)
    for lo, n, r in [(0, n1, r1), (n1, n2, r2)]:
        lam = 1 + (n - 1) * r
        off = (lam - m) / n
        want[lo:lo + n, lo:lo + n] = off / (off + m)
    np.fill_diagonal(want, 1.0)
    assert np.max(np.abs(out - want)) < 1e-12
    assert np.allclose(np.sort(w), np.sort([1 + 29 * 0.6, 1 + 19 * 0.3] + [0.4] * 29 + [0.7] * 19),
                       atol=1e-12)


def test_clean_all_noise_is_identity(orc):
    out, w, n_noise = orc.clean_rmt(np.eye(10), 100)
    assert n_noise == 10
    assert np.array_equal(out, np.eye(10))


def test_clean_nothing_in_range_leaves_c(orc):
    """One factor b = 0.5 over N = 10: eigenvalues 5.5 and 0.5; at q = 0.01
    the range [0.81, 1.21] holds neither, so C comes back unchanged."""
    C = 0.5 * np.ones((10, 10)) + 0.5 * np.eye(10)
    out, w, n_noise = orc.clean_rmt(C, 1000)
    assert n_noise == 0
    assert np.array_equal(out, C)


@pytest.mark.parametrize("work", ["n100", "n500"])
def test_clean_invariants(orc, work):
    """On sample correlations of planted returns: C' keeps the trace, its kept
    eigenpairs, and maps each noise eigenvector to m v; C'' is symmetric, has
    unit diagonal, entries in [-1, 1] and no negative eigenvalue."""
    pl = getattr(synth, work)()
    T, N = pl.R.shape
    C = orc.pearson(pl.R)
    Cp, w, noise, m = orc.rmt_clip(C, T)
    assert 0 < noise.sum() < N
    assert np.trace(Cp) == pytest.approx(np.trace(C), abs=1e-10)
    _, V = np.linalg.eigh(C)
    lam = np.where(noise, m, w)
    assert np.max(np.abs(Cp @ V - V * lam)) < 1e-10
    out, w2, n_noise = orc.clean_rmt(C, T)
    assert n_noise == int(noise.sum())
    assert np.array_equal(out, out.T)
    assert np.all(np.diag(out) == 1.0)
    assert np.all(np.abs(out) <= 1.0)
    assert np.linalg.eigvalsh(out).min() > -1e-12


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_clean_reduces_estimation_noise(orc, seed):
    """The purpose the paper gives (Sec. 4.2): cleaning reduces the Gaussian
    noise of the estimate. Planted returns with a known population correlation
    (market beta^2 between all pairs, + (1 - beta^2) g_s inside cluster s), N =
    100 over T = 400: the cleaned matrix is nearer to it in Frobenius norm."""
    rng = np.random.default_rng(seed)
    N, T, beta = 100, 400, 0.3
    sizes, g = [25, 25, 20], np.array([0.3, 0.5, 0.2])
    pl = synth.planted_returns(rng, T, sizes, g, n_noise=N - sum(sizes), beta=beta,
                               shuffle=False)
    t = pl.truth
    gi = np.array([g[x] if x < len(sizes) else 0.0 for x in t])
    inside = (t[:, None] == t[None, :]) & (t[:, None] < len(sizes))
    Ct = beta ** 2 + (1 - beta ** 2) * np.where(inside, gi[:, None], 0.0)
    np.fill_diagonal(Ct, 1.0)
    C = orc.pearson(pl.R)
    out, _, n_noise = orc.clean_rmt(C, T)
    assert n_noise > 0
    assert np.linalg.norm(out - Ct) < 0.95 * np.linalg.norm(C - Ct)
