"""Random-matrix cleaning of C on the GPU (parallel cyclic Jacobi in FP64 +
trace-preserving clipping of the Wishart-range eigenvalues, Sec. 4.2) against
the oracle: eigenvalues, noise-set sizes and the cleaned matrices, single and
batched, single-tile and multi-tile, odd and even N, plus the edge cases."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu

# Jacobi stops at max |a_ij| <= 1e-14 ||A||_F: eigenvalues then agree with
# LAPACK to ~1e-13 |lambda|_max, the kept eigenvectors to ~1e-14 ||A||_F / gap
EIG_TOL = 1e-11
C_TOL = 1e-9


@pytest.fixture(scope="module")
def g():
    from paper_1403_4099_gb300 import gpga
    gpga.lib()
    return gpga


def _margin_ok(orc, C, T):
    """No eigenvalue within 1e-8 of a range edge, so both sides take the same
    noise set whatever their rounding."""
    lo, hi = orc.wishart_range(C.shape[0], T)
    w = np.linalg.eigvalsh(C)
    return np.min(np.abs(np.concatenate([w - lo, w - hi]))) > 1e-8


def _check(g, orc, C, T):
    assert _margin_ok(orc, C, T)
    Cd = dev(C)
    ev, nn, sweeps = g.corr_clean_rmt(Cd, T)
    ref, w, n_ref = orc.clean_rmt(C, T)
    assert nn == [n_ref]
    assert sweeps <= 40
    assert np.max(np.abs(ev.cpu().numpy()[0] - w)) < EIG_TOL * max(1.0, np.abs(w).max())
    got = Cd.cpu().numpy()
    assert np.max(np.abs(got - ref)) < C_TOL
    assert np.array_equal(got, got.T)
    assert np.all(np.diag(got) == 1.0)
    return got, n_ref


@pytest.mark.parametrize("work", ["small16", "n100", "n500"])
def test_clean_matches_oracle_on_workloads(g, orc, work):
    pl = getattr(synth, work)()
    T = pl.R.shape[0]
    C = orc.pearson(pl.R)
    _check(g, orc, C, T)


@pytest.mark.parametrize("N,T", [(5, 40), (18, 1800), (33, 150), (37, 120), (64, 200), (101, 300)])
def test_clean_matches_oracle_sizes(g, orc, N, T):
    """One tile (N <= 32) and several, odd N (a padding index), short windows."""
    pl = synth.planted_returns(np.random.default_rng(N), T, [N // 3, N // 4], [0.5, 0.3],
                               n_noise=N - N // 3 - N // 4, beta=0.2)
    C = orc.pearson(pl.R)
    _check(g, orc, C, T)


def test_clean_two_blocks_closed_form(g, orc):
    n1, r1, n2, r2 = 30, 0.6, 20, 0.3
    C = np.zeros((50, 50))
    C[:n1, :n1] = r1
    C[n1:, n1:] = r2
    np.fill_diagonal(C, 1.0)
    got, n_noise = _check(g, orc, C, 100)
    assert n_noise == 48


def _batch_check(g, orc, Cs, T):
    Cs = [C for C in Cs if _margin_ok(orc, C, T)]
    B = np.stack(Cs)
    Bd = dev(B)
    ev, nn, sweeps = g.corr_clean_rmt(Bd, T)
    got = Bd.cpu().numpy()
    evh = ev.cpu().numpy()
    for k, C in enumerate(Cs):
        ref, w, n_ref = orc.clean_rmt(C, T)
        assert nn[k] == n_ref
        assert np.max(np.abs(evh[k] - w)) < EIG_TOL * max(1.0, np.abs(w).max())
        assert np.max(np.abs(got[k] - ref)) < C_TOL
    # one matrix alone agrees with its slot of the batch
    one = dev(Cs[-1])
    g.corr_clean_rmt(one, T)
    assert np.max(np.abs(one.cpu().numpy() - got[-1])) < C_TOL
    return nn


def test_clean_batch_of_paper_windows(g, orc):
    """The paper's stream shape: N = 18 over windows of 1800 bars, one batch.
    Its within-cluster modes lie below the range and nothing falls inside it,
    so every window comes back unchanged."""
    st = synth.paper_stream(windows=64)
    Cs = [orc.pearson(st.R[k:k + st.W]) for k in range(64)]
    nn = _batch_check(g, orc, Cs, st.W)
    assert set(nn) == {0}


def test_clean_batch_of_short_windows(g, orc):
    """48 windows of 150 bars (q = 0.12) slid by 30 over the same stream: most
    eigenvalues are noise; cleaned together and one by one by the oracle."""
    st = synth.paper_stream(windows=64)
    Cs = [orc.pearson(st.R[30 * k:30 * k + 150]) for k in range(48)]
    nn = _batch_check(g, orc, Cs, 150)
    assert min(nn) > 0


def test_clean_known_spectrum_not_unit_diagonal(g, orc):
    rng = np.random.default_rng(11)
    Q, R = np.linalg.qr(rng.standard_normal((6, 6)))
    Q = Q * np.sign(np.diag(R))
    C = (Q * np.array([0.1, 0.3, 1.0, 2.0, 2.5, 5.0])) @ Q.T
    C = 0.5 * (C + C.T)
    Cd = dev(C)
    ev, nn, _ = g.corr_clean_rmt(Cd, 24)
    assert nn == [3]
    assert np.max(np.abs(ev.cpu().numpy()[0] - [0.1, 0.3, 1.0, 2.0, 2.5, 5.0])) < 1e-12
    ref, _, _ = orc.clean_rmt(C, 24)
    assert np.max(np.abs(Cd.cpu().numpy() - ref)) < C_TOL


def test_clean_identity_and_empty_range(g, orc):
    Cd = dev(np.eye(10))
    _, nn, _ = g.corr_clean_rmt(Cd, 100)
    assert nn == [10]
    assert np.array_equal(Cd.cpu().numpy(), np.eye(10))
    C = 0.5 * np.ones((10, 10)) + 0.5 * np.eye(10)
    Cd = dev(C)
    _, nn, _ = g.corr_clean_rmt(Cd, 1000)
    assert nn == [0]
    assert np.array_equal(Cd.cpu().numpy(), C)  # untouched


def test_clean_rejects_bad_input(g):
    import torch
    C = dev(np.eye(8))
    with pytest.raises(g.GpgaError):
        g.corr_clean_rmt(C, 0.0)
    with pytest.raises(g.GpgaError):
        g.corr_clean_rmt(C, float("nan"))
    bad = np.eye(8)
    bad[2, 3] = bad[3, 2] = np.nan
    with pytest.raises(g.GpgaError):
        g.corr_clean_rmt(dev(bad), 100)
    with pytest.raises(TypeError):
        g.corr_clean_rmt(torch.eye(8, dtype=torch.float64), 100)  # host memory


# ---------------------------------------------------------------------------
# The tridiagonal solver (Householder reduction, bisection, inverse iteration),
# which cleans one matrix at a time from 33 stocks up (and every batch from
# 128 stocks up): the cases above with N > 32 already run it; these add its
# own edge cases.
# ---------------------------------------------------------------------------
def test_tri_known_spectrum(g, orc):
    """A random orthogonal basis with a prescribed spectrum (no eigenvalue near
    a range edge): the eigenvalues come back to 1e-12 and C' matches."""
    N, T = 80, 400
    rng = np.random.default_rng(23)
    Q, R = np.linalg.qr(rng.standard_normal((N, N)))
    Q = Q * np.sign(np.diag(R))
    lo, hi = orc.wishart_range(N, T)
    lam = np.concatenate([np.linspace(0.05, lo - 0.05, 10), np.linspace(lo + 0.05, hi - 0.05, 60),
                          np.linspace(hi + 0.1, 9.0, 10)])
    C = (Q * lam) @ Q.T
    C = 0.5 * (C + C.T)
    got, n_ref = _check(g, orc, C, T)
    assert n_ref == 60


def test_tri_exact_multiplicity_in_the_expanded_set(g, orc):
    """One block of 10 stocks at correlation 0.9 among 110 independent ones:
    the kept set is 0.1 nine times over (exactly) and 9.1; the noise set is 1
    110 times, equal to its mean, so C' = C. Inverse iteration must span the
    nine-fold eigenspace (distinct starts, Gram-Schmidt in the group)."""
    N, T = 120, 1200
    C = np.eye(N)
    C[:10, :10] = 0.9
    np.fill_diagonal(C, 1.0)
    Cd = dev(C)
    ev, nn, sweeps = g.corr_clean_rmt(Cd, T)
    assert nn == [110] and sweeps == 0
    assert np.max(np.abs(ev.cpu().numpy()[0] - np.sort(np.linalg.eigvalsh(C)))) < 1e-12
    ref, _, _ = orc.clean_rmt(C, T)
    assert np.max(np.abs(Cd.cpu().numpy() - ref)) < C_TOL
    assert np.max(np.abs(Cd.cpu().numpy() - C)) < C_TOL


def test_tri_identity_and_empty_range(g, orc):
    N = 100
    Cd = dev(np.eye(N))
    _, nn, sweeps = g.corr_clean_rmt(Cd, 1000)
    assert nn == [N] and sweeps == 0
    assert np.array_equal(Cd.cpu().numpy(), np.eye(N))
    C = 0.5 * np.ones((N, N)) + 0.5 * np.eye(N)
    Cd = dev(C)
    _, nn, _ = g.corr_clean_rmt(Cd, 5000)  # range [0.7, 1.3]: 0.5 and 50.5 outside
    assert nn == [0]
    assert np.array_equal(Cd.cpu().numpy(), C)  # untouched


def test_tri_small_batch_matches_oracle_one_by_one(g, orc):
    """Three matrices of 150 stocks in one call (the tridiagonal solver takes
    them in turn)."""
    Cs = []
    for k in range(3):
        pl = synth.planted_returns(np.random.default_rng(300 + k), 600, [40, 30, 20], [0.6, 0.4, 0.3],
                                   n_noise=60, beta=0.25)
        Cs.append(orc.pearson(pl.R))
    nn = _batch_check(g, orc, Cs, 600)
    assert min(nn) > 0


def test_tri_rejects_non_finite_and_leaves_c(g):
    bad = np.eye(64)
    bad[5, 9] = bad[9, 5] = np.inf
    Cd = dev(bad)
    with pytest.raises(g.GpgaError) as e:
        g.corr_clean_rmt(Cd, 500)
    assert e.value.code == g.ERR_ARG
    assert np.array_equal(Cd.cpu().numpy(), bad)


def test_tri_timeout_then_recovers(g, orc):
    """A wait budget of 0 cycles makes the reduction's first grid barrier give
    up at once (nothing hangs): GPGA_ERR_TIMEOUT and C unchanged; with the
    default budget the same call then matches the oracle."""
    pl = synth.n100()
    C = orc.pearson(pl.R)
    T = pl.R.shape[0]
    Cd = dev(C)
    g.set_wait_budget(0)
    try:
        with pytest.raises(g.GpgaError) as e:
            g.corr_clean_rmt(Cd, T)
    finally:
        g.set_wait_budget(-1)
    assert e.value.code == g.ERR_TIMEOUT
    assert np.array_equal(Cd.cpu().numpy(), C)
    _check(g, orc, C, T)
