"""Pins of the oracle's Giada-Marsili likelihood (Eq. 5, 6, 8).

What fixes it, other than itself:
  * Eq. 8 on an equicorrelated block (C = rho off the diagonal) equals
    -1/2 log det C_s; checked with numpy's slogdet (a library routine), per block,
    with unequal block sizes and rho, so a dropped term, a wrong sign, a swapped
    n_s / c_s or an off-by-one in (n_s - 1) all fail.
  * the two-element case -1/2 log(1 - rho^2), again via slogdet;
  * Eq. 6 as a matrix product: c_s = diag(S^T C S) with one-hot S (numpy matmul);
  * the derived invariants: L = 0 for singletons and for c_s = n_s, every term
    >= 0, relabelling invariance, stock-permutation invariance, locality.
"""
import numpy as np

from paper_1403_4099_gb300 import synth


def _onehot(s, N):
    S = np.zeros((N, N))
    S[np.arange(N), s] = 1.0
    return S


def _block_C(sizes, rhos, cross=0.0):
    N = sum(sizes)
    C = np.full((N, N), cross)
    s = np.concatenate([np.full(n, k) for k, n in enumerate(sizes)]).astype(np.int32)
    o = 0
    for n, r in zip(sizes, rhos):
        C[o:o + n, o:o + n] = r
        o += n
    np.fill_diagonal(C, 1.0)
    return C, s


def test_singletons_are_zero(orc):
    C = orc.pearson(synth.small16().R)
    assert orc.loglik(np.arange(16), C) == 0.0
    rng = np.random.default_rng(0)
    assert orc.loglik(rng.permutation(16), C) == 0.0


def test_two_element_closed_form(orc):
    for rho in [-0.95, -0.4, 0.0, 0.1, 0.5, 0.99]:
        C = np.array([[1.0, rho], [rho, 1.0]])
        L = orc.loglik([0, 0], C)
        assert abs(L - (-0.5 * np.linalg.slogdet(C)[1])) < 1e-13
    # the same pair inside a larger matrix with a singleton: only the pair counts
    C = np.array([[1.0, 0.3, 0.2], [0.3, 1.0, -0.1], [0.2, -0.1, 1.0]])
    assert abs(orc.loglik([1, 2, 1], C) + 0.5 * np.log(1 - 0.2 ** 2)) < 1e-14


def test_equicorrelated_blocks_equal_minus_half_logdet(orc):
    sizes = [7, 2, 5, 11, 3]
    rhos = [0.35, 0.8, -0.2, 0.05, 0.6]
    C, s = _block_C(sizes, rhos)
    expect = 0.0
    o = 0
    for n in sizes:
        expect += -0.5 * np.linalg.slogdet(C[o:o + n, o:o + n])[1]
        o += n
    L = orc.loglik(s, C)
    assert abs(L - expect) < 1e-11 * max(1.0, abs(expect))
    # the terms are separately positive: each block alone
    o = 0
    for n, r in zip(sizes, rhos):
        lab = np.arange(C.shape[0], dtype=np.int32)
        lab[o:o + n] = o
        Lb = orc.loglik(lab, C)
        assert abs(Lb - (-0.5 * np.linalg.slogdet(C[o:o + n, o:o + n])[1])) < 1e-11
        assert Lb >= 0.0
        o += n


def test_locality_cross_cluster_entries_do_not_matter(orc):
    sizes = [4, 6, 3]
    C0, s = _block_C(sizes, [0.5, 0.3, 0.7], cross=0.0)
    C1, _ = _block_C(sizes, [0.5, 0.3, 0.7], cross=0.07)
    assert orc.loglik(s, C0) == orc.loglik(s, C1)


def test_c_equal_n_gives_zero(orc):
    # off-diagonal entries that sum to zero: c_s = n_s, g* = 0 (Eq. 4) and the term vanishes
    C = np.eye(3)
    C[0, 1] = C[1, 0] = 0.2
    C[0, 2] = C[2, 0] = -0.1
    C[1, 2] = C[2, 1] = -0.1
    assert abs(orc.loglik([0, 0, 0], C)) < 1e-15


def test_cluster_sums_match_matrix_form(orc):
    rng = np.random.default_rng(5)
    p = synth.n100()
    C = orc.pearson(p.R)
    for s in [p.truth, rng.integers(0, 100, 100), rng.integers(0, 7, 100)]:
        s = np.asarray(s, np.int32)
        n, c, d = orc.cluster_sums(s, C)
        S = _onehot(s, 100)
        np.testing.assert_array_equal(n, S.sum(axis=0).astype(np.int32))
        np.testing.assert_allclose(c, np.diag(S.T @ C @ S), rtol=0, atol=1e-10)
        np.testing.assert_allclose(c + d, n.astype(np.float64) ** 2, rtol=0, atol=1e-10)
        assert d.min() >= 0.0


def test_relabelling_is_bit_exact(orc):
    rng = np.random.default_rng(6)
    C = orc.pearson(synth.n100().R)
    for _ in range(20):
        s = rng.integers(0, rng.integers(2, 100), 100).astype(np.int32)
        pi = rng.permutation(100).astype(np.int32)
        assert orc.loglik(s, C) == orc.loglik(pi[s], C)


def test_stock_permutation_invariance(orc):
    rng = np.random.default_rng(7)
    p = synth.n100()
    C = orc.pearson(p.R)
    for s in [p.truth, rng.integers(0, 30, 100).astype(np.int32)]:
        pi = rng.permutation(100)
        L0 = orc.loglik(s, C)
        L1 = orc.loglik(s[pi], C[np.ix_(pi, pi)])
        assert abs(L0 - L1) <= 1e-12 * max(1.0, abs(L0))


def test_terms_nonnegative_random(orc):
    rng = np.random.default_rng(8)
    for t in range(30):
        T = int(rng.integers(5, 80))
        R = rng.standard_normal((T, 24)) + rng.standard_normal((T, 1)) * rng.uniform(0, 2)
        C = orc.pearson(R)
        s = rng.integers(0, rng.integers(1, 24), 24).astype(np.int32)
        assert orc.loglik(s, C) >= -1e-12


def test_batch_equals_single(orc):
    rng = np.random.default_rng(9)
    C = orc.pearson(synth.n100().R)
    pop = rng.integers(0, 100, (33, 100)).astype(np.int32)
    L = orc.loglik_batch(pop, C, nthreads=4)
    assert all(L[i] == orc.loglik(pop[i], C) for i in range(33))


def test_degenerate_identical_series_are_clamped(orc):
    C = np.ones((4, 4))  # four identical series: d_s = 0
    L, k = orc.loglik([0, 0, 0, 1], C, with_clamps=True)
    assert k == 1 and np.isfinite(L) and L > 0
