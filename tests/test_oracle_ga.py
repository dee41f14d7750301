"""Pins of the oracle's GA operators (Sec. 3.1, Algorithm 1, Table 3) by
properties that hold whatever the random draws: sorting against numpy, exact
integer weights, the defining property of stochastic universal sampling, the
structure of each crossover child, mutation rate, elitism, termination."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1403_4099_gb300 import synth


def test_init_range_and_determinism(orc):
    a = orc.ga_init(64, 16, seed=123)
    b = orc.ga_init(64, 16, seed=123)
    c = orc.ga_init(64, 16, seed=124)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0 and a.max() < 16
    k = orc.ga_init(400, 50, seed=5, K0=7)
    assert k.min() == 0 and k.max() == 6
    counts = np.bincount(k.ravel(), minlength=7)
    expect = k.size / 7
    assert np.all(np.abs(counts - expect) < 6 * math.sqrt(expect))


def test_rank_matches_lexsort(orc):
    rng = np.random.default_rng(0)
    L = np.round(rng.standard_normal(1000), 1)  # many ties
    L[5] = -np.inf
    L[9] = np.nan  # ranks as -inf
    perm = orc.ga_rank(L)
    key = np.where(np.isnan(L), -np.inf, L)
    ref = np.lexsort((np.arange(1000), -key))
    assert np.array_equal(perm, ref)


def test_rank_weights_exact(orc):
    P = 5000
    w = orc.ga_weights(np.zeros(P), np.arange(P, dtype=np.int32), orc.SCALING_RANK)
    exact = np.array([math.isqrt((1 << 64) // (r + 1)) for r in range(P)], dtype=np.uint64)
    # floor(2^32 / sqrt(r)) computed exactly with integers; FP64 may round across by 1
    diff = w.astype(np.int64) - exact.astype(np.int64)
    assert np.abs(diff).max() <= 1
    assert (diff == 0).mean() > 0.99
    assert w[0] == 1 << 32 and np.all(np.diff(w.astype(np.int64)) <= 0)


def test_prop_weights(orc):
    rng = np.random.default_rng(1)
    L = rng.uniform(-1, 10, 300)
    perm = orc.ga_rank(L)
    w = orc.ga_weights(L, perm, orc.SCALING_PROP)
    assert w[0] == 1 << 32 and np.all(np.diff(w.astype(np.int64)) <= 0)
    for r in range(300):
        x = max(L[perm[r]], 0.0)
        exact = Fraction(x) / Fraction(L[perm[0]]) * (1 << 32)
        assert abs(int(w[r]) - math.floor(exact)) <= 1
    assert np.all(orc.ga_weights(-np.abs(L), orc.ga_rank(-np.abs(L)), orc.SCALING_PROP) == 1)


@pytest.mark.parametrize("P,M", [(64, 62), (1000, 990), (37, 37), (4096, 4094), (10, 3)])
def test_sus_counts_are_floor_or_ceil_of_expectation(orc, P, M):
    rng = np.random.default_rng(P + M)
    w = orc.ga_weights(np.zeros(P), np.arange(P, dtype=np.int32), orc.SCALING_RANK)
    w = (w * rng.integers(1, 4, P).astype(np.uint64)).astype(np.uint64)
    W = int(w.astype(object).sum())
    for u in [0, 1, 2**31, 2**32 - 1, int(rng.integers(0, 2**32))]:
        sel = orc.ga_sus(w, M, u)
        assert np.all(np.diff(sel) >= 0) and sel.min() >= 0 and sel.max() < P
        counts = np.bincount(sel, minlength=P)
        for r in range(P):
            e = Fraction(M * int(w[r]), W)
            assert math.floor(e) <= counts[r] <= math.ceil(e)


def _classify_child(child, a, b):
    """Which crossover shapes explain child (no mutation)."""
    N = a.shape[0]
    kinds = set()
    if np.array_equal(child, a):
        kinds.add("copy")
    for cut in range(1, N):
        if np.array_equal(child[:cut], a[:cut]) and np.array_equal(child[cut:], b[cut:]):
            kinds.add("onepoint")
            break
    # merge: some cluster Q of b, all of whose genes now carry the a-label of one
    # of its members, everything else as in a
    for lab in np.unique(b):
        Q = b == lab
        if not np.array_equal(child[~Q], a[~Q]):
            continue
        v = child[Q]
        if np.all(v == v[0]) and v[0] in set(a[Q].tolist()):
            kinds.add("merge")
    return kinds


@pytest.mark.parametrize("pc,pkb,kind", [(0.0, 0.0, "copy"), (1.0, 0.0, "onepoint"),
                                          (1.0, 1.0, "merge")])
def test_crossover_structure(orc, pc, pkb, kind):
    rng = np.random.default_rng(11)
    P, N = 40, 12
    pop = rng.integers(0, 5, (P, N)).astype(np.int32)
    L = rng.standard_normal(P)
    prm = orc.params(P, N, elite=3, pc=pc, pkb=pkb, pm=0.0)
    nxt, perm, par = orc.ga_evolve(pop, L, prm, seed=99, g=4)
    M = P - 3
    assert np.array_equal(nxt[:3], pop[perm[:3]])
    for k in range(M):
        a, b = pop[par[k]], pop[par[(k + M // 2) % M]]
        assert kind in _classify_child(nxt[3 + k], a, b), k


def test_mixed_crossover_rates(orc):
    rng = np.random.default_rng(12)
    P, N = 2000, 20
    pop = rng.integers(0, 20, (P, N)).astype(np.int32)
    L = rng.standard_normal(P)
    prm = orc.params(P, N, elite=0, pc=0.9, pkb=0.0, pm=0.0)
    nxt, perm, par = orc.ga_evolve(pop, L, prm, seed=3, g=0)
    copies = sum(np.array_equal(nxt[k], pop[par[k]]) for k in range(P))
    # 10% no-crossover plus the rare one-point cut that reproduces a
    assert 0.07 * P < copies < 0.14 * P
    prm = orc.params(P, N, elite=0, pc=1.0, pkb=0.5, pm=0.0)
    nxt, perm, par = orc.ga_evolve(pop, L, prm, seed=4, g=0)
    M = P
    kinds = [_classify_child(nxt[k], pop[par[k]], pop[par[(k + M // 2) % M]]) for k in range(P)]
    merges = sum("merge" in k and "onepoint" not in k for k in kinds)
    onepoints = sum("onepoint" in k and "merge" not in k for k in kinds)
    assert abs(merges - onepoints) < 0.15 * P


def test_mutation_rate_and_elites_untouched(orc):
    rng = np.random.default_rng(13)
    P, N, E = 500, 100, 5
    pop = rng.integers(0, N, (P, N)).astype(np.int32)
    L = rng.standard_normal(P)
    pm = 0.02
    prm = orc.params(P, N, elite=E, pc=0.0, pm=pm)
    nxt, perm, par = orc.ga_evolve(pop, L, prm, seed=7, g=2)
    assert np.array_equal(nxt[:E], pop[perm[:E]])
    changed = (nxt[E:] != pop[par]).sum()
    n = (P - E) * N
    p = pm * (1 - 1 / N)
    assert abs(changed - n * p) < 6 * math.sqrt(n * p * (1 - p))
    assert nxt.min() >= 0 and nxt.max() < N


def test_selection_follows_rank(orc):
    rng = np.random.default_rng(14)
    P, N = 256, 8
    pop = rng.integers(0, N, (P, N)).astype(np.int32)
    L = rng.standard_normal(P)
    prm = orc.params(P, N, elite=2, pc=0.0, pm=0.0)
    _, perm, par = orc.ga_evolve(pop, L, prm, seed=1, g=0)
    rank_of = np.empty(P, np.int64)
    rank_of[perm] = np.arange(P)
    r = rank_of[par]
    assert np.all(np.diff(r) >= 0)  # pointers walk the line in rank order
    assert (r < P // 4).mean() > 0.4  # 1/sqrt(rank) favours the fittest


def test_termination_rule(orc):
    prm = orc.params(10, 5, max_gens=30, stall_gens=5, tol=1e-5)
    h = np.concatenate([np.linspace(1, 2, 10), np.full(21, 2.0)])
    done = [g for g in range(31) if orc.ga_terminated(h, g, prm)]
    assert done[0] == 14  # best_14 - best_9 = 0
    h2 = np.linspace(1, 100, 31)
    assert [g for g in range(31) if orc.ga_terminated(h2, g, prm)] == [30]
    prm_off = orc.params(10, 5, max_gens=30, stall_gens=5, tol=-1.0)
    assert [g for g in range(31) if orc.ga_terminated(h, g, prm_off)] == [30]


def test_run_elitism_monotone_and_recovers_small16(orc):
    p = synth.small16()
    C = orc.pearson(p.R)
    prm = orc.params(64, 16, elite=2, max_gens=200, stall_gens=50, tol=1e-5, pm=0.01)
    out = orc.ga_run(C, prm, seed=synth.seed_for(1), ring=True)
    assert np.all(np.diff(out["hist"]) >= 0)
    assert orc.ari(out["best"], p.truth) >= 0.99
    assert out["L"] == orc.loglik(out["best"], C)
    assert np.array_equal(out["ring"][-1], out["best"])


def test_threshold_init_matches_scipy_components(orc):
    """Components of {C > tau} against scipy's connected_components (a library
    routine), for the tau each individual draws."""
    sp = pytest.importorskip("scipy.sparse.csgraph")
    from scipy.sparse import csr_matrix
    p = synth.n100()
    C = orc.pearson(p.R)
    pop = orc.ga_init_threshold(C, 40, seed=77, tau_lo=0.05, tau_hi=0.6)
    seen_tau = []
    for q in range(40):
        w = orc.philox((0, q, 0, 4), (77, 0))
        tau = 0.05 + (0.6 - 0.05) * (float(w[0]) * 2.0 ** -32)
        seen_tau.append(tau)
        A = csr_matrix(np.triu(C > tau, 1))
        _, comp = sp.connected_components(A, directed=False)
        assert orc.ari(pop[q], comp.astype(np.int32)) == 1.0
        # label = the member joining Prim's tree first
        order = orc.prim_order(C)
        pos = np.empty(100, np.int64); pos[order] = np.arange(100)
        for lab in np.unique(pop[q]):
            members = np.flatnonzero(pop[q] == lab)
            assert lab == members[np.argmin(pos[members])]
    assert max(seen_tau) - min(seen_tau) > 0.3


def test_prim_order_is_a_maximum_spanning_tree(orc):
    """Total weight of the tree Prim's order implies equals scipy's minimum
    spanning tree of -C (a library routine)."""
    sp = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(21)
    C = orc.pearson(rng.standard_normal((60, 30)))
    order = orc.prim_order(C)
    assert sorted(order.tolist()) == list(range(30)) and order[0] == 0
    # attach each vertex to its best earlier vertex: the Prim tree
    tot = 0.0
    for k in range(1, 30):
        tot += max(C[order[k], order[:k]])
    mst = sp.minimum_spanning_tree(-(C - np.eye(30)) + 10.0)  # shift keeps weights positive
    assert abs((-(mst.sum() - 10.0 * 29)) - tot) < 1e-9


def _mutation_indicator(orc, P, N, pm, seed=21, labels=False):
    """Per gene: did mutation change it? (pc = 0, no elites: child = parent + mutation)."""
    rng = np.random.default_rng(seed)
    pop = rng.integers(0, N, (P, N)).astype(np.int32)
    L = rng.standard_normal(P)
    prm = orc.params(P, N, elite=0, pc=0.0, pm=pm)
    nxt, perm, par = orc.ga_evolve(pop, L, prm, seed=seed, g=5)
    assert nxt.min() >= 0 and nxt.max() < N
    x = nxt != pop[par]
    return (x, nxt[x]) if labels else x


def test_mutation_law_is_independent_per_gene(orc):
    """Mutation is drawn as geometric gaps inside blocks of 16 genes; the law must
    still be one independent Bernoulli(P_m) per gene: every position (first,
    middle and last of a block, and of the short last block) mutates at the same
    rate, neighbours are uncorrelated, and the count per child has the binomial
    variance. A lost step after a mutated gene, a gap counted from the wrong
    position or a block offset error shows up as a position bias or a
    correlation."""
    P, N, pm = 6000, 37, 0.25
    x, new = _mutation_indicator(orc, P, N, pm, labels=True)
    x = x.astype(np.float64)
    # the new labels are uniform on [0, N) and independent of the gap draws
    # (a label taken from the gap word would crowd the top of the range)
    hist = np.bincount(new, minlength=N)
    e = new.size / N
    assert np.all(np.abs(hist - e) < 6 * math.sqrt(e)), hist
    assert abs(new.mean() - (N - 1) / 2) < 6 * math.sqrt((N * N - 1) / 12 / new.size)
    p = pm * (1 - 1 / N)  # a redrawn label equals the old one with probability 1/N
    sd = math.sqrt(p * (1 - p) / P)
    rates = x.mean(axis=0)
    assert np.all(np.abs(rates - p) < 5 * sd), rates
    for j in range(N - 1):  # neighbours, across block boundaries too (15|16, 31|32)
        c = np.corrcoef(x[:, j], x[:, j + 1])[0, 1]
        assert abs(c) < 5 / math.sqrt(P), (j, c)
    counts = x.sum(axis=1)
    assert abs(counts.var() - N * p * (1 - p)) < 0.1 * N * p * (1 - p)


def test_mutation_extremes(orc):
    """P_m = 1 replaces every gene (a block then needs eight Philox calls);
    P_m below 2^-32 replaces none."""
    P, N = 400, 50
    x = _mutation_indicator(orc, P, N, 1.0)
    frac = x.mean()
    assert abs(frac - (1 - 1 / N)) < 5 * math.sqrt((1 / N) * (1 - 1 / N) / (P * N))
    assert not _mutation_indicator(orc, P, N, 1e-12).any()


def test_paper_shaped_inputs():
    """The paper-shaped generators: 40 stocks in 4 clusters of 10; an 18-stock
    series long enough for 1760 windows of 1800 bars with 3 clusters of 6."""
    from paper_1403_4099_gb300 import synth
    tr = synth.paper_training()
    assert tr.R.shape == (1800, 40)
    assert sorted(np.bincount(tr.truth).tolist()) == [10, 10, 10, 10]
    st = synth.paper_stream()
    assert st.R.shape == (1800 + 1760 - 1, 18) and st.W == 1800 and st.windows == 1760
    assert sorted(np.bincount(st.truth).tolist()) == [6, 6, 6]


def test_island_migration_ring(orc):
    """Ring migration: island k's first m members land, in order, on the last m
    slots of island k + 1 (the last island feeds the first); the rest of every
    island is untouched, and the fitness travels with the members."""
    rng = np.random.default_rng(41)
    K, P, N, m = 4, 10, 6, 3
    pops = rng.integers(0, N, (K, P, N)).astype(np.int32)
    Ls = rng.standard_normal((K, P))
    new, nl = orc.island_migrate(pops, Ls, m)
    for k in range(K):
        to = (k + 1) % K
        assert np.array_equal(new[to, P - m:], pops[k, :m])
        assert np.array_equal(nl[to, P - m:], Ls[k, :m])
        assert np.array_equal(new[to, :P - m], pops[to, :P - m])
    with pytest.raises(Exception):
        orc.island_migrate(pops, Ls, 6)  # 2 m > P
