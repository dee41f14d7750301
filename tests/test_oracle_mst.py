"""Oracle per-cluster minimum spanning trees (the cluster trees of Sec. 4, on
the correlation distance d = sqrt(2 (1 - C))) against SciPy's minimum
spanning tree of each cluster's distance submatrix (a library routine), plus
the special cases: singletons have no edge, one cluster of N has N - 1."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth


def _scipy_forest(s, C):
    sp = pytest.importorskip("scipy.sparse.csgraph")
    edges = set()
    total = 0.0
    order = []
    for i, lab in enumerate(s):
        if lab not in order:
            order.append(lab)
    for lab in order:
        m = np.flatnonzero(s == lab)
        if m.size < 2:
            continue
        d = np.sqrt(2.0 * (1.0 - C[np.ix_(m, m)]))
        np.fill_diagonal(d, 0.0)
        t = sp.minimum_spanning_tree(d).tocoo()
        for a, b, w in zip(t.row, t.col, t.data):
            u, v = sorted((int(m[a]), int(m[b])))
            edges.add((u, v))
            total += w
    return edges, total


@pytest.mark.parametrize("rep", range(4))
def test_cluster_mst_matches_scipy(orc, rep):
    rng = np.random.default_rng(30 + rep)
    pl = synth.n100(replicate=rep)
    C = orc.pearson(pl.R)
    for s in (pl.truth, rng.integers(0, 12, 100).astype(np.int32)):
        u, v, w = orc.cluster_mst(s, C)
        assert np.all(u < v)
        assert len(u) == 100 - len(np.unique(s))
        edges, total = _scipy_forest(s, C)
        assert set(zip(u.tolist(), v.tolist())) == edges
        assert w.sum() == pytest.approx(total, rel=1e-12)
        # every edge joins two genes of the same cluster, each cluster a tree
        assert np.all(s[u] == s[v])


def test_cluster_mst_special_cases(orc):
    pl = synth.small16()
    C = orc.pearson(pl.R)
    u, v, w = orc.cluster_mst(np.arange(16, dtype=np.int32), C)
    assert len(u) == 0
    u, v, w = orc.cluster_mst(np.zeros(16, np.int32), C)
    assert len(u) == 15 and len(set(u.tolist()) | set(v.tolist())) == 16
    # the weight is the correlation distance of the pair
    assert np.allclose(w, np.sqrt(2 * (1 - C[u, v])))
