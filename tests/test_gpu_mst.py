"""Per-cluster minimum spanning trees through the C ABI (cluster_mst) against
the oracle's Kruskal trees: same edges and exactly the same distances (both
sides evaluate sqrt(2 (1 - C_uv)) on the same entry), clusters in
first-occurrence order."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1403_4099_gb300 import gpga
    gpga.lib()
    return gpga


def _by_cluster(s, u, v, w):
    """{cluster label: {(u, v): w}} keeping the clusters' first-occurrence order."""
    out = {}
    for a, b, d in zip(u.tolist(), v.tolist(), w.tolist()):
        out.setdefault(int(s[a]), {})[(a, b)] = d
    return out


@pytest.mark.parametrize("case", ["planted", "random", "few", "one", "singletons"])
def test_cluster_mst_matches_oracle(g, orc, case):
    import torch
    pl = synth.n100(replicate=3)
    C = orc.pearson(pl.R)
    rng = np.random.default_rng(5)
    s = {"planted": pl.truth,
         "random": rng.integers(0, 100, 100),
         "few": rng.integers(0, 4, 100),
         "one": np.zeros(100),
         "singletons": np.arange(100)}[case].astype(np.int32)
    u, v, w = g.cluster_mst(dev(C), dev(s, torch.int32))
    ou, ov, ow = orc.cluster_mst(s, C)
    assert len(u) == len(ou) == 100 - len(np.unique(s))
    assert np.all(u < v)
    gb, ob = _by_cluster(s, u, v, w), _by_cluster(s, ou, ov, ow)
    assert list(gb) == list(ob)  # clusters in first-occurrence order
    for lab in ob:
        assert gb[lab] == ob[lab]  # same edges, bit-identical distances


def test_cluster_mst_n500_and_bad_label(g, orc):
    import torch
    pl = synth.n500()
    C = orc.pearson(pl.R)
    u, v, w = g.cluster_mst(dev(C), dev(pl.truth, torch.int32))
    ou, ov, ow = orc.cluster_mst(pl.truth, C)
    assert set(zip(u.tolist(), v.tolist())) == set(zip(ou.tolist(), ov.tolist()))
    assert np.sum(w) == pytest.approx(np.sum(ow), rel=1e-12)
    bad = pl.truth.copy()
    bad[7] = 500
    with pytest.raises(g.GpgaError):
        g.cluster_mst(dev(C), dev(bad, torch.int32))
