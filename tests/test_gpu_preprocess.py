"""Pre-processing upstream of C on the GPU against the oracle: the EWMA
correlation (within the prelude's 1e-6) and the market-mode removal."""
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


@pytest.mark.parametrize("lam", [1.0, 0.98, 0.9])
@pytest.mark.parametrize("shape", [(400, 100), (1300, 37), (5000, 500)])
def test_ewma_matches_oracle(g, orc, lam, shape):
    T, N = shape
    R = synth.n500().R[:T, :N] if N == 500 else synth.n100().R[:T, :N]
    got = g.cluster_corr_ewma(dev(R), lam).cpu().numpy()
    ref = orc.pearson_ewma(R, lam)
    assert np.max(np.abs(got - ref)) < 1e-6
    if lam == 1.0:  # the same numbers as cluster_corr
        assert np.array_equal(got, g.cluster_corr(dev(R)).cpu().numpy())


@pytest.mark.parametrize("which", ["n100", "n500", "one_factor"])
def test_market_removal_matches_oracle(g, orc, which):
    if which == "one_factor":
        N, b = 64, 0.3
        C = (1 - b) * np.eye(N) + b * np.ones((N, N))
    else:
        pl = synth.n100() if which == "n100" else synth.n500()
        C = orc.pearson(pl.R)
    Cd = dev(C)
    lam, it = g.corr_remove_market(Cd)
    ref, lref = orc.remove_market(C)
    assert lam == pytest.approx(lref, rel=1e-12)
    assert it < 1000
    assert np.max(np.abs(Cd.cpu().numpy() - ref)) < 1e-9


def test_market_removal_drops_the_market_cluster(g, orc):
    """On the N=100 workload (market loading 0.3) the market mode alone makes
    "every stock in one cluster" score well; once it is removed that
    configuration scores about nothing while the planted partition still
    scores far above it."""
    import torch
    pl = synth.n100()
    C = orc.pearson(pl.R)
    Cm, _ = orc.remove_market(C)
    lab = torch.from_numpy(np.stack([pl.truth, np.zeros(100, np.int32)])).int().cuda()
    L0 = g.ga_score(lab, dev(C), form=g.FORM_GATHER).cpu().numpy()
    L1 = g.ga_score(lab, dev(Cm), form=g.FORM_GATHER).cpu().numpy()
    assert L0[1] > 1.0                # the market mode rewards one big cluster
    assert abs(L1[1]) < 1e-2          # gone with the market mode
    assert L1[0] > 100 * abs(L1[1])   # the planted clusters remain
