"""The paper-shaped workload (Sec. 4, Table 3): the 40-stock training set with
4 planted clusters and the 18-stock window stream, run through the library
with Table 3 parameters (P = 1000, <= 400 generations, P_c = P_kb = 0.9,
stall 50 generations at tolerance 1e-5, 10 elites)."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import metrics, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpga():
    from paper_1403_4099_gb300 import gpga as g
    g.lib()
    return g


def _params(gpga, **kw):
    base = dict(P=1000, elite=10, max_gens=400, stall_gens=50, tol=1e-5, pc=0.9, pkb=0.9,
                pm=0.1, form=gpga.FORM_GATHER)
    base.update(kw)
    return gpga.default_params(**base)


def test_training_set_recovered(gpga):
    """Most seeds recover the 4 planted clusters of the 40-stock training set."""
    import torch
    tr = synth.paper_training()
    C = gpga.cluster_corr(torch.from_numpy(tr.R).cuda())
    b = gpga.Batch([C] * 8, _params(gpga, pm=0.01), [100 + k for k in range(8)])
    while b.step(16) > 0:
        pass
    aris = [metrics.ari(b.best(k)[0], tr.truth) for k in range(8)]
    b.close()
    assert sum(a >= 0.99 for a in aris) >= 7, aris


def test_window_stream_recovered(gpga):
    """Windows of the 18-stock stream (3 planted clusters of 6, market mode)
    are clustered as planted, and a window's result in the fleet is the result
    of the same run alone."""
    import torch
    st = synth.paper_stream(windows=24)
    R = torch.from_numpy(st.R).cuda()
    Cs = [gpga.cluster_corr(R[k:k + st.W].contiguous()) for k in range(st.windows)]
    prm = _params(gpga)
    seeds = [5000 + k for k in range(st.windows)]
    b = gpga.Batch(Cs, prm, seeds)
    while b.step(16) > 0:
        pass
    aris = [metrics.ari(b.best(k)[0], st.truth) for k in range(st.windows)]
    assert np.mean(aris) >= 0.95, aris
    ga = gpga.GA(Cs[3], prm, seed=seeds[3])
    ga.step(prm.max_gens)
    lab, L, g = ga.best()
    ga.close()
    lb, Lb, gb = b.best(3)
    b.close()
    np.testing.assert_array_equal(lb, lab)
    assert Lb == L and gb == g
