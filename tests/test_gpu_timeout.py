"""Failure detection without a GPU fault: the bounded mbarrier waits of the
tensor form's tcgen05 pipeline give up when their budget runs out, the kernel
drains the MMAs it issued, frees its tensor memory and returns, and the call
reports GPGA_ERR_TIMEOUT. A budget of 0 cycles makes the first wait give up at
once (nothing hangs, nothing faults); the next call with the default budget on
the same process must score correctly, which shows that the context and the
tensor memory survived."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth
from gpu_util import assert_L_close, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1403_4099_gb300 import build, gpga
    build.build()
    return gpga


def test_ga_score_timeout_then_recovers(g, orc):
    import torch
    p = synth.n100()
    C = orc.pearson(p.R)
    rng = np.random.default_rng(17)
    pop = synth.random_labels(rng, 300, 100)
    labels, Cd = dev(pop, torch.int32), dev(C)
    g.set_wait_budget(0)
    try:
        with pytest.raises(g.GpgaError) as e:
            g.ga_score(labels, Cd, form=g.FORM_TENSOR)
    finally:
        g.set_wait_budget(-1)
    assert e.value.code == g.ERR_TIMEOUT
    for _ in range(2):  # the default budget again: correct scores, twice
        L = g.ga_score(labels, Cd, form=g.FORM_TENSOR)
        torch.cuda.synchronize()
        assert_L_close(L.cpu().numpy(), orc.loglik_batch(pop, C), "after timeout")


def test_ga_run_reports_timeout(g, orc):
    p = synth.small16()
    C = orc.pearson(p.R)
    prm = g.default_params(P=64, elite=2, max_gens=20, tol=-1.0, form=g.FORM_TENSOR)
    g.set_wait_budget(0)
    try:
        ga = g.GA(dev(C), prm, seed=3)  # generation 0 is scored with the zero budget
    finally:
        g.set_wait_budget(-1)
    with pytest.raises(g.GpgaError) as e:
        ga.best()
    assert e.value.code == g.ERR_TIMEOUT
    ga.reset(dev(C), 4)  # clears the run's error word
    ga.step(5)
    lab, L, gen = ga.best()
    assert gen == 5 and abs(L - orc.loglik(lab, C)) <= 1e-9 * max(1.0, abs(L))
    ga.close()
