"""ga_score_noalloc: the allocation-free scoring entry point, for callers that
cannot let the library allocate device memory (their own allocator owns the
GPU, or their loop forbids allocator calls). Checked through the C-ABI against
the FP64 oracle and against ga_score's gather form, on two calls in a row (the
shared fixed scratch keeps the previous call's contents, which must not leak
into the next result), and across a refused call: a call with a label outside
[0, N) reports GPGA_ERR_ARG with NaN in that row, and the next clean call must
succeed with oracle-matching values (its error flags start from zero again).
Collected last so that a failure here comes after every other test has run."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth
from gpu_util import assert_L_close, dev

pytestmark = pytest.mark.gpu


def test_noalloc_matches_oracle_and_ga_score_two_calls(orc):
    import torch
    from paper_1403_4099_gb300 import build, gpga
    build.build()
    rng = np.random.default_rng(2024)
    cases = [(synth.n500(), 4096), (synth.n100(), 333)]
    for p, P in cases:
        N = p.R.shape[1]
        Ch = orc.pearson(p.R)
        C = dev(Ch)
        pops = [synth.random_labels(rng, P, N), synth.perturbed_population(rng, p.truth, P, 0.05)]
        for pop in pops:  # two calls in a row on different inputs
            labels = dev(pop, torch.int32)
            ref = gpga.ga_score(labels, C, form=gpga.FORM_GATHER)
            out = torch.full((P,), np.nan, dtype=torch.float64, device="cuda")
            gpga.ga_score_noalloc(labels, C, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert_L_close(got, orc.loglik_batch(pop, Ch), f"noalloc vs oracle N={N}")
            assert_L_close(got, ref.cpu().numpy(), f"noalloc vs ga_score N={N}")
    # sizes beyond the fixed scratch are refused with a clear error
    big = torch.zeros((2, 1025), dtype=torch.int32, device="cuda")
    Cbig = torch.eye(1025, dtype=torch.float64, device="cuda")
    L = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(gpga.GpgaError) as e:
        gpga.ga_score_noalloc(big, Cbig, L)
    assert e.value.code == gpga.ERR_ARG and "1024" in str(e.value)


def test_noalloc_bad_label_then_clean_call(orc):
    import torch
    from paper_1403_4099_gb300 import gpga
    p = synth.n100()
    Ch = orc.pearson(p.R)
    C = dev(Ch)
    rng = np.random.default_rng(7)
    pop = synth.random_labels(rng, 64, 100)
    bad = pop.copy()
    bad[5, 17] = 100  # outside [0, N)
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(gpga.GpgaError) as e:
        gpga.ga_score_noalloc(dev(bad, torch.int32), C, out)
    assert e.value.code == gpga.ERR_ARG
    got = out.cpu().numpy()
    assert np.isnan(got[5]) and np.isfinite(np.delete(got, 5)).all()
    # the next clean call starts from cleared flags and an empty error message
    gpga.ga_score_noalloc(dev(pop, torch.int32), C, out)
    torch.cuda.synchronize()
    assert gpga.lib().gpga_last_error() == b""
    assert_L_close(out.cpu().numpy(), orc.loglik_batch(pop, Ch), "clean call after a refused one")
