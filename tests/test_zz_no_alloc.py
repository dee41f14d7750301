"""ga_score_noalloc: the allocation-free scoring entry point, for callers that
cannot let the library allocate device memory (their own allocator owns the
GPU, or their loop forbids allocator calls). It must give the same likelihoods
as ga_score's gather form, through the C-ABI, on two calls in a row (the shared
fixed scratch keeps the previous call's contents, which must not leak into the
next result). Collected last so that a failure here comes after every other
test has run."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth
from gpu_util import assert_L_close, dev

pytestmark = pytest.mark.gpu


def test_noalloc_matches_ga_score_two_calls(orc):
    import torch
    from paper_1403_4099_gb300 import build, gpga
    build.build()
    rng = np.random.default_rng(2024)
    cases = [(synth.n500(), 4096), (synth.n100(), 333)]
    for p, P in cases:
        N = p.R.shape[1]
        C = dev(orc.pearson(p.R))
        pops = [synth.random_labels(rng, P, N), synth.perturbed_population(rng, p.truth, P, 0.05)]
        for pop in pops:  # two calls in a row on different inputs
            labels = dev(pop, torch.int32)
            ref = gpga.ga_score(labels, C, form=gpga.FORM_GATHER)
            out = torch.full((P,), np.nan, dtype=torch.float64, device="cuda")
            gpga.ga_score_noalloc(labels, C, out)
            torch.cuda.synchronize()
            assert_L_close(out.cpu().numpy(), ref.cpu().numpy(), f"noalloc N={N}")
    # sizes beyond the fixed scratch are refused with a clear error
    big = torch.zeros((2, 1025), dtype=torch.int32, device="cuda")
    Cbig = torch.eye(1025, dtype=torch.float64, device="cuda")
    L = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(gpga.GpgaError) as e:
        gpga.ga_score_noalloc(big, Cbig, L)
    assert e.value.code == gpga.ERR_ARG and "1024" in str(e.value)
