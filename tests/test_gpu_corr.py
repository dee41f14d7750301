"""GPU Pearson prelude (cluster_corr) against the FP64 oracle."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu

C_TOL = 1e-6


@pytest.fixture(scope="module")
def g():
    from paper_1403_4099_gb300 import build, gpga
    build.build()
    return gpga


def _corr(g, R):
    import torch
    C = g.cluster_corr(dev(R))
    torch.cuda.synchronize()
    return C.cpu().numpy()


@pytest.mark.parametrize("which", ["small16", "n100", "n500"])
def test_matches_oracle(g, orc, which):
    p = getattr(synth, which)()
    C = _corr(g, p.R)
    ref = orc.pearson(p.R)
    err = np.abs(C - ref).max()
    print(which, "max |dC|", err)
    assert err <= C_TOL
    assert np.all(np.diag(C) == 1.0) and np.array_equal(C, C.T)


@pytest.mark.parametrize("T,N", [(37, 2), (100, 63), (64, 65), (500, 130), (17, 200)])
def test_ragged(g, orc, T, N):
    rng = np.random.default_rng(T * 1000 + N)
    R = rng.standard_normal((T, N)) * rng.uniform(0.5, 2, N) + rng.uniform(-3, 3, N)
    assert np.abs(_corr(g, R) - orc.pearson(R)).max() <= C_TOL


def test_degenerate_and_bad_args(g):
    import torch
    rng = np.random.default_rng(5)
    R = rng.standard_normal((50, 8))
    R[:, 3] = 1.5
    with pytest.raises(g.GpgaError) as e:
        g.cluster_corr(dev(R))
    assert e.value.code == g.ERR_DEGENERATE
    R = rng.standard_normal((50, 8))
    R[10, 2] = np.nan
    with pytest.raises(g.GpgaError) as e:
        g.cluster_corr(dev(R))
    assert e.value.code == g.ERR_DEGENERATE
    with pytest.raises(g.GpgaError) as e:
        g.cluster_corr(dev(rng.standard_normal((1, 8))))
    assert e.value.code == g.ERR_ARG
    torch.cuda.synchronize()
