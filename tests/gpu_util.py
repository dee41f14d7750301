"""Helpers shared by the GPU tests: device tensors, the likelihood tolerance."""
import numpy as np


def tol(L):
    """Per-individual likelihood bar: |dL| <= 1e-4 + 1e-6 |L|."""
    return 1e-4 + 1e-6 * np.abs(L)


def dev(x, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def assert_L_close(got, ref, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    bad = err > tol(ref)
    assert not bad.any(), (f"{what}: {bad.sum()} of {len(ref)} outside 1e-4+1e-6|L|; "
                           f"max err {err.max():.3e} at {int(err.argmax())}")
    return float(err.max())
