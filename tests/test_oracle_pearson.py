"""Pins of the oracle's Pearson prelude (Eq. 7) against numpy and closed forms."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth


def test_matches_numpy_corrcoef(orc):
    rng = np.random.default_rng(1)
    for T, N in [(500, 16), (37, 9), (2000, 60)]:
        R = rng.standard_normal((T, N)) * rng.uniform(0.1, 10, N) + rng.uniform(-5, 5, N)
        C = orc.pearson(R)
        np.testing.assert_allclose(C, np.corrcoef(R, rowvar=False), rtol=0, atol=1e-14)


def test_planted_workload_matches_numpy(orc):
    p = synth.n100()
    C = orc.pearson(p.R)
    np.testing.assert_allclose(C, np.corrcoef(p.R, rowvar=False), rtol=0, atol=1e-14)


def test_orthogonal_centred_columns_give_identity(orc):
    rng = np.random.default_rng(2)
    X = rng.standard_normal((200, 12))
    X -= X.mean(axis=0)
    Q, _ = np.linalg.qr(X)  # columns span the centred space, orthonormal
    C = orc.pearson(Q * rng.uniform(0.5, 3.0, 12) + 7.0)
    np.testing.assert_allclose(C, np.eye(12), atol=1e-13)


def test_affine_copies_are_plus_minus_one(orc):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(300)
    R = np.stack([x, 2.5 * x + 4.0, -0.3 * x + 1.0, rng.standard_normal(300)], axis=1)
    C = orc.pearson(R)
    assert abs(C[0, 1] - 1.0) < 1e-15 and abs(C[0, 2] + 1.0) < 1e-15 and abs(C[1, 2] + 1.0) < 1e-15


def test_structure_diag_symmetric_psd_bounded(orc):
    p = synth.small16()
    C = orc.pearson(p.R)
    assert np.all(np.diag(C) == 1.0)
    assert np.array_equal(C, C.T)
    assert np.abs(C).max() <= 1.0
    assert np.linalg.eigvalsh(C).min() >= -1e-12


def test_degenerate_inputs(orc):
    rng = np.random.default_rng(4)
    R = rng.standard_normal((50, 5))
    R2 = R.copy(); R2[:, 3] = 2.0
    assert orc.pearson_status(R2) == -4
    R3 = R.copy(); R3[7, 1] = np.nan
    assert orc.pearson_status(R3) == -4
    R4 = R.copy(); R4[7, 1] = np.inf
    assert orc.pearson_status(R4) == -4
    assert orc.pearson_status(R[:1]) == -1
    with pytest.raises(RuntimeError):
        orc.pearson(R2)
