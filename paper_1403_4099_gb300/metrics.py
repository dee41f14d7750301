"""Recovery measurement: adjusted Rand index (Hubert & Arabie, 1985) between a
found configuration and the planted one, from the pair-counting form:
    ARI = (sum C(n_ij,2) - E) / (1/2 (sum C(a_i,2) + sum C(b_j,2)) - E),
    E   = sum C(a_i,2) sum C(b_j,2) / C(n,2),
with the contingency counts n_ij and margins a_i, b_j. Evaluation only: not part
of the method."""
from __future__ import annotations

import numpy as np


def ari(a, b) -> float:
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    n = a.shape[0]
    if n < 2:
        return 1.0
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    table = np.zeros((ai.max() + 1, bi.max() + 1), np.int64)
    np.add.at(table, (ai, bi), 1)
    pairs = lambda x: (x * (x - 1) // 2).sum()
    idx = float(pairs(table))
    sa = float(pairs(table.sum(axis=1)))
    sb = float(pairs(table.sum(axis=0)))
    total = n * (n - 1) / 2.0
    expected = sa * sb / total
    top = 0.5 * (sa + sb)
    if top == expected:
        return 1.0
    return (idx - expected) / (top - expected)
