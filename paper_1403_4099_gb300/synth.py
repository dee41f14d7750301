"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only -- none of the method's arithmetic (no
correlation, no likelihood, no GA operator). Both the oracle-side tests and the
GPU path draw their inputs from here.

The returns follow the one-factor-per-cluster model of Eq. 2 (Noh's model, as
used by Giada and Marsili): series i of cluster s is

    r_i(t) = beta m(t) + sqrt(1 - beta^2) [ sqrt(g_s) eta_s(t) + sqrt(1 - g_s) eps_i(t) ]

with a market mode m (loading beta, 0 for none), cluster factors eta_s and
idiosyncratic noise eps_i, all iid N(0, 1). g_s here is the within-cluster
correlation of the non-market part, i.e. Eq. 2's g_s squared. Noise series are
singleton clusters: beta m + sqrt(1 - beta^2) eps_i. Columns are shuffled so that
clusters are not contiguous. Pearson correlation is invariant to per-column
affine maps, so no standardisation is applied here.

Seeds: base 14034099; workload c, replicate r uses 14034099 + 1000 c + r, PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 14034099


def seed_for(config: int, replicate: int = 0) -> int:
    return BASE_SEED + 1000 * int(config) + int(replicate)


@dataclass
class Planted:
    R: np.ndarray        # T x N float64 returns, row-major
    truth: np.ndarray    # N int32 planted labels; each noise series its own label
    sizes: list          # planted cluster sizes (noise excluded)
    g: np.ndarray        # per-cluster g_s


def dirichlet_sizes(rng: np.random.Generator, total: int, k: int, min_size: int = 2) -> list:
    """k sizes summing to `total` from total * Dirichlet(1), largest-remainder
    rounding, redrawn until every size is >= min_size."""
    if k * min_size > total:
        raise ValueError("too many clusters for the series available")
    while True:
        x = rng.dirichlet(np.ones(k)) * total
        base = np.floor(x).astype(np.int64)
        rem = int(total - base.sum())
        order = np.argsort(-(x - base), kind="stable")
        base[order[:rem]] += 1
        if base.min() >= min_size:
            return [int(v) for v in base]


def planted_returns(rng: np.random.Generator, T: int, sizes, g, n_noise: int = 0,
                    beta: float = 0.0, shuffle: bool = True) -> Planted:
    sizes = [int(s) for s in sizes]
    g = np.broadcast_to(np.asarray(g, np.float64), (len(sizes),)).copy()
    N = sum(sizes) + int(n_noise)
    labels = np.concatenate([np.full(s, k, np.int64) for k, s in enumerate(sizes)]
                            + [len(sizes) + np.arange(n_noise)])
    perm = rng.permutation(N) if shuffle else np.arange(N)
    labels = labels[perm]
    m = rng.standard_normal(T)
    eta = rng.standard_normal((T, len(sizes)))
    eps = rng.standard_normal((T, N))
    R = np.empty((T, N), np.float64)
    side = np.sqrt(1.0 - beta * beta)
    for i in range(N):
        s = labels[i]
        if s < len(sizes):
            part = np.sqrt(g[s]) * eta[:, s] + np.sqrt(1.0 - g[s]) * eps[:, i]
        else:
            part = eps[:, i]
        R[:, i] = beta * m + side * part
    # canonical truth labels (first occurrence order) so that comparisons are easy
    _, first = np.unique(labels, return_index=True)
    order = np.argsort(first)
    remap = np.empty(labels.max() + 1, np.int64)
    remap[np.unique(labels)[order]] = np.arange(order.shape[0])
    truth = remap[labels].astype(np.int32)
    return Planted(np.ascontiguousarray(R), truth, sizes, g)


# --- the workloads -------------------------------------------------------------

def small16(replicate: int = 0) -> Planted:
    """N=16, T=500, three planted clusters 6/5/5, g=0.5, no market, no noise."""
    rng = np.random.default_rng(seed_for(1, replicate))
    return planted_returns(rng, 500, [6, 5, 5], 0.5)


def small10(replicate: int = 0) -> Planted:
    """N=10 for the exhaustive check: 4/3/3, g=0.5, T=500."""
    rng = np.random.default_rng(seed_for(1, 100 + replicate))
    return planted_returns(rng, 500, [4, 3, 3], 0.5)


def wishart10(replicate: int) -> np.ndarray:
    """A T=20 x N=10 iid Gaussian returns matrix (its Pearson C is a random
    Wishart-type correlation matrix) for the brute-force comparison."""
    rng = np.random.default_rng(seed_for(1, 200 + replicate))
    return rng.standard_normal((20, 10))


def market_clusters(config: int, N: int, T: int, k: int, glo: float, ghi: float,
                    noise_frac: float = 0.1, beta: float = 0.3, replicate: int = 0) -> Planted:
    """Market mode (loading beta) + k planted clusters with Dirichlet(1) sizes
    (each >= 2) over the non-noise series, g_s ~ U[glo, ghi], noise_frac * N
    singleton noise series."""
    rng = np.random.default_rng(seed_for(config, replicate))
    n_noise = int(round(noise_frac * N))
    sizes = dirichlet_sizes(rng, N - n_noise, k)
    g = rng.uniform(glo, ghi, size=k)
    return planted_returns(rng, T, sizes, g, n_noise=n_noise, beta=beta)


def n100(replicate: int = 0) -> Planted:
    """N=100, T=2000, market 0.3, 8 clusters g~U[0.2,0.8], 10 noise series."""
    return market_clusters(2, 100, 2000, 8, 0.2, 0.8, replicate=replicate)


def n500(replicate: int = 0) -> Planted:
    """N=500, T=5000, market 0.3, 20 clusters g~U[0.1,0.9], 50 noise series."""
    return market_clusters(3, 500, 5000, 20, 0.1, 0.9, replicate=replicate)


def serving_request(N: int, replicate: int) -> Planted:
    """A request of the serving stream: T = 4N, clusters as in the N=100 recipe
    scaled (k = max(2, round(8 N / 100)) clusters, g~U[0.2,0.8], 10% noise)."""
    k = max(2, int(round(8 * N / 100)))
    k = min(k, max(1, (N - int(round(0.1 * N))) // 2))
    return market_clusters(5, N, 4 * N, k, 0.2, 0.8, replicate=replicate)


def random_labels(rng: np.random.Generator, P: int, N: int, K: int | None = None) -> np.ndarray:
    """P x N int32 labels uniform in [0, K) (K = N by default)."""
    return rng.integers(0, N if K is None else K, size=(P, N), dtype=np.int64).astype(np.int32)


def perturbed_population(rng: np.random.Generator, truth: np.ndarray, P: int, flip: float) -> np.ndarray:
    """P copies of `truth` with a fraction `flip` of genes replaced by uniform
    labels in [0, N): the shape of a late, converged population."""
    N = truth.shape[0]
    pop = np.tile(np.asarray(truth, np.int32), (P, 1))
    mask = rng.random((P, N)) < flip
    pop[mask] = rng.integers(0, N, size=int(mask.sum()), dtype=np.int64).astype(np.int32)
    return pop


@dataclass
class Intraday:
    R: np.ndarray          # T x N float64 one-minute returns
    truth_before: np.ndarray  # N int32 labels of the first regime (noise: singletons)
    truth_after: np.ndarray   # N int32 labels of the second regime
    switch: int            # first minute of the second regime


def intraday(N: int = 400, windows: int = 256, W: int = 390, stride: int = 30,
             k_before: int = 12, k_after: int = 9, replicate: int = 0) -> Intraday:
    """An intraday series of W + (windows - 1) stride one-minute returns over N
    stocks whose planted structure switches at the midpoint: k_before clusters
    before, a fresh draw of k_after clusters after (g ~ U[0.2, 0.8], market
    loading 0.3, 10% singleton noise series in each regime)."""
    rng = np.random.default_rng(seed_for(4, replicate))
    T = W + (windows - 1) * stride
    sw = T // 2
    n_noise = int(round(0.1 * N))
    parts = []
    truths = []
    for k, T_part in ((k_before, sw), (k_after, T - sw)):
        sizes = dirichlet_sizes(rng, N - n_noise, k)
        g = rng.uniform(0.2, 0.8, size=k)
        pl = planted_returns(rng, T_part, sizes, g, n_noise=n_noise, beta=0.3)
        parts.append(pl.R)
        truths.append(pl.truth)
    return Intraday(np.ascontiguousarray(np.vstack(parts)), truths[0], truths[1], sw)


def window_subsets(N: int, windows: int, nmin: int = 20, nmax: int | None = None,
                   replicate: int = 0) -> list:
    """Per window a sorted random column subset of size N_k ~ U{nmin..nmax}."""
    rng = np.random.default_rng(seed_for(4, 500 + replicate))
    nmax = N if nmax is None else nmax
    out = []
    for _ in range(windows):
        n = int(rng.integers(nmin, nmax + 1))
        out.append(np.sort(rng.choice(N, size=n, replace=False)).astype(np.int32))
    return out


# --- paper-shaped workloads (Sec. 4: a 40-stock training set with 4 planted
# clusters; an 18-stock test stream, ~1800 bars per window, 1760 windows) ----

def paper_training(replicate: int = 0, T: int = 1800, g: float = 0.5) -> Planted:
    """40 simulated stocks in 4 disjoint planted clusters of 10 (no market mode,
    no noise series); T and g are ours (the paper states neither)."""
    rng = np.random.default_rng(seed_for(6, replicate))
    return planted_returns(rng, T, [10, 10, 10, 10], g)


@dataclass
class Stream:
    R: np.ndarray       # (W + windows - 1) x N returns
    truth: np.ndarray   # N planted labels
    W: int              # bars per window
    windows: int        # window k covers bars [k, k + W)


def paper_stream(N: int = 18, W: int = 1800, windows: int = 1760, replicate: int = 0) -> Stream:
    """An 18-stock series of W + windows - 1 bars with 3 planted clusters of 6
    (g ~ U[0.2, 0.8], market loading 0.3): the shape of the paper's test set,
    1760 windows of about 1800 three-minute bars, each window one step later."""
    rng = np.random.default_rng(seed_for(6, 100 + replicate))
    k = 3
    g = rng.uniform(0.2, 0.8, size=k)
    pl = planted_returns(rng, W + windows - 1, [N // k] * k, g, beta=0.3)
    return Stream(pl.R, pl.truth, W, windows)
