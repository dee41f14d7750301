"""Python face of the FP64 CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The GPU library never
imports, links or runs anything here, and nothing here imports the GPU package.

Each wrapper names the passage of arXiv:1403.4099 it follows (see oracle.c).
Parity unpinned: none -- every function is pinned by a test in
``tests/test_oracle_*.py`` (known-answer vectors, library routines, closed forms,
brute force, counting properties).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STREAM_INIT, STREAM_SUS, STREAM_XOVER, STREAM_MUT = 0, 1, 2, 3
SCALING_RANK, SCALING_PROP = 0, 1


class GaParams(ct.Structure):
    """Mirror of the oracle's own parameter struct (not the GPU library's)."""

    _fields_ = [
        ("P", ct.c_int32),
        ("N", ct.c_int32),
        ("elite", ct.c_int32),
        ("max_gens", ct.c_int32),
        ("stall_gens", ct.c_int32),
        ("scaling", ct.c_int32),
        ("init_labels", ct.c_int32),
        ("reserved", ct.c_int32),
        ("tol", ct.c_double),
        ("pc", ct.c_double),
        ("pkb", ct.c_double),
        ("pm", ct.c_double),
    ]


def params(P, N, elite=2, max_gens=200, stall_gens=50, tol=1e-5, pc=0.9, pkb=0.9, pm=0.01,
           scaling=SCALING_RANK, init_labels=0) -> GaParams:
    """Table 3 defaults except P_m, read per gene (0.01)."""
    return GaParams(P, N, elite, max_gens, stall_gens, scaling, init_labels, 0,
                    float(tol), float(pc), float(pkb), float(pm))


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall"]
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        # a host without libgomp still gets a (single-threaded) oracle
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ct.CDLL(build())
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        sig = {
            "orc_philox4x32_10": (None, [u32p, u32p, u32p]),
            "orc_threshold": (ct.c_uint64, [ct.c_double]),
            "orc_pearson": (ct.c_int, [f64p, ct.c_int, ct.c_int, ct.c_int, f64p]),
            "orc_cluster_sums": (ct.c_int, [i32p, ct.c_int, f64p, i32p, f64p, f64p]),
            "orc_loglik": (ct.c_int, [i32p, ct.c_int, f64p, ct.POINTER(ct.c_double),
                                      ct.POINTER(ct.c_int32)]),
            "orc_loglik_batch": (ct.c_int, [i32p, ct.c_int, ct.c_int, ct.c_int, f64p, f64p,
                                            ct.c_int]),
            "orc_max_threads": (ct.c_int, []),
            "orc_canonicalize": (ct.c_int, [i32p, ct.c_int, i32p]),
            "orc_ga_init": (ct.c_int, [ct.c_int, ct.c_int, ct.c_int, ct.c_uint64, i32p]),
            "orc_ga_rank": (ct.c_int, [f64p, ct.c_int, i32p]),
            "orc_prim_order": (ct.c_int, [f64p, ct.c_int, i32p]),
            "orc_ga_init_threshold": (ct.c_int, [f64p, ct.c_int, ct.c_int, ct.c_double,
                                                 ct.c_double, ct.c_uint64, i32p]),
            "orc_ga_weights": (ct.c_int, [f64p, i32p, ct.c_int, ct.c_int, u64p]),
            "orc_ga_sus": (ct.c_int, [u64p, ct.c_int, ct.c_int, ct.c_uint32, i32p]),
            "orc_ga_evolve": (ct.c_int, [i32p, f64p, ct.POINTER(GaParams), ct.c_uint64,
                                         ct.c_int32, i32p, ct.c_void_p, ct.c_void_p]),
            "orc_ga_terminated": (ct.c_int, [f64p, ct.c_int, ct.POINTER(GaParams)]),
            "orc_ga_run": (ct.c_int, [f64p, ct.POINTER(GaParams), ct.c_uint64, ct.c_int, i32p,
                                      ct.POINTER(ct.c_double), ct.POINTER(ct.c_int32), f64p,
                                      ct.c_void_p]),
            "orc_brute_force": (ct.c_int, [f64p, ct.c_int, i32p, ct.POINTER(ct.c_double),
                                           ct.POINTER(ct.c_int64)]),
            "orc_ari": (ct.c_double, [i32p, i32p, ct.c_int]),
            "orc_cluster_mst": (ct.c_int, [i32p, ct.c_int, f64p, i32p, i32p, f64p,
                                           ct.POINTER(ct.c_int32)]),
            "orc_island_migrate": (ct.c_int, [i32p, f64p, ct.c_int, ct.c_int, ct.c_int,
                                              ct.c_int]),
            "orc_pearson_ewma": (ct.c_int, [f64p, ct.c_int, ct.c_int, ct.c_int, ct.c_double,
                                            f64p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key."""
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def threshold(p: float) -> int:
    return int(_load().orc_threshold(float(p)))


def pearson(R) -> np.ndarray:
    """Eq. 7 on a T x N returns matrix."""
    R = _f64(R)
    T, N = R.shape
    C = np.zeros((N, N), np.float64)
    _check(_load().orc_pearson(R, T, N, N, C), "pearson")
    return C


def pearson_status(R) -> int:
    R = _f64(R)
    T, N = R.shape
    C = np.zeros((N, N), np.float64)
    return int(_load().orc_pearson(R, T, N, N, C))


def cluster_sums(s, C):
    """(n_s, c_s, d_s) for every label s in [0, N): Eq. 5, Eq. 6 and n_s^2 - c_s."""
    s = _i32(s)
    N = s.shape[0]
    n = np.zeros(N, np.int32)
    c = np.zeros(N, np.float64)
    d = np.zeros(N, np.float64)
    _check(_load().orc_cluster_sums(s, N, _f64(C), n, c, d), "cluster_sums")
    return n, c, d


def loglik(s, C, with_clamps: bool = False):
    """Eq. 8 for one configuration."""
    s = _i32(s)
    L = ct.c_double()
    k = ct.c_int32()
    _check(_load().orc_loglik(s, s.shape[0], _f64(C), ct.byref(L), ct.byref(k)), "loglik")
    return (L.value, k.value) if with_clamps else L.value


def loglik_batch(labels, C, nthreads: int = 0) -> np.ndarray:
    """Eq. 8 for a P x N population."""
    labels = _i32(labels)
    P, N = labels.shape
    L = np.zeros(P, np.float64)
    _check(_load().orc_loglik_batch(labels, P, N, N, _f64(C), L, int(nthreads)), "loglik_batch")
    return L


def canonicalize(s) -> np.ndarray:
    s = _i32(s)
    out = np.zeros_like(s)
    _check(_load().orc_canonicalize(s, s.shape[0], out), "canonicalize")
    return out


def ga_init(P, N, seed, K0=None) -> np.ndarray:
    pop = np.zeros((P, N), np.int32)
    _check(_load().orc_ga_init(P, N, N if K0 is None else K0, seed, pop), "ga_init")
    return pop


def prim_order(C) -> np.ndarray:
    C = _f64(C)
    order = np.zeros(C.shape[0], np.int32)
    _check(_load().orc_prim_order(C, C.shape[0], order), "prim_order")
    return order


def ga_init_threshold(C, P, seed, tau_lo=0.05, tau_hi=0.6) -> np.ndarray:
    """Correlation-threshold initial population (components of C > tau_p)."""
    C = _f64(C)
    N = C.shape[0]
    pop = np.zeros((P, N), np.int32)
    _check(_load().orc_ga_init_threshold(C, P, N, float(tau_lo), float(tau_hi), seed, pop),
           "ga_init_threshold")
    return pop


def ga_rank(L) -> np.ndarray:
    L = _f64(L)
    perm = np.zeros(L.shape[0], np.int32)
    _check(_load().orc_ga_rank(L, L.shape[0], perm), "ga_rank")
    return perm


def ga_weights(L, perm, scaling=SCALING_RANK) -> np.ndarray:
    L = _f64(L)
    w = np.zeros(L.shape[0], np.uint64)
    _check(_load().orc_ga_weights(L, _i32(perm), L.shape[0], scaling, w), "ga_weights")
    return w


def ga_sus(w, M, u) -> np.ndarray:
    w = np.ascontiguousarray(w, np.uint64)
    sel = np.zeros(M, np.int32)
    _check(_load().orc_ga_sus(w, w.shape[0], M, int(u), sel), "ga_sus")
    return sel


def ga_evolve(pop, L, prm: GaParams, seed, g):
    """One generation of operators; returns (next, perm, parents)."""
    pop = _i32(pop)
    P, N = pop.shape
    nxt = np.zeros_like(pop)
    perm = np.zeros(P, np.int32)
    par = np.zeros(P - prm.elite, np.int32)
    _check(_load().orc_ga_evolve(pop, _f64(L), ct.byref(prm), seed, g, nxt,
                                 perm.ctypes.data, par.ctypes.data), "ga_evolve")
    return nxt, perm, par


def ga_terminated(best_hist, g, prm: GaParams) -> bool:
    return bool(_load().orc_ga_terminated(_f64(best_hist), g, ct.byref(prm)))


def ga_run(C, prm: GaParams, seed, nthreads: int = 0, ring: bool = False):
    """A whole run of Algorithm 1; returns dict(best, L, gens, hist[, ring])."""
    C = _f64(C)
    N = prm.N
    best = np.zeros(N, np.int32)
    L = ct.c_double()
    g = ct.c_int32()
    hist = np.zeros(prm.max_gens + 1, np.float64)
    ringbuf = np.zeros((prm.max_gens + 1, N), np.int32) if ring else None
    _check(_load().orc_ga_run(C, ct.byref(prm), seed, nthreads, best, ct.byref(L), ct.byref(g),
                              hist, ringbuf.ctypes.data if ring else None), "ga_run")
    out = dict(best=best, L=L.value, gens=g.value, hist=hist[: g.value + 1])
    if ring:
        out["ring"] = ringbuf[: g.value + 1]
    return out


def brute_force(C):
    """Exhaustive max of Eq. 8 over set partitions (N <= 12)."""
    C = _f64(C)
    N = C.shape[0]
    best = np.zeros(N, np.int32)
    L = ct.c_double()
    cnt = ct.c_int64()
    _check(_load().orc_brute_force(C, N, best, ct.byref(L), ct.byref(cnt)), "brute_force")
    return best, L.value, cnt.value


def ari(a, b) -> float:
    a = _i32(a)
    return float(_load().orc_ari(a, _i32(b), a.shape[0]))


def cluster_mst(s, C):
    """Per-cluster minimum spanning trees on d = sqrt(2 (1 - C)) (Kruskal):
    (u, v, d) arrays, clusters in first-occurrence order, u < v."""
    s = _i32(s)
    N = s.shape[0]
    eu = np.zeros(max(N, 1), np.int32)
    ev = np.zeros(max(N, 1), np.int32)
    ew = np.zeros(max(N, 1), np.float64)
    n = ct.c_int32()
    _check(_load().orc_cluster_mst(s, N, _f64(C), eu, ev, ew, ct.byref(n)), "cluster_mst")
    k = n.value
    return eu[:k], ev[:k], ew[:k]


def island_migrate(pops, Ls, m):
    """Ring migration of the island model: island k's first m members (and
    fitness) replace the last m of island k + 1. pops: K x P x N int32, Ls:
    K x P FP64; returns new arrays."""
    pops = np.array(pops, dtype=np.int32, order="C", copy=True)
    Ls = np.array(Ls, dtype=np.float64, order="C", copy=True)
    K, P, N = pops.shape
    _check(_load().orc_island_migrate(pops.reshape(-1), Ls.reshape(-1), K, P, N, int(m)),
           "island_migrate")
    return pops, Ls


def pearson_ewma(R, lam: float) -> np.ndarray:
    """EWMA-weighted Pearson (rows weighted lam^(T-1-t)); lam = 1 is Eq. 7."""
    R = _f64(R)
    T, N = R.shape
    C = np.zeros((N, N), np.float64)
    _check(_load().orc_pearson_ewma(R, T, N, N, float(lam), C), "pearson_ewma")
    return C


def remove_market(C):
    """Market-mode removal: the largest eigenpair (lambda_1, v) of C (LAPACK's
    symmetric eigensolver as the step), C' = C - lambda_1 v v^T, renormalised
    to unit diagonal, C''_ij = C'_ij / sqrt(C'_ii C'_jj), clamped to [-1, 1].
    Returns (C'', lambda_1)."""
    C = _f64(C)
    w, V = np.linalg.eigh(C)
    lam, v = float(w[-1]), V[:, -1]
    Cp = C - lam * np.outer(v, v)
    d = np.diag(Cp).copy()
    if not np.all(d > 0):
        raise RuntimeError("oracle remove_market: a diagonal entry is not positive after the removal")
    out = Cp / np.sqrt(np.outer(d, d))
    np.fill_diagonal(out, 1.0)
    return np.clip(out, -1.0, 1.0), lam


def wishart_range(N, T):
    """Marchenko-Pastur support of the eigenvalues of a sample correlation
    matrix of N independent series over T observations, q = N / T:
    [(1 - sqrt q)^2, (1 + sqrt q)^2]."""
    q = N / float(T)
    r = np.sqrt(q)
    return (1.0 - r) ** 2, (1.0 + r) ** 2


def rmt_clip(C, T):
    """The trace-preserving eigenvalue clipping of Sec. 4.2 before the
    renormalisation: C = sum_k lambda_k v_k v_k^T (LAPACK's symmetric
    eigensolver as the step); the eigenvalues inside the Wishart range are the
    noise set and are replaced by their mean m, so
    C' = m I + sum_{k kept} (lambda_k - m) v_k v_k^T (same trace). With an
    empty noise set C' = C. Returns (C', eigenvalues ascending, noise mask, m)."""
    C = _f64(C)
    N = C.shape[0]
    lo, hi = wishart_range(N, T)
    w, V = np.linalg.eigh(C)
    noise = (w >= lo) & (w <= hi)
    if not noise.any():
        return C.copy(), w, noise, float("nan")
    m = float(w[noise].mean())
    keep = ~noise
    Vk = V[:, keep]
    Cp = (Vk * (w[keep] - m)) @ Vk.T
    Cp = 0.5 * (Cp + Cp.T) + m * np.eye(N)  # symmetric as defined (the product rounds unevenly)
    return Cp, w, noise, m


def clean_rmt(C, T):
    """Random-matrix cleaning of a correlation matrix estimated from T
    observations (Sec. 4.2): rmt_clip, then renormalised to unit diagonal,
    C''_ij = C'_ij / sqrt(C'_ii C'_jj), clamped to [-1, 1]; C unchanged when
    no eigenvalue lies in the Wishart range. Returns (C'', eigenvalues
    ascending, size of the noise set)."""
    Cp, w, noise, _ = rmt_clip(C, T)
    if not noise.any():
        return Cp, w, 0
    d = np.diag(Cp).copy()
    if not np.all(d > 0):
        raise RuntimeError("oracle clean_rmt: a diagonal entry is not positive after the cleaning")
    out = Cp / np.sqrt(np.outer(d, d))
    np.fill_diagonal(out, 1.0)
    return np.clip(out, -1.0, 1.0), w, int(noise.sum())
