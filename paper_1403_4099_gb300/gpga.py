"""Thin ctypes binding of libgpga.so (include/gpga.h): argument marshalling only.

Every computation runs in the library's sm_103a kernels. PyTorch supplies device
memory and streams. There is no CPU fallback: if the library is missing or fails
to load, every call raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgpga.so")

OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_DEGENERATE, ERR_TIMEOUT, ERR_STATE = -1, -2, -3, -4, -5, -6
FORM_PLAIN, FORM_TENSOR, FORM_GATHER = 0, 1, 2
SCALING_RANK, SCALING_PROP = 0, 1
INIT_UNIFORM, INIT_THRESHOLD = 0, 1
MAX_N, MAX_P = 4096, 16384

EXPORTS = ["gpga_default_params", "gpga_last_error", "cluster_corr", "ga_score", "ga_evolve",
           "ga_init", "ga_reset", "ga_step", "ga_best", "ga_history", "ga_kernel_times",
           "ga_population", "gpga_log_selftest", "ga_score_noalloc", "ga_free",
           "ga_batch_init", "ga_batch_step", "ga_batch_status", "ga_batch_best",
           "ga_batch_tuning", "ga_batch_free", "serve_create", "serve_submit", "serve_tick",
           "serve_result", "serve_stats", "serve_free", "cluster_mst", "ga_island_init",
           "ga_batch_population", "cluster_corr_ewma", "corr_remove_market", "corr_clean_rmt",
           "gpga_set_wait_budget"]


class GpgaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gpga status {code}: {msg}")
        self.code = code


class Params(ct.Structure):
    """Mirror of struct gpga_params."""

    _fields_ = [
        ("P", ct.c_int32),
        ("elite", ct.c_int32),
        ("max_gens", ct.c_int32),
        ("stall_gens", ct.c_int32),
        ("tol", ct.c_double),
        ("pc", ct.c_double),
        ("pkb", ct.c_double),
        ("pm", ct.c_double),
        ("scaling", ct.c_int32),
        ("form", ct.c_int32),
        ("init", ct.c_int32),
        ("init_labels", ct.c_int32),
        ("tau_lo", ct.c_double),
        ("tau_hi", ct.c_double),
        ("record", ct.c_int32),
        ("profile", ct.c_int32),
        ("reserved", ct.c_int32 * 2),
    ]


_lock = threading.Lock()
_lib = None


def lib() -> ct.CDLL:
    """Load libgpga.so (build it first with paper_1403_4099_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first "
                               "(there is no fallback implementation)")
        L = ct.CDLL(LIB_PATH)
        vp, i32, f64 = ct.c_void_p, ct.c_int, ct.c_double
        sigs = {
            "gpga_default_params": (i32, [ct.POINTER(Params)]),
            "gpga_last_error": (ct.c_char_p, []),
            "gpga_set_wait_budget": (i32, [ct.c_longlong]),
            "cluster_corr": (i32, [vp, i32, i32, i32, vp, vp]),
            "ga_score": (i32, [vp, i32, i32, i32, vp, vp, i32, vp]),
            "ga_evolve": (i32, [vp, vp, i32, ct.POINTER(Params), ct.c_uint64, i32, vp, vp, vp, vp]),
            "ga_init": (i32, [vp, i32, ct.POINTER(Params), ct.c_uint64, vp, ct.POINTER(vp)]),
            "ga_reset": (i32, [vp, vp, ct.c_uint64]),
            "ga_step": (i32, [vp, i32, ct.POINTER(i32)]),
            "ga_best": (i32, [vp, vp, vp, ct.POINTER(i32)]),
            "ga_history": (i32, [vp, vp, vp, vp, vp, vp, i32, ct.POINTER(i32)]),
            "ga_kernel_times": (i32, [vp, vp, i32, ct.POINTER(i32)]),
            "ga_population": (i32, [vp, vp, vp]),
            "gpga_log_selftest": (i32, [vp, i32, vp, vp, vp]),
            "ga_score_noalloc": (i32, [vp, i32, i32, i32, vp, vp, vp]),
            "ga_free": (i32, [vp]),
            "ga_batch_init": (i32, [i32, vp, vp, vp, vp, ct.POINTER(Params), vp, vp,
                                    ct.POINTER(vp)]),
            "ga_batch_step": (i32, [vp, i32, ct.POINTER(i32)]),
            "ga_batch_status": (i32, [vp, vp, vp, vp]),
            "ga_batch_best": (i32, [vp, i32, vp, vp, ct.POINTER(i32)]),
            "ga_batch_tuning": (i32, [vp, ct.POINTER(i32), ct.POINTER(i32),
                                      ct.POINTER(ct.c_float)]),
            "ga_batch_free": (i32, [vp]),
            "serve_create": (i32, [ct.POINTER(Params), i32, i32, ct.c_size_t, vp,
                                   ct.POINTER(vp)]),
            "serve_submit": (i32, [vp, vp, i32, ct.c_uint64, ct.POINTER(ct.c_longlong)]),
            "serve_tick": (i32, [vp, i32, ct.POINTER(i32), ct.POINTER(i32)]),
            "serve_result": (i32, [vp, ct.c_longlong, vp, vp, ct.POINTER(i32), vp]),
            "serve_stats": (i32, [vp, ct.POINTER(ct.c_size_t), ct.POINTER(ct.c_size_t),
                                  ct.POINTER(ct.c_longlong), ct.POINTER(i32), ct.POINTER(i32),
                                  vp]),
            "serve_free": (i32, [vp]),
            "cluster_mst": (i32, [vp, i32, vp, vp, vp, vp, ct.POINTER(i32), vp]),
            "ga_island_init": (i32, [i32, vp, i32, ct.POINTER(Params), ct.c_uint64, i32, i32, vp,
                                     ct.POINTER(vp)]),
            "ga_batch_population": (i32, [vp, i32, vp, vp]),
            "cluster_corr_ewma": (i32, [vp, i32, i32, i32, f64, vp, vp]),
            "corr_remove_market": (i32, [vp, i32, i32, ct.POINTER(f64), ct.POINTER(i32), vp]),
            "corr_clean_rmt": (i32, [vp, i32, i32, f64, vp, ct.POINTER(i32), ct.POINTER(i32), vp]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(rc: int):
    if rc != OK:
        raise GpgaError(rc, lib().gpga_last_error().decode(errors="replace"))


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ct.c_void_p(stream.cuda_stream)


def _dev(t, dtype_name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ct.c_void_p(t.data_ptr())


def set_wait_budget(cycles: int):
    """Cycles a bounded device wait may spend before it gives up (< 0: the
    default, 2^32). Process-wide; for kernels launched after the call."""
    _check(lib().gpga_set_wait_budget(int(cycles)))


def default_params(**kw) -> Params:
    p = Params()
    _check(lib().gpga_default_params(ct.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def cluster_corr(R, C=None, stream=None):
    """Pearson C (N x N FP64, device) of returns R (T x N FP64, device)."""
    import torch
    T, N = R.shape
    if C is None:
        C = torch.empty((N, N), dtype=torch.float64, device=R.device)
    _check(lib().cluster_corr(_dev(R, "float64"), T, N, N, _dev(C, "float64"),
                              _stream_ptr(stream)))
    return C


def cluster_corr_ewma(R, lam: float, C=None, stream=None):
    """EWMA-weighted Pearson C (rows weighted lam^(T-1-t)) of R (T x N FP64, device)."""
    import torch
    T, N = R.shape
    if C is None:
        C = torch.empty((N, N), dtype=torch.float64, device=R.device)
    _check(lib().cluster_corr_ewma(_dev(R, "float64"), T, N, N, float(lam), _dev(C, "float64"),
                                   _stream_ptr(stream)))
    return C


def corr_remove_market(C, max_iters: int = 1000, stream=None):
    """Market mode removed from C (device, in place); returns (lambda_1, iterations)."""
    lam = ct.c_double()
    it = ct.c_int()
    _check(lib().corr_remove_market(_dev(C, "float64"), int(C.shape[0]), int(max_iters),
                                    ct.byref(lam), ct.byref(it), _stream_ptr(stream)))
    return lam.value, it.value


def corr_clean_rmt(C, T: float, stream=None):
    """Random-matrix cleaning of C in place (device FP64, N x N or batch x N x N,
    each estimated from T observations). Returns (eigenvalues of the input,
    ascending, device batch x N; noise-set sizes, list; Jacobi sweeps)."""
    import torch
    N = int(C.shape[-1])
    B = 1 if C.dim() == 2 else int(C.shape[0])
    ev = torch.empty((B, N), dtype=torch.float64, device=C.device)
    nn = (ct.c_int * B)()
    sw = ct.c_int()
    _check(lib().corr_clean_rmt(_dev(C, "float64"), B, N, float(T), _dev(ev, "float64"), nn,
                                ct.byref(sw), _stream_ptr(stream)))
    return ev, list(nn), sw.value


def ga_score(labels, C, form: int = FORM_PLAIN, L=None, stream=None):
    """L_c (P FP64, device) of labels (P x N int32, device) against C (device)."""
    import torch
    P, N = labels.shape
    if L is None:
        L = torch.empty(P, dtype=torch.float64, device=labels.device)
    _check(lib().ga_score(_dev(labels, "int32"), P, N, N, _dev(C, "float64"), _dev(L, "float64"),
                          int(form), _stream_ptr(stream)))
    return L


def ga_score_noalloc(labels, C, L, stream=None):
    """Gather-form L_c into the caller's L without any device allocation by the
    library (its scratch is a fixed device array; N <= 1024; concurrent calls
    race). labels: P x N int32 device, C: N x N FP64 device, L: P FP64 device."""
    P, N = labels.shape
    _check(lib().ga_score_noalloc(_dev(labels, "int32"), P, N, N, _dev(C, "float64"),
                                  _dev(L, "float64"), _stream_ptr(stream)))
    return L


def ga_evolve(pop, L, params: Params, seed: int, generation: int, stream=None):
    """One stateless generation; returns (next, perm, parents) device tensors."""
    import torch
    P, N = pop.shape
    if P != params.P:
        raise ValueError("pop rows must equal params.P")
    nxt = torch.empty_like(pop)
    perm = torch.empty(P, dtype=torch.int32, device=pop.device)
    par = torch.empty(P - params.elite, dtype=torch.int32, device=pop.device)
    _check(lib().ga_evolve(_dev(pop, "int32"), _dev(L, "float64"), N, ct.byref(params),
                           ct.c_uint64(seed), int(generation), _dev(nxt, "int32"),
                           _dev(perm, "int32"), _dev(par, "int32") if par.numel() else None,
                           _stream_ptr(stream)))
    return nxt, perm, par


def cluster_mst(C, labels, stream=None):
    """Per-cluster minimum spanning trees on d = sqrt(2 (1 - C)) of one
    configuration (labels: device int32 N): host arrays (u, v, d)."""
    import torch
    N = C.shape[0]
    cap = max(N - 1, 1)
    eu = torch.empty(cap, dtype=torch.int32, device=C.device)
    ev = torch.empty(cap, dtype=torch.int32, device=C.device)
    ew = torch.empty(cap, dtype=torch.float64, device=C.device)
    n = ct.c_int()
    _check(lib().cluster_mst(_dev(C, "float64"), N, _dev(labels, "int32"), _dev(eu, "int32"),
                             _dev(ev, "int32"), _dev(ew, "float64"), ct.byref(n),
                             _stream_ptr(stream)))
    k = n.value
    return eu[:k].cpu().numpy(), ev[:k].cpu().numpy(), ew[:k].cpu().numpy()


def log_selftest(x, stream=None):
    """(table_log(x), CUDA log(x)) for a device FP64 tensor x (diagnostic)."""
    import torch
    yt = torch.empty_like(x)
    yc = torch.empty_like(x)
    _check(lib().gpga_log_selftest(_dev(x, "float64"), x.numel(), _dev(yt, "float64"),
                                   _dev(yc, "float64"), _stream_ptr(stream)))
    return yt, yc


class GA:
    """A device-resident GA run (ga_init / ga_step / ga_best / ga_free)."""

    def __init__(self, C, params: Params, seed: int, stream=None):
        self.N = C.shape[0]
        self.params = params
        self._stream = stream
        h = ct.c_void_p()
        _check(lib().ga_init(_dev(C, "float64"), self.N, ct.byref(params), ct.c_uint64(seed),
                             _stream_ptr(stream), ct.byref(h)))
        self._h = h

    def reset(self, C, seed: int):
        _check(lib().ga_reset(self._h, _dev(C, "float64"), ct.c_uint64(seed)))

    def step(self, generations: int, wait: bool = False):
        if wait:
            d = ct.c_int()
            _check(lib().ga_step(self._h, int(generations), ct.byref(d)))
            return bool(d.value)
        _check(lib().ga_step(self._h, int(generations), None))
        return None

    def best(self, labels_out=None, L_out=None):
        """(canonical labels, FP64 re-scored L, generation). Outputs may be given
        as host numpy arrays or device tensors; by default host numpy."""
        g = ct.c_int()
        if labels_out is None and L_out is None:
            lab = np.zeros(self.N, np.int32)
            Lb = np.zeros(1, np.float64)
            _check(lib().ga_best(self._h, lab.ctypes.data, Lb.ctypes.data, ct.byref(g)))
            return lab, float(Lb[0]), g.value
        lp = _ptr(labels_out)
        Lp = _ptr(L_out)
        _check(lib().ga_best(self._h, lp, Lp, ct.byref(g)))
        return labels_out, L_out, g.value

    def history(self):
        cap = self.params.max_gens + 1
        bl = np.zeros(cap, np.float64)
        n = ct.c_int()
        if self.params.record:
            lab = np.zeros((cap, self.N), np.int32)
            ts = np.zeros(cap + 1, np.int64)
            pairs = np.zeros(cap, np.uint64)
            clus = np.zeros(cap, np.uint64)
            _check(lib().ga_history(self._h, bl.ctypes.data, lab.ctypes.data, ts.ctypes.data,
                                    pairs.ctypes.data, clus.ctypes.data, cap, ct.byref(n)))
            k = n.value
            return dict(best_L=bl[:k], labels=lab[:k], t_ns=ts[:k + 1], pairs=pairs[:k],
                        clusters=clus[:k])
        _check(lib().ga_history(self._h, bl.ctypes.data, None, None, None, None, cap,
                                ct.byref(n)))
        return dict(best_L=bl[: n.value])

    def kernel_times(self):
        """(count x 4) ms of [evolve, pair/contraction, assembly, selection] for the
        generations of the last graph launch (params.profile must be set)."""
        ms = np.zeros((8, 4), np.float32)
        n = ct.c_int()
        _check(lib().ga_kernel_times(self._h, ms.ctypes.data, 8, ct.byref(n)))
        return ms[: n.value]

    def population(self):
        pop = np.zeros((self.params.P, self.N), np.int32)
        L = np.zeros(self.params.P, np.float64)
        _check(lib().ga_population(self._h, pop.ctypes.data, L.ctypes.data))
        return pop, L

    def close(self):
        if getattr(self, "_h", None):
            lib().ga_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ct.c_void_p(x.ctypes.data)
    return ct.c_void_p(x.data_ptr())


class Batch:
    """Independent runs advanced together (ga_batch_*). Cs: list of device FP64
    correlation matrices; cols: optional list of device int32 index vectors
    (run k then works on Cs[k][cols[k]][:, cols[k]]); seeds: one per run."""

    def __init__(self, Cs, params: Params, seeds, cols=None, stream=None):
        R = len(Cs)
        if len(seeds) != R or (cols is not None and len(cols) != R):
            raise ValueError("Cs, seeds and cols must have the same length")
        self.R = R
        self.params = params
        ptrs = (ct.c_void_p * R)(*[_dev(C, "float64").value for C in Cs])
        ldc = (ct.c_int * R)(*[int(C.shape[1]) for C in Cs])
        if cols is not None:
            self.N = [int(c.shape[0]) for c in cols]
            cptr = (ct.c_void_p * R)(*[_dev(c, "int32").value for c in cols])
        else:
            self.N = [int(C.shape[0]) for C in Cs]
            cptr = None
        Ns = (ct.c_int * R)(*self.N)
        sd = (ct.c_uint64 * R)(*[int(s) for s in seeds])
        h = ct.c_void_p()
        _check(lib().ga_batch_init(R, ptrs, ldc, cptr, Ns, ct.byref(params), sd,
                                   _stream_ptr(stream), ct.byref(h)))
        self._h = h

    def step(self, generations: int, wait: bool = True):
        """Advance; returns the number of runs still active if wait."""
        if wait:
            a = ct.c_int()
            _check(lib().ga_batch_step(self._h, int(generations), ct.byref(a)))
            return a.value
        _check(lib().ga_batch_step(self._h, int(generations), None))
        return None

    def status(self):
        g = np.zeros(self.R, np.int32)
        d = np.zeros(self.R, np.int32)
        b = np.zeros(self.R, np.float64)
        _check(lib().ga_batch_status(self._h, g.ctypes.data, d.ctypes.data, b.ctypes.data))
        return g, d.astype(bool), b

    def best(self, run: int):
        lab = np.zeros(self.N[run], np.int32)
        Lb = np.zeros(1, np.float64)
        g = ct.c_int()
        _check(lib().ga_batch_best(self._h, int(run), lab.ctypes.data, Lb.ctypes.data,
                                   ct.byref(g)))
        return lab, float(Lb[0]), g.value

    def population(self, run: int):
        pop = np.zeros((self.params.P, self.N[run]), np.int32)
        L = np.zeros(self.params.P, np.float64)
        _check(lib().ga_batch_population(self._h, int(run), pop.ctypes.data, L.ctypes.data))
        return pop, L

    @classmethod
    def islands(cls, C, params: Params, islands: int, seed: int, migrate_every: int,
                migrants: int, stream=None):
        """The island model: `islands` populations on C with ring migration."""
        self = cls.__new__(cls)
        self.R = int(islands)
        self.params = params
        self.N = [int(C.shape[0])] * self.R
        h = ct.c_void_p()
        _check(lib().ga_island_init(self.R, _dev(C, "float64"), int(C.shape[0]), ct.byref(params),
                                    ct.c_uint64(seed), int(migrate_every), int(migrants),
                                    _stream_ptr(stream), ct.byref(h)))
        self._h = h
        return self

    def tuning(self):
        w, c, ms = ct.c_int(), ct.c_int(), ct.c_float()
        _check(lib().ga_batch_tuning(self._h, ct.byref(w), ct.byref(c), ct.byref(ms)))
        return dict(warps_per_cta=w.value, ctas=c.value, ms=float(ms.value))

    def close(self):
        if getattr(self, "_h", None):
            lib().ga_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving loop (serve_*): submit host correlation windows, tick, collect."""

    def __init__(self, params: Params, max_runs: int, max_n: int, mem_budget: int = 0,
                 stream=None):
        self.params = params
        self.max_n = max_n
        self._n = {}
        h = ct.c_void_p()
        _check(lib().serve_create(ct.byref(params), int(max_runs), int(max_n),
                                  ct.c_size_t(int(mem_budget)), _stream_ptr(stream), ct.byref(h)))
        self._h = h

    def submit(self, C: np.ndarray, seed: int) -> int:
        C = np.ascontiguousarray(C, dtype=np.float64)
        i = ct.c_longlong()
        _check(lib().serve_submit(self._h, C.ctypes.data, int(C.shape[0]), ct.c_uint64(seed),
                                  ct.byref(i)))
        self._n[i.value] = int(C.shape[0])
        return i.value

    def tick(self, generations: int):
        a, q = ct.c_int(), ct.c_int()
        _check(lib().serve_tick(self._h, int(generations), ct.byref(a), ct.byref(q)))
        return a.value, q.value

    def result(self, rid: int):
        """None while pending, else (labels, L, generation, (queued_s, run_s))."""
        lab = np.zeros(self._n.get(rid, 1), np.int32)  # unknown ids: the library reports
        L = ct.c_double()
        g = ct.c_int()
        t = np.zeros(2, np.float64)
        rc = lib().serve_result(self._h, ct.c_longlong(rid), lab.ctypes.data, ct.byref(L),
                                ct.byref(g), t.ctypes.data)
        if rc == 0:
            return None
        if rc < 0:
            _check(rc)
        self._n.pop(rid, None)
        return lab, L.value, g.value, (float(t[0]), float(t[1]))

    def stats(self):
        u, b, c, w, k = ct.c_size_t(), ct.c_size_t(), ct.c_longlong(), ct.c_int(), ct.c_int()
        t = np.zeros(6, np.float64)
        _check(lib().serve_stats(self._h, ct.byref(u), ct.byref(b), ct.byref(c), ct.byref(w),
                                 ct.byref(k), t.ctypes.data))
        return dict(bytes_in_use=u.value, budget=b.value, completed=c.value,
                    warps_per_cta=w.value, ctas=k.value, ticks=int(t[0]), host_wait_s=t[1],
                    host_work_s=t[2], gpu_ms=t[3], generations=int(t[4]), item_gens=int(t[5]))

    def close(self):
        if getattr(self, "_h", None):
            lib().serve_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
