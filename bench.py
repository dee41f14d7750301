#!/usr/bin/env python
"""Benchmark of the PGA hot path on the N=500, T=5000, P=4096 planted-cluster
workload (20 clusters, market mode 0.3, 10% noise series).

A step is one whole PGA job on one window: Pearson prelude (cluster_corr) from
device-resident returns, initial population + scoring (ga_reset), and G
generations of score / rank / select / crossover / mutate (ga_step), all on the
device. Metric: fitness evaluations per second, P (G + 1) per step. Also
reported: generations/s, ms to recover the planted clusters (ARI >= 0.99),
per-stage kernel times (CUDA events on the launching stream, live in the timed
region), the roofline of the dominant kernel, the end-to-end number through host
buffers, and the FP64 CPU oracle timed on the host cores.

Multi-GPU (torchrun): every rank runs its own independent jobs (replicas, weak
scaling); only a barrier and max-over-ranks timing cross ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, T, P = 500, 5000, 4096
ELITE = 10
WORKLOAD = "planted_n500_t5000_p4096"
METRIC = "fitness evals/s (N=500, P=4096; step = Pearson prelude + init + G generations)"
SMS = 152
ALU_LANES = 128
GRAPH_GENS = 8  # generations per captured graph in ga_step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpga", choices=["gpga", "reference"])
    ap.add_argument("--form", default="gather", choices=["plain", "tensor", "gather"])
    ap.add_argument("--gens", type=int, default=100, help="generations per step")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-recover", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="leave out the batched and serving summaries from the headline line")
    ap.add_argument("--workload", default="planted",
                    choices=["planted", "batched", "serving", "paper", "preprocess", "islands"],
                    help="planted: the N=500 headline; batched: 256 sliding intraday windows "
                         "in one fleet; serving: Poisson request stream; paper: the paper's "
                         "shapes (40-stock training set, 18-stock 1760-window stream, Table 3 "
                         "parameters, a P_m x P_c sweep); preprocess: the steps around the path "
                         "(EWMA correlation, market-mode removal, random-matrix cleaning, "
                         "per-cluster trees); islands: the island model against one population")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1403_4099_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_value(kernel: str, src_hash: str, key: str):
    """A per-launch counter (`key`) from the committed ncu summary
    profiles/<kernel>_traffic.txt, if it was taken on the current kernel
    source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != src_hash:
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def profiled_traffic(kernel: str, src_hash: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)."""
    return profiled_value(kernel, src_hash, "dram_bytes_per_launch")


def issue_fraction(warp_insts, launch_ms, sm_mhz):
    """Warp instructions of one launch over the issue slots of its duration:
    SMs x 4 schedulers x one instruction per cycle at the sampled SM clock."""
    if not warp_insts or not launch_ms or not sm_mhz:
        return None
    slots = SMS * 4 * sm_mhz * 1e6 * launch_ms / 1e3
    return warp_insts / slots


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(R, gens: int):
    """Time the FP64 oracle on one window: Pearson + initial population + `gens`
    generations (score + operators), on all host threads. Returns
    (seconds, evaluations, seconds_pearson, seconds_ga)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    C = oracle.pearson(R)
    t1 = time.perf_counter()
    prm = oracle.params(P, N, elite=ELITE, max_gens=gens, stall_gens=50, tol=-1.0, pm=0.01)
    oracle.ga_run(C, prm, seed=12345, nthreads=0)
    t2 = time.perf_counter()
    return t2 - t0, P * (gens + 1), t1 - t0, t2 - t1


def run_reference(args, ranks):
    from paper_1403_4099_gb300 import synth
    import oracle
    if ranks.rank != 0:
        return
    planted = synth.n500()
    gens = 2
    for _ in range(args.warmup):
        oracle_sample(planted.R, gens)
    secs, evals = 0.0, 0
    for _ in range(args.steps):
        s, e, _, _ = oracle_sample(planted.R, gens)
        secs += s
        evals += e
    value = evals / secs
    cores = oracle.max_threads()
    sample = (f"per step: FP64 oracle Pearson (T={T}, N={N}) + initial population + {gens} "
              f"generations at P={P}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "T": T, "P": P, "generations_per_step": gens},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
GATHER_PROFILE = ("gather_generation_n500_p4096", ("gather.cu", "gpga_internal.cuh"))


def gather_roofline(launch_ms, pk, pk_kind, pairs_per_gen, sm_mhz=None):
    """Fused generation kernel (gather form): algorithmic bytes per launch =
    per child 2 parents read + child written (2 B labels, N genes) + one 4-byte
    D entry per same-cluster pair + 8 B of fitness; pairs measured on the
    device for the timed generations. The working set is L2-resident, so the
    bound that binds is instruction issue: `issue` gives the warp instructions
    of one launch (committed ncu capture of the same source) over the issue
    slots of the live launch time at the sampled SM clock."""
    bytes_per_launch = P * (3 * 2 * N + 8) + 4.0 * pairs_per_gen
    t = launch_ms / 1e3
    gbs = bytes_per_launch / t / 1e9
    peak = pk["hbm_gbs"]
    kern, srcs = GATHER_PROFILE
    h = source_hash(*srcs)
    insts = profiled_value(kern, h, "warp_instructions_per_launch")
    frac_issue = issue_fraction(insts, launch_ms, sm_mhz)
    return {"bound": "hbm", "kernel": "gather_generation", "achieved": gbs, "peak": peak,
            "unit": "GB/s", "frac": gbs / peak,
            "traffic": profiled_traffic(kern, h),
            "peak_source": f"hbm_gbs ({pk_kind})", "algorithmic_bytes_per_launch": bytes_per_launch,
            "same_cluster_pairs_per_launch": pairs_per_gen, "launch_ms": launch_ms,
            "issue": None if frac_issue is None else {
                "bound": "issue", "frac": frac_issue,
                "warp_instructions_per_launch": insts,
                "warp_instructions_per_individual": insts / P,
                "sm_mhz": sm_mhz,
                "peak_source": f"{SMS} SMs x 4 schedulers x 1 warp instruction per cycle at "
                               "the median SM clock sampled in the timed region"}}

# arithmetic type of the path per form (what it computes in) and its detail
DTYPE = {
    "gather": ("int64", "pair sums of D = 1 - C as int32 fixed point 2^-30 added in int64 "
                        "(exact); Eq. 8 assembled in integer fixed point (Q62 table log, "
                        "result in Q40); Pearson prelude: integer column statistics, the "
                        "centred returns split three ways into BF16 on tcgen05 with FP32 "
                        "accumulation and exact fixed-point partial sums; integer GA "
                        "operators"),
    "plain": ("f32", "FP32 pair accumulation of D = 1 - C, fixed-point per-cluster sums, "
                     "integer Eq. 8 assembly; integer GA operators"),
    "tensor": ("bf16", "one-hot x D split BF16 hi + lo on tcgen05, FP32 accumulation in TMEM, "
                       "fixed-point per-cluster sums, integer Eq. 8 assembly; integer GA "
                       "operators"),
}


def launches_per_step(form: str, gens: int) -> int:
    corr = 7                      # colsum x2, colfinal x2, normalise, gram, gram_final
    score = {"plain": 2, "tensor": 4, "gather": 1}[form]
    start = 3 + score + 1         # state, prep_d, init, score, select (the rank and SUS
                                  # tables are built once per handle, before the timed steps)
    per_gen = (1 if form == "gather" else 1 + score) + 1  # (fused | evolve + score), select
    return corr + start + gens * per_gen


def run_gpu(args, ranks):
    import torch

    from paper_1403_4099_gb300 import gpga, metrics, runtime, synth

    torch.cuda.set_device(ranks.local)
    dev = torch.device("cuda", ranks.local)
    runtime.init_dist(ranks, "nccl")
    form = {"plain": gpga.FORM_PLAIN, "tensor": gpga.FORM_TENSOR, "gather": gpga.FORM_GATHER}[args.form]
    G = args.gens
    planted = synth.n500(replicate=ranks.rank)
    R_host = torch.from_numpy(planted.R).pin_memory()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    with torch.cuda.stream(stream):
        R = R_host.to(dev, non_blocking=True)
        C = torch.empty((N, N), dtype=torch.float64, device=dev)
        gpga.cluster_corr(R, C, stream)
        prm = gpga.default_params(P=P, elite=ELITE, max_gens=G, stall_gens=50, tol=-1.0,
                                  pm=0.01, form=form, record=1, profile=1)
        # stage breakdown: a separate, untimed run with events around every stage
        prm_all = gpga.default_params(P=P, elite=ELITE, max_gens=G, stall_gens=50, tol=-1.0,
                                      pm=0.01, form=form, profile=2)
        ga = gpga.GA(C, prm, seed=1, stream=stream)

        def one_step(k):
            gpga.cluster_corr(R, C, stream)
            ga.reset(C, 1000 + k)
            ga.step(G)

        for k in range(args.warmup):
            one_step(k)
        stream.synchronize()
        runtime.barrier(ranks)

        gpu = None
        try:
            props = torch.cuda.get_device_properties(dev)
            gpu = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(ranks.local)
        except Exception:
            gpu = str(ranks.local)
        sampler = runtime.ClockSampler(gpu)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        stage = []
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev0[k].record(stream)
            one_step(args.warmup + k)
            ev1[k].record(stream)
            stage.append(ga.kernel_times())
        stream.synchronize()
        wall = time.perf_counter() - wall0
        clocks = sampler.stop(busy_mhz_floor=600.0)
        step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        hist = ga.history()
        ga_all = gpga.GA(C, prm_all, seed=2, stream=stream)
        ga_all.step(G)
        stages_all = ga_all.kernel_times()
        ga_all.close()
        converged = run_converged(args, C, stream, form) if ranks.rank == 0 else None
    runtime.barrier(ranks)

    secs = sum(step_ms) / 1e3
    evals = P * (G + 1) * args.steps
    max_secs, total_evals = runtime.aggregate(ranks, secs, evals, device=dev)
    value = total_evals / max_secs
    gens_per_s = value / P

    names = {gpga.FORM_PLAIN: ["evolve", "pair_plain", "assemble", "select"],
             gpga.FORM_TENSOR: ["evolve", "tc_contract", "assemble", "select"],
             gpga.FORM_GATHER: ["gather_generation", "-", "-", "select"]}[form]
    # dominant kernel: events live in the timed region (only around that kernel)
    stage = np.concatenate(stage)
    main_col = 0 if form == gpga.FORM_GATHER else 1
    main_ms = float(stage[:, main_col].mean())
    # breakdown from the untimed all-stage run (each event adds ~2 us to its stage)
    kernel_ms = {n: float(v) for n, v in zip(names, stages_all.mean(axis=0)) if n != "-"}
    kernel_ms[names[main_col]] = main_ms
    dominant = max(kernel_ms, key=kernel_ms.get)

    pk, pk_kind = peaks()
    if form == gpga.FORM_PLAIN:
        # compare + predicated add per unordered gene pair (i < j) per individual
        ops = float(P) * N * (N - 1)
        t = main_ms / 1e3
        peak = SMS * ALU_LANES * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        traffic = profiled_traffic("pair_plain_n500_p4096",
                                   source_hash("score.cu", "gpga_internal.cuh"))
        roof = {"bound": "alu", "kernel": "pair_plain", "achieved": ops / t / 1e12, "peak": peak,
                "unit": "Tops/s", "frac": (ops / t / 1e12) / peak, "traffic": traffic,
                "peak_source": f"{SMS} SMs x {ALU_LANES} FP32/INT32 lanes x "
                               f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz ({pk_kind} max clock)",
                "algorithmic_ops_per_launch": ops, "launch_ms": main_ms}
    elif form == gpga.FORM_TENSOR:
        # issued tcgen05 work: column tiles of 128 clusters x row tiles of 256 x
        # K = Np, two MMAs (D_hi, D_lo) of 2 M N K FLOPs each
        Np = (N + 63) // 64 * 64
        NTt = min(256, Np)
        tg = G if G % GRAPH_GENS else G - GRAPH_GENS + 1  # the timed generation
        cols = float(hist["clusters"][tg]) if tg < len(hist["clusters"]) else 0.0
        n_ct = 2 * int(np.ceil(cols / 256.0))  # pairs of 128-column tiles per CTA
        flops = n_ct * int(np.ceil(Np / NTt)) * 2 * 2.0 * 128 * NTt * Np
        t = main_ms / 1e3
        peak = pk["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "kernel": "tc_mma (with column prep)", "achieved": flops / t / 1e12,
                "peak": peak, "unit": "TFLOP/s", "frac": flops / t / 1e12 / peak,
                "traffic": profiled_traffic("tc_mma_n500_p4096",
                                            source_hash("score_tc.cu", "gpga_internal.cuh")),
                "peak_source": f"bf16_tflops_sustained ({pk_kind})",
                "issued_mma_flops_per_launch": flops, "columns_per_launch": cols,
                "launch_ms": main_ms}
    elif form == gpga.FORM_GATHER:
        # the timed launch is the first generation of the step's last graph
        # launch (graphs of GRAPH_GENS generations, then single generations)
        tg = G if G % GRAPH_GENS else G - GRAPH_GENS + 1
        pairs = hist["pairs"]
        roof = gather_roofline(main_ms, pk, pk_kind, float(pairs[tg]) if tg < len(pairs) else 0.0,
                               (clocks or {}).get("sm_mhz"))
        roof["timed_generation"] = int(tg)
    else:
        roof = None  # filled by the tensor form

    # recovery within the timed step itself (first generation whose best
    # individual has ARI >= 0.99 vs the planted labels)
    rec = first_recovery(hist, planted.truth)
    ms_rec = {"within_timed_step": {"generations": G, **rec}}

    # end-to-end leg on every rank, aggregated like the device-timed value
    runtime.barrier(ranks)
    e2e = run_e2e(args, ranks, R_host, dev, form, G)
    e2e_secs, e2e_evals = runtime.aggregate(ranks, e2e.pop("seconds"), e2e.pop("evals"), device=dev)
    e2e["value"] = e2e_evals / e2e_secs
    e2e["ms_per_step"] = 1e3 * e2e_secs / args.e2e_steps
    e2e["h2d_bytes_per_step"] *= ranks.world
    e2e["d2h_bytes_per_step"] *= ranks.world
    out = {"e2e": e2e}
    if ranks.rank == 0:
        out["recover"] = None if args.no_recover else run_recover(args, ranks, planted, dev, form)
        if out["recover"]:
            ms_rec.update(out["recover"])

    # the batched workload (256 sliding windows in one fleet, one timed job) and
    # the serving stream (Poisson arrivals for --serve-seconds), carried in the
    # headline line so that one run records them too
    secondary = None
    if ranks.rank == 0 and ranks.world == 1 and not args.no_secondary:
        secondary = {}
        keep = {"batched": ("metric", "value", "unit", "ms_per_step", "evals_per_s",
                            "generations", "config", "ari_single_regime_windows"),
                "serving": ("metric", "value", "unit", "config", "latency_ms", "evals_per_s",
                            "generations_mean", "active_runs")}
        for name, fn in (("batched", run_batched), ("serving", run_serving)):
            try:
                sl = fn(argparse.Namespace(**{**vars(args), "steps": 10}), ranks, emit=False)
                secondary[name] = {k: sl[k] for k in keep[name]}
            except Exception as exc:  # reported, never hides the headline
                secondary[name] = {"error": repr(exc)[:300]}

    cpu = None
    if ranks.rank == 0 and ranks.world == 1 and not args.no_cpu_baseline:
        import oracle
        g_cpu = 3
        s, e, sp, sg = oracle_sample(planted.R, g_cpu)
        # extrapolate the GA part linearly to G generations
        s_full = sp + sg * (G + 1) / (g_cpu + 1)
        cpu = {"value": P * (G + 1) / s_full, "unit": "evals/s", "cores": oracle.max_threads(),
               "kind": "oracle",
               "sample": (f"FP64 oracle on this workload: Pearson once ({sp:.2f} s, 1 thread) + "
                          f"initial population + {g_cpu} generations ({sg:.2f} s, all threads), "
                          f"GA time extrapolated linearly to {G} generations")}

    if ranks.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ranks.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * max_secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.form][0], "dtype_detail": DTYPE[args.form][1],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "T": T, "P": P, "elite": ELITE,
                       "generations_per_step": G, "form": args.form, "init": "uniform",
                       "l2": "flushed between steps (256 MB memset outside the step events)"},
            "generations_per_s": gens_per_s,
            **({"non_singleton_clusters_per_individual": {
                "first_generation": float(hist["clusters"][0]) / P,
                "last_generation": float(hist["clusters"][-1]) / P}}
               if form == gpga.FORM_TENSOR else {}),
            "converged_regime": converged,
            "same_cluster_pairs_per_individual": {
                "first_generation": float(hist["pairs"][0]) / P,
                "last_generation": float(hist["pairs"][-1]) / P,
                "dense_pairs_per_individual": N * (N - 1) / 2},
            "ms_to_recover": ms_rec,
            "kernel_ms": kernel_ms, "dominant_kernel": dominant,
            "roofline": roof,
            "e2e": out.get("e2e"),
            "cpu_baseline": cpu,
            "secondary": secondary,
            "gpu_launches": launches_per_step(args.form, G) * args.steps,
            "clocks": clocks,
            "wall_s_timed_region": wall,
        }
        print(json.dumps(line), flush=True)
    runtime.barrier(ranks)


def run_converged(args, C, stream, form):
    """The same G generations from a converged start: the correlation-threshold
    initial population (components of C > tau, tau ~ U[0.05, 0.6)), whose
    configurations hold the planted clusters, so that every child has large
    clusters and the same-cluster pair gathers dominate. Only ga_step is
    timed (CUDA events on the run's stream, L2 flushed before each step)."""
    import torch

    from paper_1403_4099_gb300 import gpga
    G = args.gens
    prm = gpga.default_params(P=P, elite=ELITE, max_gens=G, stall_gens=50, tol=-1.0, pm=0.01,
                              form=form, init=gpga.INIT_THRESHOLD, record=1, profile=1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=C.device)
    ga = gpga.GA(C, prm, seed=11, stream=stream)
    ms, kern = [], []
    steps = max(3, args.steps // 4)
    for k in range(2 + steps):
        ga.reset(C, 500 + k)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ga.step(G)
        e1.record(stream)
        kt = ga.kernel_times()
        stream.synchronize()
        if k >= 2:
            ms.append(e0.elapsed_time(e1))
            kern.append(float(kt[:, 0 if form == gpga.FORM_GATHER else 1].mean()))
    h = ga.history()
    ga.close()
    t = float(np.mean(ms))
    return {"init": "threshold (tau ~ U[0.05, 0.6))", "generations": G, "steps": steps,
            "value": P * G / (t / 1e3), "unit": "evals/s", "ms_per_step": t,
            "dominant_kernel_ms": float(np.mean(kern)),
            "same_cluster_pairs_per_individual": {
                "first_generation": float(h["pairs"][1]) / P,
                "last_generation": float(h["pairs"][-1]) / P}}


def run_e2e(args, ranks, R_host, dev, form, G):
    """The same metric through the public API from pinned host returns to the
    host-side best configuration: H2D of R, prelude, init, G generations,
    FP64 re-score, D2H of the labels and L, every step. Returns this rank's
    seconds and evaluations over `e2e_steps` steps (one untimed step first)."""
    import torch

    from paper_1403_4099_gb300 import gpga
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        R = torch.empty(R_host.shape, dtype=torch.float64, device=dev)
        C = torch.empty((N, N), dtype=torch.float64, device=dev)
        R.copy_(R_host, non_blocking=True)
        gpga.cluster_corr(R, C, stream)
        prm = gpga.default_params(P=P, elite=ELITE, max_gens=G, tol=-1.0, pm=0.01, form=form)
        ga = gpga.GA(C, prm, seed=7, stream=stream)
        lab = np.zeros(N, np.int32)
        Lb = np.zeros(1, np.float64)
        times = []
        for k in range(args.e2e_steps + 1):
            stream.synchronize()
            t0 = time.perf_counter()
            R.copy_(R_host, non_blocking=True)
            gpga.cluster_corr(R, C, stream)
            ga.reset(C, 50 + k)
            ga.step(G)
            ga.best(lab, Lb)
            times.append(time.perf_counter() - t0)
        ga.close()
    t = float(np.sum(times[1:]))
    return {"unit": "evals/s", "seconds": t, "evals": float(P * (G + 1) * args.e2e_steps),
            "h2d_bytes_per_step": int(R_host.numel() * 8), "d2h_bytes_per_step": int(N * 4 + 8)}


RECOVER_CONFIGS = (
    # name, planted workload, P, E, generation cap, initial label range K0 (0: N),
    # mutation probability per gene
    ("small16_p64", "small16", 64, 2, 2000, 0, 0.01),
    ("n100_p1024", "n100", 1024, 10, 3000, 0, 0.01),
    ("n500_p4096", "n500", 4096, 10, 5000, 0, 0.01),
    # one mutation per child on average at N = 500 (P_m = 1/N)
    ("n500_p4096_pm002", "n500", 4096, 10, 3000, 0, 0.002),
    # the same GA from labels uniform in [0, round(sqrt(N))) instead of [0, N)
    # (the reading of "create initial population" allows a smaller label
    # range; sqrt(N) is a generic choice, not the planted cluster count)
    ("n100_p1024_k0_10", "n100", 1024, 10, 3000, 10, 0.01),
)
RECOVER_SEEDS = (101, 202, 303)


def planted_members(truth):
    """Mask of the genes that belong to a planted cluster (two or more members);
    the noise series are planted as singletons and have no cluster to recover."""
    t = np.asarray(truth)
    return np.bincount(t, minlength=t.max() + 1)[t] >= 2


def first_recovery(h, truth):
    """Recovery of the planted clusters along a run's records: the generation and
    device ms (from the start of ga_reset to the end of that generation) of the
    first best configuration whose ARI over the members of the planted clusters
    is >= 0.99 (None if none), with the best such ARI and its generation, and
    the ARI over all N genes (noise series included) at the same points. The
    noise series are left out of the criterion because the likelihood itself
    places them in clusters: on the n500 workload each of them raises L by
    joining one, so the likelihood's optimum is not the planted partition over
    all N (pinned by the oracle tests)."""
    from paper_1403_4099_gb300 import metrics
    labs = h["labels"]
    mem = planted_members(truth)
    ari_m = np.empty(len(labs))
    ari_all = np.empty(len(labs))
    prev, prev_m, prev_a = None, 0.0, 0.0
    for g, l in enumerate(labs):
        if prev is None or not np.array_equal(l, prev):  # the best changes rarely
            prev = l
            prev_m = metrics.ari(l[mem], truth[mem])
            prev_a = metrics.ari(l, truth)
        ari_m[g] = prev_m
        ari_all[g] = prev_a
    hit = np.flatnonzero(ari_m >= 0.99)
    g0 = int(hit[0]) if hit.size else None
    ms = None if g0 is None else float(h["t_ns"][1 + g0] - h["t_ns"][0]) / 1e6
    gb = int(ari_m.argmax())
    # the departures of the final best configuration from the planted clusters
    # (members only): planted clusters whose members share a found cluster with
    # members of another planted cluster, and planted clusters spread over
    # more than one found cluster
    fin, tm = np.asarray(labs[-1])[mem], np.asarray(truth)[mem]
    merged = {int(c) for f in np.unique(fin) for c in np.unique(tm[fin == f])
              if np.unique(tm[fin == f]).size > 1}
    split = sum(int(np.unique(fin[tm == c]).size > 1) for c in np.unique(tm))
    return {"generation": g0, "ms": ms, "best_ari_members": float(ari_m[gb]),
            "final_planted_clusters_merged": len(merged), "final_planted_clusters_split": split,
            "best_ari_members_generation": gb,
            "ari_all_genes_at_recovery": None if g0 is None else float(ari_all[g0]),
            "best_ari_all_genes": float(ari_all.max()),
            "best_L_final": float(h["best_L"][-1])}


def run_recover(args, ranks, planted, dev, form):
    """Recovery of the planted clusters by the GA itself (Algorithm 1 from the
    uniform initial population): for each workload and seed, device time from
    the start of ga_reset to the first generation whose best individual has
    ARI >= 0.99 against the planted partition over the members of the planted
    clusters (stall rule off, up to a cap of generations); the ARI over all N
    genes and the planted partition's own L are reported beside it. Also the correlation-threshold initialiser, reported apart:
    it is a single-linkage cut of C and recovers the partition before any GA
    operator runs (generation 0)."""
    import torch

    from paper_1403_4099_gb300 import gpga, metrics, synth
    stream = torch.cuda.Stream(device=dev)
    out = {"uniform_init": {}}
    with torch.cuda.stream(stream):
        for name, wl, Pw, Ew, cap, K0, pm in RECOVER_CONFIGS:
            pl = planted if wl == "n500" else getattr(synth, wl)()
            Rw = torch.from_numpy(pl.R).to(dev)
            Nw = pl.R.shape[1]
            Cw = torch.empty((Nw, Nw), dtype=torch.float64, device=dev)
            gpga.cluster_corr(Rw, Cw, stream)
            prm = gpga.default_params(P=Pw, elite=Ew, max_gens=cap, stall_gens=50, tol=-1.0,
                                      pm=pm, form=form, record=1, init_labels=K0)
            ga = gpga.GA(Cw, prm, seed=1, stream=stream)
            runs = []
            for sd in RECOVER_SEEDS:
                ga.reset(Cw, sd)
                ga.step(cap)
                h = ga.history()
                runs.append({"seed": sd, **first_recovery(h, pl.truth),
                             "ms_per_generation": float(h["t_ns"][-1] - h["t_ns"][0]) / 1e6 /
                                                  (len(h["t_ns"]) - 1)})
            ga.close()
            # the planted partition's own L (gather form on the device), beside
            # the best L the runs end with
            tl = torch.from_numpy(pl.truth.astype(np.int32)[None]).to(dev)
            L_pl = float(gpga.ga_score(tl, Cw, gpga.FORM_GATHER, stream=stream).cpu()[0])
            ok = [r["ms"] for r in runs if r["ms"] is not None]
            out["uniform_init"][name] = {
                "N": Nw, "P": Pw, "elite": Ew, "pm": pm, "generation_cap": cap,
                "initial_labels": K0 or Nw, "L_planted_partition": L_pl,
                "recovered": f"{len(ok)}/{len(runs)}",
                "median_ms": float(np.median(ok)) if ok else None,
                "runs": runs}
        # the single-linkage initialiser at the headline workload (not the GA)
        R = torch.from_numpy(planted.R).to(dev)
        C = torch.empty((N, N), dtype=torch.float64, device=dev)
        gpga.cluster_corr(R, C, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gpga.cluster_corr(R, C, stream)
        e1.record(stream)
        stream.synchronize()
        corr_ms = e0.elapsed_time(e1)
        prm = gpga.default_params(P=P, elite=ELITE, max_gens=200, tol=-1.0, pm=0.01, form=form,
                                  init=gpga.INIT_THRESHOLD, record=1)
        ga = gpga.GA(C, prm, seed=3, stream=stream)
        ga.step(50)
        ga.reset(C, 4)
        ga.step(50)
        h = ga.history()
        ga.close()
    rec = first_recovery(h, planted.truth)
    out["single_linkage_initialiser"] = {
        "what": "correlation-threshold initial population (components of C > tau_p, a "
                "single-linkage cut); recovers before any GA operator runs",
        **rec, "prelude_ms": corr_ms,
        "ms_with_prelude": None if rec["ms"] is None else rec["ms"] + corr_ms}
    return out


# ---------------------------------------------------------------------------
# Batched: 256 sliding windows (W=390, stride 30) of an N=400 intraday series
# whose planted structure switches at the midpoint; run k works on a random
# column subset of N_k ~ U{20..400}; P=1024; all runs in one fleet.
# ---------------------------------------------------------------------------
B_WINDOWS, B_W, B_STRIDE, B_N, B_P = 256, 390, 30, 400, 1024


def run_batched(args, ranks, emit=True):
    """Config 4: 256 sliding windows in one fleet. Prints its JSON line (emit)
    or returns it (as the secondary object of the headline line)."""
    import torch

    from paper_1403_4099_gb300 import gpga, metrics, runtime, synth
    torch.cuda.set_device(ranks.local)
    dev = torch.device("cuda", ranks.local)
    runtime.init_dist(ranks, "nccl")
    win = synth.intraday(B_N, B_WINDOWS, B_W, B_STRIDE, replicate=ranks.rank)
    subs = synth.window_subsets(B_N, B_WINDOWS, 20, B_N, replicate=ranks.rank)
    stream = torch.cuda.Stream(device=dev)
    prm = gpga.default_params(P=B_P, elite=10, max_gens=400, stall_gens=50, tol=1e-5, pm=0.01,
                              form=gpga.FORM_GATHER)
    with torch.cuda.stream(stream):
        R = torch.from_numpy(win.R).to(dev)
        cols = [torch.from_numpy(s).to(dev) for s in subs]
        Cs = [torch.empty((B_N, B_N), dtype=torch.float64, device=dev) for _ in range(B_WINDOWS)]
        seeds = [9000 + k for k in range(B_WINDOWS)]

        def job():
            for k in range(B_WINDOWS):
                gpga.cluster_corr(R[B_STRIDE * k: B_STRIDE * k + B_W], Cs[k], stream)
            b = gpga.Batch(Cs, prm, seeds, cols=cols, stream=stream)
            t_init = time.perf_counter()
            while b.step(16) > 0:
                pass
            return b, t_init

        b, _ = job()  # warm-up (builds, tunes, captures)
        b.close()
        stream.synchronize()
        runtime.barrier(ranks)
        times, gens_tot = [], []
        for _ in range(max(1, args.steps // 10)):
            t0 = time.perf_counter()
            b, t_init = job()
            stream.synchronize()
            t1 = time.perf_counter()
            g, done, best = b.status()
            times.append((t1 - t0, t_init - t0))
            gens_tot.append(g.copy())
            last = b
            if _ < max(1, args.steps // 10) - 1:
                b.close()
    secs = float(np.mean([t for t, _ in times]))
    g = gens_tot[-1]
    evals = float(B_P * np.sum(g + 1))
    max_secs, total_evals = runtime.aggregate(ranks, secs, evals, device=dev)
    tune = last.tuning()
    aris_b, aris_a = [], []
    for k in range(B_WINDOWS):
        lab, L, gg = last.best(k)
        lo, hi = B_STRIDE * k, B_STRIDE * k + B_W
        if hi <= win.switch:
            aris_b.append(metrics.ari(lab, win.truth_before[subs[k]]))
        elif lo >= win.switch:
            aris_a.append(metrics.ari(lab, win.truth_after[subs[k]]))
    last.close()
    if ranks.rank == 0:
        line = {"metric": "windows/s (256 sliding intraday windows, N_k in [20,400], P=1024, "
                          "each run to 400 generations or stall)",
                "value": B_WINDOWS * ranks.world / max_secs, "unit": "windows/s",
                "n_gpus": ranks.world, "steps": len(times), "warmup": 1,
                "ms_per_step": 1e3 * max_secs, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPE["gather"][0],
                "dtype_detail": DTYPE["gather"][1], "data": "synthetic",
                "config": {"workload": "intraday_n400_w390_s30_x256_p1024", "P": B_P,
                           "N_range": [20, B_N], "windows": B_WINDOWS, "form": "gather"},
                "evals_per_s": total_evals / max_secs,
                "generations": {"mean": float(np.mean(g)), "min": int(g.min()), "max": int(g.max())},
                "init_ms": 1e3 * float(np.mean([t for _, t in times])),
                "tuning": tune,
                "ari_single_regime_windows": {
                    "before_switch": {"n": len(aris_b), "mean": float(np.mean(aris_b)),
                                      "min": float(np.min(aris_b))},
                    "after_switch": {"n": len(aris_a), "mean": float(np.mean(aris_a)),
                                     "min": float(np.min(aris_a))}}}
        if not emit:
            return line
        print(json.dumps(line), flush=True)
    runtime.barrier(ranks)
    return None


# ---------------------------------------------------------------------------
# Serving: Poisson arrivals of correlation windows, N in {30, 100, 300, 1000}
# (T = 4N returns, planted clusters), P=2048, each run to 300 generations or
# stall (50, 1e-5); latency from arrival to the collected result.
# ---------------------------------------------------------------------------
S_NS, S_P, S_POOL = (30, 100, 300, 1000), 2048, 8


def run_serving(args, ranks, emit=True):
    """Config 5: a Poisson stream of correlation windows. Prints its JSON line
    (emit) or returns it (as a secondary object of the headline line)."""
    import torch

    from paper_1403_4099_gb300 import gpga, runtime, synth
    torch.cuda.set_device(ranks.local)
    dev = torch.device("cuda", ranks.local)
    runtime.init_dist(ranks, "nccl")
    rng = np.random.default_rng(synth.seed_for(5, 900 + ranks.rank))
    pool = {}
    for n in S_NS:
        pool[n] = []
        for r in range(S_POOL):
            pl = synth.serving_request(n, replicate=100 * ranks.rank + r)
            C = gpga.cluster_corr(torch.from_numpy(pl.R).to(dev))
            pool[n].append(C.cpu().numpy())
    torch.cuda.synchronize()
    prm = gpga.default_params(P=S_P, elite=10, max_gens=300, stall_gens=50, tol=1e-5, pm=0.01,
                              form=gpga.FORM_GATHER)
    dur, rate = args.serve_seconds, args.serve_rate
    arr = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * dur * 1.5) + 16))
    arr = arr[arr < dur]
    reqN = rng.choice(S_NS, size=arr.shape[0])
    reqP = rng.integers(0, S_POOL, size=arr.shape[0])
    stream = torch.cuda.Stream(device=dev)
    srv = gpga.Server(prm, max_runs=1024, max_n=max(S_NS), stream=stream)
    # warm-up request (tuning, graph capture)
    wid = srv.submit(pool[S_NS[-1]][0], 1)
    while srv.result(wid) is None:
        srv.tick(8)
    runtime.barrier(ranks)
    lat, qs, gens, active_hist = [], [], [], []
    pending = {}
    nxt = 0
    t0 = time.perf_counter()
    done_n = 0
    while done_n < arr.shape[0]:
        now = time.perf_counter() - t0
        while nxt < arr.shape[0] and arr[nxt] <= now:
            i = srv.submit(pool[int(reqN[nxt])][int(reqP[nxt])], 10_000 + nxt)
            pending[i] = nxt
            nxt += 1
        a, q = srv.tick(8)
        active_hist.append(a)
        tnow = time.perf_counter() - t0
        for i in list(pending):
            r = srv.result(i)
            if r is not None:
                k = pending.pop(i)
                lat.append(tnow - arr[k])
                qs.append(r[3][0])
                gens.append(r[2])
                done_n += 1
        if a == 0 and q == 0 and nxt < arr.shape[0]:
            time.sleep(max(0.0, min(0.001, arr[nxt] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat_ms = 1e3 * np.array(lat)
    n_done = len(lat)
    max_wall, total = runtime.aggregate(ranks, wall, float(n_done), device=dev)
    evals = float(S_P * np.sum(np.array(gens) + 1))
    if ranks.rank == 0:
        line = {"metric": "windows/s (Poisson stream, N in {30,100,300,1000}, P=2048, "
                          "<=300 generations or stall)",
                "value": total / max_wall, "unit": "windows/s", "n_gpus": ranks.world,
                "steps": 1, "warmup": 1, "ms_per_step": 1e3 * max_wall,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE["gather"][0], "dtype_detail": DTYPE["gather"][1],
                "data": "synthetic",
                "config": {"workload": "serving_poisson", "rate_per_s": rate, "seconds": dur,
                           "requests": int(arr.shape[0]), "P": S_P, "Ns": list(S_NS)},
                "latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                               "p99": float(np.percentile(lat_ms, 99)),
                               "max": float(lat_ms.max())},
                "queue_ms_mean": 1e3 * float(np.mean(qs)),
                "evals_per_s": evals / wall,
                "generations_mean": float(np.mean(gens)),
                "active_runs": {"mean": float(np.mean(active_hist)), "max": int(max(active_hist))},
                "launch_shape": {"warps_per_cta": st["warps_per_cta"], "ctas": st["ctas"]},
                "ticks": st["ticks"], "generations_per_tick": 8,
                "host_s": {"waiting_for_gpu": st["host_wait_s"], "tick_work": st["host_work_s"]},
                "gpu_generation_graphs_s": st["gpu_ms"] / 1e3,
                "individual_generations_per_gpu_s": (st["item_gens"] / (st["gpu_ms"] / 1e3)
                                                     if st["gpu_ms"] > 0 else None)}
        if not emit:
            return line
        print(json.dumps(line), flush=True)
    runtime.barrier(ranks)
    return None


# ---------------------------------------------------------------------------
# Paper-shaped workload (Sec. 4, Table 3): P = 1000, at most 400 generations,
# P_c = 0.9, P_kb = 0.9, P_m = 0.1 per gene, tolerance 1e-5 over 50 stall
# generations, 10 elites. (1) the 40-stock training set, (2) a P_m x P_c sweep
# on it (8 seeds each), (3) the 18-stock stream of 1760 windows of 1800 bars
# as one fleet.
# ---------------------------------------------------------------------------
def _table3(gpga, **kw):
    base = dict(P=1000, elite=10, max_gens=400, stall_gens=50, tol=1e-5, pc=0.9, pkb=0.9,
                pm=0.1, form=gpga.FORM_GATHER)
    base.update(kw)
    return gpga.default_params(**base)


def run_paper(args, ranks):
    import torch

    from paper_1403_4099_gb300 import gpga, metrics, runtime, synth
    torch.cuda.set_device(ranks.local)
    dev = torch.device("cuda", ranks.local)
    runtime.init_dist(ranks, "nccl")
    stream = torch.cuda.Stream(device=dev)
    out = {}
    with torch.cuda.stream(stream):
        # (1) training set, one run with the history recorded
        tr = synth.paper_training(replicate=ranks.rank)
        C = gpga.cluster_corr(torch.from_numpy(tr.R).to(dev), stream=stream)
        ga = gpga.GA(C, _table3(gpga, record=1), seed=21, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        while not ga.step(8, wait=True):
            pass
        e1.record(stream)
        stream.synchronize()
        h = ga.history()
        lab, L, g = ga.best()
        ga.close()
        ari = [metrics.ari(l, tr.truth) for l in h["labels"]]
        rec = next((k for k, a in enumerate(ari) if a >= 0.99), None)
        out["training_40"] = {"generations": int(g), "final_ari": float(metrics.ari(lab, tr.truth)),
                              "first_generation_ari_0.99": rec, "L": float(L),
                              "ms": float(e0.elapsed_time(e1))}
        # (2) sweep: 8 seeds per (P_m, P_c), each combination one batch
        sweep = []
        for pm in (0.01, 0.05, 0.1):
            for pc in (0.6, 0.9):
                b = gpga.Batch([C] * 8, _table3(gpga, pm=pm, pc=pc), [100 + k for k in range(8)],
                               stream=stream)
                while b.step(16) > 0:
                    pass
                gens, _, _ = b.status()
                aris = [metrics.ari(b.best(k)[0], tr.truth) for k in range(8)]
                b.close()
                sweep.append({"pm": pm, "pc": pc, "recovered": int(sum(a >= 0.99 for a in aris)),
                              "of": 8, "mean_ari": float(np.mean(aris)),
                              "mean_generations": float(np.mean(gens))})
        out["sweep_training_40"] = sweep
        # (3) the stream: 1760 windows as one fleet
        st = synth.paper_stream(replicate=ranks.rank)
        R = torch.from_numpy(st.R).to(dev)
        Cs = [torch.empty((18, 18), dtype=torch.float64, device=dev) for _ in range(st.windows)]
        runtime.barrier(ranks)
        stream.synchronize()
        t0 = time.perf_counter()
        for k in range(st.windows):
            gpga.cluster_corr(R[k:k + st.W], Cs[k], stream)
        b = gpga.Batch(Cs, _table3(gpga), [5000 + k for k in range(st.windows)], stream=stream)
        while b.step(16) > 0:
            pass
        stream.synchronize()
        secs = time.perf_counter() - t0
        gens, _, _ = b.status()
        sample = range(0, st.windows, 40)
        aris = [metrics.ari(b.best(k)[0], st.truth) for k in sample]
        b.close()
    max_secs, total = runtime.aggregate(ranks, secs, float(st.windows), device=dev)
    evals = float(1000 * np.sum(gens + 1))
    if ranks.rank == 0:
        line = {"metric": "windows/s (18-stock stream: 1760 windows of 1800 bars, Table 3 "
                          "parameters, each run to 400 generations or stall)",
                "value": total / max_secs, "unit": "windows/s", "n_gpus": ranks.world,
                "steps": 1, "warmup": 0, "ms_per_step": 1e3 * max_secs,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE["gather"][0], "dtype_detail": DTYPE["gather"][1],
                "data": "synthetic",
                "config": {"workload": "paper_stream_n18_w1800_x1760_p1000", "P": 1000,
                           "max_gens": 400, "pm": 0.1, "pc": 0.9, "pkb": 0.9, "elite": 10},
                "evals_per_s": evals / secs,
                "generations": {"mean": float(np.mean(gens)), "min": int(gens.min()),
                                "max": int(gens.max())},
                "stream_ari_sampled": {"n": len(aris), "mean": float(np.mean(aris)),
                                       "min": float(np.min(aris))},
                **out}
        print(json.dumps(line), flush=True)
    runtime.barrier(ranks)


# FP64 rate of a GB300 (nominal; no measured FP64 peak is available): the
# Jacobi rotations are plain FP64 multiply-adds
FP64_TFLOPS_NOMINAL = 1.25


def run_preprocess(args, ranks):
    """The pre-processing upstream of C through the library's public calls (each
    blocks until its stream is done, so host wall time is the call's time):
    EWMA correlation and market-mode removal at N = 500, random-matrix cleaning
    of one N = 500 matrix and of the 18-stock stream's 1760 windows as one
    batch; the FP64 oracle's cleaning timed on the host beside it."""
    import torch

    import oracle
    from paper_1403_4099_gb300 import gpga, runtime, synth
    torch.cuda.set_device(ranks.local)
    dev = torch.device("cuda", ranks.local)
    runtime.init_dist(ranks, "nccl")
    stream = torch.cuda.Stream(device=dev)

    def timed(fn, reps):
        fn()
        stream.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        stream.synchronize()
        return (time.perf_counter() - t0) / reps

    pl = synth.n500(replicate=ranks.rank)
    T = pl.R.shape[0]
    st = synth.paper_stream(replicate=ranks.rank)
    with torch.cuda.stream(stream):
        R = torch.from_numpy(pl.R).to(dev)
        C = gpga.cluster_corr(R, stream=stream)
        ewma_s = timed(lambda: gpga.cluster_corr_ewma(R, 0.98, stream=stream), max(3, args.steps // 4))
        mkt_s = timed(lambda: gpga.corr_remove_market(C.clone(), stream=stream), 3)
        rmt_one = lambda: gpga.corr_clean_rmt(C.clone(), T, stream=stream)  # noqa: E731
        rmt500_s = timed(rmt_one, 2)
        _, nn500, sw500 = rmt_one()
        Rs = torch.from_numpy(st.R).to(dev)
        Cs = torch.empty((st.windows, 18, 18), dtype=torch.float64, device=dev)
        for k in range(st.windows):
            gpga.cluster_corr(Rs[k:k + st.W], Cs[k], stream)
        rmt_batch = lambda: gpga.corr_clean_rmt(Cs.clone(), st.W, stream=stream)  # noqa: E731
        runtime.barrier(ranks)
        rmtB_s = timed(rmt_batch, 3)
        _, nnB, swB = rmt_batch()
        lab = torch.from_numpy(pl.truth.astype(np.int32)).to(dev)
        mst_s = timed(lambda: gpga.cluster_mst(C, lab, stream=stream), 3)
    max_secs, total = runtime.aggregate(ranks, rmtB_s, float(st.windows), device=dev)
    if ranks.rank != 0:
        runtime.barrier(ranks)
        return
    # Jacobi FP64 work: per Jacobi round 3 n2^2 flops on A (upper pair-blocks, 24 flops
    # per 2 x 2 block) and 3 n2^2 on V, n2 - 1 rounds per sweep
    def jacobi_flops(N, sweeps, B=1):
        n2 = N + (N & 1)
        return float(B) * sweeps * (n2 - 1) * 6.0 * n2 * n2
    fB = jacobi_flops(18, swB, st.windows) / rmtB_s / 1e12
    # the oracle (NumPy / LAPACK, its default threads) on the same inputs
    Ch = C.cpu().numpy()
    t0 = time.perf_counter()
    oracle.clean_rmt(Ch, T)
    orc500 = time.perf_counter() - t0
    Csh = Cs.cpu().numpy()
    nb = 200
    t0 = time.perf_counter()
    for k in range(nb):
        oracle.clean_rmt(Csh[k], st.W)
    orcB = (time.perf_counter() - t0) / nb
    t0 = time.perf_counter()
    oracle.cluster_mst(pl.truth, Ch)
    orc_mst = time.perf_counter() - t0
    line = {"metric": "windows/s (random-matrix cleaning of the 18-stock stream: 1760 "
                      "correlation windows of 1800 bars, one batch)",
            "value": total / max_secs, "unit": "windows/s", "n_gpus": ranks.world, "steps": 3,
            "warmup": 1, "ms_per_step": 1e3 * max_secs, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "rmt_clean_n18_w1800_x1760"},
            "rmt_stream": {"sweeps": swB, "noise_set_sizes": sorted(set(nnB))},
            "rmt_n500": {"ms": 1e3 * rmt500_s, "noise_set": nn500[0],
                         "solver": "Householder tridiagonal reduction + bisection + inverse "
                                   "iteration" if sw500 == 0 else f"cyclic Jacobi, {sw500} sweeps"},
            "roofline": {"bound": "alu", "kernel": "jacobi_round (N=18, 1760 matrices)",
                         "achieved": fB, "peak": FP64_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                         "frac": fB / FP64_TFLOPS_NOMINAL, "traffic": None,
                         "peak_source": "nominal FP64 rate (fallback: no measured FP64 peak)"},
            "ewma_corr_n500_t5000_ms": 1e3 * ewma_s,
            "market_removal_n500_ms": 1e3 * mkt_s,
            "cluster_mst_n500_planted_ms": 1e3 * mst_s,
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(),
                             "rmt_n500_ms": 1e3 * orc500,
                             "cluster_mst_n500_planted_ms": 1e3 * orc_mst,
                             "value": 1.0 / orcB, "unit": "windows/s",
                             "sample": f"{nb} of the 1760 windows, one by one (NumPy eigh, its "
                                       "default threads), and the N=500 matrix once"}}
    print(json.dumps(line), flush=True)
    runtime.barrier(ranks)


def run_islands(args, ranks):
    """The island model (the variant the paper proposes, Sec. 5.2 and 6) against one
    population of the same total size, on the N = 100 workload: 8 islands of 512
    with ring migration of 2 elites every 10 generations, and one population of
    4096; 200 generations each without the stall rule, so both make the same
    number of evaluations. Each timed from its start call to its last step."""
    import torch

    from paper_1403_4099_gb300 import gpga, metrics, runtime, synth
    torch.cuda.set_device(ranks.local)
    dev = torch.device("cuda", ranks.local)
    runtime.init_dist(ranks, "nccl")
    stream = torch.cuda.Stream(device=dev)
    G, K, PI = 200, 8, 512
    pl = synth.n100(replicate=ranks.rank)
    with torch.cuda.stream(stream):
        C = gpga.cluster_corr(torch.from_numpy(pl.R).to(dev), stream=stream)
        stream.synchronize()

        def island_job(seed):
            prm = gpga.default_params(P=PI, elite=10, max_gens=G, tol=-1.0, pm=0.01,
                                      form=gpga.FORM_GATHER)
            t0 = time.perf_counter()
            b = gpga.Batch.islands(C, prm, K, seed=seed, migrate_every=10, migrants=2,
                                   stream=stream)
            while b.step(16) > 0:
                pass
            stream.synchronize()
            secs = time.perf_counter() - t0
            best = max((b.best(k) for k in range(K)), key=lambda t: t[1])
            b.close()
            return secs, best

        def single_job(seed):
            prm = gpga.default_params(P=K * PI, elite=10, max_gens=G, tol=-1.0, pm=0.01,
                                      form=gpga.FORM_GATHER)
            t0 = time.perf_counter()
            ga = gpga.GA(C, prm, seed=seed, stream=stream)
            ga.step(G)
            stream.synchronize()
            secs = time.perf_counter() - t0
            best = ga.best()
            ga.close()
            return secs, best

        island_job(1)  # warm-up (library, tuner, graphs)
        single_job(1)
        runtime.barrier(ranks)
        res_i = [island_job(100 + k) for k in range(args.steps // 4 or 1)]
        res_s = [single_job(100 + k) for k in range(args.steps // 4 or 1)]
    ti = float(np.median([r[0] for r in res_i]))
    ts = float(np.median([r[0] for r in res_s]))
    evals = float(K * PI * (G + 1))
    max_t, total = runtime.aggregate(ranks, ti, evals, device=dev)
    if ranks.rank == 0:
        def summary(res):
            return {"best_L": [float(r[1][1]) for r in res],
                    "ari": [float(metrics.ari(r[1][0], pl.truth)) for r in res]}
        line = {"metric": "fitness evals/s (island model: 8 islands x P=512, N=100, 200 "
                          "generations, ring migration of 2 elites every 10)",
                "value": total / max_t, "unit": "evals/s", "n_gpus": ranks.world,
                "steps": len(res_i), "warmup": 1, "ms_per_step": 1e3 * max_t,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE["gather"][0],
                "dtype_detail": DTYPE["gather"][1], "data": "synthetic",
                "config": {"workload": "islands_n100_t2000_k8_p512_g200", "migrate_every": 10,
                           "migrants": 2, "pm": 0.01},
                "islands": summary(res_i),
                "single_population_p4096": {"evals_per_s": evals / ts, "ms": 1e3 * ts,
                                            **summary(res_s)}}
        print(json.dumps(line), flush=True)
    runtime.barrier(ranks)


def main():
    args = parse()
    from paper_1403_4099_gb300 import runtime
    ranks = runtime.ranks_from_env()
    if args.impl == "reference":
        run_reference(args, ranks)
        return
    if args.workload == "batched":
        run_batched(args, ranks)
        return
    if args.workload == "serving":
        run_serving(args, ranks)
        return
    if args.workload == "paper":
        run_paper(args, ranks)
        return
    if args.workload == "preprocess":
        run_preprocess(args, ranks)
        return
    if args.workload == "islands":
        run_islands(args, ranks)
        return
    run_gpu(args, ranks)


if __name__ == "__main__":
    main()
