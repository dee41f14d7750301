// fleet.cu -- many independent GA runs on one GPU: the batch calls
// (ga_batch_*: a fixed set of runs, e.g. one per sliding window) and the
// serving loop (serve_*: requests admitted while others run, by free device
// memory), both over one "fleet" of runs.
//
// Every run keeps its own C, N, population, fitness, state and Philox key in
// device memory for its whole life. One generation of the whole fleet is two
// launches: the fused generation kernel over all (run, slot) work items (a
// grid of resident CTAs striding over the items, runs ordered by decreasing N
// so the costly ones start first) and the selection kernel with one grid
// slice per run. Both read the run table from device memory, so the CUDA
// graph of U generations captured once stays valid while runs come and go.
// Per slot the arithmetic is that of the single-run gather form, so a run's
// result does not depend on which other runs share the fleet.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "gpga_internal.cuh"

namespace gpga {

namespace {

struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(char *b) : base(b) {}
    template <typename T> T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

// one run's device memory
struct RunMem {
    char *block = nullptr;
    size_t bytes = 0;
    double *C64 = nullptr;
    int32_t *canon = nullptr;
    double *Lbest = nullptr;
    int *err = nullptr;
    int *diag = nullptr;
    int32_t *mst_order = nullptr, *mst_from = nullptr;
    double *mst_w = nullptr;
    FleetRun d{};
};

struct Slot {
    bool used = false;
    long long since = -1; // first tick whose run table holds this run (-1: not yet)
    int N = 0;
    uint64_t seed = 0;
    long long id = -1;
    RunMem m;
    std::chrono::steady_clock::time_point t_submit, t_admit;
};

} // namespace

struct Fleet {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    gpga_params prm{};
    int P = 0, E = 0, M = 0;
    int cap = 0, Nmax = 0, Np_max = 0;
    char *shared = nullptr;        // rank table, log tables, run table, states
    uint64_t *rank_prefix = nullptr;
    int32_t *sus_tab = nullptr; // SUS brackets of rank_prefix (M + 1)
    double *logtab = nullptr;
    FleetRun *d_runs = nullptr;
    FleetHdr *d_hdr = nullptr;
    DevState *d_st = nullptr;      // cap states, indexed by slot
    // pinned mirrors, two of each: a serving tick fills one while the copies
    // of the previous tick may still read the other
    FleetRun *h_runs[2] = {nullptr, nullptr};
    FleetHdr *h_hdr[2] = {nullptr, nullptr};
    DevState *h_st[2] = {nullptr, nullptr};
    std::vector<Slot> slots;
    int nactive = 0, nitems = 0;
    int warps = 0, ctas = 0;
    float tune_ms = 0.f;
    bool flat_ok = false;    // a grid sized to the items is allowed (fixed set of runs)
    long long tune_items = 0; // work items when the shape was last tuned
    bool retune = false;      // tune again when the items double
    cudaGraphExec_t gU = nullptr, g1 = nullptr;
    int U = 8;
    int migrate_every = 0, migrants = 0; // island model (0: independent runs)
};

static size_t run_bytes(const Fleet *f, int N, char *base, RunMem *m)
{
    Carve c(base);
    const size_t Np = pad_n(N), P = f->P, G = (size_t)f->prm.max_gens + 1;
    RunMem t;
    t.C64 = c.take<double>((size_t)N * N);
    t.d.Dfix = c.take<int32_t>(Np * Np);
    t.d.pop0 = c.take<uint16_t>(P * Np);
    t.d.pop1 = c.take<uint16_t>(P * Np);
    t.d.L = c.take<double>(P);
    t.d.perm = c.take<int32_t>(P);
    t.d.rank = c.take<int>(P);
    t.d.ticket = c.take<unsigned>(TICKETS);
    t.d.work_prefix = c.take<uint64_t>(P);
    t.d.hist = c.take<double>(G);

    t.canon = c.take<int32_t>(N);
    t.Lbest = c.take<double>(1);
    t.err = c.take<int>(1);
    t.diag = c.take<int>(1);
    if (f->prm.init == GPGA_INIT_THRESHOLD) {
        t.mst_order = c.take<int32_t>(N);
        t.mst_from = c.take<int32_t>(N);
        t.mst_w = c.take<double>(N);
    }
    t.d.diag = t.diag;
    t.d.N = N;
    t.d.Np = (int)Np;
    if (m) *m = t;
    return c.off + 256;
}

static SelectCfg fleet_select_cfg(const Fleet *f, int N, int gen_off)
{
    SelectCfg c;
    c.P = f->P;
    c.E = f->E;
    c.M = f->M;
    c.N = N;
    c.ldp = pad_n(N);
    c.scaling = f->prm.scaling;
    c.max_gens = f->prm.max_gens;
    c.stall_gens = f->prm.stall_gens;
    c.tol = f->prm.tol;
    c.k0 = 0;
    c.k1 = 0;
    c.gen_off = gen_off;
    c.record = 0;
    return c;
}

static EvolveCfg fleet_evolve_cfg(const Fleet *f)
{
    EvolveCfg e;
    e.P = f->P;
    e.E = f->E;
    e.M = f->M;
    e.N = 0; // per run
    e.ldp = 0;
    e.thr_pc = prob_threshold(f->prm.pc);
    e.thr_pkb = prob_threshold(f->prm.pkb);
    set_mutation(&e, f->prm.pm);
    set_sus_divisor(&e, f->M);
    e.k0 = 0;
    e.k1 = 0;
    e.gen = 0;
    e.sus_tab = f->prm.scaling == GPGA_SCALING_PROP ? nullptr : f->sus_tab;
    return e;
}

static void fleet_destroy(Fleet *f)
{
    if (!f) return;
    if (f->gU) cudaGraphExecDestroy(f->gU);
    if (f->g1) cudaGraphExecDestroy(f->g1);
    for (auto &s : f->slots)
        if (s.m.block) cudaFreeAsync(s.m.block, f->stream);
    if (f->shared) cudaFreeAsync(f->shared, f->stream);
    if (f->stream) cudaStreamSynchronize(f->stream);
    for (int b = 0; b < 2; ++b) {
        if (f->h_runs[b]) cudaFreeHost(f->h_runs[b]);
        if (f->h_hdr[b]) cudaFreeHost(f->h_hdr[b]);
        if (f->h_st[b]) cudaFreeHost(f->h_st[b]);
    }
    if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
    delete f;
}

static int fleet_create(const gpga_params *p, int cap, int Nmax, void *stream, Fleet **out)
{
    int rc = check_params(p, Nmax);
    if (rc) return rc;
    if (p->form != GPGA_FORM_GATHER)
        return set_error(GPGA_ERR_ARG, "fleet: only the gather form runs batched (form=%d)", p->form);
    if (p->record || p->profile)
        return set_error(GPGA_ERR_ARG, "fleet: record and profile are single-run options");
    if (cap < 1 || cap > 65535) return set_error(GPGA_ERR_ARG, "fleet: %d runs outside [1, 65535]", cap);
    rc = prepare_device();
    if (rc) return rc;
    Fleet *f = new (std::nothrow) Fleet;
    if (!f) return set_error(GPGA_ERR_OOM, "fleet: host allocation");
    f->prm = *p;
    f->P = p->P;
    f->E = p->elite;
    f->M = p->P - p->elite;
    f->cap = cap;
    f->Nmax = Nmax;
    f->Np_max = pad_n(Nmax);
    cudaGetDevice(&f->dev);
    if (stream) {
        f->stream = (cudaStream_t)stream;
    } else if (cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete f;
        return set_error(GPGA_ERR_CUDA, "fleet: stream creation failed");
    } else {
        f->own_stream = true;
    }
    f->slots.resize(cap);
    size_t bytes = 0;
    for (int pass = 0; pass < 2; ++pass) {
        Carve c(f->shared);
        uint64_t *rp = c.take<uint64_t>(f->P);
        int32_t *stab = c.take<int32_t>((size_t)f->M + 1);
        double *lt = c.take<double>(logtab_len(Nmax));
        FleetRun *dr = c.take<FleetRun>(cap);
        FleetHdr *dh = c.take<FleetHdr>(1);
        DevState *ds = c.take<DevState>(cap);
        if (pass == 0) {
            bytes = c.off + 256;
            cudaError_t e = cudaMallocAsync((void **)&f->shared, bytes, f->stream);
            if (e != cudaSuccess) {
                fleet_destroy(f);
                return cuda_error(e, "fleet: device allocation", __FILE__, __LINE__);
            }
        } else {
            f->rank_prefix = rp;
            f->sus_tab = stab;
            f->logtab = lt;
            f->d_runs = dr;
            f->d_hdr = dh;
            f->d_st = ds;
        }
    }
    for (int b = 0; b < 2; ++b) {
        if (cudaMallocHost((void **)&f->h_runs[b], (size_t)cap * sizeof(FleetRun)) != cudaSuccess ||
            cudaMallocHost((void **)&f->h_hdr[b], sizeof(FleetHdr)) != cudaSuccess ||
            cudaMallocHost((void **)&f->h_st[b], (size_t)cap * sizeof(DevState)) != cudaSuccess) {
            fleet_destroy(f);
            return set_error(GPGA_ERR_OOM, "fleet: pinned host allocation");
        }
        memset(f->h_st[b], 0, (size_t)cap * sizeof(DevState));
        f->h_hdr[b]->nruns = 0;
        f->h_hdr[b]->nitems = 0;
    }
    rc = rank_prefix_table(f->rank_prefix, f->P, f->M, f->sus_tab, f->stream);
    if (!rc) rc = launch_logtab(f->logtab, Nmax, f->stream);
    if (!rc && cudaMemsetAsync(f->d_hdr, 0, sizeof(FleetHdr), f->stream) != cudaSuccess)
        rc = set_error(GPGA_ERR_CUDA, "fleet: memset failed");
    if (!rc && cudaMemsetAsync(f->d_st, 0, (size_t)cap * sizeof(DevState), f->stream) != cudaSuccess)
        rc = set_error(GPGA_ERR_CUDA, "fleet: memset failed");
    if (rc) {
        fleet_destroy(f);
        return rc;
    }
    *out = f;
    return GPGA_OK;
}

// Start run `slot` on C (device; ld ldc; optional device column subset cols).
// C == nullptr: the caller has already written the dense C into m.C64.
static int fleet_start(Fleet *f, int slot, const double *C, int ldc, const int32_t *cols, int N,
                       uint64_t seed)
{
    Slot &s = f->slots[slot];
    RunMem &m = s.m;
    cudaStream_t st = f->stream;
    const int Np = pad_n(N), P = f->P;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    m.d.st = f->d_st + slot;
    GPGA_CUDA(cudaMemsetAsync(m.err, 0, sizeof(int), st));
    GPGA_CUDA(cudaMemsetAsync(m.diag, 0, sizeof(int), st));
    GPGA_CUDA(cudaMemsetAsync(m.d.rank, 0, (size_t)P * sizeof(int), st));
    GPGA_CUDA(cudaMemsetAsync(m.d.ticket, 0, TICKETS * sizeof(unsigned), st));
    int rc = launch_state_init(m.d.st, nullptr, k0, k1, st);
    if (rc) return rc;
    rc = C ? launch_fleet_prep(C, ldc, cols, N, Np, m.C64, const_cast<int32_t *>(m.d.Dfix), m.diag, st)
           : launch_fleet_prep(m.C64, N, nullptr, N, Np, nullptr, const_cast<int32_t *>(m.d.Dfix),
                               m.diag, st);
    if (rc) return rc;
    if (f->prm.init == GPGA_INIT_THRESHOLD) {
        rc = launch_mst(m.C64, N, m.mst_order, m.mst_from, m.mst_w, st);
        if (!rc)
            rc = launch_init_threshold<uint16_t>(m.d.pop0, Np, P, N, m.mst_order, m.mst_from,
                                                 m.mst_w, f->prm.tau_lo, f->prm.tau_hi, k0, k1, st);
    } else {
        const int K0 = f->prm.init_labels > 0 ? std::min(f->prm.init_labels, N) : N;
        rc = launch_init_uniform<uint16_t>(m.d.pop0, Np, P, N, K0, k0, k1, st);
    }
    if (rc) return rc;
    GPGA_CUDA(cudaMemsetAsync(m.d.pop1, 0, (size_t)P * Np * sizeof(uint16_t), st));
    const uint16_t *lab2[2] = {m.d.pop0, m.d.pop1};
    rc = launch_gather_score<uint16_t>(lab2, Np, 0, P, N, Np, m.d.Dfix, m.diag, f->logtab, m.d.L,
                                       m.err, m.d.st, nullptr, ScoreTab{}, st);
    if (rc) return rc;
    return launch_select<uint16_t>(m.d.L, fleet_select_cfg(f, N, 0), m.d.rank, m.d.perm,
                                   m.d.work_prefix, m.d.ticket, m.d.st, m.d.hist, lab2, nullptr,
                                   nullptr, st);
}

static int fleet_alloc_run(Fleet *f, int slot, int N)
{
    Slot &s = f->slots[slot];
    const size_t bytes = run_bytes(f, N, nullptr, nullptr);
    char *block = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&block, bytes, f->stream));
    run_bytes(f, N, block, &s.m);
    s.m.block = block;
    s.m.bytes = bytes;
    s.N = N;
    return GPGA_OK;
}

static void fleet_release_run(Fleet *f, int slot)
{
    Slot &s = f->slots[slot];
    if (s.m.block) cudaFreeAsync(s.m.block, f->stream);
    s = Slot{};
}

// the run table: used slots by decreasing N (ties by slot), and the header,
// from pinned mirror `b`; runs entering the table are stamped with `tick`
static int fleet_upload(Fleet *f, int b, long long tick)
{
    std::vector<int> order;
    for (int i = 0; i < f->cap; ++i)
        if (f->slots[i].used) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int c) { return f->slots[a].N > f->slots[c].N; });
    for (size_t k = 0; k < order.size(); ++k) f->h_runs[b][k] = f->slots[order[k]].m.d;
    f->nactive = (int)order.size();
    f->nitems = f->nactive * f->P;
    f->h_hdr[b]->nruns = f->nactive;
    f->h_hdr[b]->nitems = f->nitems;
    if (f->nactive)
        GPGA_CUDA(cudaMemcpyAsync(f->d_runs, f->h_runs[b], (size_t)f->nactive * sizeof(FleetRun),
                                  cudaMemcpyHostToDevice, f->stream));
    GPGA_CUDA(cudaMemcpyAsync(f->d_hdr, f->h_hdr[b], sizeof(FleetHdr), cudaMemcpyHostToDevice,
                              f->stream));
    for (int i : order)
        if (f->slots[i].since < 0) f->slots[i].since = tick;
    return GPGA_OK;
}

// pdl: the launch directly follows the fleet's selection in a captured graph
static int fleet_gen_launch(Fleet *f, int warps, int ctas, bool pdl = false)
{
    return launch_fleet_generation(f->d_runs, f->d_hdr, fleet_evolve_cfg(f), f->rank_prefix,
                                   f->logtab, f->Np_max, warps, ctas,
                                   f->prm.scaling == GPGA_SCALING_PROP, f->stream, pdl);
}

// Autotuner: warps per CTA (individuals per CTA) and grid shape of the fused
// generation kernel, timed on the fleet's current runs. The kernel is
// idempotent between selections (it rewrites the next population and its
// fitness from the same parents and Philox counters), so the trials leave the
// runs' results unchanged. Shapes: 1, 2 or 4 waves of resident CTAs striding
// over the items and, when f->flat_ok (a fixed set of runs), one warp per item.
static int fleet_tune(Fleet *f)
{
    int sms = 0;
    GPGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->dev));
    const int wmax = fleet_max_warps(f->Np_max);
    struct Cand {
        int warps, ctas;
    };
    std::vector<Cand> cands;
    for (int w = 2; w <= wmax; w <<= 1) {
        int occ = 0;
        int rc = fleet_ctas_per_sm(f->Np_max, w, &occ);
        if (rc) return rc;
        if (occ < 1) continue;
        const int flat = (f->nitems + w - 1) / w;
        for (int waves = 1; waves <= 4; waves <<= 1)
            if (waves == 1 || sms * occ * waves < flat) cands.push_back({w, sms * occ * waves});
        if (f->flat_ok && flat > sms * occ) cands.push_back({w, flat});
    }
    if (cands.empty()) return set_error(GPGA_ERR_ARG, "fleet: no launch shape fits N=%d", f->Nmax);
    if (f->nactive == 0) { // nothing to time: the widest one-wave shape
        for (const Cand &c : cands)
            if (c.ctas <= sms * 64) {
                f->warps = c.warps;
                f->ctas = c.ctas;
            }
        return GPGA_OK;
    }
    cudaEvent_t e0, e1;
    GPGA_CUDA(cudaEventCreate(&e0));
    GPGA_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int rc = GPGA_OK;
    for (const Cand &c : cands) {
        rc = fleet_gen_launch(f, c.warps, c.ctas); // warm-up
        if (rc) break;
        cudaEventRecord(e0, f->stream);
        for (int r = 0; r < 3 && !rc; ++r) rc = fleet_gen_launch(f, c.warps, c.ctas);
        cudaEventRecord(e1, f->stream);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = set_error(GPGA_ERR_CUDA, "fleet: tuning sync failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        if (ms < best) {
            best = ms;
            f->warps = c.warps;
            f->ctas = c.ctas;
            f->tune_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    f->tune_items = f->nitems;
    // the trials rewrote each run's fitness with that of the next population:
    // score the current populations again (the selection already used the
    // right values, so the runs' results do not change)
    for (int i = 0; i < f->cap && !rc; ++i) {
        const Slot &s = f->slots[i];
        if (!s.used) continue;
        const uint16_t *lab2[2] = {s.m.d.pop0, s.m.d.pop1};
        rc = launch_gather_score<uint16_t>(lab2, s.m.d.Np, 0, f->P, s.N, s.m.d.Np, s.m.d.Dfix,
                                           s.m.diag, f->logtab, s.m.d.L, s.m.err, s.m.d.st,
                                           nullptr, ScoreTab{}, f->stream);
    }
    return rc;
}

static int fleet_graph(Fleet *f, int gens, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    GPGA_CUDA(cudaStreamBeginCapture(f->stream, cudaStreamCaptureModeThreadLocal));
    int rc = GPGA_OK;
    for (int k = 0; k < gens && !rc; ++k) {
        rc = fleet_gen_launch(f, f->warps, f->ctas, k > 0);
        if (!rc && f->migrate_every > 0)
            rc = launch_fleet_migrate(f->d_runs, f->d_hdr, f->P, f->migrate_every, f->migrants,
                                      f->cap, f->stream);
        if (!rc) rc = launch_fleet_select(f->d_runs, f->d_hdr, fleet_select_cfg(f, f->Nmax, 1),
                                          f->cap, f->stream);
    }
    cudaError_t e = cudaStreamEndCapture(f->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_error(e, "fleet: cudaStreamEndCapture", __FILE__, __LINE__);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(e, "fleet: cudaGraphInstantiate", __FILE__, __LINE__);
    return GPGA_OK;
}

static int fleet_step(Fleet *f, int generations)
{
    if (generations <= 0 || f->nactive == 0) return GPGA_OK;
    int rc;
    if (!f->warps || (f->retune && f->nitems > 2 * f->tune_items)) {
        rc = fleet_tune(f);
        if (rc) return rc;
        if (f->gU) cudaGraphExecDestroy(f->gU);
        if (f->g1) cudaGraphExecDestroy(f->g1);
        f->gU = f->g1 = nullptr;
    }
    if (generations >= f->U && !f->gU) {
        rc = fleet_graph(f, f->U, &f->gU);
        if (rc) return rc;
    }
    if (generations % f->U && !f->g1) {
        rc = fleet_graph(f, 1, &f->g1);
        if (rc) return rc;
    }
    int left = generations;
    for (; left >= f->U; left -= f->U) GPGA_CUDA(cudaGraphLaunch(f->gU, f->stream));
    for (; left > 0; --left) GPGA_CUDA(cudaGraphLaunch(f->g1, f->stream));
    return GPGA_OK;
}

static int fleet_status(Fleet *f)
{
    GPGA_CUDA(cudaMemcpyAsync(f->h_st[0], f->d_st, (size_t)f->cap * sizeof(DevState),
                              cudaMemcpyDeviceToHost, f->stream));
    GPGA_CUDA(cudaStreamSynchronize(f->stream));
    return GPGA_OK;
}

// FP64 re-score + canonical labels of run `slot`'s best into its canon/Lbest
static int fleet_rescore(Fleet *f, int slot)
{
    RunMem &m = f->slots[slot].m;
    return launch_rescore_fp64(m.d.pop0, m.d.pop1, m.d.Np, m.d.st, m.C64, m.d.N, m.canon, m.Lbest,
                               f->stream);
}

} // namespace gpga

using namespace gpga;

// ---------------------------------------------------------------------------
// batch
// ---------------------------------------------------------------------------
struct gpga_batch {
    Fleet *f = nullptr;
    int runs = 0;
};

extern "C" {

GPGA_API int ga_batch_init(int runs, const double *const *C, const int *ldc,
                           const int32_t *const *cols, const int *N, const gpga_params *p,
                           const uint64_t *seeds, void *stream, gpga_batch **out)
{
    if (!out) return set_error(GPGA_ERR_ARG, "ga_batch_init: out is NULL");
    *out = nullptr;
    if (runs < 1 || !C || !N || !seeds)
        return set_error(GPGA_ERR_ARG, "ga_batch_init: runs=%d or a NULL array", runs);
    int Nmax = 0;
    for (int k = 0; k < runs; ++k) {
        if (!C[k]) return set_error(GPGA_ERR_ARG, "ga_batch_init: C[%d] is NULL", k);
        if (N[k] < 2 || N[k] > GPGA_MAX_N)
            return set_error(GPGA_ERR_ARG, "ga_batch_init: N[%d]=%d outside [2, %d]", k, N[k], GPGA_MAX_N);
        if (ldc && ldc[k] < (cols && cols[k] ? 1 : N[k]))
            return set_error(GPGA_ERR_ARG, "ga_batch_init: ldc[%d]=%d too small", k, ldc[k]);
        Nmax = std::max(Nmax, N[k]);
    }
    Fleet *f = nullptr;
    int rc = fleet_create(p, runs, Nmax, stream, &f);
    if (rc) return rc;
    for (int k = 0; k < runs && !rc; ++k) {
        rc = fleet_alloc_run(f, k, N[k]);
        if (rc) break;
        f->slots[k].used = true;
        f->slots[k].seed = seeds[k];
        rc = fleet_start(f, k, C[k], ldc ? ldc[k] : N[k], cols ? cols[k] : nullptr, N[k], seeds[k]);
    }
    f->flat_ok = true;
    if (!rc) rc = fleet_upload(f, 0, 0);
    if (!rc) rc = fleet_tune(f);
    if (!rc) rc = fleet_status(f);
    if (rc) {
        fleet_destroy(f);
        return rc;
    }
    gpga_batch *h = new (std::nothrow) gpga_batch;
    if (!h) {
        fleet_destroy(f);
        return set_error(GPGA_ERR_OOM, "ga_batch_init: host allocation");
    }
    h->f = f;
    h->runs = runs;
    *out = h;
    return GPGA_OK;
}

GPGA_API int ga_island_init(int islands, const double *C, int N, const gpga_params *p,
                            uint64_t seed, int migrate_every, int migrants, void *stream,
                            gpga_batch **out)
{
    if (!out) return set_error(GPGA_ERR_ARG, "ga_island_init: out is NULL");
    *out = nullptr;
    if (islands < 2 || !C || !p)
        return set_error(GPGA_ERR_ARG, "ga_island_init: islands=%d (>= 2) or a NULL argument",
                         islands);
    if (migrate_every < 1 || migrants < 1 || migrants > p->elite || 2 * migrants > p->P)
        return set_error(GPGA_ERR_ARG,
                         "ga_island_init: migrate_every=%d, migrants=%d (1 <= migrants <= elite, "
                         "2 migrants <= P)",
                         migrate_every, migrants);
    std::vector<const double *> Cs(islands, C);
    std::vector<int> Ns(islands, N);
    std::vector<uint64_t> seeds(islands);
    for (int k = 0; k < islands; ++k) seeds[k] = seed + (uint64_t)k;
    gpga_batch *h = nullptr;
    int rc = ga_batch_init(islands, Cs.data(), nullptr, nullptr, Ns.data(), p, seeds.data(),
                           stream, &h);
    if (rc) return rc;
    // migration enters the captured generation graphs (none is built yet)
    h->f->migrate_every = migrate_every;
    h->f->migrants = migrants;
    *out = h;
    return GPGA_OK;
}

GPGA_API int ga_batch_population(gpga_batch *h, int run, int32_t *pop, double *L)
{
    if (!h) return set_error(GPGA_ERR_ARG, "ga_batch_population: NULL handle");
    if (run < 0 || run >= h->runs) return set_error(GPGA_ERR_ARG, "ga_batch_population: run %d", run);
    Fleet *f = h->f;
    int rc = fleet_status(f);
    if (rc) return rc;
    const RunMem &m = f->slots[run].m;
    const int P = f->P, N = m.d.N, Np = m.d.Np;
    if (pop) {
        std::vector<uint16_t> tmp((size_t)P * Np);
        const uint16_t *buf = (f->h_st[0][run].gen & 1) ? m.d.pop1 : m.d.pop0;
        GPGA_CUDA(cudaMemcpy(tmp.data(), buf, tmp.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost));
        for (int q = 0; q < P; ++q)
            for (int j = 0; j < N; ++j) pop[(size_t)q * N + j] = tmp[(size_t)q * Np + j];
    }
    if (L) GPGA_CUDA(cudaMemcpy(L, m.d.L, (size_t)P * sizeof(double), cudaMemcpyDeviceToHost));
    return GPGA_OK;
}

GPGA_API int ga_batch_step(gpga_batch *h, int generations, int *active)
{
    if (!h) return set_error(GPGA_ERR_ARG, "ga_batch_step: NULL handle");
    if (generations < 0) return set_error(GPGA_ERR_ARG, "ga_batch_step: generations < 0");
    int rc = fleet_step(h->f, generations);
    if (rc) return rc;
    if (active) {
        rc = fleet_status(h->f);
        if (rc) return rc;
        int a = 0;
        for (int k = 0; k < h->runs; ++k) a += h->f->h_st[0][k].done ? 0 : 1;
        *active = a;
    }
    return GPGA_OK;
}

GPGA_API int ga_batch_status(gpga_batch *h, int32_t *generation, int32_t *done, double *best)
{
    if (!h) return set_error(GPGA_ERR_ARG, "ga_batch_status: NULL handle");
    int rc = fleet_status(h->f);
    if (rc) return rc;
    for (int k = 0; k < h->runs; ++k) {
        const DevState &s = h->f->h_st[0][k];
        if (generation) generation[k] = s.gen;
        if (done) done[k] = s.done;
        if (best) best[k] = s.best;
    }
    return GPGA_OK;
}

GPGA_API int ga_batch_best(gpga_batch *h, int run, int32_t *labels, double *L, int *generation)
{
    if (!h) return set_error(GPGA_ERR_ARG, "ga_batch_best: NULL handle");
    if (run < 0 || run >= h->runs) return set_error(GPGA_ERR_ARG, "ga_batch_best: run %d", run);
    Fleet *f = h->f;
    RunMem &m = f->slots[run].m;
    int rc = fleet_rescore(f, run);
    if (rc) return rc;
    if (labels)
        GPGA_CUDA(cudaMemcpyAsync(labels, m.canon, (size_t)m.d.N * sizeof(int32_t),
                                  is_device_ptr(labels) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyDeviceToHost,
                                  f->stream));
    if (L)
        GPGA_CUDA(cudaMemcpyAsync(L, m.Lbest, sizeof(double),
                                  is_device_ptr(L) ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyDeviceToHost,
                                  f->stream));
    rc = fleet_status(f);
    if (rc) return rc;
    if (generation) *generation = f->h_st[0][run].gen;
    return GPGA_OK;
}

GPGA_API int ga_batch_tuning(gpga_batch *h, int *warps_per_cta, int *ctas, float *ms)
{
    if (!h) return set_error(GPGA_ERR_ARG, "ga_batch_tuning: NULL handle");
    if (warps_per_cta) *warps_per_cta = h->f->warps;
    if (ctas) *ctas = h->f->ctas;
    if (ms) *ms = h->f->tune_ms;
    return GPGA_OK;
}

GPGA_API int ga_batch_free(gpga_batch *h)
{
    if (!h) return GPGA_OK;
    fleet_destroy(h->f);
    delete h;
    return GPGA_OK;
}

} // extern "C"

// ---------------------------------------------------------------------------
// serving
//
// A tick k, on the host: wait until the GPU has finished tick k-2 (its status
// copy), collect the results copied out at tick k-1, retire the runs that
// tick k-2 left terminated (FP64 re-score and copy-out enqueued, memory freed
// in stream order), admit queued requests, upload the run table and launch the
// generations of tick k, then the status copy. The GPU runs tick k-1 while the
// host prepares tick k, so it never waits for the host; results come back two
// to three ticks after their run terminates.
// ---------------------------------------------------------------------------
struct gpga_server {
    Fleet *f = nullptr;
    size_t budget = 0;     // bytes of run memory the server may hold
    size_t in_use = 0;
    size_t reserve = 0;    // device memory always left free
    long long next_id = 0;
    long long completed = 0;
    long long tick = 0;
    struct Req {
        long long id;
        int N;
        uint64_t seed;
        std::vector<double> C;
        std::chrono::steady_clock::time_point t_submit;
    };
    std::deque<Req> queue;
    struct Result {
        std::vector<int32_t> labels;
        double L;
        int gen;
        double queue_s, run_s;
    };
    std::unordered_map<long long, Result> results;
    std::unordered_map<long long, int> running; // id -> slot
    // results in flight: copied at tick t into the pinned arena, collected at t+1
    struct Out {
        long long id;
        int slot, N, gen;
        std::chrono::steady_clock::time_point t_submit, t_admit;
    };
    std::vector<Out> out[2];
    int32_t *arena_lab = nullptr; // pinned, cap x Nmax
    double *arena_L = nullptr;    // pinned, cap
    double *stage[2] = {nullptr, nullptr}; // pinned request matrices of a tick
    size_t stage_cap[2] = {0, 0};
    cudaEvent_t ev_status[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    cudaEvent_t ev_g0[2] = {nullptr, nullptr}, ev_g1[2] = {nullptr, nullptr};
    bool g_timed[2] = {false, false};
    // counters
    double gpu_ms = 0.0;          // device time of the generation graphs
    long long gens = 0;           // fleet generations launched
    long long item_gens = 0;      // sum over launched generations of the work items
    double host_wait_s = 0.0, host_work_s = 0.0;
};

namespace {

void serve_release(gpga_server *h)
{
    if (!h) return;
    if (h->f) fleet_destroy(h->f); // synchronises the stream
    for (int b = 0; b < 2; ++b) {
        if (h->stage[b]) cudaFreeHost(h->stage[b]);
        if (h->ev_status[b]) cudaEventDestroy(h->ev_status[b]);
        if (h->ev_out[b]) cudaEventDestroy(h->ev_out[b]);
        if (h->ev_g0[b]) cudaEventDestroy(h->ev_g0[b]);
        if (h->ev_g1[b]) cudaEventDestroy(h->ev_g1[b]);
    }
    if (h->arena_lab) cudaFreeHost(h->arena_lab);
    if (h->arena_L) cudaFreeHost(h->arena_L);
    delete h;
}

// move the results copied out at the previous tick (its copies are complete)
void serve_collect(gpga_server *h, int b)
{
    const auto now = std::chrono::steady_clock::now();
    const int Nmax = h->f->Nmax;
    for (const gpga_server::Out &o : h->out[b]) {
        gpga_server::Result r;
        r.labels.assign(h->arena_lab + (size_t)o.slot * Nmax, h->arena_lab + (size_t)o.slot * Nmax + o.N);
        r.L = h->arena_L[o.slot];
        r.gen = o.gen;
        r.queue_s = std::chrono::duration<double>(o.t_admit - o.t_submit).count();
        r.run_s = std::chrono::duration<double>(now - o.t_admit).count();
        h->results[o.id] = std::move(r);
        h->running.erase(o.id);
        ++h->completed;
    }
    h->out[b].clear();
}

// retire the runs whose status (from tick `tick` - 2, mirror b) says done:
// FP64 re-score, copy-out into the arena, memory freed in stream order
int serve_retire(gpga_server *h, int b)
{
    Fleet *f = h->f;
    const int Nmax = f->Nmax;
    for (int i = 0; i < f->cap; ++i) {
        Slot &s = f->slots[i];
        if (!s.used || s.since < 0 || s.since > h->tick - 2 || !f->h_st[b][i].done) continue;
        int rc = fleet_rescore(f, i);
        if (rc) return rc;
        GPGA_CUDA(cudaMemcpyAsync(h->arena_lab + (size_t)i * Nmax, s.m.canon,
                                  (size_t)s.N * sizeof(int32_t), cudaMemcpyDeviceToHost, f->stream));
        GPGA_CUDA(cudaMemcpyAsync(h->arena_L + i, s.m.Lbest, sizeof(double),
                                  cudaMemcpyDeviceToHost, f->stream));
        h->out[b].push_back({s.id, i, s.N, f->h_st[b][i].gen, s.t_submit, s.t_admit});
        h->in_use -= s.m.bytes;
        fleet_release_run(f, i);
    }
    return GPGA_OK;
}

int serve_admit(gpga_server *h, int b)
{
    Fleet *f = h->f;
    // matrices of this tick's admissions go through pinned staging buffer b
    // (free: tick - 2, its last user, has finished)
    size_t staged = 0;
    while (!h->queue.empty()) {
        gpga_server::Req &q = h->queue.front();
        int slot = -1;
        for (int i = 0; i < f->cap; ++i)
            if (!f->slots[i].used) {
                slot = i;
                break;
            }
        if (slot < 0) break;
        const size_t need = run_bytes(f, q.N, nullptr, nullptr);
        if (h->in_use + need > h->budget) break;
        size_t free_b = 0, total_b = 0;
        GPGA_CUDA(cudaMemGetInfo(&free_b, &total_b));
        if (free_b < need + h->reserve) break;
        const size_t nn = (size_t)q.N * q.N;
        if (staged + nn > h->stage_cap[b]) {
            if (staged) break; // this tick's buffer is full: admit the rest next tick
            if (h->stage[b]) cudaFreeHost(h->stage[b]);
            h->stage[b] = nullptr;
            h->stage_cap[b] = 0;
            const size_t want = std::max(nn, (size_t)1 << 24);
            GPGA_CUDA(cudaMallocHost((void **)&h->stage[b], want * sizeof(double)));
            h->stage_cap[b] = want;
        }
        double *src = h->stage[b] + staged;
        memcpy(src, q.C.data(), nn * sizeof(double));
        staged += nn;
        int rc = fleet_alloc_run(f, slot, q.N);
        if (rc) return rc;
        Slot &s = f->slots[slot];
        s.used = true;
        s.since = -1;
        s.seed = q.seed;
        s.id = q.id;
        s.t_submit = q.t_submit;
        s.t_admit = std::chrono::steady_clock::now();
        GPGA_CUDA(cudaMemcpyAsync(s.m.C64, src, nn * sizeof(double), cudaMemcpyHostToDevice,
                                  f->stream));
        rc = fleet_start(f, slot, nullptr, q.N, nullptr, q.N, q.seed);
        if (rc) return rc;
        h->in_use += need;
        h->running[q.id] = slot;
        h->queue.pop_front();
    }
    return GPGA_OK;
}

} // namespace

extern "C" {

GPGA_API int serve_create(const gpga_params *p, int max_runs, int max_n, size_t mem_budget,
                          void *stream, gpga_server **out)
{
    if (!out) return set_error(GPGA_ERR_ARG, "serve_create: out is NULL");
    *out = nullptr;
    gpga_server *h = new (std::nothrow) gpga_server;
    if (!h) return set_error(GPGA_ERR_OOM, "serve_create: host allocation");
    int rc = fleet_create(p, max_runs, max_n, stream, &h->f);
    if (rc) {
        h->f = nullptr;
        serve_release(h);
        return rc;
    }
    h->f->retune = true;
    const int Nmax = h->f->Nmax;
    bool ok = cudaMallocHost((void **)&h->arena_lab, (size_t)max_runs * Nmax * sizeof(int32_t)) ==
                  cudaSuccess &&
              cudaMallocHost((void **)&h->arena_L, (size_t)max_runs * sizeof(double)) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaEventCreateWithFlags(&h->ev_status[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->ev_out[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreate(&h->ev_g0[b]) == cudaSuccess &&
             cudaEventCreate(&h->ev_g1[b]) == cudaSuccess;
    if (!ok) {
        serve_release(h);
        return set_error(GPGA_ERR_OOM, "serve_create: pinned memory or events");
    }
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        serve_release(h);
        return cuda_error(e, "serve_create: cudaMemGetInfo", __FILE__, __LINE__);
    }
    h->reserve = std::min<size_t>((size_t)1 << 30, free_b / 10);
    h->budget = mem_budget ? mem_budget : (free_b > h->reserve ? free_b - h->reserve : 0);
    *out = h;
    return GPGA_OK;
}

GPGA_API int serve_submit(gpga_server *h, const double *C, int N, uint64_t seed, long long *id)
{
    if (!h || !C || !id) return set_error(GPGA_ERR_ARG, "serve_submit: NULL argument");
    if (N < 2 || N > h->f->Nmax)
        return set_error(GPGA_ERR_ARG, "serve_submit: N=%d outside [2, %d]", N, h->f->Nmax);
    gpga_server::Req q;
    q.id = h->next_id++;
    q.N = N;
    q.seed = seed;
    try {
        q.C.assign(C, C + (size_t)N * N);
    } catch (...) {
        return set_error(GPGA_ERR_OOM, "serve_submit: host allocation");
    }
    q.t_submit = std::chrono::steady_clock::now();
    h->queue.push_back(std::move(q));
    *id = h->queue.back().id;
    return GPGA_OK;
}

GPGA_API int serve_tick(gpga_server *h, int generations, int *active, int *queued)
{
    if (!h) return set_error(GPGA_ERR_ARG, "serve_tick: NULL handle");
    if (generations < 0) return set_error(GPGA_ERR_ARG, "serve_tick: generations < 0");
    Fleet *f = h->f;
    const int b = (int)(h->tick & 1), pb = b ^ 1;
    const auto t0 = std::chrono::steady_clock::now();
    // tick - 2 finished (its status is in mirror b); tick - 1's copy-out landed
    if (h->tick >= 2) GPGA_CUDA(cudaEventSynchronize(h->ev_status[b]));
    if (h->tick >= 1) GPGA_CUDA(cudaEventSynchronize(h->ev_out[pb]));
    const auto t1 = std::chrono::steady_clock::now();
    if (h->g_timed[b]) { // tick - 2's generation graphs
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev_g0[b], h->ev_g1[b]) == cudaSuccess) h->gpu_ms += ms;
        h->g_timed[b] = false;
    }
    serve_collect(h, pb);
    int rc = h->tick >= 2 ? serve_retire(h, b) : GPGA_OK;
    if (!rc) GPGA_CUDA(cudaEventRecord(h->ev_out[b], f->stream));
    if (!rc) rc = serve_admit(h, b);
    if (!rc) rc = fleet_upload(f, b, h->tick);
    if (rc) return rc;
    if (generations > 0 && f->nactive > 0) {
        // (the first launch, and the first after the work doubled, tunes the
        // launch shape and waits for the GPU)
        GPGA_CUDA(cudaEventRecord(h->ev_g0[b], f->stream));
        rc = fleet_step(f, generations);
        if (rc) return rc;
        GPGA_CUDA(cudaEventRecord(h->ev_g1[b], f->stream));
        h->g_timed[b] = true;
        h->gens += generations;
        h->item_gens += (long long)generations * f->nitems;
    }
    GPGA_CUDA(cudaMemcpyAsync(f->h_st[b], f->d_st, (size_t)f->cap * sizeof(DevState),
                              cudaMemcpyDeviceToHost, f->stream));
    GPGA_CUDA(cudaEventRecord(h->ev_status[b], f->stream));
    ++h->tick;
    const auto t2 = std::chrono::steady_clock::now();
    h->host_wait_s += std::chrono::duration<double>(t1 - t0).count();
    h->host_work_s += std::chrono::duration<double>(t2 - t1).count();
    if (active) *active = f->nactive;
    if (queued) *queued = (int)h->queue.size();
    return GPGA_OK;
}

GPGA_API int serve_result(gpga_server *h, long long id, int32_t *labels, double *L,
                          int *generation, double *times)
{
    if (!h) return set_error(GPGA_ERR_ARG, "serve_result: NULL handle");
    auto it = h->results.find(id);
    if (it == h->results.end()) {
        if (h->running.count(id)) return 0;
        for (const auto &q : h->queue)
            if (q.id == id) return 0;
        return set_error(GPGA_ERR_ARG, "serve_result: unknown or already collected id %lld", id);
    }
    const gpga_server::Result &r = it->second;
    if (labels) memcpy(labels, r.labels.data(), r.labels.size() * sizeof(int32_t));
    if (L) *L = r.L;
    if (generation) *generation = r.gen;
    if (times) {
        times[0] = r.queue_s;
        times[1] = r.run_s;
    }
    h->results.erase(it);
    return 1;
}

GPGA_API int serve_stats(gpga_server *h, size_t *bytes_in_use, size_t *budget,
                         long long *completed, int *warps_per_cta, int *ctas, double *timing)
{
    if (!h) return set_error(GPGA_ERR_ARG, "serve_stats: NULL handle");
    if (bytes_in_use) *bytes_in_use = h->in_use;
    if (budget) *budget = h->budget;
    if (completed) *completed = h->completed;
    if (warps_per_cta) *warps_per_cta = h->f->warps;
    if (ctas) *ctas = h->f->ctas;
    if (timing) {
        timing[0] = (double)h->tick;
        timing[1] = h->host_wait_s;
        timing[2] = h->host_work_s;
        timing[3] = h->gpu_ms;
        timing[4] = (double)h->gens;
        timing[5] = (double)h->item_gens;
    }
    return GPGA_OK;
}

GPGA_API int serve_free(gpga_server *h)
{
    serve_release(h);
    return GPGA_OK;
}

} // extern "C"
