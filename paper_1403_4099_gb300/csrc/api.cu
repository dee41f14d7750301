// api.cu -- the extern "C" boundary of libgpga.so (declared in include/gpga.h):
// argument checks, status codes, the GA handle and its device memory, and the
// per-generation launch sequence, captured once into CUDA graphs.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>

#include "gpga_internal.cuh"
#include "score_tc.cuh"

namespace gpga {

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

static std::atomic<long long> g_wait_budget{1ll << 32};

long long wait_budget() { return g_wait_budget.load(std::memory_order_relaxed); }

int device_error_status(int err_word, const char *what)
{
    if (err_word & 4)
        return set_error(GPGA_ERR_TIMEOUT,
                         "%s: a bounded device wait gave up (the affected fitness values are NaN)",
                         what);
    if (err_word & 1)
        return set_error(GPGA_ERR_ARG, "%s: a label lies outside [0, N) (its L is NaN)", what);
    return GPGA_OK;
}

int cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    const int code = (e == cudaErrorMemoryAllocation) ? GPGA_ERR_OOM : GPGA_ERR_CUDA;
    return set_error(code, "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_params(const gpga_params *p, int N)
{
    if (!p) return set_error(GPGA_ERR_ARG, "params is NULL");
    if (N < 2 || N > GPGA_MAX_N) return set_error(GPGA_ERR_ARG, "N=%d outside [2, %d]", N, GPGA_MAX_N);
    if (p->P < 2 || p->P > GPGA_MAX_P) return set_error(GPGA_ERR_ARG, "P=%d outside [2, %d]", p->P, GPGA_MAX_P);
    if (p->elite < 0 || p->elite >= p->P) return set_error(GPGA_ERR_ARG, "elite=%d outside [0, P)", p->elite);
    if (p->max_gens < 0) return set_error(GPGA_ERR_ARG, "max_gens < 0");
    if (p->scaling != GPGA_SCALING_RANK && p->scaling != GPGA_SCALING_PROP)
        return set_error(GPGA_ERR_ARG, "unknown scaling %d", p->scaling);
    if (p->form != GPGA_FORM_PLAIN && p->form != GPGA_FORM_TENSOR && p->form != GPGA_FORM_GATHER)
        return set_error(GPGA_ERR_ARG, "unknown form %d", p->form);
    if (p->init != GPGA_INIT_UNIFORM && p->init != GPGA_INIT_THRESHOLD)
        return set_error(GPGA_ERR_ARG, "unknown init %d", p->init);
    if (p->init_labels < 0 || p->init_labels > N) return set_error(GPGA_ERR_ARG, "init_labels outside [0, N]");
    if (!(p->pc >= 0.0 && p->pc <= 1.0) || !(p->pkb >= 0.0 && p->pkb <= 1.0) ||
        !(p->pm >= 0.0 && p->pm <= 1.0))
        return set_error(GPGA_ERR_ARG, "probabilities must lie in [0, 1]");
    if (p->init == GPGA_INIT_THRESHOLD && !(p->tau_hi >= p->tau_lo))
        return set_error(GPGA_ERR_ARG, "tau_hi < tau_lo");
    return GPGA_OK;
}

// kernels with large dynamic shared memory: raise their limit once per device
int prepare_device()
{
    static std::mutex mu;
    static bool ready[64] = {false};
    int dev = 0;
    GPGA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(GPGA_ERR_ARG, "device ordinal %d unsupported", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (ready[dev]) return GPGA_OK;
    int maxsmem = 0;
    GPGA_CUDA(cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int rc = prepare_score_kernels(maxsmem);
    if (!rc) rc = prepare_ga_kernels(maxsmem);
    if (!rc) rc = prepare_init_kernels(maxsmem);
    if (!rc) rc = prepare_tc_kernels(maxsmem);
    if (!rc) rc = prepare_gather_kernels(maxsmem);
    if (!rc) rc = prepare_corr_kernels(maxsmem);
    if (!rc) rc = prepare_rmt_tri_kernels(maxsmem);
    if (rc) return rc;
    ready[dev] = true;
    return GPGA_OK;
}

} // namespace gpga

using namespace gpga;

struct gpga_ga {
    int dev = 0;
    int N = 0, Np = 0, P = 0, E = 0, M = 0;
    gpga_params prm{};
    uint64_t seed = 0;
    uint32_t k0 = 0, k1 = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char *block = nullptr; // one device allocation, carved below
    double *C64 = nullptr;
    float *D32 = nullptr;
    __nv_bfloat16 *Dhi = nullptr, *Dlo = nullptr;
    int32_t *Dfix = nullptr;
    double *logtab = nullptr;
    uint16_t *pop[2] = {nullptr, nullptr};
    double *L = nullptr;
    float *acc = nullptr;
    int32_t *perm = nullptr;
    int *rank = nullptr;
    unsigned *ticket = nullptr;
    uint64_t *rank_prefix = nullptr, *work_prefix = nullptr;
    int32_t *sus_tab = nullptr; // SUS brackets of rank_prefix (P + 1)
    bool tables_ready = false;  // rank_prefix and sus_tab depend on P and E only
    DevState *st = nullptr;
    double *hist = nullptr;
    uint16_t *ring = nullptr;
    unsigned long long *ts = nullptr;
    unsigned long long *pairs = nullptr;
    unsigned long long *clusters = nullptr;
    int32_t *mst_order = nullptr, *mst_from = nullptr;
    double *mst_w = nullptr;
    int *err = nullptr;
    int *diag = nullptr;
    int32_t *canon = nullptr;
    double *Lbest = nullptr;
    ScoreTab tab{}; // gather form: per-individual score tables (delta scoring)
    TcWork tc{};
    cudaGraphExec_t g1 = nullptr, gU = nullptr;
    int U = 8;
    // profile: 5 event boundaries per generation, one set per graph shape
    static constexpr int NEV = 5;
    cudaEvent_t evU[8][NEV] = {};
    cudaEvent_t ev1[1][NEV] = {};
    int last_graph = 0; // generations in the most recently launched graph
};

namespace {

struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(char *b) : base(b) {}
    template <typename T> T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

size_t carve(gpga_ga *h, char *base)
{
    Carver c(base);
    const size_t N = h->N, Np = h->Np, P = h->P, G = (size_t)h->prm.max_gens + 1;
    h->C64 = c.take<double>(N * N);
    h->D32 = c.take<float>(Np * Np);
    h->Dhi = c.take<__nv_bfloat16>(Np * Np);
    h->Dlo = c.take<__nv_bfloat16>(Np * Np);
    h->Dfix = c.take<int32_t>(Np * Np);
    h->logtab = c.take<double>(logtab_len(h->N));
    h->pop[0] = c.take<uint16_t>(P * Np);
    h->pop[1] = c.take<uint16_t>(P * Np);
    h->L = c.take<double>(P);
    h->acc = c.take<float>(P * Np);
    h->perm = c.take<int32_t>(P);
    h->rank = c.take<int>(P);
    h->ticket = c.take<unsigned>(TICKETS);
    h->rank_prefix = c.take<uint64_t>(P);
    h->work_prefix = c.take<uint64_t>(P);
    h->sus_tab = c.take<int32_t>(P + 1);
    h->st = c.take<DevState>(1);
    h->hist = c.take<double>(G);
    h->ring = h->prm.record ? c.take<uint16_t>(G * N) : nullptr;
    h->ts = h->prm.record ? c.take<unsigned long long>(G + 1) : nullptr;
    h->pairs = h->prm.record ? c.take<unsigned long long>(G) : nullptr;
    h->clusters = h->prm.record ? c.take<unsigned long long>(G) : nullptr;
    h->mst_order = c.take<int32_t>(N);
    h->mst_from = c.take<int32_t>(N);
    h->mst_w = c.take<double>(N);
    h->err = c.take<int>(1);
    h->diag = c.take<int>(1);
    h->canon = c.take<int32_t>(N);
    h->Lbest = c.take<double>(1);
    if (h->prm.form == GPGA_FORM_TENSOR) tc_carve(&h->tc, h->N, h->Np, h->P, &c.off, c.base);
    if (h->prm.form == GPGA_FORM_GATHER && uses_delta(h->N)) {
        h->tab.ldt = (int)Np;
        for (int b = 0; b < 2; ++b) {
            h->tab.d[b] = c.take<long long>(P * Np);
            h->tab.lf[b] = c.take<long long>(P);
            h->tab.np[b] = c.take<long long>(P);
        }
    }
    return c.off + 256;
}

static int mark(gpga_ga *h, cudaEvent_t *evs, int k);

int enqueue_score(gpga_ga *h, int sel_off, cudaEvent_t *evs = nullptr)
{
    const uint16_t *lab2[2] = {h->pop[0], h->pop[1]};
    const int tensor = h->prm.form == GPGA_FORM_TENSOR;
    int rc;
    if (h->prm.form == GPGA_FORM_GATHER) {
        rc = launch_gather_score<uint16_t>(lab2, h->Np, sel_off, h->P, h->N, h->Np, h->Dfix,
                                           h->diag, h->logtab, h->L, h->err, h->st, h->pairs,
                                           h->tab, h->stream);
        if (!rc) rc = mark(h, evs, 2);
        if (!rc) rc = mark(h, evs, 3);
        return rc;
    }
    if (tensor) { // columns + tcgen05 contraction, then the assembly
        rc = tc_contract<uint16_t>(&h->tc, h->Dhi, h->Dlo, h->Np, lab2, h->Np, sel_off, h->P,
                                   h->N, h->err, h->st, h->pairs, h->clusters, h->stream);
        if (!rc) rc = mark(h, evs, 2);
        if (!rc)
            rc = tc_finish<uint16_t>(&h->tc, lab2, h->Np, sel_off, h->P, h->N, h->logtab, h->L,
                                     h->err, h->st, h->stream);
        if (!rc) rc = mark(h, evs, 3);
        return rc;
    }
        rc = launch_pair_plain<uint16_t>(h->D32, h->Np, lab2, h->Np, sel_off, h->P, h->N, h->acc,
                                         h->st, h->stream);
    if (!rc) rc = mark(h, evs, 2);
    if (!rc)
        rc = launch_assemble<uint16_t>(lab2, h->Np, sel_off, h->acc, h->Np, h->D32, 0, h->P, h->N,
                                       h->logtab, h->L, h->err, h->st, h->pairs, h->stream);
    if (!rc) rc = mark(h, evs, 3);
    return rc;
}

SelectCfg select_cfg(const gpga_ga *h, int gen_off)
{
    SelectCfg c;
    c.P = h->P;
    c.E = h->E;
    c.M = h->M;
    c.N = h->N;
    c.ldp = h->Np;
    c.scaling = h->prm.scaling;
    c.max_gens = h->prm.max_gens;
    c.stall_gens = h->prm.stall_gens;
    c.tol = h->prm.tol;
    c.k0 = h->k0;
    c.k1 = h->k1;
    c.gen_off = gen_off;
    c.record = h->prm.record;
    return c;
}

int enqueue_select(gpga_ga *h, int gen_off)
{
    const uint16_t *pop2[2] = {h->pop[0], h->pop[1]};
    return launch_select<uint16_t>(h->L, select_cfg(h, gen_off), h->rank, h->perm,
                                   h->work_prefix, h->ticket, h->st, h->hist, pop2, h->ring,
                                   h->ts, h->stream);
}

// event boundaries 0..4 of a generation: before evolve, after evolve (or the
// fused kernel), after the main scoring kernel, after assembly, after selection.
// profile 1 records only the boundaries of the dominant kernel, profile 2 all.
static bool marked(const gpga_ga *h, int k)
{
    if (h->prm.profile >= 2) return true;
    if (h->prm.form == GPGA_FORM_GATHER) return k == 0 || k == 1;
    return k == 1 || k == 2;
}

static int mark(gpga_ga *h, cudaEvent_t *evs, int k)
{
    if (!evs || !marked(h, k)) return GPGA_OK;
    GPGA_CUDA(cudaEventRecordWithFlags(evs[k], h->stream, cudaEventRecordExternal));
    return GPGA_OK;
}

// after_kernel: the node captured last before this generation is a kernel
// (the selection; not the start of the graph, not an event). The fused
// generation kernel is then launched as a programmatic dependent of it.
int enqueue_generation(gpga_ga *h, cudaEvent_t *evs, bool after_kernel)
{
    EvolveCfg e;
    e.P = h->P;
    e.E = h->E;
    e.M = h->M;
    e.N = h->N;
    e.ldp = h->Np;
    e.thr_pc = prob_threshold(h->prm.pc);
    e.thr_pkb = prob_threshold(h->prm.pkb);
    set_mutation(&e, h->prm.pm);
    set_sus_divisor(&e, h->M);
    e.k0 = h->k0;
    e.k1 = h->k1;
    e.gen = 0;
    e.sus_tab = h->prm.scaling == GPGA_SCALING_PROP ? nullptr : h->sus_tab;
    const uint16_t *pop2[2] = {h->pop[0], h->pop[1]};
    uint16_t *next2[2] = {h->pop[1], h->pop[0]};
    const uint64_t *prefix = h->prm.scaling == GPGA_SCALING_PROP ? h->work_prefix : h->rank_prefix;
    int rc = mark(h, evs, 0);
    if (h->prm.form == GPGA_FORM_GATHER) {
        // selection, crossover, mutation, replacement and scoring in one kernel
        const bool pdl_gen = after_kernel && !(evs && marked(h, 0));
        if (!rc)
            rc = launch_gather_generation(pop2, next2, e, h->perm, prefix, h->Np, h->Dfix,
                                          h->diag, h->logtab, h->L, h->st, h->pairs, h->tab,
                                          pdl_gen, h->stream);
        if (!rc) rc = mark(h, evs, 1);
        if (!rc) rc = mark(h, evs, 2);
        if (!rc) rc = mark(h, evs, 3);
    } else {
        if (!rc) rc = launch_evolve<uint16_t>(pop2, next2, e, h->perm, prefix, nullptr, h->st, h->stream);
        if (!rc) rc = mark(h, evs, 1);
        if (!rc) rc = enqueue_score(h, 1, evs);
    }
    if (!rc) rc = enqueue_select(h, 1);
    if (!rc) rc = mark(h, evs, 4);
    return rc;
}

int enqueue_start(gpga_ga *h, const double *C)
{
    const size_t nn = (size_t)h->N * h->N * sizeof(double);
    GPGA_CUDA(cudaMemcpyAsync(h->C64, C, nn, cudaMemcpyDeviceToDevice, h->stream));
    GPGA_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    GPGA_CUDA(cudaMemsetAsync(h->rank, 0, (size_t)h->P * sizeof(int), h->stream));
    GPGA_CUDA(cudaMemsetAsync(h->ticket, 0, TICKETS * sizeof(unsigned), h->stream));
    GPGA_CUDA(cudaMemsetAsync(h->diag, 0, sizeof(int), h->stream));
    if (h->pairs)
        GPGA_CUDA(cudaMemsetAsync(h->pairs, 0, ((size_t)h->prm.max_gens + 1) * sizeof(unsigned long long),
                                  h->stream));
    if (h->clusters)
        GPGA_CUDA(cudaMemsetAsync(h->clusters, 0,
                                  ((size_t)h->prm.max_gens + 1) * sizeof(unsigned long long), h->stream));
    int rc = launch_state_init(h->st, h->ts, h->k0, h->k1, h->stream);
    if (rc) return rc;
    rc = launch_prep_d(h->C64, h->N, h->N, h->Np, h->D32, h->Dhi, h->Dlo, h->Dfix, h->logtab,
                       h->diag, h->stream);
    if (rc) return rc;
    if (!h->tables_ready) { // once per handle: a reset keeps P and E
        rc = rank_prefix_table(h->rank_prefix, h->P, h->M, h->sus_tab, h->stream);
        if (rc) return rc;
        h->tables_ready = true;
    }
    if (h->prm.init == GPGA_INIT_THRESHOLD) {
        rc = launch_mst(h->C64, h->N, h->mst_order, h->mst_from, h->mst_w, h->stream);
        if (rc) return rc;
        rc = launch_init_threshold<uint16_t>(h->pop[0], h->Np, h->P, h->N, h->mst_order,
                                             h->mst_from, h->mst_w, h->prm.tau_lo, h->prm.tau_hi,
                                             h->k0, h->k1, h->stream);
    } else {
        const int K0 = h->prm.init_labels > 0 ? h->prm.init_labels : h->N;
        rc = launch_init_uniform<uint16_t>(h->pop[0], h->Np, h->P, h->N, K0, h->k0, h->k1,
                                           h->stream);
    }
    if (rc) return rc;
    GPGA_CUDA(cudaMemsetAsync(h->pop[1], 0, (size_t)h->P * h->Np * sizeof(uint16_t), h->stream));
    rc = enqueue_score(h, 0);
    if (rc) return rc;
    return enqueue_select(h, 0);
}

int build_graph(gpga_ga *h, int gens, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    cudaEvent_t(*evs)[gpga_ga::NEV] = gens == 1 ? h->ev1 : h->evU;
    if (h->prm.profile) {
        for (int k = 0; k < gens; ++k)
            for (int e = 0; e < gpga_ga::NEV; ++e)
                if (!evs[k][e]) GPGA_CUDA(cudaEventCreate(&evs[k][e]));
    }
    GPGA_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = GPGA_OK;
    // profile 1 times the dominant kernel of the graph's first generation only
    // (each event node costs about 2 us of the step); profile 2 every stage of
    // every generation
    bool after_kernel = false;
    for (int k = 0; k < gens && rc == GPGA_OK; ++k) {
        cudaEvent_t *ek =
            (h->prm.profile >= 2 || (h->prm.profile == 1 && k == 0)) ? evs[k] : nullptr;
        rc = enqueue_generation(h, ek, after_kernel);
        after_kernel = !(ek && marked(h, 4));
    }
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    return GPGA_OK;
}

} // namespace

extern "C" {

GPGA_API const char *gpga_last_error(void) { return g_err; }

GPGA_API int gpga_set_wait_budget(long long cycles)
{
    g_err[0] = 0;
    g_wait_budget.store(cycles < 0 ? (1ll << 32) : cycles, std::memory_order_relaxed);
    return GPGA_OK;
}

GPGA_API int gpga_default_params(gpga_params *p)
{
    if (!p) return set_error(GPGA_ERR_ARG, "params is NULL");
    memset(p, 0, sizeof *p);
    p->P = 1000;
    p->elite = 10;
    p->max_gens = 400;
    p->stall_gens = 50;
    p->tol = 1e-5;
    p->pc = 0.9;
    p->pkb = 0.9;
    p->pm = 0.01;
    p->scaling = GPGA_SCALING_RANK;
    p->form = GPGA_FORM_PLAIN;
    p->init = GPGA_INIT_UNIFORM;
    p->init_labels = 0;
    p->tau_lo = 0.05;
    p->tau_hi = 0.6;
    p->record = 0;
    return GPGA_OK;
}

GPGA_API int cluster_corr(const double *R, int T, int N, int ld, double *C, void *stream)
{
    g_err[0] = 0;
    if (!R || !C) return set_error(GPGA_ERR_ARG, "cluster_corr: NULL pointer");
    if (T < 2 || N < 2 || N > GPGA_MAX_N || ld < N)
        return set_error(GPGA_ERR_ARG, "cluster_corr: T=%d N=%d ld=%d out of range", T, N, ld);
    int rc = prepare_device();
    if (rc) return rc;
    return corr_run(R, T, N, ld, C, (cudaStream_t)stream);
}

GPGA_API int cluster_corr_ewma(const double *R, int T, int N, int ld, double lambda, double *C,
                               void *stream)
{
    g_err[0] = 0;
    if (!R || !C) return set_error(GPGA_ERR_ARG, "cluster_corr_ewma: NULL pointer");
    if (T < 2 || N < 2 || N > GPGA_MAX_N || ld < N)
        return set_error(GPGA_ERR_ARG, "cluster_corr_ewma: T=%d N=%d ld=%d out of range", T, N, ld);
    if (!(lambda > 0.0 && lambda <= 1.0))
        return set_error(GPGA_ERR_ARG, "cluster_corr_ewma: lambda must lie in (0, 1]");
    int rc = prepare_device();
    if (rc) return rc;
    return corr_run_weighted(R, T, N, ld, lambda, C, (cudaStream_t)stream);
}

GPGA_API int corr_remove_market(double *C, int N, int max_iters, double *lambda1, int *iters,
                                void *stream)
{
    g_err[0] = 0;
    if (!C) return set_error(GPGA_ERR_ARG, "corr_remove_market: NULL pointer");
    if (N < 2 || N > GPGA_MAX_N || max_iters < 1)
        return set_error(GPGA_ERR_ARG, "corr_remove_market: N=%d max_iters=%d", N, max_iters);
    int rc = prepare_device();
    if (rc) return rc;
    return market_remove(C, N, max_iters, lambda1, iters, (cudaStream_t)stream);
}

GPGA_API int corr_clean_rmt(double *C, int batch, int N, double T, double *eigvals, int *n_noise,
                           int *sweeps, void *stream)
{
    g_err[0] = 0;
    if (!C) return set_error(GPGA_ERR_ARG, "corr_clean_rmt: NULL pointer");
    if (batch < 1 || batch > 65535 || N < 2 || N > GPGA_MAX_N || !(T > 0.0) || !isfinite(T))
        return set_error(GPGA_ERR_ARG, "corr_clean_rmt: batch=%d N=%d T=%g out of range", batch, N,
                         T);
    if (!is_device_ptr(C) || (eigvals && !is_device_ptr(eigvals)))
        return set_error(GPGA_ERR_ARG, "corr_clean_rmt: C and eigvals must be device memory");
    int rc = prepare_device();
    if (rc) return rc;
    return rmt_clean(C, batch, N, T, eigvals, n_noise, sweeps, (cudaStream_t)stream);
}

GPGA_API int ga_score(const int32_t *labels, int P, int N, int ld, const double *C, double *L,
                      int form, void *stream)
{
    g_err[0] = 0;
    if (!labels || !C || !L) return set_error(GPGA_ERR_ARG, "ga_score: NULL pointer");
    if (N < 2 || N > GPGA_MAX_N || P < 1 || P > (1 << 24) || ld < N)
        return set_error(GPGA_ERR_ARG, "ga_score: P=%d N=%d ld=%d out of range", P, N, ld);
    if (form != GPGA_FORM_PLAIN && form != GPGA_FORM_TENSOR && form != GPGA_FORM_GATHER)
        return set_error(GPGA_ERR_ARG, "ga_score: unknown form %d", form);
    int rc = prepare_device();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int Np = pad_n(N);
    const size_t b_d = (size_t)Np * Np * sizeof(float);
    const size_t b_h = (size_t)Np * Np * sizeof(__nv_bfloat16);
    const size_t b_acc = (size_t)P * Np * sizeof(float);
    const size_t b_log = logtab_len(N) * sizeof(double);
    const size_t b_fix = (size_t)Np * Np * sizeof(int32_t);
    size_t tc_bytes = 0;
    if (form == GPGA_FORM_TENSOR) tc_bytes = tc_scratch_bytes(N, Np, P);
    const size_t total = b_d + 2 * b_h + b_fix + b_acc + b_log + tc_bytes + 4096;
    char *ws = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&ws, total, s));
    Carver c(ws);
    float *D32 = c.take<float>((size_t)Np * Np);
    __nv_bfloat16 *Dhi = c.take<__nv_bfloat16>((size_t)Np * Np);
    __nv_bfloat16 *Dlo = c.take<__nv_bfloat16>((size_t)Np * Np);
    float *acc = c.take<float>((size_t)P * Np);
    int32_t *Dfix = c.take<int32_t>((size_t)Np * Np);
    double *logtab = c.take<double>(logtab_len(N));
    int *err = c.take<int>(2); // [0] label error, [1] diagonal flag
    TcWork tc{};
    if (form == GPGA_FORM_TENSOR) tc_carve(&tc, N, Np, P, &c.off, ws);
    int herr = 0;
    do {
        if (cudaMemsetAsync(err, 0, 2 * sizeof(int), s) != cudaSuccess) {
            rc = set_error(GPGA_ERR_CUDA, "ga_score: memset failed");
            break;
        }
        rc = launch_prep_d(C, N, N, Np, D32, form == GPGA_FORM_TENSOR ? Dhi : nullptr, Dlo,
                           form == GPGA_FORM_GATHER ? Dfix : nullptr, logtab, err + 1, s);
        if (rc) break;
        const int32_t *lab2[2] = {labels, labels};
        if (form == GPGA_FORM_GATHER) {
            rc = launch_gather_score<int32_t>(lab2, ld, 0, P, N, Np, Dfix, err + 1, logtab, L, err,
                                              nullptr, nullptr, ScoreTab{}, s);
        } else if (form == GPGA_FORM_TENSOR) {
            rc = tc_contract<int32_t>(&tc, Dhi, Dlo, Np, lab2, ld, 0, P, N, err, nullptr, nullptr,
                                      nullptr, s);
            if (!rc) rc = tc_finish<int32_t>(&tc, lab2, ld, 0, P, N, logtab, L, err, nullptr, s);
        } else {
            rc = launch_pair_plain<int32_t>(D32, Np, lab2, ld, 0, P, N, acc, nullptr, s);
            if (rc) break;
            rc = launch_assemble<int32_t>(lab2, ld, 0, acc, Np, D32, 0, P, N, logtab, L, err,
                                          nullptr, nullptr, s);
        }
        if (rc) break;
        cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "ga_score sync", __FILE__, __LINE__);
    } while (0);
    cudaFreeAsync(ws, s);
    if (rc == GPGA_OK) rc = device_error_status(herr, "ga_score");
    return rc;
}

GPGA_API int ga_evolve(const int32_t *pop, const double *L, int N, const gpga_params *p,
                       uint64_t seed, int generation, int32_t *next, int32_t *perm,
                       int32_t *parents, void *stream)
{
    g_err[0] = 0;
    if (!pop || !L || !next) return set_error(GPGA_ERR_ARG, "ga_evolve: NULL pointer");
    int rc = check_params(p, N);
    if (rc) return rc;
    if (generation < 0) return set_error(GPGA_ERR_ARG, "ga_evolve: generation < 0");
    rc = prepare_device();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int P = p->P, E = p->elite, M = P - E;
    const size_t total = (size_t)P * (2 * sizeof(uint64_t) + 3 * sizeof(int32_t)) + 2048 +
                         TICKETS * sizeof(unsigned);
    char *ws = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&ws, total, s));
    Carver c(ws);
    uint64_t *rpre = c.take<uint64_t>(P);
    uint64_t *wpre = c.take<uint64_t>(P);
    int *rank = c.take<int>(P);
    unsigned *ticket = c.take<unsigned>(TICKETS);
    int32_t *pm_ = perm ? perm : c.take<int32_t>(P);
    do {
        if (cudaMemsetAsync(rank, 0, (size_t)P * sizeof(int), s) != cudaSuccess ||
            cudaMemsetAsync(ticket, 0, TICKETS * sizeof(unsigned), s) != cudaSuccess) {
            rc = set_error(GPGA_ERR_CUDA, "ga_evolve: memset failed");
            break;
        }
        rc = rank_prefix_table(rpre, P, M, nullptr, s);
        if (rc) break;
        SelectCfg sc;
        sc.P = P;
        sc.E = E;
        sc.M = M;
        sc.N = N;
        sc.ldp = N;
        sc.scaling = p->scaling;
        sc.max_gens = p->max_gens;
        sc.stall_gens = p->stall_gens;
        sc.tol = p->tol;
        sc.k0 = (uint32_t)seed;
        sc.k1 = (uint32_t)(seed >> 32);
        sc.gen_off = generation;
        sc.record = 0;
        rc = launch_select<int32_t>(L, sc, rank, pm_, wpre, ticket, nullptr, nullptr, nullptr,
                                    nullptr, nullptr, s);
        if (rc) break;
        EvolveCfg e;
        e.P = P;
        e.E = E;
        e.M = M;
        e.N = N;
        e.ldp = N;
        e.thr_pc = prob_threshold(p->pc);
        e.thr_pkb = prob_threshold(p->pkb);
        set_mutation(&e, p->pm);
        set_sus_divisor(&e, M);
        e.k0 = sc.k0;
        e.k1 = sc.k1;
        e.gen = generation;
        e.sus_tab = nullptr; // the general search (no bracket table here)
        const int32_t *pop2[2] = {pop, pop};
        int32_t *next2[2] = {next, next};
        rc = launch_evolve<int32_t>(pop2, next2, e, pm_,
                                    p->scaling == GPGA_SCALING_PROP ? wpre : rpre, parents,
                                    nullptr, s);
    } while (0);
    cudaFreeAsync(ws, s);
    return rc;
}

GPGA_API int ga_init(const double *C, int N, const gpga_params *p, uint64_t seed, void *stream,
                     gpga_ga **out)
{
    g_err[0] = 0;
    if (!out) return set_error(GPGA_ERR_ARG, "ga_init: out is NULL");
    *out = nullptr;
    if (!C) return set_error(GPGA_ERR_ARG, "ga_init: C is NULL");
    int rc = check_params(p, N);
    if (rc) return rc;
    rc = prepare_device();
    if (rc) return rc;
    gpga_ga *h = new (std::nothrow) gpga_ga();
    if (!h) return set_error(GPGA_ERR_OOM, "ga_init: host allocation failed");
    cudaGetDevice(&h->dev);
    h->N = N;
    h->Np = pad_n(N);
    h->P = p->P;
    h->E = p->elite;
    h->M = p->P - p->elite;
    h->prm = *p;
    h->seed = seed;
    h->k0 = (uint32_t)seed;
    h->k1 = (uint32_t)(seed >> 32);
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return set_error(GPGA_ERR_CUDA, "ga_init: stream creation failed");
        }
        h->own_stream = true;
    }
    const size_t bytes = carve(h, nullptr);
    cudaError_t e = cudaMallocAsync((void **)&h->block, bytes, h->stream);
    if (e != cudaSuccess) {
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return cuda_error(e, "ga_init: device allocation", __FILE__, __LINE__);
    }
    carve(h, h->block);
    rc = enqueue_start(h, C);
    if (rc) {
        ga_free(h);
        return rc;
    }
    *out = h;
    return GPGA_OK;
}

GPGA_API int ga_reset(gpga_ga *h, const double *C, uint64_t seed)
{
    g_err[0] = 0;
    if (!h || !C) return set_error(GPGA_ERR_ARG, "ga_reset: NULL argument");
    h->seed = seed;
    h->k0 = (uint32_t)seed;
    h->k1 = (uint32_t)(seed >> 32);
    // the captured graphs stay valid: the key and the generation live in device state
    return enqueue_start(h, C);
}

GPGA_API int ga_step(gpga_ga *h, int generations, int *done)
{
    g_err[0] = 0;
    if (!h) return set_error(GPGA_ERR_ARG, "ga_step: NULL handle");
    if (generations < 0) return set_error(GPGA_ERR_ARG, "ga_step: generations < 0");
    int rc;
    if (generations >= h->U && !h->gU) {
        rc = build_graph(h, h->U, &h->gU);
        if (rc) return rc;
    }
    if (generations % h->U && !h->g1) {
        rc = build_graph(h, 1, &h->g1);
        if (rc) return rc;
    }
    int left = generations;
    while (left >= h->U) {
        GPGA_CUDA(cudaGraphLaunch(h->gU, h->stream));
        left -= h->U;
        h->last_graph = h->U;
    }
    while (left-- > 0) {
        GPGA_CUDA(cudaGraphLaunch(h->g1, h->stream));
        h->last_graph = 1;
    }
    if (done) {
        DevState st;
        int herr = 0;
        GPGA_CUDA(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, h->stream));
        GPGA_CUDA(cudaMemcpyAsync(&herr, h->err, sizeof herr, cudaMemcpyDeviceToHost, h->stream));
        GPGA_CUDA(cudaStreamSynchronize(h->stream));
        *done = st.done;
        return device_error_status(herr, "ga_step");
    }
    return GPGA_OK;
}

GPGA_API int ga_best(gpga_ga *h, int32_t *labels, double *L, int *generation)
{
    g_err[0] = 0;
    if (!h) return set_error(GPGA_ERR_ARG, "ga_best: NULL handle");
    int rc = launch_rescore_fp64(h->pop[0], h->pop[1], h->Np, h->st, h->C64, h->N, h->canon,
                                 h->Lbest, h->stream);
    if (rc) return rc;
    if (labels)
        GPGA_CUDA(cudaMemcpyAsync(labels, h->canon, (size_t)h->N * sizeof(int32_t),
                                  is_device_ptr(labels) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyDeviceToHost,
                                  h->stream));
    if (L)
        GPGA_CUDA(cudaMemcpyAsync(L, h->Lbest, sizeof(double),
                                  is_device_ptr(L) ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyDeviceToHost,
                                  h->stream));
    DevState st;
    int herr = 0;
    GPGA_CUDA(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    GPGA_CUDA(cudaMemcpyAsync(&herr, h->err, sizeof herr, cudaMemcpyDeviceToHost, h->stream));
    GPGA_CUDA(cudaStreamSynchronize(h->stream));
    if (generation) *generation = st.gen;
    return device_error_status(herr, "ga_best");
}

GPGA_API int ga_history(gpga_ga *h, double *best_L, int32_t *best_labels, int64_t *t_ns,
                        uint64_t *pairs, uint64_t *clusters, int cap, int *count)
{
    g_err[0] = 0;
    if (!h) return set_error(GPGA_ERR_ARG, "ga_history: NULL handle");
    DevState st;
    GPGA_CUDA(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    GPGA_CUDA(cudaStreamSynchronize(h->stream));
    int n = st.gen + 1;
    if (n > cap) n = cap;
    if (count) *count = n;
    if (n <= 0) return GPGA_OK;
    if (best_L) GPGA_CUDA(cudaMemcpy(best_L, h->hist, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost));
    if (best_labels || t_ns || pairs || clusters) {
        if (!h->prm.record) return set_error(GPGA_ERR_STATE, "ga_history: run created with record = 0");
    }
    if (best_labels) {
        const size_t cnt = (size_t)n * h->N;
        uint16_t *tmp = new (std::nothrow) uint16_t[cnt];
        if (!tmp) return set_error(GPGA_ERR_OOM, "ga_history: host allocation");
        cudaError_t e = cudaMemcpy(tmp, h->ring, cnt * sizeof(uint16_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            for (size_t i = 0; i < cnt; ++i) best_labels[i] = tmp[i];
        delete[] tmp;
        if (e != cudaSuccess) return cuda_error(e, "ga_history copy", __FILE__, __LINE__);
    }
    if (pairs) GPGA_CUDA(cudaMemcpy(pairs, h->pairs, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (clusters)
        GPGA_CUDA(cudaMemcpy(clusters, h->clusters, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (t_ns) GPGA_CUDA(cudaMemcpy(t_ns, h->ts, (size_t)(n + 1) * sizeof(int64_t),
                                   cudaMemcpyDeviceToHost));
    return GPGA_OK;
}

GPGA_API int ga_kernel_times(gpga_ga *h, float *ms, int cap, int *count)
{
    g_err[0] = 0;
    if (!h || !ms) return set_error(GPGA_ERR_ARG, "ga_kernel_times: NULL argument");
    if (!h->prm.profile) return set_error(GPGA_ERR_STATE, "ga_kernel_times: run created with profile = 0");
    GPGA_CUDA(cudaStreamSynchronize(h->stream));
    const int timed = h->prm.profile >= 2 ? h->last_graph : (h->last_graph ? 1 : 0);
    const int n = timed < cap ? timed : cap;
    cudaEvent_t(*evs)[gpga_ga::NEV] = h->last_graph == 1 ? h->ev1 : h->evU;
    for (int k = 0; k < n; ++k)
        for (int e = 0; e < 4; ++e) {
            float t = 0.f;
            const int stage_end = e == 3 ? 4 : e + 1;
            if (marked(h, e) && marked(h, stage_end))
                GPGA_CUDA(cudaEventElapsedTime(&t, evs[k][e], evs[k][stage_end]));
            ms[k * 4 + e] = t;
        }
    if (count) *count = n;
    return GPGA_OK;
}

GPGA_API int ga_population(gpga_ga *h, int32_t *pop, double *L)
{
    g_err[0] = 0;
    if (!h) return set_error(GPGA_ERR_ARG, "ga_population: NULL handle");
    DevState st;
    GPGA_CUDA(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    GPGA_CUDA(cudaStreamSynchronize(h->stream));
    if (pop) {
        const size_t cnt = (size_t)h->P * h->Np;
        uint16_t *tmp = new (std::nothrow) uint16_t[cnt];
        if (!tmp) return set_error(GPGA_ERR_OOM, "ga_population: host allocation");
        cudaError_t e = cudaMemcpy(tmp, h->pop[st.gen & 1], cnt * sizeof(uint16_t),
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            delete[] tmp;
            return cuda_error(e, "ga_population copy", __FILE__, __LINE__);
        }
        int32_t *h32 = new (std::nothrow) int32_t[(size_t)h->P * h->N];
        if (!h32) {
            delete[] tmp;
            return set_error(GPGA_ERR_OOM, "ga_population: host allocation");
        }
        for (int p = 0; p < h->P; ++p)
            for (int j = 0; j < h->N; ++j) h32[(size_t)p * h->N + j] = tmp[(size_t)p * h->Np + j];
        delete[] tmp;
        e = cudaMemcpy(pop, h32, (size_t)h->P * h->N * sizeof(int32_t), cudaMemcpyDefault);
        delete[] h32;
        if (e != cudaSuccess) return cuda_error(e, "ga_population copy out", __FILE__, __LINE__);
    }
    if (L) GPGA_CUDA(cudaMemcpy(L, h->L, (size_t)h->P * sizeof(double), cudaMemcpyDefault));
    return GPGA_OK;
}

GPGA_API int cluster_mst(const double *C, int N, const int32_t *labels, int32_t *edge_u,
                         int32_t *edge_v, double *edge_w, int *n_edges, void *stream)
{
    g_err[0] = 0;
    if (!C || !labels || !edge_u || !edge_v || !edge_w)
        return set_error(GPGA_ERR_ARG, "cluster_mst: NULL pointer");
    if (N < 1 || N > GPGA_MAX_N) return set_error(GPGA_ERR_ARG, "cluster_mst: N=%d out of range", N);
    int rc = prepare_device();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int *grp = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&grp, cluster_mst_scratch_ints(N) * sizeof(int), s));
    int hinfo[2] = {0, 0};
    rc = launch_cluster_mst(C, N, labels, edge_u, edge_v, edge_w, grp, s);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(hinfo, grp, sizeof hinfo, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "cluster_mst sync", __FILE__, __LINE__);
    }
    cudaFreeAsync(grp, s);
    if (rc) return rc;
    if (hinfo[0]) return set_error(GPGA_ERR_ARG, "cluster_mst: a label lies outside [0, N)");
    if (n_edges) *n_edges = N - hinfo[1];
    return GPGA_OK;
}

GPGA_API int gpga_log_selftest(const double *x, int n, double *y_table, double *y_cuda,
                               void *stream)
{
    g_err[0] = 0;
    if (!x || !y_table || !y_cuda || n < 0) return set_error(GPGA_ERR_ARG, "gpga_log_selftest: bad argument");
    if (n == 0) return GPGA_OK;
    return launch_log_selftest(x, n, y_table, y_cuda, (cudaStream_t)stream);
}

GPGA_API int ga_free(gpga_ga *h)
{
    if (!h) return GPGA_OK;
    if (h->gU) cudaGraphExecDestroy(h->gU);
    if (h->g1) cudaGraphExecDestroy(h->g1);
    if (h->block) cudaFreeAsync(h->block, h->stream);
    cudaStreamSynchronize(h->stream);
    for (auto &row : h->evU)
        for (auto &e : row)
            if (e) cudaEventDestroy(e);
    for (auto &row : h->ev1)
        for (auto &e : row)
            if (e) cudaEventDestroy(e);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return GPGA_OK;
}

} // extern "C"
