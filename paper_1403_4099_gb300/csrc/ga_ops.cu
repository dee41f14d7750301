// ga_ops.cu -- the device-resident GA generation of Algorithm 1 after scoring:
// evaluate state and statistics, termination test, isolate fittest, elitism,
// scaling, SUS selection (one grid launch per generation), then crossover, mutation and
// replacement (one warp per child). All decisions are integer or exact
// comparisons of FP64 values, so the result is bit-identical to any other
// implementation of the same rules fed the same fitness vector and Philox key.
#include <math.h>

#include "gpga_internal.cuh"

namespace gpga {

uint64_t prob_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(p * 4294967296.0);
}

void set_sus_divisor(EvolveCfg *cfg, int M)
{
    int l = 0;
    while ((1ll << l) < (long long)M) ++l; // l = ceil(log2 M)
    const int s = 60 + l;
    // magic = ceil(2^s / M) < 2^61, by long division in 128 bits
    const unsigned __int128 num = (unsigned __int128)1 << s;
    unsigned __int128 q = num / (unsigned)M;
    if (q * (unsigned)M != num) q += 1;
    cfg->m_magic = (uint64_t)q;
    cfg->m_shift = s;
}

void set_mutation(EvolveCfg *cfg, double pm)
{
    cfg->thr_pm = prob_threshold(pm);
    // (1 - P_m)^t as a running FP64 product, t = 1..MUT_BLOCK, scaled to 32 bits
    const double keep = 1.0 - pm;
    double run = 1.0;
    for (int t = 0; t < MUT_BLOCK; ++t) {
        run *= keep;
        const double v = floor(run * 4294967296.0);
        cfg->gap[t] = v >= 4294967295.0 ? 0xffffffffu : (uint32_t)v;
    }
}

// ---------------------------------------------------------------------------
// "Create initial population": gene j of individual p uniform in [0, K0) from
// word j mod 4 of Philox(0, p, j / 4, INIT). One thread per 4 genes.
// ---------------------------------------------------------------------------
template <typename LabT>
__global__ void init_uniform_kernel(LabT *__restrict__ pop, int ldp, int P, int N, int K0,
                                    uint32_t k0, uint32_t k1)
{
    const int nb = (ldp + 3) >> 2;
    const long long total = (long long)P * nb;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(t / nb), b = (int)(t - (long long)p * nb);
        const U4 w = philox(0u, (uint32_t)p, (uint32_t)b, STREAM_INIT, k0, k1);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = 4 * b + r;
            if (j < ldp) pop[(size_t)p * ldp + j] = (LabT)(j < N ? draw_below(ws[r], (uint32_t)K0) : 0);
        }
    }
}

template <typename LabT>
int launch_init_uniform(LabT *pop, int ldp, int P, int N, int K0, uint32_t k0, uint32_t k1,
                        cudaStream_t s)
{
    const long long total = (long long)P * ((ldp + 3) >> 2);
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    init_uniform_kernel<LabT><<<blocks, 256, 0, s>>>(pop, ldp, P, N, K0, k0, k1);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template int launch_init_uniform<uint16_t>(uint16_t *, int, int, int, int, uint32_t, uint32_t,
                                           cudaStream_t);
template int launch_init_uniform<int32_t>(int32_t *, int, int, int, int, uint32_t, uint32_t,
                                          cudaStream_t);

// ---------------------------------------------------------------------------
// Rank scaling table: inclusive prefix of w(r) = floor(2^32 / sqrt(r + 1)),
// IEEE FP64 sqrt and division (no contraction possible), r = 0..P-1.
// ---------------------------------------------------------------------------
__global__ void rank_prefix_kernel(uint64_t *__restrict__ prefix, int P)
{
    // one CTA: chunked sequential scan, deterministic
    __shared__ uint64_t part[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (P + nt - 1) / nt;
    const int lo = t * chunk, hi = min(P, lo + chunk);
    uint64_t s = 0;
    for (int r = lo; r < hi; ++r) {
        const double v = __ddiv_rn(4294967296.0, __dsqrt_rn((double)(r + 1)));
        s += (uint64_t)floor(v);
        prefix[r] = s;
    }
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        uint64_t run = 0;
        for (int k = 0; k < nt; ++k) {
            const uint64_t v = part[k];
            part[k] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int r = lo; r < hi; ++r) prefix[r] += part[t];
}

// SUS brackets of the fixed prefix: tab[k] = first rank r with
// prefix[r] > floor(k W / M), k = 0..M, W = prefix[P - 1] (k W < 2^56)
__global__ void sus_table_kernel(const uint64_t *__restrict__ prefix, int P, int M,
                                 int32_t *__restrict__ tab)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > M) return;
    const uint64_t x = (uint64_t)k * prefix[P - 1] / (uint64_t)M;
    int lo = 0, hi = P;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] > x)
            hi = mid;
        else
            lo = mid + 1;
    }
    tab[k] = lo;
}

int rank_prefix_table(uint64_t *prefix, int P, int M, int32_t *sus_tab, cudaStream_t s)
{
    rank_prefix_kernel<<<1, 1024, 0, s>>>(prefix, P);
    GPGA_LAUNCH_CHECK();
    if (sus_tab) {
        sus_table_kernel<<<(M + 1 + 255) / 256, 256, 0, s>>>(prefix, P, M, sus_tab);
        GPGA_LAUNCH_CHECK();
    }
    return GPGA_OK;
}

__global__ void state_init_kernel(DevState *st, unsigned long long *ts0, uint32_t k0, uint32_t k1)
{
    st->k0 = k0;
    st->k1 = k1;
    st->gen = 0;
    st->done = 0;
    st->best_idx = 0;
    st->err = 0;
    st->lsum = 0;
    st->best = 0.0;
    st->mean = 0.0;
    st->gnext = 0;
    if (ts0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        ts0[0] = t;
    }
}

int launch_state_init(DevState *st, unsigned long long *ts0, uint32_t k0, uint32_t k1,
                      cudaStream_t s)
{
    state_init_kernel<<<1, 1, 0, s>>>(st, ts0, k0, k1);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

// FP64 fitness as an unsigned key with the same order (NaN mapped to -inf and
// -0 to +0 first): flip all bits of negatives, set the sign bit of the rest. Integer compares
// keep the sort off the FP64 pipe.
__device__ __forceinline__ unsigned long long order_key(double x)
{
    if (isnan(x)) x = -INFINITY;
    if (x == 0.0) x = 0.0; // -0 ties with +0, as in an FP64 comparison
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// the same key from the bit pattern with integer operations only (the FP64
// pipe runs at a small fraction of the integer rate on this part)
__device__ __forceinline__ unsigned long long order_key_bits(unsigned long long b)
{
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    if (mag > 0x7ff0000000000000ull) b = 0xfff0000000000000ull; // NaN -> -inf
    else if (mag == 0ull) b = 0ull;                            // -0 -> +0
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// trunc(x 2^30) of a finite FP64 bit pattern with |x| < 2^32 as an integer
// (0 for non-finite values, which the mean leaves out), integer operations only
__device__ __forceinline__ long long fix30_bits(unsigned long long b)
{
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0x7ff || e == 0) return 0; // non-finite; zero and subnormals
    const long long m = (long long)((b & 0x000fffffffffffffull) | 0x0010000000000000ull);
    const int sh = e - 1075 + 30; // x 2^30 = m 2^(e - 1075 + 30)
    long long v = sh >= 0 ? (sh < 11 ? (m << sh) : 0x7fffffffffffffffll)
                          : (sh > -64 ? (m >> -sh) : 0ll);
    return (b >> 63) ? -v : v;
}

// strict "fitter than" of (key, index) pairs: key descending, index ascending
__device__ __forceinline__ bool fitter(unsigned long long ka, int ia, unsigned long long kb, int ib)
{
    return ka > kb || (ka == kb && ia < ib);
}

// ---------------------------------------------------------------------------
// "Isolate fittest individuals" and the per-generation bookkeeping, one launch.
// rank_i = #{j : (L_j, j) fitter than (L_i, i)} (key descending, index
// ascending; NaN as -inf). CTA (x, y) sorts the 256 keys of chunk y
// (bitonic, shuffles below distance 32, shared memory above) and counts, for
// each key i of chunk x, the fitter keys of chunk y by binary search; integer
// atomics sum the counts, so the ranks are exact and order-independent.
// Ticket (no CTA ever waits): the last CTA scatters perm[rank_i] = i (zeroing
// rank for the next use) and does "evaluate state and statistics" (best; the
// mean from the fixed-point sum the CTAs of row 0 add), the record of the best
// configuration and the device clock, "determine if termination criteria are
// met", and for proportional scaling the weights by rank with their inclusive
// prefix.
// Stateful use: g = st->gen + gen_off.
// ---------------------------------------------------------------------------
constexpr int RANK_CHUNK = 256;

struct SelectSmem {
    unsigned long long sk[RANK_CHUNK];
    int si[RANK_CHUNK];
    uint64_t s_part[RANK_CHUNK];
    int s_last;
    int s_best;      // the individual of rank 0
    double s_bestL;  // its fitness
};

// the body of one CTA (blockIdx.x, blockIdx.y) of the selection grid of one run
template <typename LabT>
__device__ __forceinline__ void select_cta(const double *__restrict__ L, const SelectCfg &cfg,
                                           int *__restrict__ rank, int32_t *__restrict__ perm,
                                           uint64_t *__restrict__ work_prefix,
                                           unsigned *__restrict__ ticket, DevState *st,
                                           double *__restrict__ hist, const LabT *pop0,
                                           const LabT *pop1, LabT *__restrict__ ring,
                                           unsigned long long *__restrict__ ts, SelectSmem &sm)
{
    if (st && st->done) return;
    const int P = cfg.P;
    unsigned long long *sk = sm.sk;
    int *si = sm.si;
    int &s_last = sm.s_last;
    uint64_t *s_part = sm.s_part;
    const int tid = threadIdx.x, nt = blockDim.x;
    {
        // chunk y sorted fitter-first by a bitonic network, one key per thread:
        // exchanges at distance < 32 through warp shuffles, wider ones through
        // shared memory (6 of the 36 stages); padding (key 0, index above every
        // real one) sorts last and is fitter than no real key
        const int jy = blockIdx.y * RANK_CHUNK + tid;
        unsigned long long mk = jy < P ? order_key(L[jy]) : 0ull;
        int mi = jy < P ? jy : 0x7fffffff;
        const int i = blockIdx.x * RANK_CHUNK + tid;
        const unsigned long long ki = i < P ? order_key(L[i]) : 0ull;
        for (int k = 2; k <= RANK_CHUNK; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                unsigned long long pk;
                int pi;
                if (j >= 32) {
                    sk[tid] = mk;
                    si[tid] = mi;
                    __syncthreads();
                    pk = sk[tid ^ j];
                    pi = si[tid ^ j];
                    __syncthreads();
                } else {
                    pk = __shfl_xor_sync(0xffffffffu, mk, j);
                    pi = __shfl_xor_sync(0xffffffffu, mi, j);
                }
                // the lower position of an ascending (fitter-first) block keeps
                // the fitter key, and so on
                const bool keep_fitter = ((tid & j) == 0) == ((tid & k) == 0);
                const bool mine_fitter = fitter(mk, mi, pk, pi);
                if (keep_fitter != mine_fitter) {
                    mk = pk;
                    mi = pi;
                }
            }
        }
        sk[tid] = mk;
        si[tid] = mi;
        __syncthreads();
        if (i < P) {
            // fitter keys of chunk y form a prefix of the sorted chunk
            int pos = 0;
#pragma unroll
            for (int step = RANK_CHUNK / 2; step; step >>= 1)
                if (fitter(sk[pos + step - 1], si[pos + step - 1], ki, i)) pos += step;
            if (fitter(sk[pos], si[pos], ki, i)) ++pos; // pos = RANK_CHUNK - 1 case
            if (pos) atomicAdd(&rank[i], pos);
        }
    }
    // the population mean in fixed point 2^-30 (exact integer sum, non-finite
    // fitness left out): the CTAs of row y = 0 add chunk x's share
    if (st && blockIdx.y == 0) {
        const int i = blockIdx.x * RANK_CHUNK + tid;
        long long f = 0;
        if (i < P) {
            const double v = L[i];
            if (isfinite(v)) f = __double2ll_rn(v * 1073741824.0);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if ((tid & 31) == 0 && f)
            atomicAdd(reinterpret_cast<unsigned long long *>(&st->lsum), (unsigned long long)f);
    }
    // ticket: the last of the nc x nc CTAs holds the final ranks, scatters
    // perm[rank_i] = i (zeroing rank for the next use) and does the
    // generation's bookkeeping
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&ticket[0], 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // a generation kernel launched as a programmatic dependent may be scheduled
    // now; it waits for this grid to complete before it reads anything written here
    griddep_launch();
    const int g = st ? __ldcg(&st->gen) + cfg.gen_off : 0; // (loaded while perm is built)
    // the bookkeeping inputs that do not depend on the ranks, loaded alongside them
    const bool stall = st && cfg.tol >= 0.0 && cfg.stall_gens > 0 && g >= cfg.stall_gens;
    long long lsum = 0;
    double prev = 0.0;
    if (st && tid == 0) {
        lsum = __ldcg(&st->lsum);
        if (stall) prev = hist[g - cfg.stall_gens];
    }
    for (int i0 = tid; i0 < P; i0 += 16 * nt) { // 16 rank loads in flight per thread
        int r[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int i = i0 + u * nt;
            r[u] = i < P ? __ldcg(rank + i) : 0;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int i = i0 + u * nt;
            if (i < P) {
                perm[r[u]] = i;
                rank[i] = 0;
                if (r[u] == 0) { // the fittest: its index and fitness, without a perm read
                    sm.s_best = i;
                    sm.s_bestL = L[i];
                }
            }
        }
    }
    __syncthreads(); // perm is visible to the whole CTA
    if (tid == 0) ticket[0] = 0u;
    const int bidx = sm.s_best;
    if (st) {
        if (cfg.record && ring) {
            const LabT *src = ((g & 1) ? pop1 : pop0) + (size_t)bidx * cfg.ldp;
            for (int j = tid; j < cfg.N; j += nt) ring[(size_t)g * cfg.N + j] = src[j];
        }
        if (tid == 0) {
            double best = sm.s_bestL;
            if (isnan(best)) best = -INFINITY;
            st->gen = g;
            st->best = best;
            st->best_idx = bidx;
            hist[g] = best;
            int done = g >= cfg.max_gens;
            if (!done && stall) done = (best - prev) <= cfg.tol * fmax(1.0, fabs(best));
            if (cfg.record && ts) {
                unsigned long long t;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                ts[1 + g] = t;
            }
            st->done = done;
            s_last = done;
            st->mean = (double)lsum * 9.313225746154785e-10 / (double)P;
            st->lsum = 0;
        }
        __syncthreads();
        if (s_last) return;
    }
    if (cfg.scaling != GPGA_SCALING_PROP) return;
    // proportional weights by rank, w = floor(max(L, 0) / L_max 2^32) (all 1 if
    // L_max <= 0), and their inclusive prefix: chunked sequential scan
    double lmax = sm.s_bestL;
    if (isnan(lmax)) lmax = -INFINITY;
    const int chunk = (P + nt - 1) / nt;
    const int lo = tid * chunk, hi = min(P, lo + chunk);
    uint64_t sacc = 0;
    for (int r = lo; r < hi; ++r) {
        uint64_t w = 1;
        if (lmax > 0.0) {
            double x = L[__ldcg(perm + r)];
            if (!(x > 0.0)) x = 0.0;
            w = (uint64_t)floor(__dmul_rn(__ddiv_rn(x, lmax), 4294967296.0));
        }
        sacc += w;
        work_prefix[r] = sacc;
    }
    s_part[tid] = sacc;
    __syncthreads();
    if (tid == 0) {
        uint64_t run = 0;
        for (int k = 0; k < nt; ++k) {
            const uint64_t v = s_part[k];
            s_part[k] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int r = lo; r < hi; ++r) work_prefix[r] += s_part[tid];
}

template <typename LabT>
__global__ void __launch_bounds__(RANK_CHUNK)
    select_kernel(const double *__restrict__ L, SelectCfg cfg, int *__restrict__ rank,
                  int32_t *__restrict__ perm, uint64_t *__restrict__ work_prefix,
                  unsigned *__restrict__ ticket, DevState *st, double *__restrict__ hist,
                  const LabT *pop0, const LabT *pop1, LabT *__restrict__ ring,
                  unsigned long long *__restrict__ ts)
{
    __shared__ SelectSmem sm;
    select_cta<LabT>(L, cfg, rank, perm, work_prefix, ticket, st, hist, pop0, pop1, ring, ts, sm);
}

// Selection of every active run of a fleet: CTA (x, y, z) plays CTA (x, y) of
// the runs at table positions z, z + gridDim.z, ... < hdr->nruns in turn (the
// per-run tickets never make a CTA wait, so the order is free).
__global__ void __launch_bounds__(RANK_CHUNK)
    fleet_select_kernel(const FleetRun *__restrict__ runs, const FleetHdr *__restrict__ hdr,
                        SelectCfg cfg)
{
    __shared__ SelectSmem sm;
    const int nruns = hdr->nruns;
    for (int z = blockIdx.z; z < nruns; z += gridDim.z) {
        const FleetRun &r = runs[z];
        SelectCfg c = cfg;
        c.N = r.N;
        c.ldp = r.Np;
        select_cta<uint16_t>(r.L, c, r.rank, r.perm, r.work_prefix, r.ticket, r.st, r.hist,
                             r.pop0, r.pop1, nullptr, nullptr, sm);
        __syncthreads(); // shared memory is reused by the next run
    }
}

int launch_fleet_select(const FleetRun *runs, const FleetHdr *hdr, const SelectCfg &cfg,
                        int cap, cudaStream_t s)
{
    const int nc = (cfg.P + RANK_CHUNK - 1) / RANK_CHUNK;
    // at most ~4096 CTAs in flight, the rest of the runs taken in turn
    int z = 4096 / (nc * nc);
    if (z < 1) z = 1;
    if (z > cap) z = cap;
    fleet_select_kernel<<<dim3(nc, nc, z), RANK_CHUNK, 0, s>>>(runs, hdr, cfg);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

// ---------------------------------------------------------------------------
// Island model (the variant the paper proposes, Sec. 5.2 and 6): the runs of a fleet
// are islands on one C, in a ring by table position. When the generation
// being built, g + 1, is a multiple of `every`, island z copies the first m
// slots of its new population -- its m best of generation g, placed there by
// elitism (m <= E) -- with their fitness over the last m slots (children) of
// island (z + 1) mod K, before the selection ranks the new populations. Both
// islands must be active and at the same generation. Runs after the fused
// generation kernel, every generation (a no-op between migrations).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
    fleet_migrate_kernel(const FleetRun *__restrict__ runs, const FleetHdr *__restrict__ hdr,
                         int P, int every, int m)
{
    const int K = hdr->nruns;
    if (K < 2) return;
    for (int z = blockIdx.x; z < K; z += gridDim.x) {
        const FleetRun &a = runs[z];
        const FleetRun &b = runs[(z + 1) % K];
        if (a.st->done || b.st->done) continue;
        const int g = a.st->gen;
        if (b.st->gen != g || (g + 1) % every != 0) continue;
        // the new population (generation g + 1) is buffer (g + 1) & 1
        const uint16_t *src = ((g + 1) & 1) ? a.pop1 : a.pop0;
        uint16_t *dst = ((g + 1) & 1) ? b.pop1 : b.pop0;
        const int Np = a.Np;
        for (int idx = threadIdx.x; idx < m * Np; idx += blockDim.x) {
            const int r = idx / Np, j = idx - r * Np;
            dst[(size_t)(P - m + r) * Np + j] = src[(size_t)r * Np + j];
        }
        for (int r = threadIdx.x; r < m; r += blockDim.x) b.L[P - m + r] = a.L[r];
    }
}

int launch_fleet_migrate(const FleetRun *runs, const FleetHdr *hdr, int P, int every, int m,
                         int cap, cudaStream_t s)
{
    const int grid = cap < 152 ? cap : 152;
    fleet_migrate_kernel<<<grid, 256, 0, s>>>(runs, hdr, P, every, m);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

// ---------------------------------------------------------------------------
// "Isolate fittest individuals" by counting, for rank scaling (whose weights
// by rank are fixed, so nothing after the ranks needs a second pass): CTA c
// owns the 32 keys i = 32 c + lane; every CTA holds all P keys in shared
// memory, and warp w counts, for its lane's key, the fitter keys of slice w
// of the population: rank_i = #{j < i : k_j >= k_i} + #{j > i : k_j > k_i}
// (key descending, index ascending; NaN as -inf). The slices' counts add up
// to the exact rank, so perm[rank_i] = i is written at once: no atomics, no
// ticket, no CTA waits for another. The CTA that holds rank 0 does the
// generation's bookkeeping (best, the record of the best configuration and the
// device clock, the termination test); CTA 0 writes the mean, from the
// fixed-point sum of all fitness values.
// Stateful use: g = st->gen + gen_off (read only by the CTA that holds rank 0,
// which is also the only writer of the state).
// ---------------------------------------------------------------------------
constexpr int SEL_WARPS = 32;

// count of keys of s_key[j0, j1) (pairs of 16 bytes; j0, j1 even) that are
// >= ki (ge) or > ki
template <bool GE>
__device__ __forceinline__ int count_fitter(const unsigned long long *s_key, int j0, int j1,
                                            unsigned long long ki)
{
    int c = 0;
    const ulonglong2 *k2 = reinterpret_cast<const ulonglong2 *>(s_key);
#pragma unroll 4
    for (int j = j0 >> 1; j < (j1 >> 1); ++j) {
        const ulonglong2 v = k2[j];
        if (GE) {
            c += v.x >= ki ? 1 : 0;
            c += v.y >= ki ? 1 : 0;
        } else {
            c += v.x > ki ? 1 : 0;
            c += v.y > ki ? 1 : 0;
        }
    }
    return c;
}

template <typename LabT>
__global__ void __launch_bounds__(32 * SEL_WARPS)
    select_count_kernel(const double *__restrict__ L, SelectCfg cfg, int32_t *__restrict__ perm,
                        DevState *st, double *__restrict__ hist, const LabT *pop0,
                        const LabT *pop1, LabT *__restrict__ ring,
                        unsigned long long *__restrict__ ts)
{
    extern __shared__ unsigned long long s_key[]; // P keys, zero-padded to Pp
    __shared__ int s_cnt[SEL_WARPS][32];
    __shared__ long long s_sum[SEL_WARPS];
    __shared__ int s_best;
    if (st && st->done) return; // a run that terminated selects nothing
    const int P = cfg.P, Pp = (P + 2 * SEL_WARPS - 1) & ~(2 * SEL_WARPS - 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x;
    // keys (a padding key 0 is below every real key, so it is never fitter),
    // four loads in flight per thread; CTA 0 alone forms the fixed-point sum
    // for the mean
    const bool mean_cta = st && blockIdx.x == 0;
    long long fsum = 0;
    for (int j0 = tid; j0 < Pp; j0 += 4 * nt) {
        unsigned long long u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + q * nt;
            u[q] = j < P ? (unsigned long long)__double_as_longlong(__ldg(L + j)) : 0ull;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + q * nt;
            if (j < Pp) s_key[j] = j < P ? order_key_bits(u[q]) : 0ull;
            if (mean_cta && j < P) fsum += fix30_bits(u[q]);
        }
    }
    if (mean_cta) {
#pragma unroll
        for (int o = 16; o; o >>= 1) fsum += __shfl_xor_sync(0xffffffffu, fsum, o);
        if (lane == 0) s_sum[warp] = fsum;
    }
    if (tid == 0) s_best = -1;
    __syncthreads();
    const int b0 = blockIdx.x * 32, i = b0 + lane;
    const unsigned long long ki = i < P ? s_key[i] : 0ull;
    const int per = Pp / SEL_WARPS; // even
    const int j0 = warp * per, j1 = j0 + per;
    // j below the CTA's block: fitter iff k_j >= k_i (lower index wins ties);
    // inside the block: per lane; above it: fitter iff k_j > k_i
    int c = count_fitter<true>(s_key, j0, min(j1, b0), ki);
    for (int j = max(j0, b0); j < min(j1, b0 + 32); ++j) {
        const unsigned long long kj = s_key[j];
        c += (kj > ki || (kj == ki && j < i)) ? 1 : 0;
    }
    c += count_fitter<false>(s_key, max(j0, b0 + 32), j1, ki);
    s_cnt[warp][lane] = c;
    __syncthreads();
    if (warp == 0) {
        int r = 0;
#pragma unroll
        for (int w = 0; w < SEL_WARPS; ++w) r += s_cnt[w][lane];
        if (i < P) {
            perm[r] = i;
            if (r == 0) s_best = i;
        }
    }
    __syncthreads();
    // the next generation kernel (a programmatic dependent) may be scheduled
    // now; it waits for this grid to complete before it reads anything written here
    griddep_launch();
    if (mean_cta && tid == 0) {
        long long lsum = 0;
#pragma unroll
        for (int w = 0; w < SEL_WARPS; ++w) lsum += s_sum[w];
        st->mean = (double)lsum * 9.313225746154785e-10 / (double)P;
    }
    const int bidx = s_best;
    if (!st || bidx < 0) return;
    const int g = st->gen + cfg.gen_off;
    if (cfg.record && ring) {
        const LabT *src = ((g & 1) ? pop1 : pop0) + (size_t)bidx * cfg.ldp;
        for (int j = tid; j < cfg.N; j += blockDim.x) ring[(size_t)g * cfg.N + j] = src[j];
    }
    if (tid == 0) {
        double best = L[bidx];
        if (isnan(best)) best = -INFINITY;
        st->gen = g;
        st->best = best;
        st->best_idx = bidx;
        hist[g] = best;
        int done = g >= cfg.max_gens;
        if (!done && cfg.tol >= 0.0 && cfg.stall_gens > 0 && g >= cfg.stall_gens)
            done = (best - hist[g - cfg.stall_gens]) <= cfg.tol * fmax(1.0, fabs(best));
        if (cfg.record && ts) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            ts[1 + g] = t;
        }
        st->done = done;
    }
}

// selection by counting for rank scaling (one launch, no ticket), else the
// chunked sort + search with the ticketed last CTA (proportional scaling needs
// the weights in rank order after all ranks are known)
template <typename LabT>
int launch_select(const double *L, const SelectCfg &cfg, int *rank, int32_t *perm,
                  uint64_t *work_prefix, unsigned *ticket, DevState *st, double *hist,
                  const LabT *const *pop2, LabT *ring, unsigned long long *ts, cudaStream_t s)
{
    if (cfg.scaling == GPGA_SCALING_RANK) {
        const int grid = (cfg.P + 31) / 32;
        const size_t smem = (size_t)((cfg.P + 2 * SEL_WARPS - 1) & ~(2 * SEL_WARPS - 1)) *
                            sizeof(unsigned long long);
        select_count_kernel<LabT><<<grid, 32 * SEL_WARPS, smem, s>>>(
            L, cfg, perm, st, hist, pop2 ? pop2[0] : nullptr, pop2 ? pop2[1] : nullptr, ring, ts);
        GPGA_LAUNCH_CHECK();
        return GPGA_OK;
    }
    const int nc = (cfg.P + RANK_CHUNK - 1) / RANK_CHUNK;
    select_kernel<LabT><<<dim3(nc, nc), RANK_CHUNK, 0, s>>>(
        L, cfg, rank, perm, work_prefix, ticket, st, hist, pop2 ? pop2[0] : nullptr,
        pop2 ? pop2[1] : nullptr, ring, ts);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template int launch_select<uint16_t>(const double *, const SelectCfg &, int *, int32_t *,
                                     uint64_t *, unsigned *, DevState *, double *,
                                     const uint16_t *const *, uint16_t *, unsigned long long *,
                                     cudaStream_t);
template int launch_select<int32_t>(const double *, const SelectCfg &, int *, int32_t *,
                                    uint64_t *, unsigned *, DevState *, double *,
                                    const int32_t *const *, int32_t *, unsigned long long *,
                                    cudaStream_t);

// ---------------------------------------------------------------------------
// "Apply genetic operator: selection" (SUS), crossover, mutation and
// replacement, one warp per slot of the next population.
// Slots 0..E-1: elites in rank order, copied. Slot E + k: child k.
// Selection: the P individuals lie on a line in rank order over segments of
// their scaled weights (prefix[r] inclusive, W = prefix[P-1]); pointer
// x_k = floor((k 2^32 + u) W / (M 2^32)), u = word 0 of Philox(g, 0, 0, SUS),
// selects rank r with prefix[r-1] <= x_k < prefix[r]. Child k pairs
// a = parent(k) with b = parent((k + M/2) mod M).
// Crossover: Philox(g, k, 0, XOVER) = (x, y, z, .): if x < thr(P_c), then the
// knowledge-based merge if y < thr(P_kb) with anchor q = draw(z, N):
// child_j = a_q where b_j = b_q, else a_j; otherwise one-point at
// cut = 1 + draw(z, N - 1): child_j = a_j for j < cut, b_j after.
// Mutation, gene pair (2m, 2m+1): Philox(g, k, m, MUT) = (f0, v0, f1, v1):
// child_j = draw(v, N) if f < thr(P_m).
// Every gene is a function of (a_j, b_j) and warp-uniform values, so lanes
// stream gene pairs with no shared memory.
// ---------------------------------------------------------------------------
template <typename LabT>
__global__ void __launch_bounds__(256)
    evolve_kernel(const LabT *pop0, const LabT *pop1, LabT *next0, LabT *next1, EvolveCfg cfg,
                  const int32_t *__restrict__ perm, const uint64_t *__restrict__ prefix,
                  int32_t *__restrict__ parents_out, const DevState *__restrict__ st)
{
    int g = cfg.gen;
    uint32_t k0 = cfg.k0, k1 = cfg.k1;
    const LabT *cur = pop0;
    LabT *nxt = next0;
    if (st) {
        if (st->done) return;
        g = st->gen;
        k0 = st->k0;
        k1 = st->k1;
        cur = (g & 1) ? pop1 : pop0;
        nxt = (g & 1) ? next1 : next0;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = blockIdx.x * 8 + warp;
    if (slot >= cfg.P) return;
    const int N = cfg.N, ldp = cfg.ldp;
    LabT *dst = nxt + (size_t)slot * ldp;
    if (slot < cfg.E) {
        const LabT *src = cur + (size_t)perm[slot] * ldp;
        for (int j = lane; j < N; j += 32) dst[j] = src[j];
        return;
    }
    child_genes<LabT>(cur, ldp, N, cfg, g, slot - cfg.E, k0, k1, perm, prefix, parents_out, dst,
                      nullptr, lane);
}

template <typename LabT>
int launch_evolve(const LabT *const *pop2, LabT *const *next2, const EvolveCfg &cfg,
                  const int32_t *perm, const uint64_t *prefix, int32_t *parents_out,
                  const DevState *st, cudaStream_t s)
{
    const int grid = (cfg.P + 7) / 8;
    evolve_kernel<LabT><<<grid, 256, 0, s>>>(pop2[0], pop2[1], next2[0], next2[1], cfg, perm,
                                             prefix, parents_out, st);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template int launch_evolve<uint16_t>(const uint16_t *const *, uint16_t *const *,
                                     const EvolveCfg &, const int32_t *, const uint64_t *,
                                     int32_t *, const DevState *, cudaStream_t);
template int launch_evolve<int32_t>(const int32_t *const *, int32_t *const *, const EvolveCfg &,
                                    const int32_t *, const uint64_t *, int32_t *,
                                    const DevState *, cudaStream_t);

int prepare_ga_kernels(int maxsmem)
{
    // select_count_kernel holds all P keys (up to 128 KB at GPGA_MAX_P)
    if (int rc = raise_smem(select_count_kernel<uint16_t>, maxsmem)) return rc;
    if (int rc = raise_smem(select_count_kernel<int32_t>, maxsmem)) return rc;
    return GPGA_OK;
}

} // namespace gpga
