// gather.cu -- gather form of the likelihood (Eq. 5, 6, 8) and the fused GA
// generation (selection, crossover, mutation, replacement + scoring).
//
// Work per configuration is what Eq. 6 needs, not N^2: genes are sorted by
// label (stable counting sort), and only same-cluster pairs are visited:
//   d_s = sum_{i,j in s} D_ij = 2 sum_{a<b} D_{m_a m_b} + sum_a D_{m_a m_a},
// sum_s n_s (n_s - 1) / 2 gathers of D (L2-resident) instead of a dense
// sweep. D is read as int32 fixed point (2^-30), so every cluster sum is an
// exact integer sum: independent of the order of the members, which are
// therefore scattered with plain atomics, and deterministic. One warp per
// individual; labels, counts and members live in that warp's 8 N-byte slice of
// shared memory. A cluster of at most 8 members is summed by one lane, a larger one by
// the whole warp. Eq. 8 then follows in the one-log product form.
#include <math.h>

#include "gpga_internal.cuh"

namespace gpga {

// per-warp shared-memory slice for Np padded genes (8 Np bytes), in order:
//   list  (2 Np bytes) int32 list of the non-singleton clusters, label order,
//         (start << 16 | n), at most N/2 entries;
//   cnt   (2 Np bytes) label counts, then cluster starts, then cluster ends;
//   lab   (2 Np bytes) labels;
//   mem   (2 Np bytes) gene indices grouped by label.
// Counts and starts are 16-bit (N < 65536), two per 32-bit word (label 2w in
// the low half of word w), updated with 32-bit shared-memory atomics: a half
// never carries into its neighbour because no count or start exceeds N. After
// the scatter, cnt and lab (contiguous) are dead and hold the pair sums.
struct GatherSlice {
    int *list;
    uint32_t *cnt;
    uint16_t *lab;
    uint16_t *mem;
};

__host__ __device__ inline size_t gather_slice_bytes(int Np) { return (size_t)Np * 8; }

__device__ inline GatherSlice gather_slice(unsigned char *base, int Np)
{
    GatherSlice s;
    s.list = reinterpret_cast<int *>(base);
    s.cnt = reinterpret_cast<uint32_t *>(base + (size_t)2 * Np);
    s.lab = reinterpret_cast<uint16_t *>(base + (size_t)4 * Np);
    s.mem = reinterpret_cast<uint16_t *>(base + (size_t)6 * Np);
    return s;
}

// clusters up to this size are summed by one lane (at most 28 pairs); larger
// ones by the whole warp
constexpr int SMALL_CLUSTER = 8;

// d_s of one cluster of 3 <= n <= K members m[0..n): every pair load issued
// at once (predicated on n), so one L2 round trip instead of n (n - 1) / 2
template <int K>
__device__ __forceinline__ long long small_cluster_sum(const uint16_t *m, int n,
                                                       const int32_t *__restrict__ Dfix, int Np,
                                                       int diag)
{
    int idx[K];
#pragma unroll
    for (int a = 0; a < K; ++a) idx[a] = a < n ? (int)m[a] : 0;
    int32_t v[K * (K - 1) / 2];
    int t = 0;
#pragma unroll
    for (int a = 0; a < K - 1; ++a)
#pragma unroll
        for (int b = a + 1; b < K; ++b, ++t)
            v[t] = b < n ? __ldg(Dfix + (size_t)idx[a] * Np + idx[b]) : 0;
    long long s = 0;
#pragma unroll
    for (int q = 0; q < K * (K - 1) / 2; ++q) s += v[q];
    s *= 2;
    if (diag)
#pragma unroll
        for (int a = 0; a < K; ++a)
            if (a < n) s += Dfix[(size_t)idx[a] * (Np + 1)];
    return s;
}

// Score one configuration held in sl.lab[0..N) (labels < N, N < 65536).
// Returns L on all lanes. Dfix: Np x Np int32, D = 1 - C in fixed point
// 2^-DFIX_BITS; diag: nonzero if some D_ii != 0. pairs_out (optional):
// += sum_s n_s (n_s - 1) / 2.
__device__ double gather_score_warp(const GatherSlice &sl, int N, int Np,
                                    const int32_t *__restrict__ Dfix, int diag,
                                    const long long *__restrict__ ltab,
                                    const long long *__restrict__ kfix, int lane,
                                    unsigned long long *pairs_out)
{
    const unsigned lt = (1u << lane) - 1u;
    const int nwd = (N + 1) >> 1; // words holding the labels 0..N-1
    // histogram
    for (int w = lane; w < nwd; w += 32) sl.cnt[w] = 0u;
    __syncwarp();
    for (int i = lane; i < N; i += 32) {
        const int s = sl.lab[i];
        atomicAdd(&sl.cnt[s >> 1], 1u << ((s & 1) << 4));
    }
    __syncwarp();
    // cluster starts (exclusive scan of the counts, written over the counts)
    // and the list of non-singleton clusters, in one pass: lane l takes the 4
    // consecutive count words 4 l .. 4 l + 3 of each 128-word chunk
    int nlist = 0;
    {
        int carry = 0;
        for (int cb = 0; cb < nwd; cb += 128) {
            const int w0 = cb + 4 * lane;
            uint32_t c2[4];
            int tot = 0, nns = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                c2[q] = w0 + q < nwd ? sl.cnt[w0 + q] : 0u;
                const int x0 = (int)(c2[q] & 0xffffu), x1 = (int)(c2[q] >> 16);
                tot += x0 + x1;
                nns += (x0 >= 2) + (x1 >= 2);
            }
            int it = tot, in = nns; // inclusive scans over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t1 = __shfl_up_sync(0xffffffffu, it, o);
                const int t2 = __shfl_up_sync(0xffffffffu, in, o);
                if (lane >= o) {
                    it += t1;
                    in += t2;
                }
            }
            int run = carry + it - tot, li = nlist + in - nns;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (w0 + q < nwd) {
                    const int x0 = (int)(c2[q] & 0xffffu), x1 = (int)(c2[q] >> 16);
                    sl.cnt[w0 + q] = (uint32_t)run | ((uint32_t)(run + x0) << 16);
                    if (x0 >= 2) sl.list[li++] = (run << 16) | x0;
                    run += x0;
                    if (x1 >= 2) sl.list[li++] = (run << 16) | x1;
                    run += x1;
                }
            }
            carry += __shfl_sync(0xffffffffu, it, 31);
            nlist += __shfl_sync(0xffffffffu, in, 31);
        }
    }
    __syncwarp();
    // scatter gene indices by label (order inside a cluster is irrelevant: the
    // pair sums below are exact integer sums), four atomics in flight per lane
    for (int i0 = lane; i0 < N; i0 += 128) {
        int sv[4];
        uint32_t old[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) sv[u] = i0 + 32 * u < N ? (int)sl.lab[i0 + 32 * u] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            old[u] = sv[u] >= 0 ? atomicAdd(&sl.cnt[sv[u] >> 1], 1u << ((sv[u] & 1) << 4)) : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (sv[u] >= 0)
                sl.mem[(old[u] >> ((sv[u] & 1) << 4)) & 0xffffu] = (uint16_t)(i0 + 32 * u);
    }
    __syncwarp();
    const int *list = sl.list;
    // Pair sums first, then the terms: the sums of the clusters hold no
    // dependency on one another, so a lane's loads of successive clusters
    // overlap instead of waiting behind each cluster's log-product step.
    // csum (int64 per listed cluster) fills the dead count and label space
    // (4 Np contiguous bytes) from the front, the list of big clusters (n > 8)
    // from the back: 8 nlist + 4 nbig <= 4 N bytes.
    long long *csum = reinterpret_cast<long long *>(sl.cnt);
    int *big_end = reinterpret_cast<int *>(sl.lab + Np);
    int nbig = 0;
    long long ksum = 0; // sum of K(n_s) in 2^-44, loaded alongside the pair sums
    // small clusters: one lane each, all pair loads of the cluster at once
    for (int base = 0; base < nlist; base += 32) {
        const int c = base + lane;
        int v = 0, n = 0;
        if (c < nlist) {
            v = list[c];
            n = v & 0xffff;
        }
        if (n >= 2 && n <= SMALL_CLUSTER) {
            const uint16_t *m = sl.mem + (v >> 16);
            ksum += __ldg(kfix + n);
            csum[c] = n <= 4 ? small_cluster_sum<4>(m, n, Dfix, Np, diag)
                             : small_cluster_sum<SMALL_CLUSTER>(m, n, Dfix, Np, diag);
        }
        const unsigned bm = __ballot_sync(0xffffffffu, n > SMALL_CLUSTER);
        if (n > SMALL_CLUSTER) big_end[-1 - (nbig + __popc(bm & lt))] = c;
        nbig += __popc(bm);
    }
    __syncwarp();
    // big clusters one at a time, rows a over lanes, eight loads in flight per lane
    for (int q = 0; q < nbig; ++q) {
        const int c = big_end[-1 - q];
        const int v = list[c];
        const uint16_t *m = sl.mem + (v >> 16);
        const int n = v & 0xffff;
        long long sum = 0;
        for (int a = lane; a < n - 1; a += 32) {
            const int32_t *row = Dfix + (size_t)m[a] * Np;
            long long s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            int b = a + 1;
            for (; b + 8 <= n; b += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) s[u] += __ldg(row + m[b + u]);
            }
#pragma unroll
            for (int u = 0; u < 7; ++u)
                if (b + u < n) s[u] += __ldg(row + m[b + u]);
            sum += ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
        }
        sum *= 2;
        if (diag)
            for (int a = lane; a < n; a += 32) sum += Dfix[(size_t)m[a] * (Np + 1)];
#pragma unroll
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) {
            csum[c] = sum;
            ksum += __ldg(kfix + n);
        }
    }
    __syncwarp();
    // the terms, one lane per cluster: two running mantissa products per lane
    // (alternate clusters), so two independent multiply chains overlap
    LogProd acc, acc2;
    acc.k = ksum;
    long long npairs = 0;
    for (int c = lane; c < nlist; c += 64) {
        const int n = list[c] & 0xffff;
        logprod_mul(acc, n, csum[c], DFIX_BITS);
        npairs += n * (n - 1) / 2;
        if (c + 32 < nlist) {
            const int n2 = list[c + 32] & 0xffff;
            logprod_mul(acc2, n2, csum[c + 32], DFIX_BITS);
            npairs += n2 * (n2 - 1) / 2;
        }
    }
    mant_mul(acc.m, acc.e, acc2.m, acc2.e); // (adds acc2's exponent too)
    if (pairs_out) {
#pragma unroll
        for (int o = 16; o; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        if (lane == 0) atomicAdd(pairs_out, (unsigned long long)npairs);
    }
    const double L = logprod_finish(acc, ltab, nlist);
    __syncwarp();
    return L;
}

// ---------------------------------------------------------------------------
// Score-only: one warp per individual of lab (stateful: the buffer selected by
// st->gen + sel_off).
// ---------------------------------------------------------------------------
template <typename LabT>
__global__ void __launch_bounds__(256, 4)
    gather_score_kernel(const LabT *lab0, const LabT *lab1, int ldl, int sel_off, int P, int N,
                        int Np, const int32_t *__restrict__ Dfix, const int *__restrict__ diag_flag,
                        const double *__restrict__ logtab, double *__restrict__ L,
                        int *__restrict__ err, const DevState *__restrict__ st,
                        unsigned long long *__restrict__ pairs)
{
    const LabT *__restrict__ lab = lab0;
    unsigned long long *pairs_g = nullptr;
    if (st) {
        if (st->done) return;
        const int gen = st->gen + sel_off;
        lab = (gen & 1) ? lab1 : lab0;
        if (pairs) pairs_g = pairs + gen;
    }
    extern __shared__ unsigned char smem_g[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const GatherSlice sl = gather_slice(smem_g + (size_t)warp * gather_slice_bytes(Np), Np);
    const long long *ltab = reinterpret_cast<const long long *>(logtab);
    const long long *ktab = kfix_of(logtab);
    const int diag = *diag_flag;
    for (int p = blockIdx.x * nw + warp; p < P; p += gridDim.x * nw) {
        bool bad = false;
        const LabT *lp = lab + (size_t)p * ldl;
        for (int i = lane; i < N; i += 32) {
            const int v = (int)lp[i];
            const bool ok = v >= 0 && v < N;
            bad |= !ok;
            sl.lab[i] = (uint16_t)(ok ? v : 0);
        }
        bad = __any_sync(0xffffffffu, bad);
        __syncwarp();
        const double v = gather_score_warp(sl, N, Np, Dfix, diag, ltab, ktab, lane, pairs_g);
        if (lane == 0) {
            L[p] = bad ? __longlong_as_double(0x7ff8000000000000ll) : v;
            if (bad && err) atomicOr(err, 1);
        }
    }
}

// ---------------------------------------------------------------------------
// Fused generation: warp `slot` builds slot of the next population exactly as
// the evolve kernel does (elite copy, or SUS parents + crossover + mutation)
// into global memory and its shared slice, then scores it.
// ---------------------------------------------------------------------------
// one slot of the next population (all lanes of the warp call)
template <typename LabT>
__device__ __forceinline__ void generation_slot(const LabT *cur, LabT *nxt, const EvolveCfg &cfg,
                                                int g, uint32_t k0, uint32_t k1, int slot,
                                                const int32_t *__restrict__ perm,
                                                const uint64_t *__restrict__ prefix, int Np,
                                                const int32_t *__restrict__ Dfix, int diag,
                                                const double *__restrict__ logtab,
                                                double *__restrict__ L, const GatherSlice &sl,
                                                int lane, unsigned long long *pairs_out,
                                                const SusPre *pre = nullptr)
{
    const int N = cfg.N, ldp = cfg.ldp;
    LabT *dst = nxt + (size_t)slot * ldp;
    if (slot < cfg.E) {
        const LabT *src = cur + (size_t)perm[slot] * ldp;
        for (int j = lane; j < N; j += 32) {
            const LabT v = src[j];
            dst[j] = v;
            sl.lab[j] = (uint16_t)v;
        }
    } else {
        const int k = slot - cfg.E;
        child_genes<LabT>(cur, ldp, N, cfg, g, k, k0, k1, perm, prefix, nullptr, dst, sl.lab,
                          lane, pre);
    }
    __syncwarp();
    const double v = gather_score_warp(sl, N, Np, Dfix, diag,
                                       reinterpret_cast<const long long *>(logtab), kfix_of(logtab),
                                       lane, pairs_out);
    if (lane == 0) L[slot] = v;
}

template <typename LabT>
__global__ void __launch_bounds__(256, 4)
    gather_generation_kernel(const LabT *pop0, const LabT *pop1, LabT *next0, LabT *next1,
                             EvolveCfg cfg, const int32_t *__restrict__ perm,
                             const uint64_t *__restrict__ prefix, int Np,
                             const int32_t *__restrict__ Dfix, const int *__restrict__ diag_flag,
                             const double *__restrict__ logtab,
                             double *__restrict__ L, const DevState *__restrict__ st,
                             unsigned long long *__restrict__ pairs)
{
    extern __shared__ unsigned char smem_g[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int slot = blockIdx.x * nw + warp;
    if (slot >= cfg.P) return;
    // the SUS loads that depend on no generation (fixed tables written at the
    // start of the run), issued before the wait below
    SusPre pre;
    const bool use_pre = cfg.sus_tab != nullptr && slot >= cfg.E;
    if (use_pre) pre = sus_prefetch((uint32_t)(slot - cfg.E), cfg.M, cfg.P, prefix, cfg.sus_tab, lane);
    // launched as a programmatic dependent of the selection (which lets it be
    // scheduled while its last CTA finishes): wait for that grid before reading
    // perm and the state. (Letting the selection in turn be scheduled early,
    // from here, measured slower: its waiting CTAs cost the generation more
    // than the launch gap they hide.)
    griddep_wait();
    if (st->done) return;
    const int g = st->gen;
    const LabT *cur = (g & 1) ? pop1 : pop0;
    LabT *nxt = (g & 1) ? next1 : next0;
    const GatherSlice sl = gather_slice(smem_g + (size_t)warp * gather_slice_bytes(Np), Np);
    generation_slot<LabT>(cur, nxt, cfg, g, st->k0, st->k1, slot, perm, prefix, Np, Dfix,
                          *diag_flag, logtab, L, sl, lane, pairs ? pairs + g + 1 : nullptr,
                          use_pre ? &pre : nullptr);
}

// ---------------------------------------------------------------------------
// Fleet generation: work item i is slot i mod P of the run at table position
// i / P (the table is ordered by decreasing N, so the costly runs start
// first); the CTAs stride over the items. Runs whose state is done are
// skipped. Per slot the work is exactly that of gather_generation_kernel.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512, 2)
    fleet_generation_kernel(const FleetRun *__restrict__ runs, const FleetHdr *__restrict__ hdr,
                            EvolveCfg base, const uint64_t *__restrict__ rank_prefix,
                            const double *__restrict__ logtab, int Np_max, int prop)
{
    // may be launched as a programmatic dependent of the fleet's selection:
    // wait for that grid before reading any run's state, permutation or prefix
    griddep_wait();
    extern __shared__ unsigned char smem_g[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    unsigned char *slice = smem_g + (size_t)warp * gather_slice_bytes(Np_max);
    const int nitems = hdr->nitems, P = base.P;
    for (int item = blockIdx.x * nw + warp; item < nitems; item += gridDim.x * nw) {
        const int ri = item / P, slot = item - ri * P;
        const FleetRun &r = runs[ri];
        const DevState *st = r.st;
        if (st->done) continue;
        const int g = st->gen;
        EvolveCfg cfg = base;
        cfg.N = r.N;
        cfg.ldp = r.Np;
        const uint16_t *cur = (g & 1) ? r.pop1 : r.pop0;
        uint16_t *nxt = (g & 1) ? r.pop0 : r.pop1;
        const uint64_t *prefix = prop ? r.work_prefix : rank_prefix;
        const GatherSlice sl = gather_slice(slice, r.Np);
        generation_slot<uint16_t>(cur, nxt, cfg, g, st->k0, st->k1, slot, r.perm, prefix, r.Np,
                                  r.Dfix, *r.diag, logtab, r.L, sl, lane, nullptr);
        __syncwarp();
    }
}

// warps per CTA of the single-run gather kernels: 4 (measured at N=500,
// P=4096: 1024 CTAs of 4 warps spread over the SMs more evenly than 512 of 8,
// 4% less time per generation), fewer if the slices do not fit
static int warps_for(int Np)
{
    const size_t per = gather_slice_bytes(Np);
    int nw = 4;
    while (nw > 1 && nw * per > (size_t)200 * 1024) nw >>= 1;
    return nw;
}

template <typename LabT>
int launch_gather_score(const LabT *const *lab2, int ldl, int sel_off, int P, int N, int Np,
                        const int32_t *Dfix, const int *diag_flag, const double *logtab,
                        double *L, int *err, const DevState *st, unsigned long long *pairs,
                        cudaStream_t s)
{
    const int nw = warps_for(Np);
    const size_t smem = nw * gather_slice_bytes(Np);
    const int grid = (P + nw - 1) / nw;
    gather_score_kernel<LabT><<<grid, 32 * nw, smem, s>>>(lab2[0], lab2[1], ldl, sel_off, P, N,
                                                          Np, Dfix, diag_flag, logtab, L, err,
                                                          st, pairs);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template <typename LabT>
int launch_gather_generation(const LabT *const *pop2, LabT *const *next2, const EvolveCfg &cfg,
                             const int32_t *perm, const uint64_t *prefix, int Np,
                             const int32_t *Dfix, const int *diag_flag, const double *logtab,
                             double *L, const DevState *st, unsigned long long *pairs, bool pdl,
                             cudaStream_t s)
{
    const int nw = warps_for(Np);
    const size_t smem = nw * gather_slice_bytes(Np);
    const int grid = (cfg.P + nw - 1) / nw;
    GPGA_CUDA(launch_pdl(gather_generation_kernel<LabT>, dim3(grid), dim3(32 * nw), smem, s, pdl,
                         pop2[0], pop2[1], next2[0], next2[1], cfg, perm, prefix, Np, Dfix,
                         diag_flag, logtab, L, st, pairs));
    return GPGA_OK;
}

int fleet_max_warps(int Np_max)
{
    int nw = 16;
    while (nw > 1 && nw * gather_slice_bytes(Np_max) > (size_t)200 * 1024) nw >>= 1;
    return nw;
}

int fleet_ctas_per_sm(int Np_max, int warps, int *out)
{
    GPGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        out, fleet_generation_kernel, 32 * warps, warps * gather_slice_bytes(Np_max)));
    return GPGA_OK;
}

int launch_fleet_generation(const FleetRun *runs, const FleetHdr *hdr, const EvolveCfg &cfg,
                            const uint64_t *rank_prefix, const double *logtab, int Np_max,
                            int warps, int ctas, int prop, cudaStream_t s, bool pdl)
{
    if (warps < 1 || warps > 16 || ctas < 1)
        return set_error(GPGA_ERR_ARG, "fleet generation: %d warps x %d CTAs", warps, ctas);
    const size_t smem = warps * gather_slice_bytes(Np_max);
    GPGA_CUDA(launch_pdl(fleet_generation_kernel, dim3(ctas), dim3(32 * warps), smem, s, pdl, runs,
                         hdr, cfg, rank_prefix, logtab, Np_max, prop));
    return GPGA_OK;
}

template int launch_gather_score<uint16_t>(const uint16_t *const *, int, int, int, int, int,
                                           const int32_t *, const int *, const double *, double *,
                                           int *, const DevState *, unsigned long long *,
                                           cudaStream_t);
template int launch_gather_score<int32_t>(const int32_t *const *, int, int, int, int, int,
                                          const int32_t *, const int *, const double *, double *,
                                          int *, const DevState *, unsigned long long *,
                                          cudaStream_t);
template int launch_gather_generation<uint16_t>(const uint16_t *const *, uint16_t *const *,
                                                const EvolveCfg &, const int32_t *,
                                                const uint64_t *, int, const int32_t *,
                                                const int *, const double *, double *,
                                                const DevState *, unsigned long long *, bool,
                                                cudaStream_t);

int prepare_gather_kernels(int maxsmem)
{
    if (int rc = raise_smem(gather_score_kernel<uint16_t>, maxsmem)) return rc;
    if (int rc = raise_smem(gather_score_kernel<int32_t>, maxsmem)) return rc;
    if (int rc = raise_smem(gather_generation_kernel<uint16_t>, maxsmem)) return rc;
    if (int rc = raise_smem(fleet_generation_kernel, maxsmem)) return rc;
    return GPGA_OK;
}

} // namespace gpga
