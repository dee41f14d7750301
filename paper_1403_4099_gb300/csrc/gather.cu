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
// individual; labels, counts and members live in that warp's slice of shared
// memory. A cluster of at most 8 members is summed by one lane, a larger one
// by the whole warp.
//
// Eq. 8 is a sum of one term per cluster with n_s >= 2,
//   L = sum_s T(n_s, d_s),  T(n, d) = K(n) - 1/2 log(c d^(n-1)),  c = n^2 - d,
// each term evaluated in integer fixed point (Q40) from the exact (n_s, d_s),
// so L is an exact integer sum of terms that depend on their own cluster only.
//
// Delta scoring of children (stateful runs): each individual keeps its table
// of d_s per label (valid where n_s >= 2), its L in Q40 and its pair count.
// A child differs from its first parent a in a few genes X (a knowledge-based
// merge moves one of b's clusters, mutation redraws about N P_m genes). With
// U_t the members of cluster t that did not move, Out_t the genes of X that
// left t and In_t those that joined it,
//   d'_t = d_t + 2 [D(U_t, In_t) - D(U_t, Out_t)] + D(In_t, In_t) - D(Out_t, Out_t),
// so only the clusters X touches are updated, with sum_t |U_t| (|In_t| +
// |Out_t|) + |X|^2 gathers, and L' = L + sum_t [T(n'_t, d'_t) - T(n_t, d_t)].
// All sums are exact integers and T depends on (n, d) alone, so the result is
// bit-identical to scoring the child from scratch. Children with more than
// DELTA_X changed genes (one-point crossovers, mostly) are scored from scratch.
#include <math.h>

#include "gpga_internal.cuh"

namespace gpga {

// ---------------------------------------------------------------------------
// Per-warp shared-memory slice for Np padded genes: 8 Np bytes, in order
//   list  (2 Np bytes) int32 list of the non-singleton clusters, label order,
//         (start << 16 | n), at most N/2 entries;
//   cnt   (2 Np bytes) label counts, then cluster starts, then cluster ends;
//   lab   (2 Np bytes) labels;
//   mem   (2 Np bytes) gene indices grouped by label;
// then the delta region (delta_bytes(Np)): the changed genes X of a child and
// the affected clusters (delta path), or the labels of the listed clusters
// (full path).
// Counts and starts are 16-bit (N < 65536), two per 32-bit word (label 2w in
// the low half of word w), updated with 32-bit shared-memory atomics: a half
// never carries into its neighbour because no count or start exceeds N. After
// the scatter, cnt and lab (contiguous) are dead and hold the pair sums.
// ---------------------------------------------------------------------------
// at most DELTA_X changed genes (bits of a 32-bit mask) and 2 DELTA_X touched
// clusters; 30 bytes per touched cluster and 6 per changed gene (2.1 KB), so
// that the slices of a 4-warp CTA at N = 500 leave room for the 8 CTAs per SM
// the registers allow (one wave of the 4096 children)
constexpr int DELTA_X = 32;
constexpr int DELTA_A = 2 * DELTA_X;
__host__ __device__ inline size_t delta_bytes(int Np)
{
    const size_t b = 6 * (size_t)DELTA_X + 30 * (size_t)DELTA_A;
    const size_t need = b > (size_t)Np ? b : (size_t)Np;
    return (need + 15) & ~(size_t)15;
}
// slice of a warp: the delta region only where the per-cluster form runs
// (N >= DELTA_MIN_N; its full path keeps the listed clusters' labels there)
__host__ __device__ inline size_t gather_slice_bytes(int Np, bool delta)
{
    return (size_t)Np * 8 + (delta ? delta_bytes(Np) : 0);
}

constexpr uint16_t NO_SLOT = 0xffffu;

// the slice of one warp: its base and Np; the regions are computed on use
// (a struct of pointers would be kept in local memory)
struct GatherSlice {
    unsigned char *base;
    int Np;
    __device__ __forceinline__ int *list() const { return reinterpret_cast<int *>(base); }
    __device__ __forceinline__ uint32_t *cnt() const
    {
        return reinterpret_cast<uint32_t *>(base + (size_t)2 * Np);
    }
    __device__ __forceinline__ uint16_t *lab() const
    {
        return reinterpret_cast<uint16_t *>(base + (size_t)4 * Np);
    }
    __device__ __forceinline__ uint16_t *mem() const
    {
        return reinterpret_cast<uint16_t *>(base + (size_t)6 * Np);
    }
    // delta region: per affected cluster the change of d (then the new d),
    // the parent's d, the bits over X of the genes that joined / left it, its
    // member count in the child, its label and a member left in place; per
    // changed gene its index and its labels in a and in the child; in the
    // full path, the labels of the listed clusters
    __device__ __forceinline__ long long *dacc() const
    {
        return reinterpret_cast<long long *>(base + (size_t)8 * Np);
    }
    __device__ __forceinline__ long long *dold() const { return dacc() + DELTA_A; }
    __device__ __forceinline__ unsigned *in_mask() const
    {
        return reinterpret_cast<unsigned *>(dold() + DELTA_A);
    }
    __device__ __forceinline__ unsigned *out_mask() const { return in_mask() + DELTA_A; }
    __device__ __forceinline__ uint16_t *nnew() const
    {
        return reinterpret_cast<uint16_t *>(out_mask() + DELTA_A);
    }
    __device__ __forceinline__ uint16_t *slab() const { return nnew() + DELTA_A; }
    __device__ __forceinline__ uint16_t *um() const { return slab() + DELTA_A; }
    __device__ __forceinline__ uint16_t *xs() const { return um() + DELTA_A; }
    __device__ __forceinline__ uint16_t *xa() const { return xs() + DELTA_X; }
    __device__ __forceinline__ uint16_t *xc() const { return xa() + DELTA_X; }
    __device__ __forceinline__ uint16_t *lablist() const
    {
        return reinterpret_cast<uint16_t *>(base + (size_t)8 * Np);
    }
};

__device__ __forceinline__ GatherSlice gather_slice(unsigned char *base, int Np)
{
    GatherSlice s;
    s.base = base;
    s.Np = Np;
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

// T(n, d) = K(n) - 1/2 [log c + (n - 1) log d] of one cluster (n >= 2) in
// fixed point 2^-40, from d as the exact fixed-point integer df = d 2^DFIX_BITS,
// c = n^2 - d, with Eq. 8's domain floors (c >= n 2^-40, d >= n (n - 1) 2^-40,
// at least one unit). Each of c, d is a 63-bit mantissa m and an exponent e
// (v = m 2^(e - 62)), log v = log(m 2^-62) + e ln 2 with the table log; the two
// logs are independent chains, and the bracket is summed exactly in 128 bits
// (Q62) before the one final shift, so T depends on (n, df) alone.
__device__ __forceinline__ long long cluster_term(int n, long long df,
                                                  const long long *__restrict__ ltab,
                                                  const long long *__restrict__ kfix)
{
    long long cf = (((long long)n * n) << DFIX_BITS) - df;
    const int sh = 40 - DFIX_BITS;
    long long cmin = (long long)n >> sh, dmin = ((long long)n * (n - 1)) >> sh;
    if (cmin < 1) cmin = 1;
    if (dmin < 1) dmin = 1;
    if (cf < cmin) cf = cmin;
    if (df < dmin) df = dmin;
    unsigned long long mc, md;
    long long ec, ed;
    mant_of(cf, mc, ec);
    mant_of(df, md, ed);
    const long long lc = log_q62(mc, ltab), ld = log_q62(md, ltab);
    const long long n1 = n - 1;
    const __int128 s = (__int128)lc + (__int128)n1 * ld +
                       (__int128)((ec - DFIX_BITS) + n1 * (ed - DFIX_BITS)) * LN2_Q62;
    return (__ldg(kfix + n) >> (KFIX_BITS - 40)) - (long long)(s >> 23);
}

// L from its Q40 fixed point
__device__ __forceinline__ double lfix_to_double(long long lf) { return dbl_scaled(lf, 40); }

// Score one configuration held in sl.lab()[0..N) (labels < N, N < 65536) from
// scratch. Returns L in Q40 on all lanes and the pair count sum_s n_s (n_s -
// 1) / 2 in *npairs_out (all lanes). Dfix: Np x Np int32, D = 1 - C in fixed
// point 2^-DFIX_BITS; diag: nonzero if some D_ii != 0. trow (optional): the
// individual's row of the d table, written where n_s >= 2.
template <bool PROD>
__device__ __forceinline__ long long score_full_warp(const GatherSlice &sl, int N, int Np,
                                     const int32_t *__restrict__ Dfix, int diag,
                                     const long long *__restrict__ ltab,
                                     const long long *__restrict__ kfix, int lane,
                                     long long *__restrict__ trow, long long *npairs_out)
{
    const unsigned lt = (1u << lane) - 1u;
    const int nwd = (N + 1) >> 1; // words holding the labels 0..N-1
    // histogram
    for (int w = lane; w < nwd; w += 32) sl.cnt()[w] = 0u;
    __syncwarp();
    for (int i = lane; i < N; i += 32) {
        const int s = sl.lab()[i];
        atomicAdd(&sl.cnt()[s >> 1], 1u << ((s & 1) << 4));
    }
    __syncwarp();
    // cluster starts (exclusive scan of the counts, written over the counts)
    // and the list of non-singleton clusters with their labels, in one pass:
    // lane l takes the 4 consecutive count words 4 l .. 4 l + 3 of each
    // 128-word chunk
    int nlist = 0;
    {
        int carry = 0;
        for (int cb = 0; cb < nwd; cb += 128) {
            const int w0 = cb + 4 * lane;
            uint32_t c2[4];
            int tot = 0, nns = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                c2[q] = w0 + q < nwd ? sl.cnt()[w0 + q] : 0u;
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
                    sl.cnt()[w0 + q] = (uint32_t)run | ((uint32_t)(run + x0) << 16);
                    if (x0 >= 2) {
                        if (!PROD && trow) sl.lablist()[li] = (uint16_t)(2 * (w0 + q));
                        sl.list()[li++] = (run << 16) | x0;
                    }
                    run += x0;
                    if (x1 >= 2) {
                        if (!PROD && trow) sl.lablist()[li] = (uint16_t)(2 * (w0 + q) + 1);
                        sl.list()[li++] = (run << 16) | x1;
                    }
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
        for (int u = 0; u < 4; ++u) sv[u] = i0 + 32 * u < N ? (int)sl.lab()[i0 + 32 * u] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            old[u] = sv[u] >= 0 ? atomicAdd(&sl.cnt()[sv[u] >> 1], 1u << ((sv[u] & 1) << 4)) : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (sv[u] >= 0)
                sl.mem()[(old[u] >> ((sv[u] & 1) << 4)) & 0xffffu] = (uint16_t)(i0 + 32 * u);
    }
    __syncwarp();
    const int *list = sl.list();
    // Pair sums of every listed cluster first, then the terms: the sums hold
    // no dependency on one another, so a lane's loads of successive clusters
    // overlap. csum (int64 per listed cluster) fills the dead count and label
    // space (4 Np contiguous bytes) from the front, the list of big clusters
    // (n > 8) from the back: 8 nlist + 4 nbig <= 4 N bytes.
    long long *csum = reinterpret_cast<long long *>(sl.cnt());
    int *big_end = reinterpret_cast<int *>(sl.lab() + Np);
    int nbig = 0;
    long long ksum = 0; // product form: sum of K(n_s) in 2^-44, loaded alongside the pair sums
    // small clusters: one lane each, all pair loads of the cluster at once
    for (int base = 0; base < nlist; base += 32) {
        const int c = base + lane;
        int v = 0, n = 0;
        if (c < nlist) {
            v = list[c];
            n = v & 0xffff;
        }
        if (n >= 2 && n <= SMALL_CLUSTER) {
            const uint16_t *m = sl.mem() + (v >> 16);
            if (PROD) ksum += __ldg(kfix + n);
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
        const uint16_t *m = sl.mem() + (v >> 16);
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
            if (PROD) ksum += __ldg(kfix + n);
        }
    }
    __syncwarp();
    if (PROD) {
        // Eq. 8 as one log of the product of the clusters' factors c d^(n-1):
        // one lane per cluster, two running products per lane (alternate
        // clusters) so that two multiply chains overlap
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
#pragma unroll
        for (int o = 16; o; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        const long long lq = logprod_finish_q40(acc, ltab, nlist);
        __syncwarp();
        *npairs_out = npairs;
        return lq;
    }
    // the terms, one lane per cluster, summed exactly
    long long lf = 0, npairs = 0;
    for (int c = lane; c < nlist; c += 32) {
        const int n = list[c] & 0xffff;
        const long long d = csum[c];
        lf += cluster_term(n, d, ltab, kfix);
        npairs += n * (n - 1) / 2;
        if (trow) trow[sl.lablist()[c]] = d;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lf += __shfl_xor_sync(0xffffffffu, lf, o);
        npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    }
    __syncwarp();
    *npairs_out = npairs;
    return lf;
}

// ---------------------------------------------------------------------------
// Child construction for the 16-bit populations of the gather form, in blocks
// of 16 genes (the mutation blocks): lane l owns blocks l, l + 32, ... for the
// crossover, the mutation and the comparison with parent a, so the changed
// genes X are found in registers. The result is gene for gene that of
// child_genes (same draws, same rules); only the work split differs.
// ---------------------------------------------------------------------------
// the draws of child k of generation g that depend on neither parent: the rank
// of this half-warp's SUS pointer (lanes 0-15 parent a, 16-31 parent b) when
// the fixed rank brackets give it directly (-1: searched later), the crossover
// words, and the mutations of the lane's first block (gene mask and the first
// four new labels in gene order; more than four: drawn again when applied)
struct ChildPlan {
    int g;
    int rank;
    uint32_t x0, x1, x2;
    uint32_t mmask;
    uint32_t mlab[2];
    int mover;
};

__device__ __forceinline__ ChildPlan plan_child(const EvolveCfg &cfg, int N, int g, int k,
                                                uint32_t k0, uint32_t k1, const SusPre *pre,
                                                int lane)
{
    ChildPlan c;
    c.g = g;
    c.rank = -1;
    const int M = cfg.M;
    if (pre && __all_sync(0xffffffffu, pre->hi - pre->lo <= 16)) {
        const uint32_t kp = lane < 16 ? (uint32_t)k : (uint32_t)((k + M / 2) % M);
        const uint32_t su = philox((uint32_t)g, 0u, 0u, STREAM_SUS, k0, k1).x;
        const uint64_t x = sus_pointer(kp, su, pre->W, cfg.m_magic, cfg.m_shift);
        const unsigned half = lane < 16 ? 0x0000ffffu : 0xffff0000u;
        const bool le = (lane & 15) < pre->hi - pre->lo && pre->cand <= x;
        c.rank = pre->lo + __popc(__ballot_sync(0xffffffffu, le) & half);
    }
    const U4 xw = philox((uint32_t)g, (uint32_t)k, 0u, STREAM_XOVER, k0, k1);
    c.x0 = xw.x;
    c.x1 = xw.y;
    c.x2 = xw.z;
    c.mmask = 0u;
    c.mlab[0] = c.mlab[1] = 0u;
    c.mover = 0;
    const int len = min(MUT_BLOCK, N - MUT_BLOCK * lane);
    if (cfg.thr_pm && len > 0) {
        int pos = 0, cnt = 0;
        auto rec = [&](int p, int v) {
            c.mmask |= 1u << p;
            if (cnt < 2) c.mlab[0] |= (uint32_t)v << ((cnt & 1) << 4);
            else if (cnt < 4) c.mlab[1] |= (uint32_t)v << ((cnt & 1) << 4);
            else c.mover = 1;
            ++cnt;
        };
        for (uint32_t e = 0;; ++e) {
            const U4 w = philox((uint32_t)g, (uint32_t)k, (uint32_t)lane + 65536u * e, STREAM_MUT,
                                k0, k1);
            pos += mutation_skip(w.x, cfg);
            if (pos >= len) break;
            rec(pos, draw_below(w.y, (uint32_t)N));
            if (++pos >= len) break;
            pos += mutation_skip(w.z, cfg);
            if (pos >= len) break;
            rec(pos, draw_below(w.w, (uint32_t)N));
            if (++pos >= len) break;
        }
    }
    return c;
}

// mutations of block blk of child k (g), written into the block's 16 labels
// in shared memory (the lane's own block: no other lane touches it)
__device__ __forceinline__ void mutate_block_smem(const EvolveCfg &cfg, int N, int g, int k,
                                                  uint32_t k0, uint32_t k1, int blk,
                                                  uint16_t *lab_s)
{
    const int len = min(MUT_BLOCK, N - MUT_BLOCK * blk);
    if (!cfg.thr_pm || len <= 0) return;
    uint16_t *b = lab_s + MUT_BLOCK * blk;
    int pos = 0;
    for (uint32_t e = 0;; ++e) {
        const U4 w = philox((uint32_t)g, (uint32_t)k, (uint32_t)blk + 65536u * e, STREAM_MUT, k0, k1);
        pos += mutation_skip(w.x, cfg);
        if (pos >= len) break;
        b[pos] = (uint16_t)draw_below(w.y, (uint32_t)N);
        if (++pos >= len) break;
        pos += mutation_skip(w.z, cfg);
        if (pos >= len) break;
        b[pos] = (uint16_t)draw_below(w.w, (uint32_t)N);
        if (++pos >= len) break;
    }
}

// Build child k from plan c: SUS parents (perm read here), crossover,
// mutation; writes the child to dst (global, padded row of Np genes) and
// sl.lab(), and the changed genes X (against parent a) to sl.xs() / xa / xc when
// there are at most DELTA_X of them. Returns the number of changed genes
// (all lanes) and parent a's index in *ia_out.
__device__ __forceinline__ int build_child(const uint16_t *cur, int N, int ldp, int Np,
                                           const EvolveCfg &cfg,
                           const ChildPlan &c, int k, uint32_t k0, uint32_t k1,
                           const int32_t *__restrict__ perm, const uint64_t *__restrict__ prefix,
                           uint16_t *__restrict__ dst, const GatherSlice &sl, int lane,
                           int *ia_out)
{
    const int M = cfg.M, g = c.g;
    const unsigned lt = (1u << lane) - 1u;
    int par;
    if (c.rank >= 0) {
        par = perm[c.rank];
    } else {
        const uint32_t kp = lane < 16 ? (uint32_t)k : (uint32_t)((k + M / 2) % M);
        const uint32_t su = philox((uint32_t)g, 0u, 0u, STREAM_SUS, k0, k1).x;
        const uint64_t W = __ldg(prefix + cfg.P - 1);
        par = cfg.sus_tab ? sus_parent_tab(kp, su, W, M, cfg.P, cfg.m_magic, cfg.m_shift, prefix,
                                           cfg.sus_tab, perm, lane)
                          : sus_parent_half(kp, su, W, M, cfg.P, cfg.m_magic, cfg.m_shift, prefix,
                                            perm, lane);
    }
    const int ia = __shfl_sync(0xffffffffu, par, 0);
    const int ib = __shfl_sync(0xffffffffu, par, 16);
    *ia_out = ia;
    const uint16_t *__restrict__ a = cur + (size_t)ia * ldp;
    const uint16_t *__restrict__ b = cur + (size_t)ib * ldp;
    int mode = 0, cut = N, q = 0;
    if ((uint64_t)c.x0 < cfg.thr_pc) {
        if ((uint64_t)c.x1 < cfg.thr_pkb) {
            mode = 2;
            q = draw_below(c.x2, (uint32_t)N);
        } else {
            mode = 1;
            cut = 1 + draw_below(c.x2, (uint32_t)(N - 1));
        }
    }
    const uint4 *a4 = reinterpret_cast<const uint4 *>(a);
    const uint4 *b4 = reinterpret_cast<const uint4 *>(b);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    uint4 *s4 = reinterpret_cast<uint4 *>(sl.lab());
    const int nblk = Np / MUT_BLOCK;
    int nx = 0;
    for (int blk = lane; blk - lane < nblk; blk += 32) {
        const bool act = blk < nblk;
        uint4 av[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        uint4 bv[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        int aq = 0, bq = 0;
        // every load of the block (and the anchor genes) issued together
        if (act) {
            av[0] = __ldg(a4 + 2 * blk);
            av[1] = __ldg(a4 + 2 * blk + 1);
            if (mode) {
                bv[0] = __ldg(b4 + 2 * blk);
                bv[1] = __ldg(b4 + 2 * blk + 1);
            }
        }
        if (mode == 2) {
            aq = __ldg(a + q);
            bq = __ldg(b + q);
        }
        const uint32_t aw[8] = {av[0].x, av[0].y, av[0].z, av[0].w, av[1].x, av[1].y, av[1].z, av[1].w};
        const uint32_t bw[8] = {bv[0].x, bv[0].y, bv[0].z, bv[0].w, bv[1].x, bv[1].y, bv[1].z, bv[1].w};
        uint32_t v[8];
        const int base = MUT_BLOCK * blk;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int j0 = base + 2 * w, j1 = j0 + 1;
            const int a0 = (int)(aw[w] & 0xffffu), a1 = (int)(aw[w] >> 16);
            const int b0 = (int)(bw[w] & 0xffffu), b1 = (int)(bw[w] >> 16);
            int c0 = a0, c1 = a1;
            if (mode == 1) {
                if (j0 >= cut) c0 = b0;
                if (j1 >= cut) c1 = b1;
            } else if (mode == 2) {
                if (b0 == bq) c0 = aq;
                if (b1 == bq) c1 = aq;
            }
            v[w] = (uint32_t)c0 | ((uint32_t)c1 << 16);
        }
        // mutation: the planned draws of the first block (positions known at
        // compile time after unrolling, so v stays in registers); other blocks,
        // and a first block with more than four mutations, drawn here through
        // the lane's own labels in shared memory
        if (act) {
            if (blk == lane && !c.mover) {
                const uint32_t mm = c.mmask;
                if (mm) {
                    int cnt = 0;
#pragma unroll
                    for (int p = 0; p < 16; ++p) {
                        if ((mm >> p) & 1u) {
                            const uint32_t lw = cnt < 2 ? c.mlab[0] : c.mlab[1];
                            const uint32_t lab = (lw >> ((cnt & 1) << 4)) & 0xffffu;
                            ++cnt;
                            const uint32_t hsh = (uint32_t)(p & 1) << 4;
                            v[p >> 1] = (v[p >> 1] & ~(0xffffu << hsh)) | (lab << hsh);
                        }
                    }
                }
            } else if (cfg.thr_pm) {
                s4[2 * blk] = make_uint4(v[0], v[1], v[2], v[3]);
                s4[2 * blk + 1] = make_uint4(v[4], v[5], v[6], v[7]);
                mutate_block_smem(cfg, N, g, k, k0, k1, blk, sl.lab());
                const uint4 r0 = s4[2 * blk], r1 = s4[2 * blk + 1];
                v[0] = r0.x; v[1] = r0.y; v[2] = r0.z; v[3] = r0.w;
                v[4] = r1.x; v[5] = r1.y; v[6] = r1.z; v[7] = r1.w;
            }
        }
        // genes past N are zero; the changed genes
        uint32_t diff = 0u;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int j0 = base + 2 * w;
            if (j0 >= N) v[w] = 0u;
            else if (j0 + 1 >= N) v[w] &= 0xffffu;
            const uint32_t x = v[w] ^ aw[w];
            if (j0 < N && (x & 0xffffu)) diff |= 1u << (2 * w);
            if (j0 + 1 < N && (x >> 16)) diff |= 1u << (2 * w + 1);
        }
        if (!act) diff = 0u;
        // positions of this lane's changed genes in the list (warp scan)
        const int cnt = __popc(diff);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int pos = nx + incl - cnt;
        if (diff) {
#pragma unroll
            for (int p = 0; p < 16; ++p) {
                if ((diff >> p) & 1u) {
                    if (pos < DELTA_X) {
                        const int hsh = (p & 1) << 4;
                        sl.xs()[pos] = (uint16_t)(base + p);
                        sl.xa()[pos] = (uint16_t)((aw[p >> 1] >> hsh) & 0xffffu);
                        sl.xc()[pos] = (uint16_t)((v[p >> 1] >> hsh) & 0xffffu);
                    }
                    ++pos;
                }
            }
        }
        nx += __shfl_sync(0xffffffffu, incl, 31);
        if (act) {
            const uint4 o0 = make_uint4(v[0], v[1], v[2], v[3]), o1 = make_uint4(v[4], v[5], v[6], v[7]);
            d4[2 * blk] = o0;
            d4[2 * blk + 1] = o1;
            s4[2 * blk] = o0;
            s4[2 * blk + 1] = o1;
        }
    }
    (void)lt;
    __syncwarp();
    return nx;
}

// ---------------------------------------------------------------------------
// Delta scoring of a child (sl.lab() holds it, sl.xs() / xa / xc its nx <=
// DELTA_X changed genes) against its first parent a (d table row ta, Lfix
// lfa, pair count npa): writes the child's d table row tc (a's row with the
// touched clusters updated) and returns its Lfix and pair count. REG: the
// table row (Np <= 512) passes through registers, eight 16-byte loads per
// lane issued before the affected clusters are found and stored once they
// are (the parent's d of those clusters taken from them on the way).
// ---------------------------------------------------------------------------
template <bool REG>
__device__ __forceinline__ void score_delta_warp(const GatherSlice &sl, int N, int Np, int nx,
                                 const long long *__restrict__ ta, long long lfa, long long npa,
                                 long long *__restrict__ tc, const int32_t *__restrict__ Dfix,
                                 int diag, const long long *__restrict__ ltab,
                                 const long long *__restrict__ kfix, int lane, long long *lf_out,
                                 long long *np_out)
{
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
    const longlong2 *ta2 = reinterpret_cast<const longlong2 *>(ta);
    longlong2 *tc2 = reinterpret_cast<longlong2 *>(tc);
    const int nv = Np >> 1; // 16-byte vectors of the row (two labels each)
    longlong2 tv[8];
    if (REG) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (lane + 32 * i < nv) tv[i] = __ldg(ta2 + lane + 32 * i);
    } else {
#pragma unroll 8
        for (int v = lane; v < nv; v += 32) tc2[v] = __ldg(ta2 + v);
    }
    // no label affected yet; bitmap of the changed genes in the list space
    uint16_t *aslot = reinterpret_cast<uint16_t *>(sl.cnt());
    uint32_t *isx = reinterpret_cast<uint32_t *>(sl.list());
    for (int w = lane; w < (Np >> 1); w += 32) reinterpret_cast<uint32_t *>(aslot)[w] = 0xffffffffu;
    for (int w = lane; w < (Np >> 5); w += 32) isx[w] = 0u;
    __syncwarp();
    if (lane < nx) atomicOr(&isx[sl.xs()[lane] >> 5], 1u << (sl.xs()[lane] & 31));
    // the affected clusters: the old and new labels of X, each once
    int na = 0;
    for (int base = 0; base < 2 * nx; base += 32) {
        const int q = base + lane;
        int lab = -1;
        if (q < 2 * nx) lab = q < nx ? (int)sl.xa()[q] : (int)sl.xc()[q - nx];
        const bool fresh = lab >= 0 && aslot[lab] == NO_SLOT;
        const unsigned grp = __match_any_sync(FULL, fresh ? lab : -1 - lane);
        const bool leader = fresh && (__ffs(grp) - 1) == lane;
        const unsigned lb = __ballot_sync(FULL, leader);
        if (leader) {
            const int k = na + __popc(lb & lt);
            aslot[lab] = (uint16_t)k;
            sl.slab()[k] = (uint16_t)lab;
            sl.in_mask()[k] = 0u;
            sl.out_mask()[k] = 0u;
            sl.dacc()[k] = 0;
            sl.dold()[k] = 0;
            sl.nnew()[k] = 0;
            sl.um()[k] = NO_SLOT;
        }
        na += __popc(lb);
        __syncwarp();
    }
    if (lane < nx) {
        atomicOr(&sl.out_mask()[aslot[sl.xa()[lane]]], 1u << lane);
        atomicOr(&sl.in_mask()[aslot[sl.xc()[lane]]], 1u << lane);
    }
    __syncwarp();
    if (REG) {
        // the row arrives: the parent's d of the affected clusters to shared
        // memory, and the row stored to the child unchanged (the touched
        // clusters are overwritten at the end)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int v = lane + 32 * i;
            if (v < nv) {
                const int k0 = aslot[2 * v], k1 = aslot[2 * v + 1];
                if (k0 != NO_SLOT) sl.dold()[k0] = tv[i].x;
                if (k1 != NO_SLOT) sl.dold()[k1] = tv[i].y;
                tc2[v] = tv[i];
            }
        }
    }
    // members of the affected clusters in the child, two genes per lane and
    // step: counted, and those that stayed in place (U) listed in the member space
    uint16_t *ulist = sl.mem();
    const uint32_t *lab2 = reinterpret_cast<const uint32_t *>(sl.lab());
    unsigned *nn2 = reinterpret_cast<unsigned *>(sl.nnew());
    int nu = 0;
#pragma unroll 2
    for (int j0 = 0; j0 < N; j0 += 64) {
        const int j = j0 + 2 * lane;
        int ka = NO_SLOT, kb = NO_SLOT;
        bool sa = false, sb = false;
        if (j < N) {
            const uint32_t w = lab2[j >> 1];
            const uint32_t xb = isx[j >> 5] >> (j & 31);
            ka = aslot[w & 0xffffu];
            if (j + 1 < N) kb = aslot[w >> 16];
            if (ka != NO_SLOT) {
                atomicAdd(nn2 + (ka >> 1), 1u << ((ka & 1) << 4));
                sa = (xb & 1u) == 0u;
                if (sa) sl.um()[ka] = (uint16_t)j; // any one of them
            }
            if (kb != NO_SLOT) {
                atomicAdd(nn2 + (kb >> 1), 1u << ((kb & 1) << 4));
                sb = (xb & 2u) == 0u;
                if (sb) sl.um()[kb] = (uint16_t)(j + 1);
            }
        }
        const unsigned ba = __ballot_sync(FULL, sa), bb = __ballot_sync(FULL, sb);
        const int pa = nu + __popc(ba & lt) + __popc(bb & lt);
        if (sa) ulist[pa] = (uint16_t)j;
        if (sb) ulist[pa + (sa ? 1 : 0)] = (uint16_t)(j + 1);
        nu += __popc(ba) + __popc(bb);
    }
    __syncwarp();
    // 2 [D(U_t, In_t) - D(U_t, Out_t)]: per member left in place, its row of D
    // at the genes that joined or left its cluster; two members per lane and
    // step, four gathers each in flight
    for (int e0 = lane; e0 < nu; e0 += 64) {
        int jj[2], kk[2];
        unsigned mi[2], mm[2];
        long long s[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = e0 + 32 * h;
            jj[h] = e < nu ? (int)ulist[e] : 0;
            kk[h] = e < nu ? (int)aslot[sl.lab()[jj[h]]] : 0;
            mi[h] = e < nu ? sl.in_mask()[kk[h]] : 0u;
            mm[h] = e < nu ? (mi[h] | sl.out_mask()[kk[h]]) : 0u;
        }
        while (mm[0] | mm[1]) {
            int32_t val[2][4];
            unsigned bit[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int32_t *row = Dfix + (size_t)jj[h] * Np;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    bit[h][u] = mm[h] & (~mm[h] + 1u);
                    mm[h] ^= bit[h][u];
                    val[h][u] = bit[h][u] ? __ldg(row + sl.xs()[__ffs(bit[h][u]) - 1]) : 0;
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    s[h] += (bit[h][u] & mi[h]) ? (long long)val[h][u] : -(long long)val[h][u];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (e0 + 32 * h < nu)
                atomicAdd(reinterpret_cast<unsigned long long *>(&sl.dacc()[kk[h]]),
                          (unsigned long long)(2 * s[h]));
    }
    // D(In_t, In_t) - D(Out_t, Out_t): per changed gene, its row at the genes
    // that joined its new cluster with it and at those that left its old one
    if (lane < nx) {
        const int kin = aslot[sl.xc()[lane]], kout = aslot[sl.xa()[lane]];
        const int32_t *row = Dfix + (size_t)sl.xs()[lane] * Np;
        long long si = 0, so = 0;
        for (unsigned m = sl.in_mask()[kin]; m; m &= m - 1) si += __ldg(row + sl.xs()[__ffs(m) - 1]);
        for (unsigned m = sl.out_mask()[kout]; m; m &= m - 1) so += __ldg(row + sl.xs()[__ffs(m) - 1]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&sl.dacc()[kin]), (unsigned long long)si);
        atomicAdd(reinterpret_cast<unsigned long long *>(&sl.dacc()[kout]), (unsigned long long)(-so));
    }
    __syncwarp(); // also orders the table copy before the writes below
    // the touched terms: new minus old
    long long dl = 0, dp = 0;
    for (int k = lane; k < na; k += 32) {
        const int t = sl.slab()[k];
        const unsigned mi = sl.in_mask()[k], mo = sl.out_mask()[k];
        const int nn = (int)sl.nnew()[k];
        const int no = nn - __popc(mi) + __popc(mo);
        long long dold = 0;
        if (no >= 2) {
            dold = REG ? sl.dold()[k] : __ldg(ta + t);
        } else if (no == 1 && diag) { // a singleton's d is its own D_jj
            const int m = mo ? (int)sl.xs()[__ffs(mo) - 1] : (int)sl.um()[k];
            dold = Dfix[(size_t)m * (Np + 1)];
        }
        const long long dnew = dold + sl.dacc()[k];
        const long long tn = nn >= 2 ? cluster_term(nn, dnew, ltab, kfix) : 0;
        const long long to = no >= 2 ? cluster_term(no, dold, ltab, kfix) : 0;
        dl += tn - to;
        dp += (long long)(nn * (nn - 1) / 2) - (long long)(no * (no - 1) / 2);
        if (nn >= 2) tc[t] = dnew;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        dl += __shfl_xor_sync(FULL, dl, o);
        dp += __shfl_xor_sync(FULL, dp, o);
    }
    __syncwarp();
    *lf_out = lfa + dl;
    *np_out = npa + dp;
}

// ---------------------------------------------------------------------------
// Score-only: one warp per individual of lab (stateful: the buffer selected by
// st->gen + sel_off, whose score tables are written when tab is given).
// ---------------------------------------------------------------------------
template <typename LabT>
__global__ void __launch_bounds__(256, 4)
    gather_score_kernel(const LabT *lab0, const LabT *lab1, int ldl, int sel_off, int P, int N,
                        int Np, const int32_t *__restrict__ Dfix, const int *__restrict__ diag_flag,
                        const double *__restrict__ logtab, double *__restrict__ L,
                        int *__restrict__ err, const DevState *__restrict__ st,
                        unsigned long long *__restrict__ pairs, ScoreTab tab)
{
    const LabT *__restrict__ lab = lab0;
    unsigned long long *pairs_g = nullptr;
    int b = 0;
    if (st) {
        if (st->done) return;
        const int gen = st->gen + sel_off;
        b = gen & 1;
        lab = b ? lab1 : lab0;
        if (pairs) pairs_g = pairs + gen;
    }
    extern __shared__ unsigned char smem_g[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const GatherSlice sl =
        gather_slice(smem_g + (size_t)warp * gather_slice_bytes(Np, tab.dbuf(0) != nullptr), Np);
    const long long *ltab = reinterpret_cast<const long long *>(logtab);
    const long long *ktab = kfix_of(logtab);
    const int diag = *diag_flag;
    // the per-cluster form for a single run with score tables and for
    // stateless scoring from DELTA_MIN_N genes up; the product form otherwise
    // (fleet runs included)
    const bool per_cluster = tab.dbuf(0) != nullptr || (!st && uses_delta(N));
    for (int p = blockIdx.x * nw + warp; p < P; p += gridDim.x * nw) {
        bool bad = false;
        const LabT *lp = lab + (size_t)p * ldl;
        for (int i = lane; i < N; i += 32) {
            const int v = (int)lp[i];
            const bool ok = v >= 0 && v < N;
            bad |= !ok;
            sl.lab()[i] = (uint16_t)(ok ? v : 0);
        }
        bad = __any_sync(0xffffffffu, bad);
        __syncwarp();
        long long npairs = 0;
        long long *trow = tab.dbuf(b) ? tab.dbuf(b) + (size_t)p * tab.ldt : nullptr;
        const long long lf =
            per_cluster ? score_full_warp<false>(sl, N, Np, Dfix, diag, ltab, ktab, lane, trow,
                                                 &npairs)
                        : score_full_warp<true>(sl, N, Np, Dfix, diag, ltab, ktab, lane, nullptr,
                                                &npairs);
        if (lane == 0) {
            L[p] = bad ? __longlong_as_double(0x7ff8000000000000ll) : lfix_to_double(lf);
            if (bad && err) atomicOr(err, 1);
            if (tab.lfbuf(b)) {
                tab.lfbuf(b)[p] = lf;
                tab.npbuf(b)[p] = npairs;
            }
            if (pairs_g) atomicAdd(pairs_g, (unsigned long long)npairs);
        }
    }
}

// ---------------------------------------------------------------------------
// Fused generation: warp `slot` builds slot of the next population exactly as
// the evolve kernel does (elite copy, or SUS parents + crossover + mutation)
// into global memory and its shared slice, then scores it: an elite keeps its
// parent's score; a child is scored by delta from its first parent, or from
// scratch when too many genes changed. b: the buffer of the current
// generation g (g & 1); the next one is written to 1 - b. plan: the child's
// draws for generation g (slot >= E). REG_OK: table rows may pass through
// registers (the single-run kernel; the fleet kernel streams them, which
// keeps its item loop within its registers).
// PATH (fixed per instantiation, so that a kernel holds only the code its runs
// use): GEN_PRODUCT, no score tables, every child scored from scratch in the
// product form; GEN_DELTA_REG / GEN_DELTA_STREAM, score tables, children
// scored by delta, the table row through registers (Np <= 512) or streamed.
// ---------------------------------------------------------------------------
enum GenPath : int { GEN_PRODUCT = 0, GEN_DELTA_REG = 1, GEN_DELTA_STREAM = 2 };

template <bool REG_OK, int PATH>
__device__ __forceinline__ void generation_slot(const uint16_t *cur, uint16_t *nxt, int N, int ldp,
                                                const EvolveCfg &cfg, const ChildPlan &plan,
                                                uint32_t k0, uint32_t k1, int slot,
                                                const int32_t *__restrict__ perm,
                                                const uint64_t *__restrict__ prefix, int Np,
                                                const int32_t *__restrict__ Dfix, int diag,
                                                const double *__restrict__ logtab,
                                                double *__restrict__ L, const ScoreTab &tab,
                                                const GatherSlice &sl, int lane,
                                                unsigned long long *pairs_out,
                                                const SusPre *pre = nullptr)
{
    const int b = plan.g & 1, nb = b ^ 1;
    uint16_t *dst = nxt + (size_t)slot * ldp;
    const long long *ltab = reinterpret_cast<const long long *>(logtab);
    const long long *kfix = kfix_of(logtab);
    long long lf, np;
    if (PATH == GEN_PRODUCT) {
        // no score tables (N < DELTA_MIN_N, or a fleet): the child is built by
        // the pair loop of child_genes and scored from scratch in the
        // one-log product form
        if (slot < cfg.E) {
            const uint16_t *src = cur + (size_t)perm[slot] * ldp;
            for (int j = lane; j < N; j += 32) {
                const uint16_t v = src[j];
                dst[j] = v;
                sl.lab()[j] = v;
            }
        } else {
            EvolveCfg c2 = cfg;
            c2.N = N;
            c2.ldp = ldp;
            child_genes<uint16_t>(cur, ldp, N, c2, plan.g, slot - cfg.E, k0, k1, perm, prefix,
                                  nullptr, dst, sl.lab(), lane, pre);
        }
        __syncwarp();
        lf = score_full_warp<true>(sl, N, Np, Dfix, diag, ltab, kfix, lane, nullptr, &np);
        if (lane == 0) {
            L[slot] = lfix_to_double(lf);
            if (pairs_out) atomicAdd(pairs_out, (unsigned long long)np);
        }
        return;
    }
    long long *tc = tab.dbuf(nb) + (size_t)slot * tab.ldt;
    if (slot < cfg.E) {
        // elite: labels, table and score of the parent, unchanged
        const int src_i = perm[slot];
        const uint16_t *src = cur + (size_t)src_i * ldp;
        for (int j = lane; j < N; j += 32) dst[j] = src[j];
        const int4 *ts = reinterpret_cast<const int4 *>(tab.dbuf(b) + (size_t)src_i * tab.ldt);
        int4 *td = reinterpret_cast<int4 *>(tc);
#pragma unroll 8
        for (int v = lane; v < (Np >> 1); v += 32) td[v] = __ldg(ts + v);
        lf = tab.lfbuf(b)[src_i];
        np = tab.npbuf(b)[src_i];
    } else {
        const int k = slot - cfg.E;
        int ia;
        const int nx = build_child(cur, N, ldp, Np, cfg, plan, k, k0, k1, perm, prefix, dst, sl,
                                   lane, &ia);
        const long long lfa = tab.lfbuf(b)[ia], npa = tab.npbuf(b)[ia];
        const long long *ta = tab.dbuf(b) + (size_t)ia * tab.ldt;
        if (nx <= DELTA_X) {
            if (REG_OK && PATH == GEN_DELTA_REG)
                score_delta_warp<true>(sl, N, Np, nx, ta, lfa, npa, tc, Dfix, diag, ltab, kfix,
                                       lane, &lf, &np);
            else
                score_delta_warp<false>(sl, N, Np, nx, ta, lfa, npa, tc, Dfix, diag, ltab, kfix,
                                        lane, &lf, &np);
        } else {
            lf = score_full_warp<false>(sl, N, Np, Dfix, diag, ltab, kfix, lane, tc, &np);
        }
    }
    if (lane == 0) {
        L[slot] = lfix_to_double(lf);
        tab.lfbuf(nb)[slot] = lf;
        tab.npbuf(nb)[slot] = np;
        if (pairs_out) atomicAdd(pairs_out, (unsigned long long)np);
    }
}

template <int PATH>
__global__ void __launch_bounds__(128, 7)
    gather_generation_kernel(const uint16_t *pop0, const uint16_t *pop1, uint16_t *next0,
                             uint16_t *next1, EvolveCfg cfg, const int32_t *__restrict__ perm,
                             const uint64_t *__restrict__ prefix, int Np,
                             const int32_t *__restrict__ Dfix, const int *__restrict__ diag_flag,
                             const double *__restrict__ logtab, double *__restrict__ L,
                             DevState *__restrict__ st, unsigned long long *__restrict__ pairs,
                             ScoreTab tab)
{
    extern __shared__ unsigned char smem_g[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int slot = blockIdx.x * nw + warp;
    if (slot >= cfg.P) return;
    // the run's Philox key (written when the run started, long before)
    const uint32_t k0 = st->k0, k1 = st->k1;
    // Everything of the child that depends on neither parent, drawn before the
    // wait below for the generation read from the state now (the selection
    // writes it before it lets this kernel be scheduled; if the value read is
    // stale, the draws are made again after the wait): the SUS brackets of
    // the fixed rank prefix and the pointer's rank, the crossover words, the
    // mutations of the lane's first block.
    SusPre pre;
    const bool use_pre = cfg.sus_tab != nullptr && slot >= cfg.E;
    if (use_pre) pre = sus_prefetch((uint32_t)(slot - cfg.E), cfg.M, cfg.P, prefix, cfg.sus_tab, lane);
    constexpr bool delta = PATH != GEN_PRODUCT;
    const int g_hint = *reinterpret_cast<volatile const int *>(&st->gnext);
    ChildPlan plan;
    plan.g = g_hint;
    if (delta && slot >= cfg.E)
        plan = plan_child(cfg, cfg.N, g_hint, slot - cfg.E, k0, k1, use_pre ? &pre : nullptr, lane);
    // launched as a programmatic dependent of the selection: wait for that grid
    // before reading perm and the state
    griddep_wait();
    if (st->done) return;
    const int g = st->gen;
    if (slot == 0 && lane == 0) st->gnext = g + 1;
    if (delta && slot >= cfg.E && g != plan.g)
        plan = plan_child(cfg, cfg.N, g, slot - cfg.E, k0, k1, use_pre ? &pre : nullptr, lane);
    plan.g = g;
    const uint16_t *cur = (g & 1) ? pop1 : pop0;
    uint16_t *nxt = (g & 1) ? next1 : next0;
    const GatherSlice sl = gather_slice(smem_g + (size_t)warp * gather_slice_bytes(Np, delta), Np);
    generation_slot<true, PATH>(cur, nxt, cfg.N, cfg.ldp, cfg, plan, k0, k1, slot, perm, prefix, Np, Dfix,
                          *diag_flag, logtab, L, tab, sl, lane, pairs ? pairs + g + 1 : nullptr,
                          use_pre ? &pre : nullptr);
}

// ---------------------------------------------------------------------------
// Fleet generation: work item i is slot i mod P of the run at table position
// i / P (the table is ordered by decreasing N, so the costly runs start
// first); the CTAs stride over the items. Runs whose state is done are
// skipped. Per slot the work is that of gather_generation_kernel without
// score tables: every child is scored from scratch in the product form, so
// a run's result equals the same run alone for N < DELTA_MIN_N (from
// DELTA_MIN_N genes up a single run uses the per-cluster form, whose L can
// differ from the product form's in the last bits).
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
    unsigned char *slice = smem_g + (size_t)warp * gather_slice_bytes(Np_max, false);
    const int nitems = hdr->nitems, P = base.P;
    for (int item = blockIdx.x * nw + warp; item < nitems; item += gridDim.x * nw) {
        const int ri = item / P, slot = item - ri * P;
        const FleetRun &r = runs[ri];
        const DevState *st = r.st;
        if (st->done) continue;
        const int g = st->gen;
        const uint16_t *cur = (g & 1) ? r.pop1 : r.pop0;
        uint16_t *nxt = (g & 1) ? r.pop0 : r.pop1;
        const uint64_t *prefix = prop ? r.work_prefix : rank_prefix;
        const GatherSlice sl = gather_slice(slice, r.Np);
        ChildPlan plan;
        plan.g = g;
        SusPre pre;
        const bool use_pre = slot >= base.E && !prop && base.sus_tab != nullptr;
        if (use_pre)
            pre = sus_prefetch((uint32_t)(slot - base.E), base.M, P, prefix, base.sus_tab, lane);
        generation_slot<false, GEN_PRODUCT>(cur, nxt, r.N, r.Np, base, plan, st->k0, st->k1, slot,
                                      r.perm, prefix, r.Np, r.Dfix, *r.diag, logtab, r.L,
                                      ScoreTab{}, sl, lane, nullptr, use_pre ? &pre : nullptr);
        __syncwarp();
    }
}

// warps per CTA of the single-run gather kernels: 4 (measured at N=500,
// P=4096: 1024 CTAs of 4 warps spread over the SMs more evenly than 512 of 8,
// 4% less time per generation), fewer if the slices do not fit
static int warps_for(int Np, bool delta)
{
    const size_t per = gather_slice_bytes(Np, delta);
    int nw = 4;
    while (nw > 1 && nw * per > (size_t)200 * 1024) nw >>= 1;
    return nw;
}

size_t score_tab_row_bytes(int Np) { return (size_t)Np * sizeof(long long); }

template <typename LabT>
int launch_gather_score(const LabT *const *lab2, int ldl, int sel_off, int P, int N, int Np,
                        const int32_t *Dfix, const int *diag_flag, const double *logtab,
                        double *L, int *err, const DevState *st, unsigned long long *pairs,
                        const ScoreTab &tab, cudaStream_t s)
{
    const bool delta = tab.dbuf(0) != nullptr;
    const int nw = warps_for(Np, delta);
    const size_t smem = nw * gather_slice_bytes(Np, delta);
    const int grid = (P + nw - 1) / nw;
    gather_score_kernel<LabT><<<grid, 32 * nw, smem, s>>>(lab2[0], lab2[1], ldl, sel_off, P, N,
                                                          Np, Dfix, diag_flag, logtab, L, err,
                                                          st, pairs, tab);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

int launch_gather_generation(const uint16_t *const *pop2, uint16_t *const *next2,
                             const EvolveCfg &cfg, const int32_t *perm, const uint64_t *prefix,
                             int Np, const int32_t *Dfix, const int *diag_flag,
                             const double *logtab, double *L, DevState *st,
                             unsigned long long *pairs, const ScoreTab &tab, bool pdl,
                             cudaStream_t s)
{
    const bool delta = tab.dbuf(0) != nullptr;
    const int nw = warps_for(Np, delta);
    const size_t smem = nw * gather_slice_bytes(Np, delta);
    const int grid = (cfg.P + nw - 1) / nw;
    const int path = !delta ? GEN_PRODUCT : (Np <= 512 ? GEN_DELTA_REG : GEN_DELTA_STREAM);
    if (path == GEN_PRODUCT)
        GPGA_CUDA(launch_pdl(gather_generation_kernel<GEN_PRODUCT>, dim3(grid), dim3(32 * nw), smem,
                             s, pdl, pop2[0], pop2[1], next2[0], next2[1], cfg, perm, prefix, Np,
                             Dfix, diag_flag, logtab, L, st, pairs, tab));
    else if (path == GEN_DELTA_REG)
        GPGA_CUDA(launch_pdl(gather_generation_kernel<GEN_DELTA_REG>, dim3(grid), dim3(32 * nw),
                             smem, s, pdl, pop2[0], pop2[1], next2[0], next2[1], cfg, perm, prefix,
                             Np, Dfix, diag_flag, logtab, L, st, pairs, tab));
    else
        GPGA_CUDA(launch_pdl(gather_generation_kernel<GEN_DELTA_STREAM>, dim3(grid), dim3(32 * nw),
                             smem, s, pdl, pop2[0], pop2[1], next2[0], next2[1], cfg, perm, prefix,
                             Np, Dfix, diag_flag, logtab, L, st, pairs, tab));
    return GPGA_OK;
}

int fleet_max_warps(int Np_max)
{
    int nw = 16;
    while (nw > 1 && nw * gather_slice_bytes(Np_max, false) > (size_t)200 * 1024) nw >>= 1;
    return nw;
}

int fleet_ctas_per_sm(int Np_max, int warps, int *out)
{
    GPGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        out, fleet_generation_kernel, 32 * warps, warps * gather_slice_bytes(Np_max, false)));
    return GPGA_OK;
}

int launch_fleet_generation(const FleetRun *runs, const FleetHdr *hdr, const EvolveCfg &cfg,
                            const uint64_t *rank_prefix, const double *logtab, int Np_max,
                            int warps, int ctas, int prop, cudaStream_t s, bool pdl)
{
    if (warps < 1 || warps > 16 || ctas < 1)
        return set_error(GPGA_ERR_ARG, "fleet generation: %d warps x %d CTAs", warps, ctas);
    const size_t smem = warps * gather_slice_bytes(Np_max, false);
    GPGA_CUDA(launch_pdl(fleet_generation_kernel, dim3(ctas), dim3(32 * warps), smem, s, pdl, runs,
                         hdr, cfg, rank_prefix, logtab, Np_max, prop));
    return GPGA_OK;
}

template int launch_gather_score<uint16_t>(const uint16_t *const *, int, int, int, int, int,
                                           const int32_t *, const int *, const double *, double *,
                                           int *, const DevState *, unsigned long long *,
                                           const ScoreTab &, cudaStream_t);
template int launch_gather_score<int32_t>(const int32_t *const *, int, int, int, int, int,
                                          const int32_t *, const int *, const double *, double *,
                                          int *, const DevState *, unsigned long long *,
                                          const ScoreTab &, cudaStream_t);

int prepare_gather_kernels(int maxsmem)
{
    if (int rc = raise_smem(gather_score_kernel<uint16_t>, maxsmem)) return rc;
    if (int rc = raise_smem(gather_score_kernel<int32_t>, maxsmem)) return rc;
    if (int rc = raise_smem(gather_generation_kernel<GEN_PRODUCT>, maxsmem)) return rc;
    if (int rc = raise_smem(gather_generation_kernel<GEN_DELTA_REG>, maxsmem)) return rc;
    if (int rc = raise_smem(gather_generation_kernel<GEN_DELTA_STREAM>, maxsmem)) return rc;
    if (int rc = raise_smem(fleet_generation_kernel, maxsmem)) return rc;
    return GPGA_OK;
}

} // namespace gpga
