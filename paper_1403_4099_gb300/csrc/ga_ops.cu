// ga_ops.cu -- the device-resident GA generation of Algorithm 1 after scoring:
// evaluate state and statistics, termination test, isolate fittest, elitism,
// scaling, SUS selection (one single-CTA kernel), then crossover, mutation and
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

int rank_prefix_table(uint64_t *prefix, int P, cudaStream_t s)
{
    rank_prefix_kernel<<<1, 1024, 0, s>>>(prefix, P);
    GPGA_LAUNCH_CHECK();
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
    st->best = 0.0;
    st->mean = 0.0;
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

// ---------------------------------------------------------------------------
// SUS pointer x_k = floor((k 2^32 + u) W / (M 2^32)) in exact integer
// arithmetic: A = (k 2^32 + u) W < 2^127 as two 64-bit words, divided by M with
// 32-bit long division, then shifted right by 32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sus_pointer(uint32_t k, uint32_t u, uint64_t W, uint32_t M)
{
    const uint64_t num = ((uint64_t)k << 32) | u;
    const uint64_t lo = num * W;
    const uint64_t hi = __umul64hi(num, W);
    // 128-bit (hi:lo) / M, limb by limb (32-bit limbs, most significant first)
    const uint32_t limb[4] = {(uint32_t)(hi >> 32), (uint32_t)hi, (uint32_t)(lo >> 32),
                              (uint32_t)lo};
    uint32_t q[4];
    uint64_t rem = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const uint64_t cur = (rem << 32) | limb[t];
        q[t] = (uint32_t)(cur / M);
        rem = cur % M;
    }
    // quotient >> 32 = limbs q0 q1 q2 (q0 is zero since the pointer is below W)
    return ((uint64_t)q[1] << 32) | q[2];
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

// strict "fitter than" of (key, index) pairs: key descending, index ascending
__device__ __forceinline__ bool fitter(unsigned long long ka, int ia, unsigned long long kb, int ib)
{
    return ka > kb || (ka == kb && ia < ib);
}

// ---------------------------------------------------------------------------
// Selection kernel (one CTA of 1024 threads). Stateful use (st != nullptr):
// g = st->gen + gen_off becomes the current generation; records best L, best
// labels and the device clock; tests termination and sets st->done.
// Then: bitonic sort of (L, index) -> perm; scaling weights -> inclusive
// prefix (RANK: precomputed table; PROP: computed and scanned here); SUS.
// Shared memory: Pp keys (double, later reused for the uint64 prefix) and
// Pp indices, Pp = next power of two >= P.
// ---------------------------------------------------------------------------
template <typename LabT>
__global__ void __launch_bounds__(1024)
    select_kernel(const double *__restrict__ L, SelectCfg cfg,
                  const uint64_t *__restrict__ rank_prefix, int32_t *__restrict__ perm,
                  int32_t *__restrict__ parents, DevState *st, double *__restrict__ hist,
                  const LabT *pop0, const LabT *pop1, LabT *__restrict__ ring,
                  unsigned long long *__restrict__ ts, int Pp)
{
    extern __shared__ unsigned long long sm_key[];
    int *sm_idx = reinterpret_cast<int *>(sm_key + Pp);
    __shared__ int s_done;
    __shared__ double s_red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    int g = cfg.gen_off;
    uint32_t k0 = cfg.k0, k1 = cfg.k1;
    if (st) {
        if (st->done) return;
        g = st->gen + cfg.gen_off;
        k0 = st->k0;
        k1 = st->k1;
    }
    const int P = cfg.P;
    for (int i = tid; i < Pp; i += nt) {
        sm_key[i] = i < P ? order_key(L[i]) : 0ull; // padding below every real key
        sm_idx[i] = i;
    }
    __syncthreads();
    // bitonic sort into "fitter first" order
    for (int k = 2; k <= Pp; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = tid; t < (Pp >> 1); t += nt) {
                const int i = ((t / j) * 2 * j) + (t % j);
                const int l = i + j;
                const unsigned long long ki = sm_key[i], kl = sm_key[l];
                const int ii = sm_idx[i], il = sm_idx[l];
                const bool up = (i & k) == 0;
                const bool swap = up ? fitter(kl, il, ki, ii) : fitter(ki, ii, kl, il);
                if (swap) {
                    sm_key[i] = kl;
                    sm_key[l] = ki;
                    sm_idx[i] = il;
                    sm_idx[l] = ii;
                }
            }
            __syncthreads();
        }
    }

    if (st) {
        // statistics: best, mean (fixed-order reduction)
        double part = 0.0;
        for (int i = tid; i < P; i += nt) part += L[i];
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = part;
        __syncthreads();
        const int bidx = sm_idx[0];
        double best = L[bidx];
        if (isnan(best)) best = -INFINITY;
        if (tid == 0) {
            double m = 0.0;
            for (int w = 0; w < (nt >> 5); ++w) m += s_red[w];
            st->gen = g;
            st->best = best;
            st->best_idx = bidx;
            st->mean = m / (double)P;
            hist[g] = best;
            int done = g >= cfg.max_gens;
            if (!done && cfg.tol >= 0.0 && cfg.stall_gens > 0 && g >= cfg.stall_gens) {
                const double prev = hist[g - cfg.stall_gens];
                done = (best - prev) <= cfg.tol * fmax(1.0, fabs(best));
            }
            s_done = done;
        }
        if (cfg.record && ring) {
            const LabT *src = ((g & 1) ? pop1 : pop0) + (size_t)bidx * cfg.ldp;
            for (int j = tid; j < cfg.N; j += nt) ring[(size_t)g * cfg.N + j] = src[j];
        }
        __syncthreads();
        if (cfg.record && ts && tid == 0) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            ts[1 + g] = t;
        }
        if (s_done) {
            if (tid == 0) st->done = 1;
            return;
        }
    }

    for (int r = tid; r < P; r += nt) perm[r] = sm_idx[r];

    // scaling -> inclusive prefix in the key array (reinterpreted as uint64)
    uint64_t *pre = reinterpret_cast<uint64_t *>(sm_key);
    if (cfg.scaling == GPGA_SCALING_RANK) {
        __syncthreads();
        for (int r = tid; r < P; r += nt) pre[r] = rank_prefix[r];
        __syncthreads();
    } else {
        double lmax = L[sm_idx[0]];
        if (isnan(lmax)) lmax = -INFINITY;
        __syncthreads();
        for (int r = tid; r < P; r += nt) {
            uint64_t w = 1;
            if (lmax > 0.0) {
                double x = L[sm_idx[r]];
                if (!(x > 0.0)) x = 0.0;
                w = (uint64_t)floor(__dmul_rn(__ddiv_rn(x, lmax), 4294967296.0));
            }
            pre[r] = w; // same slot, read above by this thread only
        }
        __syncthreads();
        // chunked inclusive scan
        const int chunk = (P + nt - 1) / nt;
        const int lo = tid * chunk, hi = min(P, lo + chunk);
        uint64_t s = 0;
        for (int r = lo; r < hi; ++r) {
            s += pre[r];
            pre[r] = s;
        }
        __shared__ uint64_t s_part[1024];
        s_part[tid] = s;
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
        for (int r = lo; r < hi; ++r) pre[r] += s_part[tid];
        __syncthreads();
    }

    // SUS: M pointers, parent = first rank whose prefix exceeds the pointer.
    // Thread t takes a contiguous run of pointers: the first by exact 128-bit
    // division, the next ones by exact increments (numerator + 2^32 W, carried
    // against the divisor M 2^32).
    const uint64_t W = pre[P - 1];
    const U4 w = philox((uint32_t)g, 0u, 0u, STREAM_SUS, k0, k1);
    const int M = cfg.M;
    const int per = (M + nt - 1) / nt;
    const int k_lo = tid * per, k_hi = min(M, k_lo + per);
    if (k_lo < k_hi) {
        uint64_t x = sus_pointer((uint32_t)k_lo, w.x, W, (uint32_t)M);
        // remainder of the first numerator modulo M 2^32, as (rem_hi < M, rem_lo)
        const uint64_t num = ((uint64_t)(uint32_t)k_lo << 32) | w.x;
        const uint64_t plo = num * W, phi = __umul64hi(num, W);
        // (phi:plo) - x * M * 2^32
        const uint64_t xm_lo = (x * (uint64_t)M) << 32;
        const uint64_t xm_hi = __umul64hi(x, (uint64_t)M << 32);
        uint64_t r_lo = plo - xm_lo;
        uint64_t r_hi = phi - xm_hi - (plo < xm_lo ? 1ull : 0ull);
        // step 2^32 W = qs (M 2^32) + rs, qs = W / M, rs = (W mod M) 2^32
        const uint64_t qs = W / (uint64_t)M, rsm = W % (uint64_t)M;
        const uint64_t dm = (uint64_t)M; // divisor is dm * 2^32: compare (r_hi:r_lo) >= (dm:0)
        int lo = 0;
        for (int k = k_lo; k < k_hi; ++k) {
            if (k > k_lo) {
                x += qs;
                // remainder += rsm * 2^32
                const uint64_t add_lo = rsm << 32, add_hi = rsm >> 32;
                const uint64_t nlo = r_lo + add_lo;
                r_hi = r_hi + add_hi + (nlo < r_lo ? 1ull : 0ull);
                r_lo = nlo;
                if (r_hi > (dm >> 32) || (r_hi == (dm >> 32) && r_lo >= (dm << 32))) {
                    const uint64_t sub_lo = dm << 32, sub_hi = dm >> 32;
                    const uint64_t n2 = r_lo - sub_lo;
                    r_hi = r_hi - sub_hi - (r_lo < sub_lo ? 1ull : 0ull);
                    r_lo = n2;
                    x += 1;
                }
            }
            int hi = P - 1;
            while (lo < hi) { // pointers grow with k: the search restarts at the last hit
                const int mid = (lo + hi) >> 1;
                if (pre[mid] > x)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            parents[k] = sm_idx[lo];
        }
    }
}

template <typename LabT>
int launch_select(const double *L, const SelectCfg &cfg, const uint64_t *rank_prefix,
                  int32_t *perm, int32_t *parents, DevState *st, double *hist,
                  const LabT *const *pop2, LabT *ring, unsigned long long *ts, cudaStream_t s)
{
    int Pp = 1;
    while (Pp < cfg.P) Pp <<= 1;
    const size_t smem = (size_t)Pp * (sizeof(unsigned long long) + sizeof(int));
    select_kernel<LabT><<<1, 1024, smem, s>>>(L, cfg, rank_prefix, perm, parents, st, hist,
                            pop2 ? pop2[0] : nullptr, pop2 ? pop2[1] : nullptr, ring, ts, Pp);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template int launch_select<uint16_t>(const double *, const SelectCfg &, const uint64_t *,
                                     int32_t *, int32_t *, DevState *, double *,
                                     const uint16_t *const *, uint16_t *, unsigned long long *,
                                     cudaStream_t);
template int launch_select<int32_t>(const double *, const SelectCfg &, const uint64_t *,
                                    int32_t *, int32_t *, DevState *, double *,
                                    const int32_t *const *, int32_t *, unsigned long long *,
                                    cudaStream_t);

// ---------------------------------------------------------------------------
// Crossover + mutation + replacement, one warp per slot of the next population.
// Slots 0..E-1: elites in rank order, copied. Slot E + k: child k of
//   a = parents[k], b = parents[(k + M/2) mod M];
//   Philox(g, k, 0, XOVER) = (x, y, z, .): crossover if x < thr(P_c); then
//   knowledge-based merge if y < thr(P_kb) with anchor q = draw(z, N):
//   child_j = a_q where b_j = b_q, else a_j; otherwise one-point at
//   cut = 1 + draw(z, N - 1): child_j = a_j for j < cut, b_j after.
//   Mutation, gene pair (2m, 2m+1): Philox(g, k, m, MUT) = (f0, v0, f1, v1):
//   child_j = draw(v, N) if f < thr(P_m).
// Every gene is a function of (a_j, b_j) and warp-uniform values, so lanes
// stream gene pairs with no shared memory.
// ---------------------------------------------------------------------------
template <typename LabT>
__global__ void __launch_bounds__(256)
    evolve_kernel(const LabT *pop0, const LabT *pop1, LabT *next0, LabT *next1, EvolveCfg cfg,
                  const int32_t *__restrict__ perm, const int32_t *__restrict__ parents,
                  const DevState *__restrict__ st)
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
    const int k = slot - cfg.E;
    const int M = cfg.M;
    const LabT *a = cur + (size_t)parents[k] * ldp;
    const LabT *b = cur + (size_t)parents[(k + M / 2) % M] * ldp;
    const U4 xw = philox((uint32_t)g, (uint32_t)k, 0u, STREAM_XOVER, k0, k1);
    int mode = 0, cut = N;
    int bq = 0, aq = 0;
    if ((uint64_t)xw.x < cfg.thr_pc) {
        if ((uint64_t)xw.y < cfg.thr_pkb) {
            mode = 2;
            const int q = draw_below(xw.z, (uint32_t)N);
            bq = (int)b[q];
            aq = (int)a[q];
        } else {
            mode = 1;
            cut = 1 + draw_below(xw.z, (uint32_t)(N - 1));
        }
    }
    const int npair = (N + 1) >> 1;
    for (int m = lane; m < npair; m += 32) {
        const int j0 = 2 * m, j1 = 2 * m + 1;
        int a0 = (int)a[j0], b0 = (int)b[j0];
        int a1 = 0, b1 = 0;
        if (j1 < N) {
            a1 = (int)a[j1];
            b1 = (int)b[j1];
        }
        int c0 = a0, c1 = a1;
        if (mode == 1) {
            if (j0 >= cut) c0 = b0;
            if (j1 >= cut) c1 = b1;
        } else if (mode == 2) {
            if (b0 == bq) c0 = aq;
            if (b1 == bq) c1 = aq;
        }
        const U4 mw = philox((uint32_t)g, (uint32_t)k, (uint32_t)m, STREAM_MUT, k0, k1);
        if ((uint64_t)mw.x < cfg.thr_pm) c0 = draw_below(mw.y, (uint32_t)N);
        if ((uint64_t)mw.z < cfg.thr_pm) c1 = draw_below(mw.w, (uint32_t)N);
        dst[j0] = (LabT)c0;
        if (j1 < N) dst[j1] = (LabT)c1;
    }
}

template <typename LabT>
int launch_evolve(const LabT *const *pop2, LabT *const *next2, const EvolveCfg &cfg,
                  const int32_t *perm, const int32_t *parents, const DevState *st,
                  cudaStream_t s)
{
    const int grid = (cfg.P + 7) / 8;
    evolve_kernel<LabT><<<grid, 256, 0, s>>>(pop2[0], pop2[1], next2[0], next2[1], cfg, perm,
                                             parents, st);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template int launch_evolve<uint16_t>(const uint16_t *const *, uint16_t *const *,
                                     const EvolveCfg &, const int32_t *, const int32_t *,
                                     const DevState *, cudaStream_t);
template int launch_evolve<int32_t>(const int32_t *const *, int32_t *const *, const EvolveCfg &,
                                    const int32_t *, const int32_t *, const DevState *,
                                    cudaStream_t);

int prepare_ga_kernels(int maxsmem)
{
    if (int rc = raise_smem(select_kernel<uint16_t>, maxsmem)) return rc;
    if (int rc = raise_smem(select_kernel<int32_t>, maxsmem)) return rc;
    return GPGA_OK;
}

} // namespace gpga
