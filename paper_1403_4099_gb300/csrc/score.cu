// score.cu -- Giada-Marsili log-likelihood L_c of a population (Eq. 5, 6, 8),
// plain form on CUDA cores, plus the FP64 assembly shared with the tensor form
// and the FP64 final re-score of one configuration.
//
// Split of the work (D = 1 - C, symmetric, zero diagonal for a Pearson C):
//   d_s = sum_{i,j in s} D_ij = sum_{i in s} (2 u_i + D_ii),
//   u_i = sum_{j > i, s_j = s_i} D_ij        (pair kernel, FP32, upper triangle)
//   n_s, d_s per cluster -> c_s = n_s^2 - d_s -> Eq. 8 terms in FP64 (assembly)
// Accumulating 1 - C_ij directly keeps n_s^2 - c_s free of cancellation.
#include <math.h>

#include <cooperative_groups.h>

#include "gpga_internal.cuh"

namespace gpga {

int fix_bits_for(int N)
{
    // 2 N^2 2^bits < 2^62 with margin
    double need = log2(2.0 * (double)N * (double)N + 1.0);
    int bits = 61 - (int)ceil(need);
    if (bits > 40) bits = 40;
    if (bits < 20) bits = 20;
    return bits;
}

// entry k of the log_q62() table: inv_k = fl(1 / c_k) 2^62 (exact: a 53-bit
// double scaled by a power of two), t_k = -log(inv_k 2^-62) in Q62
__device__ __forceinline__ void log_tab_entry(int k, long long *out)
{
    const double c = 1.0 + ((double)k + 0.5) / (double)LOG_TAB;
    const double v = 1.0 / c;
    out[0] = (long long)(v * 4611686018427387904.0);
    out[1] = __double2ll_rn(-log(v) * 4611686018427387904.0);
}

// the log tables (threads tid of nt): log_q62()'s table, then the per-size
// constant of the assembly, K[n] = 1/2 (log n + (n - 1) log(n (n - 1))), in
// fixed point 2^-44, n = 0..N
__device__ __forceinline__ void fill_logtab(double *logtab, int N, int tid, int nt)
{
    for (int k = tid; k < LOG_TAB; k += nt)
        log_tab_entry(k, reinterpret_cast<long long *>(logtab) + 2 * k);
    long long *kfix = reinterpret_cast<long long *>(logtab + 2 * LOG_TAB);
    for (int n = tid; n <= N; n += nt) {
        double v = 0.0;
        if (n >= 2) {
            const double dn = (double)n;
            v = 0.5 * (log(dn) + (dn - 1.0) * (log(dn) + log(dn - 1.0)));
        }
        kfix[n] = __double2ll_rn(v * 17592186044416.0); // 2^44
    }
}

// D 2^30 rounded, saturated to the int32 range (D in [-2, 2))
__device__ __forceinline__ int32_t dfix_of(double d)
{
    double v = rint(d * 1073741824.0);
    if (v > 2147483647.0) v = 2147483647.0;
    if (v < -2147483648.0) v = -2147483648.0;
    return (int32_t)v;
}

// ---------------------------------------------------------------------------
// D forms: D32 = fp32(1 - (C + C^T)/2), Dhi = bf16(D), Dlo = bf16(D - Dhi),
// Dfix = int32(D 2^30), all Np x Np, zero outside N x N; and the log tables.
// ---------------------------------------------------------------------------
__global__ void prep_d_kernel(const double *__restrict__ C, int N, int ldc, int Np,
                              float *__restrict__ D32, __nv_bfloat16 *__restrict__ Dhi,
                              __nv_bfloat16 *__restrict__ Dlo, int32_t *__restrict__ Dfix,
                              double *__restrict__ logtab, int *__restrict__ diag_flag)
{
    const size_t total = (size_t)Np * Np;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / Np), j = (int)(idx - (size_t)i * Np);
        double d = 0.0;
        if (i < N && j < N) {
            const double cij = C[(size_t)i * ldc + j], cji = C[(size_t)j * ldc + i];
            d = 1.0 - 0.5 * (cij + cji);
        }
        const float df = (float)d;
        D32[idx] = df;
        if (diag_flag && i == j && df != 0.f) *diag_flag = 1;
        if (Dfix) Dfix[idx] = dfix_of(d);
        if (Dhi) {
            const __nv_bfloat16 hi = __double2bfloat16(d);
            const double rem = d - (double)__bfloat162float(hi);
            Dhi[idx] = hi;
            Dlo[idx] = __double2bfloat16(rem);
        }
    }
    if (logtab)
        fill_logtab(logtab, N, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void logtab_kernel(double *__restrict__ logtab, int N)
{
    fill_logtab(logtab, N, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

int launch_logtab(double *logtab, int N, cudaStream_t s)
{
    logtab_kernel<<<(N + 1 + 255) / 256 + 1, 256, 0, s>>>(logtab, N);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

// One fleet run's inputs: C gathered through the optional column subset into
// a dense N x N copy (for the final re-score; C64 == nullptr when C already is
// that copy), and the fixed-point D of the gather form with its diagonal
// flag, element for element as prep_d_kernel.
__global__ void fleet_prep_kernel(const double *__restrict__ C, int ldc,
                                  const int32_t *__restrict__ cols, int N, int Np,
                                  double *__restrict__ C64, int32_t *__restrict__ Dfix,
                                  int *__restrict__ diag_flag)
{
    const size_t total = (size_t)Np * Np;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / Np), j = (int)(idx - (size_t)i * Np);
        double d = 0.0;
        if (i < N && j < N) {
            const int ci = cols ? cols[i] : i, cj = cols ? cols[j] : j;
            const double cij = C[(size_t)ci * ldc + cj], cji = C[(size_t)cj * ldc + ci];
            if (C64) C64[(size_t)i * N + j] = cij;
            d = 1.0 - 0.5 * (cij + cji);
        }
        if (diag_flag && i == j && (float)d != 0.f) *diag_flag = 1;
        Dfix[idx] = dfix_of(d);
    }
}

int launch_fleet_prep(const double *C, int ldc, const int32_t *cols, int N, int Np, double *C64,
                      int32_t *Dfix, int *diag_flag, cudaStream_t s)
{
    const size_t total = (size_t)Np * Np;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    fleet_prep_kernel<<<blocks, 256, 0, s>>>(C, ldc, cols, N, Np, C64, Dfix, diag_flag);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

int launch_prep_d(const double *C, int N, int ldc, int Np, float *D32, __nv_bfloat16 *Dhi,
                  __nv_bfloat16 *Dlo, int32_t *Dfix, double *logtab, int *diag_flag,
                  cudaStream_t s)
{
    const size_t total = (size_t)Np * Np;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    prep_d_kernel<<<blocks, 256, 0, s>>>(C, N, ldc, Np, D32, Dhi, Dlo, Dfix, logtab, diag_flag);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

// ---------------------------------------------------------------------------
// Pair kernel (plain form, row u_i of the upper triangle).
//
// A CTA of 8 warps owns IPC individuals per group and G groups (G > 1 only for
// small N). Rows are cut into 32-row blocks I (NB = Np/32); row block I needs
// the tiles (I, J >= I): NB - I of them. Block I is paired with block NB-1-I so
// that every warp item costs NB + 1 tiles. Lane l of a warp owns row
// i = 32 I + l of all IPC individuals: per column j it loads D_ij once (a
// coalesced 128-byte row of the symmetric D from L2) and compares s_j with s_i
// for the IPC individuals (labels transposed in shared memory, one broadcast
// 16-byte load per 4 individuals). The only per-pair work is compare + add.
// ---------------------------------------------------------------------------
template <typename LabT, int IPC>
__global__ void __launch_bounds__(256, 2)
    pair_plain_kernel(const float *__restrict__ D, int Np, const LabT *lab0, const LabT *lab1,
                      int ldl, int sel_off, int P, int N, float *__restrict__ acc_out,
                      const DevState *__restrict__ st)
{
    const LabT *__restrict__ lab = lab0;
    if (st) {
        if (st->done) return;
        lab = ((st->gen + sel_off) & 1) ? lab1 : lab0;
    }
    extern __shared__ int4 smem_i4[];
    int *lab_s = reinterpret_cast<int *>(smem_i4);
    const int NB = Np >> 5;
    const int npairs = (NB + 1) >> 1;
    const int G = npairs >= 8 ? 1 : (8 / npairs);
    const int p_base = blockIdx.x * G * IPC;

    // labels, transposed: lab_s[(g * Np + j) * IPC + q]
    for (int idx = threadIdx.x; idx < G * IPC * Np; idx += blockDim.x) {
        const int gq = idx / Np, j = idx - gq * Np;
        const int p = p_base + gq;
        int v = 0x7fffffff; // padding genes: D is zero there anyway
        if (p < P && j < N) v = (int)lab[(size_t)p * ldl + j];
        const int g = gq / IPC, q = gq - g * IPC;
        lab_s[(g * Np + j) * IPC + q] = v;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int items = G * npairs;
    for (int it = warp; it < items; it += 8) {
        const int g = it / npairs, t = it - g * npairs;
        const int *ls = lab_s + (size_t)g * Np * IPC;
        const int pg = p_base + g * IPC;
        for (int half = 0; half < 2; ++half) {
            const int I = half ? (NB - 1 - t) : t;
            if (half && I == t) break;
            const int i = (I << 5) + lane;
            int my[IPC];
            float acc[IPC];
#pragma unroll
            for (int q4 = 0; q4 < IPC / 4; ++q4) {
                const int4 v = *reinterpret_cast<const int4 *>(ls + i * IPC + 4 * q4);
                my[4 * q4 + 0] = v.x;
                my[4 * q4 + 1] = v.y;
                my[4 * q4 + 2] = v.z;
                my[4 * q4 + 3] = v.w;
            }
#pragma unroll
            for (int q = 0; q < IPC; ++q) acc[q] = 0.f;

            for (int J = I; J < NB; ++J) {
                float dv[32];
                const float *Dp = D + (size_t)(J << 5) * Np + i;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) dv[jj] = __ldg(Dp + (size_t)jj * Np);
                if (J == I) {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj)
                        if (jj <= lane) dv[jj] = 0.f;
                }
                const int *lj = ls + (J << 5) * IPC;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
#pragma unroll
                    for (int q4 = 0; q4 < IPC / 4; ++q4) {
                        const int4 v = *reinterpret_cast<const int4 *>(lj + jj * IPC + 4 * q4);
                        if (v.x == my[4 * q4 + 0]) acc[4 * q4 + 0] += dv[jj];
                        if (v.y == my[4 * q4 + 1]) acc[4 * q4 + 1] += dv[jj];
                        if (v.z == my[4 * q4 + 2]) acc[4 * q4 + 2] += dv[jj];
                        if (v.w == my[4 * q4 + 3]) acc[4 * q4 + 3] += dv[jj];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < IPC; ++q)
                if (pg + q < P) acc_out[(size_t)(pg + q) * Np + i] = acc[q];
        }
    }
}

template <typename LabT>
int launch_pair_plain(const float *D32, int Np, const LabT *const *lab2, int ldl, int sel_off,
                      int P, int N, float *acc, const DevState *st, cudaStream_t s)
{
    const int NB = Np >> 5;
    const int npairs = (NB + 1) >> 1;
    const int G = npairs >= 8 ? 1 : (8 / npairs);
    if (Np <= 2048) {
        constexpr int IPC = 16;
        const size_t smem = (size_t)G * Np * IPC * sizeof(int);
        const int per_cta = G * IPC;
        const int grid = (P + per_cta - 1) / per_cta;
        pair_plain_kernel<LabT, IPC><<<grid, 256, smem, s>>>(D32, Np, lab2[0], lab2[1], ldl,
                                                             sel_off, P, N, acc, st);
    } else {
        constexpr int IPC = 8;
        const size_t smem = (size_t)G * Np * IPC * sizeof(int);
        const int per_cta = G * IPC;
        const int grid = (P + per_cta - 1) / per_cta;
        pair_plain_kernel<LabT, IPC><<<grid, 256, smem, s>>>(D32, Np, lab2[0], lab2[1], ldl,
                                                             sel_off, P, N, acc, st);
    }
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

// ---------------------------------------------------------------------------
// Assembly (Eq. 5 and Eq. 8): one warp per individual. Row sums are turned into
// fixed point (scale 2^b) and added into per-label bins with integer shared-
// memory atomics, so d_s is independent of the order of the additions (the score
// is deterministic). The non-singleton clusters are compacted and Eq. 8 is
// evaluated from the exact integers dfix = d_s 2^b, cfix = n_s^2 2^b - dfix by
// the one-log product form (LogProd, gpga_internal.cuh).
//   full_rows = 0: row value = 2 u_i + D_ii (upper-triangle sums of the plain form)
//   full_rows = 1: row value = y_i = sum_j D_ij [s_j = s_i] (tensor form)
// ---------------------------------------------------------------------------
template <typename LabT>
__global__ void __launch_bounds__(256)
    assemble_kernel(const LabT *lab0, const LabT *lab1, int ldl, int sel_off,
                    const float *__restrict__ acc, int Np, const float *__restrict__ D32,
                    int full_rows, int P, int N, const double *__restrict__ logtab, int fix_bits,
                    double *__restrict__ L, int *__restrict__ err, const DevState *__restrict__ st,
                    unsigned long long *__restrict__ pairs)
{
    const LabT *__restrict__ lab = lab0;
    int gen = 0;
    if (st) {
        if (st->done) return;
        gen = st->gen + sel_off;
        lab = (gen & 1) ? lab1 : lab0;
    }
    extern __shared__ unsigned long long smem_u64[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    unsigned long long *dfx = smem_u64 + (size_t)warp * Np;
    int *cnt = reinterpret_cast<int *>(smem_u64 + (size_t)nw * Np) + warp * Np;
    const long long *__restrict__ ltab = reinterpret_cast<const long long *>(logtab);
    const long long *__restrict__ ktab = kfix_of(logtab);

    for (int p = blockIdx.x * nw + warp; p < P; p += gridDim.x * nw) {
        for (int s = lane; s < N; s += 32) {
            cnt[s] = 0;
            dfx[s] = 0ull;
        }
        __syncwarp();
        bool bad = false;
        const LabT *lp = lab + (size_t)p * ldl;
        const float *ap = acc + (size_t)p * Np;
        for (int i = lane; i < N; i += 32) {
            const int s = (int)lp[i];
            if (s < 0 || s >= N) {
                bad = true;
                continue;
            }
            const float y = ap[i];
            long long f;
            if (full_rows) {
                f = fix_of(y, fix_bits);
            } else {
                f = fix_of(y, fix_bits + 1) + fix_of(D32[(size_t)i * Np + i], fix_bits);
            }
            atomicAdd(&cnt[s], 1);
            atomicAdd(&dfx[s], (unsigned long long)f);
        }
        bad = __any_sync(0xffffffffu, bad);
        __syncwarp();
        // compact the non-singleton clusters to the front of the bins (in place:
        // every entry moves left, and each chunk is read before it is written) so
        // that the FP64 log terms run on full warps
        int nlist = 0;
        for (int base = 0; base < N; base += 32) {
            const int s = base + lane;
            int n = 0;
            unsigned long long f = 0ull;
            if (s < N) {
                n = cnt[s];
                f = dfx[s];
            }
            const unsigned m = __ballot_sync(0xffffffffu, n >= 2);
            __syncwarp();
            if (n >= 2) {
                const int k = nlist + __popc(m & ((1u << lane) - 1u));
                cnt[k] = n;
                dfx[k] = f;
            }
            nlist += __popc(m);
            __syncwarp();
        }
        LogProd acc_l;
        int npairs = 0;
        for (int k = lane; k < nlist; k += 32) {
            logprod_add(acc_l, cnt[k], (long long)dfx[k], fix_bits, ktab);
            npairs += cnt[k] * (cnt[k] - 1) / 2;
        }
        if (pairs) {
#pragma unroll
            for (int o = 16; o; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
            if (lane == 0) atomicAdd(pairs + gen, (unsigned long long)npairs);
        }
        const double part = logprod_finish(acc_l, ltab, nlist);
        if (lane == 0) {
            L[p] = bad ? __longlong_as_double(0x7ff8000000000000ll) : part;
            if (bad && err) atomicOr(err, 1);
        }
        __syncwarp();
    }
}

template <typename LabT>
int launch_assemble(const LabT *const *lab2, int ldl, int sel_off, const float *acc, int Np,
                    const float *D32, int full_rows, int P, int N, const double *logtab,
                    double *L, int *err, const DevState *st, unsigned long long *pairs,
                    cudaStream_t s)
{
    // 8 warps (one individual each) unless the per-warp bins of a large N need
    // fewer to fit the 227 KB of shared memory
    const size_t per_warp = (size_t)Np * (sizeof(unsigned long long) + sizeof(int));
    int nw = 8;
    while (nw > 1 && nw * per_warp > (size_t)200 * 1024) nw >>= 1;
    const size_t smem = nw * per_warp;
    const int grid = (P + nw - 1) / nw;
    assemble_kernel<LabT><<<grid, 32 * nw, smem, s>>>(lab2[0], lab2[1], ldl, sel_off, acc, Np, D32,
                                                  full_rows, P, N, logtab, fix_bits_for(N), L,
                                                  err, st, pairs);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template int launch_pair_plain<uint16_t>(const float *, int, const uint16_t *const *, int, int,
                                         int, int, float *, const DevState *, cudaStream_t);
template int launch_pair_plain<int32_t>(const float *, int, const int32_t *const *, int, int,
                                        int, int, float *, const DevState *, cudaStream_t);
template int launch_assemble<uint16_t>(const uint16_t *const *, int, int, const float *, int,
                                       const float *, int, int, int, const double *, double *,
                                       int *, const DevState *, unsigned long long *,
                                       cudaStream_t);
template int launch_assemble<int32_t>(const int32_t *const *, int, int, const float *, int,
                                      const float *, int, int, int, const double *, double *,
                                      int *, const DevState *, unsigned long long *,
                                      cudaStream_t);

// ---------------------------------------------------------------------------
// Final re-score of one configuration in FP64 straight from C (Eq. 5, 6, 8),
// plus its canonical relabelling (first occurrence -> 0, 1, 2, ...), on a
// thread-block cluster of RESCORE_CTAS CTAs (one CTA when the cluster cannot
// be placed). Every CTA forms the canonical ids (first gene of each label by
// atomicMin, a block scan) and the member list of every cluster in ascending
// gene order (a counting sort, stable through warp match masks). The rows of
// C are then dealt out over the cluster in chunks of 32 list positions, so a
// warp's lanes take rows of the same cluster: a thread sums C_ij and 1 - C_ij
// over its row's members j in ascending order with Neumaier compensation.
// An FP64 instruction holds the FP64 pipe whatever the number of active lanes,
// so the loops run over members only and keep the lanes busy. After a cluster
// barrier CTA 0 reads the other CTAs' row sums from their shared memory (the
// others wait at a second barrier until it has), sums each cluster's rows in
// ascending order (one thread per cluster), takes the Eq. 8 terms and adds
// them in canonical order as 32 compensated runs combined by a two-sum
// butterfly. Every sum is in the same order as a sequential one over the
// members, within about one ulp of the exact value.
// ---------------------------------------------------------------------------
constexpr int RESCORE_CTAS = 8;

__device__ __forceinline__ void neu_add(double &s, double &c, double x)
{
    const double t = s + x;
    if (fabs(s) >= fabs(x))
        c += (s - t) + x;
    else
        c += (x - t) + s;
    s = t;
}

// s + c += x exactly (Knuth's two-sum): the rounded sum and its error
__device__ __forceinline__ void two_sum_add(double &s, double &c, double x)
{
    const double t = s + x;
    const double bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

// CTA of the cluster that owns list position p: positions go out in chunks
// of 32, chunk q to warp q mod (ncta nw) counted CTA-fastest
__device__ __forceinline__ int rescore_owner(int p, int ncta) { return (p >> 5) % ncta; }

__global__ void __launch_bounds__(1024)
    rescore_kernel(const uint16_t *pop0, const uint16_t *pop1, int ldp,
                   const DevState *__restrict__ st, const double *__restrict__ C, int N,
                   int32_t *__restrict__ canon, double *__restrict__ L_out)
{
    namespace cg = cooperative_groups;
    const cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), ncta = (int)cluster.num_blocks();
    const uint16_t *lab = ((st->gen & 1) ? pop1 : pop0) + (size_t)st->best_idx * ldp;
    extern __shared__ double sm_d[];
    double *rc = sm_d;           // N row sums of C over same-cluster columns (by gene)
    double *rd = sm_d + N;       // N row sums of (1 - C)
    double *term = sm_d + 2 * N; // per canonical cluster: its Eq. 8 term (0 for singletons)
    int *li = reinterpret_cast<int *>(sm_d + 3 * N); // labels, then fill counters
    int *first = li + N;         // label -> first gene carrying it, then cluster sizes
    int *gid = first + N;        // gene -> canonical id (scan of first occurrences)
    int *start = gid + N;        // canonical id -> its first list position
    int *mem = start + N;        // the member list: genes by cluster, ascending in each
    __shared__ int s_part[32];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int i = tid; i < N; i += nt) {
        li[i] = lab[i];
        first[i] = N;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) atomicMin(&first[li[i]], i);
    __syncthreads();
    // canonical ids by first occurrence: exclusive scan of the first-occurrence
    // flags over the genes (chunked: thread t scans genes t*chunk ..)
    const int chunk = (N + nt - 1) / nt;
    const int lo = min(N, tid * chunk), hi = min(N, lo + chunk);
    int cnt = 0;
    for (int i = lo; i < hi; ++i) cnt += first[li[i]] == i;
    int v = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_part[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? s_part[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_part[lane] = w; // inclusive per warp
    }
    __syncthreads();
    int run = v - cnt + (wid ? s_part[wid - 1] : 0);
    for (int i = lo; i < hi; ++i) {
        gid[i] = run; // provisional: valid at first occurrences
        if (first[li[i]] == i) ++run;
    }
    const int K = s_part[nw - 1];
    __syncthreads();
    int g_own[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = tid + u * nt;
        g_own[u] = i < N ? gid[first[li[i]]] : 0;
    }
    __syncthreads();
    // canonical id of every gene; cluster sizes (over first[]), fill counters
    // (over li[])
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = tid + u * nt;
        if (i < N) gid[i] = g_own[u];
    }
    for (int k = tid; k < N; k += nt) {
        first[k] = 0;
        li[k] = 0;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) atomicAdd(&first[gid[i]], 1);
    __syncthreads();
    // list starts: exclusive scan of the sizes over the K clusters
    {
        const int kc = (K + nt - 1) / nt;
        const int k0 = min(K, tid * kc), k1 = min(K, k0 + kc);
        int sz = 0;
        for (int k = k0; k < k1; ++k) sz += first[k];
        int x = sz;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        __syncthreads(); // s_part is reused
        if (lane == 31) s_part[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = lane < nw ? s_part[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            s_part[lane] = w;
        }
        __syncthreads();
        int at = x - sz + (wid ? s_part[wid - 1] : 0);
        for (int k = k0; k < k1; ++k) {
            start[k] = at;
            at += first[k];
        }
    }
    __syncthreads();
    // member lists, ascending gene order inside each cluster: warp 0 walks the
    // genes 32 at a time; lanes with the same id are ordered by lane
    if (wid == 0) {
        const unsigned lt = (1u << lane) - 1u;
        for (int b = 0; b < N; b += 32) {
            const int i = b + lane;
            const int k = i < N ? gid[i] : -1 - lane; // a distinct key per idle lane
            const unsigned same = __match_any_sync(0xffffffffu, k);
            if (i < N) {
                const int r = __popc(same & lt);
                mem[start[k] + li[k] + r] = i;
            }
            __syncwarp();
            if (i < N && (same & lt) == 0) li[k] += __popc(same);
            __syncwarp();
        }
    }
    __syncthreads();
    // row sums of the list positions this CTA owns; singletons need none
    const int lanes_all = ncta * nt;
    for (int p0 = (wid * ncta + rank) * 32; p0 < N; p0 += lanes_all) {
        const int p = p0 + lane;
        if (p >= N) continue;
        const int i = mem[p], k = gid[i], n = first[k];
        if (n < 2) continue;
        const double *row = C + (size_t)i * N;
        const int q0 = start[k];
        double sc = 0.0, cc = 0.0, sd = 0.0, cd = 0.0;
        for (int q = q0; q < q0 + n; ++q) {
            const double x = __ldg(row + mem[q]);
            neu_add(sc, cc, x);
            neu_add(sd, cd, 1.0 - x);
        }
        rc[i] = sc + cc;
        rd[i] = sd + cd;
    }
    cluster.sync(); // every row sum is in its CTA's shared memory
    if (rank == 0 && ncta > 1) {
        for (int p = tid; p < N; p += nt) {
            const int owner = rescore_owner(p, ncta);
            const int i = mem[p];
            if (owner != 0 && first[gid[i]] >= 2) {
                rc[i] = *cluster.map_shared_rank(rc + i, owner);
                rd[i] = *cluster.map_shared_rank(rd + i, owner);
            }
        }
    }
    cluster.sync(); // CTA 0 has read the others' shared memory: they may exit
    if (rank != 0) return;
    // one thread per cluster: its members' row sums in ascending index, then its term
    for (int k = tid; k < K; k += nt) {
        const int n = first[k];
        double t = 0.0;
        if (n >= 2) {
            double c = 0.0, cc = 0.0, d = 0.0, dc = 0.0;
            for (int q = start[k]; q < start[k] + n; ++q) {
                const int j = mem[q];
                neu_add(c, cc, rc[j]);
                neu_add(d, dc, rd[j]);
            }
            const double dn = (double)n;
            double cs = c + cc, ds = d + dc;
            const double eps = 9.094947017729282e-13;
            if (!(cs >= dn * eps)) cs = dn * eps;
            if (!(ds >= dn * (dn - 1.0) * eps)) ds = dn * (dn - 1.0) * eps;
            t = 0.5 * (log(dn / cs) + (dn - 1.0) * log((dn * dn - dn) / ds));
        }
        term[k] = t;
    }
    __syncthreads();
    // terms in canonical order: lane l of warp 0 sums a contiguous run with
    // compensation, then the 32 (sum, error) pairs are combined by a two-sum
    // butterfly
    if (wid == 0) {
        const int per = (K + 31) / 32;
        const int a0 = min(K, lane * per), a1 = min(K, a0 + per);
        double s = 0.0, c = 0.0;
        for (int k = a0; k < a1; ++k) two_sum_add(s, c, term[k]);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
            const double c2 = __shfl_xor_sync(0xffffffffu, c, o);
            // the lower lane of each pair keeps the sum in lane order
            const bool low = (lane & o) == 0;
            double x = low ? s : s2, y = low ? s2 : s;
            double e = low ? c + c2 : c2 + c;
            two_sum_add(x, e, y);
            s = x;
            c = e;
        }
        if (lane == 0) *L_out = s + c;
    }
    for (int i = tid; i < N; i += nt) canon[i] = gid[i];
}

// cluster size the re-score launches with (RESCORE_CTAS, or 1 when a cluster
// of that size with this shared memory cannot be placed); set at preparation
static int g_rescore_ctas = 1;

static size_t rescore_smem(int N)
{
    return (size_t)N * (3 * sizeof(double) + 5 * sizeof(int));
}

int launch_rescore_fp64(const uint16_t *pop0, const uint16_t *pop1, int ldp, const DevState *st,
                        const double *C, int N, int32_t *canon_out, double *L_out, cudaStream_t s)
{
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3(g_rescore_ctas);
    c.blockDim = dim3(1024);
    c.dynamicSmemBytes = rescore_smem(N);
    c.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = g_rescore_ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    c.attrs = at;
    c.numAttrs = 1;
    GPGA_CUDA(cudaLaunchKernelEx(&c, rescore_kernel, pop0, pop1, ldp, st, C, N, canon_out, L_out));
    return GPGA_OK;
}

// diagnostic: log_q62() (with the exponent term) and CUDA's log on the same
// positive normal inputs
__global__ void log_selftest_kernel(const double *__restrict__ x, int n, double *__restrict__ yt,
                                    double *__restrict__ yc)
{
    __shared__ long long tab[2 * LOG_TAB];
    for (int k = threadIdx.x; k < LOG_TAB; k += blockDim.x) log_tab_entry(k, tab + 2 * k);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long b = __double_as_longlong(x[i]);
        const int e = (int)(b >> 52) - 1023;
        const unsigned long long m = (((unsigned long long)b & 0x000fffffffffffffull) |
                                      0x0010000000000000ull) << 10; // Q62
        const long long lq = log_q62(m, tab);
        yt[i] = fma((double)e, 0.6931471805599453, (double)lq * 2.168404344971009e-19);
        yc[i] = log(x[i]);
    }
}

int launch_log_selftest(const double *x, int n, double *yt, double *yc, cudaStream_t s)
{
    log_selftest_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(x, n, yt, yc);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

int prepare_score_kernels(int maxsmem)
{
    if (int rc = raise_smem(pair_plain_kernel<uint16_t, 16>, maxsmem)) return rc;
    if (int rc = raise_smem(pair_plain_kernel<uint16_t, 8>, maxsmem)) return rc;
    if (int rc = raise_smem(pair_plain_kernel<int32_t, 16>, maxsmem)) return rc;
    if (int rc = raise_smem(pair_plain_kernel<int32_t, 8>, maxsmem)) return rc;
    if (int rc = raise_smem(assemble_kernel<uint16_t>, maxsmem)) return rc;
    if (int rc = raise_smem(assemble_kernel<int32_t>, maxsmem)) return rc;
    if (int rc = raise_smem(rescore_kernel, maxsmem)) return rc;
    // the re-score's cluster: RESCORE_CTAS CTAs if that many can be placed with
    // the shared memory of the largest N, else a single CTA does all the rows
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3(RESCORE_CTAS);
    c.blockDim = dim3(1024);
    c.dynamicSmemBytes = rescore_smem(GPGA_MAX_N);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = RESCORE_CTAS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    c.attrs = at;
    c.numAttrs = 1;
    int nclusters = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, rescore_kernel, &c);
    if (e != cudaSuccess) (void)cudaGetLastError(); // not placeable: one CTA
    g_rescore_ctas = (e == cudaSuccess && nclusters >= 1) ? RESCORE_CTAS : 1;
    return GPGA_OK;
}

} // namespace gpga
