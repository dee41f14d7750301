// gpga_internal.cuh -- device helpers and host-side declarations shared by the
// translation units of libgpga.so (sm_103a). Nothing here is part of the ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gpga.h"

namespace gpga {

// ---------------------------------------------------------------------------
// errors (host)
// ---------------------------------------------------------------------------
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what, const char *file, int line);
// empty this thread's error message (every exported call starts with it)
void clear_error();
// cycles a bounded device wait may spend before it gives up (gpga_set_wait_budget)
long long wait_budget();
// the status of a run's device error word: bit 0 (value 1) a label outside
// [0, N), bit 2 (value 4) a bounded wait that gave up
int device_error_status(int err_word, const char *what);

#define GPGA_CUDA(expr)                                                              \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess) return ::gpga::cuda_error(e_, #expr, __FILE__, __LINE__); \
    } while (0)

#define GPGA_LAUNCH_CHECK()                                                          \
    do {                                                                             \
        cudaError_t e_ = cudaGetLastError();                                         \
        if (e_ != cudaSuccess) return ::gpga::cuda_error(e_, "kernel launch", __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------------------------
// Programmatic dependent launch. A kernel launched with pdl = true may be
// scheduled while the previous kernel of the stream is still running; it calls
// griddep_wait() before its first access to anything that kernel writes (the
// wait returns once that grid has completed and its memory is visible; for a
// kernel launched without the attribute it returns at once). griddep_launch()
// lets the next kernel be scheduled once every CTA of this grid has called it
// or exited; it changes nothing about memory visibility.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, bool pdl, Args... args)
{
    cudaLaunchConfig_t c = {};
    c.gridDim = grid;
    c.blockDim = block;
    c.dynamicSmemBytes = smem;
    c.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    c.attrs = at;
    c.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&c, k, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): two 32x32 -> 64-bit
// multiplies per round, ten rounds, key bumped by the Weyl constants.
// Counter layout of the GA: (generation, index, block, stream).
// ---------------------------------------------------------------------------
enum : uint32_t { STREAM_INIT = 0u, STREAM_SUS = 1u, STREAM_XOVER = 2u, STREAM_MUT = 3u };

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// uniform integer in [0, n): high word of u * n
__device__ __forceinline__ int draw_below(uint32_t u, uint32_t n) { return (int)__umulhi(u, n); }

// ---------------------------------------------------------------------------
// run state kept in device memory (read by every kernel of a generation)
// ---------------------------------------------------------------------------
struct DevState {
    int gen;      // generation scored most recently
    int done;     // termination reached
    int best_idx; // fittest individual of generation `gen`
    int err;      // device-side error bits
    double best;  // its L
    double mean;  // population mean L
    uint32_t k0, k1; // Philox key (the run's seed), read by the graphed kernels
    long long lsum;  // fixed-point (2^-30) sum of the generation's fitness, for the mean
    int gnext;       // the generation the next generation kernel starts from, as a hint
                     // it may read before its grid wait (written by the generation
                     // kernel after its wait, and at the start of a run)
    int pad_;
};

// label storage traits: the handle stores labels as uint16 (N <= 65535), the
// stateless calls take the caller's int32
template <typename T> struct LabPair;
template <> struct LabPair<uint16_t> {
    using type = ushort2;
};
template <> struct LabPair<int32_t> {
    using type = int2;
};

// padded gene count: multiple of 64 (tensor-form K tiles, 32-row pair tiles)
inline int pad_n(int N) { return (N + 63) & ~63; }

// The gather form scores configurations of N >= DELTA_MIN_N genes as a sum of
// per-cluster fixed-point terms (single runs, stateless scoring), which lets a
// single GA run keep per-individual score tables and score most children by
// delta from a parent; smaller N, and every fleet run, use the one-log
// product form without tables (a full scoring in the product form is cheaper
// than in the per-cluster form, which needs two logs per cluster). Both forms
// are exact fixed-point evaluations of Eq. 8 that agree to ~1e-12.
constexpr int DELTA_MIN_N = 448;
__host__ __device__ inline bool uses_delta(int N) { return N >= DELTA_MIN_N; }

// fixed-point scale (bits) for the order-independent per-cluster sums of
// FP32 row sums: |row sum| <= 2 N, n_s <= N, so 2 N^2 2^bits < 2^62
int fix_bits_for(int N);

constexpr int LOG_TAB = 256; // cells of the table-driven logarithm (log_q62)

// layout of the per-run log table (8-byte slots): LOG_TAB pairs (inv_k, t_k)
// of log_q62() as int64, then K[n] = 1/2 (log n + (n - 1) log(n (n - 1))) for
// n = 0..N as int64 fixed point 2^-44 (kfix_of)
inline size_t logtab_len(int N) { return 2 * LOG_TAB + (size_t)N + 1; }
__host__ __device__ inline const long long *kfix_of(const double *logtab)
{
    return reinterpret_cast<const long long *>(logtab + 2 * LOG_TAB);
}

// ---------------------------------------------------------------------------
// Eq. 8 of one configuration from its non-singleton clusters, with one log:
//   L = sum_s K[n_s] - 1/2 log prod_s c_s d_s^(n_s - 1)
// (the bracket of Eq. 8 is log(n/c) + (n-1) log(n(n-1)/d)). c_s, d_s arrive as
// exact fixed-point integers cf = c_s 2^b, df = d_s 2^b; the product is kept as
// a mantissa in [1, 2) and an integer exponent, renormalised after every
// multiply from the bit pattern (no overflow, no FP64 log per cluster), and
// the 2^(b n_s) of each cluster's factor is removed from the exponent exactly.
// Domain floor of Eq. 8 (degenerate data only): c_s >= n_s 2^-40,
// d_s >= n_s (n_s - 1) 2^-40, applied in fixed point (at least 1 unit).
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Exact conversions on the integer pipe (the FP64 pipe, which the hardware's
// float <-> int64 conversions use, is ~1/64 of the FP32 rate here).
//   fix_of(y, b) = trunc(y 2^b) for float y with |y| 2^b < 2^62
//   dbl_of(v)    = v as double, rounded toward zero (v > 0, relative error
//                  below 2^-52)
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long fix_of(float y, int bits)
{
    const unsigned u = __float_as_uint(y);
    const int e = (int)((u >> 23) & 0xff);
    if (e == 0) return 0; // zero (no subnormals in these sums)
    const long long m = (long long)((u & 0x7fffffu) | 0x800000u);
    const int sh = e - 150 + bits; // y 2^b = m 2^(e - 150 + b)
    long long v = sh >= 0 ? (m << sh) : (sh > -24 ? (m >> -sh) : 0ll);
    return (u >> 31) ? -v : v;
}

__device__ __forceinline__ double dbl_of(long long v)
{
    const int lz = __clzll(v);
    const int e = 63 - lz;                                         // leading bit
    const unsigned long long mant = ((unsigned long long)v << lz) >> 11; // 53 bits, top set
    return __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) |
                                            (mant & 0x000fffffffffffffull)));
}

// Running product as an integer mantissa m in [2^62, 2^63) (value m 2^-62,
// in [1, 2)) with a binary exponent e; products are 64 x 64 -> 128-bit integer
// multiplies truncated back to 63 bits (relative error < 2^-62 each), so the
// FP64 pipe is not used per cluster. k: sum of K[n_s] in fixed point 2^-44
// (exact integer adds).
constexpr int KFIX_BITS = 44;
// fixed-point D of the gather form: int32 D 2^30 (D = 1 - C in [-2, 2))
constexpr int DFIX_BITS = 30;

struct LogProd {
    unsigned long long m = 1ull << 62;
    long long e = 0;
    long long k = 0;
};

// (mantissa, exponent) of an integer v > 0
__device__ __forceinline__ void mant_of(long long v, unsigned long long &m, long long &e)
{
    const int lz = __clzll(v); // >= 1
    m = (unsigned long long)v << (lz - 1);
    e = 63 - lz;
}

// m 2^-62 <- (m 2^-62)(x 2^-62), exponent carried in e
__device__ __forceinline__ void mant_mul(unsigned long long &m, long long &e, unsigned long long x,
                                         long long ex)
{
    const unsigned long long lo = m * x, hi = __umul64hi(m, x); // m x in [2^124, 2^126)
    if (hi >> 61) {
        m = (hi << 1) | (lo >> 63);
        e += ex + 1;
    } else {
        m = (hi << 2) | (lo >> 62);
        e += ex;
    }
}

// the product part of logprod_add: c d^(n-1) into the running mantissa
// product (the caller sums K(n) itself)
__device__ __forceinline__ void logprod_mul(LogProd &a, int n, long long df, int fix_bits)
{
    long long cf = (((long long)n * n) << fix_bits) - df;
    const int sh = 40 - fix_bits; // fix_bits <= 40
    long long cmin = (long long)n >> sh, dmin = ((long long)n * (n - 1)) >> sh;
    if (cmin < 1) cmin = 1;
    if (dmin < 1) dmin = 1;
    if (cf < cmin) cf = cmin;
    if (df < dmin) df = dmin;
    unsigned long long x;
    long long ex;
    mant_of(cf, x, ex);
    mant_mul(a.m, a.e, x, ex);
    unsigned long long md;
    long long ed;
    mant_of(df, md, ed);
    for (int q = n - 1;;) { // d^(n-1) by binary exponentiation
        if (q & 1) mant_mul(a.m, a.e, md, ed);
        q >>= 1;
        if (!q) break;
        mant_mul(md, ed, md, ed);
    }
    a.e -= (long long)fix_bits * n; // c and the n - 1 factors d each carried 2^b
}

__device__ __forceinline__ void logprod_add(LogProd &a, int n, long long df, int fix_bits,
                                            const long long *__restrict__ kfix)
{
    logprod_mul(a, n, df, fix_bits);
    a.k += kfix[n];
}

// signed Q62 product (a b) >> 62
__device__ __forceinline__ long long mulq62(long long a, long long b)
{
    const long long hi = __mul64hi(a, b);
    const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
    return (long long)(((unsigned long long)hi << 2) | (lo >> 62));
}

// log(m 2^-62) in Q62 for m in [2^62, 2^63), table-driven (Tang's method in
// fixed point): the top 8 fraction bits pick inv_k ~ 2^62 / c_k with
// c_k = 1 + (k + 1/2)/256 and t_k = -log(inv_k 2^-62) (tab[2k], tab[2k+1]);
// r = m inv_k 2^-124 - 1 (|r| <= 2^-9), log = t_k + log1p(r), log1p by its
// series to r^6 (truncation < 2^-65). Integer pipe only.
__device__ __forceinline__ long long log_q62(unsigned long long m,
                                             const long long *__restrict__ tab)
{
    const int k = (int)((m >> 54) & 0xff);
    const unsigned long long inv = (unsigned long long)tab[2 * k];
    const unsigned long long lo = m * inv, hi = __umul64hi(m, inv);
    const long long r = (long long)(((hi << 2) | (lo >> 62)) - (1ull << 62));
    long long q = 922337203685477581ll - mulq62(r, 768614336404564651ll); // 1/5 - r/6
    q = -1152921504606846976ll + mulq62(r, q);                             // -1/4 + r q
    q = 1537228672809129301ll + mulq62(r, q);                              // 1/3 + r q
    q = -2305843009213693952ll + mulq62(r, q);                             // -1/2 + r q
    q = 4611686018427387904ll + mulq62(r, q);                              // 1 + r q
    return tab[2 * k + 1] + mulq62(r, q);
}

// x 2^-s as a double for a signed integer x (integer pipe; rounding toward zero)
__device__ __forceinline__ double dbl_scaled(long long x, int s)
{
    if (x == 0) return 0.0;
    const unsigned long long sign = x < 0 ? 0x8000000000000000ull : 0ull;
    const long long b = __double_as_longlong(dbl_of(x < 0 ? -x : x)) - ((long long)s << 52);
    return __longlong_as_double((long long)((unsigned long long)b | sign));
}

constexpr long long LN2_Q62 = 3196577161300663915ll; // round(ln 2 2^62)

// combine the lanes' partial products (fixed xor butterfly: every lane ends
// with the same value) and return L = k 2^-44 - 1/2 (e ln 2 + log(m 2^-62)),
// evaluated in fixed point Q40 (absolute error ~1e-12), as that integer
__device__ __forceinline__ long long logprod_finish_q40(LogProd a,
                                                        const long long *__restrict__ ltab,
                                                        int nclusters)
{
    if (nclusters == 0) return 0; // all singletons: Eq. 8 is an empty sum
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, a.m, o);
        const long long e2 = __shfl_xor_sync(0xffffffffu, a.e, o);
        const long long k2 = __shfl_xor_sync(0xffffffffu, a.k, o);
        mant_mul(a.m, a.e, m2, e2);
        a.k += k2;
    }
    const long long ph = __mul64hi(a.e, LN2_Q62);
    const unsigned long long pl = (unsigned long long)a.e * (unsigned long long)LN2_Q62;
    const long long elog = (long long)(((unsigned long long)ph << 42) | (pl >> 22));
    const long long tot = elog + (log_q62(a.m, ltab) >> 22);
    return (a.k >> (KFIX_BITS - 40)) - (tot >> 1);
}

__device__ __forceinline__ double logprod_finish(LogProd a, const long long *__restrict__ ltab,
                                                 int nclusters)
{
    if (nclusters == 0) return 0.0; // all singletons: Eq. 8 is an empty sum
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, a.m, o);
        const long long e2 = __shfl_xor_sync(0xffffffffu, a.e, o);
        const long long k2 = __shfl_xor_sync(0xffffffffu, a.k, o);
        mant_mul(a.m, a.e, m2, e2);
        a.k += k2;
    }
    // e ln2 in Q40 from the exact 128-bit product e LN2_Q62, then + log m
    const long long ph = __mul64hi(a.e, LN2_Q62);
    const unsigned long long pl = (unsigned long long)a.e * (unsigned long long)LN2_Q62;
    const long long elog = (long long)(((unsigned long long)ph << 42) | (pl >> 22));
    const long long tot = elog + (log_q62(a.m, ltab) >> 22);
    const long long Lq = (a.k >> (KFIX_BITS - 40)) - (tot >> 1);
    return dbl_scaled(Lq, 40);
}

// ---------------------------------------------------------------------------
// host launchers (score.cu)
// ---------------------------------------------------------------------------
// D forms and log tables; *diag_flag (zeroed by the caller) becomes nonzero if
// some D_ii != 0
int launch_prep_d(const double *C, int N, int ldc, int Np, float *D32, __nv_bfloat16 *Dhi,
                  __nv_bfloat16 *Dlo, int32_t *Dfix, double *logtab, int *diag_flag,
                  cudaStream_t s);

template <typename LabT>
int launch_pair_plain(const float *D32, int Np, const LabT *const *lab2, int ldl, int sel_off,
                      int P, int N, float *acc, const DevState *st, cudaStream_t s);

// pairs (optional, stateful): per-generation sum of n_s (n_s - 1) / 2, indexed
// by the generation being scored
template <typename LabT>
int launch_assemble(const LabT *const *lab2, int ldl, int sel_off, const float *acc, int Np,
                    const float *D32, int full_rows, int P, int N, const double *logtab,
                    double *L, int *err, const DevState *st, unsigned long long *pairs,
                    cudaStream_t s);

// the log tables alone (length logtab_len(N)), as launch_prep_d writes them
int launch_logtab(double *logtab, int N, cudaStream_t s);
// one fleet run: C (ld ldc, optional column subset cols[0..N)) -> dense C64
// (N x N) and Dfix (Np x Np) with its diagonal flag (zeroed by the caller)
int launch_fleet_prep(const double *C, int ldc, const int32_t *cols, int N, int Np, double *C64,
                      int32_t *Dfix, int *diag_flag, cudaStream_t s);

int launch_log_selftest(const double *x, int n, double *yt, double *yc, cudaStream_t s);

int launch_rescore_fp64(const uint16_t *pop0, const uint16_t *pop1, int ldp, const DevState *st,
                        const double *C, int N, int32_t *canon_out, double *L_out, cudaStream_t s);

// raise a kernel's dynamic shared-memory limit to what the device allows beside
// the kernel's static shared memory
template <typename F> inline int raise_smem(F *f, int maxsmem)
{
    cudaFuncAttributes a;
    GPGA_CUDA(cudaFuncGetAttributes(&a, (const void *)f));
    GPGA_CUDA(cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   maxsmem - (int)a.sharedSizeBytes));
    return GPGA_OK;
}

// one-time per-device raise of the dynamic shared-memory limit of the kernels
// that need more than 48 KB (outside any stream capture)
int prepare_device();
bool is_device_ptr(const void *p);
int check_params(const gpga_params *p, int N);
int prepare_score_kernels(int maxsmem);
int prepare_ga_kernels(int maxsmem);
int prepare_init_kernels(int maxsmem);
int prepare_tc_kernels(int maxsmem);
int prepare_gather_kernels(int maxsmem);
int prepare_corr_kernels(int maxsmem);
// market-mode removal in place (corr.cu): lambda1 / iters optional (host)
int market_remove(double *C, int N, int max_iters, double *lambda1, int *iters, cudaStream_t s);
// random-matrix cleaning of B matrices N x N in place (rmt.cu): eig_sorted
// (device, B x N, optional) the input's eigenvalues ascending; n_noise (host,
// B, optional) the noise-set sizes; sweeps (host, optional) Jacobi sweeps run
int rmt_clean(double *C, int B, int N, double T, double *eig_sorted, int *n_noise, int *sweeps,
              cudaStream_t s);
// the same through a tridiagonal reduction, one matrix at a time (rmt_tri.cu)
int rmt_clean_tri(double *C, int B, int N, double T, double *eig_sorted, int *n_noise,
                  cudaStream_t s);
int prepare_rmt_tri_kernels(int maxsmem);


// ---------------------------------------------------------------------------
// host launchers (ga_ops.cu)
// ---------------------------------------------------------------------------
struct SelectCfg {
    int P, E, M, N, ldp;
    int scaling;
    int max_gens, stall_gens;
    double tol;
    uint32_t k0, k1;
    int gen_off; // stateful: g = st->gen + gen_off; stateless: g = gen_off
    int record;
};

// the fixed rank-scaling prefix (P entries) and, if sus_tab is given, its SUS
// brackets (M + 1 entries, see sus_parent_tab)
int rank_prefix_table(uint64_t *prefix, int P, int M, int32_t *sus_tab, cudaStream_t s);

template <typename LabT>
int launch_init_uniform(LabT *pop, int ldp, int P, int N, int K0, uint32_t k0, uint32_t k1,
                        cudaStream_t s);

// ---------------------------------------------------------------------------
// Fleet: many independent GA runs (each its own C, N, population, state and
// Philox key) advanced together, one launch per step for all of them. The
// descriptor table lives in device memory and is read by the graphed kernels,
// so the set of runs can change between graph launches.
// ---------------------------------------------------------------------------
// Per-run score tables of the gather form, two buffers by generation parity
// like the populations. For individual p of buffer b:
//   d[b][p * ldt + s]  d_s = sum_{i,j in s} D_ij in fixed point 2^-30, valid
//                      where n_s >= 2 (other entries unspecified)
//   lf[b][p]           L_c in fixed point 2^-40 (exact sum of per-cluster terms)
//   np[b][p]           sum_s n_s (n_s - 1) / 2
// All pointers null: no tables (stateless scoring).
struct ScoreTab {
    long long *d[2] = {nullptr, nullptr};
    long long *lf[2] = {nullptr, nullptr};
    long long *np[2] = {nullptr, nullptr};
    int ldt = 0;
    // buffer b selected without a run-time array index (which would keep the
    // kernel-parameter copy of this struct in local memory)
    __host__ __device__ __forceinline__ long long *dbuf(int b) const { return b ? d[1] : d[0]; }
    __host__ __device__ __forceinline__ long long *lfbuf(int b) const { return b ? lf[1] : lf[0]; }
    __host__ __device__ __forceinline__ long long *npbuf(int b) const { return b ? np[1] : np[0]; }
};

struct FleetRun {
    int N, Np;               // genes, padded row length of pop and Dfix
    uint16_t *pop0, *pop1;   // P x Np label buffers (ping-pong by generation parity)
    const int32_t *Dfix;     // Np x Np fixed-point D
    const int *diag;         // nonzero if some D_ii != 0
    double *L;               // P fitness values
    int32_t *perm;           // P: index by rank
    int *rank;               // P: zero between launches
    unsigned *ticket;        // TICKETS: zero between launches
    uint64_t *work_prefix;   // P: proportional-scaling prefix
    DevState *st;            // the run's state
    double *hist;            // max_gens + 1 best values
};

struct FleetHdr {
    int nruns;  // active descriptors 0 .. nruns-1
    int nitems; // nruns * P work items of the generation kernel
};

// rank (chunked sort + search, grid) + finalize (perm, stats, termination,
// records, PROP prefix); rank[] and ticket[0 .. 1 + P/256] must be zero on
// entry and are left zero
constexpr int TICKETS = 2 + GPGA_MAX_P / 256;
template <typename LabT>
int launch_select(const double *L, const SelectCfg &cfg, int *rank, int32_t *perm,
                  uint64_t *work_prefix, unsigned *ticket, DevState *st, double *hist,
                  const LabT *const *pop2, LabT *ring, unsigned long long *ts, cudaStream_t s);

// mutation gaps: genes in blocks of MUT_BLOCK; gap[t] = min(floor((1 - P_m)^(t+1)
// 2^32), 2^32 - 1), the probability (times 2^32) that the next t + 1 genes
// keep their labels
constexpr int MUT_BLOCK = 16;

struct EvolveCfg {
    int P, E, M, N, ldp;
    uint64_t m_magic; // exact division by M of values below 2^60 (set_sus_divisor)
    int m_shift;
    uint64_t thr_pc, thr_pkb, thr_pm;
    uint32_t k0, k1;
    int gen; // stateless generation (when st == nullptr)
    uint32_t gap[MUT_BLOCK];
    const int32_t *sus_tab; // SUS brackets of a fixed prefix (rank scaling), or nullptr
};

// fill cfg->thr_pm and cfg->gap for mutation probability pm (host)
void set_mutation(EvolveCfg *cfg, double pm);
// fill cfg->m_magic / m_shift for the M pointers of SUS (host)
void set_sus_divisor(EvolveCfg *cfg, int M);

// prefix: inclusive prefix of the scaled weights by rank (RANK: the fixed
// table; PROP: the work prefix written by finalize); parents_out optional
// ---------------------------------------------------------------------------
// One child of the next population (warp-cooperative; all lanes call).
// "Apply genetic operator: selection" (SUS): the P individuals lie on a line
// in rank order over segments of their scaled weights (prefix[r] inclusive,
// W = prefix[P-1]); pointer x_k = floor((k 2^32 + u) W / (M 2^32)) with
// u = word 0 of Philox(g, 0, 0, SUS) selects rank r with
// prefix[r-1] <= x_k < prefix[r]. Child k pairs a = parent(k) with
// b = parent((k + M/2) mod M).
// Crossover: Philox(g, k, 0, XOVER) = (x, y, z, .): if x < thr(P_c), then the
// knowledge-based merge if y < thr(P_kb) with anchor q = draw(z, N):
// child_j = a_q where b_j = b_q, else a_j; otherwise one-point at
// cut = 1 + draw(z, N - 1): child_j = a_j for j < cut, b_j after.
// Mutation, gene pair (2m, 2m+1): Philox(g, k, m, MUT) = (f0, v0, f1, v1):
// child_j = draw(v, N) if f < thr(P_m).
// Every gene is a function of (a_j, b_j) and warp-uniform values, so lanes
// stream gene pairs. Writes dst (global) and, if given, lab_s (shared).
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// SUS pointer x_k = floor((k 2^32 + u) W / (M 2^32)), exact, on the integer
// pipe: y = (k 2^32 + u) W as a 128-bit product, Y = floor(y / 2^32) (< 2^60
// for k < M <= 2^14 and W <= P 2^32 <= 2^46), x_k = floor(Y / M) by the
// multiply-shift division of set_sus_divisor: magic = ceil(2^(60 + l) / M),
// l = ceil(log2 M), x = (Y magic) >> (60 + l), exact for every Y < 2^60
// because the error term Y (magic M - 2^(60 + l)) / (M 2^(60 + l)) stays below 1/M.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sus_pointer(uint32_t k, uint32_t u, uint64_t W, uint64_t magic,
                                                int shift)
{
    const uint64_t num = ((uint64_t)k << 32) | u;
    const uint64_t ylo = num * W, yhi = __umul64hi(num, W);
    const uint64_t Y = (yhi << 32) | (ylo >> 32);
    const uint64_t plo = Y * magic, phi = __umul64hi(Y, magic);
    return shift >= 64 ? (phi >> (shift - 64)) : ((phi << (64 - shift)) | (plo >> shift));
}

// Parent of SUS pointer k for each half-warp (lanes 0-15 and 16-31 may ask
// for different k): the rank r with prefix[r-1] <= x_k < prefix[r], found by a
// 16-ary search (each round the half-warp loads 16 evenly spaced prefix values
// and counts those <= x_k: three dependent loads for P = 4096 instead of
// twelve), then perm[r]. All lanes of the warp call; returns the half's parent.
__device__ __forceinline__ int sus_parent_half(uint32_t k, uint32_t u, uint64_t W, int M, int P,
                                               uint64_t magic, int shift,
                                               const uint64_t *__restrict__ prefix,
                                               const int32_t *__restrict__ perm, int lane)
{
    const uint64_t x = sus_pointer(k, u, W, magic, shift);
    const int l = lane & 15;
    const unsigned half = lane < 16 ? 0x0000ffffu : 0xffff0000u;
    int top = 1;
    while (top * 16 < P) top *= 16;
    // invariant: the answer lies in [lo, lo + 16 step)
    int lo = 0;
    for (int step = top; step >= 1; step >>= 4) {
        const int idx = lo + l * step;
        const bool le = idx < P && __ldg(prefix + idx) <= x;
        const int c = __popc(__ballot_sync(0xffffffffu, le) & half);
        if (c) lo += (c - 1) * step + 1;
    }
    return perm[lo];
}

// The same parent with the brackets of a prefix that does not change between
// generations (rank scaling): tab[k] = first rank r with prefix[r] > floor(k W / M),
// k = 0..M. Pointer k lies in [floor(k W / M), floor((k + 1) W / M)], so its rank
// is tab[k] + #{r in [tab[k], tab[k+1]) : prefix[r] <= x_k}: the bracket loads
// do not wait for x_k, and one round of at most 16 prefix loads per half-warp
// replaces the 16-ary search. A wider bracket (very few pointers for the
// ranks) takes the general search.
__device__ __forceinline__ int sus_parent_tab(uint32_t k, uint32_t u, uint64_t W, int M, int P,
                                              uint64_t magic, int shift,
                                              const uint64_t *__restrict__ prefix,
                                              const int32_t *__restrict__ tab,
                                              const int32_t *__restrict__ perm, int lane)
{
    const int lo = __ldg(tab + k), hi = __ldg(tab + k + 1);
    if (__all_sync(0xffffffffu, hi - lo <= 16)) {
        const uint64_t x = sus_pointer(k, u, W, magic, shift);
        const int l = lane & 15;
        const unsigned half = lane < 16 ? 0x0000ffffu : 0xffff0000u;
        const bool le = l < hi - lo && __ldg(prefix + lo + l) <= x;
        return perm[lo + __popc(__ballot_sync(0xffffffffu, le) & half)];
    }
    return sus_parent_half(k, u, W, M, P, magic, shift, prefix, perm, lane);
}

// The loads of sus_parent_tab that do not depend on the generation: the bracket
// of the lane's pointer (k for lanes 0-15, (k + M/2) mod M for 16-31), the
// lane's candidate prefix value in it and W. Both tables are fixed for the run,
// so a kernel issues these before it waits for the selection.
struct SusPre {
    int lo, hi;    // bracket [lo, hi) of the lane's pointer
    uint64_t cand; // prefix[lo + (lane & 15)] if that rank is inside the bracket
    uint64_t W;    // prefix[P - 1]
};

__device__ __forceinline__ SusPre sus_prefetch(uint32_t k, int M, int P,
                                               const uint64_t *__restrict__ prefix,
                                               const int32_t *__restrict__ tab, int lane)
{
    SusPre s;
    const uint32_t kp = lane < 16 ? k : (k + (uint32_t)M / 2) % (uint32_t)M;
    s.lo = __ldg(tab + kp);
    s.hi = __ldg(tab + kp + 1);
    s.W = __ldg(prefix + P - 1);
    const int l = lane & 15;
    s.cand = l < s.hi - s.lo ? __ldg(prefix + s.lo + l) : 0ull;
    return s;
}

// number of genes the next mutation skips for word u: #{t : u < gap[t]}
__device__ __forceinline__ int mutation_skip(uint32_t u, const EvolveCfg &cfg)
{
    int s = 0;
#pragma unroll
    for (int t = 0; t < MUT_BLOCK; ++t) s += u < cfg.gap[t] ? 1 : 0;
    return s;
}

// "Apply genetic operator: mutation" (random replacement, each gene with
// probability P_m), drawn as geometric gaps: lane handles the blocks of
// MUT_BLOCK genes b = lane, lane + 32, ...; from position pos the next
// mutated gene is pos + skip(u) and takes label draw(v, N), with (u, v) the
// words (x, y) then (z, w) of Philox(g, k, b + 65536 e, MUT), e = 0, 1, ...
// The crossover result must already be in dst / lab_s (all lanes, synced here).
template <typename LabT>
__device__ __forceinline__ void mutate_child(const EvolveCfg &cfg, int N, int g, int k,
                                             uint32_t k0, uint32_t k1, LabT *dst,
                                             uint16_t *lab_s, int lane)
{
    __syncwarp();
    if (!cfg.thr_pm) return;
    const int nblk = (N + MUT_BLOCK - 1) / MUT_BLOCK;
    for (int blk = lane; blk < nblk; blk += 32) {
        const int base = blk * MUT_BLOCK;
        const int len = min(MUT_BLOCK, N - base);
        int pos = 0;
        for (uint32_t e = 0;; ++e) {
            const U4 w = philox((uint32_t)g, (uint32_t)k, (uint32_t)blk + 65536u * e, STREAM_MUT,
                                k0, k1);
            pos += mutation_skip(w.x, cfg);
            if (pos >= len) break;
            {
                const int v = draw_below(w.y, (uint32_t)N);
                dst[base + pos] = (LabT)v;
                if (lab_s) lab_s[base + pos] = (uint16_t)v;
            }
            if (++pos >= len) break;
            pos += mutation_skip(w.z, cfg);
            if (pos >= len) break;
            {
                const int v = draw_below(w.w, (uint32_t)N);
                dst[base + pos] = (LabT)v;
                if (lab_s) lab_s[base + pos] = (uint16_t)v;
            }
            if (++pos >= len) break;
        }
    }
    __syncwarp();
}

// pre (optional): this child's sus_prefetch, issued earlier by the caller.
// Returns the index of parent a (all lanes).
template <typename LabT>
__device__ __forceinline__ int child_genes(const LabT *cur, int ldp, int N, const EvolveCfg &cfg,
                                            int g, int k, uint32_t k0, uint32_t k1,
                                            const int32_t *__restrict__ perm,
                                            const uint64_t *__restrict__ prefix,
                                            int32_t *__restrict__ parents_out,
                                            LabT *__restrict__ dst, uint16_t *lab_s, int lane,
                                            const SusPre *pre = nullptr)
{
    const int M = cfg.M;
    const uint64_t W = pre ? pre->W : __ldg(prefix + cfg.P - 1);
    const U4 su = philox((uint32_t)g, 0u, 0u, STREAM_SUS, k0, k1);
    const uint32_t kp = lane < 16 ? (uint32_t)k : (uint32_t)((k + M / 2) % M);
    int par;
    if (pre && __all_sync(0xffffffffu, pre->hi - pre->lo <= 16)) {
        // sus_parent_tab with its loads already in registers
        const uint64_t x = sus_pointer(kp, su.x, W, cfg.m_magic, cfg.m_shift);
        const unsigned half = lane < 16 ? 0x0000ffffu : 0xffff0000u;
        const bool le = (lane & 15) < pre->hi - pre->lo && pre->cand <= x;
        par = perm[pre->lo + __popc(__ballot_sync(0xffffffffu, le) & half)];
    } else {
        par = cfg.sus_tab ? sus_parent_tab(kp, su.x, W, M, cfg.P, cfg.m_magic, cfg.m_shift, prefix,
                                           cfg.sus_tab, perm, lane)
                          : sus_parent_half(kp, su.x, W, M, cfg.P, cfg.m_magic, cfg.m_shift, prefix,
                                            perm, lane);
    }
    const int ia = __shfl_sync(0xffffffffu, par, 0);
    const int ib = __shfl_sync(0xffffffffu, par, 16);
    if (parents_out && lane == 0) parents_out[k] = ia;
    const LabT *__restrict__ a = cur + (size_t)ia * ldp;
    const LabT *__restrict__ b = cur + (size_t)ib * ldp;
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
    if constexpr (sizeof(LabT) == 2) {
        // 16-bit labels: one 32-bit load per parent and gene pair (rows are
        // 128-byte aligned); a padding gene (j = N for odd N) is written as 0
        const uint32_t *__restrict__ a2 = reinterpret_cast<const uint32_t *>(a);
        const uint32_t *__restrict__ b2 = reinterpret_cast<const uint32_t *>(b);
        uint32_t *__restrict__ d2 = reinterpret_cast<uint32_t *>(dst);
        uint32_t *s2 = reinterpret_cast<uint32_t *>(lab_s);
#pragma unroll 8
        for (int m = lane; m < npair; m += 32) {
            const int j0 = 2 * m, j1 = 2 * m + 1;
            const uint32_t av = __ldg(a2 + m), bv = __ldg(b2 + m);
            const int a0 = (int)(av & 0xffffu), a1 = (int)(av >> 16);
            const int b0 = (int)(bv & 0xffffu), b1 = (int)(bv >> 16);
            int c0 = a0, c1 = a1;
            if (mode == 1) {
                if (j0 >= cut) c0 = b0;
                if (j1 >= cut) c1 = b1;
            } else if (mode == 2) {
                if (b0 == bq) c0 = aq;
                if (b1 == bq) c1 = aq;
            }
            if (j1 >= N) c1 = 0;
            const uint32_t cv = (uint32_t)c0 | ((uint32_t)c1 << 16);
            d2[m] = cv;
            if (s2) s2[m] = cv;
        }
        mutate_child<LabT>(cfg, N, g, k, k0, k1, dst, lab_s, lane);
        return ia;
    }
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
        dst[j0] = (LabT)c0;
        if (lab_s) lab_s[j0] = (uint16_t)c0;
        if (j1 < N) {
            dst[j1] = (LabT)c1;
            if (lab_s) lab_s[j1] = (uint16_t)c1;
        }
    }
    mutate_child<LabT>(cfg, N, g, k, k0, k1, dst, lab_s, lane);
    return ia;
}

template <typename LabT>
int launch_evolve(const LabT *const *pop2, LabT *const *next2, const EvolveCfg &cfg,
                  const int32_t *perm, const uint64_t *prefix, int32_t *parents_out,
                  const DevState *st, cudaStream_t s);

// gather form (gather.cu). tab: the score tables written for the scored
// buffer (stateful runs), or empty.
template <typename LabT>
int launch_gather_score(const LabT *const *lab2, int ldl, int sel_off, int P, int N, int Np,
                        const int32_t *Dfix, const int *diag_flag, const double *logtab,
                        double *L, int *err, const DevState *st, unsigned long long *pairs,
                        const ScoreTab &tab, cudaStream_t s);
int launch_gather_generation(const uint16_t *const *pop2, uint16_t *const *next2,
                             const EvolveCfg &cfg, const int32_t *perm, const uint64_t *prefix,
                             int Np, const int32_t *Dfix, const int *diag_flag,
                             const double *logtab, double *L, DevState *st,
                             unsigned long long *pairs, const ScoreTab &tab, bool pdl,
                             cudaStream_t s);
// bytes of one row of the d table for padded gene count Np
size_t score_tab_row_bytes(int Np);

int launch_state_init(DevState *st, unsigned long long *ts0, uint32_t k0, uint32_t k1,
                      cudaStream_t s);

// fleet launches: selection of every active run (grid nc x nc x cap), and the
// fused generation over all (run, slot) items, `warps` warps per CTA, `ctas`
// CTAs striding over the items; smem slices sized for Np_max; prop: the runs
// use proportional scaling (their own work prefix), else the shared rank table
int launch_fleet_select(const FleetRun *runs, const FleetHdr *hdr, const SelectCfg &cfg,
                        int cap, cudaStream_t s);
int launch_fleet_generation(const FleetRun *runs, const FleetHdr *hdr, const EvolveCfg &cfg,
                            const uint64_t *rank_prefix, const double *logtab, int Np_max,
                            int warps, int ctas, int prop, cudaStream_t s, bool pdl = false);

// island migration over the fleet's runs (ring by table position): every
// `every` generations, the m elites of each run replace the last m children
// of the next run
int launch_fleet_migrate(const FleetRun *runs, const FleetHdr *hdr, int P, int every, int m,
                         int cap, cudaStream_t s);
// largest warps per CTA whose shared-memory slices fit, and the resident CTAs
// per SM of the fleet generation kernel at that shape
int fleet_max_warps(int Np_max);
int fleet_ctas_per_sm(int Np_max, int warps, int *out);

// threshold initialisation (init.cu)
// per-cluster minimum spanning trees of one configuration (labels device,
// int32 N); grp: device scratch of cluster_mst_scratch_ints(N) ints, of
// which grp[0] = 1 on a label outside [0, N) and grp[1] = the cluster count
size_t cluster_mst_scratch_ints(int N);
int launch_cluster_mst(const double *C, int N, const int32_t *labels, int32_t *eu, int32_t *ev,
                       double *ew, int *grp, cudaStream_t s);
int launch_mst(const double *C, int N, int32_t *edge_u, int32_t *edge_v, double *edge_w,
               cudaStream_t s);
template <typename LabT>
int launch_init_threshold(LabT *pop, int ldp, int P, int N, const int32_t *edge_u,
                          const int32_t *edge_v, const double *edge_w, double tau_lo,
                          double tau_hi, uint32_t k0, uint32_t k1, cudaStream_t s);

// ---------------------------------------------------------------------------
// host launchers (corr.cu)
// ---------------------------------------------------------------------------
int corr_run(const double *R, int T, int N, int ld, double *C, cudaStream_t s);
// unit weights on the tensor cores (corr_tc.cu)
int corr_run_tc(const double *R, int T, int N, int ld, double *C, cudaStream_t s);
int prepare_corr_tc_kernels(int maxsmem);
// EWMA-weighted Pearson: rows weighted lambda^(T-1-t) in the means, the
// variances and the cross products (lambda = 1: plain Pearson)
int corr_run_weighted(const double *R, int T, int N, int ld, double lambda, double *C,
                      cudaStream_t s);

// uint64 threshold of a probability: floor(p 2^32), 2^32 for p >= 1
uint64_t prob_threshold(double p);

} // namespace gpga
