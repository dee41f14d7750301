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

// fixed-point scale (bits) for the order-independent per-cluster sums of
// FP32 row sums: |row sum| <= 2 N, n_s <= N, so 2 N^2 2^bits < 2^62
int fix_bits_for(int N);

// ---------------------------------------------------------------------------
// Natural log in FP64 for x > 0 normal, table-driven (P. T. P. Tang, "Table-
// driven implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16(4), 1990): x = 2^e m, m in [1, 2); the top 8
// mantissa bits pick c_k = 1 + (k + 1/2)/256, with tab[k] = (inv_k, -log inv_k)
// and inv_k = fl(1/c_k); r = m inv_k - 1 (one FMA, |r| <= 2^-9 + ulp) and
// log x = e ln2 - log inv_k + log1p(r), log1p by its Taylor series to r^6
// (truncation < |r|^7/7 < 2e-20). About 9 FP64 operations.
// ---------------------------------------------------------------------------
constexpr int LOG_TAB = 256;

__device__ __forceinline__ double table_log(double x, const double2 *__restrict__ tab)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)(b >> 52) - 1023;
    const int k = (int)((b >> 44) & 0xff);
    const double m = __longlong_as_double((b & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
    const double2 t = tab[k];
    const double r = fma(m, t.x, -1.0);
    double q = fma(r, -1.0 / 6.0, 0.2);
    q = fma(r, q, -0.25);
    q = fma(r, q, 1.0 / 3.0);
    q = fma(r, q, -0.5);
    q = fma(r, q, 1.0);
    return fma((double)e, 0.6931471805599453, fma(r, q, t.y));
}

// layout of the per-run log table (doubles): LOG_TAB pairs (inv_k, -log inv_k),
// then K1[n], n = 0..N (see score.cu)
inline size_t logtab_len(int N) { return 2 * LOG_TAB + (size_t)N + 1; }

// ---------------------------------------------------------------------------
// host launchers (score.cu)
// ---------------------------------------------------------------------------
int launch_prep_d(const double *C, int N, int ldc, int Np, float *D32, __nv_bfloat16 *Dhi,
                  __nv_bfloat16 *Dlo, double *logtab, cudaStream_t s);

template <typename LabT>
int launch_pair_plain(const float *D32, int Np, const LabT *const *lab2, int ldl, int sel_off,
                      int P, int N, float *acc, const DevState *st, cudaStream_t s);

template <typename LabT>
int launch_assemble(const LabT *const *lab2, int ldl, int sel_off, const float *acc, int Np,
                    const float *D32, int full_rows, int P, int N, const double *logtab,
                    double *L, int *err, const DevState *st, cudaStream_t s);

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
int prepare_score_kernels(int maxsmem);
int prepare_ga_kernels(int maxsmem);
int prepare_init_kernels(int maxsmem);
int prepare_tc_kernels(int maxsmem);

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

int rank_prefix_table(uint64_t *prefix, int P, cudaStream_t s);

template <typename LabT>
int launch_init_uniform(LabT *pop, int ldp, int P, int N, int K0, uint32_t k0, uint32_t k1,
                        cudaStream_t s);

// rank (counting, grid) + finalize (perm, stats, termination, records, PROP
// prefix); rank[] and *ticket must be zero on entry and are left zero
template <typename LabT>
int launch_select(const double *L, const SelectCfg &cfg, int *rank, int32_t *perm,
                  uint64_t *work_prefix, unsigned *ticket, DevState *st, double *hist,
                  const LabT *const *pop2, LabT *ring, unsigned long long *ts, cudaStream_t s);

struct EvolveCfg {
    int P, E, M, N, ldp;
    uint64_t thr_pc, thr_pkb, thr_pm;
    uint32_t k0, k1;
    int gen; // stateless generation (when st == nullptr)
};

// prefix: inclusive prefix of the scaled weights by rank (RANK: the fixed
// table; PROP: the work prefix written by finalize); parents_out optional
template <typename LabT>
int launch_evolve(const LabT *const *pop2, LabT *const *next2, const EvolveCfg &cfg,
                  const int32_t *perm, const uint64_t *prefix, int32_t *parents_out,
                  const DevState *st, cudaStream_t s);

int launch_state_init(DevState *st, unsigned long long *ts0, uint32_t k0, uint32_t k1,
                      cudaStream_t s);

// threshold initialisation (init.cu)
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

// uint64 threshold of a probability: floor(p 2^32), 2^32 for p >= 1
uint64_t prob_threshold(double p);

} // namespace gpga
