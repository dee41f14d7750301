// corr_tc.cu -- the Pearson prelude, Eq. 7 (Sec. 2.1; the standardisation
// below Eq. 2), with the T-contraction on the tensor cores (sm_103a tcgen05):
//   C_ij = <z_i, z_j> / sqrt(<z_i, z_i> <z_j, z_j>),  z = R - column mean.
//
// The column statistics stay off the FP64 pipe (a small fraction of the
// integer rate on this part):
//   1. colscan:  the largest binary exponent of each column (integer field)
//                and a finiteness check;
//   2. colfix:   X_tj = trunc(R_tj 2^s_j), s_j from that exponent so that
//                |X| < 2^(60 - B) (T < 2^B), and S1_j = sum_t X_tj, exact in int64;
//   3. zsplit:   Z_tj = T X_tj - S1_j = T (X_tj - mean_j), an exact integer
//                (|Z| < 2^61), scaled by 2^-61 and split into three BF16
//                parts hi + mid + lo (24 significant bits), written
//                transposed (column j's values contiguous in t);
//   4. gram_tc:  S = Z^T Z on 128 x 128 upper-triangle tiles, the T range
//                split over CTAs: six BF16 products (hi hi, hi mid, mid hi,
//                hi lo, lo hi, mid mid; the dropped ones are below 2^-24 of
//                each product) accumulated in FP32 in tensor memory, the
//                K-blocks of a CTA taken in turn by four accumulators (the
//                accumulation error grows with an accumulator's magnitude and
//                step count), per-split partial tiles in FP32;
//   5. gram_diag / gram_out: the partials added as exact fixed-point
//                integers in a fixed order, C_ij = S_ij / sqrt(S_ii S_jj)
//                (FP64), diagonal 1, clamped to [-1, 1], both triangles.
// A column whose values are all equal gives Z = 0 exactly: zero variance.
// Resolution of the centring: 2^-(60 - B) of the column's largest magnitude.
#include <math.h>

#include "gpga_internal.cuh"
#include "tc_ptx.cuh"

namespace gpga {

constexpr int G_TILE = 128;                   // rows of a Gram tile (MMA M and N)
constexpr int G_KB = 64;                      // rows of T per K-block (128 bytes of BF16)
constexpr int G_OP_BYTES = G_TILE * G_KB * 2; // one operand plane of a K-block: 16 KB
constexpr int G_STAGE = 6 * G_OP_BYTES;       // A hi/mid/lo + B hi/mid/lo: 96 KB
constexpr int G_SMEM = 2 * G_STAGE + 1024;
constexpr int G_THREADS = 128;
constexpr int G_NACC = 4;                      // accumulators, K-blocks taken in turn
constexpr int G_TMEM_COLS = G_NACC * G_TILE;   // 512 columns
constexpr int CT_ROWS = 256; // rows of R per column-statistics CTA

// bits needed for T (T < 2^B)
static int bitlen(int T)
{
    int b = 0;
    while ((1ll << b) <= (long long)T) ++b;
    return b;
}

__global__ void __launch_bounds__(256)
    colscan_kernel(const double *__restrict__ R, int T, int N, int ld, int *__restrict__ emax,
                   int *__restrict__ err)
{
    __shared__ int red[8][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = blockIdx.x * 32 + tx;
    const int t0 = blockIdx.y * CT_ROWS, t1 = min(T, t0 + CT_ROWS);
    int e = 0, bad = 0;
    if (j < N) {
        for (int t = t0 + ty; t < t1; t += 8) {
            const unsigned long long b =
                (unsigned long long)__double_as_longlong(R[(size_t)t * ld + j]);
            const int x = (int)((b >> 52) & 0x7ff);
            bad |= x == 0x7ff;
            e = max(e, x);
        }
    }
    red[ty][tx] = e;
    if (bad) atomicOr(err, 2);
    __syncthreads();
    if (ty == 0 && j < N) {
        for (int r = 1; r < 8; ++r) e = max(e, red[r][tx]);
        atomicMax(emax + j, e);
    }
}

// X = trunc(x 2^s) of an FP64 bit pattern, with the column's shift folded in
// sh0 = s - 1075 (x = M 2^(e - 1075), M the 53-bit significand); zero and
// subnormals give 0
__device__ __forceinline__ long long fix_col(unsigned long long b, int sh0)
{
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;
    const long long M = (long long)((b & 0x000fffffffffffffull) | 0x0010000000000000ull);
    const int sh = e + sh0;
    const long long v = sh >= 0 ? (M << sh) : (sh > -63 ? (M >> -sh) : 0ll);
    return (b >> 63) ? -v : v;
}

// the column's shift: s_j = (60 - B) - (emax_j - 1022), folded with -1075
__device__ __forceinline__ int col_sh0(int emax, int B) { return (60 - B) - (emax - 1022) - 1075; }

__global__ void __launch_bounds__(256)
    colfix_kernel(const double *__restrict__ R, int T, int N, int ld, const int *__restrict__ emax,
                  int B, unsigned long long *__restrict__ S1)
{
    __shared__ long long red[8][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = blockIdx.x * 32 + tx;
    const int t0 = blockIdx.y * CT_ROWS, t1 = min(T, t0 + CT_ROWS);
    long long s = 0;
    if (j < N) {
        const int sh0 = col_sh0(emax[j], B);
        for (int t = t0 + ty; t < t1; t += 8)
            s += fix_col((unsigned long long)__double_as_longlong(R[(size_t)t * ld + j]), sh0);
    }
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && j < N) {
        for (int r = 1; r < 8; ++r) s += red[r][tx];
        atomicAdd(S1 + j, (unsigned long long)s);
    }
}

// BF16 of v 2^-61 for an integer |v| < 2^62, rounded to nearest (ties away
// from zero), and the integer it stands for (so that v - *used is exact)
__device__ __forceinline__ uint16_t bf16_of_int(long long v, long long *used)
{
    if (v == 0) {
        *used = 0;
        return 0;
    }
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int L = 63 - __clzll((long long)a);
    int sh = L - 7;
    unsigned long long r;
    if (sh > 0) {
        r = (a + (1ull << (sh - 1))) >> sh;
        if (r >> 8) {
            r >>= 1;
            ++sh;
        }
        const long long u = (long long)(r << sh);
        *used = v < 0 ? -u : u;
    } else {
        r = a << (-sh);
        *used = v;
    }
    const int E = sh + 7 - 61; // value = (r / 128) 2^E, r in [128, 255]
    return (uint16_t)((v < 0 ? 0x8000u : 0u) | ((unsigned)(E + 127) << 7) | (unsigned)(r & 0x7f));
}

// Z planes (Nq x Tp BF16 each), 32 x 32 tiles through shared memory:
// block (32, 8), tile (t0 = 32 bx, j0 = 32 by)
__global__ void __launch_bounds__(256)
    zsplit_kernel(const double *__restrict__ R, int T, int N, int ld, const int *__restrict__ emax,
                  int B, const unsigned long long *__restrict__ S1, int Tp,
                  uint16_t *__restrict__ Zh, uint16_t *__restrict__ Zm, uint16_t *__restrict__ Zl)
{
    __shared__ uint16_t tile[3][32][34];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int t0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int j = j0 + tx;
    int sh0 = 0;
    long long s1 = 0;
    if (j < N) {
        sh0 = col_sh0(emax[j], B);
        s1 = (long long)S1[j];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int tt = ty + 8 * q, t = t0 + tt;
        long long z = 0;
        if (j < N && t < T)
            z = (long long)T * fix_col((unsigned long long)__double_as_longlong(R[(size_t)t * ld + j]),
                                       sh0) -
                s1;
        long long u;
        const uint16_t h = bf16_of_int(z, &u);
        z -= u;
        const uint16_t m = bf16_of_int(z, &u);
        z -= u;
        const uint16_t l = bf16_of_int(z, &u);
        tile[0][tx][tt] = h;
        tile[1][tx][tt] = m;
        tile[2][tx][tt] = l;
    }
    __syncthreads();
    // transposed: row j0 + jj, columns t0 .. t0 + 31 (coalesced over t)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int jj = ty + 8 * q;
        const size_t off = (size_t)(j0 + jj) * Tp + t0 + tx;
        Zh[off] = tile[0][jj][tx];
        Zm[off] = tile[1][jj][tx];
        Zl[off] = tile[2][jj][tx];
    }
}

// upper-triangle tile index -> (bi, bj), bi <= bj
__device__ __forceinline__ void tile_pair(int tile, int nb, int *bi, int *bj)
{
    int b = 0;
    while (tile >= nb - b) {
        tile -= nb - b;
        ++b;
    }
    *bi = b;
    *bj = b + tile;
}

// ---------------------------------------------------------------------------
// The contraction: CTA (tile, split) accumulates S over its K-blocks
// [kb0, kb1) of T in one 128 x 128 FP32 accumulator in tensor memory. Per
// K-block all 128 threads cp.async the six operand planes (hi, mid, lo of
// the A rows bi and the B rows bj) into 128-byte-swizzled K-major tiles (two
// stages); thread 0 issues 4 x 6 tcgen05.mma (M128 N128 K16, BF16 in, FP32
// accumulate) and commits to the stage's mbarrier. Every pipeline wait is
// bounded by `budget` cycles; a timeout sets bit 4 of err, stops issuing,
// waits (full bound) for the committed MMAs and frees the tensor memory.
// Epilogue: thread r reads row r of the accumulator (tcgen05.ld) and writes
// it to the split's FP32 partial tile.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(G_THREADS, 1)
    gram_tc_kernel(const uint16_t *__restrict__ Zh, const uint16_t *__restrict__ Zm,
                   const uint16_t *__restrict__ Zl, int Tp, int nb, int kb_per, int nkb,
                   float *__restrict__ part, long long budget, int *__restrict__ err)
{
    extern __shared__ unsigned char g_raw[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int ntiles = gridDim.x;
    int bi, bj;
    tile_pair(blockIdx.x, nb, &bi, &bj);
    const int kb0 = blockIdx.y * kb_per, kb1 = min(nkb, kb0 + kb_per);
    float *dst = part + ((size_t)blockIdx.y * ntiles + blockIdx.x) * (G_TILE * G_TILE);
    if (kb0 >= kb1) { // an empty split contributes zeros
        for (int e = tid; e < G_TILE * G_TILE; e += G_THREADS) dst[e] = 0.f;
        return;
    }
    const uint32_t raw = smem_u32(g_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    const uint32_t stage0 = raw + pad;
    // instruction descriptor: D F32, A BF16, B BF16, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(G_TILE >> 3) << 17) |
                           ((uint32_t)(G_TILE >> 4) << 24);
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(G_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    // the six planes of K-block kb into stage s (one commit group)
    auto copy_k = [&](int kb, int s) {
        const uint32_t sa = stage0 + (uint32_t)s * G_STAGE;
        for (int q = tid; q < 6 * G_TILE * 8; q += G_THREADS) {
            const int pl = q >> 10, rem = q & 1023;
            const int row = rem >> 3, ch = rem & 7;
            const int grow = (pl < 3 ? bi : bj) * G_TILE + row;
            const int p3 = pl < 3 ? pl : pl - 3;
            const uint16_t *src = (p3 == 0 ? Zh : (p3 == 1 ? Zm : Zl)) + (size_t)grow * Tp +
                                  (size_t)kb * G_KB + ch * 8;
            const uint32_t d = sa + (uint32_t)pl * G_OP_BYTES + row * 128 + ((ch ^ (row & 7)) * 16);
            cp_async16(d, src, 16);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // products (A plane, B plane): hi hi, hi mid, mid hi, hi lo, lo hi, mid mid
    const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
    int it = 0;
    copy_k(kb0, 0);
    for (int kb = kb0; kb < kb1; ++kb, ++it) {
        const int s = it & 1;
        const uint32_t sa = stage0 + (uint32_t)s * G_STAGE;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int kk = 0; kk < G_KB / 16; ++kk)
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint64_t ad = sw128_desc(sa + (uint32_t)pa[p] * G_OP_BYTES + 32 * kk);
                    const uint64_t bd = sw128_desc(sa + (uint32_t)(3 + pb[p]) * G_OP_BYTES + 32 * kk);
                    const int q = kb - kb0;
                    mma_bf16(tmem + (uint32_t)((q % G_NACC) * G_TILE), ad, bd, idesc,
                             (q >= G_NACC || kk || p) ? 1u : 0u);
                }
            mma_commit(smem_u32(&mbar[s]));
        }
        if (kb + 1 < kb1) {
            // the other stage is free once the MMAs of the previous block are done
            if (it >= 1) {
                if (tid == 0 &&
                    !mbar_wait(smem_u32(&mbar[(it - 1) & 1]), ((it - 1) >> 1) & 1, budget))
                    s_abort = 1;
                __syncthreads();
                if (s_abort) {
                    ++it;
                    break;
                }
            }
            copy_k(kb + 1, s ^ 1);
        }
    }
    if (!s_abort) {
        const int last = it - 1;
        if (tid == 0 && !mbar_wait(smem_u32(&mbar[last & 1]), (last >> 1) & 1, budget)) s_abort = 1;
        __syncthreads();
    }
    if (!s_abort) {
        // the used accumulators added in FP32 (each holds a quarter of the
        // K-blocks, which keeps the accumulation error of the tensor cores,
        // relative to the accumulator's magnitude and step count, small)
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int row = warp * 32 + (tid & 31);
        const int nacc = min(G_NACC, kb1 - kb0);
        float *drow = dst + (size_t)row * G_TILE;
#pragma unroll 1
        for (int q = 0; q < G_TILE / 32; ++q) {
            float acc[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0.f;
#pragma unroll 1
            for (int a = 0; a < nacc; ++a) {
                uint32_t v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                    "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, "
                    "%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
                      "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]),
                      "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * G_TILE) + 32u * q));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int c = 0; c < 32; ++c) acc[c] += __uint_as_float(v[c]);
            }
            float4 *o = reinterpret_cast<float4 *>(drow + 32 * q);
#pragma unroll
            for (int c = 0; c < 8; ++c)
                o[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
        }
    }
    __syncthreads();
    if (s_abort && tid == 0) {
        atomicOr(err, 4);
        if (it >= 1) mbar_wait(smem_u32(&mbar[(it - 1) & 1]), ((it - 1) >> 1) & 1);
        if (it >= 2) mbar_wait(smem_u32(&mbar[(it - 2) & 1]), ((it - 2) >> 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(G_TMEM_COLS));
    }
}

// S_ij of one tile element: the splits' FP32 partials as fixed-point
// integers (2^-fixb), added exactly in split order
__device__ __forceinline__ long long gram_sum(const float *__restrict__ part, int nsplit,
                                              int ntiles, int tile, int r, int c, int fixb)
{
    long long s = 0;
    const size_t stride = (size_t)ntiles * G_TILE * G_TILE;
    const float *p = part + (size_t)tile * G_TILE * G_TILE + (size_t)r * G_TILE + c;
    for (int k = 0; k < nsplit; ++k) s += fix_of(p[k * stride], fixb);
    return s;
}

// 1 / sqrt(S_jj) per column; zero variance flagged (bit 1)
__global__ void gram_diag_kernel(const float *__restrict__ part, int nsplit, int ntiles, int nb,
                                 int N, int fixb, double *__restrict__ inv, int *__restrict__ err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int b = j / G_TILE, r = j - b * G_TILE;
    const int tile = b * nb - b * (b - 1) / 2; // index of (b, b)
    const long long s = gram_sum(part, nsplit, ntiles, tile, r, r, fixb);
    if (s <= 0) {
        atomicOr(err, 2);
        inv[j] = 0.0;
    } else {
        inv[j] = 1.0 / sqrt(dbl_scaled(s, fixb));
    }
}

// C of tile blockIdx.x, rows 8 blockIdx.y .. + 7: both triangles, diagonal 1
__global__ void __launch_bounds__(256)
    gram_out_kernel(const float *__restrict__ part, int nsplit, int ntiles, int nb, int N,
                    int fixb, const double *__restrict__ inv, double *__restrict__ C)
{
    int bi, bj;
    tile_pair(blockIdx.x, nb, &bi, &bj);
    for (int e = threadIdx.x; e < 8 * G_TILE; e += blockDim.x) {
        const int rr = e / G_TILE, c = e - rr * G_TILE, r = blockIdx.y * 8 + rr;
        const int i = bi * G_TILE + r, j = bj * G_TILE + c;
        if (i >= N || j >= N || (bi == bj && j < i)) continue;
        double v = 1.0;
        if (i != j) {
            v = dbl_scaled(gram_sum(part, nsplit, ntiles, blockIdx.x, r, c, fixb), fixb) * inv[i] *
                inv[j];
            if (v > 1.0) v = 1.0;
            if (v < -1.0) v = -1.0;
        }
        C[(size_t)i * N + j] = v;
        C[(size_t)j * N + i] = v;
    }
}

int corr_run_tc(const double *R, int T, int N, int ld, double *C, cudaStream_t s)
{
    const int B = bitlen(T);
    if (B > 40) return set_error(GPGA_ERR_ARG, "cluster_corr: T=%d too large", T);
    const int Nq = (N + G_TILE - 1) / G_TILE * G_TILE;
    const int Tp = (T + G_KB - 1) / G_KB * G_KB;
    const int nb = Nq / G_TILE, ntiles = nb * (nb + 1) / 2, nkb = Tp / G_KB;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // about one CTA per SM: split T over the CTAs of each tile
    int nsplit = sms / ntiles;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > nkb) nsplit = nkb;
    const int kb_per = (nkb + nsplit - 1) / nsplit;
    nsplit = (nkb + kb_per - 1) / kb_per;
    // fixed point of the partial sums: |S| <= T < 2^B, so 2^fixb |S| < 2^61
    const int fixb = 60 - B < 40 ? 60 - B : 40;

    const size_t b_plane = (size_t)Nq * Tp * sizeof(uint16_t);
    const size_t b_part = (size_t)nsplit * ntiles * G_TILE * G_TILE * sizeof(float);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        const size_t o = off;
        off += bytes;
        return o;
    };
    const size_t o_h = take(b_plane), o_m = take(b_plane), o_l = take(b_plane);
    const size_t o_part = take(b_part);
    const size_t o_emax = take((size_t)N * sizeof(int));
    const size_t o_s1 = take((size_t)N * sizeof(unsigned long long));
    const size_t o_inv = take((size_t)N * sizeof(double));
    const size_t o_err = take(sizeof(int));
    const size_t total = off + 256;
    char *ws = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&ws, total, s));
    uint16_t *Zh = (uint16_t *)(ws + o_h), *Zm = (uint16_t *)(ws + o_m), *Zl = (uint16_t *)(ws + o_l);
    float *part = (float *)(ws + o_part);
    int *emax = (int *)(ws + o_emax);
    unsigned long long *S1 = (unsigned long long *)(ws + o_s1);
    double *inv = (double *)(ws + o_inv);
    int *err = (int *)(ws + o_err);
    int rc = GPGA_OK, herr = 0;
    do {
        if (cudaMemsetAsync(emax, 0, (size_t)N * sizeof(int), s) != cudaSuccess ||
            cudaMemsetAsync(S1, 0, (size_t)N * sizeof(unsigned long long), s) != cudaSuccess ||
            cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
            rc = set_error(GPGA_ERR_CUDA, "cluster_corr: memset failed");
            break;
        }
        const dim3 cgrid((N + 31) / 32, (T + CT_ROWS - 1) / CT_ROWS), cblock(32, 8);
        colscan_kernel<<<cgrid, cblock, 0, s>>>(R, T, N, ld, emax, err);
        colfix_kernel<<<cgrid, cblock, 0, s>>>(R, T, N, ld, emax, B, S1);
        zsplit_kernel<<<dim3(Tp / 32, Nq / 32), dim3(32, 8), 0, s>>>(R, T, N, ld, emax, B, S1, Tp,
                                                                     Zh, Zm, Zl);
        gram_tc_kernel<<<dim3(ntiles, nsplit), G_THREADS, G_SMEM, s>>>(
            Zh, Zm, Zl, Tp, nb, kb_per, nkb, part, wait_budget(), err);
        gram_diag_kernel<<<(N + 255) / 256, 256, 0, s>>>(part, nsplit, ntiles, nb, N, fixb, inv,
                                                          err);
        gram_out_kernel<<<dim3(ntiles, G_TILE / 8), 256, 0, s>>>(part, nsplit, ntiles, nb, N, fixb,
                                                                 inv, C);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "cluster_corr", __FILE__, __LINE__);
    } while (0);
    cudaFreeAsync(ws, s);
    if (rc) return rc;
    if (herr & 4)
        return set_error(GPGA_ERR_TIMEOUT, "cluster_corr: a bounded device wait gave up");
    if (herr & 2)
        return set_error(GPGA_ERR_DEGENERATE,
                         "cluster_corr: a column has a non-finite value or zero variance");
    return GPGA_OK;
}

int prepare_corr_tc_kernels(int maxsmem)
{
    (void)maxsmem;
    GPGA_CUDA(cudaFuncSetAttribute((const void *)gram_tc_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM));
    return GPGA_OK;
}

} // namespace gpga
