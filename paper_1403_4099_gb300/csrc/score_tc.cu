// score_tc.cu -- tensor form of Eq. 6: d_s = 1^T D_ss 1 for every non-singleton
// cluster of every individual, as one dense tcgen05 contraction per tile
//   Z^T[c, i] = sum_j S^T[c, j] D[j, i]
// with the one-hot S (exact in BF16) as the A operand (M = 128 cluster columns
// per tile, K = genes), D = 1 - C split into BF16 hi + lo (D_hi + D_lo carries
// ~16 mantissa bits) as two B operands (N = 256 rows of D per tile) accumulated
// into the same FP32 TMEM accumulator, and the epilogue
//   d_c = sum_{i in c} Z^T[c, i]
// read back with tcgen05.ld, masked by the cluster's membership bits, turned
// into fixed point and added with integer atomics (exact, deterministic).
//
// Kernels:
//   tc_prep_kernel      one warp per individual: histogram, one column per
//                       non-singleton cluster (reserved with an atomic), the
//                       column's membership bitmask (one match per 32 genes),
//                       size and zeroed sum
//   tc_mma_kernel       persistent, one CTA (4 warps) per SM: per unit
//                       (128 columns x 256 rows) and 64-gene K-block, the
//                       threads build the one-hot tile from the bitmasks and
//                       cp.async the D_hi / D_lo tiles into 128-byte-swizzled
//                       shared memory (two stages); one thread issues
//                       tcgen05.mma (M128 N256 K16, kind::f16, BF16 in, FP32
//                       accumulate) and commits to the stage's mbarrier
//   tc_assemble_kernel  one warp per individual: Eq. 8 over its columns in
//                       the fixed-point one-log form
// Every pipeline wait is bounded by the wait budget (gpga_set_wait_budget;
// default 2^32 cycles, about 2 s); a timeout sets bit 2 of the error word,
// stops issuing work, waits with the full default bound for the MMAs already
// committed, and the CTA still frees its TMEM.
#include "score_tc.cuh"
#include "tc_ptx.cuh"

namespace gpga {

constexpr int TC_M = 128;     // cluster columns per accumulator (MMA M)
constexpr int TC_ACC = 2;     // accumulators per CTA: 256 columns share every D tile
constexpr int TC_NT = 256;    // rows of D per tile (MMA N, largest)
constexpr int TC_KB = 64;     // genes per K-block: one 128-byte row of BF16
constexpr int TC_THREADS = 128;
constexpr int A_BYTES = TC_M * TC_KB * 2;                     // 16 KB per accumulator
constexpr int B_BYTES = TC_NT * TC_KB * 2;                    // 32 KB
constexpr int STAGE_BYTES = TC_ACC * A_BYTES + 2 * B_BYTES;   // 96 KB
constexpr int TC_SMEM = 2 * STAGE_BYTES + 1024 + 256;
constexpr int TC_TMEM_COLS = 512; // TC_ACC accumulators of TC_NT FP32 columns

// ---------------------------------------------------------------------------
// scratch layout
// ---------------------------------------------------------------------------
static size_t tc_layout(TcWork *w, int N, int Np, int P, size_t off, char *base)
{
    const size_t maxcols = (size_t)P * (size_t)(N / 2 > 0 ? N / 2 : 1);
    const size_t W = (size_t)Np / 32;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        char *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    char *b = take(maxcols * W * sizeof(uint32_t));
    char *n = take(maxcols * sizeof(int32_t));
    char *d = take(maxcols * sizeof(long long));
    char *cb = take((size_t)P * sizeof(int32_t));
    char *kc = take((size_t)P * sizeof(int32_t));
    char *nc = take(sizeof(unsigned));
    char *er = take(sizeof(int));
    if (w) {
        w->bits = reinterpret_cast<uint32_t *>(b);
        w->col_n = reinterpret_cast<int32_t *>(n);
        w->dfix = reinterpret_cast<long long *>(d);
        w->colbase = reinterpret_cast<int32_t *>(cb);
        w->kcount = reinterpret_cast<int32_t *>(kc);
        w->ncols = reinterpret_cast<unsigned *>(nc);
        w->err = reinterpret_cast<int *>(er);
        w->maxcols = (int)maxcols;
    }
    return off;
}

size_t tc_scratch_bytes(int N, int Np, int P) { return tc_layout(nullptr, N, Np, P, 0, nullptr) + 256; }

void tc_carve(TcWork *w, int N, int Np, int P, size_t *off, char *base)
{
    *off = tc_layout(w, N, Np, P, *off, base);
}

// ---------------------------------------------------------------------------
// prep: columns, membership bitmasks, sizes
// ---------------------------------------------------------------------------
template <typename LabT>
__global__ void __launch_bounds__(256)
    tc_prep_kernel(const LabT *lab0, const LabT *lab1, int ldl, int sel_off, int P, int N, int Np,
                   TcWork w, int *__restrict__ err, const DevState *__restrict__ st,
                   unsigned long long *__restrict__ pairs, unsigned long long *__restrict__ clusters)
{
    const LabT *__restrict__ lab = lab0;
    unsigned long long *pairs_g = nullptr, *clus_g = nullptr;
    if (st) {
        if (st->done) return;
        const int gen = st->gen + sel_off;
        lab = (gen & 1) ? lab1 : lab0;
        if (pairs) pairs_g = pairs + gen;
        if (clusters) clus_g = clusters + gen;
    }
    extern __shared__ int sm_tc[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int *cnt = sm_tc + (size_t)warp * 2 * Np;
    int *cid = cnt + Np;
    const int W = Np >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int p = blockIdx.x * nw + warp; p < P; p += gridDim.x * nw) {
        const LabT *lp = lab + (size_t)p * ldl;
        for (int s = lane; s < Np; s += 32) cnt[s] = 0;
        __syncwarp();
        for (int i = lane; i < N; i += 32) {
            const int v = (int)lp[i];
            if (v >= 0 && v < N) atomicAdd(&cnt[v], 1); // range errors: the assembly flags them
        }
        __syncwarp();
        // compact ids of the non-singleton clusters, ascending label
        int k = 0;
        long long np = 0;
        for (int base = 0; base < N; base += 32) {
            const int s = base + lane;
            const int n = s < N ? cnt[s] : 0;
            const unsigned m = __ballot_sync(0xffffffffu, n >= 2);
            if (s < Np) cid[s] = n >= 2 ? k + __popc(m & lt) : -1;
            np += n >= 2 ? (long long)n * (n - 1) / 2 : 0;
            k += __popc(m);
        }
        int cbase = 0;
        if (lane == 0) cbase = (int)atomicAdd(w.ncols, (unsigned)k);
        cbase = __shfl_sync(0xffffffffu, cbase, 0);
        if (cbase + k > w.maxcols) { // cannot happen: at most N/2 clusters per individual
            if (lane == 0) atomicOr(err, 4);
            k = 0;
        }
        if (lane == 0) {
            w.colbase[p] = cbase;
            w.kcount[p] = k;
            if (clus_g) atomicAdd(clus_g, (unsigned long long)k);
        }
        __syncwarp();
        for (int s = lane; s < N; s += 32) {
            const int c = cid[s];
            if (c >= 0 && c < k) {
                w.col_n[cbase + c] = cnt[s];
                w.dfix[cbase + c] = 0;
            }
        }
        // membership bitmasks: zero, then one word per 32 genes per cluster
        uint32_t *bits = w.bits + (size_t)cbase * W;
        for (int t = lane; t < k * W; t += 32) bits[t] = 0u;
        __syncwarp();
        for (int wd = 0; wd < W; ++wd) {
            const int i = wd * 32 + lane;
            int c = -1;
            if (i < N) {
                const int v = (int)lp[i];
                if (v >= 0 && v < N) c = cid[v];
            }
            const unsigned act = __ballot_sync(0xffffffffu, c >= 0 && c < k);
            if (c >= 0 && c < k) {
                const unsigned peers = __match_any_sync(act, c);
                if ((peers & lt) == 0u) bits[(size_t)c * W + wd] = peers;
            }
        }
        if (pairs_g) {
#pragma unroll
            for (int o = 16; o; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
            if (lane == 0) atomicAdd(pairs_g, (unsigned long long)np);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// the contraction
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_mma_kernel(TcWork w, const __nv_bfloat16 *__restrict__ Dhi,
                  const __nv_bfloat16 *__restrict__ Dlo, int Np, int NT, int fix_bits,
                  const DevState *__restrict__ st, long long budget)
{
    if (st && st->done) return;
    extern __shared__ unsigned char sm_raw[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5;
    // 1024-byte aligned stage buffers
    const uint32_t raw = smem_u32(sm_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    // stage s at a byte offset s * STAGE_BYTES (selected arithmetically: a
    // run-time index into a local array would live in local memory)
    unsigned char *const stage0 = sm_raw + pad;
    const uint32_t stage0_addr = raw + pad;

    const int ncols = (int)*w.ncols;
    const int nct = (ncols + TC_ACC * TC_M - 1) / (TC_ACC * TC_M);
    const int nnt = (Np + NT - 1) / NT;
    const int units = nct * nnt;
    if ((int)blockIdx.x >= units) return;
    const int W = Np >> 5;
    const int KB = Np / TC_KB;
    // instruction descriptor: D F32, A BF16, B BF16, both K-major, N = NT, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    // thread 0 alone waits on the mbarriers; its verdict reaches every thread
    // through s_abort after a barrier, so control flow stays CTA-uniform
    int it = 0; // K-blocks issued by this CTA (stage = it & 1, use = it >> 1)
    for (int u = blockIdx.x; u < units && !s_abort; u += gridDim.x) {
        const int ct = u / nnt, nt = u - ct * nnt;
        const int c0 = ct * TC_ACC * TC_M, n0 = nt * NT;
        // membership words of the current K-block, prefetched one block ahead
        uint32_t bw[TC_ACC][2];
#pragma unroll
        for (int acc = 0; acc < TC_ACC; ++acc) {
            const int col = c0 + acc * TC_M + tid;
            bw[acc][0] = col < ncols ? w.bits[(size_t)col * W] : 0u;
            bw[acc][1] = col < ncols ? w.bits[(size_t)col * W + 1] : 0u;
        }
        // D tiles of K-block kb into stage s (all threads; one commit group)
        auto copy_d = [&](int kb, int s) {
            const uint32_t bh = stage0_addr + (uint32_t)s * STAGE_BYTES + TC_ACC * A_BYTES,
                           bl = bh + B_BYTES;
            for (int q = tid; q < NT * 8; q += TC_THREADS) {
                const int row = q >> 3, ch = q & 7;
                const int gi = n0 + row;
                const bool in = gi < Np;
                const size_t off = (size_t)(in ? gi : 0) * Np + (size_t)kb * TC_KB + ch * 8;
                const uint32_t dofs = row * 128 + ((ch ^ (row & 7)) * 16);
                cp_async16(bh + dofs, Dhi + off, in ? 16 : 0);
                cp_async16(bl + dofs, Dlo + off, in ? 16 : 0);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        // software pipeline over the K-blocks of this unit: the D tiles of block
        // kb + 1 stream into the other stage while the MMAs of block kb run
        // (every MMA of the previous unit is complete: its epilogue waited)
        copy_d(0, it & 1);
        for (int kb = 0; kb < KB; ++kb, ++it) {
            const int s = it & 1;
            unsigned char *A = stage0 + (size_t)s * STAGE_BYTES;
            const uint32_t Aaddr = stage0_addr + (uint32_t)s * STAGE_BYTES;
            const uint32_t Bh = Aaddr + TC_ACC * A_BYTES, Bl = Bh + B_BYTES;
            // one-hot rows from the membership bits (thread = column of each
            // accumulator's tile)
#pragma unroll
            for (int acc = 0; acc < TC_ACC; ++acc) {
                const int col = c0 + acc * TC_M + tid;
                const uint32_t w0 = bw[acc][0], w1 = bw[acc][1];
                if (kb + 1 < KB) {
                    bw[acc][0] = col < ncols ? w.bits[(size_t)col * W + 2 * kb + 2] : 0u;
                    bw[acc][1] = col < ncols ? w.bits[(size_t)col * W + 2 * kb + 3] : 0u;
                }
                unsigned char *Aa = A + acc * A_BYTES;
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) {
                    const uint32_t byte = ((ch < 4 ? w0 : w1) >> (8 * (ch & 3))) & 0xffu;
                    uint32_t q[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h)
                        q[h] = ((byte >> (2 * h)) & 1u ? 0x3F80u : 0u) |
                               ((byte >> (2 * h + 1)) & 1u ? 0x3F800000u : 0u);
                    *reinterpret_cast<uint4 *>(Aa + tid * 128 + ((ch ^ (tid & 7)) * 16)) =
                        make_uint4(q[0], q[1], q[2], q[3]);
                }
            }
            asm volatile("cp.async.wait_group 0;" ::: "memory"); // block kb's D tiles
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int kk = 0; kk < TC_KB / 16; ++kk) {
                    const uint64_t bh = sw128_desc(Bh + 32 * kk), bl = sw128_desc(Bl + 32 * kk);
#pragma unroll
                    for (int acc = 0; acc < TC_ACC; ++acc) {
                        const uint64_t ad = sw128_desc(Aaddr + acc * A_BYTES + 32 * kk);
                        const uint32_t t = tmem + (uint32_t)(acc * TC_NT);
                        mma_bf16(t, ad, bh, idesc, (kb | kk) ? 1u : 0u);
                        mma_bf16(t, ad, bl, idesc, 1u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&mbar[s]))
                             : "memory");
            }
            if (kb + 1 < KB) {
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
                copy_d(kb + 1, s ^ 1);
            }
        }
        if (s_abort) break;
        // epilogue: wait for the last K-block's MMAs (all earlier ones are done too)
        const int last = it - 1;
        if (tid == 0 && !mbar_wait(smem_u32(&mbar[last & 1]), (last >> 1) & 1, budget))
            s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
        for (int a2 = 0; a2 < TC_ACC; ++a2) {
            const int col = c0 + a2 * TC_M + tid;
            float acc = 0.f;
            const uint32_t lane_base = ((uint32_t)(warp * 32) << 16) + (uint32_t)(a2 * TC_NT);
            for (int q = 0; q < NT / 32; ++q) {
                uint32_t v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                    "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, "
                    "%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                      "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                      "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                      "=r"(v[30]), "=r"(v[31])
                    : "r"(tmem + lane_base + 32u * q));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (col < ncols && n0 + 32 * q < Np) {
                    const uint32_t mk = w.bits[(size_t)col * W + (n0 >> 5) + q];
#pragma unroll
                    for (int t = 0; t < 32; ++t)
                        if ((mk >> t) & 1u) acc += __uint_as_float(v[t]);
                }
            }
            if (col < ncols)
                atomicAdd(reinterpret_cast<unsigned long long *>(w.dfix + col),
                          (unsigned long long)fix_of(acc, fix_bits));
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    // on a timeout: flag it, then wait (with the full default bound, whatever
    // the budget) for the commits still in flight before freeing TMEM
    __syncthreads();
    if (s_abort && tid == 0) {
        atomicOr(w.err, 4);
        if (it >= 1) mbar_wait(smem_u32(&mbar[(it - 1) & 1]), ((it - 1) >> 1) & 1);
        if (it >= 2) mbar_wait(smem_u32(&mbar[(it - 2) & 1]), ((it - 2) >> 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TC_TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// assembly: Eq. 8 per individual from its columns (n_s, exact d_s)
// ---------------------------------------------------------------------------
template <typename LabT>
__global__ void __launch_bounds__(256)
    tc_assemble_kernel(const LabT *lab0, const LabT *lab1, int ldl, int sel_off, int P, int N,
                       TcWork w, const double *__restrict__ logtab, int fix_bits,
                       double *__restrict__ L, int *__restrict__ err,
                       const DevState *__restrict__ st)
{
    const LabT *__restrict__ lab = lab0;
    if (st) {
        if (st->done) return;
        lab = ((st->gen + sel_off) & 1) ? lab1 : lab0;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const long long *ltab = reinterpret_cast<const long long *>(logtab);
    const long long *kfix = kfix_of(logtab);
    const bool timeout = (*w.err & 4) != 0;
    for (int p = blockIdx.x * nw + warp; p < P; p += gridDim.x * nw) {
        bool bad = false;
        const LabT *lp = lab + (size_t)p * ldl;
        for (int i = lane; i < N; i += 32) {
            const int v = (int)lp[i];
            bad |= !(v >= 0 && v < N);
        }
        bad = __any_sync(0xffffffffu, bad) || timeout;
        const int cb = w.colbase[p], k = w.kcount[p];
        LogProd acc;
        for (int c = lane; c < k; c += 32)
            logprod_add(acc, w.col_n[cb + c], w.dfix[cb + c], fix_bits, kfix);
        const double v = logprod_finish(acc, ltab, k);
        if (lane == 0) {
            L[p] = bad ? __longlong_as_double(0x7ff8000000000000ll) : v;
            if (bad && err) atomicOr(err, timeout ? 4 : 1);
        }
    }
}

template <typename LabT>
int tc_contract(TcWork *w, const __nv_bfloat16 *Dhi, const __nv_bfloat16 *Dlo, int Np,
                const LabT *const *lab2, int ldl, int sel_off, int P, int N, int *err,
                const DevState *st, unsigned long long *pairs, unsigned long long *clusters,
                cudaStream_t s)
{
    GPGA_CUDA(cudaMemsetAsync(w->ncols, 0, sizeof(unsigned), s));
    GPGA_CUDA(cudaMemsetAsync(w->err, 0, sizeof(int), s));
    {
        const size_t per = (size_t)2 * Np * sizeof(int);
        int nw = 8;
        while (nw > 1 && nw * per > (size_t)200 * 1024) nw >>= 1;
        tc_prep_kernel<LabT><<<(P + nw - 1) / nw, 32 * nw, nw * per, s>>>(
            lab2[0], lab2[1], ldl, sel_off, P, N, Np, *w, err, st, pairs, clusters);
        GPGA_LAUNCH_CHECK();
    }
    const int NT = Np < TC_NT ? Np : TC_NT;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    tc_mma_kernel<<<sms, TC_THREADS, TC_SMEM, s>>>(*w, Dhi, Dlo, Np, NT, fix_bits_for(N), st,
                                                    wait_budget());
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template <typename LabT>
int tc_finish(TcWork *w, const LabT *const *lab2, int ldl, int sel_off, int P, int N,
              const double *logtab, double *L, int *err, const DevState *st, cudaStream_t s)
{
    tc_assemble_kernel<LabT><<<(P + 7) / 8, 256, 0, s>>>(lab2[0], lab2[1], ldl, sel_off, P, N,
                                                         *w, logtab, fix_bits_for(N), L, err, st);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template int tc_contract<uint16_t>(TcWork *, const __nv_bfloat16 *, const __nv_bfloat16 *, int,
                                   const uint16_t *const *, int, int, int, int, int *,
                                   const DevState *, unsigned long long *, unsigned long long *,
                                   cudaStream_t);
template int tc_contract<int32_t>(TcWork *, const __nv_bfloat16 *, const __nv_bfloat16 *, int,
                                  const int32_t *const *, int, int, int, int, int *,
                                  const DevState *, unsigned long long *, unsigned long long *,
                                  cudaStream_t);
template int tc_finish<uint16_t>(TcWork *, const uint16_t *const *, int, int, int, int,
                                 const double *, double *, int *, const DevState *, cudaStream_t);
template int tc_finish<int32_t>(TcWork *, const int32_t *const *, int, int, int, int,
                                const double *, double *, int *, const DevState *, cudaStream_t);

int prepare_tc_kernels(int maxsmem)
{
    if (int rc = raise_smem(tc_mma_kernel, maxsmem)) return rc;
    if (int rc = raise_smem(tc_prep_kernel<uint16_t>, maxsmem)) return rc;
    if (int rc = raise_smem(tc_prep_kernel<int32_t>, maxsmem)) return rc;
    return GPGA_OK;
}

} // namespace gpga
