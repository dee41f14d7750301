// corr.cu -- Pearson correlation prelude, Eq. 7 (Sec. 2.1; the standardisation
// below Eq. 2): C_ij = <z_i, z_j> / sqrt(|z_i|^2 |z_j|^2), z = R - column mean.
// Unit weights (cluster_corr) run the tensor-core path of corr_tc.cu; this
// file holds the weighted (EWMA) path and the market-mode removal.
//
// Passes over R (T x N FP64, row-major, leading dim ld):
//   1. column sums over T-slabs (FP64 partials, fixed order) -> means, finiteness
//   2. centred sums of squares (FP64 partials) -> 1 / sqrt(q_j), zero-variance check
//   3. Z = fp32((R - mean) / sqrt(q)), T x Np, zero padding columns
//   4. C = Z^T Z on the upper-triangle 64 x 64 tiles, T split across CTAs for
//      parallelism: FP32 FMA over sub-slabs of <= 512 rows added into FP64
//      accumulators; a final pass sums the CTAs' partials in fixed order, writes
//      both triangles, diagonal 1, clamps to [-1, 1].
// The contraction is FP32 on unit-norm columns: |error| ~ 1e-7 on C.
#include <math.h>

#include "gpga_internal.cuh"

namespace gpga {

static constexpr int CS_COLS = 32, CS_ROWS = 8; // column-stat CTA: 32 columns x 8 row lanes
static constexpr int T_SLAB = 128;              // rows per column-stat CTA

// column sums over a slab of rows: sum_t w_t (R_tj - mean_j)^2 with mean, else
// sum_t w_t R_tj (w == nullptr: all weights 1)
__global__ void colsum_kernel(const double *__restrict__ R, int T, int N, int ld,
                              const double *__restrict__ mean, const double *__restrict__ w,
                              double *__restrict__ part)
{
    __shared__ double red[CS_ROWS][CS_COLS + 1];
    const int cx = threadIdx.x, ry = threadIdx.y;
    const int j = blockIdx.x * CS_COLS + cx;
    const int t0 = blockIdx.y * T_SLAB;
    const int t1 = min(T, t0 + T_SLAB);
    double s = 0.0;
    if (j < N) {
        const double mu = mean ? mean[j] : 0.0;
        // four rows in flight per thread, four partial sums (fixed order)
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        int t = t0 + ry;
        for (; t + 3 * CS_ROWS < t1; t += 4 * CS_ROWS) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = R[(size_t)(t + u * CS_ROWS) * ld + j] - mu;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double x = mean ? v[u] * v[u] : v[u];
                a[u] += w ? w[t + u * CS_ROWS] * x : x;
            }
        }
        for (; t < t1; t += CS_ROWS) {
            const double v = R[(size_t)t * ld + j] - mu;
            const double x = mean ? v * v : v;
            a[0] += w ? w[t] * x : x;
        }
        s = (a[0] + a[1]) + (a[2] + a[3]);
    }
    red[ry][cx] = s;
    __syncthreads();
    if (ry == 0 && j < N) {
        double a = 0.0;
        for (int r = 0; r < CS_ROWS; ++r) a += red[r][cx];
        part[(size_t)blockIdx.y * N + j] = a;
    }
}

// wsum: total weight (nullptr: uniform weights, T)
__global__ void colfinal_kernel(const double *__restrict__ part, int nslab, int T,
                                const double *wsum, int N, double *__restrict__ out, int mode,
                                int *__restrict__ err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double a = 0.0;
    for (int k = 0; k < nslab; ++k) a += part[(size_t)k * N + j];
    if (mode == 0) { // means
        if (!isfinite(a)) atomicOr(err, 2);
        out[j] = a / (wsum ? *wsum : (double)T);
    } else { // 1 / sqrt(q)
        if (!(a > 0.0) || !isfinite(a)) {
            atomicOr(err, 2);
            out[j] = 0.0;
        } else {
            out[j] = 1.0 / sqrt(a);
        }
    }
}

// Z_tj = sqrt(w_t) (R_tj - mean_j) / sqrt(q_j) (sw = sqrt(w), nullptr: 1);
// CTA y takes rows y, y + gridDim.y, ...; its threads the columns of a row
__global__ void normalise_kernel(const double *__restrict__ R, int T, int N, int ld, int Np,
                                 const double *__restrict__ mean, const double *__restrict__ inv,
                                 const double *__restrict__ sw, float *__restrict__ Z)
{
    for (int t = blockIdx.y; t < T; t += gridDim.y) {
        const double st = sw ? sw[t] : 1.0;
        const double *row = R + (size_t)t * ld;
        float *zr = Z + (size_t)t * Np;
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Np; j += gridDim.x * blockDim.x) {
            float z = 0.f;
            if (j < N) {
                const double x = (row[j] - mean[j]) * inv[j];
                z = (float)(sw ? st * x : x);
            }
            zr[j] = z;
        }
    }
}

// exponentially weighted rows: w_t = lambda^(T-1-t) (the newest row weighs 1),
// their square roots, and (one CTA, fixed order) their sum
__global__ void ewma_weights_kernel(int T, double lambda, double *__restrict__ w,
                                    double *__restrict__ sw, double *__restrict__ wsum)
{
    __shared__ double part[1024];
    const double ll = log(lambda);
    double s = 0.0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const double v = lambda == 1.0 ? 1.0 : exp((double)(T - 1 - t) * ll);
        w[t] = v;
        sw[t] = sqrt(v);
        s += v;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) a += part[k];
        *wsum = a;
    }
}

// C tile (bi, bj), bi <= bj, 64 x 64, over rows [t0, t1) of Z. 256 threads, each
// a 4 x 4 micro-tile; Z slices staged through shared memory 16 rows at a time.
// FP32 FMA over sub-slabs of at most SUB rows, added into FP64 accumulators.
static constexpr int GT = 64, GK = 16, SUB = 512;

__global__ void __launch_bounds__(256)
    gram_kernel(const float *__restrict__ Z, int T, int Np, int nb, int trange,
                double *__restrict__ part, int ntiles)
{
    __shared__ float As[2][GK][GT];
    __shared__ float Bs[2][GK][GT];
    // tile index -> (bi, bj) with bi <= bj
    int tile = blockIdx.x, bi = 0;
    while (tile >= nb - bi) {
        tile -= nb - bi;
        ++bi;
    }
    const int bj = bi + tile;
    const int t0 = blockIdx.y * trange;
    const int t1 = min(T, t0 + trange);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc64[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc64[a][b] = 0.0;
    // 16 rows x 64 columns of each operand per slice: 1024 floats, 4 per thread
    float ra[4], rb[4];
    auto fetch = [&](int t, int te) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = threadIdx.x + 256 * r;
            const int tt = t + (e >> 6), c = e & 63;
            ra[r] = tt < te ? Z[(size_t)tt * Np + bi * GT + c] : 0.f;
            rb[r] = tt < te ? Z[(size_t)tt * Np + bj * GT + c] : 0.f;
        }
    };
    auto stage = [&](int buf) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = threadIdx.x + 256 * r;
            As[buf][e >> 6][e & 63] = ra[r];
            Bs[buf][e >> 6][e & 63] = rb[r];
        }
    };
    for (int ts = t0; ts < t1; ts += SUB) {
        const int te = min(t1, ts + SUB);
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        // double-buffered slices: the next slice's loads are in flight while the
        // current one is multiplied (one barrier per slice)
        fetch(ts, te);
        stage(0);
        __syncthreads();
        int buf = 0;
        for (int t = ts; t < te; t += GK) {
            const bool more = t + GK < te;
            if (more) fetch(t + GK, te);
#pragma unroll
            for (int kk = 0; kk < GK; ++kk) {
                float a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = As[buf][kk][ty * 4 + q];
                    b[q] = Bs[buf][kk][tx * 4 + q];
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
            }
            if (more) stage(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc64[x][y] += (double)acc[x][y];
    }
    double *dst = part + ((size_t)blockIdx.y * ntiles + blockIdx.x) * (GT * GT);
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) dst[(ty * 4 + x) * GT + tx * 4 + y] = acc64[x][y];
}

// CTA (tile, y): rows 16 y .. 16 y + 15 of tile `tile` (upper triangle, bi <= bj);
// the partials summed in slab order, then written as rows (coalesced) and, from
// shared memory, as the columns of the mirrored tile
__global__ void __launch_bounds__(256)
    gram_final_kernel(const double *__restrict__ part, int nslab, int ntiles, int nb, int N,
                      double *__restrict__ C)
{
    __shared__ double a_s[16][GT + 1];
    int tile = blockIdx.x, bi = 0;
    while (tile >= nb - bi) {
        tile -= nb - bi;
        ++bi;
    }
    const int bj = bi + tile;
    const int r0 = blockIdx.y * 16;
    const size_t tstride = (size_t)ntiles * (GT * GT);
    for (int e = threadIdx.x; e < 16 * GT; e += blockDim.x) {
        const int rr = e / GT, c = e - rr * GT, r = r0 + rr;
        const double *src = part + (size_t)blockIdx.x * (GT * GT) + r * GT + c;
        double a = 0.0;
        for (int k = 0; k < nslab; ++k) a += src[(size_t)k * tstride];
        const int i = bi * GT + r, j = bj * GT + c;
        if (i == j) a = 1.0;
        if (a > 1.0) a = 1.0;
        if (a < -1.0) a = -1.0;
        a_s[rr][c] = a;
        if (i < N && j < N && !(bi == bj && j < i)) C[(size_t)i * N + j] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * GT; e += blockDim.x) {
        const int c = e >> 4, rr = e & 15, r = r0 + rr;
        const int i = bi * GT + r, j = bj * GT + c;
        if (i < N && j < N && !(bi == bj && j < i)) C[(size_t)j * N + i] = a_s[rr][c];
    }
}

int corr_run(const double *R, int T, int N, int ld, double *C, cudaStream_t s)
{
    return corr_run_weighted(R, T, N, ld, 1.0, C, s);
}

int corr_run_weighted(const double *R, int T, int N, int ld, double lambda, double *C,
                      cudaStream_t s)
{
    // unit weights (plain Pearson): the integer statistics and the tcgen05
    // contraction of corr_tc.cu; below, the FP64 / FP32 path of the EWMA weights
    if (lambda == 1.0) return corr_run_tc(R, T, N, ld, C, s);
    const bool weighted = lambda != 1.0;
    const int Np = pad_n(N);
    const int nslab_c = (T + T_SLAB - 1) / T_SLAB;
    const int nb = Np / GT;
    const int ntiles = nb * (nb + 1) / 2;
    // split T so that the grid covers the GPU about twice (152 SMs)
    int nsplit = (2 * 152 + ntiles - 1) / ntiles;
    if (nsplit < 1) nsplit = 1;
    int trange = (T + nsplit - 1) / nsplit;
    trange = ((trange + GK - 1) / GK) * GK;
    nsplit = (T + trange - 1) / trange;

    const size_t b_part = (size_t)nslab_c * N * sizeof(double);
    const size_t b_vec = (size_t)N * sizeof(double);
    const size_t b_z = (size_t)T * Np * sizeof(float);
    const size_t b_g = (size_t)nsplit * ntiles * GT * GT * sizeof(double);
    const size_t b_w = weighted ? (size_t)2 * T * sizeof(double) : 0;
    const size_t total = b_part + 2 * b_vec + b_z + b_g + b_w + 512;
    char *ws = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&ws, total, s));
    double *part = (double *)ws;
    double *mean = (double *)(ws + b_part);
    double *inv = mean + N;
    float *Z = (float *)(ws + b_part + 2 * b_vec);
    double *gpart = (double *)(ws + b_part + 2 * b_vec + b_z);
    double *wv = weighted ? (double *)(ws + b_part + 2 * b_vec + b_z + b_g) : nullptr;
    double *swv = weighted ? wv + T : nullptr;
    double *wsum = (double *)(ws + total - 512);
    int *err = (int *)(ws + total - 256);
    int rc = GPGA_OK;
    int herr = 0;
    do {
        if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
            rc = set_error(GPGA_ERR_CUDA, "cluster_corr: memset failed");
            break;
        }
        if (weighted) ewma_weights_kernel<<<1, 1024, 0, s>>>(T, lambda, wv, swv, wsum);
        const double *ws_ = weighted ? wsum : nullptr;
        dim3 cgrid((N + CS_COLS - 1) / CS_COLS, nslab_c), cblock(CS_COLS, CS_ROWS);
        colsum_kernel<<<cgrid, cblock, 0, s>>>(R, T, N, ld, nullptr, wv, part);
        colfinal_kernel<<<(N + 255) / 256, 256, 0, s>>>(part, nslab_c, T, ws_, N, mean, 0, err);
        colsum_kernel<<<cgrid, cblock, 0, s>>>(R, T, N, ld, mean, wv, part);
        colfinal_kernel<<<(N + 255) / 256, 256, 0, s>>>(part, nslab_c, T, ws_, N, inv, 1, err);
        const int zx = (Np + 255) / 256;
        const int zy = T < 65535 / zx ? T : 65535 / zx;
        normalise_kernel<<<dim3(zx, zy), 256, 0, s>>>(R, T, N, ld, Np, mean, inv, swv, Z);
        gram_kernel<<<dim3(ntiles, nsplit), 256, 0, s>>>(Z, T, Np, nb, trange, gpart, ntiles);
        gram_final_kernel<<<dim3(ntiles, GT / 16), 256, 0, s>>>(gpart, nsplit, ntiles, nb, N, C);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_error(e, "cluster_corr kernels", __FILE__, __LINE__);
            break;
        }
        e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "cluster_corr sync", __FILE__, __LINE__);
            break;
        }
    } while (0);
    cudaFreeAsync(ws, s);
    if (rc == GPGA_OK && herr)
        rc = set_error(GPGA_ERR_DEGENERATE,
                       "cluster_corr: a column has a non-finite value or zero variance");
    return rc;
}

// ---------------------------------------------------------------------------
// Market-mode removal (pre-processing upstream of C): the largest eigenpair
// (lambda_1, v) of C by power iteration from the uniform vector (FP64; stops
// when no component of v moves by more than 1e-14, or after max_iters), then
// C' = C - lambda_1 v v^T renormalised to unit diagonal:
// C''_ij = C'_ij / sqrt(C'_ii C'_jj), diagonal 1, clamped to [-1, 1].
// ---------------------------------------------------------------------------
__global__ void market_diag_kernel(const double *__restrict__ C, int N,
                                   const double *__restrict__ v, const double *__restrict__ info,
                                   double *__restrict__ dg, int *__restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double d = C[(size_t)i * N + i] - info[0] * v[i] * v[i];
    if (!(d > 0.0)) atomicOr(err, 1);
    dg[i] = d > 0.0 ? d : 1.0;
}

__global__ void market_clean_kernel(double *__restrict__ C, int N, const double *__restrict__ v,
                                    const double *__restrict__ info,
                                    const double *__restrict__ dg)
{
    const size_t total = (size_t)N * N;
    const double lam = info[0];
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / N), j = (int)(idx - (size_t)i * N);
        double c = 1.0;
        if (i != j) {
            c = (C[idx] - lam * v[i] * v[j]) / sqrt(dg[i] * dg[j]);
            if (c > 1.0) c = 1.0;
            if (c < -1.0) c = -1.0;
        }
        C[idx] = c;
    }
}

// ---------------------------------------------------------------------------
// The same power iteration over the whole GPU, one launch per iteration k
// (k = 0 .. max_iters): v_0 = 1/sqrt(N), v_k = u_{k-1} / |u_{k-1}|, u_k = C v_k,
// one warp per row of C. Every CTA forms v_k, v_{k-1}, |u_{k-1}| and
// lambda_{k-1} = v_{k-1} . u_{k-1} itself (fixed-order sums, so all CTAs agree)
// and tests iteration k-1: if no component of v moved by more than 1e-14, or
// k = max_iters, the run stops with lambda_{k-1}, k iterations and v_k (CTA 0
// writes them and the stop flag; later launches return at once). u rotates
// through three buffers.
// ---------------------------------------------------------------------------
constexpr int MP_THREADS = 256;

__device__ double mp_block_sum(double x, double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if (lane == 0) red[wid] = x;
    __syncthreads();
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a += red[k];
    return a;
}

__device__ double mp_block_max(double x, double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    __syncthreads();
    if (lane == 0) red[wid] = x;
    __syncthreads();
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a = fmax(a, red[k]);
    return a;
}

__global__ void __launch_bounds__(MP_THREADS)
    market_iter_kernel(const double *__restrict__ C, int N, int k, int max_iters,
                       double *__restrict__ U, double *__restrict__ vout,
                       double *__restrict__ info)
{
    if (info[2] != 0.0) return;
    extern __shared__ double vk[]; // N
    __shared__ double red[MP_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const double *u1 = U + (size_t)((k + 2) % 3) * N; // u_{k-1}
    const double *u2 = U + (size_t)((k + 1) % 3) * N; // u_{k-2}
    double *uk = U + (size_t)(k % 3) * N;
    const double v0 = 1.0 / sqrt((double)N);
    if (k == 0) {
        for (int j = tid; j < N; j += blockDim.x) vk[j] = v0;
    } else {
        double q = 0.0, q2 = 0.0;
        for (int j = tid; j < N; j += blockDim.x) {
            q += u1[j] * u1[j];
            if (k >= 2) q2 += u2[j] * u2[j];
        }
        const double inv1 = 1.0 / sqrt(mp_block_sum(q, red));
        const double inv2 = k >= 2 ? 1.0 / sqrt(mp_block_sum(q2, red)) : 0.0;
        double lam = 0.0, dv = 0.0;
        for (int j = tid; j < N; j += blockDim.x) {
            const double vprev = k >= 2 ? u2[j] * inv2 : v0; // v_{k-1}
            const double x = u1[j] * inv1;                   // v_k
            lam += vprev * u1[j];
            dv = fmax(dv, fabs(x - vprev));
            vk[j] = x;
        }
        lam = mp_block_sum(lam, red);
        dv = mp_block_max(dv, red);
        if (dv <= 1e-14 || k >= max_iters) {
            if (blockIdx.x == 0) {
                for (int j = tid; j < N; j += blockDim.x) vout[j] = vk[j];
                if (tid == 0) {
                    info[0] = lam;
                    info[1] = (double)k;
                    info[2] = 1.0;
                }
            }
            return;
        }
    }
    __syncthreads();
    for (int r = blockIdx.x * nw + wid; r < N; r += gridDim.x * nw) {
        double a = 0.0;
        for (int j = lane; j < N; j += 32) a += C[(size_t)r * N + j] * vk[j];
#pragma unroll
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) uk[r] = a;
    }
}

int market_remove(double *C, int N, int max_iters, double *lambda1, int *iters, cudaStream_t s)
{
    const size_t bytes = (size_t)N * 5 * sizeof(double) + 4 * sizeof(double) + 256;
    char *ws = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&ws, bytes, s));
    double *v = (double *)ws, *dg = v + N, *U = dg + N, *info = U + 3 * (size_t)N;
    int *err = (int *)(ws + bytes - 64);
    double hinfo[3] = {0.0, 0.0, 0.0};
    int herr = 0, rc = GPGA_OK;
    do {
        if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
            cudaMemsetAsync(info, 0, 4 * sizeof(double), s) != cudaSuccess) {
            rc = set_error(GPGA_ERR_CUDA, "corr_remove_market: memset failed");
            break;
        }
        // one launch per iteration over the whole GPU, the stop flag read back
        // every 16 launches (the launches after the stop return at once)
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int rows_per_cta = MP_THREADS / 32;
        int grid = (N + rows_per_cta - 1) / rows_per_cta;
        if (grid > sms) grid = sms;
        const size_t smem = (size_t)N * sizeof(double);
        cudaError_t e = cudaSuccess;
        for (int k = 0; k <= max_iters && e == cudaSuccess;) {
            const int stop = k + 16 <= max_iters + 1 ? k + 16 : max_iters + 1;
            for (; k < stop; ++k)
                market_iter_kernel<<<grid, MP_THREADS, smem, s>>>(C, N, k, max_iters, U, v, info);
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (hinfo[2] != 0.0) break;
        }
        if (e != cudaSuccess) {
            rc = cuda_error(e, "corr_remove_market power iteration", __FILE__, __LINE__);
            break;
        }
        market_diag_kernel<<<(N + 255) / 256, 256, 0, s>>>(C, N, v, info, dg, err);
        const size_t total = (size_t)N * N;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        market_clean_kernel<<<blocks, 256, 0, s>>>(C, N, v, info, dg);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "corr_remove_market", __FILE__, __LINE__);
    } while (0);
    cudaFreeAsync(ws, s);
    if (rc) return rc;
    if (lambda1) *lambda1 = hinfo[0];
    if (iters) *iters = (int)hinfo[1];
    if (herr)
        return set_error(GPGA_ERR_DEGENERATE,
                         "corr_remove_market: a diagonal entry is not positive after the removal");
    return GPGA_OK;
}

int prepare_corr_kernels(int maxsmem)
{
    if (int rc = prepare_corr_tc_kernels(maxsmem)) return rc;
    return raise_smem(market_iter_kernel, maxsmem);
}

} // namespace gpga

