// corr.cu -- Pearson correlation prelude, Eq. 7 (Sec. 2.1; the standardisation
// below Eq. 2): C_ij = <z_i, z_j> / sqrt(|z_i|^2 |z_j|^2), z = R - column mean.
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
static constexpr int T_SLAB = 512;              // rows per column-stat CTA

__global__ void colsum_kernel(const double *__restrict__ R, int T, int N, int ld,
                              const double *__restrict__ mean, double *__restrict__ part)
{
    __shared__ double red[CS_ROWS][CS_COLS + 1];
    const int cx = threadIdx.x, ry = threadIdx.y;
    const int j = blockIdx.x * CS_COLS + cx;
    const int t0 = blockIdx.y * T_SLAB;
    const int t1 = min(T, t0 + T_SLAB);
    double s = 0.0;
    if (j < N) {
        const double mu = mean ? mean[j] : 0.0;
        for (int t = t0 + ry; t < t1; t += CS_ROWS) {
            const double v = R[(size_t)t * ld + j] - mu;
            s += mean ? v * v : v;
        }
    }
    red[ry][cx] = s;
    __syncthreads();
    if (ry == 0 && j < N) {
        double a = 0.0;
        for (int r = 0; r < CS_ROWS; ++r) a += red[r][cx];
        part[(size_t)blockIdx.y * N + j] = a;
    }
}

__global__ void colfinal_kernel(const double *__restrict__ part, int nslab, int T, int N,
                                double *__restrict__ out, int mode, int *__restrict__ err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double a = 0.0;
    for (int k = 0; k < nslab; ++k) a += part[(size_t)k * N + j];
    if (mode == 0) { // means
        if (!isfinite(a)) atomicOr(err, 2);
        out[j] = a / (double)T;
    } else { // 1 / sqrt(q)
        if (!(a > 0.0) || !isfinite(a)) {
            atomicOr(err, 2);
            out[j] = 0.0;
        } else {
            out[j] = 1.0 / sqrt(a);
        }
    }
}

__global__ void normalise_kernel(const double *__restrict__ R, int T, int N, int ld, int Np,
                                 const double *__restrict__ mean, const double *__restrict__ inv,
                                 float *__restrict__ Z)
{
    const size_t total = (size_t)T * Np;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(idx / Np), j = (int)(idx - (size_t)t * Np);
        float z = 0.f;
        if (j < N) z = (float)((R[(size_t)t * ld + j] - mean[j]) * inv[j]);
        Z[idx] = z;
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
    __shared__ float As[GK][GT];
    __shared__ float Bs[GK][GT];
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
    for (int ts = t0; ts < t1; ts += SUB) {
        const int te = min(t1, ts + SUB);
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int t = ts; t < te; t += GK) {
            // 16 rows x 64 columns of each operand: 1024 floats, 4 per thread
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int e = threadIdx.x + 256 * r;
                const int kk = e >> 6, c = e & 63;
                const int tt = t + kk;
                As[kk][c] = tt < te ? Z[(size_t)tt * Np + bi * GT + c] : 0.f;
                Bs[kk][c] = tt < te ? Z[(size_t)tt * Np + bj * GT + c] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < GK; ++kk) {
                float a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = As[kk][ty * 4 + q];
                    b[q] = Bs[kk][tx * 4 + q];
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
            }
            __syncthreads();
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

__global__ void gram_final_kernel(const double *__restrict__ part, int nslab, int ntiles, int nb,
                                  int N, double *__restrict__ C)
{
    int tile = blockIdx.x, bi = 0;
    while (tile >= nb - bi) {
        tile -= nb - bi;
        ++bi;
    }
    const int bj = bi + tile;
    for (int e = threadIdx.x; e < GT * GT; e += blockDim.x) {
        const int r = e / GT, c = e - r * GT;
        const int i = bi * GT + r, j = bj * GT + c;
        if (i >= N || j >= N || (bi == bj && j < i)) continue;
        double a = 0.0;
        for (int k = 0; k < nslab; ++k) a += part[((size_t)k * ntiles + blockIdx.x) * (GT * GT) + e];
        if (i == j) a = 1.0;
        if (a > 1.0) a = 1.0;
        if (a < -1.0) a = -1.0;
        C[(size_t)i * N + j] = a;
        C[(size_t)j * N + i] = a;
    }
}

int corr_run(const double *R, int T, int N, int ld, double *C, cudaStream_t s)
{
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
    const size_t total = b_part + 2 * b_vec + b_z + b_g + 256;
    char *ws = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&ws, total, s));
    double *part = (double *)ws;
    double *mean = (double *)(ws + b_part);
    double *inv = mean + N;
    float *Z = (float *)(ws + b_part + 2 * b_vec);
    double *gpart = (double *)(ws + b_part + 2 * b_vec + b_z);
    int *err = (int *)(ws + total - 256);
    int rc = GPGA_OK;
    int herr = 0;
    do {
        if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
            rc = set_error(GPGA_ERR_CUDA, "cluster_corr: memset failed");
            break;
        }
        dim3 cgrid((N + CS_COLS - 1) / CS_COLS, nslab_c), cblock(CS_COLS, CS_ROWS);
        colsum_kernel<<<cgrid, cblock, 0, s>>>(R, T, N, ld, nullptr, part);
        colfinal_kernel<<<(N + 255) / 256, 256, 0, s>>>(part, nslab_c, T, N, mean, 0, err);
        colsum_kernel<<<cgrid, cblock, 0, s>>>(R, T, N, ld, mean, part);
        colfinal_kernel<<<(N + 255) / 256, 256, 0, s>>>(part, nslab_c, T, N, inv, 1, err);
        const size_t zt = (size_t)T * Np;
        int zb = (int)((zt + 255) / 256);
        if (zb > 8192) zb = 8192;
        normalise_kernel<<<zb, 256, 0, s>>>(R, T, N, ld, Np, mean, inv, Z);
        gram_kernel<<<dim3(ntiles, nsplit), 256, 0, s>>>(Z, T, Np, nb, trange, gpart, ntiles);
        gram_final_kernel<<<ntiles, 256, 0, s>>>(gpart, nsplit, ntiles, nb, N, C);
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

} // namespace gpga
