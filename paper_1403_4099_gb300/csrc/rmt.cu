// rmt.cu -- random-matrix cleaning of correlation matrices upstream of the
// clustering (Sec. 4.2: the eigenvalues in the Wishart range are removed in a
// trace-preserving way), batched over independent matrices.
//
// Eigen-decomposition by the parallel cyclic Jacobi method in FP64: the n2
// (= N rounded up to even) indices are paired by the round-robin schedule, so
// each of the n2 - 1 rounds of a sweep applies n2 / 2 disjoint rotations at
// once, A <- J^T A J, V <- V J. A round reads A from one buffer and writes the
// other, so every CTA computes the rotations it needs from a stable A. A padding
// index (odd N) has a zero row and column and is never rotated. Sweeps run until
// the largest off-diagonal entry is below 1e-14 of ||A||_F.
//
// Cleaning: the eigenvalues inside [(1 - sqrt q)^2, (1 + sqrt q)^2], q = N / T,
// are the noise set, replaced by their mean m:
//   C' = m I + sum_{k kept} (lambda_k - m) v_k v_k^T,
// then C''_ij = C'_ij / sqrt(C'_ii C'_jj), clamped to [-1, 1], unit diagonal.
// With an empty noise set the matrix is left as it is.
#include <math.h>

#include "gpga_internal.cuh"

namespace gpga {

constexpr int JT = 16;               // rotation pairs per tile side (32 x 32 entries)
constexpr int JACOBI_MAX_SWEEPS = 40;
constexpr double JACOBI_TOL = 1e-14; // max |a_ij| (i != j) <= tol ||A||_F

// pair k of round r of the round-robin schedule over n2 indices (m = n2 - 1
// odd): pair 0 = (r, m), pair k = ((r + k) mod m, (r - k) mod m); every pair of
// indices meets once in the m rounds of a sweep. Returns p < q.
__device__ __forceinline__ void rr_pair(int r, int k, int m, int &p, int &q)
{
    int a, b;
    if (k == 0) {
        a = r;
        b = m;
    } else {
        a = (r + k) % m;
        b = (r - k + m) % m;
    }
    p = min(a, b);
    q = max(a, b);
}

struct JRot {
    int p, q;
    double c, s, t;
};

// the rotation that zeroes a_pq (Golub and Van Loan's symmetric 2 x 2 Schur
// step): theta = (a_qq - a_pp) / (2 a_pq), t = sign(theta) / (|theta| +
// sqrt(1 + theta^2)), c = 1 / sqrt(1 + t^2), s = t c; the identity if a_pq = 0
__device__ __forceinline__ JRot jacobi_rotation(const double *A, int n2, int r, int k)
{
    JRot o;
    rr_pair(r, k, n2 - 1, o.p, o.q);
    const double apq = A[(size_t)o.p * n2 + o.q];
    o.c = 1.0;
    o.s = 0.0;
    o.t = 0.0;
    if (apq != 0.0) {
        const double app = A[(size_t)o.p * n2 + o.p], aqq = A[(size_t)o.q * n2 + o.q];
        const double theta = (aqq - app) / (2.0 * apq);
        double t;
        if (fabs(theta) > 1e150)
            t = 0.5 / theta; // theta^2 would overflow; t -> 1 / (2 theta)
        else
            t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
        o.c = 1.0 / sqrt(1.0 + t * t);
        o.s = t * o.c;
        o.t = t;
    }
    return o;
}

// One round (or, for a matrix that one tile covers, rounds r0 .. r0 + nr - 1
// with the CTA alone on it) of every matrix z = blockIdx.z. CTA (x, y) owns the
// pair-blocks (a, b), a in tile x, b in tile y, a <= b (writing both (a, b) and
// its transpose), and the rows 32 x .. 32 x + 31 of V for the column pairs of
// tile y. A0 / A1 alternate as source and destination round by round.
__global__ void __launch_bounds__(256)
    jacobi_round_kernel(double *A0, double *A1, double *__restrict__ V, int n2, int r0, int nr)
{
    __shared__ int sp[2][JT], sq[2][JT];
    __shared__ double sc[2][JT], ss[2][JT], st[2][JT];
    const int h = n2 >> 1, m = n2 - 1;
    const int tx = blockIdx.x, ty = blockIdx.y, tid = threadIdx.x;
    const size_t stride = (size_t)n2 * n2;
    double *Vz = V + blockIdx.z * stride;
    for (int u = 0; u < nr; ++u) {
        const int r = (r0 + u) % m;
        const bool odd = ((r0 + u) & 1) != 0;
        const double *A = (odd ? A1 : A0) + blockIdx.z * stride;
        double *B = (odd ? A0 : A1) + blockIdx.z * stride;
        if (tid < 2 * JT) {
            const int side = tid / JT, j = tid - side * JT;
            const int k = (side ? ty : tx) * JT + j;
            if (k < h) {
                const JRot o = jacobi_rotation(A, n2, r, k);
                sp[side][j] = o.p;
                sq[side][j] = o.q;
                sc[side][j] = o.c;
                ss[side][j] = o.s;
                st[side][j] = o.t;
            }
        }
        __syncthreads();
        {
            const int ia = tid / JT, ib = tid - (tid / JT) * JT;
            const int a = tx * JT + ia, b = ty * JT + ib;
            if (a < h && b < h && a <= b) {
                const int p = sp[0][ia], q = sq[0][ia];
                if (a == b) {
                    // the rotated 2 x 2 diagonal block: a_pq -> 0 exactly
                    const double apq = A[(size_t)p * n2 + q], t = st[0][ia];
                    B[(size_t)p * n2 + p] = A[(size_t)p * n2 + p] - t * apq;
                    B[(size_t)q * n2 + q] = A[(size_t)q * n2 + q] + t * apq;
                    B[(size_t)p * n2 + q] = 0.0;
                    B[(size_t)q * n2 + p] = 0.0;
                } else {
                    const int p2 = sp[1][ib], q2 = sq[1][ib];
                    const double c = sc[0][ia], s = ss[0][ia], c2 = sc[1][ib], s2 = ss[1][ib];
                    const double x00 = A[(size_t)p * n2 + p2], x01 = A[(size_t)p * n2 + q2];
                    const double x10 = A[(size_t)q * n2 + p2], x11 = A[(size_t)q * n2 + q2];
                    // rows p, q by (c, s), then columns p2, q2 by (c2, s2)
                    const double y00 = c * x00 - s * x10, y01 = c * x01 - s * x11;
                    const double y10 = s * x00 + c * x10, y11 = s * x01 + c * x11;
                    const double z00 = c2 * y00 - s2 * y01, z01 = s2 * y00 + c2 * y01;
                    const double z10 = c2 * y10 - s2 * y11, z11 = s2 * y10 + c2 * y11;
                    B[(size_t)p * n2 + p2] = z00;
                    B[(size_t)p * n2 + q2] = z01;
                    B[(size_t)q * n2 + p2] = z10;
                    B[(size_t)q * n2 + q2] = z11;
                    B[(size_t)p2 * n2 + p] = z00;
                    B[(size_t)q2 * n2 + p] = z01;
                    B[(size_t)p2 * n2 + q] = z10;
                    B[(size_t)q2 * n2 + q] = z11;
                }
            }
        }
        // V <- V J on rows 32 tx .. 32 tx + 31, column pairs of tile y
        for (int w = tid; w < 2 * JT * JT; w += blockDim.x) {
            const int i = tx * 2 * JT + w / JT, jb = w - (w / JT) * JT;
            const int b = ty * JT + jb;
            if (i < n2 && b < h) {
                double *row = Vz + (size_t)i * n2;
                const int p2 = sp[1][jb], q2 = sq[1][jb];
                const double c2 = sc[1][jb], s2 = ss[1][jb];
                const double v0 = row[p2], v1 = row[q2];
                row[p2] = c2 * v0 - s2 * v1;
                row[q2] = s2 * v0 + c2 * v1;
            }
        }
        __syncthreads(); // (single-tile rounds: this round's writes before the next round's reads)
    }
}

// A0 <- C (N x N, padded to n2 with zeros), V <- I; err bit 1 on a
// non-finite entry
__global__ void jacobi_init_kernel(const double *__restrict__ C, int N, int n2,
                                   double *__restrict__ A0, double *__restrict__ V,
                                   int *__restrict__ err)
{
    const size_t stride = (size_t)n2 * n2;
    const double *Cz = C + blockIdx.y * (size_t)N * N;
    double *Az = A0 + blockIdx.y * stride, *Vz = V + blockIdx.y * stride;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < stride;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n2), j = (int)(idx - (size_t)i * n2);
        double a = 0.0;
        if (i < N && j < N) {
            a = Cz[(size_t)i * N + j];
            if (!isfinite(a)) {
                atomicOr(err, 1);
                a = 0.0;
            }
        }
        Az[idx] = a;
        Vz[idx] = i == j ? 1.0 : 0.0;
    }
}

// per matrix (one CTA): largest |a_ij|, i != j, against tol ||A||_F;
// *unconverged += 1 if above
__global__ void __launch_bounds__(256)
    jacobi_check_kernel(const double *__restrict__ A, int n2, int *__restrict__ unconverged)
{
    __shared__ double s_off[8], s_fro[8];
    const double *Az = A + blockIdx.x * (size_t)n2 * n2;
    double off = 0.0, fro = 0.0;
    const size_t total = (size_t)n2 * n2;
    for (size_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const double a = Az[idx];
        const int i = (int)(idx / n2), j = (int)(idx - (size_t)i * n2);
        fro += a * a;
        if (i != j) off = fmax(off, fabs(a));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
        fro += __shfl_xor_sync(0xffffffffu, fro, o);
    }
    if (lane == 0) {
        s_off[wid] = off;
        s_fro[wid] = fro;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mo = 0.0, f = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            mo = fmax(mo, s_off[k]);
            f += s_fro[k];
        }
        if (!(mo <= JACOBI_TOL * sqrt(f))) atomicAdd(unconverged, 1);
    }
}

// per matrix (one CTA): eigenvalues lambda_k = a_kk (k < N), the noise set
// inside [lo, hi], its mean m, the kept list (index, lambda_k - m) in index
// order, the eigenvalues in ascending order (rank by counting), the noise
// count. Fixed-order reductions.
__global__ void __launch_bounds__(256)
    rmt_stats_kernel(const double *__restrict__ A, int N, int n2, double lo, double hi,
                     int *__restrict__ kidx, double *__restrict__ kw, int *__restrict__ kcount,
                     int *__restrict__ ncount, double *__restrict__ mean,
                     double *__restrict__ eig_sorted)
{
    __shared__ double s_sum[8];
    __shared__ int s_cnt[8];
    __shared__ int s_base;
    const int z = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = blockDim.x >> 5;
    const double *Az = A + z * (size_t)n2 * n2;
    double sum = 0.0;
    int cnt = 0;
    for (int k = tid; k < N; k += blockDim.x) {
        const double l = Az[(size_t)k * n2 + k];
        if (l >= lo && l <= hi) {
            sum += l;
            ++cnt;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        s_sum[wid] = sum;
        s_cnt[wid] = cnt;
    }
    __syncthreads();
    double tot = 0.0;
    int n_noise = 0;
    for (int k = 0; k < nw; ++k) {
        tot += s_sum[k];
        n_noise += s_cnt[k];
    }
    const double mval = n_noise ? tot / (double)n_noise : 0.0;
    // kept list in index order: chunks of blockDim.x indices, ballot prefix
    if (tid == 0) s_base = 0;
    __syncthreads();
    int *kz = kidx + (size_t)z * n2;
    double *wz = kw + (size_t)z * n2;
    for (int k0 = 0; k0 < N; k0 += blockDim.x) {
        const int k = k0 + tid;
        double l = 0.0;
        bool keep = false;
        if (k < N) {
            l = Az[(size_t)k * n2 + k];
            keep = !(l >= lo && l <= hi);
        }
        const unsigned bm = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_cnt[wid] = __popc(bm);
        __syncthreads();
        int off = s_base;
        for (int q = 0; q < wid; ++q) off += s_cnt[q];
        if (keep) {
            const int pos = off + __popc(bm & ((1u << lane) - 1u));
            kz[pos] = k;
            wz[pos] = l - mval;
        }
        __syncthreads();
        if (tid == 0) {
            int add = 0;
            for (int q = 0; q < nw; ++q) add += s_cnt[q];
            s_base += add;
        }
        __syncthreads();
    }
    if (eig_sorted) {
        double *ez = eig_sorted + (size_t)z * N;
        for (int k = tid; k < N; k += blockDim.x) {
            const double l = Az[(size_t)k * n2 + k];
            int rk = 0;
            for (int j = 0; j < N; ++j) {
                const double x = Az[(size_t)j * n2 + j];
                rk += (x < l || (x == l && j < k)) ? 1 : 0;
            }
            ez[rk] = l;
        }
    }
    if (tid == 0) {
        kcount[z] = s_base;
        ncount[z] = n_noise;
        mean[z] = mval;
    }
}

// C'_ij = m delta_ij + sum over the kept list of w_k (V_ik V_jk), into Cp
// (n2 stride), one entry per thread; tiles (x, y), matrix z
__global__ void __launch_bounds__(256)
    rmt_rebuild_kernel(const double *__restrict__ V, int N, int n2, const int *__restrict__ kidx,
                       const double *__restrict__ kw, const int *__restrict__ kcount,
                       const int *__restrict__ ncount, const double *__restrict__ mean,
                       double *__restrict__ Cp)
{
    const int z = blockIdx.z;
    if (ncount[z] == 0) return;
    const int i = blockIdx.y * 16 + (threadIdx.x >> 4), j = blockIdx.x * 16 + (threadIdx.x & 15);
    if (i >= N || j >= N) return;
    const size_t stride = (size_t)n2 * n2;
    const double *Vz = V + z * stride;
    const int *kz = kidx + (size_t)z * n2;
    const double *wz = kw + (size_t)z * n2;
    const int K = kcount[z];
    double acc = 0.0;
    for (int u = 0; u < K; ++u) {
        const int k = kz[u];
        acc += wz[u] * (Vz[(size_t)i * n2 + k] * Vz[(size_t)j * n2 + k]);
    }
    if (i == j) acc += mean[z];
    Cp[z * stride + (size_t)i * n2 + j] = acc;
}

// C_ij <- C'_ij / sqrt(C'_ii C'_jj), clamped, unit diagonal (matrices with an
// empty noise set untouched); err bit 2 on a non-positive C'_ii
__global__ void rmt_normalise_kernel(const double *__restrict__ Cp, int N, int n2,
                                     const int *__restrict__ ncount, double *__restrict__ C,
                                     int *__restrict__ err)
{
    const int z = blockIdx.y;
    if (ncount[z] == 0) return;
    const size_t stride = (size_t)n2 * n2;
    const double *Pz = Cp + z * stride;
    double *Cz = C + z * (size_t)N * N;
    const size_t total = (size_t)N * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / N), j = (int)(idx - (size_t)i * N);
        const double di = Pz[(size_t)i * n2 + i], dj = Pz[(size_t)j * n2 + j];
        double c = 1.0;
        if (!(di > 0.0) || !(dj > 0.0)) {
            atomicOr(err, 2);
        } else if (i != j) {
            c = Pz[(size_t)i * n2 + j] / sqrt(di * dj);
            if (c > 1.0) c = 1.0;
            if (c < -1.0) c = -1.0;
        }
        Cz[idx] = c;
    }
}

int rmt_normalise(const double *Cp, int B, int N, int n2, const int *ncount, double *C, int *err,
                  cudaStream_t s)
{
    int blocks = (int)(((size_t)N * N + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    rmt_normalise_kernel<<<dim3(blocks, B), 256, 0, s>>>(Cp, N, n2, ncount, C, err);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

// the Jacobi rounds of a sweep cost a launch each once a matrix spans more
// than one 32 x 32 tile; from there a few matrices go through the tridiagonal
// reduction of rmt_tri.cu (one matrix at a time), large batches stay here
static bool use_tridiagonal(int B, int N) { return N > 2 * JT && (N >= 128 || B <= 4); }

int rmt_clean(double *C, int B, int N, double T, double *eig_sorted, int *n_noise, int *sweeps,
              cudaStream_t s)
{
    if (use_tridiagonal(B, N)) {
        if (sweeps) *sweeps = 0;
        return rmt_clean_tri(C, B, N, T, eig_sorted, n_noise, s);
    }
    const int n2 = (N + 1) & ~1, h = n2 >> 1, tiles = (h + JT - 1) / JT;
    const size_t stride = (size_t)n2 * n2;
    const size_t mat = (size_t)B * stride * sizeof(double);
    const size_t vec = (size_t)B * n2;
    // the scratch, carved in 256-byte aligned pieces; the sizes are summed with
    // the same rounding the carving applies
    const size_t sizes[9] = {mat, mat, mat, vec * sizeof(int), vec * sizeof(double),
                             (size_t)B * sizeof(int), (size_t)B * sizeof(int),
                             (size_t)B * sizeof(double), 2 * sizeof(int)};
    size_t bytes = 0;
    for (size_t n : sizes) bytes += (n + 255) & ~(size_t)255;
    char *ws = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&ws, bytes, s));
    char *piece[9];
    {
        size_t off = 0;
        for (int k = 0; k < 9; ++k) {
            piece[k] = ws + off;
            off += (sizes[k] + 255) & ~(size_t)255;
        }
    }
    double *A0 = (double *)piece[0], *A1 = (double *)piece[1], *V = (double *)piece[2];
    int *kidx = (int *)piece[3];
    double *kw = (double *)piece[4];
    int *kcount = (int *)piece[5];
    int *ncount = (int *)piece[6];
    double *mean = (double *)piece[7];
    int *flags = (int *)piece[8]; // [0] error bits, [1] unconverged matrices
    const double q = (double)N / T, rq = sqrt(q);
    const double lo = (1.0 - rq) * (1.0 - rq), hi = (1.0 + rq) * (1.0 + rq);
    int rc = GPGA_OK, hflags[2] = {0, 0}, sw = 0;
    do {
        if (cudaMemsetAsync(flags, 0, 2 * sizeof(int), s) != cudaSuccess) {
            rc = set_error(GPGA_ERR_CUDA, "corr_clean_rmt: memset failed");
            break;
        }
        {
            int blocks = (int)((stride + 255) / 256);
            if (blocks > 1024) blocks = 1024;
            jacobi_init_kernel<<<dim3(blocks, B), 256, 0, s>>>(C, N, n2, A0, V, flags);
        }
        const int m = n2 - 1;
        // a sweep is m rounds (odd), so the current buffer alternates sweep by sweep
        for (sw = 0; sw < JACOBI_MAX_SWEEPS; ++sw) {
            const int rbase = sw * m; // round index parity selects the source buffer
            if (tiles == 1) {
                jacobi_round_kernel<<<dim3(1, 1, B), 256, 0, s>>>(A0, A1, V, n2, rbase, m);
            } else {
                for (int r = 0; r < m; ++r)
                    jacobi_round_kernel<<<dim3(tiles, tiles, B), 256, 0, s>>>(A0, A1, V, n2,
                                                                              rbase + r, 1);
            }
            const double *Acur = ((rbase + m) & 1) ? A1 : A0;
            cudaError_t e = cudaMemsetAsync(flags + 1, 0, sizeof(int), s);
            if (e == cudaSuccess) {
                jacobi_check_kernel<<<B, 256, 0, s>>>(Acur, n2, flags + 1);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                rc = cuda_error(e, "corr_clean_rmt: Jacobi sweep", __FILE__, __LINE__);
                break;
            }
            if (hflags[0] || hflags[1] == 0) {
                ++sw;
                break;
            }
        }
        if (rc) break;
        if (hflags[0] & 1) {
            rc = set_error(GPGA_ERR_ARG, "corr_clean_rmt: non-finite entry in C");
            break;
        }
        if (hflags[1]) {
            rc = set_error(GPGA_ERR_DEGENERATE,
                           "corr_clean_rmt: Jacobi did not converge in %d sweeps (%d matrices)",
                           JACOBI_MAX_SWEEPS, hflags[1]);
            break;
        }
        // after sw sweeps of m rounds the eigenvalues sit in the buffer the last round wrote
        const bool in_a1 = ((sw * m) & 1) != 0;
        const double *Aev = in_a1 ? A1 : A0;
        double *Cp = in_a1 ? A0 : A1; // the free buffer holds C'
        rmt_stats_kernel<<<B, 256, 0, s>>>(Aev, N, n2, lo, hi, kidx, kw, kcount, ncount, mean,
                                          eig_sorted);
        const int t16 = (N + 15) / 16;
        rmt_rebuild_kernel<<<dim3(t16, t16, B), 256, 0, s>>>(V, N, n2, kidx, kw, kcount, ncount,
                                                             mean, Cp);
        {
            int blocks = (int)(((size_t)N * N + 255) / 256);
            if (blocks > 1024) blocks = 1024;
            rmt_normalise_kernel<<<dim3(blocks, B), 256, 0, s>>>(Cp, N, n2, ncount, C, flags);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && n_noise)
            e = cudaMemcpyAsync(n_noise, ncount, (size_t)B * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "corr_clean_rmt", __FILE__, __LINE__);
            break;
        }
        if (hflags[0] & 2)
            rc = set_error(GPGA_ERR_DEGENERATE,
                           "corr_clean_rmt: a diagonal entry is not positive after the cleaning");
    } while (0);
    cudaFreeAsync(ws, s);
    if (sweeps) *sweeps = sw;
    return rc;
}

} // namespace gpga
