// rmt_tri.cu -- random-matrix cleaning (Sec. 4.2: the eigenvalues in the
// Wishart range are removed in a trace-preserving way) of large correlation
// matrices through a tridiagonal reduction, in place of the cyclic Jacobi of
// rmt.cu, whose n - 1 rounds per sweep each cost a launch at these sizes.
// One matrix at a time, in FP64:
//
//   1. tri_reduce (one cooperative launch): Householder reduction
//      A = Q T Q^T, Q = H_0 H_1 ... H_{N-3}, H_k = I - tau_k u_k u_k^T acting
//      on rows k+1 .. N-1 (u_k(0) = 1). Step k updates the trailing matrix
//      A' <- H_k A' H_k by p = tau A' u, K = tau/2 p^T u, w = p - K u,
//      A' <- A' - u w^T - w u^T. Every CTA forms the reflectors, K and w
//      itself (the same arithmetic in the same order, so the same bits); a
//      warp owns rows; the update of step k and the product A' u_{k+1} of
//      step k+1 share one pass over a row, the matrix and p ping-pong between
//      two buffers, so one grid barrier per step remains.
//   2. tri_bisect: every eigenvalue of T by bisection on the Sturm count
//      (sign changes of the leading principal minors of T - x I, scaled by
//      powers of two), one warp per eigenvalue testing 32 points per round.
//   3. tri_stats: the noise set (eigenvalues in [(1 - sqrt q)^2,
//      (1 + sqrt q)^2]), its mean m; the smaller of the kept set and the noise
//      set is expanded: C' = m I + sum_kept (l - m) v v^T, or equivalently
//      C' = C - sum_noise (l - m) v v^T; eigenvalues closer than 1e-10 ||T||
//      form groups.
//   4. tri_invit: eigenvectors of T for that set by inverse iteration (LU of
//      T - l I with partial pivoting, two solves from a pseudo-random start),
//      members of a group orthogonalised against each other (Gram-Schmidt)
//      after every solve.
//   5. two Newton-Schulz steps Z <- Z - 1/2 (Z Z^T - I) Z restore
//      orthogonality across groups to working precision.
//   6. back-transformation V = Q Z (the reflectors applied in reverse order),
//      C' from V, then the normalisation of rmt.cu.
// No step sums in an order that depends on the launch: the result is
// reproducible run to run.
#include <float.h>
#include <math.h>

#include "gpga_internal.cuh"

namespace gpga {

constexpr int RED_THREADS = 128; // the reduction: 4 warps per CTA, one CTA per SM at most
constexpr int RED_WARPS = RED_THREADS / 32;
constexpr int RED_PREFETCH = 16; // entries per lane of a warp's first row loaded ahead (N <= 513)
constexpr int TRI_INV_ITERS = 2;
constexpr double TRI_GROUP_TOL = 1e-10; // eigenvalues this close (relative to ||T||) form a group
constexpr int TRI_TILE = 32;            // output tile of the small dense products

// grid barrier of a cooperative launch: one counter that only grows; the
// b-th barrier of a launch waits until it reaches b x gridDim.x arrivals.
// Every wait is bounded by `budget` cycles; a CTA that gives up sets `abort`,
// which makes every later barrier return false at once.
struct GridBar {
    unsigned count;
    int abort;
    int pad[2];
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool grid_barrier(GridBar *b, unsigned *target, long long budget)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile int *vab = &b->abort;
        *target += gridDim.x;
        if (*vab) {
            ok = 0;
        } else {
            __threadfence();
            atomicAdd(&b->count, 1u);
            const long long t0 = clock64();
            while (ld_acquire_gpu(&b->count) < *target) {
                if (*vab || clock64() - t0 > budget) {
                    ok = 0;
                    atomicExch(&b->abort, 1);
                    break;
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// sum over the CTA in a fixed order (the butterfly gives every lane the same
// bits; the warps' sums are added in warp order): every thread gets the sum
__device__ double cta_sum(double x, double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if (lane == 0) red[wid] = x;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += red[k];
    return s;
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Householder vector of x[0..n) (n >= 2): u(0) = 1, H x = beta e_1 with
// H = I - tau u u^T, beta = -sign(x0) ||x|| (tau = 0, beta = x0 when x(1..) = 0).
// Every thread of the CTA returns the same tau and beta.
__device__ void householder(const double *x, int n, double *u, double *red, double *tau,
                            double *beta)
{
    double s = 0.0;
    for (int j = 1 + threadIdx.x; j < n; j += blockDim.x) s += x[j] * x[j];
    const double sig2 = cta_sum(s, red);
    const double x0 = x[0];
    if (sig2 == 0.0) {
        *tau = 0.0;
        *beta = x0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) u[j] = j == 0 ? 1.0 : 0.0;
    } else {
        const double mu = sqrt(x0 * x0 + sig2);
        const double bt = x0 >= 0.0 ? -mu : mu;
        const double dn = x0 - bt;             // |dn| >= |bt| > 0
        const double q = 1.0 / (bt * dn);      // one division for both reciprocals
        const double inv = bt * q;             // 1 / (x0 - beta)
        *tau = -dn * (dn * q);                 // (beta - x0) / beta
        *beta = bt;
        for (int j = threadIdx.x; j < n; j += blockDim.x) u[j] = j == 0 ? 1.0 : x[j] * inv;
    }
    __syncthreads();
}

// copy C into the work matrix, flag a non-finite entry (err bit 1)
__global__ void tri_copy_kernel(const double *__restrict__ C, int N, double *__restrict__ A,
                                int *__restrict__ err)
{
    const size_t total = (size_t)N * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const double v = C[i];
        if (!isfinite(v)) atomicOr(err, 1);
        A[i] = v;
    }
}

// Step 1. A0: the matrix (full, row-major, N x N), A1: the second buffer;
// P0, P1: p ping-pong (N); outputs d (N), e (N - 1), tau (N - 2), U (row k
// holds u_k at columns k+1 .. N-1). Needs N >= 3. Dynamic shared memory: 4 N
// doubles. err bit 4: a barrier gave up. At the start of a step every load
// that depends only on the previous step (p, the row of the next reflector,
// the first row a warp updates) is issued at once.
__global__ void __launch_bounds__(RED_THREADS)
    tri_reduce_kernel(double *A0, double *A1, int N, double *P0, double *P1, double *__restrict__ d,
                      double *__restrict__ e, double *__restrict__ tau, double *__restrict__ U,
                      GridBar *bar, long long budget, int *__restrict__ err)
{
    extern __shared__ double sm_tri[];
    double *u = sm_tri, *un = sm_tri + N, *w = sm_tri + 2 * N, *r = sm_tri + 3 * N;
    __shared__ double red[RED_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gw = blockIdx.x * RED_WARPS + wid, GW = gridDim.x * RED_WARPS;
    const bool lead = blockIdx.x == 0;
    double tk, bk;
    // step 0's reflector from row 0, and p = tau_0 A' u_0 for rows 1 .. N-1
    for (int j = tid; j < N - 1; j += blockDim.x) r[j] = A0[j + 1];
    __syncthreads();
    householder(r, N - 1, u, red, &tk, &bk);
    if (lead) {
        if (tid == 0) {
            d[0] = A0[0];
            e[0] = bk;
            tau[0] = tk;
        }
        for (int j = tid; j < N - 1; j += blockDim.x) U[1 + j] = u[j];
    }
    for (int i = 1 + gw; i < N; i += GW) {
        const double *row = A0 + (size_t)i * N + 1;
        double acc = 0.0;
        for (int j = lane; j < N - 1; j += 32) acc += row[j] * u[j];
        acc = warp_sum(acc) * tk;
        if (lane == 0) P0[i] = acc;
    }
    unsigned target = 0; // arrivals the next barrier waits for (thread 0)
    if (!grid_barrier(bar, &target, budget)) {
        if (tid == 0) atomicOr(err, 4);
        return;
    }
    double *cur = A0, *nxt = A1, *Pc = P0, *Pn = P1;
    for (int k = 0; k <= N - 3; ++k) {
        const int n = N - k - 1; // trailing rows / columns k+1 .. N-1 (local 0 .. n-1)
        // loads ahead: the first row this warp updates (if any)
        const int i0 = k + 2 + gw;
        double ra[RED_PREFETCH];
        if (i0 < N) {
            const double *src0 = cur + (size_t)i0 * N + (k + 1);
#pragma unroll
            for (int t = 0; t < RED_PREFETCH; ++t) {
                const int j = 1 + lane + 32 * t;
                ra[t] = j < n ? src0[j] : 0.0;
            }
        }
        // p (into w) and row k+1 (into r), and p^T u
        const double *rk = cur + (size_t)(k + 1) * N + (k + 1);
        double s = 0.0;
        for (int j = tid; j < n; j += blockDim.x) {
            const double p = Pc[k + 1 + j];
            r[j] = rk[j];
            w[j] = p;
            s += p * u[j];
        }
        // w = p - (tau/2)(p^T u) u
        const double K = 0.5 * tk * cta_sum(s, red);
        for (int j = tid; j < n; j += blockDim.x) w[j] -= K * u[j];
        __syncthreads();
        if (k == N - 3) {
            // the last 2 x 2 trailing block after its update
            if (lead && tid == 0) {
                d[N - 2] = r[0] - 2.0 * u[0] * w[0];
                d[N - 1] = cur[(size_t)(N - 1) * N + (N - 1)] - 2.0 * u[1] * w[1];
                e[N - 2] = r[1] - u[0] * w[1] - w[0] * u[1];
            }
            break;
        }
        // row k+1 after the update (local row 0): its diagonal is d_{k+1},
        // the rest the vector of the next reflector
        {
            const double u0 = u[0], w0 = w[0];
            for (int j = tid; j < n; j += blockDim.x) r[j] = r[j] - u0 * w[j] - w0 * u[j];
        }
        __syncthreads();
        double t1, b1;
        householder(r + 1, n - 1, un, red, &t1, &b1);
        if (lead) {
            if (tid == 0) {
                d[k + 1] = r[0];
                e[k + 1] = b1;
                tau[k + 1] = t1;
            }
            double *Ur = U + (size_t)(k + 1) * N + (k + 2);
            for (int j = tid; j < n - 1; j += blockDim.x) Ur[j] = un[j];
        }
        // rows k+2 .. N-1: the update of step k and p of step k+1 in one pass
        bool first = true;
        for (int i = i0; i < N; i += GW, first = false) {
            const int li = i - (k + 1);
            const double ui = u[li], wi = w[li];
            const double *src = cur + (size_t)i * N + (k + 1);
            double *dst = nxt + (size_t)i * N + (k + 1);
            double acc = 0.0;
#pragma unroll
            for (int t = 0; t < RED_PREFETCH; ++t) {
                const int j = 1 + lane + 32 * t;
                if (j < n) {
                    const double a = (first ? ra[t] : src[j]) - ui * w[j] - wi * u[j];
                    dst[j] = a;
                    acc += a * un[j - 1];
                }
            }
            for (int j = 1 + lane + 32 * RED_PREFETCH; j < n; j += 32) {
                const double a = src[j] - ui * w[j] - wi * u[j];
                dst[j] = a;
                acc += a * un[j - 1];
            }
            acc = warp_sum(acc) * t1;
            if (lane == 0) Pn[i] = acc;
        }
        if (!grid_barrier(bar, &target, budget)) {
            if (tid == 0) atomicOr(err, 4);
            return;
        }
        double *t = cur;
        cur = nxt;
        nxt = t;
        t = Pc;
        Pc = Pn;
        Pn = t;
        t = u;
        u = un;
        un = t;
        tk = t1;
    }
}

// Sturm count: the number of eigenvalues of T below x, as the number of sign
// changes in p_0 = 1, p_1, ..., p_N with p_i = (d_i - x) p_{i-1} -
// e_{i-1}^2 p_{i-2}, the leading principal minors of T - x I (Sturm's
// theorem; p_i / p_{i-1} are the LDL^T pivots). A zero p_i is replaced by
// -2^-600 p_{i-1}, a tiny value of the opposite sign (a pivot just below
// zero). Every 8 steps p_i and p_{i-1} are scaled by the same power of two,
// which keeps them near 1 and leaves every sign as it is; sign and exponent
// tests run on the integer pipe. No division: one FMA per step lies on the
// dependency chain.
__device__ __forceinline__ bool dneg(double v) { return __double2hiint(v) < 0; }

__device__ __forceinline__ bool dzero(double v)
{
    return ((unsigned)__double2hiint(v) & 0x7ff00000u) == 0u; // zero or subnormal
}

// 2^-e(v) for the binary exponent e of a normal v (|e| < 1000)
__device__ __forceinline__ double dscale_of(double v)
{
    const int e = ((__double2hiint(v) >> 20) & 0x7ff) - 1023;
    return __hiloint2double((1023 - e) << 20, 0);
}

__device__ __forceinline__ int sturm_count(const double *d, const double *e2, int N, double x)
{
    const double tiny = 0x1p-600;
    double p2 = 1.0, p1 = d[0] - x;
    if (dzero(p1)) p1 = -tiny;
    int c = dneg(p1) ? 1 : 0;
    int i = 1;
    for (; i + 8 <= N; i += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            double p = fma(d[i + q] - x, p1, -(e2[i + q - 1] * p2));
            if (dzero(p)) p = -tiny * p1;
            c += dneg(p) != dneg(p1) ? 1 : 0;
            p2 = p1;
            p1 = p;
        }
        const double sc = dscale_of(p1);
        p1 *= sc;
        p2 *= sc;
    }
    for (; i < N; ++i) {
        double p = fma(d[i] - x, p1, -(e2[i - 1] * p2));
        if (dzero(p)) p = -tiny * p1;
        c += dneg(p) != dneg(p1) ? 1 : 0;
        p2 = p1;
        p1 = p;
    }
    return c;
}

// Step 2. lam[k] = the k-th smallest eigenvalue of T. One warp per
// eigenvalue: its 32 lanes test 32 points per round, which splits the bracket
// [lo, hi] (count(lo) <= k < count(hi)) into 33 parts, until it is below
// 4 eps ||T|| (absolute) or 2 eps |lambda| (about 11 rounds). On this part an
// FP64 warp instruction holds its SM sub-partition's FP64 pipe for ~64
// cycles, whatever the number of active lanes, so one warp per eigenvalue
// (N warps over the 4 x 152 sub-partitions) bounds the time best.
// Dynamic shared memory: 2 N doubles.
constexpr int BIS_THREADS = 128; // one warp per SM sub-partition
constexpr int BIS_WARPS = BIS_THREADS / 32;
__global__ void __launch_bounds__(BIS_THREADS)
    tri_bisect_kernel(const double *__restrict__ d, const double *__restrict__ e, int N,
                      double *__restrict__ lam, double *__restrict__ tnorm_out)
{
    extern __shared__ double sm_bis[];
    double *sd = sm_bis, *se2 = sm_bis + N;
    __shared__ double red_lo[BIS_WARPS], red_hi[BIS_WARPS], red_e[BIS_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double glo = INFINITY, ghi = -INFINITY, emax = 0.0;
    for (int i = tid; i < N; i += blockDim.x) {
        const double di = d[i];
        const double el = i > 0 ? fabs(e[i - 1]) : 0.0, er = i < N - 1 ? fabs(e[i]) : 0.0;
        sd[i] = di;
        if (i < N - 1) {
            se2[i] = e[i] * e[i];
            emax = fmax(emax, se2[i]);
        }
        glo = fmin(glo, di - el - er);
        ghi = fmax(ghi, di + el + er);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
        ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
        emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    if (lane == 0) {
        red_lo[wid] = glo;
        red_hi[wid] = ghi;
        red_e[wid] = emax;
    }
    __syncthreads();
    glo = red_lo[0];
    ghi = red_hi[0];
    emax = red_e[0];
    for (int k = 1; k < BIS_WARPS; ++k) {
        glo = fmin(glo, red_lo[k]);
        ghi = fmax(ghi, red_hi[k]);
        emax = fmax(emax, red_e[k]);
    }
    const double tnorm = fmax(fabs(glo), fabs(ghi));
    const double pivmin = DBL_MIN * fmax(1.0, emax);
    const double atol = 4.0 * DBL_EPSILON * tnorm;
    // widen the Gershgorin bracket so that its ends are strictly outside
    glo -= 2.0 * DBL_EPSILON * tnorm * N + 2.0 * pivmin;
    ghi += 2.0 * DBL_EPSILON * tnorm * N + 2.0 * pivmin;
    if (blockIdx.x == 0 && tid == 0 && tnorm_out) *tnorm_out = tnorm;
    const int k = blockIdx.x * BIS_WARPS + wid;
    if (k >= N) return;
    double lo = glo, hi = ghi;
    for (int round = 0; round < 40; ++round) {
        const double tol = fmax(atol, 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)));
        if (hi - lo <= tol) break;
        const double x = lo + (hi - lo) * ((double)(lane + 1) / 33.0);
        const int c = sturm_count(sd, se2, N, x);
        const unsigned m = __ballot_sync(0xffffffffu, c >= k + 1);
        const int l = m ? __ffs(m) - 1 : 32; // first point with count > k
        const double xl = __shfl_sync(0xffffffffu, x, l < 32 ? l : 31);
        const double xp = __shfl_sync(0xffffffffu, x, l > 0 ? (l < 32 ? l - 1 : 31) : 0);
        if (l == 32) {
            lo = xl;
        } else {
            if (l > 0) lo = xp;
            hi = xl;
        }
    }
    if (lane == 0) lam[k] = 0.5 * (lo + hi);
}

// Step 3 (one CTA). The noise set of lam (inside [mlo, mhi]), its size and
// mean m; the expanded set S (the kept set when it is not larger than the
// noise set, else the noise set) as indices idx[0..K) in ascending order with
// weights w_s (l_s - m for the kept set, m - l_s for the noise set) and the
// groups of S: gfirst[0..ngroups] (members gfirst[g] .. gfirst[g+1]-1).
// info: [0] K, [1] ngroups, [2] 1 if the noise set is expanded (C' = C + ...),
// [3] n_noise. mean_out: m. A set bit 0 or 2 of *errflag (non-finite input,
// reduction timed out) reports an empty noise set, so that C is left as it is.
__global__ void __launch_bounds__(1024)
    tri_stats_kernel(const double *__restrict__ lam, int N, double mlo, double mhi,
                     const double *__restrict__ tnorm_p, const int *__restrict__ errflag,
                     int *__restrict__ idx,
                     double *__restrict__ w, int *__restrict__ gfirst, int *__restrict__ info,
                     double *__restrict__ mean_out, int *__restrict__ ncount)
{
    __shared__ double s_sum[32];
    __shared__ int s_cnt[32];
    __shared__ int s_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    double sum = 0.0;
    int cnt = 0;
    for (int k = tid; k < N; k += blockDim.x) {
        const double l = lam[k];
        if (l >= mlo && l <= mhi) {
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
    int nn = 0;
    for (int q = 0; q < nw; ++q) {
        tot += s_sum[q];
        nn += s_cnt[q];
    }
    // a non-finite input or a reduction that gave up leaves C as it is (an
    // empty noise set and an empty S)
    const bool off = (*errflag & 5) != 0;
    if (off) nn = 0;
    const double m = nn ? tot / (double)nn : 0.0;
    const bool noise_form = (N - nn) > nn;
    const double gtol = TRI_GROUP_TOL * *tnorm_p;
    __syncthreads();
    if (tid == 0) s_base = 0;
    __syncthreads();
    // S in index order (ballot prefix per chunk of blockDim.x indices)
    for (int k0 = 0; k0 < N; k0 += blockDim.x) {
        const int k = k0 + tid;
        bool in = false;
        double l = 0.0;
        if (k < N) {
            l = lam[k];
            const bool noise = l >= mlo && l <= mhi;
            in = !off && (noise_form ? noise : !noise);
        }
        const unsigned bm = __ballot_sync(0xffffffffu, in);
        if (lane == 0) s_cnt[wid] = __popc(bm);
        __syncthreads();
        int off = s_base;
        for (int q = 0; q < wid; ++q) off += s_cnt[q];
        if (in) {
            const int pos = off + __popc(bm & ((1u << lane) - 1u));
            idx[pos] = k;
            w[pos] = noise_form ? m - l : l - m;
        }
        __syncthreads();
        if (tid == 0) {
            int add = 0;
            for (int q = 0; q < nw; ++q) add += s_cnt[q];
            s_base += add;
        }
        __syncthreads();
    }
    const int K = s_base;
    // groups: a member starts one unless it directly follows the previous
    // member in index order with an eigenvalue within gtol
    if (tid == 0) {
        int ng = 0;
        for (int s = 0; s < K; ++s) {
            const bool start = s == 0 || idx[s] != idx[s - 1] + 1 ||
                               lam[idx[s]] - lam[idx[s - 1]] > gtol;
            if (start) gfirst[ng++] = s;
        }
        gfirst[ng] = K;
        info[0] = K;
        info[1] = ng;
        info[2] = noise_form ? 1 : 0;
        info[3] = nn;
        *mean_out = m;
        *ncount = nn;
    }
}

// a pseudo-random start component in [-1, 1) for vector s, entry i (SplitMix64
// finaliser of a counter)
__device__ __forceinline__ double start_component(int s, int i)
{
    unsigned long long z = ((unsigned long long)(unsigned)s << 32 | (unsigned)i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// LU factorisation with partial pivoting of the tridiagonal T - l I (Gaussian
// elimination, rows i and i+1 exchanged when |sub| > |pivot|): on return dd
// (the reciprocals of U's diagonal), du (first superdiagonal), du2 (second,
// from exchanges), dl (multipliers), piv (1 where rows were exchanged); pivots
// below `pert` in magnitude are raised to it first (inverse iteration on a
// shift at an eigenvalue)
__device__ void tri_lu(const double *d, const double *e, int N, double l, double pert, double *dd,
                       double *du, double *du2, double *dl, unsigned char *piv)
{
    for (int i = 0; i < N; ++i) {
        dd[i] = d[i] - l;
        if (i < N - 1) {
            du[i] = e[i];
            dl[i] = e[i];
        }
        du2[i] = 0.0;
    }
    for (int i = 0; i < N - 1; ++i) {
        if (fabs(dd[i]) >= fabs(dl[i])) {
            piv[i] = 0;
            const double f = dd[i] != 0.0 ? dl[i] / dd[i] : 0.0;
            dl[i] = f;
            dd[i + 1] -= f * du[i];
        } else {
            piv[i] = 1;
            const double f = dd[i] / dl[i];
            dd[i] = dl[i];
            dl[i] = f;
            const double t = du[i];
            du[i] = dd[i + 1];
            dd[i + 1] = t - f * dd[i + 1];
            if (i < N - 2) {
                du2[i] = du[i + 1];
                du[i + 1] = -f * du[i + 1];
            }
        }
    }
    for (int i = 0; i < N; ++i) {
        double v = dd[i];
        if (fabs(v) < pert) v = v < 0.0 ? -pert : pert;
        dd[i] = 1.0 / v;
    }
}

// solve (LU) x = b in place with the factors of tri_lu (rd: reciprocal pivots)
__device__ void tri_solve(int N, const double *rd, const double *du, const double *du2,
                          const double *dl, const unsigned char *piv, double *b)
{
    for (int i = 0; i < N - 1; ++i) {
        if (piv[i] == 0) {
            b[i + 1] -= dl[i] * b[i];
        } else {
            const double t = b[i];
            b[i] = b[i + 1];
            b[i + 1] = t - dl[i] * b[i + 1];
        }
    }
    b[N - 1] *= rd[N - 1];
    if (N >= 2) b[N - 2] = (b[N - 2] - du[N - 2] * b[N - 1]) * rd[N - 2];
    for (int i = N - 3; i >= 0; --i) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) * rd[i];
}

// Step 4. One warp per group of S: each member's eigenvector of T by inverse
// iteration, orthogonalised against the members before it after every
// solve; written to row s of Z (K x N). Dynamic shared memory: 5 N doubles +
// N bytes.
__global__ void __launch_bounds__(32)
    tri_invit_kernel(const double *__restrict__ d, const double *__restrict__ e, int N,
                     const double *__restrict__ lam, const int *__restrict__ idx,
                     const int *__restrict__ gfirst, const int *__restrict__ info,
                     const double *__restrict__ tnorm_p, double *__restrict__ Z)
{
    extern __shared__ double sm_inv[];
    const int g = blockIdx.x;
    if (g >= info[1]) return;
    double *dd = sm_inv, *du = sm_inv + N, *du2 = sm_inv + 2 * N, *dl = sm_inv + 3 * N,
           *x = sm_inv + 4 * N;
    unsigned char *piv = reinterpret_cast<unsigned char *>(sm_inv + 5 * N);
    const int lane = threadIdx.x;
    const double pert = DBL_EPSILON * fmax(*tnorm_p, DBL_MIN);
    const int s0 = gfirst[g], s1 = gfirst[g + 1];
    for (int s = s0; s < s1; ++s) {
        const double l = lam[idx[s]];
        if (lane == 0) tri_lu(d, e, N, l, pert, dd, du, du2, dl, piv);
        for (int i = lane; i < N; i += 32) x[i] = start_component(idx[s], i);
        __syncwarp();
        for (int it = 0; it < TRI_INV_ITERS; ++it) {
            if (lane == 0) tri_solve(N, dd, du, du2, dl, piv, x);
            __syncwarp();
            for (int pass = 0; pass < 2; ++pass) {
                // Gram-Schmidt against the group's earlier members, twice
                for (int t = s0; t < s; ++t) {
                    const double *zt = Z + (size_t)t * N;
                    double a = 0.0;
                    for (int i = lane; i < N; i += 32) a += x[i] * zt[i];
                    a = warp_sum(a);
                    for (int i = lane; i < N; i += 32) x[i] -= a * zt[i];
                    __syncwarp();
                }
                double q = 0.0;
                for (int i = lane; i < N; i += 32) q += x[i] * x[i];
                q = warp_sum(q);
                const double inv = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
                for (int i = lane; i < N; i += 32) x[i] *= inv;
                __syncwarp();
                if (s == s0) break;
            }
        }
        double *zs = Z + (size_t)s * N;
        for (int i = lane; i < N; i += 32) zs[i] = x[i];
        __syncwarp();
    }
}

// Step 5a. E = Z Z^T - I (K x K), 16 x 16 tiles of the upper triangle (one
// entry per thread), each written to both triangles
constexpr int NS_TILE = 16;
__global__ void __launch_bounds__(256)
    tri_gram_kernel(const double *__restrict__ Z, int N, const int *__restrict__ info,
                    double *__restrict__ E, int ldE)
{
    __shared__ double sa[NS_TILE][33], sb[NS_TILE][33];
    const int K = info[0];
    if (blockIdx.x < blockIdx.y) return;
    const int a0 = blockIdx.y * NS_TILE, b0 = blockIdx.x * NS_TILE;
    if (a0 >= K || b0 >= K) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc = 0.0;
    for (int i0 = 0; i0 < N; i0 += 32) {
        for (int q = threadIdx.x; q < NS_TILE * 32; q += blockDim.x) {
            const int r = q >> 5, c = q & 31, i = i0 + c;
            sa[r][c] = (a0 + r < K && i < N) ? Z[(size_t)(a0 + r) * N + i] : 0.0;
            sb[r][c] = (b0 + r < K && i < N) ? Z[(size_t)(b0 + r) * N + i] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < 32; ++c) acc += sa[ty][c] * sb[tx][c];
        __syncthreads();
    }
    const int a = a0 + ty, b = b0 + tx;
    if (a < K && b < K) {
        const double v = acc - (a == b ? 1.0 : 0.0);
        E[(size_t)a * ldE + b] = v;
        E[(size_t)b * ldE + a] = v;
    }
}

// Step 5b. Zo = Z - 1/2 E Z (K x N), 16 x 16 tiles, one entry per thread
__global__ void __launch_bounds__(256)
    tri_ns_apply_kernel(const double *__restrict__ Z, int N, const int *__restrict__ info,
                        const double *__restrict__ E, int ldE, double *__restrict__ Zo)
{
    __shared__ double se[NS_TILE][33], sz[32][NS_TILE + 1];
    const int K = info[0];
    const int a0 = blockIdx.y * NS_TILE, i0 = blockIdx.x * NS_TILE;
    if (a0 >= K || i0 >= N) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc = 0.0;
    for (int b0 = 0; b0 < K; b0 += 32) {
        for (int q = threadIdx.x; q < NS_TILE * 32; q += blockDim.x) {
            const int r = q >> 5, c = q & 31;
            se[r][c] = (a0 + r < K && b0 + c < K) ? E[(size_t)(a0 + r) * ldE + b0 + c] : 0.0;
            const int rb = q >> 4, ci = q & 15;
            sz[rb][ci] = (b0 + rb < K && i0 + ci < N) ? Z[(size_t)(b0 + rb) * N + i0 + ci] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < 32; ++c) acc += se[ty][c] * sz[c][tx];
        __syncthreads();
    }
    const int a = a0 + ty, i = i0 + tx;
    if (a < K && i < N) Zo[(size_t)a * N + i] = Z[(size_t)a * N + i] - 0.5 * acc;
}

// Step 6a. V = Q Z in place: H_{N-3} first, H_0 last. One CTA per row of Z
// (the vector, held in shared memory), its elements split over four warps
// (one per SM sub-partition: the FP64 pipe bounds this step); the next
// reflector row is fetched (cp.async) while the current one is applied.
// Dynamic shared memory: 3 N doubles.
constexpr int BACK_THREADS = 128;

__device__ __forceinline__ void cp_async8(double *dst_smem, const double *src)
{
    const uint32_t dsm = (uint32_t)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dsm), "l"(src) : "memory");
}

__global__ void __launch_bounds__(BACK_THREADS)
    tri_back_kernel(double *__restrict__ Z, int N, const int *__restrict__ info,
                    const double *__restrict__ U, const double *__restrict__ tau)
{
    extern __shared__ double sm_back[];
    __shared__ double red[BACK_THREADS / 32];
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31, nt = blockDim.x;
    const int s = blockIdx.x;
    if (s >= info[0]) return;
    double *ub = sm_back; // two reflector rows
    double *z = sm_back + 2 * (size_t)N;
    double *zs = Z + (size_t)s * N;
    for (int i = tid; i < N; i += nt) z[i] = zs[i];
    // entries k+2 .. N-1 of reflector row k into buffer b (u_k(0) = 1 at k+1)
    auto fetch = [&](int k, int b) {
        const double *src = U + (size_t)k * N;
        double *dst = ub + (size_t)b * N;
        for (int j = k + 2 + tid; j < N; j += nt) cp_async8(dst + j, src + j);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    fetch(N - 3, 0);
    int b = 0;
    for (int k = N - 3; k >= 0; --k, b ^= 1) {
        if (k > 0) {
            fetch(k - 1, b ^ 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const double tk = tau[k];
        if (tk != 0.0) {
            const double *uk = ub + (size_t)b * N;
            // thread tid owns the elements j = tid (mod nt) of [k+1, N)
            double a = 0.0;
            for (int j = k + 1 + tid; j < N; j += nt) a += (j == k + 1 ? 1.0 : uk[j]) * z[j];
            a = warp_sum(a);
            if (lane == 0) red[wid] = a;
            __syncthreads();
            a = 0.0;
            for (int q = 0; q < (nt >> 5); ++q) a += red[q];
            a *= tk;
            for (int j = k + 1 + tid; j < N; j += nt) z[j] -= a * (j == k + 1 ? 1.0 : uk[j]);
        }
        // every thread is done with buffer b and red before they are reused
        __syncthreads();
    }
    for (int i = tid; i < N; i += nt) zs[i] = z[i];
}

// Step 6b. Cp = base + sum_s w_s v_s v_s^T, base = C (noise set expanded) or
// m I (kept set), 32 x 32 tiles of the upper triangle (w_s folded into the
// staged j operand: one FMA per term); entries with i <= j are written to
// both triangles, so C' is exactly symmetric. Nothing to do with an empty
// noise set.
__global__ void __launch_bounds__(256)
    tri_rebuild_kernel(const double *__restrict__ V, int N, const int *__restrict__ info,
                       const double *__restrict__ w, const double *__restrict__ mean,
                       const double *__restrict__ C, double *__restrict__ Cp)
{
    __shared__ double si[TRI_TILE][TRI_TILE + 1], sj[TRI_TILE][TRI_TILE + 1];
    if (info[3] == 0 || blockIdx.x < blockIdx.y) return;
    const int K = info[0];
    const bool noise_form = info[2] != 0;
    const int i0 = blockIdx.y * TRI_TILE, j0 = blockIdx.x * TRI_TILE;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int s0 = 0; s0 < K; s0 += TRI_TILE) {
        for (int r = ty; r < TRI_TILE; r += 8) {
            const int s = s0 + r;
            const bool in = s < K;
            si[r][tx] = (in && i0 + tx < N) ? V[(size_t)s * N + i0 + tx] : 0.0;
            sj[r][tx] = (in && j0 + tx < N) ? w[s] * V[(size_t)s * N + j0 + tx] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < TRI_TILE; ++c) {
            const double bj = sj[c][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += si[c][ty + 8 * q] * bj;
        }
        __syncthreads();
    }
    const double m = *mean;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < N && j < N && i <= j) {
            const double base = noise_form ? C[(size_t)i * N + j] : (i == j ? m : 0.0);
            const double v = base + acc[q];
            Cp[(size_t)i * N + j] = v;
            Cp[(size_t)j * N + i] = v;
        }
    }
}

int prepare_rmt_tri_kernels(int maxsmem)
{
    const int need = 4 * GPGA_MAX_N * (int)sizeof(double);
    if (need > maxsmem) return set_error(GPGA_ERR_CUDA, "rmt: %d bytes of shared memory needed", need);
    GPGA_CUDA(cudaFuncSetAttribute((const void *)tri_reduce_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, need));
    GPGA_CUDA(cudaFuncSetAttribute((const void *)tri_bisect_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   2 * GPGA_MAX_N * (int)sizeof(double)));
    GPGA_CUDA(cudaFuncSetAttribute((const void *)tri_invit_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   5 * GPGA_MAX_N * (int)sizeof(double) + GPGA_MAX_N));
    GPGA_CUDA(cudaFuncSetAttribute((const void *)tri_back_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   3 * GPGA_MAX_N * (int)sizeof(double)));
    return GPGA_OK;
}

// the normalisation of rmt.cu (C_ij <- C'_ij / sqrt(C'_ii C'_jj), clamped)
int rmt_normalise(const double *Cp, int B, int N, int n2, const int *ncount, double *C, int *err,
                  cudaStream_t s);

int rmt_clean_tri(double *C, int B, int N, double T, double *eig_sorted, int *n_noise,
                  cudaStream_t s)
{
    if (N < 3) return set_error(GPGA_ERR_ARG, "corr_clean_rmt: N=%d too small for the reduction", N);
    int dev = 0, sms = 0, per_sm = 0;
    GPGA_CUDA(cudaGetDevice(&dev));
    GPGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem_red = 4 * (size_t)N * sizeof(double);
    GPGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tri_reduce_kernel, RED_THREADS,
                                                            smem_red));
    if (per_sm < 1) return set_error(GPGA_ERR_CUDA, "corr_clean_rmt: reduction kernel does not fit");
    int G = (N + RED_WARPS - 1) / RED_WARPS;
    if (G > sms) G = sms; // one CTA per SM at most: all co-resident
    const int Kmax = N / 2 + 1;
    const size_t nn = (size_t)N * N;
    // scratch, 256-byte aligned pieces
    const size_t sizes[] = {nn * 8, nn * 8, nn * 8,                     // A0, A1 (then C'), U
                            (size_t)Kmax * N * 8, (size_t)Kmax * N * 8, // Z, Z2
                            (size_t)Kmax * Kmax * 8,                    // E
                            (size_t)N * 8, (size_t)N * 8,               // P0, P1
                            (size_t)N * 8, (size_t)N * 8, (size_t)N * 8, (size_t)N * 8, // d e tau lam
                            (size_t)N * 4, (size_t)N * 8, (size_t)(N + 2) * 4,          // idx w gfirst
                            8 * 4, 8 * 8, sizeof(GridBar), 4 * sizeof(int)};
    constexpr int NP = sizeof(sizes) / sizeof(sizes[0]);
    size_t bytes = 0;
    for (size_t v : sizes) bytes += (v + 255) & ~(size_t)255;
    char *ws = nullptr;
    GPGA_CUDA(cudaMallocAsync((void **)&ws, bytes, s));
    char *pc[NP];
    {
        size_t off = 0;
        for (int k = 0; k < NP; ++k) {
            pc[k] = ws + off;
            off += (sizes[k] + 255) & ~(size_t)255;
        }
    }
    double *A0 = (double *)pc[0], *A1 = (double *)pc[1], *U = (double *)pc[2];
    double *Z = (double *)pc[3], *Z2 = (double *)pc[4], *E = (double *)pc[5];
    double *P0 = (double *)pc[6], *P1 = (double *)pc[7];
    double *d = (double *)pc[8], *e = (double *)pc[9], *tau = (double *)pc[10],
           *lam = (double *)pc[11];
    int *idx = (int *)pc[12];
    double *wv = (double *)pc[13];
    int *gfirst = (int *)pc[14];
    int *info = (int *)pc[15];
    double *scal = (double *)pc[16]; // [0] mean, [1] ||T||
    GridBar *bar = (GridBar *)pc[17];
    int *flags = (int *)pc[18]; // [0] error bits, [1] noise count
    const double q = (double)N / T, rq = sqrt(q);
    const double mlo = (1.0 - rq) * (1.0 - rq), mhi = (1.0 + rq) * (1.0 + rq);
    const long long budget = wait_budget();
    int rc = GPGA_OK, hflags = 0;
    for (int z = 0; z < B && !rc; ++z) {
        double *Cz = C + (size_t)z * nn;
        cudaError_t ce = cudaMemsetAsync(flags, 0, 4 * sizeof(int), s);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(U, 0, nn * sizeof(double), s);
        if (ce != cudaSuccess) {
            rc = cuda_error(ce, "corr_clean_rmt: memset", __FILE__, __LINE__);
            break;
        }
        {
            int blocks = (int)((nn + 255) / 256);
            if (blocks > 1024) blocks = 1024;
            tri_copy_kernel<<<blocks, 256, 0, s>>>(Cz, N, A0, flags);
        }
        {
            int Nv = N;
            long long bv = budget;
            void *args[] = {&A0, &A1, &Nv, &P0, &P1, &d, &e, &tau, &U, &bar, &bv, &flags};
            ce = cudaLaunchCooperativeKernel((const void *)tri_reduce_kernel, dim3(G),
                                             dim3(RED_THREADS), args, smem_red, s);
            if (ce != cudaSuccess) {
                rc = cuda_error(ce, "corr_clean_rmt: reduction launch", __FILE__, __LINE__);
                break;
            }
        }
        tri_bisect_kernel<<<(N + BIS_WARPS - 1) / BIS_WARPS, BIS_THREADS,
                            2 * (size_t)N * sizeof(double), s>>>(d, e, N, lam, scal + 1);
        tri_stats_kernel<<<1, 1024, 0, s>>>(lam, N, mlo, mhi, scal + 1, flags, idx, wv, gfirst,
                                            info, scal, flags + 1);
        tri_invit_kernel<<<Kmax, 32, 5 * (size_t)N * sizeof(double) + N, s>>>(
            d, e, N, lam, idx, gfirst, info, scal + 1, Z);
        const int kt = (Kmax + NS_TILE - 1) / NS_TILE, it16 = (N + NS_TILE - 1) / NS_TILE;
        const int nt = (N + TRI_TILE - 1) / TRI_TILE;
        for (int it = 0; it < 2; ++it) {
            double *zin = it ? Z2 : Z, *zout = it ? Z : Z2;
            tri_gram_kernel<<<dim3(kt, kt), 256, 0, s>>>(zin, N, info, E, Kmax);
            tri_ns_apply_kernel<<<dim3(it16, kt), 256, 0, s>>>(zin, N, info, E, Kmax, zout);
        }
        tri_back_kernel<<<Kmax, BACK_THREADS, 3 * (size_t)N * sizeof(double), s>>>(Z, N, info, U,
                                                                                 tau);
        tri_rebuild_kernel<<<dim3(nt, nt), 256, 0, s>>>(Z, N, info, wv, scal, Cz, A1);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) {
            rc = cuda_error(ce, "corr_clean_rmt: kernels", __FILE__, __LINE__);
            break;
        }
        if ((rc = rmt_normalise(A1, 1, N, N, flags + 1, Cz, flags, s))) break;
        if (eig_sorted) {
            ce = cudaMemcpyAsync(eig_sorted + (size_t)z * N, lam, (size_t)N * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s);
            if (ce != cudaSuccess) {
                rc = cuda_error(ce, "corr_clean_rmt: eigenvalues", __FILE__, __LINE__);
                break;
            }
        }
        int hf[2] = {0, 0};
        ce = cudaMemcpyAsync(hf, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
            rc = cuda_error(ce, "corr_clean_rmt", __FILE__, __LINE__);
            break;
        }
        hflags |= hf[0];
        if (n_noise) n_noise[z] = hf[1];
        if (hf[0] & 1)
            rc = set_error(GPGA_ERR_ARG, "corr_clean_rmt: non-finite entry in C");
        else if (hf[0] & 4)
            rc = set_error(GPGA_ERR_TIMEOUT, "corr_clean_rmt: a bounded device wait gave up");
        else if (hf[0] & 2)
            rc = set_error(GPGA_ERR_DEGENERATE,
                           "corr_clean_rmt: a diagonal entry is not positive after the cleaning");
    }
    cudaFreeAsync(ws, s);
    return rc;
}

} // namespace gpga
