// init.cu -- correlation-threshold initial population (reading of "create
// initial population", Algorithm 1, which the paper leaves to a thesis).
//
// Individual p starts as the connected components of the graph
// {(i, j) : C_ij > tau_p}, tau_p = tau_lo + (tau_hi - tau_lo) u_p / 2^32 with u_p
// word 0 of Philox(0, p, 0, TAU): single-linkage cuts of C at a spread of levels,
// which the GA then refines. Components of {C > tau} equal those of the maximum
// spanning tree's edges above tau, so the tree is built once (Prim, one CTA) and
// each individual needs one O(N) pass:
//   vertices in Prim order v_0 = 0, v_1, ...; vertex v_k joined the tree through
//   edge (from_k, v_k) of weight w_k; label(v_0) = v_0 and
//   label(v_k) = w_k > tau ? label(from_k) : v_k.
// Prim's rule: the next vertex has the largest key (ties to the lower index);
// a key improves only on a strictly larger C. The comparisons are those of
// FP64 values, made exactly on order-preserving integer images.
#include <math.h>

#include "gpga_internal.cuh"

namespace gpga {

static constexpr uint32_t STREAM_TAU = 4u;

// Order-preserving integer image of an FP64 value, so that Prim's
// comparisons run on the integer pipe (an FP64 instruction holds the FP64 pipe
// for tens of cycles whatever its active lanes): for non-NaN a and b,
// a > b iff prim_key(a) > prim_key(b) and a == b iff the keys are equal
// (-0 and +0 share a key). NaN takes the key of -inf. Every key is above 0.
__device__ __forceinline__ unsigned long long prim_key(double x)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    if (mag > 0x7ff0000000000000ull) b = 0xfff0000000000000ull; // NaN -> -inf
    else if (mag == 0ull) b = 0ull;                            // -0 -> +0
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// larger key first, ties to the lower vertex
__device__ __forceinline__ void prim_max(unsigned long long &bk, int &bi, unsigned long long k, int i)
{
    if (k > bk || (k == bk && i < bi)) {
        bk = k;
        bi = i;
    }
}

__global__ void __launch_bounds__(1024)
    mst_kernel(const double *__restrict__ C, int N, int32_t *__restrict__ order,
               int32_t *__restrict__ from, double *__restrict__ w_out)
{
    extern __shared__ unsigned long long sm_key[];
    unsigned long long *key = sm_key;                  // N: image of the best edge weight
    double *val = reinterpret_cast<double *>(key + N); // N: that weight
    int *src = reinterpret_cast<int *>(val + N);       // N
    int *in = src + N;                                 // N
    __shared__ unsigned long long s_bk[32];
    __shared__ int s_bi[32];
    __shared__ int s_pick;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, nw = nt >> 5;
    for (int j = tid; j < N; j += nt) {
        const double c = C[j]; // row 0
        key[j] = prim_key(c);
        val[j] = c;
        src[j] = 0;
        in[j] = j == 0;
    }
    if (tid == 0) {
        order[0] = 0;
        from[0] = 0;
        w_out[0] = INFINITY;
    }
    __syncthreads();
    for (int step = 1; step < N; ++step) {
        // argmax of key over vertices not in the tree, ties to the lower index
        // (key 0 is below every real key, so a vertex is always found)
        unsigned long long bk = 0ull;
        int bi = 0x7fffffff;
        for (int j = tid; j < N; j += nt)
            if (!in[j]) prim_max(bk, bi, key[j], j);
#pragma unroll
        for (int o = 16; o; o >>= 1)
            prim_max(bk, bi, __shfl_xor_sync(0xffffffffu, bk, o), __shfl_xor_sync(0xffffffffu, bi, o));
        if (lane == 0) {
            s_bk[tid >> 5] = bk;
            s_bi[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid < 32) {
            bk = tid < nw ? s_bk[tid] : 0ull;
            bi = tid < nw ? s_bi[tid] : 0x7fffffff;
#pragma unroll
            for (int o = 16; o; o >>= 1)
                prim_max(bk, bi, __shfl_xor_sync(0xffffffffu, bk, o),
                         __shfl_xor_sync(0xffffffffu, bi, o));
            if (tid == 0) {
                s_pick = bi;
                order[step] = bi;
                from[step] = src[bi];
                w_out[step] = val[bi];
                in[bi] = 1;
            }
        }
        __syncthreads();
        const int v = s_pick;
        const double *row = C + (size_t)v * N;
        for (int j = tid; j < N; j += nt) {
            if (in[j]) continue;
            const double c = row[j];
            const unsigned long long ck = prim_key(c);
            if (ck > key[j]) {
                key[j] = ck;
                val[j] = c;
                src[j] = v;
            }
        }
        __syncthreads();
    }
}

int launch_mst(const double *C, int N, int32_t *order, int32_t *from, double *w,
               cudaStream_t s)
{
    const size_t smem = (size_t)N * (sizeof(unsigned long long) + sizeof(double) + 2 * sizeof(int));
    mst_kernel<<<1, 1024, smem, s>>>(C, N, order, from, w);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

// one warp per individual; the Prim-order pass is made parallel by pointer
// jumping: up(v_k) = w_k > tau ? from_k : v_k, then label = up^(log N)(v).
template <typename LabT>
__global__ void __launch_bounds__(256)
    init_threshold_kernel(LabT *__restrict__ pop, int ldp, int P, int N,
                          const int32_t *__restrict__ order, const int32_t *__restrict__ from,
                          const double *__restrict__ w, double tau_lo, double tau_span,
                          uint32_t k0, uint32_t k1)
{
    extern __shared__ int sm_up[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *up = sm_up + warp * N;
    for (int p = blockIdx.x * 8 + warp; p < P; p += gridDim.x * 8) {
        const U4 r = philox(0u, (uint32_t)p, 0u, STREAM_TAU, k0, k1);
        const double frac = (double)r.x * 2.3283064365386963e-10; // u / 2^32, exact
        const double tau = __dadd_rn(tau_lo, __dmul_rn(tau_span, frac));
        for (int k = lane; k < N; k += 32) {
            const int v = order[k];
            up[v] = (k > 0 && w[k] > tau) ? from[k] : v;
        }
        __syncwarp();
        // pointer jumping to the component root (the earliest vertex in Prim order);
        // every value ever stored in up[v] is an ancestor of v, so updating in
        // place only moves pointers further up, and ceil(log2 N) rounds suffice
        for (int round = 0; (1 << round) < N; ++round) {
            for (int v = lane; v < N; v += 32) up[v] = up[up[v]];
            __syncwarp();
        }
        LabT *dst = pop + (size_t)p * ldp;
        for (int j = lane; j < ldp; j += 32) dst[j] = (LabT)(j < N ? up[j] : 0);
        __syncwarp();
    }
}

template <typename LabT>
int launch_init_threshold(LabT *pop, int ldp, int P, int N, const int32_t *order,
                          const int32_t *from, const double *w, double tau_lo, double tau_hi,
                          uint32_t k0, uint32_t k1, cudaStream_t s)
{
    const size_t smem = (size_t)8 * N * sizeof(int);
    const int grid = (P + 7) / 8;
    init_threshold_kernel<LabT><<<grid, 256, smem, s>>>(pop, ldp, P, N, order, from, w, tau_lo, tau_hi - tau_lo, k0, k1);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

template int launch_init_threshold<uint16_t>(uint16_t *, int, int, int, const int32_t *,
                                             const int32_t *, const double *, double, double,
                                             uint32_t, uint32_t, cudaStream_t);
template int launch_init_threshold<int32_t>(int32_t *, int, int, int, const int32_t *,
                                            const int32_t *, const double *, double, double,
                                            uint32_t, uint32_t, cudaStream_t);

// ---------------------------------------------------------------------------
// Minimum spanning tree of every cluster of one configuration (the cluster
// trees drawn in Sec. 4.2) on the correlation distance d_ij = sqrt(2 (1 - C_ij)),
// by Prim's algorithm from each cluster's first gene. One CTA: canonical ids
// by first occurrence (atomicMin + block scan), members grouped by cluster,
// then the clusters one after another, every Prim step a block-wide argmin
// (distance, then gene index). Edges: clusters in first-occurrence order, each
// cluster's n_s - 1 edges (u < v, d) in Prim order.
// ---------------------------------------------------------------------------
// the distance of genes a != b from the upper-triangle entry of C
__device__ __forceinline__ double corr_dist(const double *C, int N, int a, int b)
{
    const int u = min(a, b), v = max(a, b);
    return sqrt(2.0 * (1.0 - C[(size_t)u * N + v]));
}

// ---------------------------------------------------------------------------
// Per-cluster minimum spanning trees, in two launches:
//   cluster_group_kernel  (one CTA) labels -> clusters in first-occurrence
//                         order: sizes, starts and the genes grouped by
//                         cluster, written to the scratch grp
//   cluster_prim_kernel   one CTA per cluster (CTAs beyond the cluster count
//                         return): Prim from the cluster's first gene; a
//                         cluster of at most 32 genes is done by one warp with
//                         shuffles only, a larger one by the CTA
// Scratch grp (int32): [0] bad-label flag, [1] cluster count K, [2 .. 2+N]
// starts (K + 1 used), [3+N .. 3+2N) genes grouped by cluster.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
    cluster_group_kernel(int N, const int32_t *__restrict__ labels, int *__restrict__ grp)
{
    extern __shared__ int sm_grp[];
    int *li = sm_grp;          // N labels
    int *first = li + N;       // N: label -> first gene
    int *cid = first + N;      // N: gene -> canonical cluster (at first genes)
    int *cnt = cid + N;        // N + 1: sizes, then starts
    int *fill = cnt + N + 1;   // N: fill counters
    __shared__ int s_part[32];
    __shared__ int s_bad;
    int *start = grp + 2, *mem = grp + 3 + N;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    const int nwarps = nt >> 5;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int i = tid; i < N; i += nt) {
        int v = labels[i];
        if (v < 0 || v >= N) {
            s_bad = 1;
            v = 0;
        }
        li[i] = v;
        first[i] = N;
        cnt[i] = 0;
        fill[i] = 0;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            grp[0] = 1;
            grp[1] = 0;
        }
        return;
    }
    for (int i = tid; i < N; i += nt) atomicMin(&first[li[i]], i);
    __syncthreads();
    // canonical ids: exclusive scan of the first-occurrence flags (chunked)
    const int chunk = (N + nt - 1) / nt;
    const int lo = min(N, tid * chunk), hi = min(N, lo + chunk);
    int c0 = 0;
    for (int i = lo; i < hi; ++i) c0 += first[li[i]] == i;
    int v = c0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_part[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nwarps ? s_part[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_part[lane] = w;
    }
    __syncthreads();
    int run = v - c0 + (wid ? s_part[wid - 1] : 0);
    for (int i = lo; i < hi; ++i)
        if (first[li[i]] == i) cid[i] = run++; // cid of a cluster's first gene
    const int K = s_part[nwarps - 1];
    __syncthreads();
    for (int i = tid; i < N; i += nt) atomicAdd(&cnt[cid[first[li[i]]]], 1);
    __syncthreads();
    // cluster starts (sequential over K by thread 0: K <= N, integer work)
    if (tid == 0) {
        int acc = 0;
        for (int c = 0; c < K; ++c) {
            const int n = cnt[c];
            cnt[c] = acc;
            acc += n;
        }
        cnt[K] = acc;
        grp[0] = 0;
        grp[1] = K;
    }
    __syncthreads();
    for (int c = tid; c <= K; c += nt) start[c] = cnt[c];
    // group the genes by cluster, ascending gene index inside a cluster
    // (Prim's ties go to the lower gene index, not the position, so any order
    // would do; this one keeps the first gene at position 0)
    for (int i = tid; i < N; i += nt) {
        const int c = cid[first[li[i]]];
        mem[atomicAdd(&fill[c], 1) + cnt[c]] = i;
    }
}

// Integer image of a tree distance for the minimum search: for finite a, b,
// a < b iff dist_img(a) < dist_img(b) and a == b iff the images are equal;
// +inf (the search's starting value) and NaN share the largest image, so a
// member is always picked and any finite distance is preferred to them.
__device__ __forceinline__ unsigned long long dist_img(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const bool nan = (b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
    const bool pinf = b == 0x7ff0000000000000ull;
    return (nan || pinf) ? ~0ull : prim_key(x);
}

// better Prim candidate: smaller key, ties to the lower gene index (compared
// on the integer pipe)
__device__ __forceinline__ bool prim_better(double k, int g, double bk, int bg)
{
    const unsigned long long ik = dist_img(k), ib = dist_img(bk);
    return ik < ib || (ik == ib && g < bg);
}

__global__ void __launch_bounds__(256)
    cluster_prim_kernel(const double *__restrict__ C, int N, const int *__restrict__ grp,
                        int32_t *__restrict__ eu, int32_t *__restrict__ ev,
                        double *__restrict__ ew)
{
    extern __shared__ double sm_prim[];
    const int c = blockIdx.x;
    if (grp[0] || c >= grp[1]) return;
    const int *start = grp + 2, *memg = grp + 3 + N;
    const int st = start[c], n = start[c + 1] - st;
    if (n < 2) return;
    const int *mem = memg + st;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    int root = N;
    for (int t = 0; t < n; ++t) root = min(root, mem[t]); // the cluster's first gene
    const int ebase = st - c;
    if (n <= 32) {
        // one warp: member t = lane
        if (wid) return;
        const int g = lane < n ? mem[lane] : 0x7fffffff;
        double key = (lane < n && g != root) ? corr_dist(C, N, root, g) : INFINITY;
        int src = root;
        bool in = lane >= n || g == root;
        for (int step = 0; step < n - 1; ++step) {
            double bk = in ? INFINITY : key;
            int bg = in ? 0x7fffffff : g, bl = lane;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const double ok = __shfl_xor_sync(0xffffffffu, bk, o);
                const int og = __shfl_xor_sync(0xffffffffu, bg, o);
                const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
                if (prim_better(ok, og, bk, bg)) {
                    bk = ok;
                    bg = og;
                    bl = ol;
                }
            }
            const int vs = __shfl_sync(0xffffffffu, src, bl);
            if (lane == bl) {
                in = true;
                eu[ebase + step] = min(vs, g);
                ev[ebase + step] = max(vs, g);
                ew[ebase + step] = bk;
            }
            if (!in) {
                const double d = corr_dist(C, N, bg, g);
                if (dist_img(d) < dist_img(key)) {
                    key = d;
                    src = bg;
                }
            }
        }
        return;
    }
    // the CTA: members t = tid, tid + 256, ...
    double *key = sm_prim;                          // n
    int *src = reinterpret_cast<int *>(key + n);    // n
    int *intree = src + n;                          // n
    __shared__ double s_bk[8];
    __shared__ int s_bg[8], s_bt[8];
    __shared__ int s_pick;
    for (int t = tid; t < n; t += blockDim.x) {
        const int g = mem[t];
        key[t] = g == root ? 0.0 : corr_dist(C, N, root, g);
        src[t] = root;
        intree[t] = g == root;
    }
    __syncthreads();
    for (int step = 0; step < n - 1; ++step) {
        double bk = INFINITY;
        int bg = 0x7fffffff, bt = -1;
        for (int t = tid; t < n; t += blockDim.x) {
            if (intree[t]) continue;
            const double k = key[t];
            const int g = mem[t];
            if (prim_better(k, g, bk, bg)) {
                bk = k;
                bg = g;
                bt = t;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const double ok = __shfl_xor_sync(0xffffffffu, bk, o);
            const int og = __shfl_xor_sync(0xffffffffu, bg, o);
            const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
            if (prim_better(ok, og, bk, bg)) {
                bk = ok;
                bg = og;
                bt = ot;
            }
        }
        if (lane == 0) {
            s_bk[wid] = bk;
            s_bg[wid] = bg;
            s_bt[wid] = bt;
        }
        __syncthreads();
        if (wid == 0) {
            bk = lane < nw ? s_bk[lane] : INFINITY;
            bg = lane < nw ? s_bg[lane] : 0x7fffffff;
            bt = lane < nw ? s_bt[lane] : -1;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const double ok = __shfl_xor_sync(0xffffffffu, bk, o);
                const int og = __shfl_xor_sync(0xffffffffu, bg, o);
                const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
                if (prim_better(ok, og, bk, bg)) {
                    bk = ok;
                    bg = og;
                    bt = ot;
                }
            }
            if (lane == 0) {
                s_pick = bt;
                const int a = src[bt], b = mem[bt];
                eu[ebase + step] = min(a, b);
                ev[ebase + step] = max(a, b);
                ew[ebase + step] = bk;
                intree[bt] = 1;
            }
        }
        __syncthreads();
        const int vg = mem[s_pick];
        for (int t = tid; t < n; t += blockDim.x) {
            if (intree[t]) continue;
            const double d = corr_dist(C, N, vg, mem[t]);
            if (dist_img(d) < dist_img(key[t])) {
                key[t] = d;
                src[t] = vg;
            }
        }
        __syncthreads();
    }
}

size_t cluster_mst_scratch_ints(int N) { return (size_t)3 + 2 * (size_t)N; }

int launch_cluster_mst(const double *C, int N, const int32_t *labels, int32_t *eu, int32_t *ev,
                       double *ew, int *grp, cudaStream_t s)
{
    const size_t gsmem = (size_t)(5 * N + 1) * sizeof(int);
    cluster_group_kernel<<<1, 1024, gsmem, s>>>(N, labels, grp);
    GPGA_LAUNCH_CHECK();
    const size_t psmem = (size_t)N * (sizeof(double) + 2 * sizeof(int));
    cluster_prim_kernel<<<N, 256, psmem, s>>>(C, N, grp, eu, ev, ew);
    GPGA_LAUNCH_CHECK();
    return GPGA_OK;
}

int prepare_init_kernels(int maxsmem)
{
    if (int rc = raise_smem(cluster_group_kernel, maxsmem)) return rc;
    if (int rc = raise_smem(cluster_prim_kernel, maxsmem)) return rc;
    if (int rc = raise_smem(mst_kernel, maxsmem)) return rc;
    if (int rc = raise_smem(init_threshold_kernel<uint16_t>, maxsmem)) return rc;
    if (int rc = raise_smem(init_threshold_kernel<int32_t>, maxsmem)) return rc;
    return GPGA_OK;
}

} // namespace gpga
