/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the hot path of the master-slave
 * parallel genetic algorithm of Hendricks, Gebbie & Wilcox (arXiv:1403.4099):
 * the Pearson prelude, the Giada-Marsili log-likelihood L_c used as fitness, and
 * the generation step of the GA.
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark are the only code that loads this library. The GPU library
 * neither links, includes nor calls it, and the two share no code, header, table
 * or constant generator.
 *
 * Every function names the passage of the paper it follows. The paper names but
 * does not define several GA operators (scaling, the "knowledge-based" crossover,
 * initialisation, the exact termination rule); for those the rule implemented
 * here is the project's written reading, stated beside each function.
 *
 * Pins (what fixes this file to something other than itself) live in tests/:
 * Philox known-answer vectors, numpy.corrcoef, closed forms of Eq. 8 (two
 * elements, equicorrelated blocks = -1/2 log det), brute force over set
 * partitions, the SUS counting property, exact integer weights, sklearn's ARI.
 *
 * Compiled with -ffp-contract=off so that no a*b+c is fused on any host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-3)
#define ORC_ERR_DEGENERATE (-4)

/* Philox counter word 3 selects the stream of draws. */
#define ORC_STREAM_INIT 0u
#define ORC_STREAM_SUS 1u
#define ORC_STREAM_XOVER 2u
#define ORC_STREAM_MUT 3u

#define ORC_SCALING_RANK 0
#define ORC_SCALING_PROP 1

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, the key   */
/* bumped by the Weyl constants between rounds.                                */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static void philox_draw(uint64_t seed, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                        uint32_t out[4])
{
    uint32_t ctr[4] = {w0, w1, w2, w3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* A uniform draw in [0, n): the high word of u*n. */
static int32_t label_draw(uint32_t u, int32_t n)
{
    return (int32_t)(((uint64_t)u * (uint64_t)(uint32_t)n) >> 32);
}

/* Probability p as a 32-bit threshold: an event fires when u < floor(p * 2^32). */
uint64_t orc_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(p * 4294967296.0);
}

/* ------------------------------------------------------------------------- */
/* Neumaier-compensated FP64 sum.                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
    double s, c;
} neu_t;

static void neu_add(neu_t *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double neu_val(const neu_t *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------- */
/* Pearson correlation, Eq. 7 (Sec. 2.1 and the standardisation below Eq. 2):  */
/* each column is centred over T; C_ij = <z_i, z_j> / sqrt(|z_i|^2 |z_j|^2).   */
/* Reading: the garbled norm is the squared Euclidean norm of the centred      */
/* vector; the diagonal is exactly 1; rounding excursions beyond [-1, 1]       */
/* (Cauchy-Schwarz) are clamped. R is T x N row-major with leading dim ld.     */
/* Returns ORC_ERR_DEGENERATE for a non-finite value or a zero-variance column.*/
/* ------------------------------------------------------------------------- */
int orc_pearson(const double *R, int T, int N, int ld, double *C)
{
    if (T < 2 || N < 1 || ld < N || !R || !C) return ORC_ERR_ARG;
    double *z = (double *)malloc((size_t)T * (size_t)N * sizeof(double));
    double *q = (double *)malloc((size_t)N * sizeof(double));
    if (!z || !q) {
        free(z);
        free(q);
        return ORC_ERR_OOM;
    }
    for (int j = 0; j < N; ++j) {
        neu_t s = {0.0, 0.0};
        for (int t = 0; t < T; ++t) {
            double r = R[(size_t)t * ld + j];
            if (!isfinite(r)) {
                free(z);
                free(q);
                return ORC_ERR_DEGENERATE;
            }
            neu_add(&s, r);
        }
        double mu = neu_val(&s) / (double)T;
        neu_t ss = {0.0, 0.0};
        for (int t = 0; t < T; ++t) {
            double v = R[(size_t)t * ld + j] - mu;
            z[(size_t)t * N + j] = v;
            neu_add(&ss, v * v);
        }
        q[j] = neu_val(&ss);
        if (!(q[j] > 0.0) || !isfinite(q[j])) {
            free(z);
            free(q);
            return ORC_ERR_DEGENERATE;
        }
    }
    for (int i = 0; i < N; ++i) {
        C[(size_t)i * N + i] = 1.0;
        for (int j = i + 1; j < N; ++j) {
            neu_t s = {0.0, 0.0};
            for (int t = 0; t < T; ++t) neu_add(&s, z[(size_t)t * N + i] * z[(size_t)t * N + j]);
            double v = neu_val(&s) / sqrt(q[i] * q[j]);
            if (v > 1.0) v = 1.0;
            if (v < -1.0) v = -1.0;
            C[(size_t)i * N + j] = v;
            C[(size_t)j * N + i] = v;
        }
    }
    free(z);
    free(q);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Cluster statistics of one configuration S (labels in [0, N)):               */
/*   n_s = sum_i delta(s_i, s)                          (Eq. 5)                */
/*   c_s = sum_{i,j} C_ij delta(s_i,s) delta(s_j,s)     (Eq. 6)                */
/*   d_s = sum_{i,j} (1 - C_ij) delta(s_i,s) delta(s_j,s)  (= n_s^2 - c_s)     */
/* Both sums run over ordered pairs, the diagonal included, members taken in   */
/* ascending index; Neumaier-compensated. d_s is accumulated directly so that  */
/* n_s^2 - c_s suffers no cancellation for tight clusters.                     */
/* ------------------------------------------------------------------------- */
static int check_labels(const int32_t *s, int N)
{
    for (int i = 0; i < N; ++i)
        if (s[i] < 0 || s[i] >= N) return ORC_ERR_ARG;
    return ORC_OK;
}

int orc_cluster_sums(const int32_t *s, int N, const double *C, int32_t *n, double *c, double *d)
{
    if (N < 1 || !s || !C || !n || !c || !d) return ORC_ERR_ARG;
    if (check_labels(s, N) != ORC_OK) return ORC_ERR_ARG;
    int32_t *start = (int32_t *)calloc((size_t)N + 1, sizeof(int32_t));
    int32_t *members = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *fill = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!start || !members || !fill) {
        free(start);
        free(members);
        free(fill);
        return ORC_ERR_OOM;
    }
    for (int l = 0; l < N; ++l) n[l] = 0;
    for (int i = 0; i < N; ++i) n[s[i]]++;
    for (int l = 0; l < N; ++l) start[l + 1] = start[l] + n[l];
    for (int l = 0; l < N; ++l) fill[l] = start[l];
    for (int i = 0; i < N; ++i) members[fill[s[i]]++] = i; /* stable: ascending i */
    for (int l = 0; l < N; ++l) {
        neu_t cs = {0.0, 0.0}, ds = {0.0, 0.0};
        for (int a = start[l]; a < start[l + 1]; ++a) {
            int i = members[a];
            for (int b = start[l]; b < start[l + 1]; ++b) {
                int j = members[b];
                double cij = C[(size_t)i * N + j];
                neu_add(&cs, cij);
                neu_add(&ds, 1.0 - cij);
            }
        }
        c[l] = neu_val(&cs);
        d[l] = neu_val(&ds);
    }
    free(start);
    free(members);
    free(fill);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Giada-Marsili log-likelihood, Eq. 8:                                        */
/*   L_c(S) = 1/2 sum_{s: n_s > 1} [ log(n_s / c_s)                            */
/*                    + (n_s - 1) log((n_s^2 - n_s) / (n_s^2 - c_s)) ]         */
/* with n_s^2 - c_s taken as the directly accumulated d_s. Natural log.        */
/* Reading of the domain edge (c_s <= 0 or d_s <= 0, reachable only from       */
/* degenerate data): c_s is floored at n_s 2^-40 and d_s at n_s(n_s-1) 2^-40;  */
/* *nclamp counts the floors applied. Terms are summed in the order in which   */
/* the clusters first occur along i, so that relabelling the clusters leaves   */
/* L bit-identical.                                                            */
/* ------------------------------------------------------------------------- */
static const double CLAMP_EPS = 9.094947017729282e-13; /* 2^-40 */

int orc_loglik(const int32_t *s, int N, const double *C, double *L, int32_t *nclamp)
{
    if (N < 1 || !s || !C || !L) return ORC_ERR_ARG;
    int32_t *n = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    double *c = (double *)malloc((size_t)N * sizeof(double));
    double *d = (double *)malloc((size_t)N * sizeof(double));
    unsigned char *seen = (unsigned char *)calloc((size_t)N, 1);
    if (!n || !c || !d || !seen) {
        free(n);
        free(c);
        free(d);
        free(seen);
        return ORC_ERR_OOM;
    }
    int rc = orc_cluster_sums(s, N, C, n, c, d);
    if (rc != ORC_OK) {
        free(n);
        free(c);
        free(d);
        free(seen);
        return rc;
    }
    neu_t acc = {0.0, 0.0};
    int32_t clamps = 0;
    for (int i = 0; i < N; ++i) {
        int l = s[i];
        if (seen[l]) continue;
        seen[l] = 1;
        if (n[l] <= 1) continue;
        double ns = (double)n[l];
        double cs = c[l], ds = d[l];
        double cmin = ns * CLAMP_EPS, dmin = ns * (ns - 1.0) * CLAMP_EPS;
        if (!(cs >= cmin)) {
            cs = cmin;
            clamps++;
        }
        if (!(ds >= dmin)) {
            ds = dmin;
            clamps++;
        }
        double term = 0.5 * (log(ns / cs) + (ns - 1.0) * log((ns * ns - ns) / ds));
        neu_add(&acc, term);
    }
    *L = neu_val(&acc);
    if (nclamp) *nclamp = clamps;
    free(n);
    free(c);
    free(d);
    free(seen);
    return ORC_OK;
}

/* L_c for P configurations (row p at labels + p*ld), over nthreads host threads
 * (<= 0: all). Returns the first error met. */
int orc_loglik_batch(const int32_t *labels, int P, int N, int ld, const double *C, double *L,
                     int nthreads)
{
    if (P < 0 || N < 1 || ld < N || !labels || !C || !L) return ORC_ERR_ARG;
    int err = ORC_OK;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
    /* a small batch runs on one thread: a team's start-up and barrier cost
     * more than its work there, and far more when the host is oversubscribed */
    if ((long long)P * N < 32768) nt = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
#endif
    for (int p = 0; p < P; ++p) {
        int rc = orc_loglik(labels + (size_t)p * ld, N, C, &L[p], NULL);
        if (rc != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            err = rc;
        }
    }
    (void)nthreads;
    return err;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Relabel by first occurrence: 0, 1, 2, ... (the canonical form of S). */
int orc_canonicalize(const int32_t *s, int N, int32_t *out)
{
    if (check_labels(s, N) != ORC_OK) return ORC_ERR_ARG;
    int32_t *map = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!map) return ORC_ERR_OOM;
    for (int l = 0; l < N; ++l) map[l] = -1;
    int32_t next = 0;
    for (int i = 0; i < N; ++i) {
        if (map[s[i]] < 0) map[s[i]] = next++;
        out[i] = map[s[i]];
    }
    free(map);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* GA operators (Sec. 3.1, Algorithm 1, Table 3). Parameters: P individuals   */
/* of N genes (Eq. 9, labels in [0, N) so that K = N permits all-singleton    */
/* configurations), `elite` fittest kept (E), M = P - E children.             */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t P, N, elite, max_gens, stall_gens, scaling, init_labels, reserved;
    double tol, pc, pkb, pm;
} orc_ga_params;

/* "Create initial population" (Algorithm 1). Reading: gene j of individual p is
 * uniform in [0, K0), K0 = init_labels (default N), drawn from word (j mod 4) of
 * Philox at counter (0, p, j/4, INIT). */
int orc_ga_init(int P, int N, int K0, uint64_t seed, int32_t *pop)
{
    if (P < 1 || N < 1 || K0 < 1 || K0 > N || !pop) return ORC_ERR_ARG;
    for (int p = 0; p < P; ++p) {
        for (int j = 0; j < N; ++j) {
            uint32_t w[4];
            philox_draw(seed, 0u, (uint32_t)p, (uint32_t)(j / 4), ORC_STREAM_INIT, w);
            pop[(size_t)p * N + j] = label_draw(w[j % 4], K0);
        }
    }
    return ORC_OK;
}

/* Reading of "create initial population" with domain knowledge (optional): the
 * connected components of {(i, j) : C_ij > tau_p} for a per-individual level
 * tau_p = tau_lo + (tau_hi - tau_lo) * (u / 2^32), u = word 0 of Philox
 * (0, p, 0, TAU=4). Built here by brute force: union of every pair above the
 * level (union-find), each component labelled with its member that joins the
 * maximum spanning tree first under Prim's rule (start at 0; next = largest key,
 * ties to the lower index; keys improve only on a strictly larger C). */
#define ORC_STREAM_TAU 4u

int orc_prim_order(const double *C, int N, int32_t *order)
{
    if (N < 1 || !C || !order) return ORC_ERR_ARG;
    double *key = (double *)malloc((size_t)N * sizeof(double));
    unsigned char *in = (unsigned char *)calloc((size_t)N, 1);
    if (!key || !in) {
        free(key);
        free(in);
        return ORC_ERR_OOM;
    }
    in[0] = 1;
    order[0] = 0;
    for (int j = 0; j < N; ++j) key[j] = C[j];
    for (int step = 1; step < N; ++step) {
        int best = -1;
        for (int j = 0; j < N; ++j)
            if (!in[j] && (best < 0 || key[j] > key[best])) best = j;
        in[best] = 1;
        order[step] = best;
        for (int j = 0; j < N; ++j)
            if (!in[j] && C[(size_t)best * N + j] > key[j]) key[j] = C[(size_t)best * N + j];
    }
    free(key);
    free(in);
    return ORC_OK;
}

static int uf_find(int32_t *par, int x)
{
    while (par[x] != x) x = par[x] = par[par[x]];
    return x;
}

int orc_ga_init_threshold(const double *C, int P, int N, double tau_lo, double tau_hi,
                          uint64_t seed, int32_t *pop)
{
    if (P < 1 || N < 1 || !C || !pop || !(tau_hi >= tau_lo)) return ORC_ERR_ARG;
    int32_t *order = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *pos = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *par = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *rep = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int rc = (order && pos && par && rep) ? orc_prim_order(C, N, order) : ORC_ERR_OOM;
    if (rc == ORC_OK) {
        for (int k = 0; k < N; ++k) pos[order[k]] = k;
        const double span = tau_hi - tau_lo;
        for (int p = 0; p < P; ++p) {
            uint32_t w[4];
            philox_draw(seed, 0u, (uint32_t)p, 0u, ORC_STREAM_TAU, w);
            const double tau = tau_lo + span * ((double)w[0] * 2.3283064365386963e-10);
            for (int i = 0; i < N; ++i) par[i] = i;
            for (int i = 0; i < N; ++i)
                for (int j = i + 1; j < N; ++j)
                    if (C[(size_t)i * N + j] > tau) {
                        int a = uf_find(par, i), b = uf_find(par, j);
                        if (a != b) par[a] = b;
                    }
            /* label: the member of the component that comes first in Prim order */
            for (int i = 0; i < N; ++i) rep[i] = -1;
            for (int i = 0; i < N; ++i) {
                int r = uf_find(par, i);
                if (rep[r] < 0 || pos[i] < pos[rep[r]]) rep[r] = i;
            }
            for (int i = 0; i < N; ++i) pop[(size_t)p * N + i] = rep[uf_find(par, i)];
        }
    }
    free(order);
    free(pos);
    free(par);
    free(rep);
    return rc;
}

/* "Isolate fittest individuals": perm[r] is the individual of rank r, ranked by
 * L descending, ties by lower index first (a stable merge sort of 0..P-1); a NaN
 * fitness ranks as -inf. */
static double rank_key(double x) { return isnan(x) ? -INFINITY : x; }

int orc_ga_rank(const double *L, int P, int32_t *perm)
{
    if (P < 1 || !L || !perm) return ORC_ERR_ARG;
    int32_t *tmp = (int32_t *)malloc((size_t)P * sizeof(int32_t));
    if (!tmp) return ORC_ERR_OOM;
    for (int p = 0; p < P; ++p) perm[p] = p;
    for (int width = 1; width < P; width *= 2) {
        for (int lo = 0; lo < P; lo += 2 * width) {
            int mid = lo + width < P ? lo + width : P;
            int hi = lo + 2 * width < P ? lo + 2 * width : P;
            int i = lo, j = mid, o = lo;
            while (i < mid && j < hi) {
                /* take from the right run only when strictly fitter: stability */
                if (rank_key(L[perm[j]]) > rank_key(L[perm[i]]))
                    tmp[o++] = perm[j++];
                else
                    tmp[o++] = perm[i++];
            }
            while (i < mid) tmp[o++] = perm[i++];
            while (j < hi) tmp[o++] = perm[j++];
        }
        memcpy(perm, tmp, (size_t)P * sizeof(int32_t));
    }
    free(tmp);
    return ORC_OK;
}

/* "Apply scaling" (Algorithm 1; undefined in the paper). Reading: weights are
 * 32.32 fixed point so that selection is exact integer arithmetic.
 *   RANK: w(r) = floor(2^32 / sqrt(r + 1)) for 0-based rank r, IEEE FP64 sqrt
 *         and division.
 *   PROP: w = floor(max(L, 0) / L_max * 2^32); all weights 1 if L_max <= 0.
 * Output is indexed by rank. */
int orc_ga_weights(const double *L, const int32_t *perm, int P, int scaling, uint64_t *w)
{
    if (P < 1 || !perm || !w) return ORC_ERR_ARG;
    if (scaling == ORC_SCALING_RANK) {
        for (int r = 0; r < P; ++r) w[r] = (uint64_t)floor(4294967296.0 / sqrt((double)(r + 1)));
        return ORC_OK;
    }
    if (scaling != ORC_SCALING_PROP || !L) return ORC_ERR_ARG;
    double lmax = L[perm[0]];
    for (int r = 0; r < P; ++r) {
        if (!(lmax > 0.0)) {
            w[r] = 1;
            continue;
        }
        double x = L[perm[r]];
        if (!(x > 0.0)) x = 0.0;
        w[r] = (uint64_t)floor(x / lmax * 4294967296.0);
    }
    return ORC_OK;
}

/* "Apply genetic operator: selection" -- stochastic universal sampling
 * (Sec. 3.1, Baker): the P individuals lie on a line in rank order, each over a
 * segment of length w; M pointers at x_k = floor((k 2^32 + u) W / (M 2^32)),
 * k = 0..M-1, with W = sum w and one 32-bit offset u, pick the individual whose
 * segment [prefix_{r-1}, prefix_r) holds x_k. Exact 128-bit arithmetic.
 * sel[k] receives the selected rank. */
int orc_ga_sus(const uint64_t *w, int P, int M, uint32_t u, int32_t *sel)
{
    if (P < 1 || M < 1 || !w || !sel) return ORC_ERR_ARG;
    unsigned __int128 W = 0;
    for (int r = 0; r < P; ++r) W += w[r];
    if (W == 0) return ORC_ERR_ARG;
    int r = 0;
    unsigned __int128 edge = w[0]; /* prefix_r, exclusive upper end of rank r */
    for (int k = 0; k < M; ++k) {
        unsigned __int128 num = (((unsigned __int128)(uint32_t)k) << 32) + u;
        unsigned __int128 x = num * W / (((unsigned __int128)(uint32_t)M) << 32);
        while (x >= edge) {
            ++r;
            edge += w[r];
        }
        sel[k] = r;
    }
    return ORC_OK;
}

/* Reading of the "knowledge-based crossover" (Sec. 3.1, Table 3; defined only in
 * a thesis not available here): a cluster merge. The child starts as parent a;
 * Q = {j : b_j = b_q} is the cluster of parent b that holds anchor gene q; every
 * gene of Q joins the cluster that holds q in a (child_j = a_q on Q). Members of
 * a cluster in b thus end up together in the child, whatever b's label names,
 * and clusters grow by union -- the domain knowledge that co-clustered stocks of
 * a fit parent belong together. */
static void kb_merge(const int32_t *a, const int32_t *b, int N, int q, int32_t *child)
{
    int32_t bq = b[q], aq = a[q];
    for (int j = 0; j < N; ++j) child[j] = (b[j] == bq) ? aq : a[j];
}

/* Mutation by random replacement, each gene with probability P_m (Sec. 3.1,
 * Table 3), drawn as geometric gaps between mutated genes instead of one test
 * per gene (the same law). Genes are taken in blocks of 16 consecutive genes.
 * Within a block, from position pos the next mutated gene is pos + G(u) with
 *   G(u) = #{t in 1..16 : u < T_t},  T_t = min(floor((1 - P_m)^t 2^32), 2^32 - 1),
 * so that P(none of the next t genes mutates) = T_t / 2^32 = (1 - P_m)^t; the
 * gene takes the label draw(v, N), and the search goes on after it. The (u, v)
 * pairs are words (0, 1) then (2, 3) of Philox(g, k, block + 65536 e, MUT) for
 * e = 0, 1, ... (a block with more than two mutations uses further calls).
 * (1 - P_m)^t is the FP64 product of t factors (1 - P_m), left to right.
 * floor(P_m 2^32) = 0 means no mutation at all. */
#define ORC_MUT_BLOCK 16

static void mutation_gap_table(double pm, uint32_t T[ORC_MUT_BLOCK])
{
    const double r = 1.0 - pm;
    double q = 1.0;
    for (int t = 0; t < ORC_MUT_BLOCK; ++t) {
        q = q * r; /* (1 - P_m)^(t + 1) */
        double v = floor(q * 4294967296.0);
        if (v > 4294967295.0) v = 4294967295.0;
        T[t] = (uint32_t)v;
    }
}

static int mutation_gap(uint32_t u, const uint32_t T[ORC_MUT_BLOCK])
{
    int s = 0;
    for (int t = 0; t < ORC_MUT_BLOCK; ++t)
        if (u < T[t]) ++s;
    return s;
}

static void mutate_child(int32_t *child, int N, uint64_t seed, int32_t g, int k,
                         const uint32_t T[ORC_MUT_BLOCK])
{
    for (int blk = 0; blk * ORC_MUT_BLOCK < N; ++blk) {
        const int base = blk * ORC_MUT_BLOCK;
        const int len = N - base < ORC_MUT_BLOCK ? N - base : ORC_MUT_BLOCK;
        int pos = 0;
        for (uint32_t e = 0;; ++e) {
            uint32_t w[4];
            philox_draw(seed, (uint32_t)g, (uint32_t)k, (uint32_t)blk + 65536u * e,
                        ORC_STREAM_MUT, w);
            int done = 0;
            for (int h = 0; h < 2 && !done; ++h) {
                pos += mutation_gap(w[2 * h], T);
                if (pos >= len) {
                    done = 1;
                    break;
                }
                child[base + pos] = label_draw(w[2 * h + 1], N);
                ++pos;
                if (pos >= len) done = 1;
            }
            if (done) break;
        }
    }
}

/* One generation of Algorithm 1 after scoring: isolate fittest, elitism,
 * scaling, SUS selection, crossover (P_c; cluster merge with P_kb, else one-point),
 * random-replacement mutation per gene (P_m), replacement. Draws for parent
 * generation g:
 *   SUS offset   u = word 0 of Philox(g, 0, 0, SUS)
 *   child k      words of Philox(g, k, 0, XOVER): x crossover?, y merge?,
 *                z anchor q = draw(z, N) or cut = 1 + draw(z, N - 1)
 *   mutation     per block of 16 genes (see mutate_child): gaps between
 *                mutated genes from Philox(g, k, block + 65536 e, MUT)
 * Pairing: a = parent[k], b = parent[(k + M/2) mod M]. Elites fill slots
 * 0..E-1 in rank order, unchanged; child k fills slot E + k.
 * Optional outputs: perm (P ranks), parents (M indices). */
int orc_ga_evolve(const int32_t *pop, const double *L, const orc_ga_params *prm, uint64_t seed,
                  int32_t g, int32_t *next, int32_t *perm_out, int32_t *parents_out)
{
    if (!pop || !L || !prm || !next) return ORC_ERR_ARG;
    const int P = prm->P, N = prm->N, E = prm->elite;
    if (P < 2 || N < 1 || E < 0 || E >= P) return ORC_ERR_ARG;
    const int M = P - E;
    int32_t *perm = (int32_t *)malloc((size_t)P * sizeof(int32_t));
    uint64_t *w = (uint64_t *)malloc((size_t)P * sizeof(uint64_t));
    int32_t *sel = (int32_t *)malloc((size_t)M * sizeof(int32_t));
    int32_t *par = (int32_t *)malloc((size_t)M * sizeof(int32_t));
    int rc = ORC_OK;
    if (!perm || !w || !sel || !par) {
        rc = ORC_ERR_OOM;
        goto done;
    }
    rc = orc_ga_rank(L, P, perm);
    if (rc) goto done;
    rc = orc_ga_weights(L, perm, P, prm->scaling, w);
    if (rc) goto done;
    uint32_t wsus[4];
    philox_draw(seed, (uint32_t)g, 0u, 0u, ORC_STREAM_SUS, wsus);
    rc = orc_ga_sus(w, P, M, wsus[0], sel);
    if (rc) goto done;
    for (int k = 0; k < M; ++k) par[k] = perm[sel[k]];

    const uint64_t thr_pc = orc_threshold(prm->pc);
    const uint64_t thr_pkb = orc_threshold(prm->pkb);
    const uint64_t thr_pm = orc_threshold(prm->pm);
    uint32_t gaps[ORC_MUT_BLOCK];
    mutation_gap_table(prm->pm, gaps);

    for (int e = 0; e < E; ++e)
        memcpy(next + (size_t)e * N, pop + (size_t)perm[e] * N, (size_t)N * sizeof(int32_t));

    for (int k = 0; k < M; ++k) {
        const int32_t *a = pop + (size_t)par[k] * N;
        const int32_t *b = pop + (size_t)par[(k + M / 2) % M] * N;
        int32_t *child = next + (size_t)(E + k) * N;
        uint32_t xw[4];
        philox_draw(seed, (uint32_t)g, (uint32_t)k, 0u, ORC_STREAM_XOVER, xw);
        memcpy(child, a, (size_t)N * sizeof(int32_t));
        if ((uint64_t)xw[0] < thr_pc) {
            if ((uint64_t)xw[1] < thr_pkb) {
                kb_merge(a, b, N, label_draw(xw[2], N), child);
            } else {
                int cut = 1 + label_draw(xw[2], N - 1);
                for (int j = cut; j < N; ++j) child[j] = b[j];
            }
        }
        if (thr_pm) mutate_child(child, N, seed, g, k, gaps);
    }
    if (perm_out) memcpy(perm_out, perm, (size_t)P * sizeof(int32_t));
    if (parents_out) memcpy(parents_out, par, (size_t)M * sizeof(int32_t));
done:
    free(perm);
    free(w);
    free(sel);
    free(par);
    return rc;
}

/* Island model (the variant proposed in Sec. 5.2 and 6), ring migration after the
 * operators of one generation: K populations of P x N (pops, island-major)
 * with the fitness of their members (Ls); island k's first m members (its
 * elites, m <= E) replace, with their fitness, the last m members of island
 * (k + 1) mod K. Every island reads its own first m members before any is
 * overwritten (2 m <= P keeps the two ranges apart). */
int orc_island_migrate(int32_t *pops, double *Ls, int K, int P, int N, int m)
{
    if (!pops || !Ls || K < 2 || m < 1 || 2 * m > P) return ORC_ERR_ARG;
    int32_t *head = (int32_t *)malloc((size_t)K * m * N * sizeof(int32_t));
    double *hl = (double *)malloc((size_t)K * m * sizeof(double));
    if (!head || !hl) {
        free(head);
        free(hl);
        return ORC_ERR_OOM;
    }
    for (int k = 0; k < K; ++k) {
        memcpy(head + (size_t)k * m * N, pops + (size_t)k * P * N, (size_t)m * N * sizeof(int32_t));
        memcpy(hl + (size_t)k * m, Ls + (size_t)k * P, (size_t)m * sizeof(double));
    }
    for (int k = 0; k < K; ++k) {
        const int to = (k + 1) % K;
        memcpy(pops + ((size_t)to * P + (P - m)) * N, head + (size_t)k * m * N,
               (size_t)m * N * sizeof(int32_t));
        memcpy(Ls + (size_t)to * P + (P - m), hl + (size_t)k * m, (size_t)m * sizeof(double));
    }
    free(head);
    free(hl);
    return ORC_OK;
}

/* "Determine if termination criteria are met" (Algorithm 1; Table 3: number of
 * generations, error tolerance, stall generations). Reading: stop after scoring
 * generation g when g >= max_gens, or when g >= G_stall and
 * best_g - best_{g - G_stall} <= tol * max(1, |best_g|). tol < 0 or
 * stall_gens <= 0 switch the stall rule off. */
int orc_ga_terminated(const double *best_hist, int g, const orc_ga_params *prm)
{
    if (g >= prm->max_gens) return 1;
    if (prm->tol >= 0.0 && prm->stall_gens > 0 && g >= prm->stall_gens) {
        double b = best_hist[g];
        if (b - best_hist[g - prm->stall_gens] <= prm->tol * fmax(1.0, fabs(b))) return 1;
    }
    return 0;
}

/* A whole run of Algorithm 1 on correlation matrix C (N x N): initialise,
 * then score / record / test / evolve until termination. best_hist must hold
 * max_gens + 1 values; best_ring (optional) (max_gens + 1) x N labels: the best
 * individual of every generation. */
int orc_ga_run(const double *C, const orc_ga_params *prm, uint64_t seed, int nthreads,
               int32_t *best_labels, double *best_L, int32_t *gens_done, double *best_hist,
               int32_t *best_ring)
{
    if (!C || !prm || !best_labels || !best_L || !gens_done || !best_hist) return ORC_ERR_ARG;
    const int P = prm->P, N = prm->N;
    if (P < 2 || N < 1 || prm->max_gens < 0) return ORC_ERR_ARG;
    int32_t *pop = (int32_t *)malloc((size_t)P * N * sizeof(int32_t));
    int32_t *nxt = (int32_t *)malloc((size_t)P * N * sizeof(int32_t));
    double *L = (double *)malloc((size_t)P * sizeof(double));
    int32_t *perm = (int32_t *)malloc((size_t)P * sizeof(int32_t));
    int rc = ORC_OK;
    if (!pop || !nxt || !L || !perm) {
        rc = ORC_ERR_OOM;
        goto done;
    }
    int K0 = prm->init_labels > 0 ? prm->init_labels : N;
    rc = orc_ga_init(P, N, K0, seed, pop);
    if (rc) goto done;
    rc = orc_loglik_batch(pop, P, N, N, C, L, nthreads);
    if (rc) goto done;
    for (int g = 0;; ++g) {
        rc = orc_ga_rank(L, P, perm);
        if (rc) goto done;
        best_hist[g] = L[perm[0]];
        if (best_ring) memcpy(best_ring + (size_t)g * N, pop + (size_t)perm[0] * N, (size_t)N * sizeof(int32_t));
        if (orc_ga_terminated(best_hist, g, prm)) {
            memcpy(best_labels, pop + (size_t)perm[0] * N, (size_t)N * sizeof(int32_t));
            *best_L = L[perm[0]];
            *gens_done = g;
            break;
        }
        rc = orc_ga_evolve(pop, L, prm, seed, g, nxt, NULL, NULL);
        if (rc) goto done;
        int32_t *t = pop;
        pop = nxt;
        nxt = t;
        rc = orc_loglik_batch(pop, P, N, N, C, L, nthreads);
        if (rc) goto done;
    }
done:
    free(pop);
    free(nxt);
    free(L);
    free(perm);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Brute force: every set partition of N <= 12 objects as a restricted-growth  */
/* string (a_0 = 0, a_i <= 1 + max(a_0..a_{i-1})) in lexicographic order; the  */
/* maximum of L_c with ties to the lexicographically smallest string.          */
/* ------------------------------------------------------------------------- */
int orc_brute_force(const double *C, int N, int32_t *best, double *bestL, int64_t *count)
{
    if (N < 1 || N > 12 || !C || !best || !bestL || !count) return ORC_ERR_ARG;
    int32_t a[12] = {0};
    int64_t cnt = 0;
    int have = 0;
    for (;;) {
        double L;
        int rc = orc_loglik(a, N, C, &L, NULL);
        if (rc) return rc;
        ++cnt;
        if (!have || L > *bestL) {
            have = 1;
            *bestL = L;
            memcpy(best, a, (size_t)N * sizeof(int32_t));
        }
        int i = N - 1;
        for (; i >= 1; --i) {
            int32_t m = 0;
            for (int t = 0; t < i; ++t)
                if (a[t] > m) m = a[t];
            if (a[i] <= m) break;
        }
        if (i < 1) break;
        a[i]++;
        for (int t = i + 1; t < N; ++t) a[t] = 0;
    }
    *count = cnt;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Adjusted Rand index (Hubert & Arabie, 1985) from the contingency table of   */
/* two labelings in [0, N):                                                     */
/*   ARI = (sum_ij C(n_ij,2) - E) / (1/2 (sum_i C(a_i,2) + sum_j C(b_j,2)) - E) */
/*   E   = sum_i C(a_i,2) sum_j C(b_j,2) / C(N,2).                              */
/* The denominator vanishes only when both are all-singleton or both a single  */
/* cluster, i.e. identical: 1 is returned. NaN on bad labels.                  */
/* EWMA-weighted Pearson correlation (pre-processing upstream of C: the
 * covariance the paper computes with an online exponentially weighted filter, Sec. 4.2):
 * rows weighted w_t = lambda^(T-1-t) (the newest row weighs 1), weighted
 * means mu_j = sum_t w_t R_tj / sum_t w_t, and
 * C_ij = sum_t w_t (R_ti - mu_i)(R_tj - mu_j) / sqrt(q_i q_j),
 * q_j = sum_t w_t (R_tj - mu_j)^2; diagonal 1, clamped to [-1, 1].
 * lambda = 1 is the plain Pearson of Eq. 7. Sequential FP64 sums. */
int orc_pearson_ewma(const double *R, int T, int N, int ld, double lambda, double *C)
{
    if (!R || !C || T < 2 || N < 1 || ld < N || !(lambda > 0.0 && lambda <= 1.0))
        return ORC_ERR_ARG;
    double *w = (double *)malloc((size_t)T * sizeof(double));
    double *mu = (double *)malloc((size_t)N * sizeof(double));
    double *q = (double *)malloc((size_t)N * sizeof(double));
    if (!w || !mu || !q) {
        free(w);
        free(mu);
        free(q);
        return ORC_ERR_OOM;
    }
    double W = 0.0;
    for (int t = 0; t < T; ++t) {
        w[t] = pow(lambda, (double)(T - 1 - t));
        W += w[t];
    }
    int rc = ORC_OK;
    for (int j = 0; j < N; ++j) {
        double s = 0.0;
        for (int t = 0; t < T; ++t) s += w[t] * R[(size_t)t * ld + j];
        mu[j] = s / W;
        double v = 0.0;
        for (int t = 0; t < T; ++t) {
            const double z = R[(size_t)t * ld + j] - mu[j];
            v += w[t] * z * z;
        }
        q[j] = v;
        if (!(v > 0.0) || !isfinite(v)) rc = ORC_ERR_DEGENERATE;
    }
    if (rc == ORC_OK)
        for (int i = 0; i < N; ++i) {
            C[(size_t)i * N + i] = 1.0;
            for (int j = i + 1; j < N; ++j) {
                double s = 0.0;
                for (int t = 0; t < T; ++t)
                    s += w[t] * (R[(size_t)t * ld + i] - mu[i]) * (R[(size_t)t * ld + j] - mu[j]);
                double c = s / sqrt(q[i] * q[j]);
                if (c > 1.0) c = 1.0;
                if (c < -1.0) c = -1.0;
                C[(size_t)i * N + j] = c;
                C[(size_t)j * N + i] = c;
            }
        }
    free(w);
    free(mu);
    free(q);
    return rc;
}

/* Minimum spanning tree of every cluster of configuration s (the trees the
 * paper draws for the clusters it finds, Sec. 4.2), on the correlation distance
 * d_ij = sqrt(2 (1 - C_ij)), by Kruskal's algorithm: the cluster's pairs
 * i < j sorted by (d, i, j), each joining two components kept (union-find).
 * Output, clusters in first-occurrence order, for each its n_s - 1 edges
 * (u < v, d) in Kruskal order; *n_edges = N - number of clusters.
 * Arrays eu, ev, ew hold at least N entries. */
typedef struct {
    double d;
    int32_t u, v;
} mst_edge;

static int mst_edge_cmp(const void *a, const void *b)
{
    const mst_edge *x = (const mst_edge *)a, *y = (const mst_edge *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

int orc_cluster_mst(const int32_t *s, int N, const double *C, int32_t *eu, int32_t *ev,
                    double *ew, int32_t *n_edges)
{
    if (!s || !C || !eu || !ev || !ew || !n_edges || N < 1) return ORC_ERR_ARG;
    for (int i = 0; i < N; ++i)
        if (s[i] < 0 || s[i] >= N) return ORC_ERR_ARG;
    int32_t *seen = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    int32_t *mem = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *par = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    mst_edge *e = (mst_edge *)malloc(((size_t)N * (N - 1) / 2 + 1) * sizeof(mst_edge));
    if (!seen || !mem || !par || !e) {
        free(seen);
        free(mem);
        free(par);
        free(e);
        return ORC_ERR_OOM;
    }
    int out = 0;
    for (int i = 0; i < N; ++i) {
        const int32_t lab = s[i];
        if (seen[lab]) continue;
        seen[lab] = 1;
        int n = 0;
        for (int j = i; j < N; ++j)
            if (s[j] == lab) mem[n++] = j;
        size_t m = 0;
        for (int a = 0; a < n; ++a)
            for (int b = a + 1; b < n; ++b) {
                const double c = C[(size_t)mem[a] * N + mem[b]];
                e[m].d = sqrt(2.0 * (1.0 - c));
                e[m].u = mem[a];
                e[m].v = mem[b];
                ++m;
            }
        qsort(e, m, sizeof(mst_edge), mst_edge_cmp);
        for (int a = 0; a < n; ++a) par[mem[a]] = mem[a];
        for (size_t k = 0; k < m; ++k) {
            const int ru = uf_find(par, e[k].u), rv = uf_find(par, e[k].v);
            if (ru == rv) continue;
            par[ru] = rv;
            eu[out] = e[k].u;
            ev[out] = e[k].v;
            ew[out] = e[k].d;
            ++out;
        }
    }
    *n_edges = out;
    free(seen);
    free(mem);
    free(par);
    free(e);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
double orc_ari(const int32_t *x, const int32_t *y, int N)
{
    if (N < 1 || !x || !y || check_labels(x, N) || check_labels(y, N)) return NAN;
    if (N < 2) return 1.0;
    int32_t *cx = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *cy = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    orc_canonicalize(x, N, cx);
    orc_canonicalize(y, N, cy);
    int kx = 0, ky = 0;
    for (int i = 0; i < N; ++i) {
        if (cx[i] + 1 > kx) kx = cx[i] + 1;
        if (cy[i] + 1 > ky) ky = cy[i] + 1;
    }
    int64_t *tab = (int64_t *)calloc((size_t)kx * ky, sizeof(int64_t));
    int64_t *ra = (int64_t *)calloc((size_t)kx, sizeof(int64_t));
    int64_t *cb = (int64_t *)calloc((size_t)ky, sizeof(int64_t));
    for (int i = 0; i < N; ++i) {
        tab[(size_t)cx[i] * ky + cy[i]]++;
        ra[cx[i]]++;
        cb[cy[i]]++;
    }
    double idx = 0.0, sa = 0.0, sb = 0.0;
    for (size_t t = 0; t < (size_t)kx * ky; ++t) idx += (double)tab[t] * (double)(tab[t] - 1) / 2.0;
    for (int i = 0; i < kx; ++i) sa += (double)ra[i] * (double)(ra[i] - 1) / 2.0;
    for (int j = 0; j < ky; ++j) sb += (double)cb[j] * (double)(cb[j] - 1) / 2.0;
    double total = (double)N * (double)(N - 1) / 2.0;
    double expected = sa * sb / total;
    double maxidx = 0.5 * (sa + sb);
    double ari = (maxidx == expected) ? 1.0 : (idx - expected) / (maxidx - expected);
    free(cx);
    free(cy);
    free(tab);
    free(ra);
    free(cb);
    return ari;
}
