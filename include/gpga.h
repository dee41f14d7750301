/*
 * gpga.h -- C ABI of libgpga.so, the GB300 (sm_103a) hot path of the
 * master-slave parallel genetic algorithm for unsupervised market clustering of
 * Hendricks, Gebbie & Wilcox (arXiv:1403.4099).
 *
 * The path: Pearson correlation C of a T x N returns matrix (Eq. 7), scoring of
 * a population of cluster-label vectors with the Giada-Marsili log-likelihood
 * L_c (Eq. 5, 6, 8), and the device-resident GA generation of Algorithm 1
 * (isolate fittest, elitism, scaling, SUS selection, crossover, mutation,
 * replacement) driven by a counter-based Philox4x32-10 stream.
 *
 * Conventions for every call:
 *   - Status: 0 = GPGA_OK, negative = error (GPGA_ERR_*). No C++ exception
 *     crosses the ABI. gpga_last_error() returns a description of the last
 *     error of the calling thread (static storage, valid until the next call).
 *   - Pointers are plain addresses. "device" pointers must be readable by the
 *     current CUDA device (cudaMalloc / torch CUDA storage / managed memory);
 *     "host or device" pointers are classified with cudaPointerGetAttributes.
 *     Caller buffers are borrowed for the duration of the call only (or, for
 *     asynchronous calls, until the stream reaches the call), never retained.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Layouts are row-major. Labels are int32 in [0, N) (0-based form of the
 *     paper's 1..K labels, Eq. 9, with K = N).
 *   - The library allocates device memory only in ga_init and ga_batch_init
 *     (owned by the handle, released by ga_free / ga_batch_free), in
 *     serve_create and at each admission of a request (stream-ordered, freed
 *     when the request retires or by serve_free) and, for cluster_corr and
 *     ga_score, stream-ordered scratch (cudaMallocAsync / cudaFreeAsync)
 *     inside the call.
 */
#ifndef GPGA_H
#define GPGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GPGA_API __attribute__((visibility("default")))
#else
#define GPGA_API
#endif

/* status codes */
#define GPGA_OK 0
#define GPGA_ERR_ARG (-1)        /* bad argument: size, pointer, label range */
#define GPGA_ERR_CUDA (-2)       /* a CUDA runtime call failed */
#define GPGA_ERR_OOM (-3)        /* device allocation failed */
#define GPGA_ERR_DEGENERATE (-4) /* non-finite input or zero-variance column */
#define GPGA_ERR_TIMEOUT (-5)    /* a bounded device wait gave up */
#define GPGA_ERR_STATE (-6)      /* call not valid in the handle's state */

/* scoring forms (both end in the same FP64 log-term assembly) */
#define GPGA_FORM_PLAIN 0  /* FP32 CUDA-core pair accumulation */
#define GPGA_FORM_TENSOR 1 /* tcgen05 one-hot contraction, D split BF16 hi+lo */
#define GPGA_FORM_GATHER 2 /* same-cluster pairs only (sorted by label), FP32 gathers;
                              in a run, fused with the generation's operators */

/* fitness scaling before selection ("apply scaling", Algorithm 1) */
#define GPGA_SCALING_RANK 0 /* w(r) = floor(2^32 / sqrt(r + 1)), r = 0-based rank */
#define GPGA_SCALING_PROP 1 /* w = floor(max(L, 0) / L_max * 2^32) */

/* initial population ("create initial population", Algorithm 1) */
#define GPGA_INIT_UNIFORM 0   /* labels uniform in [0, init_labels) */
#define GPGA_INIT_THRESHOLD 1 /* components of {C_ij > tau_p}, tau_p ~ U[tau_lo, tau_hi) */

/* Limits of this build. */
#define GPGA_MAX_N 4096       /* stocks (genes per individual) */
#define GPGA_MAX_P 16384      /* population size */

/*
 * GA parameters; gpga_default_params() fills Table 3 of the paper (population
 * 1000, 400 generations, P_c 0.9, error tolerance 1e-5, stall 50, elite 10,
 * knowledge-based crossover share 0.9) with P_m read per gene as 0.01.
 */
typedef struct gpga_params {
    int32_t P;           /* population size, 2..GPGA_MAX_P */
    int32_t elite;       /* E fittest copied unchanged, 0..P-1 */
    int32_t max_gens;    /* G_max: stop after scoring generation G_max */
    int32_t stall_gens;  /* G_stall (<= 0: no stall rule) */
    double tol;          /* stall when best_g - best_{g-G_stall} <= tol*max(1,|best_g|); < 0 off */
    double pc;           /* crossover probability */
    double pkb;          /* share of crossovers that are knowledge-based (else one-point) */
    double pm;           /* mutation probability per gene (random replacement in [0, N)) */
    int32_t scaling;     /* GPGA_SCALING_* */
    int32_t form;        /* GPGA_FORM_* */
    int32_t init;        /* GPGA_INIT_* */
    int32_t init_labels; /* uniform init range K0 (0 = N) */
    double tau_lo;       /* threshold init: tau range */
    double tau_hi;
    int32_t record;      /* keep per-generation best L, best labels and device timestamps */
    int32_t profile;     /* CUDA events in every generation: 1 around the dominant
                            kernel only, 2 around every stage */
    int32_t reserved[2];
} gpga_params;

/* Opaque GA run: population (two device buffers), fitness, derived forms of C,
 * generation counter, termination state, Philox seed. */
typedef struct gpga_ga gpga_ga;

/* Fill *p with the defaults above (P = 1000). */
GPGA_API int gpga_default_params(gpga_params *p);

/* Description of the last error on this thread ("" when none). */
GPGA_API const char *gpga_last_error(void);

/*
 * gpga_set_wait_budget -- failure detection; the paper has no counterpart.
 * Every wait of a kernel of this library on a barrier (the mbarrier hand-offs
 * of the tcgen05 pipelines of GPGA_FORM_TENSOR and of the Pearson prelude, and
 * the grid barrier of corr_clean_rmt's tridiagonal reduction) gives up once it
 * has spent `cycles` SM clock cycles: the kernel then stops issuing work, waits
 * (with the full default bound) for the tensor-core operations it has already
 * issued, releases its tensor memory and returns; the call reports
 * GPGA_ERR_TIMEOUT (ga_score, cluster_corr and corr_clean_rmt at once; a GA
 * run at ga_step with `done` or at ga_best) and the device context stays
 * usable. cycles = 0 makes every such
 * wait give up at its first check; cycles < 0 restores the default, 2^32
 * cycles (about 2 s at the maximum SM clock). Process-wide; applies to kernels
 * launched after the call, and a GA handle's generation graphs keep the budget
 * in force when ga_step first captured them. Returns GPGA_OK.
 */
GPGA_API int gpga_set_wait_budget(long long cycles);

/*
 * cluster_corr -- Pearson correlation matrix, Eq. 7 (Sec. 2.1; data normalised
 * to zero mean and unit variance below Eq. 2):
 *   C_ij = sum_t z_ti z_tj / sqrt(sum_t z_ti^2 sum_t z_tj^2),  z = R - column mean.
 * R: device, T x N FP64, row-major, leading dimension ld >= N. C: device, N x N
 * FP64 (written; diagonal exactly 1, symmetric, clamped to [-1, 1]).
 * Column statistics are FP64; the T-contraction runs in FP32 on normalised
 * columns with FP64 combination of short partial sums (|error| ~1e-7).
 * Errors: GPGA_ERR_ARG if T < 2, N < 2, N > GPGA_MAX_N or ld < N;
 * GPGA_ERR_DEGENERATE if a column holds a non-finite value or has zero variance
 * (C is then left unspecified). Blocks the host until the stream reaches the
 * end of the call (the degeneracy check is data-dependent).
 */
GPGA_API int cluster_corr(const double *R, int T, int N, int ld, double *C, void *stream);

/*
 * ga_score -- L_c of P configurations, Eq. 8 with n_s (Eq. 5) and c_s (Eq. 6):
 *   L_c(S) = 1/2 sum_{s: n_s>1} [ log(n_s/c_s) + (n_s-1) log((n_s^2-n_s)/(n_s^2-c_s)) ].
 * n_s^2 - c_s is accumulated directly as d_s = sum_{i,j in s} (1 - C_ij) (no
 * cancellation for tight clusters); c_s = n_s^2 - d_s. Domain edge (degenerate
 * data only): c_s floored at n_s 2^-40 and d_s at n_s(n_s-1) 2^-40.
 * labels: device, P x N int32 in [0, N), leading dimension ld >= N.
 * C: device, N x N FP64 (read; asymmetric input is used through (C + C^T)/2,
 * which leaves Eq. 6 unchanged). L: device, P FP64 (written).
 * form: GPGA_FORM_PLAIN, GPGA_FORM_TENSOR or GPGA_FORM_GATHER.
 * Errors: GPGA_ERR_ARG for sizes out of range or any label outside [0, N)
 * (found on the device; the matching L entries are NaN); GPGA_ERR_TIMEOUT if a
 * bounded wait of the tensor form's tcgen05 pipeline gave up (every L is then
 * NaN; see gpga_set_wait_budget). Blocks the host until the stream reaches the
 * end of the call.
 */
GPGA_API int ga_score(const int32_t *labels, int P, int N, int ld, const double *C, double *L,
                      int form, void *stream);

/*
 * ga_evolve -- one stateless GA generation after scoring (Algorithm 1: isolate
 * fittest, elitism, scaling, selection, crossover, mutation, replacement) from
 * population `pop` (device, P x N int32, row stride N) with fitness `L`
 * (device, P FP64) into `next` (device, P x N int32). Draws come from
 * Philox4x32-10 keyed by `seed` with counters (generation, index, block,
 * stream): SUS (g,0,0,1) word 0; child k (g,k,0,2) words crossover?,
 * knowledge-based?, anchor/cut; gene j (g,k,j/2,3) words (0,1) or (2,3).
 * Ranking: L descending, ties to the lower index; NaN ranks as -inf.
 * Knowledge-based crossover (reading of Sec. 3.1): the child is parent a with
 * parent b's cluster of anchor gene q merged into a's cluster of q.
 * perm (device, P int32, optional) receives the rank order; parents (device,
 * P - elite int32, optional) the selected parent of each child.
 * Uses p->P, elite, pc, pkb, pm, scaling; N is the gene count.
 * Asynchronous on `stream`.
 */
GPGA_API int ga_evolve(const int32_t *pop, const double *L, int N, const gpga_params *p,
                       uint64_t seed, int generation, int32_t *next, int32_t *perm,
                       int32_t *parents, void *stream);

/*
 * ga_init -- create a GA run on correlation matrix C: Algorithm 1 "create
 * initial population" and "evaluate fitness" of generation 0. The population
 * is P label vectors in the representation of Eq. 9 (gene j = the cluster of
 * stock j; 0-based labels, K = N), drawn uniformly (params.init =
 * GPGA_INIT_UNIFORM) or as correlation-threshold components
 * (GPGA_INIT_THRESHOLD), then scored with Eq. 8; the fittest is isolated and
 * the termination test of Table 3 is applied.
 * C: device, N x N FP64 (copied and derived from, so the caller may free it
 * on return). Allocates the population buffers, the forms of D = 1 - C that
 * params.form needs and the per-generation records; the handle owns them.
 * Asynchronous on `stream`, which the handle keeps for all later calls
 * (NULL: the handle creates its own non-blocking stream).
 * Errors: GPGA_ERR_ARG (NULL C or out, N < 2, N > GPGA_MAX_N, bad params),
 * GPGA_ERR_OOM, GPGA_ERR_CUDA. *out is NULL on error.
 */
GPGA_API int ga_init(const double *C, int N, const gpga_params *p, uint64_t seed, void *stream,
                     gpga_ga **out);

/*
 * ga_reset -- restart handle h on a new correlation matrix C (device, same N,
 * copied) and seed without reallocating: Algorithm 1 "create initial
 * population" (Eq. 9) and the scoring of generation 0 (Eq. 8), exactly as
 * ga_init. Clears the device error word. Asynchronous on the handle's stream.
 * Errors: GPGA_ERR_ARG (NULL h or C), GPGA_ERR_CUDA.
 */
GPGA_API int ga_reset(gpga_ga *h, const double *C, uint64_t seed);

/*
 * ga_step -- run up to `generations` iterations of the loop of Algorithm 1
 * (Sec. 3.1 operators: isolate fittest and elitism, scaling, stochastic
 * universal sampling, crossover, mutation, replacement; then "evaluate
 * fitness" with Eq. 8 and "determine if termination criteria are met" with
 * Table 3's generation limit and stall rule), all on the device with no host
 * round trip; generations after termination are no-ops. The generations run
 * as CUDA graphs captured on the first call.
 * Asynchronous when done == NULL. Otherwise waits for the stream, writes 1 to
 * *done if the run has terminated (else 0) and reports the device error word:
 * GPGA_ERR_TIMEOUT if a bounded device wait gave up (GPGA_FORM_TENSOR; the
 * affected fitness values are NaN). Errors: GPGA_ERR_ARG (NULL h,
 * generations < 0), GPGA_ERR_CUDA.
 */
GPGA_API int ga_step(gpga_ga *h, int generations, int *done);

/*
 * ga_best -- the output of the method (Sec. 4.2: the cluster configuration of
 * the fittest individual and its likelihood): the fittest configuration of the
 * current generation, canonically relabelled by first occurrence (0, 1, 2,
 * ...), with L_c (Eq. 8) re-scored in FP64 directly from the FP64 C (the
 * final re-score, independent of the form that ranked it).
 * labels: host or device, N int32 (optional); L: host or device, 1 FP64
 * (optional); generation: host (optional). Waits for the handle's stream.
 * The outputs are written in every case; the status then reports the device
 * error word of the run: GPGA_ERR_TIMEOUT if a bounded device wait gave up
 * since the last ga_init / ga_reset (GPGA_FORM_TENSOR). Errors: GPGA_ERR_ARG
 * (NULL h), GPGA_ERR_CUDA.
 */
GPGA_API int ga_best(gpga_ga *h, int32_t *labels, double *L, int *generation);

/*
 * ga_history -- per-generation records kept when params.record != 0: best L
 * (FP64), best labels (int32, as stored), the device clock (ns, %globaltimer),
 * the number of same-cluster gene pairs sum_s n_s (n_s - 1) / 2 summed over
 * the population (the work Eq. 6 needs; gather, plain and tensor forms) and
 * the number of non-singleton clusters summed over the population (tensor
 * form: the columns of the contraction), for generations 0..count-1,
 * count <= cap. Host pointers (each optional; t_ns needs room for cap + 1
 * values, the others for cap). t_ns[0] is taken at the start of ga_init /
 * ga_reset, t_ns[1 + g] at the end of generation g (so t_ns receives
 * count + 1 values). Waits for the stream.
 */
GPGA_API int ga_history(gpga_ga *h, double *best_L, int32_t *best_labels, int64_t *t_ns,
                        uint64_t *pairs, uint64_t *clusters, int cap, int *count);

/*
 * ga_kernel_times -- stage durations (ms, CUDA events on the handle's stream) of
 * the generations run by the most recent graph launch of ga_step, available
 * when params.profile != 0. Row g of ms (count x 4, count <= cap) holds
 * [evolve (gather form: the fused generation kernel), pair accumulation
 * (plain) or contraction (tensor), assembly, selection]. With profile = 1 only
 * the first generation of each graph launch is timed, and only its dominant
 * kernel (the other entries are 0; count is 1); with profile = 2 every stage
 * of every generation. Waits for the stream. GPGA_ERR_STATE without profile.
 */
GPGA_API int ga_kernel_times(gpga_ga *h, float *ms, int cap, int *count);

/*
 * ga_population -- copy the current population (P x N int32) and its fitness
 * (P FP64) to host or device buffers (each optional). Waits for the stream.
 */
GPGA_API int ga_population(gpga_ga *h, int32_t *pop, double *L);

/*
 * cluster_corr_ewma -- pre-processing upstream of C (no counterpart in the
 * hot path; Sec. 4.2 computes the covariance with an online exponentially
 * weighted filter): the EWMA-weighted Pearson correlation of R (device, T x N FP64,
 * leading dimension ld): rows weighted w_t = lambda^(T-1-t) (the newest row
 * weighs 1) in the means, the variances and the cross products; lambda = 1 is
 * cluster_corr. C (device, N x N FP64) written, diagonal 1. Errors as
 * cluster_corr, plus GPGA_ERR_ARG for lambda outside (0, 1]. Blocks the host
 * until the stream reaches the end of the call.
 */
GPGA_API int cluster_corr_ewma(const double *R, int T, int N, int ld, double lambda, double *C,
                               void *stream);

/*
 * corr_remove_market -- pre-processing upstream of C: removes the market mode
 * from a correlation matrix in place. The largest eigenpair (lambda_1, v) of C
 * (device, N x N FP64, symmetric) by power iteration from the uniform vector
 * in FP64 (until no component of v moves by more than 1e-14, at most
 * max_iters), then C <- C - lambda_1 v v^T renormalised to unit diagonal and
 * clamped to [-1, 1]. lambda1, iters (host, optional): the eigenvalue and the
 * iterations used. GPGA_ERR_DEGENERATE if a diagonal entry is not positive
 * after the removal. Blocks the host until the stream reaches the end.
 */
GPGA_API int corr_remove_market(double *C, int N, int max_iters, double *lambda1, int *iters,
                                void *stream);

/*
 * corr_clean_rmt -- pre-processing upstream of C: random-matrix cleaning
 * (Sec. 4.2: the eigenvalues in the Wishart range are removed in a
 * trace-preserving way) of `batch` correlation matrices in place. C: device,
 * batch x N x N FP64, each symmetric, estimated from T observations.
 * Per matrix: the eigen-decomposition C = sum_k lambda_k v_k v_k^T in FP64;
 * the noise set is the eigenvalues inside the Marchenko-Pastur range
 * [(1 - sqrt q)^2, (1 + sqrt q)^2], q = N / T, and they are replaced by their
 * mean m: C' = m I + sum_{k not noise} (lambda_k - m) v_k v_k^T (same trace);
 * then C <- C'_ij / sqrt(C'_ii C'_jj), clamped to [-1, 1], unit diagonal. A
 * matrix with an empty noise set is left unchanged. Two solvers: up to 32
 * stocks, or 33 to 127 stocks in batches of more than 4, the batch goes
 * through parallel cyclic Jacobi together (until every off-diagonal entry is
 * below 1e-14 ||A||_F); otherwise each matrix in turn is reduced to
 * tridiagonal form (Householder), its eigenvalues found by bisection and the
 * eigenvectors of the smaller of the kept and noise sets by inverse iteration
 * (C' then formed as C - sum_{noise} (lambda_k - m) v_k v_k^T when the noise
 * set is the smaller one).
 * eigvals (device, optional, batch x N): the input's eigenvalues, ascending.
 * n_noise (host, optional, batch): the noise-set sizes. sweeps (host,
 * optional): Jacobi sweeps run (the batch sweeps together); 0 when the
 * tridiagonal solver ran.
 * Errors: GPGA_ERR_ARG (NULL or host C, batch outside [1, 65535], N outside
 * [2, GPGA_MAX_N], T not positive, a non-finite entry; C is left unchanged),
 * GPGA_ERR_DEGENERATE (no Jacobi convergence in 40 sweeps, or a non-positive
 * diagonal after the cleaning), GPGA_ERR_TIMEOUT (a bounded grid barrier of
 * the tridiagonal reduction gave up, see gpga_set_wait_budget; C is left
 * unchanged). Device scratch: 3 batch n2^2 doubles (Jacobi, n2 = N rounded up
 * to even) or about 4.5 N^2 doubles (tridiagonal). Blocks the host until the
 * stream reaches the end of the call.
 */
GPGA_API int corr_clean_rmt(double *C, int batch, int N, double T, double *eigvals, int *n_noise,
                           int *sweeps, void *stream);

/*
 * cluster_mst -- minimum spanning tree of every cluster of one configuration
 * (the cluster trees the paper draws for the clusters it finds, Sec. 4.2), on
 * the correlation distance d_ij = sqrt(2 (1 - C_ij)) (the upper-triangle
 * entry C_ij, i < j, is the one read), by Prim's algorithm from each
 * cluster's first gene; ties go to the lower gene index.
 * C: device, N x N FP64 row-major; labels: device, N int32 in [0, N) (e.g. the
 * canonical labels from ga_best). edge_u, edge_v, edge_w: device, room for
 * N - 1 entries each: the edges (u < v, d) of the clusters in first-occurrence
 * order, each cluster's n_s - 1 edges in the order Prim adds them;
 * *n_edges (host, optional) = N - number of clusters. Singletons have no edge.
 * Errors: GPGA_ERR_ARG (NULL pointer, N outside [1, GPGA_MAX_N], a label
 * outside [0, N)). Blocks the host until the stream reaches the end of the call.
 */
GPGA_API int cluster_mst(const double *C, int N, const int32_t *labels, int32_t *edge_u,
                         int32_t *edge_v, double *edge_w, int *n_edges, void *stream);

/*
 * gpga_log_selftest -- diagnostic with no counterpart in the paper: evaluates
 * the library's table-driven fixed-point logarithm (Q62 mantissa log plus
 * e ln 2, the kernel of the Eq. 8 assembly) and CUDA's log on the same n
 * inputs. x: device, n positive normal doubles;
 * y_table, y_cuda: device, n doubles (written). Asynchronous.
 */
GPGA_API int gpga_log_selftest(const double *x, int n, double *y_table, double *y_cuda,
                               void *stream);

/*
 * ga_score_noalloc -- the paper has no counterpart to this entry point. Same
 * result as ga_score(..., GPGA_FORM_GATHER, ...), for callers that must not
 * have the library allocate device memory while scoring (a host whose own
 * pool allocator already owns nearly all GPU memory, or a latency-critical
 * loop that forbids allocator calls). Its working memory is a fixed file-scope
 * __device__ array of about 4.3 MiB that every GPU loading the library holds
 * until the process exits; the call makes no cudaMalloc, cudaFree or other
 * allocating call. Set-up: the first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) once, with that device current, and
 * keeps it for the process; make that first call before any stream capture.
 * A cudaDeviceReset invalidates the address, so do not call this entry point
 * on a device after resetting that device in the same process. The caller
 * passes inputs and
 * outputs exactly as for ga_score: labels (device, P x N int32 in [0, N),
 * leading dimension ld >= N), C (device, N x N FP64), L (device, P FP64,
 * written).
 * Limits: 2 <= N <= 1024 (GPGA_ERR_ARG beyond), 1 <= P <= 2^24.
 * All calls share the one array and it keeps the previous call's contents
 * (the call clears what must start at zero): calls that overlap on the GPU,
 * from different streams or threads, race and must be serialised by the
 * caller. Errors as ga_score; blocks the host until the stream reaches the end
 * of the call.
 */
GPGA_API int ga_score_noalloc(const int32_t *labels, int P, int N, int ld, const double *C,
                              double *L, void *stream);

/*
 * ga_free -- release handle h (from ga_init) with all its device memory, its
 * graphs and events, and its stream if it created one; the end of the run of
 * Algorithm 1 (no counterpart in the paper beyond that). Waits for the
 * handle's stream first. NULL is a no-op. Always returns GPGA_OK.
 */
GPGA_API int ga_free(gpga_ga *h);

/* ------------------------------------------------------------------------
 * Batch: many independent GA runs (e.g. one per sliding window of a returns
 * series, each window's C being the input of one run as in Sec. 4.2) advanced
 * together. Each run is the single-run gather form with its own C, N and
 * seed: same parameters as ga_init (p->form must be GPGA_FORM_GATHER; record
 * and profile must be 0). A run of N < 448 genes gives bit-for-bit the result
 * of ga_init + ga_step on that run alone. From 448 genes up a single run
 * scores Eq. 8 as a sum of per-cluster fixed-point terms (so that it can score
 * children by delta from a parent), while a batch run scores every child from
 * scratch in the one-log product form; the two agree to about 1e-12 in L, so
 * such a run can take a different path from the single run once two
 * individuals' order depends on the last bits. One generation of all runs
 * is two kernel launches, captured in a CUDA graph; the launch shape of the fused
 * generation kernel (warps per CTA, CTAs) is chosen at init by timing the
 * candidates on the runs themselves.
 * ------------------------------------------------------------------------ */
typedef struct gpga_batch gpga_batch;

/*
 * ga_batch_init -- create `runs` runs and score their initial populations.
 * C[k]: device pointer (host array of `runs` pointers) to run k's correlation
 *   matrix, FP64 row-major with leading dimension ldc[k] (ldc NULL: N[k]).
 * cols: NULL, or host array of `runs` device pointers; cols[k] (if not NULL)
 *   holds N[k] int32 row/column indices into C[k], and run k works on the
 *   submatrix C[k][cols[k], cols[k]] (a column subset of a larger window).
 *   The indices are not checked on the device: each must lie in [0, ldc[k])
 *   and C[k] must have that many rows.
 * N[k] in [2, GPGA_MAX_N]; seeds[k] is run k's Philox key. The inputs are
 * copied: the caller may free them after the call returns.
 * Errors: GPGA_ERR_ARG (bad sizes, NULL arrays, unsupported options),
 * GPGA_ERR_OOM, GPGA_ERR_CUDA. Blocks until initialisation and the launch-shape
 * tuning have finished.
 */
GPGA_API int ga_batch_init(int runs, const double *const *C, const int *ldc,
                           const int32_t *const *cols, const int *N, const gpga_params *p,
                           const uint64_t *seeds, void *stream, gpga_batch **out);

/* ga_batch_step -- advance every run that has not terminated by up to
 * `generations` generations (terminated runs do no work). active (optional,
 * host): number of runs not yet terminated, read after a synchronisation. */
GPGA_API int ga_batch_step(gpga_batch *h, int generations, int *active);

/* ga_batch_status -- per run (host arrays of length runs, each optional): the
 * generation scored last, the termination flag, the best L of that
 * generation. Synchronises the stream. */
GPGA_API int ga_batch_status(gpga_batch *h, int32_t *generation, int32_t *done, double *best);

/* ga_batch_best -- as ga_best for run `run`: canonical labels (N[run] int32),
 * L re-scored in FP64, generation; host or device pointers. */
GPGA_API int ga_batch_best(gpga_batch *h, int run, int32_t *labels, double *L, int *generation);

/* ga_batch_tuning -- the launch shape the tuner chose and its time per
 * generation launch in ms (each output optional). */
GPGA_API int ga_batch_tuning(gpga_batch *h, int *warps_per_cta, int *ctas, float *ms);

/* ga_batch_population -- the current population of run `run` (host, P x N
 * int32) and its fitness (host, P FP64), each optional; synchronises. */
GPGA_API int ga_batch_population(gpga_batch *h, int run, int32_t *pop, double *L);

/*
 * ga_island_init -- the island variant the paper proposes (Sec. 5.2 and 6): `islands`
 * populations of the same C (device, N x N FP64, copied), island k seeded
 * with seed + k, advanced together like a batch (ga_batch_step, _status,
 * _best, _population, _free apply). Migration on a ring: when the generation
 * being built is a multiple of migrate_every, the `migrants` best individuals
 * of island k (its elites, slots 0..migrants-1 of the new population) replace
 * the last `migrants` children of island (k + 1) mod islands, with their
 * fitness, before selection; islands that terminated or stand at another
 * generation take no part. Requires islands >= 2, migrate_every >= 1,
 * 1 <= migrants <= elite and 2 migrants <= P (else GPGA_ERR_ARG).
 */
GPGA_API int ga_island_init(int islands, const double *C, int N, const gpga_params *p,
                            uint64_t seed, int migrate_every, int migrants, void *stream,
                            gpga_batch **out);

/* ga_batch_free -- release the batch and all its device memory (NULL: no-op). */
GPGA_API int ga_batch_free(gpga_batch *h);

/* ------------------------------------------------------------------------
 * Serving: a request loop over a fleet of runs. A request is one
 * correlation window (host N x N FP64 C, copied at submission) with its own
 * seed; it waits in a FIFO queue until a run slot and device memory are free
 * (admission by memory: the run's whole footprint must fit the budget and
 * leave the reserve free), then runs on the device, its population resident
 * across generations, alongside every other admitted request, until it
 * terminates (max_gens or the stall rule). Its result is the same as that of
 * ga_init + ga_step + ga_best on its C alone. Single-threaded: one host
 * thread drives a server.
 * ------------------------------------------------------------------------ */
typedef struct gpga_server gpga_server;

/* serve_create -- max_runs concurrent runs of N <= max_n; mem_budget: bytes
 * of run memory the server may hold (0: free device memory less a reserve of
 * min(1 GiB, 10%)). Parameters as ga_batch_init. */
GPGA_API int serve_create(const gpga_params *p, int max_runs, int max_n, size_t mem_budget,
                          void *stream, gpga_server **out);

/* serve_submit -- queue one request: C host pointer, N x N FP64 row-major
 * (copied), 2 <= N <= max_n; *id receives the request's id. No GPU work. */
GPGA_API int serve_submit(gpga_server *h, const double *C, int N, uint64_t seed, long long *id);

/* serve_tick -- one turn k of the loop: wait until the GPU has finished
 * turn k-2, collect the results copied out at turn k-1, retire the runs turn
 * k-2 left terminated (FP64 re-score and copy-out enqueued, memory freed in
 * stream order), admit queued requests while slots and memory allow, then
 * enqueue `generations` generations of every admitted run and return without
 * waiting for them: the GPU works on turn k-1 while the host prepares turn k.
 * A result is collected two or three turns after its run terminates.
 * active/queued (optional): runs in this turn's table and requests still
 * waiting. */
GPGA_API int serve_tick(gpga_server *h, int generations, int *active, int *queued);

/* serve_result -- 1 and the result if request `id` has finished (labels:
 * host, N int32 canonical; L; generation; times: host, 2 doubles = seconds
 * queued before admission and seconds from admission to retirement; each
 * optional), and the result is then released; 0 if it is still queued or
 * running; GPGA_ERR_ARG for an unknown or already collected id. */
GPGA_API int serve_result(gpga_server *h, long long id, int32_t *labels, double *L,
                          int *generation, double *times);

/* serve_stats -- run memory in use, the budget, requests completed so far,
 * the generation kernel's launch shape, and timing (host, 6 doubles: ticks,
 * host seconds waiting for the GPU, host seconds of tick work, GPU ms of the
 * generation graphs of ticks already waited for, fleet generations launched,
 * sum over those generations of the work items); each optional. */
GPGA_API int serve_stats(gpga_server *h, size_t *bytes_in_use, size_t *budget,
                         long long *completed, int *warps_per_cta, int *ctas, double *timing);

/* serve_free -- release the server, its queue, results and device memory. */
GPGA_API int serve_free(gpga_server *h);

#ifdef __cplusplus
}
#endif

#endif /* GPGA_H */
