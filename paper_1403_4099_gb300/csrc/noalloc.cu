// noalloc.cu -- ga_score_noalloc: the gather-form population score with its
// working memory in a fixed device array instead of cudaMallocAsync.
//
// Some callers cannot let this library allocate device memory while scoring:
// a host application whose own pool allocator has reserved nearly all of the
// GPU up front, a latency-critical serving loop that forbids allocator calls
// (they can block on device-wide synchronisation or fail under fragmentation),
// or code running where a CUDA allocation would be illegal or unwelcome. For
// them this entry point uses a file-scope __device__ array of fixed size as
// scratch; it calls no cudaMalloc, cudaFree or other allocating routine.
#include <mutex>

#include "gpga_internal.cuh"

namespace gpga {

// largest N the fixed scratch holds
constexpr int NOALLOC_MAX_N = 1024;
constexpr int NOALLOC_MAX_NP = (NOALLOC_MAX_N + 63) & ~63;

// layout of the scratch: int32 fixed-point D, log tables, two flags
constexpr size_t NA_DFIX = 0;
constexpr size_t NA_LOG = NA_DFIX + (size_t)NOALLOC_MAX_NP * NOALLOC_MAX_NP * sizeof(int32_t);
constexpr size_t NA_FLAGS =
    NA_LOG + ((2 * LOG_TAB + (size_t)NOALLOC_MAX_N + 1) * sizeof(double) + 255) / 256 * 256;
constexpr size_t NA_BYTES = NA_FLAGS + 256;

// Every device that loads the library holds this array (about 4.3 MiB) until
// the process exits. In host code the name is only a host-side stand-in; the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Set-up: the device address of g_noalloc_scratch per device ordinal, looked
// up once with that device current and kept for the process (a
// cudaDeviceReset of that device invalidates it).
static unsigned char *noalloc_base(int dev, int *rc)
{
    static std::mutex mu;
    static unsigned char *base[64] = {nullptr};
    std::lock_guard<std::mutex> lock(mu);
    if (!base[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *rc = cuda_error(e, "ga_score_noalloc: cudaGetSymbolAddress", __FILE__, __LINE__);
            return nullptr;
        }
        base[dev] = static_cast<unsigned char *>(p);
    }
    *rc = GPGA_OK;
    return base[dev];
}

} // namespace gpga

using namespace gpga;

extern "C" GPGA_API int ga_score_noalloc(const int32_t *labels, int P, int N, int ld,
                                         const double *C, double *L, void *stream)
{
    clear_error();
    if (!labels || !C || !L) return set_error(GPGA_ERR_ARG, "ga_score_noalloc: NULL pointer");
    if (N < 2 || N > NOALLOC_MAX_N || P < 1 || P > (1 << 24) || ld < N)
        return set_error(GPGA_ERR_ARG,
                         "ga_score_noalloc: P=%d N=%d ld=%d out of range (N must be in [2, %d])",
                         P, N, ld, NOALLOC_MAX_N);
    int rc = prepare_device();
    if (rc) return rc;
    int dev = 0;
    GPGA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(GPGA_ERR_ARG, "ga_score_noalloc: device %d", dev);
    unsigned char *base = noalloc_base(dev, &rc);
    if (!base) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int Np = pad_n(N);
    int32_t *Dfix = reinterpret_cast<int32_t *>(base + NA_DFIX);
    double *logtab = reinterpret_cast<double *>(base + NA_LOG);
    int *err = reinterpret_cast<int *>(base + NA_FLAGS); // [0] label error, [1] diagonal flag
    // the scratch keeps the previous call's contents: clear the flags
    GPGA_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
    // only the fixed-point D (with its diagonal flag) and the log tables: the
    // gather form reads nothing else
    rc = launch_fleet_prep(C, N, nullptr, N, Np, nullptr, Dfix, err + 1, s);
    if (!rc) rc = launch_logtab(logtab, N, s);
    if (rc) return rc;
    const int32_t *lab2[2] = {labels, labels};
    rc = launch_gather_score<int32_t>(lab2, ld, 0, P, N, Np, Dfix, err + 1, logtab, L, err,
                                      nullptr, nullptr, ScoreTab{}, s);
    if (rc) return rc;
    int herr = 0;
    GPGA_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GPGA_CUDA(cudaStreamSynchronize(s));
    if (herr & 1)
        return set_error(GPGA_ERR_ARG, "ga_score_noalloc: a label lies outside [0, N) (its L is NaN)");
    return GPGA_OK;
}
