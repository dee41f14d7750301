// score_tc.cuh -- tensor-core form of the likelihood contraction (sm_103a
// tcgen05): host-side interface used by the ABI layer.
#pragma once

#include "gpga_internal.cuh"

namespace gpga {

// device work buffers of the tensor form, carved from a caller block
struct TcWork {
    uint32_t *bits = nullptr;          // maxcols x (Np/32): membership bitmask per column
    int32_t *col_n = nullptr;          // maxcols: cluster size
    long long *dfix = nullptr;         // maxcols: d_s in fixed point 2^-b (exact sums)
    int32_t *colbase = nullptr;        // P: first column of individual p
    int32_t *kcount = nullptr;         // P: non-singleton clusters of individual p
    unsigned *ncols = nullptr;         // 1: columns used (reserved by atomics)
    int *err = nullptr;                // 1: bounded-wait timeout flag
    int maxcols = 0;
};

// bytes needed by tc_carve for (N, Np, P)
size_t tc_scratch_bytes(int N, int Np, int P);
// carve the buffers from base + *off (base == nullptr: size only), advancing *off
void tc_carve(TcWork *w, int N, int Np, int P, size_t *off, char *base);

// the contraction d_s = 1^T D_ss 1 for every non-singleton cluster on the
// tensor cores (one-hot S in BF16 x D split into BF16 hi + lo, FP32
// accumulation in TMEM): columns + bitmasks, then the tcgen05 kernel.
// clusters (optional, stateful): per-generation count of non-singleton clusters
template <typename LabT>
int tc_contract(TcWork *w, const __nv_bfloat16 *Dhi, const __nv_bfloat16 *Dlo, int Np,
                const LabT *const *lab2, int ldl, int sel_off, int P, int N, int *err,
                const DevState *st, unsigned long long *pairs, unsigned long long *clusters,
                cudaStream_t s);
// the fixed-point Eq. 8 assembly over each individual's columns
template <typename LabT>
int tc_finish(TcWork *w, const LabT *const *lab2, int ldl, int sel_off, int P, int N,
              const double *logtab, double *L, int *err, const DevState *st, cudaStream_t s);

} // namespace gpga
