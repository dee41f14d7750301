// score_tc.cuh -- tensor-core form of the likelihood contraction (sm_103a
// tcgen05): host-side interface used by the ABI layer.
#pragma once

#include "gpga_internal.cuh"

namespace gpga {

// device work buffers of the tensor form, carved from a caller block
struct TcWork {
    int32_t *colmap = nullptr; // P x Np: compact column of gene i's cluster, or -1
    int32_t *kcount = nullptr; // P: non-singleton clusters per individual
    int32_t *base = nullptr;   // P + 1: exclusive prefix of kcount
    int32_t *coltab = nullptr; // columns: (individual, label) per compact column
    int32_t *ncols = nullptr;  // 1: total columns
    int maxcols = 0;
};

// bytes needed by tc_carve for (N, Np, P)
size_t tc_scratch_bytes(int N, int Np, int P);
// carve the buffers from base + *off (base == nullptr: size only), advancing *off
void tc_carve(TcWork *w, int N, int Np, int P, size_t *off, char *base);

// y_i = sum_j D_ij [s_j = s_i] for every gene of every individual, written to
// acc (P x Np FP32), from the BF16 hi/lo split of D on the tensor cores
template <typename LabT>
int tc_score(TcWork *w, const __nv_bfloat16 *Dhi, const __nv_bfloat16 *Dlo, int Np,
             const LabT *const *lab2, int ldl, int sel_off, int P, int N, float *acc,
             const DevState *st, cudaStream_t s);

} // namespace gpga
