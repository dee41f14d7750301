// score_tc.cu -- tensor-core form (placeholder until the tcgen05 kernel lands)
#include "score_tc.cuh"

namespace gpga {

size_t tc_scratch_bytes(int, int, int) { return 0; }
void tc_carve(TcWork *, int, int, int, size_t *, char *) {}
int prepare_tc_kernels(int) { return GPGA_OK; }

template <typename LabT>
int tc_score(TcWork *, const __nv_bfloat16 *, const __nv_bfloat16 *, int, const LabT *const *,
             int, int, int, int, float *, const DevState *, cudaStream_t)
{
    return set_error(GPGA_ERR_ARG, "tensor form not available in this build");
}

template int tc_score<uint16_t>(TcWork *, const __nv_bfloat16 *, const __nv_bfloat16 *, int,
                                const uint16_t *const *, int, int, int, int, float *,
                                const DevState *, cudaStream_t);
template int tc_score<int32_t>(TcWork *, const __nv_bfloat16 *, const __nv_bfloat16 *, int,
                               const int32_t *const *, int, int, int, int, float *,
                               const DevState *, cudaStream_t);

} // namespace gpga
