// Translation unit: the FP32 CUDA-core evaluation kernels of one table type
// (NBVH_TU_TABLE: 0 FP32, 1 FP16, 2 BF16), both schedules.
#include "eval_plain.cuh"

namespace nbvh {
#if NBVH_TU_TABLE == 0
using TableT = float;
#elif NBVH_TU_TABLE == 1
using TableT = __half;
#else
using TableT = __nv_bfloat16;
#endif
template cudaError_t launch_plain_t<TableT, false>(int, const EvalArgs&, int64_t, cudaStream_t);
template cudaError_t launch_plain_t<TableT, true>(int, const EvalArgs&, int64_t, cudaStream_t);
}  // namespace nbvh
