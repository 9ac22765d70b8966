// Translation unit: the fused gather + tensor-core MLP kernels of one table
// type (NBVH_TU_TABLE: 0 FP32, 1 FP16, 2 BF16) and one mode (NBVH_TU_MODE:
// 0 segment list, 1 query, 2 training forward). The build compiles this file
// once per combination so the instantiations compile in parallel.
#include "eval_tc.cuh"
#include "eval_ws.cuh"

namespace nbvh {
#if NBVH_TU_TABLE == 0
using TableT = float;
#elif NBVH_TU_TABLE == 1
using TableT = __half;
#else
using TableT = __nv_bfloat16;
#endif
template cudaError_t launch_tc_tm<TableT, NBVH_TU_MODE>(const nbvh_model_desc*, const EvalArgs&, int64_t,
                                                        const TcPlan&, cudaStream_t);
#if NBVH_TU_MODE == 1
template cudaError_t launch_ws_t<TableT>(const nbvh_model_desc*, const EvalArgs&, cudaStream_t);
#endif
}  // namespace nbvh
