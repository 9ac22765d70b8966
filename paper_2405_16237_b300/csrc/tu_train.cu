// Translation unit: the FP32 CUDA-core training kernels (forward with stored
// activations, backward with the encoding's scatter-add) of one table type
// (NBVH_TU_TABLE: 0 FP32, 1 FP16, 2 BF16).
#include "train.cuh"

namespace nbvh {
#if NBVH_TU_TABLE == 0
using TableT = float;
#elif NBVH_TU_TABLE == 1
using TableT = __half;
#else
using TableT = __nv_bfloat16;
#endif
template cudaError_t launch_train_t<TableT>(bool, const nbvh_model_desc*, const TrainArgs&, cudaStream_t);
}  // namespace nbvh
