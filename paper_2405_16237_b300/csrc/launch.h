// Launchers defined in the library's other CUDA translation units (one per
// table type and mode, compiled in parallel); nbvh_lib.cu calls them and must
// not instantiate the kernels itself.
#pragma once
#include "eval_tc.cuh"
#include "eval_ws.cuh"
#include "train_tc.cuh"

namespace nbvh {

#define NBVH_EXTERN_TABLE_TYPES(X) X(float) X(__half) X(__nv_bfloat16)

#define NBVH_EXTERN_TC(T)                                                                                          \
  extern template cudaError_t launch_tc_tm<T, 0>(const nbvh_model_desc*, const EvalArgs&, int64_t, const TcPlan&, \
                                                 cudaStream_t);                                                   \
  extern template cudaError_t launch_tc_tm<T, 1>(const nbvh_model_desc*, const EvalArgs&, int64_t, const TcPlan&, \
                                                 cudaStream_t);                                                   \
  extern template cudaError_t launch_tc_tm<T, 2>(const nbvh_model_desc*, const EvalArgs&, int64_t, const TcPlan&, \
                                                 cudaStream_t);                                                   \
  extern template cudaError_t launch_plain_t<T, false>(int, const EvalArgs&, int64_t, cudaStream_t);              \
  extern template cudaError_t launch_plain_t<T, true>(int, const EvalArgs&, int64_t, cudaStream_t);               \
  extern template cudaError_t launch_train_t<T>(bool, const nbvh_model_desc*, const TrainArgs&, cudaStream_t);     \
  extern template cudaError_t launch_ws_t<T>(const nbvh_model_desc*, const EvalArgs&, cudaStream_t);
NBVH_EXTERN_TABLE_TYPES(NBVH_EXTERN_TC)
#undef NBVH_EXTERN_TC
#undef NBVH_EXTERN_TABLE_TYPES

cudaError_t launch_bwd_tc(const nbvh_model_desc* d, const TcBwdArgs& a, cudaStream_t s);
// W0^T of the streamed backward (bwd_w0_streamed) into img (Kp * W * 2 bytes)
cudaError_t launch_bwd_image(const nbvh_model_desc* d, const float* mlp, uint8_t* img, cudaStream_t s);
cudaError_t launch_wg_tc(bool bf16, int W, const WgTcArgs& a, cudaStream_t s);

}  // namespace nbvh
