// Translation unit: the tensor-core training kernels (MLP adjoint with the
// encoding's scatter-add, first-layer weight gradient).
#include "train_tc.cuh"

namespace nbvh {
namespace {
template <int F, int W>
cudaError_t launch_bwd_tc_fw(bool bf16, const TcBwdArgs& a, cudaStream_t s) {
  const TcBwdLayout lay = tc_bwd_layout(a.gp.n_inputs, W, a.n_hidden, a.w0t_image != nullptr);
  if (lay.total > kBwdSmemMax || lay.ncols > 512) return cudaErrorInvalidConfiguration;
  auto kern = bf16 ? train_backward_tc<F, W, true> : train_backward_tc<F, W, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lay.total));
  if (e != cudaSuccess) return e;
  constexpr int threads = bwd_threads<W>();
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, lay.total);
  if (e != cudaSuccess) return e;
  // co-resident CTAs must fit the SM's 512 TMEM columns together
  per_sm = std::min(per_sm, int(512 / lay.ncols));
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (a.n + kTcM - 1) / kTcM;
  int64_t grid = int64_t(sm_count()) * per_sm;
  if (tiles < grid) grid = tiles;
  if (grid < 1) return cudaSuccess;
  kern<<<unsigned(grid), threads, lay.total, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <int F>
cudaError_t launch_bwd_tc_f(bool bf16, int W, const TcBwdArgs& a, cudaStream_t s) {
  switch (W) {
    case 32: return launch_bwd_tc_fw<F, 32>(bf16, a, s);
    case 64: return launch_bwd_tc_fw<F, 64>(bf16, a, s);
    case 128: return launch_bwd_tc_fw<F, 128>(bf16, a, s);
  }
  return cudaErrorInvalidConfiguration;
}

}  // namespace

cudaError_t launch_bwd_image(const nbvh_model_desc* d, const float* mlp, uint8_t* img, cudaStream_t s) {
  const int K = d->n_samples * d->n_levels * d->n_features, Kp = (K + 15) & ~15;
  const int64_t n = int64_t(Kp) * d->width;
  const int blocks = int(std::min<int64_t>((n + 255) / 256, int64_t(sm_count()) * 4));
  if (d->mlp_prec == NBVH_BF16)
    bwd_w0t_image_kernel<true><<<blocks, 256, 0, s>>>(mlp, K, Kp, d->width, d->n_samples, d->n_levels,
                                                      d->n_features, img);
  else
    bwd_w0t_image_kernel<false><<<blocks, 256, 0, s>>>(mlp, K, Kp, d->width, d->n_samples, d->n_levels,
                                                       d->n_features, img);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bwd_tc(const nbvh_model_desc* d, const TcBwdArgs& a, cudaStream_t s) {
  const bool bf16 = d->mlp_prec == NBVH_BF16;
  switch (d->n_features) {
    case 1: return launch_bwd_tc_f<1>(bf16, d->width, a, s);
    case 2: return launch_bwd_tc_f<2>(bf16, d->width, a, s);
    case 4: return launch_bwd_tc_f<4>(bf16, d->width, a, s);
    case 8: return launch_bwd_tc_f<8>(bf16, d->width, a, s);
  }
  return cudaErrorInvalidValue;
}


namespace {
template <int W>
cudaError_t launch_wg_tc_w(bool bf16, const WgTcArgs& a, cudaStream_t s) {
  const uint32_t smem = wg_tc_smem(a.Kp, W);
  if (smem > 227 * 1024 || wg_tc_tiles(a.Kp) * W > 512) return cudaErrorInvalidConfiguration;
  auto kern = bf16 ? weight_grad_tc<W, true> : weight_grad_tc<W, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const int it = wg_tc_items(a.Kp, W);
  const int64_t chunks = (a.n + it - 1) / it;
  int64_t grid = sm_count();
  if (chunks < grid) grid = chunks;
  if (grid < 1) return cudaSuccess;
  kern<<<unsigned(grid), kWgTcThreads, smem, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wg_tc(bool bf16, int W, const WgTcArgs& a, cudaStream_t s) {
  switch (W) {
    case 32: return launch_wg_tc_w<32>(bf16, a, s);
    case 64: return launch_wg_tc_w<64>(bf16, a, s);
    case 128: return launch_wg_tc_w<128>(bf16, a, s);
  }
  return cudaErrorInvalidConfiguration;
}

}  // namespace nbvh
