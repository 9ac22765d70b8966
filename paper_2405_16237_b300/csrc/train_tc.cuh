// S8 backward on the tensor cores: the MLP adjoint as tcgen05 MMAs with the
// gradients in TMEM, then the adjoint of the encoding (trilinear scatter-add
// into the FP32 table gradient) straight from the dL/dfeatures accumulator.
#pragma once
#include "eval_tc.cuh"
#include "train.cuh"

namespace nbvh {

constexpr int kAggMaxRes = 64;  // warp aggregation of scatter atomics up to this level resolution

struct TcBwdArgs {
  GridParams gp;
  const float* mlp;
  int32_t n_hidden, n_out;
  RayPtrs rays;
  const int32_t* leaf;
  const int32_t* order;   // item -> ray as in the forward; nullptr: item = ray
  const float* t0;
  const float* t1;
  int64_t n;
  const float* G;         // [n][n_out] dL/d(raw), times the loss scale (by item)
  const uint16_t* H16;    // [n_hidden][n][W] hidden activations of the forward
  uint16_t* dZT;          // [n_hidden][W][ld] pre-activation gradients, neuron-major (out)
  int64_t ld;
  float* grad_table;      // FP32 [entries][F]
  const uint8_t* w0t_image;  // W0^T in its shared-memory operand layout, copied
                             // 128 features at a time (nullptr: staged whole)
};

// TMEM columns: [0, W) accumulator of dH; [W, W + W/2) the current A operand
// (dL/dout padded to 16, then dZ); [2W, 2W + 128) a 128-feature chunk of
// dL/dfeatures. Shared memory: the transposed weights as B operands; W0^T
// whole, or (streamed) one 128-feature chunk of it at a time.
struct TcBwdLayout {
  int Kp;
  uint32_t col_a, col_x, ncols;
  uint32_t w0t_off, wht_off, wot_off, row_off, u_off, bar_off, total;
};

__host__ __device__ inline TcBwdLayout tc_bwd_layout(int K, int W, int n_hidden, bool streamed) {
  TcBwdLayout L;
  L.Kp = (K + 15) & ~15;
  L.col_a = uint32_t(W);
  L.col_x = uint32_t(2 * W);
  uint32_t nc = 32;
  while (nc < L.col_x + 128u) nc <<= 1;
  L.ncols = nc;
  uint32_t off = 0;
  auto take = [&](uint32_t bytes) {
    const uint32_t o = off;
    off = (off + bytes + 127u) & ~127u;
    return o;
  };
  L.w0t_off = take(uint32_t(streamed ? (L.Kp < 128 ? L.Kp : 128) : L.Kp) * W * 2);
  L.wht_off = take(uint32_t(n_hidden - 1) * W * W * 2);
  L.wot_off = take(uint32_t(W) * 16 * 2);
  L.row_off = take(kTcM * 36);  // ray index, t0, t1, origin, direction per row
  L.u_off = take(NBVH_MAX_SAMPLES * 4);
  L.bar_off = take(64);
  L.total = off + 128;
  return L;
}

constexpr uint32_t kBwdSmemMax = 227u * 1024u;

// Whether the backward streams W0^T: its whole transpose does not fit the
// shared-memory budget next to the other operands (e.g. K = 2048 at W = 64).
__host__ __device__ inline bool bwd_w0_streamed(int K, int W, int n_hidden) {
  return tc_bwd_layout(K, W, n_hidden, false).total > kBwdSmemMax;
}

// Threads of the backward kernel: 512 lets two CTAs share an SM (2 x 256 TMEM
// columns) so one CTA's scatter overlaps the other's MMA chain; W = 128 needs
// 512 columns and runs one 1024-thread CTA per SM.
template <int W>
__host__ __device__ constexpr int bwd_threads() {
  return W >= 128 ? 1024 : 512;
}

// Level-major dL/dfeatures chunks: the dX MMA takes W0's rows permuted so one
// level's N*F features are adjacent and a 128-column chunk holds whole levels.
// The scatter then walks each ray through one level. Up to two features.
__host__ __device__ inline bool bwd_level_major(int n_samples, int F) {
  const int nf = n_samples * F;
  return F <= 2 && nf % 16 == 0 && 128 % nf == 0;
}

// Row r of W0^T (B operand of the dX MMA, K-major, rows = features): the
// feature of input order k*L*F + l*F + f, permuted level-major
// (l*N*F + k*F + f) when the scatter walks rays level by level.
__host__ __device__ inline int bwd_w0_feature(int r, int K, int NS, int L, int F, bool lmaj) {
  if (!lmaj || r >= K) return r;
  const int nf = NS * F;
  const int l = r / nf, rem = r - l * nf;
  return (rem / F) * (L * F) + l * F + rem % F;
}

// W0^T of the FP32 master weights in the backward's operand layout, written
// to global memory once per backward call for the streamed form.
template <bool BF16>
__global__ void bwd_w0t_image_kernel(const float* __restrict__ W0, int K, int Kp, int W, int NS, int L, int F,
                                     uint8_t* __restrict__ img) {
  using OT = OpType<BF16>;
  const bool lmaj = bwd_level_major(NS, F);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < int64_t(Kp) * W;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(i / W), k = int(i - int64_t(r) * W);
    const float v = r < K ? __ldg(W0 + size_t(k) * K + bwd_w0_feature(r, K, NS, L, F, lmaj)) : 0.0f;
    *reinterpret_cast<typename OT::T*>(img + op_offset(r, k, W)) = OT::one(v);
  }
}

// Adds F gradient values to an FP32 table entry (vector reductions where the
// entry width allows them).
template <int F>
__device__ __forceinline__ void add_entry(float* dst, const float* v) {
  if constexpr (F == 2) {
    atomicAdd(reinterpret_cast<float2*>(dst), make_float2(v[0], v[1]));
  } else if constexpr (F % 4 == 0) {
#pragma unroll
    for (int ff = 0; ff < F; ff += 4)
      atomicAdd(reinterpret_cast<float4*>(dst + ff), make_float4(v[ff], v[ff + 1], v[ff + 2], v[ff + 3]));
  } else {
#pragma unroll
    for (int ff = 0; ff < F; ++ff) atomicAdd(dst + ff, v[ff]);
  }
}

// Moves the eight corner sums of a cell to the cell d steps along one axis
// (BIT = 1, 2, 4 for x, y, z): shared vertices keep their sums, the others
// (already added to the table) restart at zero.
template <int F, int BIT>
__device__ __forceinline__ void shift_corners(float (&acc)[8][F], int d) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (q & BIT) continue;
#pragma unroll
    for (int ff = 0; ff < F; ++ff) {
      const float a0 = acc[q][ff], a1 = acc[q | BIT][ff];
      acc[q][ff] = d == 0 ? a0 : (d == 1 ? a1 : 0.0f);
      acc[q | BIT][ff] = d == 0 ? a1 : (d == -1 ? a0 : 0.0f);
    }
  }
}

// Adds the corner values v of a cell vertex (table entry key; 0xffffffff: none)
// to the table; when the whole warp holds the same key (coarse levels), one
// lane adds the warp's sum.
template <int F>
__device__ __forceinline__ void add_vertex_warp(float* gt, uint32_t key, float* v, bool aggregate, int lane) {
  int same = 0;
  if (aggregate) __match_all_sync(0xffffffffu, key, &same);
  if (same) {
    if (key != 0xffffffffu) {
#pragma unroll
      for (int ff = 0; ff < F; ++ff) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[ff] += __shfl_xor_sync(0xffffffffu, v[ff], o);
      }
      if (lane == 0) add_entry<F>(gt + size_t(key) * F, v);
    }
  } else if (key != 0xffffffffu) {
    add_entry<F>(gt + size_t(key) * F, v);
  }
}

template <bool BF16>
__device__ __forceinline__ float from16(uint16_t v) {
  if constexpr (BF16) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(&v));
  } else {
    return __half2float(*reinterpret_cast<const __half*>(&v));
  }
}

template <int F, int W, bool BF16>
__global__ void __launch_bounds__(bwd_threads<W>(), 1024 / bwd_threads<W>()) train_backward_tc(TcBwdArgs a) {
  using OT = OpType<BF16>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int K = a.gp.n_inputs;
  const int L = a.gp.n_levels;
  const int NS = a.gp.n_samples;
  const int nh = a.n_hidden;
  const int n_out = a.n_out;
  const bool streamed = a.w0t_image != nullptr;
  const TcBwdLayout lay = tc_bwd_layout(K, W, nh, streamed);
  const int Kp = lay.Kp;
  const bool lmaj = bwd_level_major(NS, F);
  uint8_t* sW0t = smem + lay.w0t_off;
  uint8_t* sWht = smem + lay.wht_off;
  uint8_t* sWot = smem + lay.wot_off;
  int* sray = reinterpret_cast<int*>(smem + lay.row_off);
  float* st0 = reinterpret_cast<float*>(sray + kTcM);
  float* st1 = st0 + kTcM;
  float* sro = st1 + kTcM;       // [3][kTcM] ray origins
  float* srd = sro + 3 * kTcM;   // [3][kTcM] ray directions
  float* su = reinterpret_cast<float*>(smem + lay.u_off);  // sample fractions
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + lay.bar_off + 8);

  const int64_t n_tiles = (a.n + kTcM - 1) / kTcM;
  if (int64_t(blockIdx.x) >= n_tiles) return;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (warp == 0) {
    tmem_alloc(s_tmem, lay.ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < NS) su[threadIdx.x] = sample_u(threadIdx.x, NS);
  // B operands (K-major, rows = the MMA's N): W0^T [Kp][W], W_h^T [W][W], Wo^T [W][16]
  const float* W0 = a.mlp;
  if (!streamed) {
    for (int i = threadIdx.x; i < Kp * W; i += blockDim.x) {
      const int r = i / W, k = i - r * W;
      const float v = r < K ? __ldg(W0 + size_t(k) * K + bwd_w0_feature(r, K, NS, L, F, lmaj)) : 0.0f;
      *reinterpret_cast<typename OT::T*>(sW0t + op_offset(r, k, W)) = OT::one(v);
    }
  }
  const float* p = W0 + size_t(W) * K + W;
  for (int h = 1; h < nh; ++h) {
    uint8_t* dst = sWht + size_t(h - 1) * W * W * 2;
    for (int i = threadIdx.x; i < W * W; i += blockDim.x) {
      const int r = i / W, k = i - r * W;
      *reinterpret_cast<typename OT::T*>(dst + op_offset(r, k, W)) = OT::one(__ldg(p + size_t(k) * W + r));
    }
    p += W * W + W;
  }
  for (int i = threadIdx.x; i < W * 16; i += blockDim.x) {
    const int r = i / 16, k = i - r * 16;
    const float v = k < n_out ? __ldg(p + size_t(k) * W + r) : 0.0f;
    *reinterpret_cast<typename OT::T*>(sWot + op_offset(r, k, 16)) = OT::one(v);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  const int quarter = warp & 3;
  const int cgroup = warp >> 2;
  constexpr int kGroups = bwd_threads<W>() / 128;
  constexpr int kCols = W / kGroups;
  static_assert(kCols % 8 == 0, "16-byte activation loads");
  const int row = quarter * 32 + lane;
  const uint32_t t_row = tmem + (uint32_t(quarter * 32) << 16);
  uint32_t phase = 0;
  bool failed = false;

  for (int64_t tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
    if (threadIdx.x < kTcM) {
      const int64_t i = tile * kTcM + threadIdx.x;
      const int r = i < a.n ? (a.order ? a.order[i] : int(i)) : 0;
      const bool v = i < a.n && a.leaf[r] >= 0;
      sray[threadIdx.x] = v ? r : -1;
      st0[threadIdx.x] = v ? a.t0[r] : 0.0f;
      st1[threadIdx.x] = v ? a.t1[r] : 0.0f;
      sro[threadIdx.x] = v ? a.rays.ox[r] : 0.0f;
      sro[kTcM + threadIdx.x] = v ? a.rays.oy[r] : 0.0f;
      sro[2 * kTcM + threadIdx.x] = v ? a.rays.oz[r] : 0.0f;
      srd[threadIdx.x] = v ? a.rays.dx[r] : 0.0f;
      srd[kTcM + threadIdx.x] = v ? a.rays.dy[r] : 0.0f;
      srd[2 * kTcM + threadIdx.x] = v ? a.rays.dz[r] : 0.0f;
    }
    __syncthreads();
    const int64_t grow = tile * kTcM + row;
    // dL/d(raw) as the first A operand (16 columns, zero padded)
    if (cgroup == 0) {
      float g[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) g[j] = 0.0f;
      if (grow < a.n) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (j < n_out) g[j] = a.G[grow * n_out + j];
      }
      uint32_t pk[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) pk[j] = pack2<BF16>(g[2 * j], g[2 * j + 1]);
      tmem_st8(t_row + lay.col_a, pk);
    }
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      mma_f16_ts(tmem, tmem + lay.col_a, smem_desc(smem_u32(sWot), 128, 16 * 16), idesc_f16(BF16, kTcM, W), 0u);
      mma_commit(bar);
    }
    for (int h = nh - 1; h >= 0; --h) {
      const bool ok = mbar_wait(bar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after();
      {
        float v[kCols];
        tmem_ld_cols<kCols>(t_row + uint32_t(cgroup * kCols), v);
        tmem_ld_wait();
        const int c0 = cgroup * kCols;
        uint32_t pk[kCols / 2];
        if (grow < a.n) {
          const uint4* hrow = reinterpret_cast<const uint4*>(a.H16 + (size_t(h) * size_t(a.n) + size_t(grow)) * W + c0);
#pragma unroll
          for (int q = 0; q < kCols / 8; ++q) {
            const uint4 hv = __ldg(hrow + q);
            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float hf = from16<BF16>(uint16_t(hw[i >> 1] >> (16 * (i & 1))));
              v[8 * q + i] = hf > 0.0f ? v[8 * q + i] : 0.0f;
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < kCols; ++i) v[i] = 0.0f;
        }
#pragma unroll
        for (int i = 0; i < kCols / 2; ++i) pk[i] = pack2<BF16>(v[2 * i], v[2 * i + 1]);
        tmem_st_cols<kCols / 2>(t_row + lay.col_a + uint32_t(c0 / 2), pk);
        if (grow < a.n) {  // neuron-major, as the weight gradients read it
          uint16_t* zT = a.dZT + (int64_t(h) * W + c0) * a.ld + grow;
#pragma unroll
          for (int i = 0; i < kCols / 2; ++i) {
            zT[int64_t(2 * i) * a.ld] = uint16_t(pk[i] & 0xffffu);
            zT[int64_t(2 * i + 1) * a.ld] = uint16_t(pk[i] >> 16);
          }
        }
        tmem_st_wait();
      }
      tc_fence_before();
      __syncthreads();
      if (h > 0) {
        if (threadIdx.x == 0) {
          tc_fence_after();
          const uint32_t wb = smem_u32(sWht + size_t(h - 1) * W * W * 2);
          for (int j = 0; j < W / 16; ++j)
            mma_f16_ts(tmem, tmem + lay.col_a + uint32_t(8 * j), smem_desc(wb + j * 256, 128, uint32_t(W) * 16),
                       idesc_f16(BF16, kTcM, W), j > 0);
          mma_commit(bar);
        }
        continue;
      }
      // dL/dfeatures = dZ0 W0, 128 features at a time, scattered into the table gradient
      const int ray = sray[row];
      const bool valid = ray >= 0;
      for (int c0 = 0; c0 < Kp && !failed; c0 += 128) {
        const int cw = min(128, Kp - c0);
        if (streamed) {
          // this chunk's rows of W0^T (contiguous in the operand layout); the
          // previous chunk's MMA completed before the last barrier
          const uint4* src = reinterpret_cast<const uint4*>(a.w0t_image + size_t(c0) * W * 2);
          uint4* dst = reinterpret_cast<uint4*>(sW0t);
          for (int i = threadIdx.x; i < cw * W / 8; i += blockDim.x) dst[i] = __ldg(src + i);
          fence_proxy_async_smem();
          __syncthreads();
        }
        if (threadIdx.x == 0) {
          tc_fence_after();
          const uint32_t wb = smem_u32(sW0t) + (streamed ? 0u : uint32_t(c0 / 8) * uint32_t(W) * 16);
          for (int j = 0; j < W / 16; ++j)
            mma_f16_ts(tmem + lay.col_x, tmem + lay.col_a + uint32_t(8 * j),
                       smem_desc(wb + j * 256, 128, uint32_t(W) * 16), idesc_f16(BF16, kTcM, cw), j > 0);
          mma_commit(bar);
        }
        const bool ok2 = mbar_wait(bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok2)) {
          failed = true;
          break;
        }
        tc_fence_after();
        if constexpr (F <= 2) {
          if (lmaj) {
            // Each warp takes one level of the chunk for its 32 rays and walks
            // the samples in order along the ray. The eight corner sums of the
            // current cell stay in registers; when the ray moves to another
            // cell, the vertices the two cells do not share go to the table
            // and the shared ones carry over. A level with c cells along the
            // ray costs about 4c + 4 table updates instead of 8 per sample.
            const int nf = NS * F;
            constexpr int SP = 8 / F;  // samples per 8-column TMEM load
            for (int li = cgroup; li < cw / nf; li += kGroups) {
              const int l = c0 / nf + li;
              const int N = a.gp.res[l];
              float* gt = a.grad_table + a.gp.offset[l] * F;
              float acc[8][F];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
#pragma unroll
                for (int ff = 0; ff < F; ++ff) acc[q][ff] = 0.0f;
              }
              int ccx = -1, ccy = 0, ccz = 0;  // current cell (none yet: ccx < 0)
              for (int s0 = 0; s0 < NS; s0 += SP) {
                float g8[8];
                tmem_ld8(t_row + lay.col_x + uint32_t(li * nf + s0 * F), g8);
                tmem_ld_wait();
                if (!valid) continue;
#pragma unroll
                for (int si = 0; si < SP; ++si) {
                  float x, y, z;
                  sample_point_u(a.gp, sro[row], sro[kTcM + row], sro[2 * kTcM + row], srd[row], srd[kTcM + row],
                                 srd[2 * kTcM + row], st0[row], st1[row], su[s0 + si], x, y, z);
                  int cx, cy, cz;
                  float fx, fy, fz;
                  axis_cell(x, N, cx, fx);
                  axis_cell(y, N, cy, fy);
                  axis_cell(z, N, cz, fz);
                  if (ccx >= 0 && (cx != ccx || cy != ccy || cz != ccz)) {
                    const int dx = cx - ccx, dy = cy - ccy, dz = cz - ccz;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                      const int bx = q & 1, by = (q >> 1) & 1, bz = q >> 2;
                      const bool keep =
                          unsigned(bx - dx) <= 1u && unsigned(by - dy) <= 1u && unsigned(bz - dz) <= 1u;
                      if (!keep)
                        add_entry<F>(gt + size_t(vertex_index(a.gp, l, uint32_t(ccx + bx), uint32_t(ccy + by),
                                                              uint32_t(ccz + bz))) * F,
                                     acc[q]);
                    }
                    shift_corners<F, 1>(acc, dx);
                    shift_corners<F, 2>(acc, dy);
                    shift_corners<F, 4>(acc, dz);
                  }
                  ccx = cx;
                  ccy = cy;
                  ccz = cz;
                  const float wx[2] = {1.0f - fx, fx};
                  const float wy[2] = {1.0f - fy, fy};
                  const float wz[2] = {1.0f - fz, fz};
#pragma unroll
                  for (int q = 0; q < 8; ++q) {
                    const float wq = wx[q & 1] * wy[(q >> 1) & 1] * wz[q >> 2];
#pragma unroll
                    for (int ff = 0; ff < F; ++ff) acc[q][ff] = fmaf(wq, g8[si * F + ff], acc[q][ff]);
                  }
                }
              }
              // the last cell's vertices (the whole warp takes part)
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const uint32_t key =
                    ccx >= 0 ? vertex_index(a.gp, l, uint32_t(ccx + (q & 1)), uint32_t(ccy + ((q >> 1) & 1)),
                                            uint32_t(ccz + (q >> 2)))
                             : 0xffffffffu;
                add_vertex_warp<F>(gt, key, acc[q], N <= kAggMaxRes, lane);
              }
            }
          }
        }
        if (!lmaj) {
          // Sample-major chunks: 16 features (one sample, 16 / F levels) per
          // pass; eight table updates per sample and level.
          for (int sub = cgroup * 16; sub < cw; sub += kGroups * 16) {
            float gx[16];
            tmem_ld16(t_row + lay.col_x + uint32_t(sub), gx);
            tmem_ld_wait();
            int kprev = -1;
            float x = 0.0f, y = 0.0f, z = 0.0f;
#pragma unroll
            for (int j = 0; j < 16; j += F) {
              const int f = c0 + sub + j;
              if (f >= K) continue;
              const int k = f / (L * F);
              const int l = (f / F) % L;
              if (k != kprev) {
                if (valid)
                  sample_point_u(a.gp, sro[row], sro[kTcM + row], sro[2 * kTcM + row], srd[row], srd[kTcM + row],
                                 srd[2 * kTcM + row], st0[row], st1[row], su[k], x, y, z);
                kprev = k;
              }
              Corners cr;
              level_corners(a.gp, l, x, y, z, cr);
              float* gt = a.grad_table + a.gp.offset[l] * F;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                float v[F];
#pragma unroll
                for (int ff = 0; ff < F; ++ff) v[ff] = valid ? cr.w[q] * gx[j + ff] : 0.0f;
                add_vertex_warp<F>(gt, valid ? cr.idx[q] : 0xffffffffu, v, a.gp.res[l] <= kAggMaxRes, lane);
              }
            }
          }
        }
        tc_fence_before();
        __syncthreads();
      }
    }
  }
  if (failed) set_status(NBVH_ERR_TIMEOUT);
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, lay.ncols);
  }
}

// Weight gradients from stored operands of either precision (FP32 G, 16-bit
// activations and pre-activation gradients): dW[o][j] += sum_i dZ[i][o] A[i][j],
// db[o] += sum_i dZ[i][o], FP32 accumulation, split-K over segment chunks.
// Block = 64 x 64 outputs, thread = 4 x 4 (float4 broadcasts from shared memory).
template <typename T>
__device__ __forceinline__ float to_f(T v) {
  if constexpr (std::is_same<T, float>::value) return v;
  else if constexpr (std::is_same<T, __half>::value) return __half2float(v);
  else return __bfloat162float(v);
}

constexpr int kWgT = 64;
constexpr int kWgRows = 32;
constexpr int kWgChunk2 = 4096;

// Element (i, o) of dZ is dZ[i * zi + o * zo], element (i, j) of A is
// A[i * ai + j * aj] (row-major or transposed storage).
template <typename TZ, typename TA>
__global__ void __launch_bounds__(256) weight_grad_tiled(const TZ* __restrict__ dZ, int64_t zi, int64_t zo, int n_o,
                                                         const TA* __restrict__ A, int64_t ai, int64_t aj, int n_j,
                                                         int64_t n, int64_t chunk, float* __restrict__ dW,
                                                         float* __restrict__ db) {
  __shared__ __align__(16) float sz[kWgRows][kWgT];
  __shared__ __align__(16) float sa[kWgRows][kWgT];
  const int o0 = blockIdx.x * kWgT, j0 = blockIdx.y * kWgT;
  const int64_t i0 = int64_t(blockIdx.z) * chunk;
  const int64_t i1 = min(n, i0 + chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  float bacc[4] = {0, 0, 0, 0};
  for (int64_t ib = i0; ib < i1; ib += kWgRows) {
    for (int idx = threadIdx.x; idx < kWgRows * kWgT; idx += blockDim.x) {
      const int r = idx / kWgT, c = idx - r * kWgT;
      const int64_t i = ib + r;
      sz[r][c] = (i < i1 && o0 + c < n_o) ? to_f(dZ[i * zi + int64_t(o0 + c) * zo]) : 0.0f;
      sa[r][c] = (i < i1 && j0 + c < n_j) ? to_f(A[i * ai + int64_t(j0 + c) * aj]) : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < kWgRows; ++r) {
      const float4 zv = *reinterpret_cast<const float4*>(&sz[r][ty * 4]);
      const float4 av = *reinterpret_cast<const float4*>(&sa[r][tx * 4]);
      const float z4[4] = {zv.x, zv.y, zv.z, zv.w}, a4[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
      for (int p = 0; p < 4; ++p) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(z4[p], a4[q], acc[p][q]);
        bacc[p] += z4[p];
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int o = o0 + ty * 4 + p;
    if (o >= n_o) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tx * 4 + q;
      if (j < n_j) atomicAdd(dW + size_t(o) * n_j + j, acc[p][q]);
    }
    if (blockIdx.y == 0 && tx == 0) atomicAdd(db + o, bacc[p]);
  }
}

// Output-layer weight gradients (n_o <= NO outputs, NO a multiple of 4, width
// W <= 128 a multiple of 8, rows of H 16-byte aligned): dW[o][j] += sum_i G[i][o] H[i][j], db[o] += sum_i G[i][o], G
// FP32 [n][n_o], H 16-bit [n][W]. A block takes a chunk of the items, 64 at a
// time: the tile's G and H rows are contiguous, so all threads copy them into
// shared memory with independent coalesced loads; then thread t takes column
// j = t % W of rows t / W, t / W + 256 / W, ... for all outputs at once.
constexpr int kWgOutItems = 64;
template <typename TA, int NO>
__global__ void __launch_bounds__(256) weight_grad_out(const float* __restrict__ G, int n_o,
                                                       const TA* __restrict__ H, int W, int64_t n, int64_t chunk,
                                                       float* __restrict__ dW, float* __restrict__ db) {
  __shared__ __align__(16) float sg[kWgOutItems][NO];
  __shared__ float sh[kWgOutItems][128];
  const int64_t i0 = int64_t(blockIdx.x) * chunk;
  const int64_t i1 = min(n, i0 + chunk);
  const int groups = 256 / W;
  const int j = threadIdx.x % W, g = threadIdx.x / W;
  const int pieces = W / 8;  // 16-byte pieces per row (W a multiple of 8)
  const int c8 = threadIdx.x % pieces, r8 = threadIdx.x / pieces, rstep = 256 / pieces;
  const bool active = g < groups;
  float acc[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) acc[o] = 0.0f;
  float bacc = 0.0f;
  for (int64_t ib = i0; ib < i1; ib += kWgOutItems) {
    const int cnt = int(min(int64_t(kWgOutItems), i1 - ib));
    for (int e = threadIdx.x; e < kWgOutItems * NO; e += 256) {
      const int r = e / NO, o = e - (e / NO) * NO;
      sg[r][o] = (r < cnt && o < n_o) ? __ldg(G + (ib + r) * n_o + o) : 0.0f;
    }
    // 16-byte pieces (8 entries) of the tile's rows
    for (int r = r8; r < kWgOutItems; r += rstep) {
      float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (r < cnt) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(H + (ib + r) * W + 8 * c8));
        const TA* e = reinterpret_cast<const TA*>(&q);
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = to_f(e[k]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) sh[r][8 * c8 + k] = v[k];
    }
    __syncthreads();
    if (active) {
      for (int r = g; r < cnt; r += groups) {
        const float h = sh[r][j];
#pragma unroll
        for (int o = 0; o < NO; o += 4) {
          const float4 gv = *reinterpret_cast<const float4*>(&sg[r][o]);
          acc[o] = fmaf(gv.x, h, acc[o]);
          acc[o + 1] = fmaf(gv.y, h, acc[o + 1]);
          acc[o + 2] = fmaf(gv.z, h, acc[o + 2]);
          acc[o + 3] = fmaf(gv.w, h, acc[o + 3]);
        }
      }
    }
    if (threadIdx.x < n_o)
      for (int r = 0; r < cnt; ++r) bacc += sg[r][threadIdx.x];
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) atomicAdd(dW + o * W + j, acc[o]);
  }
  if (threadIdx.x < n_o) atomicAdd(db + threadIdx.x, bacc);
}

// ---------------------------------------------------------------------------
// First-layer weight gradient on the tensor cores: dW0^T [Kp x W] =
// X^T [Kp x n] * dZ0 [n x W], K = the batch, split over CTAs. Both operands are
// stored with the batch contiguous (feature-major features, neuron-major dZ0),
// so both tiles are K-major. Each CTA accumulates its 128-feature tiles in TMEM
// over its chunks of items, then adds them into the FP32 gradient.
// ---------------------------------------------------------------------------
struct WgTcArgs {
  const uint16_t* XT;  // [Kp][ld]
  const uint16_t* ZT;  // [W][ld]
  int64_t n, ld;
  int K, Kp;
  float* dW;           // [W][K]
  float* db;           // [W]
};

constexpr int kWgTcThreads = 256;
constexpr int kWgIssuer = kWgTcThreads - 32;  // the thread that issues the MMAs (W <= 128 < kWgIssuer)

__host__ __device__ inline int wg_tc_tiles(int Kp) { return (Kp + 127) / 128; }
// One stage: the features of `it` items ([Kp][it]) and their dZ ([W][it]).
__host__ __device__ inline uint32_t wg_tc_stage_bytes(int Kp, int W, int it) {
  return uint32_t(wg_tc_tiles(Kp)) * 128 * uint32_t(it) * 2 + uint32_t(W) * uint32_t(it) * 2;
}
// Items per stage: the most of 256, 128 and 64 whose two stages (the next
// chunk copied in while the tensor cores take this one) fit shared memory;
// few features (a hidden layer's 64) take long chunks, so that each copy and
// MMA round carries enough work.
__host__ __device__ inline int wg_tc_items(int Kp, int W) {
  for (int it = 256; it > 64; it /= 2)
    if (2 * wg_tc_stage_bytes(Kp, W, it) + 256 <= 227u * 1024u) return it;
  return 64;
}
// Stages: three where they fit (two chunks in flight while the tensor cores
// take a third: the 512-feature first layer at W = 64), else two, else one.
__host__ __device__ inline int wg_tc_stages(int Kp, int W) {
  const uint32_t b = wg_tc_stage_bytes(Kp, W, wg_tc_items(Kp, W));
  return 3 * b + 256 <= 227u * 1024u ? 3 : (2 * b + 256 <= 227u * 1024u ? 2 : 1);
}
__host__ __device__ inline uint32_t wg_tc_smem(int Kp, int W) {
  return uint32_t(wg_tc_stages(Kp, W)) * wg_tc_stage_bytes(Kp, W, wg_tc_items(Kp, W)) + 128 + 128;
}

// 16 bytes global -> shared, asynchronous; bytes beyond src_bytes (0..16) are zero.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int W, bool BF16>
__global__ void __launch_bounds__(kWgTcThreads, 1) weight_grad_tc(WgTcArgs a) {
  static_assert(W < kWgIssuer, "the MMA issuer is not a bias thread");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int tiles = wg_tc_tiles(a.Kp);
  const int it = wg_tc_items(a.Kp, W);  // items per chunk
  const int stages = wg_tc_stages(a.Kp, W);
  const uint32_t stage_bytes = wg_tc_stage_bytes(a.Kp, W, it);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + size_t(stages) * stage_bytes);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 1);
  const int64_t n_chunks = (a.n + it - 1) / it;
  if (int64_t(blockIdx.x) >= n_chunks) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t ncols = 32;
  while (ncols < uint32_t(tiles * W)) ncols <<= 1;
  if (warp == 0) {
    tmem_alloc(s_tmem, ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t idesc = idesc_f16(BF16, 128, W);
  float bsum = 0.0f;  // thread t < W: sum of dZ0 over its neuron
  uint32_t phase = 0;
  bool failed = false, first = true;
  // 16-byte pieces of a [rows][it items] tile into the K-major core-matrix
  // layout, copied asynchronously (zeros past the batch and past valid_rows)
  const int ppr = it / 8;  // pieces per row
  auto stage = [&](uint8_t* dst, const uint16_t* src, int rows, int valid_rows, int64_t c0) {
    for (int p = threadIdx.x; p < rows * ppr; p += blockDim.x) {
      const int r = p / ppr, q = p - r * ppr;
      const int64_t col = c0 + 8 * q;
      const int64_t left = r < valid_rows ? a.n - col : 0;
      const uint32_t bytes = left >= 8 ? 16u : (left > 0 ? uint32_t(left) * 2u : 0u);
      const uint16_t* g = bytes ? src + int64_t(r) * a.ld + col : src;
      cp_async16(dst + op_offset(r, 8 * q, it), g, bytes);
    }
  };
  auto issue = [&](int buf, int64_t c) {
    uint8_t* sA = smem + size_t(buf) * stage_bytes;
    uint8_t* sB = sA + size_t(tiles) * 128 * it * 2;
    const int64_t c0 = c * it;
    for (int t = 0; t < tiles; ++t)
      stage(sA + size_t(t) * 128 * it * 2, a.XT + int64_t(t) * 128 * a.ld, 128, min(128, a.K - 128 * t), c0);
    stage(sB, a.ZT, W, W, c0);
    cp_async_commit();
  };
  // this CTA's chunks: blockIdx.x + j * gridDim.x for j < mine; chunk j sits
  // in buffer j % stages
  const int64_t mine = (n_chunks - 1 - blockIdx.x) / gridDim.x + 1;
  for (int j = 0; j < max(stages - 1, 1) && j < mine; ++j) issue(j, blockIdx.x + int64_t(j) * gridDim.x);
  for (int64_t i = 0; i < mine && !failed; ++i) {
    const int b = int(i % stages);
    const int64_t ahead = i + stages - 1;
    // the chunk stages - 1 ahead goes into the buffer of chunk i - 1, whose
    // MMAs have completed
    if (stages > 1 && ahead < mine) issue(int(ahead % stages), blockIdx.x + ahead * gridDim.x);
    // chunk i has landed once at most the groups committed after it are pending
    const int64_t newer = min(int64_t(stages - 1), mine - 1 - i);
    if (newer >= 2) {
      cp_async_wait<2>();
    } else if (newer == 1) {
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    fence_proxy_async_smem();
    __syncthreads();
    uint8_t* sA = smem + size_t(b) * stage_bytes;
    uint8_t* sB = sA + size_t(tiles) * 128 * it * 2;
    if (threadIdx.x < W) {
      for (int q = 0; q < it; ++q) {
        const uint16_t e = *reinterpret_cast<const uint16_t*>(sB + op_offset(threadIdx.x, q, it));
        bsum += from16<BF16>(e);
      }
    }
    if (threadIdx.x == kWgIssuer) {  // not one of the bias threads (t < W), so the MMAs start at once
      tc_fence_after();
      const uint32_t sbo = uint32_t(it) * 16;
      for (int t = 0; t < tiles; ++t) {
        const uint32_t aa = smem_u32(sA + size_t(t) * 128 * it * 2);
        for (int kk = 0; kk < it / 16; ++kk)
          mma_f16(tmem + uint32_t(t * W), smem_desc(aa + kk * 256, 128, sbo), smem_desc(smem_u32(sB) + kk * 256, 128, sbo),
                  idesc, (first && kk == 0) ? 0u : 1u);
      }
      mma_commit(bar);
    }
    first = false;
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) failed = true;
    tc_fence_after();
    if (stages == 1 && i + 1 < mine && !failed)  // the buffer is free once the MMA completed
      issue(0, blockIdx.x + (i + 1) * gridDim.x);
  }
  cp_async_wait<0>();  // no copy left in flight into the freed buffers
  if (!failed && warp < 4) {
    const int q = warp;  // lane quarter
    const uint32_t t_row = tmem + (uint32_t(q * 32) << 16);
    for (int t = 0; t < tiles; ++t) {
      const int m = 128 * t + 32 * q + lane;  // feature
#pragma unroll
      for (int c0 = 0; c0 < W; c0 += 16) {
        float v[16];
        tmem_ld16(t_row + uint32_t(t * W + c0), v);
        tmem_ld_wait();
        if (m < a.K) {
#pragma unroll
          for (int i = 0; i < 16; ++i) atomicAdd(a.dW + int64_t(c0 + i) * a.K + m, v[i]);
        }
      }
    }
  }
  if (threadIdx.x < W && !failed) atomicAdd(a.db + threadIdx.x, bsum);
  if (failed) set_status(NBVH_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

}  // namespace nbvh
