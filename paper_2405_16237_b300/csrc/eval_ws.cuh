// The persistent neural ray query as a warp-specialised pipeline (S2..S6 on
// the tensor cores). Four control warps claim tiles from the queue, stage
// their rows, issue every tcgen05.mma, run the hidden/output epilogues and
// the resolve; twelve gather warps (three per TMEM lane quarter) only encode
// features into TMEM. The two groups hand work over through mbarriers, with
// no CTA-wide barrier inside the loop: while the control warps finish tile t
// (hidden layers, output, resolve, queueing, the next claim), the gather
// warps already fill tile t + 1. TMEM holds two FP32 accumulators (tiles t
// and t + 1) and two feature chunk buffers.
#pragma once
#include "eval_tc.cuh"

namespace nbvh {

constexpr int kWsThreads = 512;     // warps 0-3 control, 4-15 gather
constexpr int kWsGatherWarps = 12;  // three per lane quarter
constexpr int kWsPerQuarter = 3;

// Geometry of the pipelined kernel. A chunk holds S_c = 3 m whole samples
// (m per gather warp of a quarter); KC = S_c * LFp features; R chunks per
// tile (the last one may hold fewer real samples). TMEM columns:
//   [0, W) D0, [W, 2W) D1 (accumulators of alternate tiles),
//   [2W, 2W + W/2) H (hidden activations), [col_a, col_a + KC) two chunk
//   buffers of KC/2 columns.
// Shared memory: the first layer's weights (R resident chunks), the hidden
// and output weights, two row buffers, barriers.
struct WsLayout {
  bool ok;
  int LFp, IPS, KP, m, S_c, KC, R;
  uint32_t col_h, col_a;
  uint32_t chunk_bytes, w1_off, wh_off, wo_off, row_off, bar_off, total;
};

__host__ __device__ inline WsLayout ws_layout(int L, int F, int N, int W, int n_hidden) {
  WsLayout T;
  T.ok = false;
  T.LFp = (L * F + kItemF - 1) / kItemF * kItemF;
  T.IPS = T.LFp / kItemF;
  T.KP = (N * T.LFp + 15) & ~15;
  T.col_h = uint32_t(2 * W);
  T.col_a = uint32_t((2 * W + W / 2 + 31) & ~31);
  const int avail = 512 - int(T.col_a);
  T.m = avail / (3 * T.LFp);  // two buffers of KC / 2 columns each: KC <= avail
  const int need = (N + kWsPerQuarter - 1) / kWsPerQuarter;
  if (T.m > need) T.m = need;
  T.S_c = kWsPerQuarter * T.m;
  T.KC = T.S_c * T.LFp;
  T.R = T.S_c > 0 ? (N + T.S_c - 1) / T.S_c : 0;
  T.chunk_bytes = uint32_t(W) * uint32_t(T.KC) * 2;
  uint32_t off = 0;
  auto take = [&](uint32_t bytes) {
    const uint32_t o = off;
    off = (off + bytes + 127u) & ~127u;
    return o;
  };
  T.w1_off = take(uint32_t(T.R) * T.chunk_bytes);
  T.wh_off = take(uint32_t(n_hidden - 1) * W * W * 2);
  T.wo_off = take(16u * W * 2);
  T.row_off = take(2 * kTcM * kRowBytes);
  T.bar_off = take(128);
  T.total = off + 128;
  T.ok = (W == 32 || W == 64) && T.m >= 1 && (T.LFp % 16) == 0 && T.total <= 227u * 1024u;
  return T;
}

// The W1 layout of the pipelined kernel: chunks of KC features, the same
// K-major core-matrix layout as the phase kernel's (w1_chunk_offset).
__host__ __device__ inline TcLayout ws_as_tc(const WsLayout& S) {
  TcLayout T;
  T.LFp = S.LFp;
  T.IPS = S.IPS;
  T.NI = 0;
  T.KP = S.KP;
  T.KC = S.KC;
  T.NB = 2;
  T.R = S.R;
  T.chunk_bytes = S.chunk_bytes;
  return T;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
// OR of pred over the `threads` threads of named barrier `id`.
__device__ __forceinline__ bool named_or(int id, int threads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(uint32_t(pred)), "r"(id), "r"(threads)
      : "memory");
  return r != 0;
}

template <typename T, int F, int W, bool BF16>
__global__ void __launch_bounds__(kWsThreads, 1) eval_ws_kernel(EvalArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int K = a.gp.n_inputs;
  const int L = a.gp.n_levels;
  const int N = a.gp.n_samples;
  const int n_out = a.n_out;
  const WsLayout lay = ws_layout(L, F, N, W, a.n_hidden);
  const TcLayout wl = ws_as_tc(lay);
  uint8_t* sW1 = smem + lay.w1_off;
  uint8_t* sWh = smem + lay.wh_off;
  uint8_t* sWo = smem + lay.wo_off;
  uint8_t* const rows_base = smem + lay.row_off;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  uint64_t* rows_full = bars + 0;  // [2] control -> gather: a tile's rows are staged
  uint64_t* a_full = bars + 2;     // [2] gather -> control: a chunk buffer is filled (12 arrivals)
  uint64_t* a_empty = bars + 4;    // [2] MMA -> gather: a chunk buffer was read
  uint64_t* d_full = bars + 6;     // [2] MMA -> control: a tile's first layer is done
  uint64_t* bar_mlp = bars + 8;    // hidden/output layer MMAs
  uint64_t* bar_fin = bars + 9;    // exit: every MMA retired
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 10);
  __shared__ int s_count[2];       // per row buffer: item count of its tile (0: drained, < 0: failed)
  __shared__ unsigned long long s_start[2];
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const bool control = warp < 4;
  const int quarter = warp & 3;
  if (warp == 0) {
    tmem_alloc(s_tmem, 512);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(rows_full + 0, 1);
    mbar_init(rows_full + 1, 1);
    mbar_init(a_full + 0, kWsGatherWarps);
    mbar_init(a_full + 1, kWsGatherWarps);
    for (int i = 4; i < 10; ++i) mbar_init(bars + i, 1);
    fence_mbar_init();
    s_fail = 0;
    s_count[0] = s_count[1] = 0;
  }
  // weights -> operand layouts, once per CTA
  const float* W1 = a.mlp;
  const float* b1 = W1 + size_t(W) * K;
  for (int i = threadIdx.x; i < W * lay.R * lay.KC; i += kWsThreads) put_w1<BF16>(sW1, W1, i, W, K, L, F, N, wl);
  const float* p = b1 + W;
  for (int h = 1; h < a.n_hidden; ++h) {
    stage_weights<BF16>(sWh + size_t(h - 1) * W * W * 2, p, W, W, W, W);
    p += W * W + W;
  }
  const float* Wo = p;
  const float* bo = Wo + size_t(n_out) * W;
  stage_weights<BF16>(sWo, Wo, n_out, 16, W, W);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t t_row = tmem + (uint32_t(quarter * 32) << 16);
  const T* table = static_cast<const T*>(a.table);
  const int R = lay.R;

  if (!control) {
    // ------------------------------------------------------------ gather warps
    const int gi = warp / 4 - 1;  // 0..2 within the quarter
    constexpr bool kSplitX = F == 2 && sizeof(T) == 2;
    for (uint32_t t = 0;; ++t) {
      const int b = int(t & 1u);
      if (!mbar_wait(rows_full + b, (t >> 1) & 1u)) {
        s_fail = 1;
        break;
      }
      const int cnt = *reinterpret_cast<volatile int*>(&s_count[b]);
      if (cnt <= 0) break;
      const RowBuf rb = row_buf(rows_base + size_t(b) * kTcM * kRowBytes);
      bool bad = false;
      for (int r = 0; r < R; ++r) {
        const uint32_t g = t * uint32_t(R) + uint32_t(r);
        const int buf = int(g & 1u);
        if (g >= 2) {
          if (!mbar_wait(a_empty + buf, ((g - 2) >> 1) & 1u)) {
            s_fail = 1;
            bad = true;
            break;
          }
          tc_fence_after();
        }
        const uint32_t t_buf = t_row + lay.col_a + uint32_t(buf * (lay.KC / 2));
        // this warp's samples of the chunk: r * S_c + gi * m + (0 .. m - 1)
        for (int s = 0; s < lay.m; ++s) {
          const int kl = gi * lay.m + s;    // sample within the chunk
          const int k = r * lay.S_c + kl;   // sample of the row
          if (k >= N) break;                // beyond the last sample: never read by the MMAs
          const uint32_t col = uint32_t(kl * lay.LFp / 2);
          if constexpr (kSplitX) {
            const int xb = lane >> 4;
            const int r0 = quarter * 32 + (lane & 15), r1 = r0 + 16;
            const bool v0 = rb.ray[r0] >= 0, v1 = rb.ray[r1] >= 0;
            float p0[3] = {0.0f, 0.0f, 0.0f}, p1[3] = {0.0f, 0.0f, 0.0f};
            if (v0) row_point(a.gp, rb, r0, k, p0);
            if (v1) row_point(a.gp, rb, r1, k, p1);
            if (L == 16) {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                uint32_t pk[4];
                split_item<T, BF16, true>(a.gp, table, 4 * q, 16, p0, p1, v0, v1, xb, pk);
                __syncwarp();
                tmem_st4(t_buf + col + 4 * q, pk);
              }
            } else {
              for (int q = 0; q < lay.IPS; ++q) {
                uint32_t pk[4];
                if (4 * q + 4 <= L)
                  split_item<T, BF16, true>(a.gp, table, 4 * q, L, p0, p1, v0, v1, xb, pk);
                else
                  split_item<T, BF16, false>(a.gp, table, 4 * q, L, p0, p1, v0, v1, xb, pk);
                __syncwarp();
                tmem_st4(t_buf + col + 4 * q, pk);
              }
            }
          } else {
            constexpr int LPC = 8 / F;
            const int row = quarter * 32 + lane;
            const bool valid = rb.ray[row] >= 0;
            float pt[3] = {0.0f, 0.0f, 0.0f};
            if (valid) row_point(a.gp, rb, row, k, pt);
            for (int q = 0; q < lay.IPS; ++q) {
              float v[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) v[j] = 0.0f;
              if (valid) row_item<T, F>(a.gp, table, q * LPC, L, pt, v);
              uint32_t pk[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) pk[j] = pack2<BF16>(v[2 * j], v[2 * j + 1]);
              __syncwarp();
              tmem_st4(t_buf + col + 4 * q, pk);
            }
          }
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(a_full + buf);
      }
      if (bad) break;
    }
  } else {
    // ------------------------------------------------------------ control warps
    const int row = threadIdx.x;  // 0..127: row of the tile, TMEM lane
    const uint32_t idesc_h = idesc_f16(BF16, kTcM, W);
    const uint32_t idesc_o = idesc_f16(BF16, kTcM, 16);
    uint32_t mlp_phase = 0;
    bool failed = false;
    // claim (blocking or not) and stage a tile into row buffer b; returns the
    // item count (0: drained, < 0: failed, kPqNoTile: nothing claimed)
    auto claim_stage = [&](int b, bool blocking) -> int {
      if (threadIdx.x == 0) {
        unsigned long long st = 0;
        s_count[b] = blocking ? pq_claim(a.pq, &st) : pq_try_claim(a.pq, &st);
        s_start[b] = st;
      }
      named_sync(1, 128);
      const int cnt = s_count[b];
      if (cnt > 0 && cnt != kPqNoTile) {
        const RowBuf rb = row_buf(rows_base + size_t(b) * kTcM * kRowBytes);
        if (row < cnt)
          pq_stage(a, s_start[b] + row, row, rb);
        else
          put_row(rb, a.rays, row, -1, 0.0f, 0.0f);
      }
      named_sync(1, 128);
      return cnt;
    };
    // publish row buffer b (its tile, or the end of work) to the gather warps
    auto publish = [&](int b) {
      if (threadIdx.x == 0) {
        __threadfence_block();
        mbar_arrive(rows_full + b);
      }
    };
    // layer-1 MMAs of chunk r of tile t, once the gather warps filled it
    auto issue_chunk = [&](uint32_t t, int r) -> bool {
      if (threadIdx.x != 0) return true;
      const uint32_t g = t * uint32_t(R) + uint32_t(r);
      const int buf = int(g & 1u);
      if (!mbar_wait(a_full + buf, (g >> 1) & 1u)) return false;
      tc_fence_after();
      const uint32_t d = tmem + uint32_t((t & 1u) * W);
      const int steps = min(lay.KC, lay.KP - r * lay.KC) / 16;
      const uint32_t wb = smem_u32(sW1 + size_t(r) * lay.chunk_bytes);
      for (int j = 0; j < steps; ++j)
        mma_f16_ts(d, tmem + lay.col_a + uint32_t(buf * (lay.KC / 2) + 8 * j),
                   smem_desc(wb + j * 256, 128, uint32_t(lay.KC) * 16), idesc_h, (r > 0 || j > 0) ? 1u : 0u);
      mma_commit(a_empty + buf);
      if (r == R - 1) mma_commit(d_full + (t & 1u));
      return true;
    };
    // hidden layers, output layer, resolve, queueing and retirement of tile t
    auto finish_tile = [&](uint32_t t) -> bool {
      const int b = int(t & 1u);
      const RowBuf rb = row_buf(rows_base + size_t(b) * kTcM * kRowBytes);
      const uint32_t d = t_row + uint32_t(b * W);
      if (!mbar_wait(d_full + b, (t >> 1) & 1u)) return false;
      tc_fence_after();
      for (int h = 0; h < a.n_hidden; ++h) {
        const float* bias = h == 0 ? b1 : b1 + W + size_t(h - 1) * (W * W + W) + size_t(W) * W;
        if (h > 0) {
          if (!mbar_wait(bar_mlp, mlp_phase)) return false;
          mlp_phase ^= 1u;
          tc_fence_after();
        }
#pragma unroll
        for (int c0 = 0; c0 < W; c0 += 16) {
          float v[16];
          tmem_ld16(d + uint32_t(c0), v);
          tmem_ld_wait();
          uint32_t pk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i)
            pk[i] = pack2<BF16>(fmaxf(v[2 * i] + __ldg(bias + c0 + 2 * i), 0.0f),
                                fmaxf(v[2 * i + 1] + __ldg(bias + c0 + 2 * i + 1), 0.0f));
          tmem_st8(t_row + lay.col_h + uint32_t(c0 / 2), pk);
        }
        tmem_st_wait();
        tc_fence_before();
        named_sync(1, 128);
        if (threadIdx.x == 0) {
          tc_fence_after();
          const uint32_t sbo = uint32_t(W) * 16;
          const uint32_t wa = smem_u32(h + 1 < a.n_hidden ? sWh + size_t(h) * W * W * 2 : sWo);
          const uint32_t idesc = h + 1 < a.n_hidden ? idesc_h : idesc_o;
          for (int j = 0; j < W / 16; ++j)
            mma_f16_ts(tmem + uint32_t(b * W), tmem + lay.col_h + uint32_t(8 * j), smem_desc(wa + j * 256, 128, sbo),
                       idesc, j > 0);
          mma_commit(bar_mlp);
        }
      }
      if (!mbar_wait(bar_mlp, mlp_phase)) return false;
      mlp_phase ^= 1u;
      tc_fence_after();
      float v[16];
      tmem_ld16(d, v);
      tmem_ld_wait();
      float raw[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) raw[j] = j < n_out ? v[j] + __ldg(bo + j) : 0.0f;
      const int ray = rb.ray[row];
      const bool push = ray >= 0 && pq_resolve(a, ray, rb.slot[row], rb.best[row], rb.next[row], raw, rb.t0[row],
                                               rb.t1[row]);
      // queue the next segments (one reservation per warp), then retire the tile
      const unsigned msk = __ballot_sync(0xffffffffu, push);
      unsigned long long base = 0;
      if (msk && lane == 0) base = atomicAdd(a.pq.reserved, (unsigned long long)__popc(msk));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (push) {
        const unsigned long long item = (unsigned long long)(rb.slot[row] + 1) << 32 | uint32_t(ray);
        if (!pq_put(a.pq, base + __popc(msk & ((1u << lane) - 1u)), pq_ring_n(a.pq), item))
          set_status(NBVH_ERR_TIMEOUT);
      }
      tc_fence_before();
      named_sync(1, 128);  // every row resolved and queued; D of this tile read
      if (threadIdx.x == 0) red_release_add_u64(a.pq.retired, (unsigned long long)s_count[b]);
      return true;
    };

    // tile 0: a blocking claim
    int cnt = claim_stage(0, true);
    publish(0);
    uint32_t published = 0;  // the last tile published to the gather warps
    if (cnt > 0) {
      for (uint32_t t = 0;; ++t) {
        const int nb = int((t + 1) & 1u);
        // first chunk of tile t (the gather warps are on it)
        if (named_or(1, 128, !issue_chunk(t, 0))) {
          failed = true;
          break;
        }
        // claim tile t + 1 now if a full one is queued, so that the gather
        // warps go on with it while this tile is finished
        int ncnt = claim_stage(nb, false);
        const bool next_staged = ncnt != kPqNoTile;
        if (next_staged) {
          publish(nb);
          published = t + 1;
        }
        for (int r = 1; r < R && !failed; ++r)
          if (named_or(1, 128, !issue_chunk(t, r))) failed = true;
        if (failed) break;
        if (named_or(1, 128, !finish_tile(t))) {
          failed = true;
          break;
        }
        if (!next_staged) {
          // nothing of this CTA is in evaluation now: a blocking claim
          ncnt = claim_stage(nb, true);
          publish(nb);
          published = t + 1;
        }
        if (ncnt <= 0) {
          failed = ncnt < 0;
          break;
        }
      }
    } else {
      failed = cnt < 0;
    }
    if (failed) {
      // the gather warps go on to the next unpublished tile and find it failed
      const int fb = int((published + 1) & 1u);
      if (threadIdx.x == 0) {
        s_fail = 1;
        s_count[fb] = -1;
      }
      named_sync(1, 128);
      publish(fb);
    }
  }
  if (s_fail) set_status(NBVH_ERR_TIMEOUT);
  __syncthreads();
  if (threadIdx.x == 0) {
    mma_commit(bar_fin);
    if (!mbar_wait(bar_fin, 0)) set_status(NBVH_ERR_TIMEOUT);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace nbvh

namespace nbvh {

// Whether the pipelined kernel runs this model (W 32 or 64, whole-sample
// chunks within TMEM, resident first layer).
inline bool ws_supported(const nbvh_model_desc* d) {
  return d->mlp_prec != NBVH_FP32 && d->n_out <= 16 &&
         ws_layout(d->n_levels, d->n_features, d->n_samples, d->width, d->n_hidden).ok;
}

template <typename T, int F, int W>
cudaError_t launch_ws_twf(const nbvh_model_desc* d, const EvalArgs& a, cudaStream_t s) {
  const WsLayout lay = ws_layout(a.gp.n_levels, F, a.gp.n_samples, W, a.n_hidden);
  if (!lay.ok || a.w1_image) return cudaErrorInvalidConfiguration;
  auto kern = d->mlp_prec == NBVH_BF16 ? eval_ws_kernel<T, F, W, true> : eval_ws_kernel<T, F, W, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lay.total));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = sms;  // one CTA per SM holds all 512 TMEM columns
  const int64_t tiles = (a.n_rays + kTcM - 1) / kTcM;
  if (tiles < grid) grid = tiles;
  if (grid < 1) return cudaSuccess;
  kern<<<unsigned(grid), kWsThreads, lay.total, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T, int F>
cudaError_t launch_ws_tf(const nbvh_model_desc* d, const EvalArgs& a, cudaStream_t s) {
  switch (d->width) {
    case 32: return launch_ws_twf<T, F, 32>(d, a, s);
    case 64: return launch_ws_twf<T, F, 64>(d, a, s);
  }
  return cudaErrorInvalidConfiguration;
}

// The pipelined persistent query of one table type (query translation units).
template <typename T>
cudaError_t launch_ws_t(const nbvh_model_desc* d, const EvalArgs& a, cudaStream_t s) {
  switch (d->n_features) {
    case 1: return launch_ws_tf<T, 1>(d, a, s);
    case 2: return launch_ws_tf<T, 2>(d, a, s);
    case 4: return launch_ws_tf<T, 4>(d, a, s);
    case 8: return launch_ws_tf<T, 8>(d, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nbvh
