// S2..S5 fused with the MLP on the 5th-generation tensor cores (tcgen05):
// the hash-grid gather writes FP16/BF16 features straight into the MMA's
// shared-memory operand layout, one elected thread issues tcgen05.mma with the
// FP32 accumulator in tensor memory (TMEM), and the epilogue reads TMEM back
// (tcgen05.ld) for bias + ReLU into the next layer's operand, or for decode and
// resolve after the output layer.
#pragma once
#include "nbvh_internal.cuh"
#include "eval_plain.cuh"

#include <algorithm>
#include <cstring>

namespace nbvh {

constexpr int kTcM = 128;          // segments per tile = MMA M = TMEM lanes
constexpr long long kWaitCycles = 4000000000LL;  // bounded mbarrier wait (~2 s)

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait: gives up after kWaitCycles SM cycles and reports false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long start = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - start > kWaitCycles) return false;
  }
  return true;
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (FP16 or BF16 operands, FP32 accumulate).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once every tcgen05 operation issued so far by this thread completes.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 bits, 8/16/32 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int COLS>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float* v) {
  if constexpr (COLS == 4) {
    tmem_ld4(taddr, v);
  } else if constexpr (COLS == 8) {
    tmem_ld8(taddr, v);
  } else {
#pragma unroll
    for (int c = 0; c < COLS; c += 16) tmem_ld16(taddr + c, v + c);
  }
}

// ---------------------------------------------------------------- operand layout
// K-major operand without swizzle, built from 8x8 "core matrices" (8 rows x
// 16 bytes, stored as 128 contiguous bytes). Element (row r, column k) of an
// operand with Kp columns sits at byte
//   (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2,
// LBO = 128 (next core matrix along K), SBO = Kp * 16 (next 8-row group).
// One MMA covers K = 16, i.e. two core matrices along K: step j starts at
// base + j * 256.
__device__ __forceinline__ uint32_t op_offset(int r, int k, int Kp) {
  return uint32_t((r >> 3) * (Kp * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version for tcgen05
  // base offset 0, absolute LBO mode, layout type 0 = no swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A/B = F16 (0) or BF16 (1),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(bool bf16, int M, int N) {
  return (1u << 4) | (uint32_t(bf16) << 7) | (uint32_t(bf16) << 10) | (uint32_t(N >> 3) << 17) |
         (uint32_t(M >> 4) << 24);
}

template <bool BF16>
struct OpType;
template <>
struct OpType<false> {
  using T = __half;
  using T2 = __half2;
  static __device__ __forceinline__ T2 pack(float a, float b) { return __floats2half2_rn(a, b); }
  static __device__ __forceinline__ T one(float a) { return __float2half_rn(a); }
};
template <>
struct OpType<true> {
  using T = __nv_bfloat16;
  using T2 = __nv_bfloat162;
  static __device__ __forceinline__ T2 pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
  static __device__ __forceinline__ T one(float a) { return __float2bfloat16_rn(a); }
};

// ---------------------------------------------------------------- tile geometry
// A sample's L*F features are padded to a multiple of 8 (one "item": 8
// features = 4 TMEM columns, one tcgen05.st); the padded input has
// KP = N * LFp features rounded up to 16 (one MMA K step) and the first
// layer's weights carry zero rows for the padding. When the whole padded
// input fits the CTA's TMEM next to the accumulator and the hidden
// activations, the first layer runs as one round (one barrier per tile).
// Otherwise it runs over K chunks of KC features (at most 32 KB of weights
// each) through two TMEM buffers: while the tensor cores multiply chunk r,
// the gather fills chunk r + 1 into the other buffer, so the feature
// footprint is bounded whatever K is.
constexpr int kItemF = 8;

// TMEM column plan (one 32-bit column holds two 16-bit operand elements):
//   [0, W)                  FP32 accumulator D of the current layer (the
//                           output layer uses its first 16 columns)
//   [W, W + W/2)            hidden activations H, the next layer's A operand
//   [2W, 2W + NB * KC/2)    NB feature buffers of KC features, the first
//                           layer's A operand
// A CTA of 256 threads keeps to 256 columns (two CTAs share an SM), one of
// 512 threads may use all 512.
// Shared memory: the first layer's weights as chunk-sized B operands (all R
// chunks resident, or two buffers that bulk copies refill from a prepared
// 16-bit image in global memory), the hidden and output weights, two row
// buffers and the barriers.
struct TcLayout {
  int LFp;                   // features per sample, padded to a multiple of 8
  int IPS;                   // items per sample (LFp / 8)
  int NI;                    // items per row (N * IPS)
  int KP;                    // padded input width (N * LFp rounded up to 16)
  int KC;                    // features per chunk (a multiple of 64)
  int NB;                    // TMEM feature buffers (1: one round; 2: double buffered)
  int R;                     // chunks (rounds per tile)
  uint32_t col_h, col_a, ncols;
  uint32_t chunk_bytes;      // one W x KC chunk of the first layer's weights
  uint32_t w1_off;           // resident: R chunks; streamed: 2 chunk buffers
  uint32_t wh_off;           // (n_hidden - 1) x W x W
  uint32_t wo_off;           // 16 x W
  uint32_t row_off;          // two row buffers
  uint32_t raw_off;          // raw outputs of a tile's rows (persistent query resolve)
  uint32_t bar_off;          // mbarriers + TMEM base address
  uint32_t total;
};

constexpr uint32_t kRowBytes = 12 * 4;  // per row: ray, t0, t1, slot, best t, next t0, origin, direction

__host__ __device__ inline TcLayout tc_layout(int L, int F, int N, int W, int n_hidden, bool stream, int threads) {
  TcLayout T;
  T.LFp = (L * F + kItemF - 1) / kItemF * kItemF;
  T.IPS = T.LFp / kItemF;
  T.NI = N * T.IPS;
  T.KP = (N * T.LFp + 15) & ~15;
  T.col_h = uint32_t(W);
  T.col_a = uint32_t(2 * W);
  const int budget = threads == 256 ? 256 : 512;
  const int avail = budget - 2 * W;         // columns for the feature buffers
  const int kp64 = (T.KP + 63) & ~63;
  if (kp64 / 2 <= avail) {
    T.NB = 1;
    T.KC = kp64;
  } else {
    T.NB = 2;
    T.KC = 2 * (avail / 2 / 32 * 32);
    // A chunk of at most 32 KB of weights (256 features at W = 64): the two
    // streamed buffers then take 64 KB of the SM's unified L1 / shared memory
    // instead of 96, which the gather uses. The 16-asset frame took 80.5 ms
    // against 85.9 with 384-feature chunks (192: 111.7, 320: 115.0 vs 105.2
    // ms untrained: chunks dividing K evenly, in few rounds, win).
    const int kc_cap = (32768 / (W * 2)) / 64 * 64;
    if (kc_cap >= 64 && T.KC > kc_cap) T.KC = kc_cap;
    if (T.KC < 64) T.KC = 64;  // no valid plan has so few columns (tc_plan rejects it)
  }
  T.R = (T.KP + T.KC - 1) / T.KC;
  const uint32_t used = T.col_a + uint32_t(T.NB * T.KC / 2);
  uint32_t nc = 32;
  while (nc < used) nc <<= 1;
  T.ncols = nc;
  T.chunk_bytes = uint32_t(W) * uint32_t(T.KC) * 2;
  uint32_t off = 0;
  auto take = [&](uint32_t bytes) {
    const uint32_t o = off;
    off = (off + bytes + 127u) & ~127u;
    return o;
  };
  T.w1_off = take((stream ? 2u : uint32_t(T.R)) * T.chunk_bytes);
  T.wh_off = take(uint32_t(n_hidden - 1) * W * W * 2);
  T.wo_off = take(16u * W * 2);
  T.row_off = take(2 * kTcM * kRowBytes);
  T.raw_off = take(kTcM * 8 * 4);
  T.bar_off = take(64);
  T.total = off + 128;  // slack for base alignment
  return T;
}

// Column c of the padded input: the original feature index, or -1 for padding.
__host__ __device__ inline int padded_feature(int c, int L, int F, int N, int LFp) {
  const int k = c / LFp, rem = c - k * LFp;
  return (k < N && rem < L * F) ? k * L * F + rem : -1;
}

// Element (row n, padded column c) of the first layer's weights in the chunked
// B-operand layout: chunk c / KC, then the K-major core-matrix layout of a
// W x KC operand.
__host__ __device__ inline uint32_t w1_chunk_offset(int n, int c, const TcLayout& T) {
  const int r = c / T.KC, cc = c - r * T.KC;
  return uint32_t(r) * T.chunk_bytes +
         uint32_t((n >> 3) * (T.KC * 16) + (cc >> 3) * 128 + (n & 7) * 16 + (cc & 7) * 2);
}

// D[tmem] (+)= A[tmem] * B[smem]^T (A from tensor memory, kind::f16).
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 32 lanes x 32 bits stores of 1/2/4/8 consecutive columns per thread.
__device__ __forceinline__ void tmem_st1(uint32_t taddr, uint32_t a) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(a) : "memory");
}
__device__ __forceinline__ void tmem_st2(uint32_t taddr, uint32_t a, uint32_t b) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(taddr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
               "r"(v[2]), "r"(v[3])
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

template <int NC>
__device__ __forceinline__ void tmem_st_cols(uint32_t taddr, const uint32_t* v) {
  if constexpr (NC == 1) {
    tmem_st1(taddr, v[0]);
  } else if constexpr (NC == 2) {
    tmem_st2(taddr, v[0], v[1]);
  } else if constexpr (NC == 4) {
    tmem_st4(taddr, v);
  } else {
#pragma unroll
    for (int c = 0; c < NC; c += 8) tmem_st8(taddr + c, v + c);
  }
}

// Copy an fp32 [rows][K] row-major weight block into the K-major operand layout
// with Kp columns (zero padding beyond K and rows beyond `rows` up to rows_p).
template <bool BF16>
__device__ __forceinline__ void stage_weights(uint8_t* dst, const float* __restrict__ src, int rows, int rows_p,
                                              int K, int Kp) {
  using OT = OpType<BF16>;
  for (int i = threadIdx.x; i < rows_p * Kp; i += blockDim.x) {
    const int r = i / Kp, k = i - r * Kp;
    const float v = (r < rows && k < K) ? __ldg(src + size_t(r) * K + k) : 0.0f;
    *reinterpret_cast<typename OT::T*>(dst + op_offset(r, k, Kp)) = OT::one(v);
  }
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  typename OpType<BF16>::T2 h = OpType<BF16>::pack(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ---------------------------------------------------------------- persistent query queue
constexpr long long kPqSpinLimit = 1LL << 22;      // default bound of the queue waits (~1 s with the back-off below)
constexpr unsigned long long kPqEmpty = ~0ull;     // an empty ring entry

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long exch_acquire_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acquire.gpu.global.exch.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long cas_release_u64(unsigned long long* p, unsigned long long cmp,
                                                              unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.release.gpu.global.cas.b64 %0, [%1], %2, %3;" : "=l"(old) : "l"(p), "l"(cmp), "l"(v)
               : "memory");
  return old;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Thread 0 of a CTA: claim up to kTcM queued items. Returns the count (start
// in *start), 0 when the CTA leaves (the queue has drained, or see below),
// -1 when the wait gave up. A partial tile is taken only when nothing is in
// evaluation (no more items can come) or after q.patience cycles of waiting:
// a tile's latency hardly shrinks with fewer rows, while other CTAs' resolves
// refill the queue within microseconds. A partial tile claims at most
// q.partial_items items: its other rows hold those rays' next segments
// (lookahead), so when the queue runs shallow, several CTAs split it and each
// ray's chain advances up to 128 / items slots per tile. The counters are polled with
// independent relaxed loads (a stale value only delays a claim; the CAS on
// head validates it); the drained state is confirmed by reading retired, then
// head, then reserved in order: equal values mean nothing is in evaluation
// or queued, so nothing more can be queued.
// With q.yield_idle = m > 0 (other kernels run beside this one: the
// instances of a hybrid trace) a CTA with nothing to claim also leaves while
// the CTAs that stay are enough for the items in evaluation: each item has at
// most one successor, so the next round needs at most ceil(in evaluation /
// kTcM) tiles (plus m - 1 spare CTAs for partial tiles with lookahead rows),
// and the CTAs evaluating them stay. Its SM then serves the other
// kernels. A stale count only makes the CTA stay. (Alone, a draining queue
// is better served by many CTAs taking partial tiles with lookahead rows.)
// Items a claim takes at once: a full tile, or with q.split > 0 at most
// max(q.split, ceil(R / CTAs)) (R: the traversal's queue length). A short
// queue then spreads over all the CTAs at once, each tile's other rows
// holding the same rays' next segments (lookahead), instead of a few CTAs
// taking full tiles one segment per ray.
__device__ __forceinline__ unsigned long long pq_full(const PQueue& q) {
  if (q.split <= 0) return kTcM;
  const int32_t n0 = __ldg(q.qlen0);
  const unsigned long long per = (unsigned long long)(n0 > 0 ? n0 : 0) / gridDim.x + 1ull;
  const unsigned long long f = per > (unsigned long long)q.split ? per : (unsigned long long)q.split;
  return f < kTcM ? f : kTcM;
}

__device__ __forceinline__ int pq_claim(const PQueue& q, unsigned long long* start) {
  const long long t0 = clock64();
  const unsigned long long full = pq_full(q);
  for (long long spin = 0; spin < q.spin_limit; ++spin) {
    const unsigned long long retired = ld_relaxed_u64(q.retired);
    const unsigned long long head = ld_relaxed_u64(q.head);
    const unsigned long long res = ld_relaxed_u64(q.reserved);
    if (res > head) {
      const unsigned long long avail = res - head;
      if (avail >= full || retired == head || clock64() - t0 > q.patience) {
        // a partial tile takes at most q.partial_items items, so that other
        // CTAs share a shallow queue and each item gets more lookahead rows
        const unsigned long long cap = avail >= full ? full : (unsigned long long)q.partial_items;
        const unsigned want = unsigned(avail < cap ? avail : cap);
        if (atomicCAS(q.head, head, head + want) == head) {
          atomicAdd(q.tiles, 1u);
          *start = head;
          return int(want);
        }
        continue;
      }
    } else if (retired == head) {
      const unsigned long long r2 = ld_acquire_u64(q.retired);
      const unsigned long long h2 = ld_acquire_u64(q.head);
      const unsigned long long s2 = ld_acquire_u64(q.reserved);
      if (r2 == h2 && s2 == h2) return 0;
      continue;
    } else if (q.yield_idle && head > retired) {
      const unsigned long long need = (head - retired + kTcM - 1) / kTcM + unsigned(q.yield_idle);
      const unsigned left = *reinterpret_cast<volatile unsigned*>(q.exited);
      if (gridDim.x > left && gridDim.x - left - 1 >= need) {
        const unsigned old = atomicAdd(q.exited, 1u);
        if (gridDim.x > old && gridDim.x - old - 1 >= need) return 0;
        atomicSub(q.exited, 1u);
      }
    }
    __nanosleep(64);
  }
  return -1;
}

// Non-blocking claim of a full tile for a CTA that is still evaluating one:
// kTcM items if that many are queued now, else kPqNoTile (the CTA then claims
// after retiring its tile, with pq_claim's waiting rules).
constexpr int kPqNoTile = -2147483647 - 1;
__device__ __forceinline__ int pq_try_claim(const PQueue& q, unsigned long long* start) {
  for (int attempt = 0; attempt < 4; ++attempt) {
    const unsigned long long head = ld_relaxed_u64(q.head);
    const unsigned long long res = ld_relaxed_u64(q.reserved);
    if (res < head + kTcM) return kPqNoTile;
    if (atomicCAS(q.head, head, head + kTcM) == head) {
      atomicAdd(q.tiles, 1u);
      *start = head;
      return kTcM;
    }
  }
  return kPqNoTile;
}

// Take the item at ring position p (its producer may still be writing it) and
// leave the entry empty for position p + n; the acquire orders the ray's
// record reads after it. Returns kPqEmpty if the wait gave up.
__device__ __forceinline__ unsigned long long pq_take(const PQueue& q, unsigned long long p, unsigned long long n) {
  unsigned long long* e = q.ring + p % n;
  for (long long spin = 0; spin < q.spin_limit; ++spin) {
    const unsigned long long v = exch_acquire_u64(e, kPqEmpty);
    if (v != kPqEmpty) return v;
    __nanosleep(32);
  }
  return kPqEmpty;
}

// Write an item into the (empty) entry of position p; the release orders this
// thread's record writes before it. Returns false if the wait gave up.
__device__ __forceinline__ bool pq_put(const PQueue& q, unsigned long long p, unsigned long long n,
                                       unsigned long long item) {
  unsigned long long* e = q.ring + p % n;
  for (long long spin = 0; spin < q.spin_limit; ++spin) {
    if (cas_release_u64(e, kPqEmpty, item) == kPqEmpty) return true;
    __nanosleep(32);
  }
  return false;
}

// ---------------------------------------------------------------- row buffers
// One tile's rows in shared memory, structure of arrays.
struct RowBuf {
  int* ray;     // -1: an empty row
  float* t0;
  float* t1;
  int* slot;    // persistent query: the item's segment slot
  float* best;  // persistent query: the ray's best t when the item was taken
  float* next;  // persistent query: the start of the ray's next segment (+inf: none)
  float* o[3];
  float* d[3];
};

__device__ __forceinline__ RowBuf row_buf(uint8_t* base) {
  RowBuf b;
  float* f = reinterpret_cast<float*>(base);
  b.ray = reinterpret_cast<int*>(f);
  b.t0 = f + kTcM;
  b.t1 = f + 2 * kTcM;
  b.slot = reinterpret_cast<int*>(f + 3 * kTcM);
  b.best = f + 4 * kTcM;
  b.next = f + 5 * kTcM;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    b.o[i] = f + (6 + i) * kTcM;
    b.d[i] = f + (9 + i) * kTcM;
  }
  return b;
}

// Row r holds segment [t0, t1] of ray `ray` (-1: empty): origin and direction
// are copied next to it so the gather reads them from shared memory.
__device__ __forceinline__ void put_row(const RowBuf& b, const RayPtrs& rays, int r, int ray, float t0, float t1) {
  b.ray[r] = ray;
  b.t0[r] = t0;
  b.t1[r] = t1;
  const bool v = ray >= 0;
  b.o[0][r] = v ? rays.ox[ray] : 0.0f;
  b.o[1][r] = v ? rays.oy[ray] : 0.0f;
  b.o[2][r] = v ? rays.oz[ray] : 0.0f;
  b.d[0][r] = v ? rays.dx[ray] : 0.0f;
  b.d[1][r] = v ? rays.dy[ray] : 0.0f;
  b.d[2][r] = v ? rays.dz[ray] : 0.0f;
}

// Sample k of row r's segment in grid coordinates (S2).
__device__ __forceinline__ void row_point(const GridParams& gp, const RowBuf& b, int r, int k, float* p) {
  sample_point(gp, b.o[0][r], b.o[1][r], b.o[2][r], b.d[0][r], b.d[1][r], b.d[2][r], b.t0[r], b.t1[r], k, p[0],
               p[1], p[2]);
}

// Stage row r of a claimed tile (item at ring position p): the ray, its
// segment's interval, its best t and its next segment's t0. Returns the ray
// (-1 if the wait gave up, or the entry holds no item of this query: only
// announced items that nothing writes, the test hook, can find one).
__device__ __forceinline__ int pq_stage(const EvalArgs& a, unsigned long long p, int r, const RowBuf& b) {
  const size_t nr = size_t(a.n_rays);
  const unsigned long long it = pq_take(a.pq, p, pq_ring_n(a.pq));
  int ray = -1;
  float t0 = 0.0f, t1 = 0.0f;
  const uint32_t iray = uint32_t(it), isl = uint32_t(it >> 32);
  if (it == kPqEmpty || iray >= uint32_t(a.n_rays) || isl >= uint32_t(a.max_segs)) {
    set_status(NBVH_ERR_TIMEOUT);
  } else {
    ray = int(iray);
    const int sl = int(isl);
    b.slot[r] = sl;
    const size_t q = size_t(sl) * nr + size_t(ray);
    t0 = a.seg_t0[q];
    t1 = a.seg_t1[q];
    b.best[r] = __ldcg(a.hits.t + ray);
    // the slot after the last holds stale data: load it with the count, use it only below the count
    const int cnt = a.seg_count[ray];
    const size_t qn = size_t(sl + 1) * nr + size_t(ray);
    const float tn = sl + 1 < a.max_segs ? fminf(a.seg_t0[qn], a.seg_t1[qn]) : 0.0f;  // its start
    b.next[r] = sl + 1 < cnt ? tn : __int_as_float(0x7f800000);
  }
  put_row(b, a.rays, r, ray, t0, t1);
  return ray;
}

// Resolve one evaluated segment (slot sl of ray `ray`) into the ray's record.
// best and next_t0 (the ray's best t and its next segment's t0, +inf if none)
// were read when the item was taken: only this item's evaluation changes the
// ray's record while it is alive. Returns whether the next segment is queued
// (it starts before the best t).
__device__ __forceinline__ bool pq_resolve(const EvalArgs& a, int ray, int sl, float best, float next_t0,
                                           const float* raw, float t0, float t1) {
  SegResult s = decode_segment(raw, t0, t1);
  if (s.hit && t0 > t1) s.hit = s.t > a.rays.tmin[ray] && s.t <= a.rays.tmax[ray];  // reversed chord
  if (s.hit && s.t < best) {
    best = s.t;
    a.hits.t[ray] = s.t;
    a.hits.hit[ray] = 1;
    a.hits.nx[ray] = s.nx;
    a.hits.ny[ray] = s.ny;
    a.hits.nz[ray] = s.nz;
    a.hits.leaf[ray] = a.seg_leaf[size_t(sl) * size_t(a.n_rays) + size_t(ray)];
    if (a.inst_out) a.inst_out[ray] = a.inst_id;
    write_albedo(a, ray, raw);
  }
  return next_t0 < best;
}

// Resolve the rows of one claimed item in slot order: row `row` holds the
// item (slot s of its ray) and, in a partial tile, rows row + c, row + 2c, ...
// hold the ray's next segments s + 1, s + 2, ... (lookahead rows staged while
// they started before the ray's best t). The closest predicted hit over them
// (ties to the earlier slot) updates the ray's record, evaluation stopping
// at the first row that starts at or beyond the best t so far. *last = the
// last slot evaluated. Returns whether the segment after it is queued (it
// starts before the best t). raw: the tile's raw outputs, 8 per row.
__device__ __forceinline__ bool pq_resolve_rows(const EvalArgs& a, const RowBuf& rb, const float* raw, int row, int c,
                                                int* last) {
  const int ray = rb.ray[row];
  const size_t nr = size_t(a.n_rays);
  float best = rb.best[row];
  int win = -1, l = rb.slot[row];
  SegResult w;
  w.hit = false;
  w.t = w.nx = w.ny = w.nz = 0.0f;
  for (int j = row, m = 0; j < kTcM; j += c, ++m) {
    if (m > 0 && (rb.ray[j] != ray || !(fminf(rb.t0[j], rb.t1[j]) < best))) break;
    SegResult s = decode_segment(raw + j * 8, rb.t0[j], rb.t1[j]);
    if (s.hit && rb.t0[j] > rb.t1[j]) s.hit = s.t > a.rays.tmin[ray] && s.t <= a.rays.tmax[ray];  // reversed chord
    if (s.hit && s.t < best) {
      best = s.t;
      win = j;
      w = s;
    }
    l = rb.slot[j];
  }
  if (win >= 0) {
    a.hits.t[ray] = w.t;
    a.hits.hit[ray] = 1;
    a.hits.nx[ray] = w.nx;
    a.hits.ny[ray] = w.ny;
    a.hits.nz[ray] = w.nz;
    a.hits.leaf[ray] = a.seg_leaf[size_t(rb.slot[win]) * nr + size_t(ray)];
    if (a.inst_out) a.inst_out[ray] = a.inst_id;
    write_albedo(a, ray, raw + win * 8);
  }
  *last = l;
  if (l + 1 >= a.seg_count[ray]) return false;
  const size_t qn = size_t(l + 1) * nr + size_t(ray);
  return fminf(a.seg_t0[qn], a.seg_t1[qn]) < best;
}

// The traversal queued the first items at ring positions [0, *qlen0).
// phantom > 0 (a test hook) announces that many further items that nothing
// ever writes, so that the waits for them run out.
static __global__ void pq_init_kernel(const int32_t* __restrict__ qlen0, PQueue q, int32_t phantom) {
  *q.reserved = (unsigned long long)(*qlen0) + (unsigned long long)(phantom > 0 ? phantom : 0);
}

// The four corners of the cell of level l at (x, y, z) whose x offset is xb:
// table indices (level-relative) for (y, z) offsets (0,0), (1,0), (0,1), (1,1)
// and the matching trilinear weights.
__device__ __forceinline__ void level_xhalf(const GridParams& gp, int l, const float* p, int xb, uint32_t* idx,
                                            float* w) {
  const int N = gp.res[l];
  int cx, cy, cz;
  float fx, fy, fz;
  axis_cell(p[0], N, cx, fx);
  axis_cell(p[1], N, cy, fy);
  axis_cell(p[2], N, cz, fz);
  const float wx = xb ? fx : 1.0f - fx;
  const float wy[2] = {1.0f - fy, fy};
  const float wz[2] = {1.0f - fz, fz};
  if (gp.dense[l]) {
    const uint32_t n1 = static_cast<uint32_t>(N) + 1u;
    const uint32_t base = static_cast<uint32_t>(cx + xb) + static_cast<uint32_t>(cy) * n1 +
                          static_cast<uint32_t>(cz) * n1 * n1;
#pragma unroll
    for (int k = 0; k < 4; ++k) idx[k] = base + (k & 1) * n1 + ((k >> 1) & 1) * n1 * n1;
  } else {
    const uint32_t hx = static_cast<uint32_t>(cx + xb);
    const uint32_t hy = static_cast<uint32_t>(cy) * kHashP1;
    const uint32_t hz = static_cast<uint32_t>(cz) * kHashP2;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t b = (k & 1) ? hy + kHashP1 : hy;
      const uint32_t d = (k & 2) ? hz + kHashP2 : hz;
      idx[k] = (hx ^ b ^ d) & gp.hash_mask;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = wx * wy[k & 1] * wz[(k >> 1) & 1];
}

// Partial features (x-offset xb corners only) of NL levels from l0 at two
// points: all 8 NL corner loads are issued before any is consumed, and the
// weights computed with the indices are kept for the interpolation. Invalid
// points contribute zeros.
template <typename T, int NL>
__device__ __forceinline__ void encode_xhalf(const GridParams& gp, const T* __restrict__ table, int l0,
                                             const float* p0, const float* p1, bool v0, bool v1, int xb,
                                             float* out0, float* out1) {
  uint32_t raw[2][NL][4];
  float w[2][NL][4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float* p = h ? p1 : p0;
    const bool v = h ? v1 : v0;
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      uint32_t idx[4];
      level_xhalf(gp, l0 + q, p, xb, idx, w[h][q]);
      const uint32_t* tab = reinterpret_cast<const uint32_t*>(table + size_t(gp.offset[l0 + q]) * 2);
#pragma unroll
      for (int k = 0; k < 4; ++k) raw[h][q][k] = v ? __ldg(tab + idx[k]) : 0u;
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float* out = h ? out1 : out0;
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float2 v;
        if constexpr (std::is_same<T, __half>::value) {
          v = __half22float2(*reinterpret_cast<const __half2*>(&raw[h][q][k]));
        } else {
          v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw[h][q][k]));
        }
        a0 = fmaf(w[h][q][k], v.x, a0);
        a1 = fmaf(w[h][q][k], v.y, a1);
      }
      out[2 * q] = a0;
      out[2 * q + 1] = a1;
    }
  }
}

// ---------------------------------------------------------------- bulk copies (TMA unit)
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Contiguous global -> shared copy of `bytes` (16-byte aligned ends, a multiple
// of 16 bytes) that completes on `bar`'s transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// The first layer's weights (FP32 [W][K] row-major) into the chunked B-operand
// layout (w1_chunk_offset) with zero rows for the padding: into shared memory
// by a CTA (resident weights) or into global memory by w1_image_kernel.
template <bool BF16>
__device__ __forceinline__ void put_w1(uint8_t* dst, const float* __restrict__ W1, int i, int W, int K, int L, int F,
                                       int N, const TcLayout& T) {
  const int cols = T.R * T.KC;
  const int n = i / cols, c = i - n * cols;
  const int f = padded_feature(c, L, F, N, T.LFp);
  const float v = f >= 0 ? __ldg(W1 + size_t(n) * K + f) : 0.0f;
  *reinterpret_cast<typename OpType<BF16>::T*>(dst + w1_chunk_offset(n, c, T)) = OpType<BF16>::one(v);
}

// Streamed first-layer weights: the 16-bit chunked image the kernel's bulk
// copies read (R * chunk_bytes bytes, 16-byte aligned).
template <bool BF16>
__global__ void __launch_bounds__(256) w1_image_kernel(const float* __restrict__ W1, int W, int K, int L, int F, int N,
                                                       TcLayout T, uint8_t* __restrict__ img) {
  const int total = W * T.R * T.KC;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
    put_w1<BF16>(img, W1, i, W, K, L, F, N, T);
}

// One item (levels l0 .. l0 + 3 of one sample, F = 2, 4-byte entries) of the
// two rows a lane pair shares (x-corner lane split): each lane gathers the
// corners with x bit xb of both rows, then the partners swap partial sums so
// that lane i returns its own row's 8 features, packed to 16 bits. Levels at
// or beyond L give zeros.
template <typename T, bool BF16, bool FULL>
__device__ __forceinline__ void split_item(const GridParams& gp, const T* __restrict__ table, int l0, int L,
                                           const float* p0, const float* p1, bool v0, bool v1, int xb,
                                           uint32_t* pk) {
  float h0[8], h1[8];  // partial features of rows r0 and r1 over this lane's x bit
  if constexpr (FULL) {
    encode_xhalf<T, 2>(gp, table, l0, p0, p1, v0, v1, xb, h0, h1);
    encode_xhalf<T, 2>(gp, table, l0 + 2, p0, p1, v0, v1, xb, h0 + 4, h1 + 4);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (l0 + q < L) {
        encode_xhalf<T, 1>(gp, table, l0 + q, p0, p1, v0, v1, xb, h0 + 2 * q, h1 + 2 * q);
      } else {
        h0[2 * q] = h0[2 * q + 1] = h1[2 * q] = h1[2 * q + 1] = 0.0f;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // send the partner the row it owns (r1 for lanes 0-15, r0 for 16-31)
    const float s0 = xb ? h0[2 * i] : h1[2 * i], s1 = xb ? h0[2 * i + 1] : h1[2 * i + 1];
    const float g0 = __shfl_xor_sync(0xffffffffu, s0, 16), g1 = __shfl_xor_sync(0xffffffffu, s1, 16);
    const float m0 = xb ? h1[2 * i] : h0[2 * i], m1 = xb ? h1[2 * i + 1] : h0[2 * i + 1];
    pk[i] = pack2<BF16>(m0 + g0, m1 + g1);
  }
}

// One item (8 / F levels from l0 of one sample) of one row; levels at or
// beyond L give zeros.
template <typename T, int F>
__device__ __forceinline__ void row_item(const GridParams& gp, const T* __restrict__ table, int l0, int L,
                                         const float* p, float* v) {
  constexpr int LPC = 8 / F;
  if (l0 + LPC <= L) {
    if constexpr (LPC == 4) {
      encode_levels<T, F, 4>(gp, table, l0, p[0], p[1], p[2], v);
    } else if constexpr (LPC % 2 == 0) {
#pragma unroll
      for (int q = 0; q < LPC; q += 2) encode_levels<T, F, 2>(gp, table, l0 + q, p[0], p[1], p[2], v + q * F);
    } else {
      encode_levels<T, F, LPC>(gp, table, l0, p[0], p[1], p[2], v);
    }
  } else {
#pragma unroll
    for (int q = 0; q < LPC; ++q) {
      if (l0 + q < L) {
        encode_level<T, F>(gp, table, l0 + q, p[0], p[1], p[2], v + q * F);
      } else {
#pragma unroll
        for (int f = 0; f < F; ++f) v[q * F + f] = 0.0f;
      }
    }
  }
}

// MODE 0: list of segments -> raw outputs; 1: query -> resolve + next segment
// queued (one launch per segment slot, or with a.pq.ring set one persistent
// launch draining the queue); 2: training forward (one segment per ray) ->
// stored 16-bit operands, raw outputs, loss and dL/d(raw).
// NT threads = NT / 128 warp groups; each warp group gathers 16 / (NT / 128)
// items of every K chunk for all 128 rows of the tile. With W <= 64 the CTA
// holds 256 TMEM columns, so two 256-thread CTAs share an SM and one CTA's
// barriers, MMAs and queue claims overlap the other's gather.
template <typename T, int F, int W, int MODE, bool BF16, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) eval_tc_kernel(EvalArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  constexpr int kGroups = NT / 128;
  constexpr int LPC = 8 / F;                  // levels per item
  constexpr int kCols = W / kGroups;          // accumulator columns per thread in hidden epilogues
  static_assert(kCols % 8 == 0 || kCols == 4 || kCols == 8, "epilogue column split");
  const int K = a.gp.n_inputs;
  const int L = a.gp.n_levels;
  const int N = a.gp.n_samples;
  const int n_out = a.n_out;
  const bool stream = a.w1_image != nullptr;
  const TcLayout lay = tc_layout(L, F, N, W, a.n_hidden, stream, NT);
  const int CI = lay.KC / kItemF;   // items per chunk
  const int IPG = CI / kGroups;     // items per warp group and chunk
  uint8_t* sW1 = smem + lay.w1_off;
  uint8_t* sWh = smem + lay.wh_off;
  uint8_t* sWo = smem + lay.wo_off;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + lay.bar_off);  // [0] hidden/output MMAs
  uint64_t* mma_done = bar + 1;                                      // [2] first-layer chunk MMAs
  uint64_t* w_full = bar + 3;                                        // [2] streamed weight chunks
  uint64_t* bar_fin = bar + 5;                                       // exit: every MMA retired
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 6);
  uint8_t* const rows_base = smem + lay.row_off;  // row buffer b at rows_base + b * kTcM * kRowBytes
  __shared__ unsigned long long s_start[2];
  __shared__ int s_count[2];  // per row buffer: its tile's item count, kPqNoTile when nothing is staged
  __shared__ int s_fail;

  // A persistent query's CTAs claim tiles from the queue until it drains.
  const bool persistent = MODE == 1 && a.pq.ring != nullptr;
  const int64_t n_items = MODE == 1 ? (persistent ? 0 : int64_t(*a.qlen)) : a.n_items;
  const int64_t n_tiles = persistent ? INT64_MAX : (n_items + kTcM - 1) / kTcM;
  if (!persistent && int64_t(blockIdx.x) >= n_tiles) return;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (warp == 0) {
    tmem_alloc(s_tmem, lay.ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 6; ++i) mbar_init(bar + i, 1);
    fence_mbar_init();
    s_count[0] = kPqNoTile;
    s_count[1] = kPqNoTile;
    s_fail = 0;
  }

  // Weights -> operand layouts (converted once per CTA; the first layer's only
  // when they stay resident).
  const float* W1 = a.mlp;
  const float* b1 = W1 + size_t(W) * K;
  if (!stream && a.w1_copy) {  // resident from the prepared image: bulk copies, waited for below
    if (threadIdx.x == 0) {
      const uint32_t bytes = uint32_t(lay.R) * lay.chunk_bytes;
      mbar_expect_tx(w_full, bytes);
      for (uint32_t o = 0; o < bytes; o += 32768u)
        bulk_g2s(sW1 + o, static_cast<const uint8_t*>(a.w1_copy) + o, min(32768u, bytes - o), w_full);
    }
  } else if (!stream) {
    for (int i = threadIdx.x; i < W * lay.R * lay.KC; i += NT) put_w1<BF16>(sW1, W1, i, W, K, L, F, N, lay);
  }
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

  const uint32_t idesc_h = idesc_f16(BF16, kTcM, W);
  const uint32_t idesc_o = idesc_f16(BF16, kTcM, 16);
  const T* table = static_cast<const T*>(a.table);
  // Warp -> TMEM lane quarter (warp % 4) and column group (warp / 4).
  const int quarter = warp & 3;
  const int cgroup = warp >> 2;
  const int row = quarter * 32 + lane;
  const uint32_t t_row = tmem + (uint32_t(quarter * 32) << 16);
  uint32_t phase = 0;         // parity of `bar`
  uint32_t g = 0;             // first-layer chunk rounds so far (buffer g & 1)
  uint32_t tma_pending[2] = {~0u, ~0u};  // thread 0: round of a streamed copy not yet seen complete
  bool failed = false;
  if (!stream && a.w1_copy && !mbar_wait(w_full, 0)) failed = true;  // the resident image copy
  constexpr bool kSplitX = F == 2 && sizeof(T) == 2;  // 4-byte entries: x-corner lane split

  int cur = 0;  // persistent query: the row buffer of the tile being evaluated
  for (int64_t tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
    int ccount = 0;       // persistent query: items in this tile
    bool staged = false;  // its rows were staged while the previous tile finished
    const RowBuf rb = row_buf(rows_base + size_t(cur) * kTcM * kRowBytes);
    if (persistent) {
      const int pre = s_count[cur];
      if (pre != kPqNoTile) {
        ccount = pre;
        staged = true;
      } else {
        __syncthreads();  // every thread has read s_count[cur]; the previous tile is retired
        if (threadIdx.x == 0) {
          unsigned long long st = 0;
          s_count[cur] = pq_claim(a.pq, &st);
          s_start[cur] = st;
        }
        __syncthreads();
        ccount = s_count[cur];
        if (ccount <= 0) {
          failed = ccount < 0;
          break;
        }
      }
    }
    if (persistent && !staged) {
      if (threadIdx.x < kTcM) {
        if (int(threadIdx.x) < ccount)
          pq_stage(a, s_start[cur] + threadIdx.x, threadIdx.x, rb);
        else
          put_row(rb, a.rays, threadIdx.x, -1, 0.0f, 0.0f);
      }
      __syncthreads();
      if (ccount < kTcM) {
        // A partial tile (the queue runs shallow): the empty rows take the
        // claimed rays' next segments (row c + (e - 1) c + i: item i's e-th
        // next slot) while they start before the ray's best t, so a ray's
        // chain of segments advances several slots per tile.
        bool staged = false;
        if (threadIdx.x >= ccount && threadIdx.x < kTcM) {
          const int j = int(threadIdx.x) - ccount;
          const int i = j % ccount, e = j / ccount + 1;
          const int ray = rb.ray[i];
          int sl = -1;
          float t0 = 0.0f, t1 = 0.0f;
          if (ray >= 0) {
            sl = rb.slot[i] + e;
            if (sl < a.seg_count[ray]) {
              const size_t q = size_t(sl) * size_t(a.n_rays) + size_t(ray);
              t0 = a.seg_t0[q];
              t1 = a.seg_t1[q];
              if (!(fminf(t0, t1) < rb.best[i])) sl = -1;
            } else {
              sl = -1;
            }
          }
          put_row(rb, a.rays, threadIdx.x, sl >= 0 ? ray : -1, t0, t1);
          rb.slot[threadIdx.x] = sl;
          staged = sl >= 0;
        }
        const int n_staged = __syncthreads_count(staged);
        if (threadIdx.x == 0 && n_staged > 0) atomicAdd(a.pq.lookahead, (unsigned long long)n_staged);
      }
    } else if (!persistent) {
      if (threadIdx.x < kTcM) {
        const int64_t i = tile * kTcM + threadIdx.x;
        int ray = -1;
        float t0 = 0.0f, t1 = 0.0f;
        if (i < n_items) {
          if constexpr (MODE == 1) {
            const size_t nr = size_t(a.n_rays);
            ray = a.queue[i];
            const size_t q = size_t(a.wave) * nr + size_t(ray);
            t0 = a.seg_t0[q];
            t1 = a.seg_t1[q];
          } else if constexpr (MODE == 2) {
            const int r = a.tr.order ? a.tr.order[i] : int(i);
            ray = a.tr.leaf[r] >= 0 ? r : -1;
            t0 = a.list_t0[r];
            t1 = a.list_t1[r];
          } else {
            ray = a.seg_ray[i];
            t0 = a.list_t0[i];
            t1 = a.list_t1[i];
          }
        }
        put_row(rb, a.rays, threadIdx.x, ray, t0, t1);
      }
      __syncthreads();
    }
    const int64_t grow = tile * kTcM + row;  // global item of this thread's row
    uint16_t* x16 = nullptr;                 // training: this item's column of the stored features
    if constexpr (MODE == 2) {
      if (grow < n_items) x16 = a.tr.X16 + grow;
    }
    const int64_t xld = MODE == 2 ? a.tr.ld : 0;
    // feature-major store of the valid features of one item (original order)
    auto store_item = [&](int k, int l0, const uint32_t* pk) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (l0 + j / F < L) x16[int64_t(k * L * F + l0 * F + j) * xld] = uint16_t(pk[j >> 1] >> (16 * (j & 1)));
      }
    };

    // ---- layer 1 over K chunks: gather chunk r into buffer g % NB while the
    // tensor cores multiply chunk r - 1
    for (int r = 0; r < lay.R; ++r, ++g) {
      const int b = lay.NB == 1 ? 0 : int(g & 1u);  // TMEM feature buffer
      const int wbuf = int(g & 1u);                 // streamed weight buffer
      if (g >= uint32_t(lay.NB)) {
        // this round's buffers were read by the MMAs of round g - NB (their
        // completion implies every earlier round's): each thread waits for it
        // itself, a failed wait shows at the next barrier
        const uint32_t gw = g - uint32_t(lay.NB);
        if (!mbar_wait(mma_done + (gw & 1u), (gw >> 1) & 1u)) s_fail = 1;
        tc_fence_after();
      }
      if (stream && threadIdx.x == 0 && !s_fail) {  // after a failed wait no further copy is issued
        mbar_expect_tx(w_full + wbuf, lay.chunk_bytes);
        bulk_g2s(sW1 + size_t(wbuf) * lay.chunk_bytes,
                 static_cast<const uint8_t*>(a.w1_image) + size_t(r) * lay.chunk_bytes, lay.chunk_bytes,
                 w_full + wbuf);
        tma_pending[wbuf] = g;
      }
      const uint32_t t_buf = t_row + lay.col_a + uint32_t(b * (lay.KC / 2));
      const int it_begin = r * CI + cgroup * IPG;  // this warp group's first item
      const int c_begin = cgroup * IPG * 4;                   // its first column in the buffer
      if constexpr (kSplitX) {
        // Lanes i and i ^ 16 share cells: lane i loads the four corners with
        // x bit (i >> 4) of rows 32q + (i & 15) and 32q + 16 + (i & 15), so one
        // warp request fetches both x-neighbours of 16 cells (one 128-byte
        // line almost always) instead of 32 cells' corners with one x bit.
        const int xb = lane >> 4;
        const int r0 = quarter * 32 + (lane & 15), r1 = r0 + 16;
        const bool v0 = rb.ray[r0] >= 0, v1 = rb.ray[r1] >= 0;
        float p0[3] = {0.0f, 0.0f, 0.0f}, p1[3] = {0.0f, 0.0f, 0.0f};
        if (L == 16 && lay.IPS == 4 && IPG % 4 == 0 && it_begin % 4 == 0) {
          // whole samples per warp group, the 16 levels unrolled
#pragma unroll 1
          for (int s = 0; s < IPG / 4; ++s) {
            const int k = it_begin / 4 + s;
            const uint32_t col = uint32_t(c_begin + 16 * s);
            if (k < N) {
              if (v0) row_point(a.gp, rb, r0, k, p0);
              if (v1) row_point(a.gp, rb, r1, k, p1);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                uint32_t pk[4];
                split_item<T, BF16, true>(a.gp, table, 4 * q, 16, p0, p1, v0, v1, xb, pk);
                if (x16) store_item(k, 4 * q, pk);
                __syncwarp();
                tmem_st4(t_buf + col + 4 * q, pk);
              }
            } else {
              const uint32_t z[4] = {0u, 0u, 0u, 0u};
#pragma unroll
              for (int q = 0; q < 4; ++q) tmem_st4(t_buf + col + 4 * q, z);
            }
          }
        } else {
          int kcur = -1;
#pragma unroll 1
          for (int i = 0; i < IPG; ++i) {
            const int it = it_begin + i;
            uint32_t pk[4] = {0u, 0u, 0u, 0u};
            if (it < lay.NI) {
              const int k = it / lay.IPS, l0 = (it - k * lay.IPS) * 4;
              if (k != kcur) {
                if (v0) row_point(a.gp, rb, r0, k, p0);
                if (v1) row_point(a.gp, rb, r1, k, p1);
                kcur = k;
              }
              if (l0 + 4 <= L)
                split_item<T, BF16, true>(a.gp, table, l0, L, p0, p1, v0, v1, xb, pk);
              else
                split_item<T, BF16, false>(a.gp, table, l0, L, p0, p1, v0, v1, xb, pk);
              if (x16) store_item(k, l0, pk);
            }
            __syncwarp();
            tmem_st4(t_buf + uint32_t(c_begin + 4 * i), pk);
          }
        }
      } else {
        const bool valid = rb.ray[row] >= 0;
        float pt[3] = {0.0f, 0.0f, 0.0f};
        int kcur = -1;
#pragma unroll 1
        for (int i = 0; i < IPG; ++i) {
          const int it = it_begin + i;
          float v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = 0.0f;
          int k = 0, l0 = 0;
          if (it < lay.NI) {
            k = it / lay.IPS;
            l0 = (it - k * lay.IPS) * LPC;
            if (valid) {
              if (k != kcur) {
                row_point(a.gp, rb, row, k, pt);
                kcur = k;
              }
              row_item<T, F>(a.gp, table, l0, L, pt, v);
            }
          }
          uint32_t pk[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) pk[j] = pack2<BF16>(v[2 * j], v[2 * j + 1]);
          if (x16 && it < lay.NI) store_item(k, l0, pk);
          __syncwarp();
          tmem_st4(t_buf + uint32_t(c_begin + 4 * i), pk);
        }
      }
      tmem_st_wait();
      tc_fence_before();
      __syncthreads();
      if (threadIdx.x == 0) {
        tc_fence_after();
        bool ok = !s_fail;
        if (stream && ok) {
          ok = mbar_wait(w_full + wbuf, (g >> 1) & 1u);
          if (ok) tma_pending[wbuf] = ~0u;
        }
        if (ok) {
          const int steps = min(lay.KC, lay.KP - r * lay.KC) / 16;
          const uint32_t wb = smem_u32(sW1 + size_t(stream ? wbuf : r) * lay.chunk_bytes);
          for (int j = 0; j < steps; ++j)
            mma_f16_ts(tmem, tmem + lay.col_a + uint32_t(b * (lay.KC / 2) + 8 * j),
                       smem_desc(wb + j * 256, 128, uint32_t(lay.KC) * 16), idesc_h, (r > 0 || j > 0) ? 1u : 0u);
        } else {
          s_fail = 1;
        }
        mma_commit(mma_done + (g & 1u));  // also when nothing was issued: keeps the phases in step
      }
    }
    if (failed) break;
    {  // the first layer's last chunk (and with it every earlier one) is done
      const uint32_t gl = g - 1;
      const bool ok = mbar_wait(mma_done + (gl & 1u), (gl >> 1) & 1u);
      if (__syncthreads_or(!ok || s_fail)) {
        failed = true;
        break;
      }
      tc_fence_after();
    }
    // ---- each hidden layer: bias + ReLU into H (TMEM), next MMA, wait
    for (int h = 0; h < a.n_hidden; ++h) {
      // bias of layer h: b0 follows W0; hidden layer h >= 1 is [W][W] then [W]
      const float* bias = h == 0 ? b1 : b1 + W + size_t(h - 1) * (W * W + W) + size_t(W) * W;
      if (h > 0) {
        const bool ok = mbar_wait(bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
          failed = true;
          break;
        }
        tc_fence_after();
      }
      {
        float v[kCols];
        tmem_ld_cols<kCols>(t_row + uint32_t(cgroup * kCols), v);
        tmem_ld_wait();
        const int c0 = cgroup * kCols;
        uint32_t pk[kCols / 2];
#pragma unroll
        for (int i = 0; i < kCols / 2; ++i)
          pk[i] = pack2<BF16>(fmaxf(v[2 * i] + __ldg(bias + c0 + 2 * i), 0.0f),
                              fmaxf(v[2 * i + 1] + __ldg(bias + c0 + 2 * i + 1), 0.0f));
        tmem_st_cols<kCols / 2>(t_row + lay.col_h + uint32_t(c0 / 2), pk);
        if constexpr (MODE == 2) {
          if (grow < n_items) {
            uint32_t* hdst = reinterpret_cast<uint32_t*>(a.tr.H16 + (size_t(h) * size_t(n_items) + size_t(grow)) * W + c0);
#pragma unroll
            for (int i = 0; i < kCols / 2; ++i) hdst[i] = pk[i];
            if (a.tr.HT16 && h + 1 < a.n_hidden) {  // the next hidden layer's weight gradient reads it neuron-major
              uint16_t* hT = a.tr.HT16 + (size_t(h) * W + c0) * size_t(xld) + size_t(grow);
#pragma unroll
              for (int i = 0; i < kCols / 2; ++i) {
                hT[size_t(2 * i) * size_t(xld)] = uint16_t(pk[i] & 0xffffu);
                hT[size_t(2 * i + 1) * size_t(xld)] = uint16_t(pk[i] >> 16);
              }
            }
          }
        }
        tmem_st_wait();
      }
      tc_fence_before();
      __syncthreads();
      if (threadIdx.x == 0) {
        tc_fence_after();
        const uint32_t sbo = uint32_t(W) * 16;
        const uint32_t wa = smem_u32(h + 1 < a.n_hidden ? sWh + size_t(h) * W * W * 2 : sWo);
        const uint32_t idesc = h + 1 < a.n_hidden ? idesc_h : idesc_o;
        for (int j = 0; j < W / 16; ++j)
          mma_f16_ts(tmem, tmem + lay.col_h + uint32_t(8 * j), smem_desc(wa + j * 256, 128, sbo), idesc, j > 0);
        mma_commit(bar);
      }
    }
    if (failed) break;
    // ---- output layer epilogue: warps 0-3 hold rows 0..127, columns 0..15
    {
      const bool ok = mbar_wait(bar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after();
      if (cgroup == 0) {
        float v[16];
        tmem_ld16(t_row, v);
        tmem_ld_wait();
        float raw[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) raw[j] = j < n_out ? v[j] + __ldg(bo + j) : 0.0f;
        const int ray = rb.ray[row];
        if constexpr (MODE == 1) {
          if (persistent) {
            // each item's thread resolves its rows (the item and its
            // lookahead rows) in slot order; the row's ray id stays in the row
            // buffer only if the ray's next segment is queued, its slot
            // becomes the last one evaluated
            float* rawbuf = reinterpret_cast<float*>(smem + lay.raw_off);
#pragma unroll
            for (int j = 0; j < 8; ++j) rawbuf[row * 8 + j] = raw[j];
            asm volatile("bar.sync 3, 128;" ::: "memory");
            int last = rb.slot[row];
            const bool push = row < ccount && ray >= 0 && pq_resolve_rows(a, rb, rawbuf, row, ccount, &last);
            asm volatile("bar.sync 3, 128;" ::: "memory");
            rb.ray[row] = push ? ray : -1;
            rb.slot[row] = last;
          } else {
            wave_resolve(a, ray >= 0, ray, raw, rb.t0[row], rb.t1[row]);
          }
        } else if constexpr (MODE == 2) {
          if (grow < n_items) {
            float gr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            float term = 0.0f;
            if (a.tr.lab.hit && ray >= 0) {
              const float inv_valid = 1.0f / float(max(1, *a.tr.n_valid));
              const float ls = a.tr.loss_scale_dev ? *a.tr.loss_scale_dev : a.tr.loss_scale;
              float alb[3];
              const bool has_alb = n_out >= 8 && a.tr.lab.ar;
              if (has_alb) {
                alb[0] = a.tr.lab.ar[ray];
                alb[1] = a.tr.lab.ag[ray];
                alb[2] = a.tr.lab.ab[ray];
              }
              term = loss_terms(raw, float(a.tr.lab.hit[ray]), a.tr.lab.depth[ray], a.tr.lab.nx[ray],
                                a.tr.lab.ny[ray], a.tr.lab.nz[ray], has_alb ? alb : nullptr, ls * inv_valid, gr);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (j < n_out) a.tr.O[grow * n_out + j] = raw[j];
            if (a.tr.lab.hit) {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (j < n_out) a.tr.G[grow * n_out + j] = gr[j];
              a.tr.loss_seg[grow] = term;
            }
          }
        } else if (ray >= 0) {
          const int64_t i = tile * kTcM + row;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j < n_out) a.out[i * n_out + j] = raw[j];
        }
      } else if (persistent && cgroup == 1) {
        // meanwhile warps 4-7 claim the next tile if a full one is queued and
        // stage its rows into the other buffer
        const int nb = cur ^ 1;
        if (threadIdx.x == 128) {
          unsigned long long st = 0;
          s_count[nb] = pq_try_claim(a.pq, &st);
          s_start[nb] = st;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (s_count[nb] != kPqNoTile)
          pq_stage(a, s_start[nb] + (threadIdx.x - 128), threadIdx.x - 128,
                   row_buf(rows_base + size_t(nb) * kTcM * kRowBytes));
      }
      tc_fence_before();
      __syncthreads();
    }
    if (persistent) {
      // Warps 0-3 queue the next segments of this tile's rays (one reservation
      // per warp, each item written into its entry) and retire the tile's
      // items, while the other warps go on to the next tile.
      if (warp < 4) {
        const int pray = rb.ray[threadIdx.x];
        const unsigned m = __ballot_sync(0xffffffffu, pray >= 0);
        unsigned long long base = 0;
        if (m && lane == 0) base = atomicAdd(a.pq.reserved, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (pray >= 0) {
          const unsigned long long item = (unsigned long long)(rb.slot[threadIdx.x] + 1) << 32 | uint32_t(pray);
          if (!pq_put(a.pq, base + __popc(m & ((1u << lane) - 1u)), pq_ring_n(a.pq), item))
            set_status(NBVH_ERR_TIMEOUT);
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (threadIdx.x == 0) red_release_add_u64(a.pq.retired, (unsigned long long)ccount);  // after the reservations
      }
      cur ^= 1;
    }
  }
  if (failed) set_status(NBVH_ERR_TIMEOUT);
  __syncthreads();
  if (threadIdx.x == 0) {
    // before the columns are freed: every MMA this thread issued has retired,
    // and no bulk copy into shared memory is still in flight (bounded waits)
    mma_commit(bar_fin);
    if (!mbar_wait(bar_fin, 0)) set_status(NBVH_ERR_TIMEOUT);
    for (int b = 0; b < 2; ++b)
      if (tma_pending[b] != ~0u && !mbar_wait(w_full + b, (tma_pending[b] >> 1) & 1u)) set_status(NBVH_ERR_TIMEOUT);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, lay.ncols);
  }
}

// ---------------------------------------------------------------- launch plan
// Threads per CTA and placement of the first layer's weights for a model:
// 256 threads (two CTAs per SM: 256 TMEM columns and at most ~113 KB of
// shared memory each) or 512 (one CTA per SM); the weights resident in shared
// memory, or streamed chunk by chunk from a prepared 16-bit image when they do
// not fit (or when the caller asks for it).
struct TcPlan {
  bool ok;           // stageable (shared memory and TMEM within the SM's limits)
  int threads;       // 256 or 512
  bool stream;       // first-layer weights streamed from the image
  uint32_t smem;     // dynamic shared memory per CTA
  uint32_t ncols;    // TMEM columns per CTA
  size_t image_bytes;  // size of the streamed image (R chunks)
};

constexpr uint32_t kSmemMax = 227 * 1024;       // per CTA
constexpr uint32_t kSmemHalf = 113 * 1024;      // per CTA with two CTAs on an SM

// w1_mode NBVH_W1_AUTO: resident when it fits the CTA's budget, except that a
// query streams a first layer of more than kResidentW1Max bytes. Resident
// weights take their size out of the SM's unified L1 / shared memory: with
// the 128 KB layers (K = 1024) resident the mixed scene ran 11 % slower,
// while 64 KB layers (K = 512) resident made the icosphere query 1.7 %, the
// sphere-cluster query 4.6 % and the mixed scene 1 % faster.
constexpr size_t kResidentW1Max = 64 * 1024;
inline TcPlan tc_plan(const nbvh_model_desc* d, int threads_opt, int w1_mode, bool query = true) {
  TcPlan p;
  std::memset(&p, 0, sizeof(p));
  const int W = d->width;
  if (W < 32 || W > 128 || d->n_out > 16) return p;
  p.threads = threads_opt != 0 ? threads_opt : 512;
  if (p.threads != 256 && p.threads != 512) return p;
  if (p.threads == 256 && W > 64) return p;
  const TcLayout res = tc_layout(d->n_levels, d->n_features, d->n_samples, W, d->n_hidden, false, p.threads);
  const TcLayout str = tc_layout(d->n_levels, d->n_features, d->n_samples, W, d->n_hidden, true, p.threads);
  const uint32_t budget = p.threads == 256 ? kSmemHalf : kSmemMax;
  if (w1_mode == NBVH_W1_RESIDENT) p.stream = false;
  else if (w1_mode == NBVH_W1_STREAMED) p.stream = true;
  else p.stream = (query && size_t(res.R) * res.chunk_bytes > kResidentW1Max) || res.total > budget;
  const TcLayout& T = p.stream ? str : res;
  p.smem = T.total;
  p.ncols = T.ncols;
  p.image_bytes = size_t(T.R) * T.chunk_bytes;
  p.ok = T.total <= kSmemMax && T.ncols <= uint32_t(p.threads == 256 ? 256 : 512);
  return p;
}

// Bytes of the streamed first-layer image of any plan of this model (the
// chunking depends on the CTA size).
inline size_t tc_image_bytes(const nbvh_model_desc* d) {
  size_t m = 0;
  for (int th : {256, 512}) {
    if (th == 256 && d->width > 64) continue;
    const TcLayout T = tc_layout(d->n_levels, d->n_features, d->n_samples, d->width, d->n_hidden, true, th);
    m = std::max(m, size_t(T.R) * T.chunk_bytes);
  }
  return m;
}

template <typename T, int F, int W, int MODE, int NT>
cudaError_t launch_tc_nt(const nbvh_model_desc* d, const EvalArgs& a, int64_t n_items_max, const TcPlan& pl,
                         cudaStream_t s) {
  const bool bf16 = d->mlp_prec == NBVH_BF16;
  auto kern = bf16 ? eval_tc_kernel<T, F, W, MODE, true, NT> : eval_tc_kernel<T, F, W, MODE, false, NT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(pl.smem));
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, pl.smem);
  if (e != cudaSuccess) return e;
  // co-resident CTAs share the SM's 512 TMEM columns
  occ = std::min(occ, int(512 / pl.ncols));
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (n_items_max + kTcM - 1) / kTcM;
  int64_t grid = int64_t(sms) * occ;
  if (tiles < grid) grid = tiles;
  if (grid < 1) return cudaSuccess;
  kern<<<unsigned(grid), NT, pl.smem, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T, int F, int W, int MODE>
cudaError_t launch_tc_twf(const nbvh_model_desc* d, const EvalArgs& a, int64_t n, const TcPlan& pl, cudaStream_t s) {
  if (!pl.ok || (pl.stream && !a.w1_image) || (!pl.stream && a.w1_image)) return cudaErrorInvalidConfiguration;
  if constexpr (W <= 64) {
    if (pl.threads == 256) return launch_tc_nt<T, F, W, MODE, 256>(d, a, n, pl, s);
  }
  if (pl.threads == 512) return launch_tc_nt<T, F, W, MODE, 512>(d, a, n, pl, s);
  return cudaErrorInvalidConfiguration;
}

template <typename T, int F, int MODE>
cudaError_t launch_tc_tf(const nbvh_model_desc* d, const EvalArgs& a, int64_t n, const TcPlan& pl, cudaStream_t s) {
  switch (a.width) {
    case 32: return launch_tc_twf<T, F, 32, MODE>(d, a, n, pl, s);
    case 64: return launch_tc_twf<T, F, 64, MODE>(d, a, n, pl, s);
    case 128: return launch_tc_twf<T, F, 128, MODE>(d, a, n, pl, s);
  }
  return cudaErrorInvalidConfiguration;
}

// The kernels of one table type and mode (one translation unit each).
template <typename T, int MODE>
cudaError_t launch_tc_tm(const nbvh_model_desc* d, const EvalArgs& a, int64_t n, const TcPlan& pl, cudaStream_t s) {
  switch (d->n_features) {
    case 1: return launch_tc_tf<T, 1, MODE>(d, a, n, pl, s);
    case 2: return launch_tc_tf<T, 2, MODE>(d, a, n, pl, s);
    case 4: return launch_tc_tf<T, 4, MODE>(d, a, n, pl, s);
    case 8: return launch_tc_tf<T, 8, MODE>(d, a, n, pl, s);
  }
  return cudaErrorInvalidValue;
}

// The prepared image of the first layer's weights (plan with stream set).
inline cudaError_t launch_w1_image(const nbvh_model_desc* d, const float* mlp, int threads, void* img,
                                   cudaStream_t s) {
  const TcLayout T = tc_layout(d->n_levels, d->n_features, d->n_samples, d->width, d->n_hidden, true, threads);
  const int K = d->n_samples * d->n_levels * d->n_features;
  const int total = d->width * T.R * T.KC;
  const unsigned grid = unsigned(std::min(1024, (total + 255) / 256));
  if (d->mlp_prec == NBVH_BF16)
    w1_image_kernel<true><<<grid, 256, 0, s>>>(mlp, d->width, K, d->n_levels, d->n_features, d->n_samples, T,
                                               static_cast<uint8_t*>(img));
  else
    w1_image_kernel<false><<<grid, 256, 0, s>>>(mlp, d->width, K, d->n_levels, d->n_features, d->n_samples, T,
                                                static_cast<uint8_t*>(img));
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace nbvh
