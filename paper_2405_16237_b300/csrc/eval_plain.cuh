// S2..S5 fused on CUDA cores in FP32: stratified samples (float-float
// positions), hash-grid gather +
// trilinear interpolation into shared memory, FP32 MLP, decode and resolve.
#pragma once
#include "nbvh_internal.cuh"

namespace nbvh {

constexpr int kPlainTM = 32;        // segments per tile
constexpr int kPlainThreads = 256;

// ---------------------------------------------------------------------------
// S8 loss (Sec. 5.2 "Combined loss"): per valid segment
//   2 BCE(sigmoid(o_hit), y) + y (2 |sigmoid(o_d) - d| + (1/3) sum |o_n - n|),
// mean over valid segments; BCE from the logit. Returns the term and writes
// dL/do (times `scale`, divided by the valid count) to g[0..4].
// ---------------------------------------------------------------------------
struct Labels {
  const uint8_t* hit;
  const float *depth, *nx, *ny, *nz;
  const float *ar, *ag, *ab;  // albedo labels (n_out >= 8), or nullptr
};

__device__ __forceinline__ float sgnf(float x) { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); }

constexpr float kAlbedoEps = 1e-2f;  // relative L2: (y' - y)^2 / (y'^2 + eps), y' not differentiated

// Sec. 5.2 "Auxiliary intersection data": with an albedo head (outputs 5-7,
// sigmoid) and albedo labels alb (3 values), the term adds
// y (1/3) sum_c (s_c - a_c)^2 / (s_c^2 + eps), s_c = sigmoid(o_{5+c}), the
// denominator taken as a constant (relative L2), weight 1 in the combined loss.
__device__ __forceinline__ float loss_terms(const float* o, float y, float d, float n0, float n1, float n2,
                                            const float* alb, float gscale, float* g) {
  const float x = o[0];
  const float bce = fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x))) - y * x;
  const float s0 = sigmoidf_(x);
  const float s1 = sigmoidf_(o[1]);
  const float dd = s1 - d;
  const float e0 = o[2] - n0, e1 = o[3] - n1, e2 = o[4] - n2;
  float term = 2.0f * bce + y * (2.0f * fabsf(dd) + (fabsf(e0) + fabsf(e1) + fabsf(e2)) * (1.0f / 3.0f));
  g[0] = gscale * 2.0f * (s0 - y);
  g[1] = gscale * y * 2.0f * sgnf(dd) * s1 * (1.0f - s1);
  g[2] = gscale * y * (1.0f / 3.0f) * sgnf(e0);
  g[3] = gscale * y * (1.0f / 3.0f) * sgnf(e1);
  g[4] = gscale * y * (1.0f / 3.0f) * sgnf(e2);
  if (alb) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float sc = sigmoidf_(o[5 + c]);
      const float den = sc * sc + kAlbedoEps;
      const float diff = sc - alb[c];
      term += y * (1.0f / 3.0f) * diff * diff / den;
      g[5 + c] = gscale * y * (1.0f / 3.0f) * 2.0f * diff / den * sc * (1.0f - sc);
    }
  }
  return term;
}

// Extra outputs of the tensor-core kernel's training forward (segment i =
// ray i; leaf < 0 does not train): 16-bit copies of the features and hidden
// activations it fed to the tensor cores, raw outputs, and with labels the
// loss terms and dL/d(raw) times the loss scale.
struct TcTrain {
  const int32_t* leaf;
  const int32_t* order;  // item -> ray (rays grouped by leaf); nullptr: item = ray
  uint16_t* X16;      // [Kp][ld] feature-major (one row per feature, items along it)
  int64_t ld;         // row stride of X16 (items, rounded up to 64)
  uint16_t* H16;      // [n_hidden][n][W]
  uint16_t* HT16;     // [n_hidden - 1][W][ld] the hidden activations that feed a hidden
                      // layer again, neuron-major (nullptr: not stored)
  float* O;           // [n][n_out]
  float* G;           // [n][n_out]
  float* loss_seg;    // [n]
  Labels lab;         // hit == nullptr: no loss
  const int32_t* n_valid;
  float loss_scale;
  const float* loss_scale_dev;
};

// Persistent query queue (tensor-core query kernel, one launch for all
// segments of all rays). An item is (segment slot << 32 | ray) in a ring of
// R 64-bit entries (position p at p % R; an empty entry holds all ones), R =
// the items the traversal queued (*qlen0, at least 1). Only those rays ever
// get items and a ray has at most one item queued or in evaluation, so at most
// R items are ever alive and position p has been taken before p + R is
// reserved. The traversal's first items fill entries [0, R), so the ring
// needs no clearing: every later position finds its entry emptied by the
// consumer of the position R before it. Producers reserve positions and write
// each item into its entry; consumers claim positions [head, reserved) and
// take each item as soon as it is there; a tile retires its items after
// queueing their successors, so head - retired counts the items in
// evaluation.
struct PQueue {
  unsigned long long* head;      // items claimed
  unsigned long long* reserved;  // items ever queued
  unsigned long long* retired;   // items resolved
  unsigned int* tiles;           // tiles claimed (statistics)
  unsigned long long* lookahead; // segments evaluated in lookahead rows, never queued (statistics)
  unsigned int* exited;          // CTAs that left before the queue drained (their SMs go to other work)
  int32_t yield_idle;            // > 0: CTAs with nothing to claim leave while the rest (with yield_idle - 1
                                 // spares) suffice; their SMs go to concurrent kernels
  long long patience;            // cycles a CTA waits for a full tile before taking a partial one
  int32_t partial_items;         // the most items a partial tile claims (the rest of it: lookahead rows)
  long long spin_limit;          // polling rounds before a queue wait gives up (NBVH_ERR_TIMEOUT)
  unsigned long long* ring;      // [n_rays] items; nullptr: one launch per segment slot instead
  const int32_t* qlen0;          // the traversal's queued items: the ring's size R
  int32_t split;                 // > 0: a claim takes at most max(split, ceil(R / CTAs)) items (see pq_full)
};

// The ring's size R (read by any thread; the traversal wrote it before the launch).
__device__ __forceinline__ unsigned long long pq_ring_n(const PQueue& q) {
  const int32_t n0 = __ldg(q.qlen0);
  return n0 > 0 ? (unsigned long long)n0 : 1ull;
}

// Everything a segment-evaluation kernel needs. Two modes:
//  - list mode  (queue == nullptr): item i is segment (seg_ray[i], t0[i], t1[i]),
//    raw outputs go to out[i * n_out + j];
//  - wave mode: item i is ray queue[i] evaluating its segment slot `wave`;
//    the closest predicted hit is kept in `hits` and the ray is queued for
//    the next wave while its next segment starts before its best t.
struct EvalArgs {
  GridParams gp;
  const void* table;
  const float* mlp;
  int32_t n_hidden, width, n_out;
  RayPtrs rays;
  // list mode
  const int32_t* seg_ray;
  const float* list_t0;
  const float* list_t1;
  int64_t n_items;
  float* out;
  // wave mode
  const int32_t* queue;
  const int32_t* qlen;
  int32_t wave;
  int64_t n_rays;
  const int32_t* seg_count;
  const int32_t* seg_leaf;
  const float* seg_t0;
  const float* seg_t1;
  nbvh_hits hits;
  int32_t* next_queue;
  int32_t* next_qlen;
  int32_t max_segs;   // segment slots per ray in the seg_* arrays
  int32_t* inst_out;  // optional (hybrid hierarchy): instance id written with each improved hit
  int32_t inst_id;
  PQueue pq;          // tensor-core query: persistent queue (when pq.ring is set)
  const void* w1_image;  // tensor-core kernel: streamed first-layer weights (nullptr: resident)
  const void* w1_copy;   // resident plan: the same 16-bit image, bulk-copied whole by each CTA
                         // (nullptr: each CTA converts the FP32 weights)
  int32_t chunk_samples; // FP32 kernel: samples per first-layer chunk (0: all, weights resident)
  // training forward (tensor-core kernel, list of one segment per ray)
  TcTrain tr;
};

// Activation layout in shared memory: [k][TM] with a per-row XOR swizzle of
// the segment index that keeps float2 pairs together and spreads the rows a
// warp writes in the dense layers over distinct banks.
__device__ __forceinline__ int act_idx(int k, int s) { return k * kPlainTM + (s ^ (((k >> 2) & 15) << 1)); }

// A dense layer over a [K][TM] activation tile (act_idx layout) with the
// weights transposed to [K][W] in shared memory: thread t owns segments s0,
// s0 + 1 and outputs n0 .. n0 + W/16 - 1. The accumulators stay in registers
// across calls, so a layer can be fed in K chunks.
template <int W>
struct DenseAcc {
  static constexpr int NPT = W / 16;
  float a0[NPT], a1[NPT];
  __device__ __forceinline__ int s0() const { return (threadIdx.x >> 4) * 2; }
  __device__ __forceinline__ int n0() const { return (threadIdx.x & 15) * NPT; }
  __device__ __forceinline__ void init(const float* __restrict__ bias) {
#pragma unroll
    for (int j = 0; j < NPT; ++j) a0[j] = a1[j] = __ldg(bias + n0() + j);
  }
  __device__ __forceinline__ void accum(const float* __restrict__ in, int K, const float* __restrict__ wt) {
    const int sa = s0(), na = n0();
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const float2 f = *reinterpret_cast<const float2*>(in + act_idx(k, sa));
      float w[NPT];
      if constexpr (NPT % 4 == 0) {
#pragma unroll
        for (int j = 0; j < NPT; j += 4) {
          const float4 q = *reinterpret_cast<const float4*>(wt + k * W + na + j);
          w[j] = q.x; w[j + 1] = q.y; w[j + 2] = q.z; w[j + 3] = q.w;
        }
      } else if constexpr (NPT == 2) {
        const float2 q = *reinterpret_cast<const float2*>(wt + k * W + na);
        w[0] = q.x; w[1] = q.y;
      } else {
        w[0] = wt[k * W + na];
      }
#pragma unroll
      for (int j = 0; j < NPT; ++j) {
        a0[j] = fmaf(w[j], f.x, a0[j]);
        a1[j] = fmaf(w[j], f.y, a1[j]);
      }
    }
  }
  template <bool RELU>
  __device__ __forceinline__ void store(float* __restrict__ out) const {
    const int sa = s0(), na = n0();
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      float2 v = make_float2(a0[j], a1[j]);
      if (RELU) { v.x = fmaxf(v.x, 0.0f); v.y = fmaxf(v.y, 0.0f); }
      *reinterpret_cast<float2*>(out + act_idx(na + j, sa)) = v;
    }
  }
};

template <int W, bool RELU>
__device__ __forceinline__ void dense_plain(const float* __restrict__ in, int K, const float* __restrict__ wt,
                                            const float* __restrict__ bias, float* __restrict__ out) {
  DenseAcc<W> acc;
  acc.init(bias);
  acc.accum(in, K, wt);
  acc.template store<RELU>(out);
}

// Decoded per-segment result (S5): hit iff logit > 0; t = t0 + sigmoid(o_d) (t1 - t0);
// normal = o_n / |o_n| or (0,0,1).
struct SegResult {
  bool hit;
  float t, nx, ny, nz;
};

// Albedo head (outputs 5-7, sigmoid) of a hit into the record, when both the
// model and the record have one.
__device__ __forceinline__ void write_albedo(const EvalArgs& a, int ray, const float* raw);

__device__ __forceinline__ SegResult decode_segment(const float* raw, float t0, float t1) {
  SegResult r;
  r.hit = raw[0] > 0.0f;
  r.t = t0 + sigmoidf_(raw[1]) * (t1 - t0);
  const float l2 = raw[2] * raw[2] + raw[3] * raw[3] + raw[4] * raw[4];
  if (l2 > 0.0f) {
    const float inv = 1.0f / sqrtf(l2);
    r.nx = raw[2] * inv; r.ny = raw[3] * inv; r.nz = raw[4] * inv;
  } else {
    r.nx = 0.0f; r.ny = 0.0f; r.nz = 1.0f;
  }
  return r;
}

// Albedo of a new closest hit: sigmoid of outputs 5-7 with an albedo head,
// 0 without one (the record may have held another instance's albedo).
__device__ __forceinline__ void write_albedo(const EvalArgs& a, int ray, const float* raw) {
  if (a.hits.ar) {
    const bool head = a.n_out >= 8;
    a.hits.ar[ray] = head ? sigmoidf_(raw[5]) : 0.0f;
    a.hits.ag[ray] = head ? sigmoidf_(raw[6]) : 0.0f;
    a.hits.ab[ray] = head ? sigmoidf_(raw[7]) : 0.0f;
  }
}

// Wave-mode epilogue for one segment of ray `ray` (one lane per item, the
// whole warp calls it): resolve into the hit record, queue the next segment.
__device__ __forceinline__ void wave_resolve(const EvalArgs& a, bool valid, int ray, const float* raw, float t0,
                                             float t1) {
  bool push = false;
  if (valid) {
    SegResult s = decode_segment(raw, t0, t1);
    if (s.hit && t0 > t1) s.hit = s.t > a.rays.tmin[ray] && s.t <= a.rays.tmax[ray];  // reversed chord
    float best = a.hits.t[ray];
    if (s.hit && s.t < best) {
      best = s.t;
      a.hits.t[ray] = s.t;
      a.hits.hit[ray] = 1;
      a.hits.nx[ray] = s.nx;
      a.hits.ny[ray] = s.ny;
      a.hits.nz[ray] = s.nz;
      a.hits.leaf[ray] = a.seg_leaf[size_t(a.wave) * size_t(a.n_rays) + size_t(ray)];
      if (a.inst_out) a.inst_out[ray] = a.inst_id;
      write_albedo(a, ray, raw);
    }
    const int nxt = a.wave + 1;
    if (nxt < a.seg_count[ray]) {
      const size_t q = size_t(nxt) * size_t(a.n_rays) + size_t(ray);
      push = fminf(a.seg_t0[q], a.seg_t1[q]) < best;  // the next segment's start
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, push);
  if (m) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(a.next_qlen, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (push) a.next_queue[base + __popc(m & ((1u << lane) - 1u))] = ray;
  }
}

// First-layer chunking of the FP32 kernel: CS samples (CS * L * F features)
// per chunk, CS = a.chunk_samples, or all N (0) with the first layer's weights
// staged once per CTA. Chunked, every tile gathers chunk c and multiplies it
// by the matching rows of the first layer's weights (reloaded per chunk), the
// accumulators staying in registers.
inline size_t plain_smem_bytes(int K, int W, int n_hidden, int n_out) {
  const int hid_w = (n_hidden - 1) * W * W + W * n_out;
  const int feat_floats = K * kPlainTM > hid_w ? K * kPlainTM : hid_w;
  return sizeof(float) * (size_t(feat_floats) + size_t(K) * W + 2 * size_t(W) * kPlainTM + 8 * kPlainTM) +
         3 * sizeof(int) * kPlainTM;
}

// Samples per chunk for an input width K = N * LF: 0 when the whole first
// layer fits shared memory, else the most samples whose chunk fits; -1 if not
// even one sample's chunk fits.
inline int plain_chunk_samples(int N, int LF, int W, int n_hidden, int n_out) {
  const size_t limit = 227 * 1024;
  if (plain_smem_bytes(N * LF, W, n_hidden, n_out) <= limit) return 0;
  for (int cs = N - 1; cs >= 1; --cs)
    if (plain_smem_bytes(cs * LF, W, n_hidden, n_out) <= limit) return cs;
  return -1;
}

template <typename T, int F, int W, bool WAVE>
__global__ void __launch_bounds__(kPlainThreads, 1) eval_plain_kernel(EvalArgs a) {
  extern __shared__ __align__(16) float smem[];
  const int K = a.gp.n_inputs;
  const int L = a.gp.n_levels;
  const int N = a.gp.n_samples;
  const int LF = L * F;
  const int n_out = a.n_out;
  const int CS = a.chunk_samples > 0 ? a.chunk_samples : N;  // samples per chunk
  const int KC = CS * LF;                                     // features per chunk
  const bool resident = CS >= N;
  const int hid_w = (a.n_hidden - 1) * W * W + W * n_out;
  const int feat_floats = max(KC * kPlainTM, hid_w);
  float* sfeat = smem;                      // [KC][TM] features, later hidden weights
  float* sW1 = sfeat + feat_floats;         // [KC][W] first-layer weights (chunk), transposed
  float* shA = sW1 + KC * W;                // [W][TM]
  float* shB = shA + W * kPlainTM;          // [W][TM]
  float* sout = shB + W * kPlainTM;         // [8][TM]
  int* sray = reinterpret_cast<int*>(sout + 8 * kPlainTM);
  float* st0 = reinterpret_cast<float*>(sray + kPlainTM);
  float* st1 = st0 + kPlainTM;

  const int64_t n_items = WAVE ? int64_t(*a.qlen) : a.n_items;
  const int64_t n_tiles = (n_items + kPlainTM - 1) / kPlainTM;
  if (int64_t(blockIdx.x) >= n_tiles) return;

  const float* W1 = a.mlp;            // [W][K]
  const float* b1 = W1 + W * K;
  // rows [c0, c0 + KC) of the transposed first layer (zero beyond K)
  auto load_w1 = [&](int c0) {
    for (int i = threadIdx.x; i < KC * W; i += blockDim.x) {
      const int n = i / KC, k = i - n * KC;
      sW1[k * W + n] = c0 + k < K ? __ldg(W1 + size_t(n) * K + c0 + k) : 0.0f;
    }
  };
  if (resident) load_w1(0);
  const T* table = static_cast<const T*>(a.table);

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    if (threadIdx.x < kPlainTM) {
      const int64_t i = tile * kPlainTM + threadIdx.x;
      int ray = -1;
      float t0 = 0.0f, t1 = 0.0f;
      if (i < n_items) {
        if (WAVE) {
          ray = a.queue[i];
          const size_t q = size_t(a.wave) * size_t(a.n_rays) + size_t(ray);
          t0 = a.seg_t0[q];
          t1 = a.seg_t1[q];
        } else {
          ray = a.seg_ray[i];
          t0 = a.list_t0[i];
          t1 = a.list_t1[i];
        }
      }
      sray[threadIdx.x] = ray;
      st0[threadIdx.x] = t0;
      st1[threadIdx.x] = t1;
    }
    __syncthreads();

    DenseAcc<W> acc;
    acc.init(b1);
    for (int ks = 0; ks < N; ks += CS) {
      const int cs = min(CS, N - ks);
      if (!resident) load_w1(ks * LF);
      // Encode: pair p = (segment s, sample k); lanes = consecutive segments.
      for (int p = threadIdx.x; p < kPlainTM * cs; p += blockDim.x) {
        const int s = p % kPlainTM;
        const int k = ks + p / kPlainTM;
        const int ray = sray[s];
        const int kb = (k - ks) * LF;
        if (ray < 0) {
          for (int j = 0; j < LF; ++j) sfeat[act_idx(kb + j, s)] = 0.0f;
          continue;
        }
        FF x, y, z;
        sample_point_ff(a.gp, a.rays.ox[ray], a.rays.oy[ray], a.rays.oz[ray], a.rays.dx[ray], a.rays.dy[ray],
                        a.rays.dz[ray], st0[s], st1[s], k, x, y, z);
        for (int l = 0; l < L; ++l) {
          float v[F];
          encode_level<T, F>(a.gp, table, l, x, y, z, v);
#pragma unroll
          for (int f = 0; f < F; ++f) sfeat[act_idx(kb + l * F + f, s)] = v[f];
        }
      }
      __syncthreads();
      acc.accum(sfeat, cs * LF, sW1);
      __syncthreads();
    }
    acc.template store<true>(shA);

    // Hidden and output weights, transposed into the (now free) feature area.
    {
      const float* src = b1 + W;
      float* dst = sfeat;
      for (int h = 1; h < a.n_hidden; ++h) {
        for (int i = threadIdx.x; i < W * W; i += blockDim.x) {
          const int n = i / W, k = i - n * W;
          dst[k * W + n] = __ldg(src + i);
        }
        src += W * W + W;
        dst += W * W;
      }
      for (int i = threadIdx.x; i < n_out * W; i += blockDim.x) {
        const int n = i / W, k = i - n * W;
        dst[k * n_out + n] = __ldg(src + i);
      }
    }
    __syncthreads();

    const float* bh = b1 + W;  // walks over hidden layers
    float* hin = shA;
    float* hout = shB;
    const float* wt = sfeat;
    for (int h = 1; h < a.n_hidden; ++h) {
      const float* bias = bh + W * W;
      dense_plain<W, true>(hin, W, wt, bias, hout);
      __syncthreads();
      float* tmp = hin; hin = hout; hout = tmp;
      bh += W * W + W;
      wt += W * W;
    }
    {
      const float* bo = bh + n_out * W;
      for (int i = threadIdx.x; i < n_out * kPlainTM; i += blockDim.x) {
        const int j = i / kPlainTM, s = i - j * kPlainTM;
        float acc_o = __ldg(bo + j);
        for (int k = 0; k < W; ++k) acc_o = fmaf(wt[k * n_out + j], hin[act_idx(k, s)], acc_o);
        sout[j * kPlainTM + s] = acc_o;
      }
    }
    __syncthreads();

    if (threadIdx.x < kPlainTM) {
      const int s = threadIdx.x;
      const int ray = sray[s];
      float raw[8];
      for (int j = 0; j < n_out; ++j) raw[j] = sout[j * kPlainTM + s];
      if (WAVE) {
        wave_resolve(a, ray >= 0, ray, raw, st0[s], st1[s]);
      } else if (ray >= 0) {
        const int64_t i = tile * kPlainTM + s;
        for (int j = 0; j < n_out; ++j) a.out[i * n_out + j] = raw[j];
      }
    }
    __syncthreads();
  }
}

// Encoder only (S2+S3), FP32 features feat[i * K + k*L*F + l*F + f].
template <typename T, int F>
__global__ void __launch_bounds__(128) encode_kernel(GridParams gp, const void* table_v, RayPtrs rays,
                                                     const int32_t* __restrict__ seg_ray,
                                                     const float* __restrict__ t0, const float* __restrict__ t1,
                                                     int64_t n_seg, float* __restrict__ feat) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int N = gp.n_samples, L = gp.n_levels;
  if (p >= n_seg * N) return;
  const int64_t i = p / N;
  const int k = int(p - i * N);
  const int ray = seg_ray[i];
  FF x, y, z;
  sample_point_ff(gp, rays.ox[ray], rays.oy[ray], rays.oz[ray], rays.dx[ray], rays.dy[ray], rays.dz[ray], t0[i],
                  t1[i], k, x, y, z);
  const T* table = static_cast<const T*>(table_v);
  float* o = feat + i * int64_t(gp.n_inputs) + int64_t(k) * L * F;
  for (int l = 0; l < L; ++l) {
    float v[F];
    encode_level<T, F>(gp, table, l, x, y, z, v);
#pragma unroll
    for (int f = 0; f < F; ++f) o[l * F + f] = v[f];
  }
}

// ---------------------------------------------------------------- launch
template <typename T, int F, int W, bool WAVE>
cudaError_t launch_plain_twf(const EvalArgs& a0, int64_t n_items_max, cudaStream_t s) {
  EvalArgs a = a0;
  const int LF = a.gp.n_levels * F;
  const int cs = plain_chunk_samples(a.gp.n_samples, LF, W, a.n_hidden, a.n_out);
  if (cs < 0) return cudaErrorInvalidConfiguration;
  a.chunk_samples = cs;
  auto kern = eval_plain_kernel<T, F, W, WAVE>;
  const size_t smem = plain_smem_bytes((cs > 0 ? cs : a.gp.n_samples) * LF, W, a.n_hidden, a.n_out);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPlainThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  int64_t tiles = (n_items_max + kPlainTM - 1) / kPlainTM;
  int64_t grid = int64_t(sm_count()) * occ;
  if (tiles < grid) grid = tiles;
  if (grid < 1) return cudaSuccess;
  kern<<<unsigned(grid), kPlainThreads, smem, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T, int F, bool WAVE>
cudaError_t launch_plain_tf(const EvalArgs& a, int64_t n, cudaStream_t s) {
  switch (a.width) {
    case 16: return launch_plain_twf<T, F, 16, WAVE>(a, n, s);
    case 32: return launch_plain_twf<T, F, 32, WAVE>(a, n, s);
    case 64: return launch_plain_twf<T, F, 64, WAVE>(a, n, s);
    case 128: return launch_plain_twf<T, F, 128, WAVE>(a, n, s);
  }
  return cudaErrorInvalidValue;
}

// The FP32 kernels of one table type and schedule (one translation unit each).
template <typename T, bool WAVE>
cudaError_t launch_plain_t(int F, const EvalArgs& a, int64_t n, cudaStream_t s) {
  switch (F) {
    case 1: return launch_plain_tf<T, 1, WAVE>(a, n, s);
    case 2: return launch_plain_tf<T, 2, WAVE>(a, n, s);
    case 4: return launch_plain_tf<T, 4, WAVE>(a, n, s);
    case 8: return launch_plain_tf<T, 8, WAVE>(a, n, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nbvh
