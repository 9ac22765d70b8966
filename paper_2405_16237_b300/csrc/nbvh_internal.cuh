// Internal device helpers of the neural ray query library (sm_103a), included
// by every CUDA translation unit of the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/nbvh.h"

namespace nbvh {

constexpr int kMaxLevels = NBVH_MAX_LEVELS;
constexpr uint32_t kHashP1 = 2654435761u;  // spatial-hash primes of the
constexpr uint32_t kHashP2 = 805459861u;   // multi-resolution hash encoding
constexpr int kNodeNone = 0x7fffffff;      // "no child" (single-leaf trees)
constexpr int kTraverseStack = 64;

// Host-side count of kernel launches made by this library (nbvh_lib.cu).
void count_launches(int64_t n);
// Multiprocessors of the current device (nbvh_lib.cu).
int sm_count();

// Device status word, one per translation unit of the library (first error
// wins). Each unit registers a reader at load time; nbvh_get_device_status
// reads and clears them all.
using StatusReader = cudaError_t (*)(int* value);
void register_status_reader(StatusReader fn);

namespace {
__device__ int g_status = 0;

cudaError_t read_clear_status(int* value) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_status, sizeof(int));
  if (e != cudaSuccess) return e;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
}

struct StatusRegistration {
  StatusRegistration() { register_status_reader(&read_clear_status); }
};
StatusRegistration g_status_registration;
}  // namespace

__device__ __forceinline__ void set_status(int code) { atomicCAS(&g_status, 0, code); }

// ---------------------------------------------------------------------------
// Grid description passed by value to kernels.
// ---------------------------------------------------------------------------
struct GridParams {
  int32_t n_levels;
  int32_t n_features;
  int32_t n_samples;
  int32_t n_inputs;         // N * L * F
  float centre[3];
  float inv_extent;
  float extent;
  uint32_t hash_mask;       // T - 1
  int32_t res[kMaxLevels];
  int32_t dense[kMaxLevels];
  int64_t offset[kMaxLevels];  // entry offset of each level
};

struct RayPtrs {
  const float *ox, *oy, *oz, *dx, *dy, *dz, *tmin, *tmax;
};

// ---------------------------------------------------------------------------
// Float-float ("double-float") arithmetic from error-free transformations
// (Knuth's TwoSum, Dekker's product via FMA). The intrinsics keep the compiler
// from contracting or reassociating the exact steps.
// ---------------------------------------------------------------------------
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return FF{s, e};
}

__device__ __forceinline__ FF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return FF{p, fmaf(a, b, -p)};
}

// ---------------------------------------------------------------------------
// Table entry loads: F features of one entry, converted to float.
// ---------------------------------------------------------------------------
template <typename T, int F>
struct EntryLoad;

template <int F>
struct EntryLoad<float, F> {
  static __device__ __forceinline__ void load(const float* __restrict__ tab, uint64_t e, float* v) {
    const float* p = tab + e * F;
    if constexpr (F == 1) {
      v[0] = __ldg(p);
    } else if constexpr (F == 2) {
      float2 a = __ldg(reinterpret_cast<const float2*>(p));
      v[0] = a.x; v[1] = a.y;
    } else {
#pragma unroll
      for (int i = 0; i < F / 4; ++i) {
        float4 a = __ldg(reinterpret_cast<const float4*>(p) + i);
        v[4 * i] = a.x; v[4 * i + 1] = a.y; v[4 * i + 2] = a.z; v[4 * i + 3] = a.w;
      }
    }
  }
};

template <int F>
struct EntryLoad<__half, F> {
  static __device__ __forceinline__ void load(const __half* __restrict__ tab, uint64_t e, float* v) {
    const __half* p = tab + e * F;
    if constexpr (F == 1) {
      v[0] = __half2float(__ldg(p));
    } else if constexpr (F == 2) {
      float2 a = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
      v[0] = a.x; v[1] = a.y;
    } else if constexpr (F == 4) {
      uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
      float2 a = __half22float2(*reinterpret_cast<__half2*>(&raw.x));
      float2 b = __half22float2(*reinterpret_cast<__half2*>(&raw.y));
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
      uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
      uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float2 a = __half22float2(*reinterpret_cast<__half2*>(&w[i]));
        v[2 * i] = a.x; v[2 * i + 1] = a.y;
      }
    }
  }
};

template <int F>
struct EntryLoad<__nv_bfloat16, F> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* __restrict__ tab, uint64_t e,
                                              float* v) {
    const __nv_bfloat16* p = tab + e * F;
    if constexpr (F == 1) {
      v[0] = __bfloat162float(__ldg(p));
    } else if constexpr (F == 2) {
      float2 a = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
      v[0] = a.x; v[1] = a.y;
    } else if constexpr (F == 4) {
      uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
      float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&raw.x));
      float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&raw.y));
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
      uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
      uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w[i]));
        v[2 * i] = a.x; v[2 * i + 1] = a.y;
      }
    }
  }
};

// ---------------------------------------------------------------------------
// S2: stratified sample k of segment [t0, t1] in grid coordinates.
// t_k = t0 + (k + 1/2)/N (t1 - t0); xhat = (o + t_k d - c) / E + 1/2 in [0,1].
// ---------------------------------------------------------------------------
// Plain FP32 form (tensor-core path: its FP16/BF16 features round far above
// the position error).
__device__ __forceinline__ float sample_u(int k, int n_samples) {
  return (static_cast<float>(k) + 0.5f) / static_cast<float>(n_samples);
}

// Sample at fraction u = sample_u(k, N) of the segment.
__device__ __forceinline__ void sample_point_u(const GridParams& gp, float ox, float oy, float oz, float dx,
                                               float dy, float dz, float t0, float t1, float u, float& x,
                                               float& y, float& z) {
  // explicit roundings: every inlined copy computes the same bits, so a row's
  // features do not depend on where the kernel evaluates it
  const float t = __fmaf_rn(u, __fsub_rn(t1, t0), t0);
  x = __saturatef(__fmaf_rn(__fsub_rn(__fmaf_rn(t, dx, ox), gp.centre[0]), gp.inv_extent, 0.5f));
  y = __saturatef(__fmaf_rn(__fsub_rn(__fmaf_rn(t, dy, oy), gp.centre[1]), gp.inv_extent, 0.5f));
  z = __saturatef(__fmaf_rn(__fsub_rn(__fmaf_rn(t, dz, oz), gp.centre[2]), gp.inv_extent, 0.5f));
}

__device__ __forceinline__ void sample_point(const GridParams& gp, float ox, float oy, float oz,
                                             float dx, float dy, float dz, float t0, float t1, int k,
                                             float& x, float& y, float& z) {
  sample_point_u(gp, ox, oy, oz, dx, dy, dz, t0, t1, sample_u(k, gp.n_samples), x, y, z);
}

// Float-float form (FP32 path): the finest level multiplies a position error by
// its resolution (thousands), so the position is carried to ~2^-44 relative
// with FP32 operations only. Returns grid coordinates as hi + lo pairs.
__device__ __forceinline__ FF grid_coord_ff(FF t, float o, float d, float c, float E) {
  FF q = two_prod(t.hi, d);
  q.lo = fmaf(t.lo, d, q.lo);
  FF s = two_sum(o, q.hi);
  s.lo = __fadd_rn(s.lo, q.lo);
  FF v = two_sum(s.hi, -c);
  v.lo = __fadd_rn(v.lo, s.lo);
  v = fast_two_sum(v.hi, v.lo);
  const float y_hi = __fdiv_rn(v.hi, E);
  const float r = __fadd_rn(fmaf(-y_hi, E, v.hi), v.lo);  // v - y_hi * E
  const float y_lo = __fdiv_rn(r, E);
  FF w = two_sum(y_hi, 0.5f);
  w.lo = __fadd_rn(w.lo, y_lo);
  w = fast_two_sum(w.hi, w.lo);
  if (w.hi < 0.0f || (w.hi == 0.0f && w.lo < 0.0f)) w = FF{0.0f, 0.0f};
  if (w.hi > 1.0f || (w.hi == 1.0f && w.lo > 0.0f)) w = FF{1.0f, 0.0f};
  return w;
}

__device__ __forceinline__ void sample_point_ff(const GridParams& gp, float ox, float oy, float oz, float dx,
                                                float dy, float dz, float t0, float t1, int k, FF& x, FF& y,
                                                FF& z) {
  const float num = static_cast<float>(k) + 0.5f;
  const float Nf = static_cast<float>(gp.n_samples);
  const float u_hi = __fdiv_rn(num, Nf);
  const float u_lo = __fdiv_rn(fmaf(-u_hi, Nf, num), Nf);
  const FF dt = two_sum(t1, -t0);
  FF p = two_prod(u_hi, dt.hi);
  p.lo = __fadd_rn(p.lo, fmaf(u_hi, dt.lo, __fmul_rn(u_lo, dt.hi)));
  FF t = two_sum(t0, p.hi);
  t.lo = __fadd_rn(t.lo, p.lo);
  t = fast_two_sum(t.hi, t.lo);
  const float E = gp.extent;
  x = grid_coord_ff(t, ox, dx, gp.centre[0], E);
  y = grid_coord_ff(t, oy, dy, gp.centre[1], E);
  z = grid_coord_ff(t, oz, dz, gp.centre[2], E);
}

// ---------------------------------------------------------------------------
// S3: one level of the multi-resolution hash encoding at grid point (x,y,z):
// the 8 vertex indices of the enclosing cell and their trilinear weights.
// Corner c selects +1 along x (bit 0), y (bit 1), z (bit 2).
// ---------------------------------------------------------------------------
struct Corners {
  uint32_t idx[8];
  float w[8];
};

// Cell index and fraction along one axis: cell = min(floor(x N), N - 1),
// frac = x N - cell (x in [0, 1]).
__device__ __forceinline__ void axis_cell(float x, int N, int& c, float& f) {
  const float p = __fmul_rn(x, static_cast<float>(N));  // no contraction: the same bits at every call site
  c = min(static_cast<int>(p), N - 1);  // p >= 0: truncation = floor
  f = __fsub_rn(p, static_cast<float>(c));
}

__device__ __forceinline__ void axis_cell(FF x, int N, int& c, float& f) {
  const float Nf = static_cast<float>(N);
  FF p = two_prod(x.hi, Nf);
  p.lo = fmaf(x.lo, Nf, p.lo);
  p = fast_two_sum(p.hi, p.lo);
  float fl = floorf(p.hi);
  if (p.hi == fl && p.lo < 0.0f) fl -= 1.0f;
  if (fl > Nf - 1.0f) fl = Nf - 1.0f;
  if (fl < 0.0f) fl = 0.0f;
  c = static_cast<int>(fl);
  f = __fadd_rn(__fsub_rn(p.hi, fl), p.lo);  // p.hi - fl is exact
}

// Table entry of grid vertex (vx, vy, vz) of level l, vertex coordinates in
// [0, N]: the mapping level_corners applies to a cell's eight corners.
__device__ __forceinline__ uint32_t vertex_index(const GridParams& gp, int l, uint32_t vx, uint32_t vy,
                                                 uint32_t vz) {
  if (gp.dense[l]) {
    const uint32_t n1 = static_cast<uint32_t>(gp.res[l]) + 1u;
    return vx + vy * n1 + vz * n1 * n1;
  }
  return (vx ^ (vy * kHashP1) ^ (vz * kHashP2)) & gp.hash_mask;
}

template <typename P>
__device__ __forceinline__ void level_corners(const GridParams& gp, int l, P x, P y, P z, Corners& c) {
  const int N = gp.res[l];
  int cx, cy, cz;
  float fx, fy, fz;
  axis_cell(x, N, cx, fx);
  axis_cell(y, N, cy, fy);
  axis_cell(z, N, cz, fz);
  const float wx[2] = {1.0f - fx, fx};
  const float wy[2] = {1.0f - fy, fy};
  const float wz[2] = {1.0f - fz, fz};
  if (gp.dense[l]) {
    const uint32_t n1 = static_cast<uint32_t>(N) + 1u;
    const uint32_t base = static_cast<uint32_t>(cx) + static_cast<uint32_t>(cy) * n1 +
                          static_cast<uint32_t>(cz) * n1 * n1;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      c.idx[k] = base + (k & 1) + ((k >> 1) & 1) * n1 + ((k >> 2) & 1) * n1 * n1;
    }
  } else {
    const uint32_t hx = static_cast<uint32_t>(cx);
    const uint32_t hy = static_cast<uint32_t>(cy) * kHashP1;
    const uint32_t hz = static_cast<uint32_t>(cz) * kHashP2;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t a = hx + (k & 1);
      const uint32_t b = (k & 2) ? hy + kHashP1 : hy;
      const uint32_t d = (k & 4) ? hz + kHashP2 : hz;
      c.idx[k] = (a ^ b ^ d) & gp.hash_mask;
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) c.w[k] = wx[k & 1] * wy[(k >> 1) & 1] * wz[(k >> 2) & 1];
}

// Corner indices (table-relative) and cell fractions of level l at (x,y,z).
template <typename P>
__device__ __forceinline__ void level_index(const GridParams& gp, int l, P x, P y, P z, uint32_t* idx,
                                            float* fr) {
  const int N = gp.res[l];
  int cx, cy, cz;
  axis_cell(x, N, cx, fr[0]);
  axis_cell(y, N, cy, fr[1]);
  axis_cell(z, N, cz, fr[2]);
  if (gp.dense[l]) {
    const uint32_t n1 = static_cast<uint32_t>(N) + 1u;
    const uint32_t base = static_cast<uint32_t>(cx) + static_cast<uint32_t>(cy) * n1 +
                          static_cast<uint32_t>(cz) * n1 * n1;
#pragma unroll
    for (int k = 0; k < 8; ++k) idx[k] = base + (k & 1) + ((k >> 1) & 1) * n1 + ((k >> 2) & 1) * n1 * n1;
  } else {
    const uint32_t hx = static_cast<uint32_t>(cx);
    const uint32_t hy = static_cast<uint32_t>(cy) * kHashP1;
    const uint32_t hz = static_cast<uint32_t>(cz) * kHashP2;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t a = hx + (k & 1);
      const uint32_t b = (k & 2) ? hy + kHashP1 : hy;
      const uint32_t d = (k & 4) ? hz + kHashP2 : hz;
      idx[k] = (a ^ b ^ d) & gp.hash_mask;
    }
  }
}

// Interpolated F features of level l at (x,y,z) (float or float-float coords).
template <typename T, int F, typename P>
__device__ __forceinline__ void encode_level(const GridParams& gp, const T* __restrict__ table, int l,
                                             P x, P y, P z, float* out) {
  Corners c;
  level_corners(gp, l, x, y, z, c);
  const T* tab = table + gp.offset[l] * F;
  float v[8][F];
#pragma unroll
  for (int k = 0; k < 8; ++k) EntryLoad<T, F>::load(tab, c.idx[k], v[k]);
#pragma unroll
  for (int f = 0; f < F; ++f) out[f] = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int f = 0; f < F; ++f) out[f] = fmaf(c.w[k], v[k][f], out[f]);
  }
}

// NL consecutive levels from l0 with every corner load issued before any is
// consumed (memory-level parallelism for the latency-bound gather). Entries of
// 4 bytes (two FP16/BF16 features) stay as raw words until the interpolation.
template <typename T, int F, int NL, typename P>
__device__ __forceinline__ void encode_levels(const GridParams& gp, const T* __restrict__ table, int l0, P x,
                                              P y, P z, float* out) {
  if constexpr (F * sizeof(T) == 4 && sizeof(T) == 2) {
    uint32_t raw[NL][8];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      uint32_t idx[8];
      float fr[3];
      level_index(gp, l0 + q, x, y, z, idx, fr);
      const uint32_t* tab = reinterpret_cast<const uint32_t*>(table + gp.offset[l0 + q] * F);
#pragma unroll
      for (int k = 0; k < 8; ++k) raw[q][k] = __ldg(tab + idx[k]);
    }
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      // cell fractions recomputed here rather than held while the loads are in flight
      const int N = gp.res[l0 + q];
      int c;
      float fr[3];
      axis_cell(x, N, c, fr[0]);
      axis_cell(y, N, c, fr[1]);
      axis_cell(z, N, c, fr[2]);
      const float wx[2] = {1.0f - fr[0], fr[0]};
      const float wy[2] = {1.0f - fr[1], fr[1]};
      const float wz[2] = {1.0f - fr[2], fr[2]};
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float w = wx[k & 1] * wy[(k >> 1) & 1] * wz[(k >> 2) & 1];
        float2 v;
        if constexpr (sizeof(T) == 2 && std::is_same<T, __half>::value) {
          v = __half22float2(*reinterpret_cast<const __half2*>(&raw[q][k]));
        } else {
          v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw[q][k]));
        }
        a0 = fmaf(w, v.x, a0);
        a1 = fmaf(w, v.y, a1);
      }
      out[q * 2] = a0;
      out[q * 2 + 1] = a1;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NL; ++q) encode_level<T, F>(gp, table, l0 + q, x, y, z, out + q * F);
  }
}


// ---------------------------------------------------------------------------
// (b - o) / d rounded once to float: b - o is formed exactly as a float pair,
// the quotient's remainder comes from an FMA, and the correction is added last.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float slab_t(float b, float o, float d) {
  const FF a = two_sum(b, -o);
  const float q = __fdiv_rn(a.hi, d);
  if (!isfinite(q)) return q;
  const float r = fmaf(-q, d, a.hi);
  return __fadd_rn(q, __fdiv_rn(__fadd_rn(r, a.lo), d));
}

// The same value from the ray's reciprocal inv = RN(1/d): q = (b - o) inv, then
// one correction with the FMA remainder (b - o) - q d, which brings q to the
// rounded quotient (the traversal computes inv once per ray instead of two
// divisions per slab).
__device__ __forceinline__ float slab_t_rcp(float b, float o, float d, float inv) {
  if (!isfinite(inv)) return slab_t(b, o, d);  // |d| below ~2^-126: divide
  const FF a = two_sum(b, -o);
  const float q = __fmul_rn(a.hi, inv);
  if (!isfinite(q)) return q;
  const float r = __fadd_rn(fmaf(-q, d, a.hi), a.lo);
  return fmaf(r, inv, q);
}

// ---------------------------------------------------------------------------
// S1: slab test of a ray against a box, FP32 with correctly rounded slabs.
// A zero direction component keeps the slab unbounded when the origin lies in
// [lo, hi] and empties it otherwise. Segment = [max(entry, tmin),
// min(exit, tmax)], non-empty iff t0 <= t1.
// ---------------------------------------------------------------------------
// Ray with per-axis reciprocals for repeated box tests.
struct RayR {
  float o[3], d[3], inv[3], tmin, tmax;
};

__device__ __forceinline__ RayR make_rayr(float ox, float oy, float oz, float dx, float dy, float dz, float tmin,
                                          float tmax) {
  RayR r;
  r.o[0] = ox; r.o[1] = oy; r.o[2] = oz;
  r.d[0] = dx; r.d[1] = dy; r.d[2] = dz;
#pragma unroll
  for (int i = 0; i < 3; ++i) r.inv[i] = __fdiv_rn(1.0f, r.d[i]);
  r.tmin = tmin;
  r.tmax = tmax;
  return r;
}

__device__ __forceinline__ bool clip_box(const RayR& r, float lx, float ly, float lz, float hx, float hy,
                                         float hz, float& t0, float& t1) {
  float en = r.tmin, ex = r.tmax;
  bool empty = false;
  const float lo[3] = {lx, ly, lz}, hi[3] = {hx, hy, hz};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (r.d[i] == 0.0f) {
      empty |= (r.o[i] < lo[i]) | (r.o[i] > hi[i]);
    } else {
      const float a = slab_t_rcp(lo[i], r.o[i], r.d[i], r.inv[i]);
      const float b = slab_t_rcp(hi[i], r.o[i], r.d[i], r.inv[i]);
      en = fmaxf(en, fminf(a, b));
      ex = fminf(ex, fmaxf(a, b));
    }
  }
  t0 = en;
  t1 = ex;
  return !empty && en <= ex;
}

__device__ __forceinline__ bool clip_box(float ox, float oy, float oz, float dx, float dy, float dz,
                                         float tmin, float tmax, float lx, float ly, float lz,
                                         float hx, float hy, float hz, float& t0, float& t1) {
  return clip_box(make_rayr(ox, oy, oz, dx, dy, dz, tmin, tmax), lx, ly, lz, hx, hy, hz, t0, t1);
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

}  // namespace nbvh
