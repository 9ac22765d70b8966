// S9: the classical BLAS of the hybrid two-level hierarchy (Sec. 7: each BLAS
// is either a classical BVH or an N-BVH, and both query types return the same
// intersection record). Closest-hit traversal of a binary triangle BVH with
// Moller-Trumbore tests, one thread per ray, FP32.
#pragma once
#include "nbvh_internal.cuh"

namespace nbvh {

struct TriBlasArgs {
  const nbvh_node* nodes;
  const float* tris;          // [n_tris][9] vertices, leaf order
  const int32_t* leaf_range;  // [n_leaves][2] begin, end into tris
  const int32_t* tri_id;      // [n_tris] caller's index of each leaf-order triangle
  const float* albedo;        // optional [n_tris][3] by caller index
  RayPtrs rays;
  int64_t n;
  nbvh_hits hits;
  int32_t* inst_out;  // optional: instance id of the record
  int32_t inst_id;
  int32_t merge;      // 1: replace the record only with a strictly closer hit
};

// Moller & Trumbore (1997): edges inclusive (u >= 0, v >= 0, u + v <= 1),
// det == 0 a miss. Returns false or the hit's t.
__device__ __forceinline__ bool tri_mt(const float* __restrict__ T, float ox, float oy, float oz, float dx,
                                       float dy, float dz, float& t) {
  const float v0x = __ldg(T), v0y = __ldg(T + 1), v0z = __ldg(T + 2);
  const float e1x = __ldg(T + 3) - v0x, e1y = __ldg(T + 4) - v0y, e1z = __ldg(T + 5) - v0z;
  const float e2x = __ldg(T + 6) - v0x, e2y = __ldg(T + 7) - v0y, e2z = __ldg(T + 8) - v0z;
  const float px = dy * e2z - dz * e2y, py = dz * e2x - dx * e2z, pz = dx * e2y - dy * e2x;
  const float det = e1x * px + e1y * py + e1z * pz;
  if (det == 0.0f) return false;
  const float inv = 1.0f / det;
  const float sx = ox - v0x, sy = oy - v0y, sz = oz - v0z;
  const float u = (sx * px + sy * py + sz * pz) * inv;
  if (u < 0.0f || u > 1.0f) return false;
  const float qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
  const float v = (dx * qx + dy * qy + dz * qz) * inv;
  if (v < 0.0f || u + v > 1.0f) return false;
  t = (e2x * qx + e2y * qy + e2z * qz) * inv;
  return true;
}

// Conservative slab test of the classical BLAS (robust traversal after Ize,
// "Robust BVH Ray Traversal", JCGT 2013): slab values from the ray's
// reciprocal, the far end grown by 2 gamma_3 (gamma_n = n eps / (1 - n eps),
// eps = 2^-24) of its magnitude, so rounding never drops a box the ray meets;
// a zero direction component keeps the slab iff lo <= o <= hi. The interval's
// upper end tmax (the best hit so far) is grown the same way, so a box whose
// entry rounds up onto it is still visited. The boxes only prune:
// Moller-Trumbore decides every hit.
constexpr float kRobustGrow = 2.0f * (3.0f * 5.9604645e-8f) / (1.0f - 3.0f * 5.9604645e-8f);

__device__ __forceinline__ bool clip_box_robust(const RayR& r, float tmax, float lx, float ly, float lz, float hx,
                                                float hy, float hz, float& t0) {
  constexpr float kGrow = kRobustGrow;
  float en = r.tmin, ex = tmax + fabsf(tmax) * kGrow;
  const float lo[3] = {lx, ly, lz}, hi[3] = {hx, hy, hz};
  bool empty = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (r.d[i] == 0.0f) {
      empty |= (r.o[i] < lo[i]) | (r.o[i] > hi[i]);
    } else {
      const float a = (lo[i] - r.o[i]) * r.inv[i];
      const float b = (hi[i] - r.o[i]) * r.inv[i];
      const float f = fmaxf(a, b);
      en = fmaxf(en, fminf(a, b));
      ex = fminf(ex, f + fabsf(f) * kGrow);
    }
  }
  t0 = en;
  return !empty && en <= ex;
}

// Closest hit with t in [tmin, tmax]; equal t goes to the lower caller index.
// The traversal visits the nearer child first and skips boxes whose
// conservative clip to [tmin, best] is empty (inclusive, so equal-t candidates
// survive).
static __global__ void __launch_bounds__(128) tri_trace_kernel(TriBlasArgs a) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= a.n) return;
  const float ox = a.rays.ox[r], oy = a.rays.oy[r], oz = a.rays.oz[r];
  const float dx = a.rays.dx[r], dy = a.rays.dy[r], dz = a.rays.dz[r];
  const float tmin = a.rays.tmin[r], tmax = a.rays.tmax[r];
  const float prev = a.merge ? a.hits.t[r] : __int_as_float(0x7f800000);
  float best = fminf(tmax, prev);
  int bid = 0x7fffffff;  // caller index of the best triangle
  int bj = -1;           // its leaf-order position
  if (!(tmin <= best)) {
    bj = -1;  // an empty interval (a ray a bounce pass retired): no reciprocals needed
  } else {
    RayR ray = make_rayr(ox, oy, oz, dx, dy, dz, tmin, best);
    int stack[kTraverseStack];
    int sp = 0;
    int cur = 0;
    for (int guard = 0; guard < (1 << 26); ++guard) {
      const float4* np = reinterpret_cast<const float4*>(a.nodes + cur);
      const float4 p = __ldg(np);
      const float4 q = __ldg(np + 1);
      const float4 c = __ldg(np + 2);
      const int4 e = __ldg(reinterpret_cast<const int4*>(np + 3));
      float a0, b0;
      const bool h0 = clip_box_robust(ray, best, p.x, p.y, p.z, p.w, q.x, q.y, a0);
      const bool h1 = (e.y != kNodeNone) && clip_box_robust(ray, best, q.z, q.w, c.x, c.y, c.z, c.w, b0);
      // leaves are tested at once (they may shrink best before the subtree is chosen)
      for (int s = 0; s < 2; ++s) {
        const bool hs = s == 0 ? h0 : h1;
        const int ch = s == 0 ? e.x : e.y;
        if (!hs || ch >= 0) continue;
        const int lf = ~ch;
        const int b = __ldg(a.leaf_range + 2 * lf), en = __ldg(a.leaf_range + 2 * lf + 1);
        for (int j = b; j < en; ++j) {
          float t;
          if (!tri_mt(a.tris + size_t(j) * 9, ox, oy, oz, dx, dy, dz, t)) continue;
          if (t < tmin || t > best) continue;
          const int id = __ldg(a.tri_id + j);
          if (t < best || id < bid) {
            best = t;
            bid = id;
            bj = j;
          }
        }
      }
      const float reach = best + fabsf(best) * kRobustGrow;
      const bool g0 = h0 && e.x >= 0 && a0 <= reach;
      const bool g1 = h1 && e.y >= 0 && b0 <= reach;
      if (g0 && g1) {
        const bool first0 = a0 <= b0;
        if (sp < kTraverseStack) {
          stack[sp++] = first0 ? e.y : e.x;
        } else {
          set_status(NBVH_ERR_UNSUPPORTED);
        }
        cur = first0 ? e.x : e.y;
      } else if (g0) {
        cur = e.x;
      } else if (g1) {
        cur = e.y;
      } else {
        if (sp == 0) break;
        cur = stack[--sp];
      }
    }
  }
  const bool found = bj >= 0 && (!a.merge || best < prev);
  if (found) {
    const float* T = a.tris + size_t(bj) * 9;
    const float e1x = T[3] - T[0], e1y = T[4] - T[1], e1z = T[5] - T[2];
    const float e2x = T[6] - T[0], e2y = T[7] - T[1], e2z = T[8] - T[2];
    float gx = e1y * e2z - e1z * e2y, gy = e1z * e2x - e1x * e2z, gz = e1x * e2y - e1y * e2x;
    const float ln = sqrtf(gx * gx + gy * gy + gz * gz);
    if (ln > 0.0f) { gx /= ln; gy /= ln; gz /= ln; }
    if (gx * dx + gy * dy + gz * dz > 0.0f) { gx = -gx; gy = -gy; gz = -gz; }
    a.hits.hit[r] = 1;
    a.hits.t[r] = best;
    a.hits.nx[r] = gx;
    a.hits.ny[r] = gy;
    a.hits.nz[r] = gz;
    a.hits.leaf[r] = bid;
    if (a.inst_out) a.inst_out[r] = a.inst_id;
    if (a.hits.ar) {
      const float* c = a.albedo ? a.albedo + 3 * size_t(__ldg(a.tri_id + bj)) : nullptr;
      a.hits.ar[r] = c ? __ldg(c) : 0.0f;
      a.hits.ag[r] = c ? __ldg(c + 1) : 0.0f;
      a.hits.ab[r] = c ? __ldg(c + 2) : 0.0f;
    }
  } else if (!a.merge) {
    a.hits.hit[r] = 0;
    a.hits.t[r] = __int_as_float(0x7f800000);
    a.hits.nx[r] = 0.0f;
    a.hits.ny[r] = 0.0f;
    a.hits.nz[r] = 0.0f;
    a.hits.leaf[r] = -1;
    if (a.inst_out) a.inst_out[r] = -1;
    if (a.hits.ar) {
      a.hits.ar[r] = 0.0f;
      a.hits.ag[r] = 0.0f;
      a.hits.ab[r] = 0.0f;
    }
  }
}

// Empty hit records (hit 0, t +inf, leaf -1, instance -1) before the merges.
static __global__ void __launch_bounds__(256) hits_clear_kernel(nbvh_hits h, int32_t* inst_out, int64_t n) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n) return;
  h.hit[r] = 0;
  h.t[r] = __int_as_float(0x7f800000);
  h.nx[r] = 0.0f;
  h.ny[r] = 0.0f;
  h.nz[r] = 0.0f;
  h.leaf[r] = -1;
  if (inst_out) inst_out[r] = -1;
  if (h.ar) {
    h.ar[r] = 0.0f;
    h.ag[r] = 0.0f;
    h.ab[r] = 0.0f;
  }
}

}  // namespace nbvh
