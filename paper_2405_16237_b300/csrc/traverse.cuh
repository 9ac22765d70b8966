// S1: N-BVH traversal, slab test, clip and per-ray ordered segment lists.
#pragma once
#include "nbvh_internal.cuh"

namespace nbvh {

struct TraverseOut {
  int32_t* seg_count;
  int32_t* seg_leaf;
  float* seg_t0;
  float* seg_t1;
  int32_t max_segs;
  // Optional (query): initialise the hit record and queue rays with >= 1 segment.
  int32_t* queue0;
  int32_t* qlen0;
  nbvh_hits hits;
  // Merge mode (hybrid hierarchy): the hit record already holds the closest
  // hit found so far; it is kept, and leaves whose clipped segment starts at or
  // beyond it are skipped (a neural hit never lies before its segment's t0).
  int32_t merge;
  // Optional (persistent query): the queued rays as 64-bit items (slot 0).
  unsigned long long* ring0;
};

// One thread per ray. Depth-first with a short stack; the nearer child is
// descended first. Child boxes are stored in the parent, so one 64-byte node
// load tests two boxes. A child box contains all boxes below it and rounding
// of the slab arithmetic is monotone, so an empty clip prunes its subtree.
// Segments are inserted into the ray's list in (t0, leaf) order; the list is
// slot-major (slot s of ray r at s * n + r) so a warp's stores coalesce.
__global__ void __launch_bounds__(256) traverse_kernel(const nbvh_node* __restrict__ nodes,
                                                       RayPtrs rays, int64_t n, TraverseOut out) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool active = r < n;
  int count = 0;
  if (active) {
    const float ox = rays.ox[r], oy = rays.oy[r], oz = rays.oz[r];
    const float dx = rays.dx[r], dy = rays.dy[r], dz = rays.dz[r];
    const float tmin = rays.tmin[r], tmax = rays.tmax[r];
    const RayR ray = make_rayr(ox, oy, oz, dx, dy, dz, tmin, tmax);
    const int max_segs = out.max_segs;
    const bool merge = out.merge != 0;
    const float best = merge ? out.hits.t[r] : 0.0f;
    bool overflow = false;
    auto emit = [&](int leaf, float t0, float t1) {
      int pos;
      if (count < max_segs) {
        pos = count++;
      } else {
        overflow = true;
        const size_t q = size_t(max_segs - 1) * size_t(n) + size_t(r);
        const float lt = out.seg_t0[q];
        const int ll = out.seg_leaf[q];
        if (t0 > lt || (t0 == lt && leaf > ll)) return;
        pos = max_segs - 1;
      }
      while (pos > 0) {
        const size_t q = size_t(pos - 1) * size_t(n) + size_t(r);
        const float pt = out.seg_t0[q];
        const int pl = out.seg_leaf[q];
        if (pt < t0 || (pt == t0 && pl < leaf)) break;
        const size_t w = size_t(pos) * size_t(n) + size_t(r);
        out.seg_t0[w] = pt;
        out.seg_t1[w] = out.seg_t1[q];
        out.seg_leaf[w] = pl;
        --pos;
      }
      const size_t w = size_t(pos) * size_t(n) + size_t(r);
      out.seg_t0[w] = t0;
      out.seg_t1[w] = t1;
      out.seg_leaf[w] = leaf;
    };

    int stack[kTraverseStack];
    int sp = 0;
    int cur = 0;
    for (int guard = 0; guard < (1 << 26); ++guard) {
      const float4* np = reinterpret_cast<const float4*>(nodes + cur);
      const float4 a = __ldg(np);
      const float4 b = __ldg(np + 1);
      const float4 c = __ldg(np + 2);
      const int4 e = __ldg(reinterpret_cast<const int4*>(np + 3));
      float a0, a1, b0, b1;
      bool h0 = clip_box(ray, a.x, a.y, a.z, a.w, b.x, b.y, a0, a1);
      bool h1 = (e.y != kNodeNone) && clip_box(ray, b.z, b.w, c.x, c.y, c.z, c.w, b0, b1);
      if (merge) {
        h0 = h0 && a0 < best;
        h1 = h1 && b0 < best;
      }
      if (h0 && e.x < 0) emit(~e.x, a0, a1);
      if (h1 && e.y < 0) emit(~e.y, b0, b1);
      const bool g0 = h0 && e.x >= 0;
      const bool g1 = h1 && e.y >= 0;
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
    out.seg_count[r] = count;
    if (overflow) set_status(NBVH_ERR_SEGMENT_OVERFLOW);
    if (out.hits.hit && !merge) {
      out.hits.hit[r] = 0;
      out.hits.t[r] = __int_as_float(0x7f800000);
      out.hits.nx[r] = 0.0f;
      out.hits.ny[r] = 0.0f;
      out.hits.nz[r] = 0.0f;
      out.hits.leaf[r] = -1;
    }
  }
  if (out.queue0 || out.ring0) {
    const bool want = active && count > 0;
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (m) {
      const int lane = threadIdx.x & 31;
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(out.qlen0, __popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      const int pos = base + __popc(m & ((1u << lane) - 1u));
      if (want && out.ring0) out.ring0[pos] = (unsigned long long)r;
      else if (want) out.queue0[pos] = int32_t(r);
    }
  }
}

}  // namespace nbvh
