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
  // A leaf whose box the ray's origin lies in (entry < tmin) is listed over its
  // whole chord with swapped endpoints (t0 = exit, t1 = entry), for a query
  // of the chord in reverse order (NBVH_FLAG_REVERSE_INSIDE).
  int32_t reverse_inside;
  // Staged merge (hybrid hierarchy, instances evaluated concurrently): the
  // record `hits` is this instance's own staging record, started at the
  // closest hit of the instances merged before (init_t, found by instance
  // init_inst; -1: none). A hit equal to it still wins for an instance with a
  // lower index than init_inst, so such an instance starts just above it.
  const float* init_t;
  const int32_t* init_inst;
  int32_t inst_id;
};

// Order key of a listed segment: its start along the ray (the entry of a
// swapped segment).
__device__ __forceinline__ float seg_key(float t0, float t1) { return fminf(t0, t1); }

// Traversal of ray r (S1). Depth-first with a short stack; the nearer child
// is descended first. Child boxes are stored in the parent, so one 64-byte
// node load tests two boxes. A child box contains all boxes below it and
// rounding of the slab arithmetic is monotone, so an empty clip prunes its
// subtree. Segments are inserted into the ray's list in (t0, leaf) order; the
// list is slot-major (slot s of ray r at s * n + r) so a warp's stores
// coalesce. Returns the ray's segment count.
__device__ __forceinline__ int traverse_ray(const nbvh_node* __restrict__ nodes, const RayPtrs& rays, int64_t n,
                                            int64_t r, const TraverseOut& out) {
  int count = 0;
  const float ox = rays.ox[r], oy = rays.oy[r], oz = rays.oz[r];
  const float dx = rays.dx[r], dy = rays.dy[r], dz = rays.dz[r];
  const float tmin = rays.tmin[r], tmax = rays.tmax[r];
  const RayR ray = make_rayr(ox, oy, oz, dx, dy, dz, tmin, tmax);
  const int max_segs = out.max_segs;
  const bool merge = out.merge != 0;
  float best = merge ? out.hits.t[r] : 0.0f;
  if (out.init_t) {
    best = out.init_t[r];
    if (out.init_inst[r] > out.inst_id) best = nextafterf(best, __int_as_float(0x7f800000));
    out.hits.t[r] = best;
    out.hits.hit[r] = 0;
  }
  bool overflow = false;
  float lo_box[3] = {0.0f, 0.0f, 0.0f}, hi_box[3] = {0.0f, 0.0f, 0.0f};  // the box being emitted
  float tail_key = 0.0f;  // order key and leaf of the list's last entry (count > 0)
  int tail_leaf = 0;
  auto emit = [&](int leaf, float t0, float t1) {
    if (out.reverse_inside) {  // origin inside the box: the whole chord, reversed
      RayR whole = ray;
      whole.tmin = -__int_as_float(0x7f800000);
      whole.tmax = __int_as_float(0x7f800000);
      float en, ex;
      if (clip_box(whole, lo_box[0], lo_box[1], lo_box[2], hi_box[0], hi_box[1], hi_box[2], en, ex) &&
          en < tmin && isfinite(en) && isfinite(ex)) {
        t0 = ex;
        t1 = en;
      }
    }
    const float key = seg_key(t0, t1);
    // usual case (near-to-far traversal): the segment goes after the list's
    // last entry, known from registers, so nothing is read back
    if (count == 0 || tail_key < key || (tail_key == key && tail_leaf < leaf)) {
      if (count < max_segs) {
        const size_t w = size_t(count) * size_t(n) + size_t(r);
        out.seg_t0[w] = t0;
        out.seg_t1[w] = t1;
        out.seg_leaf[w] = leaf;
        ++count;
        tail_key = key;
        tail_leaf = leaf;
      } else {
        overflow = true;  // beyond the last kept entry of a full list
      }
      return;
    }
    int pos;
    if (count < max_segs) {
      pos = count++;
    } else {
      overflow = true;
      const size_t q = size_t(max_segs - 1) * size_t(n) + size_t(r);
      const float lt = seg_key(out.seg_t0[q], out.seg_t1[q]);
      const int ll = out.seg_leaf[q];
      if (key > lt || (key == lt && leaf > ll)) return;
      pos = max_segs - 1;
    }
    while (pos > 0) {
      const size_t q = size_t(pos - 1) * size_t(n) + size_t(r);
      const float pt = seg_key(out.seg_t0[q], out.seg_t1[q]);
      const int pl = out.seg_leaf[q];
      if (pt < key || (pt == key && pl < leaf)) break;
      const size_t w = size_t(pos) * size_t(n) + size_t(r);
      out.seg_t0[w] = out.seg_t0[q];
      out.seg_t1[w] = out.seg_t1[q];
      out.seg_leaf[w] = pl;
      --pos;
    }
    const size_t w = size_t(pos) * size_t(n) + size_t(r);
    out.seg_t0[w] = t0;
    out.seg_t1[w] = t1;
    out.seg_leaf[w] = leaf;
    if (overflow) {  // a full list dropped its last entry: the new last one
      const size_t q = size_t(max_segs - 1) * size_t(n) + size_t(r);
      tail_key = seg_key(out.seg_t0[q], out.seg_t1[q]);
      tail_leaf = out.seg_leaf[q];
    }
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
    if (h0 && e.x < 0) {
      lo_box[0] = a.x; lo_box[1] = a.y; lo_box[2] = a.z;
      hi_box[0] = a.w; hi_box[1] = b.x; hi_box[2] = b.y;
      emit(~e.x, a0, a1);
    }
    if (h1 && e.y < 0) {
      lo_box[0] = b.z; lo_box[1] = b.w; lo_box[2] = c.x;
      hi_box[0] = c.y; hi_box[1] = c.z; hi_box[2] = c.w;
      emit(~e.y, b0, b1);
    }
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
    if (out.hits.ar) {
      out.hits.ar[r] = 0.0f;
      out.hits.ag[r] = 0.0f;
      out.hits.ab[r] = 0.0f;
    }
  }
  return count;
}

// Warp-aggregated append of the rays with segments to the first queue (the
// whole warp calls it).
__device__ __forceinline__ void queue_first(const TraverseOut& out, bool want, int64_t r) {
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

// One thread per ray.
static __global__ void __launch_bounds__(256) traverse_kernel(const nbvh_node* __restrict__ nodes,
                                                       RayPtrs rays, int64_t n, TraverseOut out) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool active = r < n;
  int count = 0;
  if (active) count = traverse_ray(nodes, rays, n, r, out);
  if (out.queue0 || out.ring0) queue_first(out, active && count > 0, r);
}

// The rays list[0 .. *list_count) only (hybrid hierarchy: the rays whose
// interval meets the instance's root boxes); grid-stride, warp-uniform loop.
static __global__ void __launch_bounds__(256) traverse_list_kernel(const nbvh_node* __restrict__ nodes, RayPtrs rays,
                                                            int64_t n, const int32_t* __restrict__ list,
                                                            const int32_t* __restrict__ list_count,
                                                            TraverseOut out) {
  const int64_t cnt = *list_count;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < cnt; base += stride) {
    const int64_t i = base + (threadIdx.x & 31);
    const bool active = i < cnt;
    const int64_t r = active ? int64_t(list[i]) : 0;
    int count = 0;
    if (active) count = traverse_ray(nodes, rays, n, r, out);
    if (out.queue0 || out.ring0) queue_first(out, active && count > 0, r);
  }
}

// Top level of the hybrid hierarchy: for every ray, each neural instance whose
// root bounding box (grown, see root_maybe) the ray's [tmin, tmax] meets
// before its current record gets the ray appended to its list: a superset of
// the rays for which the traversal's own root test passes, so a ray left out
// would find no segment there. Appends are counted per warp in shared memory,
// then reserved with one atomic per block and instance.
constexpr int kMaxInstances = 64;
struct CullArgs {
  const nbvh_node* root[kMaxInstances];
  int32_t* list[kMaxInstances];
  int32_t* count;  // [n_inst]
  int32_t n_inst;
  unsigned long long* mask;  // optional, per ray: bit k = listed for instance k
};

__device__ __forceinline__ bool root_meets(const nbvh_node* __restrict__ nodes, const RayR& ray, float best) {
  const float4* np = reinterpret_cast<const float4*>(nodes);
  const float4 a = __ldg(np);
  const float4 b = __ldg(np + 1);
  const float4 c = __ldg(np + 2);
  const int4 e = __ldg(reinterpret_cast<const int4*>(np + 3));
  float a0, a1, b0, b1;
  const bool h0 = clip_box(ray, a.x, a.y, a.z, a.w, b.x, b.y, a0, a1) && a0 < best;
  const bool h1 = (e.y != kNodeNone) && clip_box(ray, b.z, b.w, c.x, c.y, c.z, c.w, b0, b1) && b0 < best;
  return h0 || h1;
}

// The root's bounding box grown on every side by g = 1e-3 of its size +
// 1e-4 (1 + |lo| + |hi|) (computed once per CTA into gbox: lo - g, hi + g).
__device__ __forceinline__ void grow_box(const float* box, float* gbox) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float lo = box[i], hi = box[3 + i];
    const float g = 1e-3f * (hi - lo) + 1e-4f * (1.0f + fabsf(lo) + fabsf(hi));
    gbox[i] = lo - g;
    gbox[3 + i] = hi + g;
  }
}

// The ray against a grown root box (grow_box), the interval ends compared with
// a relative slack of 1e-5; ex0 = min(tmax, the ray's record). A "false" is
// conservative: these slab values and the traversal's exactly rounded ones
// differ by a few ulps of (b - o) / d, far less than g / |d|, so a ray this
// rejects fails the traversal's root test (root_meets) too. A ray with a
// direction component too small for a finite reciprocal passes every box
// (the caller's check).
__device__ __forceinline__ bool root_maybe(const float* __restrict__ gbox, const RayR& ray, float ex0) {
  float en = ray.tmin, ex = ex0;
  const float slack = 1e-5f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float glo = gbox[i], ghi = gbox[3 + i];
    if (ray.d[i] == 0.0f) {
      if (ray.o[i] < glo || ray.o[i] > ghi) return false;
    } else {
      const float ta = (glo - ray.o[i]) * ray.inv[i];
      const float tb = (ghi - ray.o[i]) * ray.inv[i];
      en = fmaxf(en, fminf(ta, tb));
      ex = fminf(ex, fmaxf(ta, tb));
    }
  }
  return en <= ex + slack * (fabsf(ex) + fabsf(en)) + 1e-30f;
}

static __global__ void __launch_bounds__(256) tlas_cull_kernel(RayPtrs rays, int64_t n, const float* __restrict__ best_t,
                                                        CullArgs c) {
  constexpr int kWarps = 256 / 32;
  __shared__ int s_cnt[kMaxInstances], s_base[kMaxInstances];
  __shared__ int s_wbase[kWarps][kMaxInstances];  // a warp's offset within the block's share
  __shared__ float s_box[kMaxInstances][6];       // grown root bounding boxes
  for (int k = threadIdx.x; k < c.n_inst; k += blockDim.x) {
    s_cnt[k] = 0;
    const nbvh_node* nd = c.root[k];
    const bool two = nd->child1 != kNodeNone;
    float box[6];
    for (int j = 0; j < 3; ++j) {
      box[j] = two ? fminf(nd->lo0[j], nd->lo1[j]) : nd->lo0[j];
      box[3 + j] = two ? fmaxf(nd->hi0[j], nd->hi1[j]) : nd->hi0[j];
    }
    grow_box(box, s_box[k]);
  }
  __syncthreads();
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool active = r < n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t mask = 0;  // instances whose root the ray meets
  if (active) {
    const float tmin = rays.tmin[r], tmax = rays.tmax[r];
    const float ex0 = fminf(tmax, best_t[r]);
    // tmin > ex0: an empty interval (a ray a bounce pass retired, or one the
    // triangles closed before tmin), which no instance's traversal gives a
    // segment: its root test needs an entry >= tmin below tmax and the record
    if (!(tmin > ex0)) {
      const RayR ray = make_rayr(rays.ox[r], rays.oy[r], rays.oz[r], rays.dx[r], rays.dy[r], rays.dz[r], tmin,
                                 tmax);
      bool tiny = false;  // a direction component too small for a finite reciprocal
#pragma unroll
      for (int i = 0; i < 3; ++i) tiny |= ray.d[i] != 0.0f && !isfinite(ray.inv[i]);
      if (tiny) {
        mask = c.n_inst >= 64 ? ~uint64_t(0) : (uint64_t(1) << c.n_inst) - 1;
      } else {
        for (int k = 0; k < c.n_inst; ++k)
          if (root_maybe(s_box[k], ray, ex0)) mask |= uint64_t(1) << k;
      }
    }
  }
  if (active && c.mask) c.mask[r] = mask;
  const bool any = __any_sync(0xffffffffu, mask != 0);  // warps with nothing to list skip both loops
  // count: one shared-memory increment per warp and instance
  if (any) {
    for (int k = 0; k < c.n_inst; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, (mask >> k) & 1);
      if (m && lane == 0) s_wbase[warp][k] = atomicAdd(&s_cnt[k], __popc(m));
    }
  }
  __syncthreads();
  // reserve: one global increment per block and instance
  for (int k = threadIdx.x; k < c.n_inst; k += blockDim.x)
    s_base[k] = s_cnt[k] > 0 ? atomicAdd(c.count + k, s_cnt[k]) : 0;
  __syncthreads();
  // write
  if (any) {
    for (int k = 0; k < c.n_inst; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, (mask >> k) & 1);
      if ((mask >> k) & 1)
        c.list[k][s_base[k] + s_wbase[warp][k] + __popc(m & ((1u << lane) - 1u))] = int32_t(r);
    }
  }
}

// Staging records of concurrently evaluated instances: slot k's record of
// ray r at index k * n + r of each array (albedo arrays optional).
struct StageArgs {
  nbvh_hits st;
  int64_t n;
  int32_t inst_of[kMaxInstances];  // instance index of slot k
};

// Per ray, the record (the triangle instances' closest hit) and the staged
// answers of the instances the ray was listed for, taken in slot order (=
// instance order): the closest hit wins, equal t to the lower instance
// index, as if the instances had been merged one after another.
static __global__ void __launch_bounds__(256) hybrid_merge_kernel(nbvh_hits out, int32_t* __restrict__ out_inst,
                                                                  const unsigned long long* __restrict__ mask,
                                                                  int64_t n, StageArgs sa) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n) return;
  unsigned long long m = mask[r];
  if (!m) return;
  float best = out.t[r];
  int best_inst = out.hit[r] ? out_inst[r] : 0x7fffffff;
  int win = -1;
  while (m) {
    const int k = __ffsll(static_cast<long long>(m)) - 1;
    m &= m - 1;
    const size_t q = size_t(k) * size_t(sa.n) + size_t(r);
    if (!sa.st.hit[q]) continue;
    const float t = sa.st.t[q];
    if (t < best || (t == best && sa.inst_of[k] < best_inst)) {
      best = t;
      best_inst = sa.inst_of[k];
      win = k;
    }
  }
  if (win < 0) return;
  const size_t q = size_t(win) * size_t(sa.n) + size_t(r);
  out.hit[r] = 1;
  out.t[r] = best;
  out.nx[r] = sa.st.nx[q];
  out.ny[r] = sa.st.ny[q];
  out.nz[r] = sa.st.nz[q];
  out.leaf[r] = sa.st.leaf[q];
  out_inst[r] = best_inst;
  if (out.ar) {
    const bool has = sa.st.ar != nullptr;
    out.ar[r] = has ? sa.st.ar[q] : 0.0f;
    out.ag[r] = has ? sa.st.ag[q] : 0.0f;
    out.ab[r] = has ? sa.st.ab[q] : 0.0f;
  }
}

}  // namespace nbvh
