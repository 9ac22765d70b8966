// S7 + S8: training rays, brute-force labels, forward with stored activations
// and fused loss, backward into the MLP and (trilinear scatter-add) into the
// hash table, weight-gradient reduction, Adam with dynamic loss scaling.
#pragma once
#include "bounce.cuh"
#include "eval_plain.cuh"
#include "nbvh_internal.cuh"

namespace nbvh {

// ---------------------------------------------------------------------------
// S7a: training rays (Sec. 4 "Encoding, inference & training": rays through
// the scene that meet a node; Sec. 5.2 "Ray distribution": a ray trains the
// first leaf it meets). Philox4x32-10 keyed by the seed, counter
// (ray, step low, step high, draw block 0/1).
//   mode 0 (probed mix): even rays pick a leaf uniformly, a point uniform in
//     its box and a uniform direction, start on the bounding sphere and train
//     that leaf; odd rays are chords of the bounding sphere and train the first
//     leaf they meet.
//   mode 1 (paper): origin uniform in the scene box inflated by 50%, uniform
//     direction, train the first leaf met.
// ---------------------------------------------------------------------------
struct TrainRayArgs {
  int32_t mode;
  uint32_t k0, k1;
  uint32_t step_lo, step_hi;
  int64_t n;
  const nbvh_node* nodes;
  const float* leaf_box;  // [L][6]
  int32_t n_leaves;
  float centre[3], lo[3], hi[3], radius;
  RayOut out;
  int32_t* leaf;
  float* t0;
  float* t1;
  int32_t* n_valid;  // incremented per ray with a trained leaf
};

__device__ __forceinline__ void sphere_dir_f(float u1, float u2, float& x, float& y, float& z) {
  z = 1.0f - 2.0f * u1;
  float s, c;
  sincosf(kTwoPi * u2, &s, &c);
  const float r = sqrtf(fmaxf(0.0f, 1.0f - z * z));
  x = r * c;
  y = r * s;
}

// Closest leaf by (t0, leaf id) along a ray: the traversal of S1 keeping only
// the minimum key.
__device__ __forceinline__ int first_leaf_dev(const nbvh_node* __restrict__ nodes, float ox, float oy, float oz,
                                              float dx, float dy, float dz, float tmin, float tmax, float& bt0,
                                              float& bt1) {
  int best = -1;
  bt0 = 0.0f;
  bt1 = 0.0f;
  int stack[kTraverseStack];
  int sp = 0, cur = 0;
  const RayR ray = make_rayr(ox, oy, oz, dx, dy, dz, tmin, tmax);
  for (int guard = 0; guard < (1 << 26); ++guard) {
    const float4* np = reinterpret_cast<const float4*>(nodes + cur);
    const float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
    const int4 e = __ldg(reinterpret_cast<const int4*>(np + 3));
    float a0, a1, b0, b1;
    bool h0 = clip_box(ray, a.x, a.y, a.z, a.w, b.x, b.y, a0, a1);
    bool h1 = (e.y != kNodeNone) && clip_box(ray, b.z, b.w, c.x, c.y, c.z, c.w, b0, b1);
    // a subtree whose box starts after the best leaf cannot hold a smaller key
    if (best >= 0) {
      h0 = h0 && a0 <= bt0;
      h1 = h1 && b0 <= bt0;
    }
    auto take = [&](int leaf, float s0, float s1) {
      if (best < 0 || s0 < bt0 || (s0 == bt0 && leaf < best)) {
        best = leaf;
        bt0 = s0;
        bt1 = s1;
      }
    };
    if (h0 && e.x < 0) take(~e.x, a0, a1);
    if (h1 && e.y < 0) take(~e.y, b0, b1);
    const bool g0 = h0 && e.x >= 0, g1 = h1 && e.y >= 0;
    if (g0 && g1) {
      const bool first0 = a0 <= b0;
      if (sp < kTraverseStack) stack[sp++] = first0 ? e.y : e.x;
      else set_status(NBVH_ERR_UNSUPPORTED);
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
  return best;
}

static __global__ void __launch_bounds__(128) train_rays_kernel(TrainRayArgs a) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const uint4 r = philox4x32_10(make_uint4(uint32_t(i), a.step_lo, a.step_hi, 0u), a.k0, a.k1);
  const uint4 q = philox4x32_10(make_uint4(uint32_t(i), a.step_lo, a.step_hi, 1u), a.k0, a.k1);
  float ox, oy, oz, dx, dy, dz, tmax = __int_as_float(0x7f800000);
  int leaf = -1;
  float s0 = 0.0f, s1 = 0.0f;
  if (a.mode == 0 && (i & 1) == 0) {
    const int lf = int((uint64_t(r.x) * uint64_t(a.n_leaves)) >> 32);
    const float* bx = a.leaf_box + size_t(lf) * 6;
    const float px = bx[0] + u24(r.y) * (bx[3] - bx[0]);
    const float py = bx[1] + u24(r.z) * (bx[4] - bx[1]);
    const float pz = bx[2] + u24(r.w) * (bx[5] - bx[2]);
    sphere_dir_f(u24(q.x), u24(q.y), dx, dy, dz);
    const float wx = px - a.centre[0], wy = py - a.centre[1], wz = pz - a.centre[2];
    const float bb = wx * dx + wy * dy + wz * dz;
    const float cc = wx * wx + wy * wy + wz * wz - a.radius * a.radius;
    const float tb = bb + sqrtf(fmaxf(0.0f, bb * bb - cc));
    ox = px - tb * dx;
    oy = py - tb * dy;
    oz = pz - tb * dz;
    if (clip_box(ox, oy, oz, dx, dy, dz, 0.0f, tmax, bx[0], bx[1], bx[2], bx[3], bx[4], bx[5], s0, s1)) leaf = lf;
  } else {
    if (a.mode == 0) {  // chord of the bounding sphere
      float ax, ay, az, ex, ey, ez;
      sphere_dir_f(u24(r.x), u24(r.y), ax, ay, az);
      sphere_dir_f(u24(r.z), u24(r.w), ex, ey, ez);
      ox = a.centre[0] + a.radius * ax;
      oy = a.centre[1] + a.radius * ay;
      oz = a.centre[2] + a.radius * az;
      const float vx = a.centre[0] + a.radius * ex - ox;
      const float vy = a.centre[1] + a.radius * ey - oy;
      const float vz = a.centre[2] + a.radius * ez - oz;
      const float ln = sqrtf(vx * vx + vy * vy + vz * vz);
      if (ln > 0.0f) {
        dx = vx / ln; dy = vy / ln; dz = vz / ln;
      } else {
        dx = 0.0f; dy = 0.0f; dz = 1.0f;
      }
      tmax = ln;
    } else {  // origin uniform in the 1.5x scene box, uniform direction
      ox = a.centre[0] + (u24(r.x) - 0.5f) * (1.5f * (a.hi[0] - a.lo[0]));
      oy = a.centre[1] + (u24(r.y) - 0.5f) * (1.5f * (a.hi[1] - a.lo[1]));
      oz = a.centre[2] + (u24(r.z) - 0.5f) * (1.5f * (a.hi[2] - a.lo[2]));
      sphere_dir_f(u24(r.w), u24(q.x), dx, dy, dz);
    }
    leaf = first_leaf_dev(a.nodes, ox, oy, oz, dx, dy, dz, 0.0f, tmax, s0, s1);
  }
  a.out.ox[i] = ox; a.out.oy[i] = oy; a.out.oz[i] = oz;
  a.out.dx[i] = dx; a.out.dy[i] = dy; a.out.dz[i] = dz;
  a.out.tmin[i] = 0.0f;
  a.out.tmax[i] = tmax;
  a.leaf[i] = leaf;
  a.t0[i] = leaf >= 0 ? s0 : 0.0f;
  a.t1[i] = leaf >= 0 ? s1 : 0.0f;
  const unsigned m = __ballot_sync(__activemask(), leaf >= 0);
  if ((threadIdx.x & 31) == __ffs(__activemask()) - 1 && m) atomicAdd(a.n_valid, __popc(m));
}

// ---------------------------------------------------------------------------
// S7b: labels, the closest Moller-Trumbore hit among the trained leaf's own
// triangles with t in [t0, t1] (Sec. 4: ground truth by intersecting the
// actual geometry). Equal t keeps the earlier triangle of the leaf's list.
// Local depth (t - t0)/(t1 - t0) (0 for t1 == t0); geometric normal turned
// to face -d (Sec. 5.2).
// ---------------------------------------------------------------------------
// With `order` (rays grouped by leaf) the lanes of a warp mostly share one
// leaf: the triangle loop is warp-uniform and its loads are broadcasts. With
// `leaf_tris` the leaf's triangles are read contiguously.
static __global__ void __launch_bounds__(128) labels_kernel(RayPtrs rays, const int32_t* __restrict__ leaf,
                                                     const float* __restrict__ t0, const float* __restrict__ t1,
                                                     int64_t n, const float* __restrict__ tris,
                                                     const int32_t* __restrict__ tri_perm,
                                                     const int32_t* __restrict__ leaf_range,
                                                     const float* __restrict__ leaf_tris,
                                                     const int32_t* __restrict__ order, uint8_t* hit,
                                                     float* depth, float* nx, float* ny, float* nz,
                                                     const float* __restrict__ tri_albedo, float* ar, float* ag,
                                                     float* ab) {
  const int64_t item = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (item >= n) return;
  const int64_t i = order ? int64_t(order[item]) : item;
  const int lf = leaf[i];
  uint8_t h = 0;
  float dep = 0.0f, gx = 0.0f, gy = 0.0f, gz = 0.0f;
  int hit_j = -1;  // leaf-order position of the hit triangle
  if (lf >= 0) {
    const float ox = rays.ox[i], oy = rays.oy[i], oz = rays.oz[i];
    const float dx = rays.dx[i], dy = rays.dy[i], dz = rays.dz[i];
    const float a0 = t0[i], a1 = t1[i];
    const int b = leaf_range[2 * lf], e = leaf_range[2 * lf + 1];
    float best = __int_as_float(0x7f800000);
    int bj = -1;
    for (int j = b; j < e; ++j) {
      const float* T = leaf_tris ? leaf_tris + size_t(j) * 9 : tris + size_t(tri_perm[j]) * 9;
      const float v0x = __ldg(T), v0y = __ldg(T + 1), v0z = __ldg(T + 2);
      const float e1x = __ldg(T + 3) - v0x, e1y = __ldg(T + 4) - v0y, e1z = __ldg(T + 5) - v0z;
      const float e2x = __ldg(T + 6) - v0x, e2y = __ldg(T + 7) - v0y, e2z = __ldg(T + 8) - v0z;
      const float px = dy * e2z - dz * e2y, py = dz * e2x - dx * e2z, pz = dx * e2y - dy * e2x;
      const float det = e1x * px + e1y * py + e1z * pz;
      if (det == 0.0f) continue;
      const float inv = 1.0f / det;
      const float sx = ox - v0x, sy = oy - v0y, sz = oz - v0z;
      const float u = (sx * px + sy * py + sz * pz) * inv;
      if (u < 0.0f || u > 1.0f) continue;
      const float qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
      const float v = (dx * qx + dy * qy + dz * qz) * inv;
      if (v < 0.0f || u + v > 1.0f) continue;
      const float t = (e2x * qx + e2y * qy + e2z * qz) * inv;
      if (t < a0 || t > a1) continue;
      if (t < best) {
        best = t;
        bj = j;
      }
    }
    if (bj >= 0) {
      h = 1;
      hit_j = bj;
      const float span = a1 - a0;
      dep = span > 0.0f ? (best - a0) / span : 0.0f;
      const float* T = leaf_tris ? leaf_tris + size_t(bj) * 9 : tris + size_t(tri_perm[bj]) * 9;
      const float e1x = T[3] - T[0], e1y = T[4] - T[1], e1z = T[5] - T[2];
      const float e2x = T[6] - T[0], e2y = T[7] - T[1], e2z = T[8] - T[2];
      gx = e1y * e2z - e1z * e2y;
      gy = e1z * e2x - e1x * e2z;
      gz = e1x * e2y - e1y * e2x;
      const float ln = sqrtf(gx * gx + gy * gy + gz * gz);
      if (ln > 0.0f) { gx /= ln; gy /= ln; gz /= ln; }
      if (gx * dx + gy * dy + gz * dz > 0.0f) { gx = -gx; gy = -gy; gz = -gz; }
    }
  }
  hit[i] = h;
  depth[i] = dep;
  nx[i] = gx;
  ny[i] = gy;
  nz[i] = gz;
  if (ar) {  // albedo of the hit triangle (0 on a miss)
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
    if (h && tri_albedo) {
      const int t = tri_perm[hit_j];
      c0 = tri_albedo[3 * size_t(t)];
      c1 = tri_albedo[3 * size_t(t) + 1];
      c2 = tri_albedo[3 * size_t(t) + 2];
    }
    ar[i] = c0;
    ag[i] = c1;
    ab[i] = c2;
  }
}

// Stored forward of one training batch (row i = segment of ray i).
struct TrainBuffers {
  float* X;         // [S][K] features
  float* H;         // [n_hidden][S][W] hidden activations (after ReLU)
  float* O;         // [S][n_out] raw outputs
  float* G;         // [S][n_out] dL/dO (scaled) or the caller's output gradient
  float* loss_seg;  // [S] per-segment loss term (0 for invalid)
  float* dZ;        // [n_hidden][S][W] pre-activation gradients
};

struct TrainArgs {
  GridParams gp;
  const void* table;
  const float* mlp;
  int32_t n_hidden, width, n_out;
  RayPtrs rays;
  const int32_t* leaf;   // < 0: the segment does not train
  const float* t0;
  const float* t1;
  int64_t n;
  Labels lab;            // null hit pointer: no loss (plain forward)
  const int32_t* n_valid;
  float loss_scale;
  const float* loss_scale_dev;  // if set, overrides loss_scale (dynamic scaling)
  TrainBuffers buf;
  float* grad_table;     // FP32 [entries][F]
};

// Forward (FP32, CUDA cores): 32 segments per tile, float-float positions,
// activations stored for the backward; with labels, loss and dL/dO fused.
template <typename T, int F, int W>
__global__ void __launch_bounds__(kPlainThreads, 1) train_forward_plain(TrainArgs a) {
  extern __shared__ __align__(16) float smem[];
  const int K = a.gp.n_inputs;
  const int L = a.gp.n_levels;
  const int N = a.gp.n_samples;
  const int n_out = a.n_out;
  const int hid_w = (a.n_hidden - 1) * W * W + W * n_out;
  const int feat_floats = max(K * kPlainTM, hid_w);
  float* sfeat = smem;
  float* sW1 = sfeat + feat_floats;
  float* shA = sW1 + K * W;
  float* shB = shA + W * kPlainTM;
  float* sout = shB + W * kPlainTM;
  int* sray = reinterpret_cast<int*>(sout + 8 * kPlainTM);
  float* st0 = reinterpret_cast<float*>(sray + kPlainTM);
  float* st1 = st0 + kPlainTM;

  const int64_t n_tiles = (a.n + kPlainTM - 1) / kPlainTM;
  if (int64_t(blockIdx.x) >= n_tiles) return;
  const float* W1 = a.mlp;
  const float* b1 = W1 + W * K;
  for (int i = threadIdx.x; i < K * W; i += blockDim.x) {
    const int n = i / K, k = i - n * K;
    sW1[k * W + n] = __ldg(W1 + i);
  }
  const T* table = static_cast<const T*>(a.table);
  const float inv_valid = a.n_valid ? 1.0f / float(max(1, *a.n_valid)) : 1.0f;
  const float lscale = a.loss_scale_dev ? *a.loss_scale_dev : a.loss_scale;

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    if (threadIdx.x < kPlainTM) {
      const int64_t i = tile * kPlainTM + threadIdx.x;
      int ray = -1;
      float t0 = 0.0f, t1 = 0.0f;
      if (i < a.n && a.leaf[i] >= 0) {
        ray = int(i);
        t0 = a.t0[i];
        t1 = a.t1[i];
      }
      sray[threadIdx.x] = ray;
      st0[threadIdx.x] = t0;
      st1[threadIdx.x] = t1;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < kPlainTM * N; p += blockDim.x) {
      const int s = p % kPlainTM;
      const int k = p / kPlainTM;
      const int ray = sray[s];
      const int kb = k * L * F;
      if (ray < 0) {
        for (int j = 0; j < L * F; ++j) sfeat[act_idx(kb + j, s)] = 0.0f;
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
    // store features [S][K]
    for (int idx = threadIdx.x; idx < kPlainTM * K; idx += blockDim.x) {
      const int s = idx / K, k = idx - s * K;
      const int64_t i = tile * kPlainTM + s;
      if (i < a.n) a.buf.X[i * K + k] = sfeat[act_idx(k, s)];
    }
    dense_plain<W, true>(sfeat, K, sW1, b1, shA);
    __syncthreads();
    auto store_h = [&](const float* h, int layer) {
      for (int idx = threadIdx.x; idx < kPlainTM * W; idx += blockDim.x) {
        const int s = idx / W, j = idx - s * W;
        const int64_t i = tile * kPlainTM + s;
        if (i < a.n) a.buf.H[(size_t(layer) * a.n + i) * W + j] = h[act_idx(j, s)];
      }
    };
    store_h(shA, 0);
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
    const float* bh = b1 + W;
    float* hin = shA;
    float* hout = shB;
    const float* wt = sfeat;
    for (int h = 1; h < a.n_hidden; ++h) {
      dense_plain<W, true>(hin, W, wt, bh + W * W, hout);
      __syncthreads();
      store_h(hout, h);
      float* tmp = hin; hin = hout; hout = tmp;
      bh += W * W + W;
      wt += W * W;
    }
    {
      const float* bo = bh + n_out * W;
      for (int i = threadIdx.x; i < n_out * kPlainTM; i += blockDim.x) {
        const int j = i / kPlainTM, s = i - j * kPlainTM;
        float acc = __ldg(bo + j);
        for (int k = 0; k < W; ++k) acc = fmaf(wt[k * n_out + j], hin[act_idx(k, s)], acc);
        sout[j * kPlainTM + s] = acc;
      }
    }
    __syncthreads();
    if (threadIdx.x < kPlainTM) {
      const int s = threadIdx.x;
      const int64_t i = tile * kPlainTM + s;
      if (i < a.n) {
        float o[8], g[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int j = 0; j < n_out; ++j) o[j] = sout[j * kPlainTM + s];
        float term = 0.0f;
        if (a.lab.hit && sray[s] >= 0) {
          float alb[3];
          const bool has_alb = n_out >= 8 && a.lab.ar;
          if (has_alb) {
            alb[0] = a.lab.ar[i];
            alb[1] = a.lab.ag[i];
            alb[2] = a.lab.ab[i];
          }
          term = loss_terms(o, float(a.lab.hit[i]), a.lab.depth[i], a.lab.nx[i], a.lab.ny[i], a.lab.nz[i],
                            has_alb ? alb : nullptr, lscale * inv_valid, g);
        }
        for (int j = 0; j < n_out; ++j) a.buf.O[i * n_out + j] = o[j];
        if (a.lab.hit) {
          for (int j = 0; j < n_out; ++j) a.buf.G[i * n_out + j] = g[j];
          a.buf.loss_seg[i] = term;
        }
      }
    }
    __syncthreads();
  }
}

// Backward (FP32, CUDA cores): from G = dL/dO through the MLP (dZ stored for
// the weight gradients) to dL/dfeatures, then the adjoint of the encoding:
// every (sample, level, corner) adds weight * dL/dfeature into its table
// entry's FP32 gradient with a vector atomic (collisions accumulate).
template <typename T, int F, int W>
__global__ void __launch_bounds__(kPlainThreads, 1) train_backward_plain(TrainArgs a) {
  extern __shared__ __align__(16) float smem[];
  const int K = a.gp.n_inputs;
  const int L = a.gp.n_levels;
  const int N = a.gp.n_samples;
  const int n_out = a.n_out;
  const int nh = a.n_hidden;
  float* sdX = smem;                       // [K][TM] dL/dfeatures
  float* sWh = sdX + K * kPlainTM;         // [(nh - 1)][W][W] hidden weights, row-major
  float* sWo = sWh + (nh - 1) * W * W;     // [n_out][W]
  float* sdA = sWo + n_out * W;            // [W][TM]
  float* sdB = sdA + W * kPlainTM;         // [W][TM]
  float* sH = sdB + W * kPlainTM;          // [W][TM] stored activation of the current layer
  float* sG = sH + W * kPlainTM;           // [8][TM]
  int* sray = reinterpret_cast<int*>(sG + 8 * kPlainTM);
  float* st0 = reinterpret_cast<float*>(sray + kPlainTM);
  float* st1 = st0 + kPlainTM;

  const int64_t n_tiles = (a.n + kPlainTM - 1) / kPlainTM;
  if (int64_t(blockIdx.x) >= n_tiles) return;
  const float* W1 = a.mlp;  // [W][K]; dX reads it at warp-uniform addresses (L1 broadcast)
  {
    const float* p = a.mlp + W * K + W;
    for (int h = 1; h < nh; ++h) {
      for (int i = threadIdx.x; i < W * W; i += blockDim.x) sWh[(h - 1) * W * W + i] = __ldg(p + i);
      p += W * W + W;
    }
    for (int i = threadIdx.x; i < n_out * W; i += blockDim.x) sWo[i] = __ldg(p + i);
  }
  __syncthreads();

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    if (threadIdx.x < kPlainTM) {
      const int64_t i = tile * kPlainTM + threadIdx.x;
      int ray = -1;
      float t0 = 0.0f, t1 = 0.0f;
      if (i < a.n && a.leaf[i] >= 0) {
        ray = int(i);
        t0 = a.t0[i];
        t1 = a.t1[i];
      }
      sray[threadIdx.x] = ray;
      st0[threadIdx.x] = t0;
      st1[threadIdx.x] = t1;
    }
    for (int idx = threadIdx.x; idx < n_out * kPlainTM; idx += blockDim.x) {
      const int j = idx / kPlainTM, s = idx - j * kPlainTM;
      const int64_t i = tile * kPlainTM + s;
      sG[j * kPlainTM + s] = i < a.n ? a.buf.G[i * n_out + j] : 0.0f;
    }
    __syncthreads();
    // layer by layer from the top: dH = (dZ_above) W_above; dZ = dH * (H > 0)
    float* dz = sdA;
    for (int h = nh - 1; h >= 0; --h) {
      for (int idx = threadIdx.x; idx < W * kPlainTM; idx += blockDim.x) {
        const int j = idx / kPlainTM, s = idx - j * kPlainTM;
        const int64_t i = tile * kPlainTM + s;
        sH[j * kPlainTM + s] = i < a.n ? a.buf.H[(size_t(h) * a.n + i) * W + j] : 0.0f;
      }
      __syncthreads();
      float* out = (h == nh - 1) ? sdA : (dz == sdA ? sdB : sdA);
      for (int idx = threadIdx.x; idx < W * kPlainTM; idx += blockDim.x) {
        const int j = idx / kPlainTM, s = idx - j * kPlainTM;
        float acc = 0.0f;
        if (h == nh - 1) {
          for (int o = 0; o < n_out; ++o) acc = fmaf(sG[o * kPlainTM + s], sWo[o * W + j], acc);
        } else {
          const float* Wa = sWh + h * W * W;  // layer h+1 weights [W][W]
          for (int o = 0; o < W; ++o) acc = fmaf(dz[o * kPlainTM + s], Wa[o * W + j], acc);
        }
        const float g = sH[j * kPlainTM + s] > 0.0f ? acc : 0.0f;
        out[j * kPlainTM + s] = g;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < W * kPlainTM; idx += blockDim.x) {
        const int s = idx / W, j = idx - s * W;
        const int64_t i = tile * kPlainTM + s;
        if (i < a.n) a.buf.dZ[(size_t(h) * a.n + i) * W + j] = out[j * kPlainTM + s];
      }
      dz = out;
      __syncthreads();
    }
    // dX = dZ1 W1
    for (int idx = threadIdx.x; idx < K * kPlainTM; idx += blockDim.x) {
      const int k = idx / kPlainTM, s = idx - k * kPlainTM;
      float acc = 0.0f;
      for (int o = 0; o < W; ++o) acc = fmaf(dz[o * kPlainTM + s], __ldg(W1 + o * K + k), acc);
      sdX[k * kPlainTM + s] = acc;
    }
    __syncthreads();
    // adjoint of the encoding: scatter into the table gradient
    for (int p = threadIdx.x; p < kPlainTM * N; p += blockDim.x) {
      const int s = p % kPlainTM;
      const int k = p / kPlainTM;
      const int ray = sray[s];
      if (ray < 0) continue;
      FF x, y, z;
      sample_point_ff(a.gp, a.rays.ox[ray], a.rays.oy[ray], a.rays.oz[ray], a.rays.dx[ray], a.rays.dy[ray],
                      a.rays.dz[ray], st0[s], st1[s], k, x, y, z);
      for (int l = 0; l < L; ++l) {
        Corners c;
        level_corners(a.gp, l, x, y, z, c);
        float gf[F];
#pragma unroll
        for (int f = 0; f < F; ++f) gf[f] = sdX[(k * L * F + l * F + f) * kPlainTM + s];
        float* gt = a.grad_table + a.gp.offset[l] * F;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float* dst = gt + size_t(c.idx[q]) * F;
          if constexpr (F == 2) {
            atomicAdd(reinterpret_cast<float2*>(dst), make_float2(c.w[q] * gf[0], c.w[q] * gf[1]));
          } else if constexpr (F % 4 == 0) {
#pragma unroll
            for (int f = 0; f < F; f += 4)
              atomicAdd(reinterpret_cast<float4*>(dst + f),
                        make_float4(c.w[q] * gf[f], c.w[q] * gf[f + 1], c.w[q] * gf[f + 2], c.w[q] * gf[f + 3]));
          } else {
            atomicAdd(dst, c.w[q] * gf[0]);
          }
        }
      }
    }
    __syncthreads();
  }
}

inline size_t train_fwd_smem(int K, int W, int nh, int n_out) { return plain_smem_bytes(K, W, nh, n_out); }

inline size_t train_bwd_smem(int K, int W, int nh, int n_out) {
  return sizeof(float) * (size_t(K) * kPlainTM + size_t(nh - 1) * W * W + size_t(n_out) * W +
                          3 * size_t(W) * kPlainTM + 8 * kPlainTM) +
         3 * sizeof(int) * kPlainTM;
}

// ---------------------------------------------------------------------------
// Weight gradients: dW_l[o][j] = sum_i dZ_l[i][o] A_{l-1}[i][j] and
// db_l[o] = sum_i dZ_l[i][o] over the batch (A_0 = features, A_l = H_l; the
// output layer uses G). Split-K over segment chunks: each block reduces a
// 32 x 32 output block over one chunk in FP32 and adds it with atomics.
// ---------------------------------------------------------------------------
constexpr int kWgTile = 32;
constexpr int kWgChunk = 2048;

static __global__ void __launch_bounds__(256) weight_grad_kernel(const float* __restrict__ dZ, int n_o,
                                                          const float* __restrict__ A, int n_j, int64_t n,
                                                          float* __restrict__ dW, float* __restrict__ db) {
  __shared__ float sz[32][kWgTile + 1];
  __shared__ float sa[32][kWgTile + 1];
  const int o0 = blockIdx.x * kWgTile;
  const int j0 = blockIdx.y * kWgTile;
  const int64_t i0 = int64_t(blockIdx.z) * kWgChunk;
  const int64_t i1 = min(n, i0 + kWgChunk);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 4 outputs
  float acc[4] = {0, 0, 0, 0};
  float bacc = 0.0f;
  for (int64_t ib = i0; ib < i1; ib += 32) {
    for (int idx = threadIdx.x; idx < 32 * kWgTile; idx += blockDim.x) {
      const int r = idx / kWgTile, c = idx - r * kWgTile;
      const int64_t i = ib + r;
      sz[r][c] = (i < i1 && o0 + c < n_o) ? dZ[i * n_o + o0 + c] : 0.0f;
      sa[r][c] = (i < i1 && j0 + c < n_j) ? A[i * n_j + j0 + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const float av = sa[r][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(sz[r][ty * 4 + q], av, acc[q]);
      if (blockIdx.y == 0 && ty == 0) bacc += sz[r][tx];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int o = o0 + ty * 4 + q, j = j0 + tx;
    if (o < n_o && j < n_j) atomicAdd(dW + size_t(o) * n_j + j, acc[q]);
  }
  if (blockIdx.y == 0 && ty == 0 && o0 + tx < n_o) atomicAdd(db + o0 + tx, bacc);
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba 2015, bias-corrected) on FP32 masters with the gradient
// unscaled by the loss scale; a step whose gradients hold inf/NaN is skipped
// and halves the scale; 2000 clean steps double it. The working copy of the
// table (the precision the kernels read) is refreshed from the master.
// ---------------------------------------------------------------------------
struct AdamState {
  float* loss_scale;   // device scalar
  int32_t* good_steps; // device scalar
  int32_t* bad;        // device scalar: set when a gradient is not finite
  int32_t* applied;    // device scalar: 1 when the last step was applied
};

// Sets *bad when a gradient is not finite (g 16-byte aligned: four at a time).
static __global__ void grad_check_kernel(const float* __restrict__ g, int64_t n, int32_t* bad) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  bool ok = true;
  const bool vec = (reinterpret_cast<uintptr_t>(g) & 15) == 0;
  const int64_t head = vec ? (n & ~int64_t(3)) : 0;
  for (int64_t q = tid; q < head / 4; q += stride) {
    const float4 x = reinterpret_cast<const float4*>(g)[q];
    ok &= isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(x.w);
  }
  for (int64_t i = head + tid; i < n; i += stride) ok &= isfinite(g[i]);
  if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0) atomicExch(bad, 1);
}

// One Adam update of one parameter (the gradient unscaled by the loss scale).
__device__ __forceinline__ float adam_update(float g, float& m, float& v, float p, float lr, float b1, float b2,
                                             float eps, float c1, float c2) {
  const float mi = b1 * m + (1.0f - b1) * g;
  const float vi = b2 * v + (1.0f - b2) * g * g;
  m = mi;
  v = vi;
  return p - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <typename T>
__device__ __forceinline__ T adam_work(float p) {
  if constexpr (std::is_same<T, __half>::value) return __float2half_rn(p);
  else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __float2bfloat16_rn(p);
  else return p;
}

// Adam over n parameters, four at a time (VEC: every pointer 16-byte aligned,
// the 16-bit working copy 8-byte aligned; the last n % 4 one at a time), the
// working copy refreshed and the gradient cleared. A step whose gradient was
// not finite only clears it.
template <typename T, bool VEC>
__global__ void adam_kernel(float* __restrict__ master, T* __restrict__ work, float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2, AdamState st) {
  const bool skip = *st.bad != 0;
  const float inv_scale = 1.0f / *st.loss_scale;
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  int64_t head = 0;  // parameters [0, head) go four at a time
  if constexpr (VEC) {
    head = n & ~int64_t(3);
    for (int64_t q = tid; q < head / 4; q += stride) {
      float4* g4 = reinterpret_cast<float4*>(grad) + q;
      if (!skip) {
        const float4 g = *g4;
        float4 mm = reinterpret_cast<const float4*>(m)[q];
        float4 vv = reinterpret_cast<const float4*>(v)[q];
        float4 p = reinterpret_cast<const float4*>(master)[q];
        p.x = adam_update(g.x * inv_scale, mm.x, vv.x, p.x, lr, b1, b2, eps, c1, c2);
        p.y = adam_update(g.y * inv_scale, mm.y, vv.y, p.y, lr, b1, b2, eps, c1, c2);
        p.z = adam_update(g.z * inv_scale, mm.z, vv.z, p.z, lr, b1, b2, eps, c1, c2);
        p.w = adam_update(g.w * inv_scale, mm.w, vv.w, p.w, lr, b1, b2, eps, c1, c2);
        reinterpret_cast<float4*>(m)[q] = mm;
        reinterpret_cast<float4*>(v)[q] = vv;
        reinterpret_cast<float4*>(master)[q] = p;
        if (work) {
          if constexpr (std::is_same<T, float>::value) {
            reinterpret_cast<float4*>(work)[q] = p;
          } else {
            T w4[4] = {adam_work<T>(p.x), adam_work<T>(p.y), adam_work<T>(p.z), adam_work<T>(p.w)};
            reinterpret_cast<uint2*>(work)[q] = *reinterpret_cast<const uint2*>(w4);
          }
        }
      }
      *g4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
  for (int64_t i = head + tid; i < n; i += stride) {
    if (!skip) {
      float mi = m[i], vi = v[i];
      const float p = adam_update(grad[i] * inv_scale, mi, vi, master[i], lr, b1, b2, eps, c1, c2);
      m[i] = mi;
      v[i] = vi;
      master[i] = p;
      if (work) work[i] = adam_work<T>(p);
    }
    grad[i] = 0.0f;
  }
}

static __global__ void loss_scale_update_kernel(AdamState st, int32_t dynamic) {
  const bool bad = *st.bad != 0;
  *st.applied = bad ? 0 : 1;
  if (dynamic) {
    if (bad) {
      *st.loss_scale = fmaxf(1.0f, *st.loss_scale * 0.5f);
      *st.good_steps = 0;
    } else if (++*st.good_steps >= 2000) {
      *st.loss_scale = *st.loss_scale * 2.0f;
      *st.good_steps = 0;
    }
  }
  *st.bad = 0;
}

// The batch loss in FP32 (sum of the per-segment terms over the valid count):
// each thread sums its grid-stride share with compensated (Kahan) summation,
// blocks reduce pairwise in shared memory into partial[blockIdx.x], and one
// block reduces the partials the same way. No atomics, so the value does not
// depend on scheduling.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
  const float y = __fsub_rn(x, comp);
  const float t = __fadd_rn(sum, y);
  comp = __fsub_rn(__fsub_rn(t, sum), y);
  sum = t;
}

__device__ __forceinline__ float block_pairwise_sum(float v, float* sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) sm[threadIdx.x] = __fadd_rn(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  return sm[0];
}

static __global__ void __launch_bounds__(256) loss_partial_kernel(const float* __restrict__ term, int64_t n,
                                                                  float* __restrict__ partial) {
  __shared__ float sm[256];
  float sum = 0.0f, comp = 0.0f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    kahan_add(sum, comp, term[i]);
  const float b = block_pairwise_sum(sum, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

static __global__ void __launch_bounds__(256) loss_final_kernel(const float* __restrict__ partial, int nb,
                                                                const int32_t* __restrict__ n_valid,
                                                                float* __restrict__ out) {
  __shared__ float sm[256];
  float sum = 0.0f, comp = 0.0f;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) kahan_add(sum, comp, partial[i]);
  const float b = block_pairwise_sum(sum, sm);
  if (threadIdx.x == 0) *out = b / float(max(1, *n_valid));
}

// The same loss with FP64 accumulation, for the finite-difference gradient
// check only (nbvh_loss_fp64): central differences subtract two nearly equal
// losses. (*out must be zero before the launch; blocks add their sums.)
static __global__ void loss_fd_fp64_kernel(const float* __restrict__ term, int64_t n, const int32_t* n_valid,
                                           double* out) {
  __shared__ double sm[256];
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    acc += double(term[i]);
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, sm[0] / double(max(1, *n_valid)));
}

// ---------------------------------------------------------------------------
// Rays grouped by trained leaf (counting sort): order[] lists the training rays
// leaf by leaf, then the rays that train nothing.
// ---------------------------------------------------------------------------
static __global__ void leaf_hist_kernel(const int32_t* __restrict__ leaf, int64_t n, int32_t* counts) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && leaf[i] >= 0) atomicAdd(counts + leaf[i], 1);
}

// Exclusive scan of n_leaves counts into cursor[0..n_leaves]; cursor[n_leaves]
// is the number of training rays (where the rays without a leaf start).
static __global__ void __launch_bounds__(1024) leaf_scan_kernel(const int32_t* __restrict__ counts, int n_leaves,
                                                         int32_t* cursor) {
  __shared__ int32_t part[1024];
  const int per = (n_leaves + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per, e = min(n_leaves, b + per);
  int32_t s = 0;
  for (int i = b; i < e; ++i) s += counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    const int32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int32_t run = part[threadIdx.x] - s;
  for (int i = b; i < e; ++i) {
    cursor[i] = run;
    run += counts[i];
  }
  if (threadIdx.x == blockDim.x - 1) cursor[n_leaves] = part[threadIdx.x];
}

static __global__ void leaf_scatter_kernel(const int32_t* __restrict__ leaf, int64_t n, int n_leaves, int32_t* cursor,
                                    int32_t* order) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int lf = leaf[i];
  const int pos = atomicAdd(cursor + (lf >= 0 ? lf : n_leaves), 1);
  order[pos] = int32_t(i);
}

}  // namespace nbvh

namespace nbvh {

// ---------------------------------------------------------------------------
// Error-driven training (Sec. 5.1 "Node error", Sec. 5.2 "Ray distribution"):
// each ray's first leaf is counted as hit; with leaf probabilities the ray
// trains that leaf only with its probability (uniform u from Philox4x32-10,
// key = seed words, counter (ray, step low, step high, 3), u = top 24 bits
// * 2^-24, trained iff u < prob[leaf]); a rejected ray trains nothing.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(256) leaf_select_kernel(int32_t* __restrict__ leaf, int64_t n, uint32_t k0,
                                                          uint32_t k1, uint32_t step_lo, uint32_t step_hi,
                                                          const float* __restrict__ prob, uint32_t* hits,
                                                          int32_t* n_valid) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int lf = leaf[i];
  if (lf < 0) return;
  if (hits) atomicAdd(hits + lf, 1u);
  if (prob) {
    const uint4 r = philox4x32_10(make_uint4(uint32_t(i), step_lo, step_hi, 3u), k0, k1);
    if (!(u24(r.x) < __ldg(prob + lf))) {
      leaf[i] = -1;
      atomicSub(n_valid, 1);
    }
  }
}

// Per-leaf sums of the trained rays' loss terms, one warp per leaf over the
// leaf's contiguous range of the grouped order (after leaf_scatter_kernel,
// cursor[l] is the range's end and counts[l] its length). The term of order
// position i is term[i] (by_item: the tensor-core forward stores terms by
// item) or term[order[i]] (by ray). Compensated per-lane sums, then a
// pairwise warp reduction; one lane adds the leaf's sum and count (FP32).
static __global__ void __launch_bounds__(256) leaf_loss_kernel(const float* __restrict__ term,
                                                               const int32_t* __restrict__ order, int by_item,
                                                               const int32_t* __restrict__ counts,
                                                               const int32_t* __restrict__ cursor, int n_leaves,
                                                               uint32_t* trained, float* loss) {
  const int l = int(blockIdx.x) * (blockDim.x >> 5) + int(threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (l >= n_leaves) return;
  const int cnt = counts[l];
  const int end = cursor[l], start = end - cnt;
  float sum = 0.0f, comp = 0.0f;
  for (int i = start + lane; i < end; i += 32) kahan_add(sum, comp, term[by_item ? i : order[i]]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, o));
  if (lane == 0 && cnt > 0) {
    trained[l] += uint32_t(cnt);
    loss[l] = __fadd_rn(loss[l], sum);
  }
}

// ---------------------------------------------------------------- launch
template <typename T, int F, int W>
cudaError_t launch_train_plain(bool backward, const TrainArgs& a, cudaStream_t s) {
  const size_t smem = backward ? train_bwd_smem(a.gp.n_inputs, W, a.n_hidden, a.n_out)
                               : train_fwd_smem(a.gp.n_inputs, W, a.n_hidden, a.n_out);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  auto kern = backward ? train_backward_plain<T, F, W> : train_forward_plain<T, F, W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPlainThreads, smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (a.n + kPlainTM - 1) / kPlainTM;
  int64_t grid = int64_t(sm_count()) * (occ < 1 ? 1 : occ);
  if (tiles < grid) grid = tiles;
  if (grid < 1) return cudaSuccess;
  kern<<<unsigned(grid), kPlainThreads, smem, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T, int F>
cudaError_t launch_train_tf(bool bwd, int W, const TrainArgs& a, cudaStream_t s) {
  switch (W) {
    case 16: return launch_train_plain<T, F, 16>(bwd, a, s);
    case 32: return launch_train_plain<T, F, 32>(bwd, a, s);
    case 64: return launch_train_plain<T, F, 64>(bwd, a, s);
    case 128: return launch_train_plain<T, F, 128>(bwd, a, s);
  }
  return cudaErrorInvalidValue;
}

// The FP32 training kernels of one table type (one translation unit each).
template <typename T>
cudaError_t launch_train_t(bool bwd, const nbvh_model_desc* d, const TrainArgs& a, cudaStream_t s) {
  switch (d->n_features) {
    case 1: return launch_train_tf<T, 1>(bwd, d->width, a, s);
    case 2: return launch_train_tf<T, 2>(bwd, d->width, a, s);
    case 4: return launch_train_tf<T, 4>(bwd, d->width, a, s);
    case 8: return launch_train_tf<T, 8>(bwd, d->width, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nbvh
