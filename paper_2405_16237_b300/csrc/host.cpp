// Host-side parts of the C ABI: status strings, level layout, MLP parameter
// count and the S0 leaf build (median split over triangle centroids).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <vector>

#include "../../include/nbvh.h"
#include "nbvh_host.h"

extern "C" const char* nbvh_status_string(nbvh_status s) {
  switch (s) {
    case NBVH_OK: return "ok";
    case NBVH_ERR_INVALID_ARG: return "invalid argument";
    case NBVH_ERR_CUDA: return "CUDA runtime error";
    case NBVH_ERR_OOM: return "out of memory";
    case NBVH_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case NBVH_ERR_SEGMENT_OVERFLOW: return "a ray crossed more leaves than max_segs";
    case NBVH_ERR_TIMEOUT: return "a bounded device wait gave up";
    case NBVH_ERR_UNSUPPORTED: return "unsupported shape or precision";
  }
  return "unknown status";
}

extern "C" int32_t nbvh_version(void) { return 1; }
extern "C" int32_t nbvh_built_arch(void) { return 1030; }

namespace nbvh_host {

bool desc_valid(const nbvh_model_desc* d) {
  if (!d) return false;
  if (d->n_levels < 1 || d->n_levels > NBVH_MAX_LEVELS) return false;
  if (!(d->n_features == 1 || d->n_features == 2 || d->n_features == 4 || d->n_features == 8))
    return false;
  if (d->log2_table < 4 || d->log2_table > 26) return false;
  if (d->base_res < 1 || !(d->growth >= 1.0f) || !std::isfinite(d->growth)) return false;
  if (d->n_samples < 1 || d->n_samples > NBVH_MAX_SAMPLES) return false;
  if (d->n_samples * d->n_levels * d->n_features > NBVH_MAX_INPUTS) return false;
  if (d->n_hidden < 1 || d->n_hidden > 8) return false;
  if (!(d->width == 16 || d->width == 32 || d->width == 64 || d->width == 128)) return false;
  if (d->n_out < 5 || d->n_out > 8) return false;
  if (d->table_prec < NBVH_FP32 || d->table_prec > NBVH_BF16) return false;
  if (d->mlp_prec < NBVH_FP32 || d->mlp_prec > NBVH_BF16) return false;
  if (!(d->frame_extent > 0.0f) || !std::isfinite(d->frame_extent)) return false;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(d->frame_centre[i])) return false;
  if ((d->flags & ~NBVH_FLAG_REVERSE_INSIDE) != 0) return false;
  return true;
}

bool layout(const nbvh_model_desc* d, int32_t* res, int32_t* dense, int64_t* size, int64_t* offset,
            int64_t* total) {
  const int64_t T = int64_t(1) << d->log2_table;
  int64_t acc = 0;
  for (int l = 0; l < d->n_levels; ++l) {
    const double n = std::floor(double(d->base_res) * std::pow(double(d->growth), double(l)));
    if (!(n >= 1.0) || n > 1.0e7) return false;
    const int64_t N = int64_t(n);
    const int64_t verts = (N + 1) * (N + 1) * (N + 1);
    res[l] = int32_t(N);
    dense[l] = verts <= T ? 1 : 0;
    size[l] = verts <= T ? verts : T;
    offset[l] = acc;
    acc += size[l];
  }
  for (int l = d->n_levels; l < NBVH_MAX_LEVELS; ++l) {
    res[l] = 0; dense[l] = 0; size[l] = 0; offset[l] = acc;
  }
  *total = acc;
  return true;
}

int64_t mlp_params(const nbvh_model_desc* d) {
  const int64_t K = int64_t(d->n_samples) * d->n_levels * d->n_features;
  int64_t n = 0, in = K;
  for (int h = 0; h < d->n_hidden; ++h) {
    n += in * d->width + d->width;
    in = d->width;
  }
  n += in * d->n_out + d->n_out;
  return n;
}

}  // namespace nbvh_host

extern "C" nbvh_status nbvh_level_layout(const nbvh_model_desc* desc, int32_t* res, int32_t* dense,
                                         int64_t* size, int64_t* offset, int64_t* total) {
  if (!nbvh_host::desc_valid(desc) || !res || !dense || !size || !offset || !total)
    return NBVH_ERR_INVALID_ARG;
  return nbvh_host::layout(desc, res, dense, size, offset, total) ? NBVH_OK : NBVH_ERR_INVALID_ARG;
}

extern "C" nbvh_status nbvh_mlp_param_count(const nbvh_model_desc* desc, int64_t* count) {
  if (!nbvh_host::desc_valid(desc) || !count) return NBVH_ERR_INVALID_ARG;
  *count = nbvh_host::mlp_params(desc);
  return NBVH_OK;
}

// ---------------------------------------------------------------------------
// S0: median-split leaf clusters.
// ---------------------------------------------------------------------------
namespace {

struct SplitNode {
  int64_t begin, end;  // range in the working index array
  int left = -1, right = -1;
};

float round_down(double x) {
  float f = float(x);
  if (double(f) > x) f = std::nextafter(f, -INFINITY);
  return f;
}

float round_up(double x) {
  float f = float(x);
  if (double(f) < x) f = std::nextafter(f, INFINITY);
  return f;
}

}  // namespace

extern "C" nbvh_status nbvh_build_leaves(const float* tris, int64_t n_tris, int32_t n_leaves,
                                         double inflate_rel, nbvh_node* nodes, int32_t node_cap,
                                         int32_t* out_n_nodes, int32_t* tri_perm, int32_t* leaf_range,
                                         float* leaf_box, nbvh_scene_info* info) {
  if (!tris || n_tris < 1 || n_tris > (int64_t(1) << 31) - 1 || n_leaves < 1 ||
      int64_t(n_leaves) > n_tris || !nodes || !out_n_nodes || !tri_perm || !leaf_range ||
      !leaf_box || !info || !(inflate_rel >= 0.0) || !std::isfinite(inflate_rel))
    return NBVH_ERR_INVALID_ARG;
  const int32_t need_nodes = std::max(1, n_leaves - 1);
  if (node_cap < need_nodes) return NBVH_ERR_INVALID_ARG;

  // Scene AABB and frame (double from float: exact).
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < n_tris * 9; ++i) {
    const double v = tris[i];
    if (!std::isfinite(v)) return NBVH_ERR_INVALID_ARG;
    lo[i % 3] = std::min(lo[i % 3], v);
    hi[i % 3] = std::max(hi[i % 3], v);
  }
  double E = 0.0, diag2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    E = std::max(E, hi[a] - lo[a]);
    diag2 += (hi[a] - lo[a]) * (hi[a] - lo[a]);
  }
  for (int a = 0; a < 3; ++a) {
    info->lo[a] = float(lo[a]);
    info->hi[a] = float(hi[a]);
    info->centre[a] = float((lo[a] + hi[a]) / 2.0);
  }
  info->extent = float(E);
  info->sphere_radius = float(1.01 * std::sqrt(diag2) / 2.0);

  // Centroids ((v0 + v1) + v2) / 3 in double.
  std::vector<double> cent(size_t(n_tris) * 3);
  for (int64_t t = 0; t < n_tris; ++t)
    for (int a = 0; a < 3; ++a)
      cent[t * 3 + a] = ((double(tris[t * 9 + a]) + double(tris[t * 9 + 3 + a])) +
                         double(tris[t * 9 + 6 + a])) / 3.0;

  std::vector<int32_t> idx(n_tris);
  for (int64_t t = 0; t < n_tris; ++t) idx[t] = int32_t(t);
  std::vector<SplitNode> sn;
  sn.reserve(size_t(2) * n_leaves);
  sn.push_back({0, n_tris});
  // Max-heap on (size, -id): the largest leaf first, ties to the lowest id.
  auto cmp = [&](int a, int b) {
    const int64_t sa = sn[a].end - sn[a].begin, sb = sn[b].end - sn[b].begin;
    if (sa != sb) return sa < sb;
    return a > b;
  };
  std::priority_queue<int, std::vector<int>, decltype(cmp)> heap(cmp);
  heap.push(0);
  int32_t leaves = 1;
  while (leaves < n_leaves) {
    const int id = heap.top();
    heap.pop();
    const int64_t b = sn[id].begin, e = sn[id].end;
    if (e - b < 2) return NBVH_ERR_INVALID_ARG;
    double cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = b; i < e; ++i)
      for (int a = 0; a < 3; ++a) {
        cmin[a] = std::min(cmin[a], cent[size_t(idx[i]) * 3 + a]);
        cmax[a] = std::max(cmax[a], cent[size_t(idx[i]) * 3 + a]);
      }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
      if (cmax[a] - cmin[a] > cmax[axis] - cmin[axis]) axis = a;
    std::sort(idx.begin() + b, idx.begin() + e, [&](int32_t p, int32_t q) {
      const double cp = cent[size_t(p) * 3 + axis], cq = cent[size_t(q) * 3 + axis];
      if (cp != cq) return cp < cq;
      return p < q;
    });
    const int64_t h = (e - b) / 2;
    const int l = int(sn.size()), r = l + 1;
    sn.push_back({b, b + h});
    sn.push_back({b + h, e});
    sn[id].left = l;
    sn[id].right = r;
    heap.push(l);
    heap.push(r);
    ++leaves;
  }

  // Number leaves in order; boxes; internal nodes in preorder.
  const double pad = inflate_rel * E;
  std::vector<int> leaf_of(sn.size(), -1), node_of(sn.size(), -1);
  std::vector<float> box(size_t(6) * n_leaves);
  int32_t next_leaf = 0, next_node = 0;
  int64_t perm_pos = 0;
  std::vector<int> order;  // preorder of split nodes
  std::vector<int> stack{0};
  while (!stack.empty()) {
    const int id = stack.back();
    stack.pop_back();
    order.push_back(id);
    if (sn[id].left >= 0) {
      stack.push_back(sn[id].right);
      stack.push_back(sn[id].left);
    }
  }
  for (int id : order) {
    if (sn[id].left >= 0) {
      node_of[id] = next_node++;
      continue;
    }
    const int32_t lf = next_leaf++;
    leaf_of[id] = lf;
    const int64_t b = sn[id].begin, e = sn[id].end;
    std::vector<int32_t> mine(idx.begin() + b, idx.begin() + e);
    std::sort(mine.begin(), mine.end());
    double blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t t : mine) {
      tri_perm[perm_pos++] = t;
      for (int v = 0; v < 3; ++v)
        for (int a = 0; a < 3; ++a) {
          const double x = tris[size_t(t) * 9 + v * 3 + a];
          blo[a] = std::min(blo[a], x);
          bhi[a] = std::max(bhi[a], x);
        }
    }
    leaf_range[2 * lf] = int32_t(perm_pos - int64_t(mine.size()));
    leaf_range[2 * lf + 1] = int32_t(perm_pos);
    for (int a = 0; a < 3; ++a) {
      box[size_t(lf) * 6 + a] = round_down(blo[a] - pad);
      box[size_t(lf) * 6 + 3 + a] = round_up(bhi[a] + pad);
    }
  }
  std::memcpy(leaf_box, box.data(), sizeof(float) * box.size());

  // Bounds of every split node (union of its leaves' boxes, exact in float).
  std::vector<float> nb(sn.size() * 6);
  for (auto it = order.rbegin(); it != order.rend(); ++it) {
    const int id = *it;
    float* o = &nb[size_t(id) * 6];
    if (sn[id].left < 0) {
      std::memcpy(o, &box[size_t(leaf_of[id]) * 6], 6 * sizeof(float));
    } else {
      const float* a = &nb[size_t(sn[id].left) * 6];
      const float* c = &nb[size_t(sn[id].right) * 6];
      for (int k = 0; k < 3; ++k) {
        o[k] = std::min(a[k], c[k]);
        o[3 + k] = std::max(a[3 + k], c[3 + k]);
      }
    }
  }
  auto child_ref = [&](int id) { return sn[id].left >= 0 ? node_of[id] : ~leaf_of[id]; };
  if (n_leaves == 1) {
    nbvh_node& n = nodes[0];
    std::memset(&n, 0, sizeof(n));
    for (int k = 0; k < 3; ++k) {
      n.lo0[k] = nb[k];
      n.hi0[k] = nb[3 + k];
      n.lo1[k] = 0.0f;
      n.hi1[k] = 0.0f;
    }
    n.child0 = ~0;
    n.child1 = 0x7fffffff;
  } else {
    for (int id : order) {
      if (sn[id].left < 0) continue;
      nbvh_node& n = nodes[node_of[id]];
      std::memset(&n, 0, sizeof(n));
      const float* a = &nb[size_t(sn[id].left) * 6];
      const float* c = &nb[size_t(sn[id].right) * 6];
      for (int k = 0; k < 3; ++k) {
        n.lo0[k] = a[k];
        n.hi0[k] = a[3 + k];
        n.lo1[k] = c[k];
        n.hi1[k] = c[3 + k];
      }
      n.child0 = child_ref(sn[id].left);
      n.child1 = child_ref(sn[id].right);
    }
  }
  *out_n_nodes = need_nodes;
  return NBVH_OK;
}

// ---------------------------------------------------------------------------
// Classical triangle BLAS (Sec. 7: a BLAS of the hybrid hierarchy is either a
// classical BVH or an N-BVH). Binned surface-area-heuristic build over
// triangle centroids: at each node, 32 bins per axis over the centroid bounds;
// the split minimising area(left) * n_left + area(right) * n_right is taken
// when it beats keeping the node as a leaf of at most max_leaf triangles; a
// node whose centroids coincide is split at its middle index.
// ---------------------------------------------------------------------------
namespace {

struct Box3 {
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const Box3& b) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], b.lo[a]);
      hi[a] = std::max(hi[a], b.hi[a]);
    }
  }
  double area() const {
    if (!(hi[0] >= lo[0])) return 0.0;
    const double x = double(hi[0]) - lo[0], y = double(hi[1]) - lo[1], z = double(hi[2]) - lo[2];
    return 2.0 * (x * y + y * z + z * x);
  }
};

struct BlasNode {
  int64_t begin, end;
  Box3 box;
  int left = -1, right = -1;
};

constexpr int kSahBins = 32;

}  // namespace

extern "C" nbvh_status nbvh_build_tri_blas(const float* tris, int64_t n_tris, int32_t max_leaf, nbvh_node* nodes,
                                           int32_t node_cap, int32_t* out_n_nodes, int32_t* tri_perm,
                                           int32_t* leaf_range, int32_t leaf_cap, int32_t* out_n_leaves) {
  if (!tris || n_tris < 1 || n_tris > (int64_t(1) << 30) || max_leaf < 1 || max_leaf > 64 || !nodes ||
      !out_n_nodes || !tri_perm || !leaf_range || !out_n_leaves)
    return NBVH_ERR_INVALID_ARG;
  if (int64_t(node_cap) < std::max<int64_t>(1, n_tris - 1) || int64_t(leaf_cap) < n_tris)
    return NBVH_ERR_INVALID_ARG;
  std::vector<Box3> tb(static_cast<size_t>(n_tris));
  std::vector<float> cent(size_t(n_tris) * 3);
  for (int64_t t = 0; t < n_tris; ++t) {
    for (int v = 0; v < 3; ++v)
      for (int a = 0; a < 3; ++a) {
        const float x = tris[size_t(t) * 9 + v * 3 + a];
        if (!std::isfinite(x)) return NBVH_ERR_INVALID_ARG;
        tb[t].lo[a] = std::min(tb[t].lo[a], x);
        tb[t].hi[a] = std::max(tb[t].hi[a], x);
      }
    for (int a = 0; a < 3; ++a) cent[size_t(t) * 3 + a] = 0.5f * (tb[t].lo[a] + tb[t].hi[a]);
  }
  std::vector<int32_t> idx(static_cast<size_t>(n_tris));
  for (int64_t t = 0; t < n_tris; ++t) idx[t] = int32_t(t);

  std::vector<BlasNode> bn;
  bn.reserve(size_t(2 * n_tris));
  BlasNode root;
  root.begin = 0;
  root.end = n_tris;
  for (int64_t t = 0; t < n_tris; ++t) root.box.grow(tb[t]);
  bn.push_back(root);
  std::vector<int> work{0};
  while (!work.empty()) {
    const int id = work.back();
    work.pop_back();
    const int64_t b = bn[id].begin, e = bn[id].end, n = e - b;
    if (n <= 1) continue;
    float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = b; i < e; ++i)
      for (int a = 0; a < 3; ++a) {
        cmin[a] = std::min(cmin[a], cent[size_t(idx[i]) * 3 + a]);
        cmax[a] = std::max(cmax[a], cent[size_t(idx[i]) * 3 + a]);
      }
    double best_cost = INFINITY;
    int best_axis = -1, best_bin = -1;
    for (int a = 0; a < 3; ++a) {
      const double ext = double(cmax[a]) - cmin[a];
      if (!(ext > 0.0)) continue;
      Box3 bb[kSahBins];
      int64_t cnt[kSahBins] = {};
      const double scale = kSahBins / ext;
      for (int64_t i = b; i < e; ++i) {
        const int32_t t = idx[i];
        int k = int((double(cent[size_t(t) * 3 + a]) - cmin[a]) * scale);
        k = std::min(std::max(k, 0), kSahBins - 1);
        ++cnt[k];
        bb[k].grow(tb[t]);
      }
      double right_area[kSahBins];
      int64_t right_cnt[kSahBins];
      Box3 acc;
      int64_t c = 0;
      for (int k = kSahBins - 1; k > 0; --k) {
        acc.grow(bb[k]);
        c += cnt[k];
        right_area[k] = acc.area();
        right_cnt[k] = c;
      }
      Box3 lacc;
      int64_t lc = 0;
      for (int k = 0; k < kSahBins - 1; ++k) {
        lacc.grow(bb[k]);
        lc += cnt[k];
        if (lc == 0 || right_cnt[k + 1] == 0) continue;
        const double cost = lacc.area() * double(lc) + right_area[k + 1] * double(right_cnt[k + 1]);
        if (cost < best_cost) {
          best_cost = cost;
          best_axis = a;
          best_bin = k;
        }
      }
    }
    // one node visit costs about one triangle test
    const double area = bn[id].box.area();
    if (n <= max_leaf && !(best_cost + area < area * double(n))) continue;
    int64_t mid;
    if (best_axis >= 0) {
      const int a = best_axis;
      const double scale = kSahBins / (double(cmax[a]) - cmin[a]);
      auto it = std::partition(idx.begin() + b, idx.begin() + e, [&](int32_t t) {
        int k = int((double(cent[size_t(t) * 3 + a]) - cmin[a]) * scale);
        k = std::min(std::max(k, 0), kSahBins - 1);
        return k <= best_bin;
      });
      mid = int64_t(it - idx.begin());
    } else {
      mid = b + n / 2;  // coincident centroids: split by index
    }
    if (mid <= b || mid >= e) mid = b + n / 2;
    BlasNode l, r;
    l.begin = b;
    l.end = mid;
    r.begin = mid;
    r.end = e;
    for (int64_t i = b; i < mid; ++i) l.box.grow(tb[idx[i]]);
    for (int64_t i = mid; i < e; ++i) r.box.grow(tb[idx[i]]);
    const int li = int(bn.size());
    bn.push_back(l);
    bn.push_back(r);
    bn[id].left = li;
    bn[id].right = li + 1;
    work.push_back(li + 1);
    work.push_back(li);
  }

  // Preorder numbering: internal nodes -> node ids, leaves -> leaf ids in
  // left-to-right order; triangles of leaf i are tri_perm[leaf_range[2i] ..
  // leaf_range[2i+1]).
  std::vector<int> order, stack{0};
  while (!stack.empty()) {
    const int id = stack.back();
    stack.pop_back();
    order.push_back(id);
    if (bn[id].left >= 0) {
      stack.push_back(bn[id].right);
      stack.push_back(bn[id].left);
    }
  }
  std::vector<int> node_of(bn.size(), -1), leaf_of(bn.size(), -1);
  int32_t nn = 0, nl = 0;
  int64_t pos = 0;
  for (int id : order) {
    if (bn[id].left >= 0) {
      node_of[id] = nn++;
      continue;
    }
    leaf_of[id] = nl;
    leaf_range[2 * nl] = int32_t(pos);
    for (int64_t i = bn[id].begin; i < bn[id].end; ++i) tri_perm[pos++] = idx[i];
    leaf_range[2 * nl + 1] = int32_t(pos);
    ++nl;
  }
  auto ref = [&](int id) { return bn[id].left >= 0 ? node_of[id] : ~leaf_of[id]; };
  auto put = [&](nbvh_node& d, int slot, const Box3& bx) {
    float* lo = slot == 0 ? d.lo0 : d.lo1;
    float* hi = slot == 0 ? d.hi0 : d.hi1;
    for (int a = 0; a < 3; ++a) {
      lo[a] = bx.lo[a];
      hi[a] = bx.hi[a];
    }
  };
  if (nn == 0) {  // a single leaf: the root holds its box and an empty second slot
    nbvh_node& d = nodes[0];
    std::memset(&d, 0, sizeof(d));
    put(d, 0, bn[0].box);
    d.child0 = ~0;
    d.child1 = 0x7fffffff;
    nn = 1;
  } else {
    for (int id : order) {
      if (bn[id].left < 0) continue;
      nbvh_node& d = nodes[node_of[id]];
      std::memset(&d, 0, sizeof(d));
      put(d, 0, bn[bn[id].left].box);
      put(d, 1, bn[bn[id].right].box);
      d.child0 = ref(bn[id].left);
      d.child1 = ref(bn[id].right);
    }
  }
  *out_n_nodes = nn;
  *out_n_leaves = nl;
  return NBVH_OK;
}

// ---------------------------------------------------------------------------
// N-BVH from a cut through a base BVH (Sec. 5.1 "Base-BVH cut optimization":
// the nodes along the cut become the N-BVH's leaves). The base BVH is in the
// nbvh_node format of nbvh_build_tri_blas; a cut entry is a base reference:
// 0 <= ref < n_base_nodes names the subtree of base node ref (0 = the whole
// tree), ref < 0 names base leaf ~ref. Every root-to-leaf path of the base
// tree must cross exactly one entry.
// ---------------------------------------------------------------------------
namespace {

struct BaseTree {
  const nbvh_node* nodes;
  int32_t n_nodes;
  const int32_t* leaf_range;
  int32_t n_leaves;
  std::vector<int> node_parent, node_slot, leaf_parent, leaf_slot;

  bool init() {
    node_parent.assign(size_t(n_nodes), -1);
    node_slot.assign(size_t(n_nodes), -1);
    leaf_parent.assign(size_t(n_leaves), -1);
    leaf_slot.assign(size_t(n_leaves), -1);
    for (int i = 0; i < n_nodes; ++i) {
      const int32_t ch[2] = {nodes[i].child0, nodes[i].child1};
      for (int s = 0; s < 2; ++s) {
        const int32_t c = ch[s];
        if (c == 0x7fffffff) continue;
        if (c >= 0) {
          if (c >= n_nodes || c == 0 || node_parent[c] >= 0) return false;
          node_parent[c] = i;
          node_slot[c] = s;
        } else {
          const int32_t l = ~c;
          if (l >= n_leaves || leaf_parent[l] >= 0) return false;
          leaf_parent[l] = i;
          leaf_slot[l] = s;
        }
      }
    }
    return true;
  }
  // box of a reference: a subtree's box is the union of its node's child boxes
  void box(int32_t ref, float* lo, float* hi) const {
    if (ref >= 0) {
      const nbvh_node& nd = nodes[ref];
      const bool two = nd.child1 != 0x7fffffff;
      for (int a = 0; a < 3; ++a) {
        lo[a] = two ? std::min(nd.lo0[a], nd.lo1[a]) : nd.lo0[a];
        hi[a] = two ? std::max(nd.hi0[a], nd.hi1[a]) : nd.hi0[a];
      }
    } else {
      const int32_t l = ~ref;
      const nbvh_node& p = nodes[leaf_parent[l]];
      const float* slo = leaf_slot[l] == 0 ? p.lo0 : p.lo1;
      const float* shi = leaf_slot[l] == 0 ? p.hi0 : p.hi1;
      for (int a = 0; a < 3; ++a) {
        lo[a] = slo[a];
        hi[a] = shi[a];
      }
    }
  }
  // triangle range of a reference (leaves of a subtree are consecutive)
  void range(int32_t ref, int32_t& b, int32_t& e) const {
    if (ref < 0) {
      b = leaf_range[2 * (~ref)];
      e = leaf_range[2 * (~ref) + 1];
      return;
    }
    int32_t first = ref, last = ref;
    while (first >= 0) first = nodes[first].child0;
    for (;;) {
      const nbvh_node& nd = nodes[last];
      const int32_t c = nd.child1 == 0x7fffffff ? nd.child0 : nd.child1;
      if (c < 0) {
        last = c;
        break;
      }
      last = c;
    }
    b = leaf_range[2 * (~first)];
    e = leaf_range[2 * (~last) + 1];
  }
};

}  // namespace

extern "C" nbvh_status nbvh_build_cut(const nbvh_node* base_nodes, int32_t n_base_nodes,
                                      const int32_t* base_leaf_range, int32_t n_base_leaves, const int32_t* cut,
                                      int32_t n_cut, double inflate_rel, float extent, nbvh_node* nodes,
                                      int32_t node_cap, int32_t* out_n_nodes, int32_t* leaf_range, float* leaf_box,
                                      int32_t* leaf_ref) {
  if (!base_nodes || n_base_nodes < 1 || !base_leaf_range || n_base_leaves < 1 || !cut || n_cut < 1 || !nodes ||
      !out_n_nodes || !leaf_range || !leaf_box || !leaf_ref || node_cap < std::max(1, n_cut - 1) ||
      !(inflate_rel >= 0.0) || !std::isfinite(inflate_rel) || !(extent > 0.0f))
    return NBVH_ERR_INVALID_ARG;
  BaseTree bt{base_nodes, n_base_nodes, base_leaf_range, n_base_leaves, {}, {}, {}, {}};
  if (!bt.init()) return NBVH_ERR_INVALID_ARG;
  // mark the cut entries
  std::vector<char> node_cut(size_t(n_base_nodes), 0), leaf_cut(size_t(n_base_leaves), 0);
  for (int i = 0; i < n_cut; ++i) {
    const int32_t r = cut[i];
    if (r >= 0) {
      if (r >= n_base_nodes || node_cut[r]) return NBVH_ERR_INVALID_ARG;
      node_cut[r] = 1;
    } else {
      if (~r >= n_base_leaves || leaf_cut[~r]) return NBVH_ERR_INVALID_ARG;
      leaf_cut[~r] = 1;
    }
  }
  // depth-first from the root: references above the cut become internal
  // N-BVH nodes, cut references leaves (numbered in this order)
  const double pad = inflate_rel * double(extent);
  int32_t n_leaf = 0, n_int = 0;
  struct Item {
    int32_t ref, parent, slot;
  };
  std::vector<Item> stack{{0, -1, 0}};
  int32_t visited_cut = 0;
  while (!stack.empty()) {
    const Item it = stack.back();
    stack.pop_back();
    const bool is_cut = it.ref >= 0 ? node_cut[it.ref] != 0 : leaf_cut[~it.ref] != 0;
    int32_t out_ref;
    float lo[3], hi[3];
    bt.box(it.ref, lo, hi);
    if (is_cut) {
      const int32_t lf = n_leaf++;
      if (lf >= n_cut) return NBVH_ERR_INVALID_ARG;
      int32_t b, e;
      bt.range(it.ref, b, e);
      leaf_range[2 * lf] = b;
      leaf_range[2 * lf + 1] = e;
      leaf_ref[lf] = it.ref;
      for (int a = 0; a < 3; ++a) {
        leaf_box[6 * lf + a] = round_down(double(lo[a]) - pad);
        leaf_box[6 * lf + 3 + a] = round_up(double(hi[a]) + pad);
      }
      ++visited_cut;
      out_ref = ~lf;
    } else {
      if (it.ref < 0) return NBVH_ERR_INVALID_ARG;  // a base leaf below no cut entry
      const int32_t id = n_int++;
      if (id >= node_cap) return NBVH_ERR_INVALID_ARG;
      std::memset(&nodes[id], 0, sizeof(nbvh_node));
      nodes[id].child1 = 0x7fffffff;
      const nbvh_node& bn = base_nodes[it.ref];
      if (bn.child1 != 0x7fffffff) stack.push_back({bn.child1, id, 1});
      stack.push_back({bn.child0, id, 0});
      out_ref = id;
    }
    if (it.parent >= 0) {
      nbvh_node& p = nodes[it.parent];
      float* plo = it.slot == 0 ? p.lo0 : p.lo1;
      float* phi = it.slot == 0 ? p.hi0 : p.hi1;
      if (is_cut) {
        for (int a = 0; a < 3; ++a) {
          plo[a] = leaf_box[6 * (~out_ref) + a];
          phi[a] = leaf_box[6 * (~out_ref) + 3 + a];
        }
      }
      if (it.slot == 0) p.child0 = out_ref;
      else p.child1 = out_ref;
    }
  }
  if (visited_cut != n_cut) return NBVH_ERR_INVALID_ARG;  // some entries lie below others
  if (n_int == 0) {  // the cut is the root alone: one leaf
    std::memset(&nodes[0], 0, sizeof(nbvh_node));
    for (int a = 0; a < 3; ++a) {
      nodes[0].lo0[a] = leaf_box[a];
      nodes[0].hi0[a] = leaf_box[3 + a];
    }
    nodes[0].child0 = ~0;
    nodes[0].child1 = 0x7fffffff;
    n_int = 1;
  } else {
    // an internal node's box in its parent: the union of its children's boxes
    for (int id = n_int - 1; id >= 0; --id) {
      nbvh_node& nd = nodes[id];
      for (int s = 0; s < 2; ++s) {
        const int32_t c = s == 0 ? nd.child0 : nd.child1;
        if (c < 0 || c == 0x7fffffff) continue;
        const nbvh_node& ch = nodes[c];
        float* dlo = s == 0 ? nd.lo0 : nd.lo1;
        float* dhi = s == 0 ? nd.hi0 : nd.hi1;
        const bool two = ch.child1 != 0x7fffffff;
        for (int a = 0; a < 3; ++a) {
          dlo[a] = two ? std::min(ch.lo0[a], ch.lo1[a]) : ch.lo0[a];
          dhi[a] = two ? std::max(ch.hi0[a], ch.hi1[a]) : ch.hi0[a];
        }
      }
    }
  }
  *out_n_nodes = n_int;
  return NBVH_OK;
}

// ---------------------------------------------------------------- error-driven cut (Sec. 5.1, Sec. 5.2)
extern "C" nbvh_status nbvh_rank_leaves(const uint32_t* hits, const uint32_t* trained, const float* loss,
                                        int32_t n_leaves, int64_t n_rays, double* q, double* p, double* r,
                                        float* prob) {
  if (!hits || !trained || !loss || n_leaves < 1 || n_rays < 0 || !q || !p || !r || !prob)
    return NBVH_ERR_INVALID_ARG;
  // q of a hit leaf that no ray trained: the mean q of the trained leaves
  double q_sum = 0.0;
  int64_t q_n = 0;
  for (int32_t i = 0; i < n_leaves; ++i)
    if (trained[i] > 0) {
      q_sum += double(loss[i]) / double(trained[i]);
      ++q_n;
    }
  const double q_mean = q_n > 0 ? q_sum / double(q_n) : 1.0;
  const double denom = double(std::max<int64_t>(1, n_rays));
  double r_max = -HUGE_VAL;
  for (int32_t i = 0; i < n_leaves; ++i) {
    q[i] = trained[i] > 0 ? double(loss[i]) / double(trained[i]) : q_mean;
    p[i] = double(hits[i]) / denom;
    r[i] = (hits[i] > 0 && q[i] > 0.0) ? 2.0 * std::log(q[i]) + std::log(p[i]) : -HUGE_VAL;
    if (std::isfinite(r[i])) r_max = std::max(r_max, r[i]);
  }
  if (!std::isfinite(r_max)) r_max = 0.0;
  for (int32_t i = 0; i < n_leaves; ++i)
    prob[i] = float(std::isfinite(r[i]) ? std::max(std::exp(r[i] - r_max), 0.005) : 0.005);
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_refine_cut(const nbvh_node* base_nodes, int32_t n_base_nodes, const int32_t* cut,
                                       int32_t n_cut, const double* r, const float* prob, int32_t k_splits,
                                       int32_t* new_cut, float* new_prob, int32_t cap, int32_t* n_new) {
  if (!base_nodes || n_base_nodes < 1 || !cut || n_cut < 1 || !r || !prob || k_splits < 0 || !new_cut ||
      !new_prob || !n_new)
    return NBVH_ERR_INVALID_ARG;
  // splittable: an internal base reference with a finite ranking
  std::vector<int32_t> cand;
  for (int32_t i = 0; i < n_cut; ++i) {
    if (cut[i] < -n_base_nodes - 1 || cut[i] >= n_base_nodes) return NBVH_ERR_INVALID_ARG;
    if (cut[i] >= 0 && std::isfinite(r[i])) cand.push_back(i);
  }
  std::stable_sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) { return r[a] > r[b]; });
  const size_t k = std::min(size_t(k_splits), cand.size());
  std::vector<uint8_t> chosen(size_t(n_cut), 0);
  for (size_t i = 0; i < k; ++i) chosen[size_t(cand[i])] = 1;
  int32_t m = 0;
  auto put = [&](int32_t ref, float pr) {
    if (m < cap) {
      new_cut[m] = ref;
      new_prob[m] = pr;
    }
    ++m;
  };
  for (int32_t i = 0; i < n_cut; ++i) {
    if (!chosen[size_t(i)]) {
      put(cut[i], prob[i]);
      continue;
    }
    const nbvh_node& nd = base_nodes[cut[i]];
    put(nd.child0, 1.0f);  // a new leaf has no statistics yet: it trains with probability 1
    if (nd.child1 != 0x7fffffff) put(nd.child1, 1.0f);
  }
  *n_new = m;
  return m <= cap ? NBVH_OK : NBVH_ERR_WORKSPACE_TOO_SMALL;
}
