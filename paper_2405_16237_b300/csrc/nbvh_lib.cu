// Device entry points of the C ABI (include/nbvh.h). The heavy kernel
// families (the fused evaluation kernels, the training kernels) are
// instantiated in their own translation units (tu_*.cu) and reached through
// launch.h; the small kernels live in the headers included here.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "nbvh_host.h"
#include "nbvh_internal.cuh"
#include "launch.h"
#include "traverse.cuh"
#include "bounce.cuh"
#include "tri_blas.cuh"
#include "probe.cuh"

namespace nbvh {

std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

// Status words of the translation units (nbvh_internal.cuh).
std::vector<StatusReader>& status_readers() {
  static std::vector<StatusReader> v;
  return v;
}
std::mutex& status_mu() {
  static std::mutex m;
  return m;
}
void register_status_reader(StatusReader fn) {
  std::lock_guard<std::mutex> lk(status_mu());
  status_readers().push_back(fn);
}

namespace {

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

bool rays_valid(const nbvh_rays& r) {
  if (r.n < 0) return false;
  if (r.n == 0) return true;
  return r.ox && r.oy && r.oz && r.dx && r.dy && r.dz && r.tmin && r.tmax;
}

RayPtrs ray_ptrs(const nbvh_rays& r) { return RayPtrs{r.ox, r.oy, r.oz, r.dx, r.dy, r.dz, r.tmin, r.tmax}; }

bool make_grid(const nbvh_model_desc* d, GridParams& gp) {
  int32_t res[NBVH_MAX_LEVELS], dense[NBVH_MAX_LEVELS];
  int64_t size[NBVH_MAX_LEVELS], offset[NBVH_MAX_LEVELS], total = 0;
  if (!nbvh_host::layout(d, res, dense, size, offset, &total)) return false;
  std::memset(&gp, 0, sizeof(gp));
  gp.n_levels = d->n_levels;
  gp.n_features = d->n_features;
  gp.n_samples = d->n_samples;
  gp.n_inputs = d->n_samples * d->n_levels * d->n_features;
  for (int i = 0; i < 3; ++i) gp.centre[i] = d->frame_centre[i];
  gp.inv_extent = 1.0f / d->frame_extent;
  gp.extent = d->frame_extent;
  gp.hash_mask = uint32_t((uint64_t(1) << d->log2_table) - 1);
  for (int l = 0; l < NBVH_MAX_LEVELS; ++l) {
    gp.res[l] = res[l];
    gp.dense[l] = dense[l];
    gp.offset[l] = offset[l];
  }
  return true;
}


template <typename T>
cudaError_t launch_encode_t(int F, const GridParams& gp, const void* table, RayPtrs r, const int32_t* seg_ray,
                            const float* t0, const float* t1, int64_t n_seg, float* feat, cudaStream_t s) {
  const int64_t work = n_seg * gp.n_samples;
  const unsigned grid = unsigned((work + 127) / 128);
  switch (F) {
    case 1: encode_kernel<T, 1><<<grid, 128, 0, s>>>(gp, table, r, seg_ray, t0, t1, n_seg, feat); break;
    case 2: encode_kernel<T, 2><<<grid, 128, 0, s>>>(gp, table, r, seg_ray, t0, t1, n_seg, feat); break;
    case 4: encode_kernel<T, 4><<<grid, 128, 0, s>>>(gp, table, r, seg_ray, t0, t1, n_seg, feat); break;
    case 8: encode_kernel<T, 8><<<grid, 128, 0, s>>>(gp, table, r, seg_ray, t0, t1, n_seg, feat); break;
    default: return cudaErrorInvalidValue;
  }
  count_launches(1);
  return cudaGetLastError();
}

EvalArgs base_args(const nbvh_model_desc* d, const GridParams& gp, const void* table, const float* mlp,
                   const nbvh_rays& rays) {
  EvalArgs a;
  std::memset(&a, 0, sizeof(a));
  a.gp = gp;
  a.table = table;
  a.mlp = mlp;
  a.n_hidden = d->n_hidden;
  a.width = d->width;
  a.n_out = d->n_out;
  a.rays = ray_ptrs(rays);
  return a;
}

nbvh_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return NBVH_OK;
  if (e == cudaErrorInvalidConfiguration) return NBVH_ERR_UNSUPPORTED;
  return NBVH_ERR_CUDA;
}

template <int MODE>
cudaError_t launch_tc(const nbvh_model_desc* d, const EvalArgs& a, int64_t n, const TcPlan& pl, cudaStream_t s) {
  switch (d->table_prec) {
    case NBVH_FP32: return launch_tc_tm<float, MODE>(d, a, n, pl, s);
    case NBVH_FP16: return launch_tc_tm<__half, MODE>(d, a, n, pl, s);
    case NBVH_BF16: return launch_tc_tm<__nv_bfloat16, MODE>(d, a, n, pl, s);
  }
  return cudaErrorInvalidValue;
}

template <bool WAVE>
cudaError_t launch_plain(const nbvh_model_desc* d, const EvalArgs& a, int64_t n, cudaStream_t s) {
  switch (d->table_prec) {
    case NBVH_FP32: return launch_plain_t<float, WAVE>(d->n_features, a, n, s);
    case NBVH_FP16: return launch_plain_t<__half, WAVE>(d->n_features, a, n, s);
    case NBVH_BF16: return launch_plain_t<__nv_bfloat16, WAVE>(d->n_features, a, n, s);
  }
  return cudaErrorInvalidValue;
}

// Options: the caller's, or the defaults.
nbvh_query_options default_options() {
  nbvh_query_options o;
  std::memset(&o, 0, sizeof(o));
  o.schedule = NBVH_SCHEDULE_PERSISTENT;
  o.patience_cycles = 4000;
  o.traverse_block = 128;
  o.eval_threads = 0;
  o.w1_mode = NBVH_W1_AUTO;
  o.eval_pipeline = NBVH_PIPELINE_AUTO;
  o.wait_spins = 0;
  o.test_phantom_items = 0;
  o.segments_out = nullptr;
  o.instance_streams = 0;
  o.partial_items = 0;
  return o;
}

bool options_valid(const nbvh_query_options& o) {
  return (o.schedule == NBVH_SCHEDULE_WAVES || o.schedule == NBVH_SCHEDULE_PERSISTENT) && o.patience_cycles >= 0 &&
         o.patience_cycles <= (int64_t(1) << 40) &&
         (o.traverse_block == 64 || o.traverse_block == 128 || o.traverse_block == 256) &&
         (o.eval_threads == 0 || o.eval_threads == 256 || o.eval_threads == 512) && o.w1_mode >= NBVH_W1_AUTO &&
         o.w1_mode <= NBVH_W1_STREAMED && o.eval_pipeline >= NBVH_PIPELINE_AUTO &&
         o.eval_pipeline <= NBVH_PIPELINE_WARP_SPECIALISED && o.wait_spins >= 0 && o.wait_spins <= (int64_t(1) << 40) &&
         o.test_phantom_items >= 0 && o.test_phantom_items <= 1024 && o.instance_streams >= 0 &&
         o.instance_streams <= 64 && o.partial_items >= 0 && o.partial_items <= 128;
}

// Whether a query with these options runs the warp-specialised persistent
// kernel: only when asked for (the automatic choice is the phase kernel,
// which measured faster on the icosphere workload; the autotuner times both).
bool use_ws(const nbvh_model_desc* d, const nbvh_query_options& o) {
  return d->mlp_prec != NBVH_FP32 && o.schedule == NBVH_SCHEDULE_PERSISTENT &&
         o.eval_pipeline == NBVH_PIPELINE_WARP_SPECIALISED;
}

// The evaluation kernels can run this model with these options (checked on
// the host before anything is enqueued). query: the options' schedule and
// pipeline apply (a segment list always runs the phase kernel).
bool eval_stageable(const nbvh_model_desc* d, const nbvh_query_options& o, bool query = true) {
  if (d->mlp_prec == NBVH_FP32)
    return plain_chunk_samples(d->n_samples, d->n_levels * d->n_features, d->width, d->n_hidden, d->n_out) >= 0;
  if (query && o.eval_pipeline == NBVH_PIPELINE_WARP_SPECIALISED)
    return o.schedule == NBVH_SCHEDULE_PERSISTENT && ws_supported(d);
  if (query && use_ws(d, o)) return true;
  return tc_plan(d, o.eval_threads, o.w1_mode).ok;
}

cudaError_t launch_ws(const nbvh_model_desc* d, const EvalArgs& a, cudaStream_t s) {
  switch (d->table_prec) {
    case NBVH_FP32: return launch_ws_t<float>(d, a, s);
    case NBVH_FP16: return launch_ws_t<__half>(d, a, s);
    case NBVH_BF16: return launch_ws_t<__nv_bfloat16>(d, a, s);
  }
  return cudaErrorInvalidValue;
}

// The evaluation's plan for desc under options o. The first layer's 16-bit
// image is written into `image` (once per call, before the evaluation
// launches): a streamed plan's CTAs copy it chunk by chunk (a.w1_image), a
// resident plan's copy it whole at their start (a.w1_copy); without an image
// buffer a resident plan's CTAs convert the FP32 weights themselves.
cudaError_t prepare_eval(const nbvh_model_desc* d, EvalArgs& a, const nbvh_query_options& o, void* image,
                         TcPlan* plan, cudaStream_t s, bool query = true) {
  std::memset(plan, 0, sizeof(*plan));
  a.w1_image = nullptr;
  a.w1_copy = nullptr;
  if (d->mlp_prec == NBVH_FP32) return cudaSuccess;
  *plan = tc_plan(d, o.eval_threads, o.w1_mode, query);
  if (!plan->ok) return cudaErrorInvalidConfiguration;
  if (plan->stream) {
    if (!image) return cudaErrorInvalidConfiguration;
    cudaError_t e = launch_w1_image(d, a.mlp, plan->threads, image, s);
    if (e != cudaSuccess) return e;
    a.w1_image = image;
  } else if (image) {
    cudaError_t e = launch_w1_image(d, a.mlp, plan->threads, image, s);
    if (e != cudaSuccess) return e;
    a.w1_copy = image;
  }
  return cudaSuccess;
}

// One evaluation launch of MODE (0 list, 1 query wave or persistent, 2
// training forward) after prepare_eval.
template <int MODE>
cudaError_t launch_eval(const nbvh_model_desc* d, const EvalArgs& a, int64_t n, const TcPlan& plan, cudaStream_t s) {
  if (d->mlp_prec == NBVH_FP32) {
    if constexpr (MODE == 2) return cudaErrorInvalidValue;
    else return launch_plain<MODE == 1>(d, a, n, s);
  }
  return launch_tc<MODE>(d, a, n, plan, s);
}

// Bytes of the first-layer image an evaluation of desc may need.
size_t image_bytes(const nbvh_model_desc* d) { return d->mlp_prec == NBVH_FP32 ? 0 : tc_image_bytes(d); }

// ---------------------------------------------------------------- kernel-class timing
// While timing is enabled (nbvh_set_timing) each timed section records a CUDA
// event pair on its stream around its launches (not while the stream is being
// captured into a graph); nbvh_get_kernel_times sums them per class.
struct TimedRecord {
  int kind;
  cudaEvent_t a, b;
  int64_t launches;
};

std::mutex g_timing_mu;
bool g_timing = false;
std::vector<TimedRecord> g_records;
std::vector<cudaEvent_t> g_free_events;

cudaEvent_t take_event() {  // under g_timing_mu
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

class TimedSection {
 public:
  TimedSection(int kind, cudaStream_t s) : kind_(kind), s_(s) {
    {
      std::lock_guard<std::mutex> lk(g_timing_mu);
      if (!g_timing) return;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_timing_mu);
    a_ = take_event();
    b_ = take_event();
    if (!a_ || !b_) {
      if (a_) g_free_events.push_back(a_);
      if (b_) g_free_events.push_back(b_);
      a_ = b_ = nullptr;
      return;
    }
    l0_ = g_launches.load();
    cudaEventRecord(a_, s_);
  }
  ~TimedSection() {
    if (!a_) return;
    cudaEventRecord(b_, s_);
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_records.push_back({kind_, a_, b_, g_launches.load() - l0_});
  }
  TimedSection(const TimedSection&) = delete;
  TimedSection& operator=(const TimedSection&) = delete;

 private:
  int kind_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  int64_t l0_ = 0;
};

struct QueryWs {
  int32_t* counters;
  int32_t* seg_count;
  int32_t* seg_leaf;
  float* seg_t0;
  float* seg_t1;
  int32_t* queue[2];
  void* image;  // the streamed first-layer image (FP16/BF16 models)
  size_t bytes;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Counter block of a query workspace: per-wave counts [0, max_segs + 2), then
// at pq_base the persistent queue's counters, one 128-byte line each.
int32_t pq_base(int32_t max_segs) { return int32_t(align256(sizeof(int32_t) * size_t(max_segs + 2)) / 4); }
size_t counters_bytes(int32_t max_segs) { return size_t(pq_base(max_segs)) * 4 + 4 * 128; }

QueryWs carve_query(void* base, int64_t n, int32_t max_segs, size_t image = 0) {
  QueryWs w;
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += align256(bytes);
    return q;
  };
  w.counters = reinterpret_cast<int32_t*>(take(counters_bytes(max_segs)));
  w.seg_count = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * size_t(n)));
  w.seg_leaf = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * size_t(n) * size_t(max_segs)));
  w.seg_t0 = reinterpret_cast<float*>(take(sizeof(float) * size_t(n) * size_t(max_segs)));
  w.seg_t1 = reinterpret_cast<float*>(take(sizeof(float) * size_t(n) * size_t(max_segs)));
  // the two wave queues, or (persistent query) one ring of n 64-bit items
  w.queue[0] = reinterpret_cast<int32_t*>(take(2 * sizeof(int32_t) * size_t(n)));
  w.queue[1] = w.queue[0] ? w.queue[0] + n : nullptr;
  w.image = image ? take(image) : nullptr;
  w.bytes = off;
  return w;
}

// Items a partial persistent tile claims by default (nbvh_query_options.partial_items = 0).
#ifndef NBVH_PARTIAL_ITEMS
#define NBVH_PARTIAL_ITEMS 16
#endif
constexpr int32_t kPartialItems = NBVH_PARTIAL_ITEMS;

// The phase kernel's claims spread a short queue over every CTA: at most
// max(kSplitItems, queue / CTAs) items each, the rest of the tile lookahead
// rows (pq_full). Measured on 4,096 rays: 167 -> 153 us per FP16 query with
// 32 (156 with 8 or 16); the 16-asset frame 0.4 % faster. Large queues (at
// least 128 items per CTA) take full tiles as before.
constexpr int32_t kSplitItems = 32;

// Persistent evaluations beside other instances' (concurrent hybrid form):
// idle CTAs leave while the CTAs that stay, with this many spares, suffice.
#ifndef NBVH_YIELD_SPARES
#define NBVH_YIELD_SPARES 8
#endif
constexpr int kYieldSpares = NBVH_YIELD_SPARES;

PQueue pq_of(const QueryWs& w, int32_t max_segs, int64_t patience, int32_t partial_items, int64_t spin_limit,
             bool yield_idle) {
  int32_t* c = w.counters + pq_base(max_segs);
  PQueue q;
  q.head = reinterpret_cast<unsigned long long*>(c);
  q.reserved = reinterpret_cast<unsigned long long*>(c + 32);
  q.retired = reinterpret_cast<unsigned long long*>(c + 64);
  q.tiles = reinterpret_cast<unsigned int*>(c + 96);
  q.lookahead = reinterpret_cast<unsigned long long*>(c + 98);
  q.exited = reinterpret_cast<unsigned int*>(c + 100);
  q.yield_idle = yield_idle ? kYieldSpares + 1 : 0;
  q.patience = patience;
  q.partial_items = partial_items;
  q.spin_limit = spin_limit > 0 ? spin_limit : kPqSpinLimit;
  q.ring = reinterpret_cast<unsigned long long*>(w.queue[0]);
  q.qlen0 = w.counters;  // the traversal's queue length
  q.split = 0;
  return q;
}

// Adds a query's evaluated segments to *out: the per-wave counts, or the
// persistent queue's queued items plus its lookahead rows (statistics).
__global__ void segments_add_kernel(const int32_t* wave_counts, int32_t n_waves, const unsigned long long* reserved,
                                    const unsigned long long* lookahead, long long* out) {
  long long v = 0;
  for (int i = threadIdx.x; i < n_waves; i += 32) v += wave_counts[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) {
    if (reserved) v += (long long)(*reserved + *lookahead);
    atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)v);
  }
}

// Traversal (S1) then the evaluation (S2..S5) on the carved query workspace:
// one wave per segment slot (FP32 form) or one persistent launch (FP16/BF16).
// merge: the hit record holds the closest hit so far (hybrid hierarchy) and
// records the instance id with every improvement.
cudaError_t launch_query_stages(const nbvh_model_desc* desc, const GridParams& gp, const void* table,
                                const float* mlp, const nbvh_node* nodes, const nbvh_rays& rays, int32_t max_segs,
                                const nbvh_hits& out, const QueryWs& w, bool merge, int32_t* inst_out,
                                int32_t inst_id, const nbvh_query_options& o, cudaStream_t s,
                                const int32_t* list = nullptr, const int32_t* list_count = nullptr,
                                const float* init_t = nullptr, const int32_t* init_inst = nullptr) {
  TraverseOut to;
  std::memset(&to, 0, sizeof(to));
  to.seg_count = w.seg_count;
  to.seg_leaf = w.seg_leaf;
  to.seg_t0 = w.seg_t0;
  to.seg_t1 = w.seg_t1;
  to.max_segs = max_segs;
  to.queue0 = w.queue[0];
  to.qlen0 = w.counters;
  to.hits = out;
  to.merge = merge ? 1 : 0;
  to.reverse_inside = (desc->flags & NBVH_FLAG_REVERSE_INSIDE) ? 1 : 0;
  to.init_t = init_t;
  to.init_inst = init_inst;
  to.inst_id = inst_id;
  const bool persistent = desc->mlp_prec != NBVH_FP32 && o.schedule == NBVH_SCHEDULE_PERSISTENT;
  if (persistent) {
    to.queue0 = nullptr;
    to.ring0 = reinterpret_cast<unsigned long long*>(w.queue[0]);  // fills entries [0, qlen0): see PQueue
  }
  const int tb = o.traverse_block;
  cudaError_t e;
  {
    TimedSection ts(NBVH_KERNEL_TRAVERSE, s);
    if (list) {  // only the listed rays (grid-stride over the device-side count)
      const int64_t blocks = std::min<int64_t>((rays.n + 255) / 256, int64_t(sm_count()) * 8);
      traverse_list_kernel<<<unsigned(std::max<int64_t>(blocks, 1)), 256, 0, s>>>(nodes, ray_ptrs(rays), rays.n,
                                                                                   list, list_count, to);
    } else {
      traverse_kernel<<<unsigned((rays.n + tb - 1) / tb), tb, 0, s>>>(nodes, ray_ptrs(rays), rays.n, to);
    }
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  TimedSection ts(NBVH_KERNEL_EVAL, s);
  EvalArgs a = base_args(desc, gp, table, mlp, rays);
  a.n_rays = rays.n;
  a.seg_count = w.seg_count;
  a.seg_leaf = w.seg_leaf;
  a.seg_t0 = w.seg_t0;
  a.seg_t1 = w.seg_t1;
  a.hits = out;
  a.inst_out = inst_out;
  a.inst_id = inst_id;
  a.max_segs = max_segs;
  const bool ws = persistent && use_ws(desc, o);
  TcPlan plan;
  std::memset(&plan, 0, sizeof(plan));
  if (!ws) {
    e = prepare_eval(desc, a, o, w.image, &plan, s);
    if (e != cudaSuccess) return e;
  }
  if (persistent) {
    // one launch drains a queue of (slot, ray) items
    // the warp-specialised pipeline has no lookahead rows: its partial tiles take every item
    const int32_t partial = ws ? int32_t(kTcM) : (o.partial_items > 0 ? o.partial_items : kPartialItems);
    a.pq = pq_of(w, max_segs, o.patience_cycles, partial, o.wait_spins, init_t != nullptr);
    a.pq.split = ws ? 0 : kSplitItems;
    pq_init_kernel<<<1, 1, 0, s>>>(w.counters, a.pq, o.test_phantom_items);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // with split claims every CTA can take a share of a short queue
    const int64_t n_max = a.pq.split > 0 ? rays.n * (kTcM / std::max(1, std::min(a.pq.split, int(kTcM)))) : rays.n;
    e = ws ? launch_ws(desc, a, s) : launch_eval<1>(desc, a, n_max, plan, s);
  } else {
    for (int wv = 0; wv < max_segs; ++wv) {
      a.wave = wv;
      a.queue = w.queue[wv & 1];
      a.qlen = w.counters + wv;
      a.next_queue = w.queue[(wv + 1) & 1];
      a.next_qlen = w.counters + wv + 1;
      e = launch_eval<1>(desc, a, rays.n, plan, s);
      if (e != cudaSuccess) return e;
    }
  }
  if (e == cudaSuccess && o.segments_out) {
    segments_add_kernel<<<1, 32, 0, s>>>(w.counters, persistent ? 0 : max_segs, persistent ? a.pq.reserved : nullptr,
                                         persistent ? a.pq.lookahead : nullptr,
                                         reinterpret_cast<long long*>(o.segments_out));
    count_launches(1);
    e = cudaGetLastError();
  }
  return e;
}
}  // namespace
}  // namespace nbvh

using namespace nbvh;

extern "C" nbvh_status nbvh_traverse(const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays, int32_t max_segs,
                                     int32_t* seg_count, int32_t* seg_leaf, float* seg_t0, float* seg_t1,
                                     void* stream) {
  if (!nodes || n_nodes < 1 || !rays_valid(rays) || max_segs < 1) return NBVH_ERR_INVALID_ARG;
  if (rays.n == 0) return NBVH_OK;
  if (!seg_count || !seg_leaf || !seg_t0 || !seg_t1) return NBVH_ERR_INVALID_ARG;
  if (rays.n > (int64_t(1) << 31) - 1) return NBVH_ERR_INVALID_ARG;
  TraverseOut out;
  std::memset(&out, 0, sizeof(out));
  out.seg_count = seg_count;
  out.seg_leaf = seg_leaf;
  out.seg_t0 = seg_t0;
  out.seg_t1 = seg_t1;
  out.max_segs = max_segs;
  const unsigned grid = unsigned((rays.n + 127) / 128);
  traverse_kernel<<<grid, 128, 0, as_stream(stream)>>>(nodes, ray_ptrs(rays), rays.n, out);
  count_launches(1);
  return status_of(cudaGetLastError());
}

extern "C" nbvh_status nbvh_encode(const nbvh_model_desc* desc, const void* table, nbvh_rays rays,
                                   const int32_t* seg_ray, const float* t0, const float* t1, int64_t n_seg,
                                   float* feat, void* stream) {
  if (!nbvh_host::desc_valid(desc) || !table || !rays_valid(rays) || n_seg < 0) return NBVH_ERR_INVALID_ARG;
  if (n_seg == 0) return NBVH_OK;
  if (!seg_ray || !t0 || !t1 || !feat) return NBVH_ERR_INVALID_ARG;
  GridParams gp;
  if (!make_grid(desc, gp)) return NBVH_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  cudaError_t e;
  switch (desc->table_prec) {
    case NBVH_FP32: e = launch_encode_t<float>(desc->n_features, gp, table, ray_ptrs(rays), seg_ray, t0, t1, n_seg, feat, s); break;
    case NBVH_FP16: e = launch_encode_t<__half>(desc->n_features, gp, table, ray_ptrs(rays), seg_ray, t0, t1, n_seg, feat, s); break;
    default: e = launch_encode_t<__nv_bfloat16>(desc->n_features, gp, table, ray_ptrs(rays), seg_ray, t0, t1, n_seg, feat, s); break;
  }
  return status_of(e);
}

extern "C" nbvh_status nbvh_query_options_default(nbvh_query_options* opt) {
  if (!opt) return NBVH_ERR_INVALID_ARG;
  *opt = default_options();
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_eval_plan(const nbvh_model_desc* desc, const nbvh_query_options* opt,
                                      int32_t* threads, int32_t* w1_streamed, int32_t* smem_bytes,
                                      int32_t* tmem_cols, int32_t* pipeline) {
  if (!nbvh_host::desc_valid(desc) || !threads || !w1_streamed || !smem_bytes || !tmem_cols || !pipeline)
    return NBVH_ERR_INVALID_ARG;
  const nbvh_query_options o = opt ? *opt : default_options();
  if (!options_valid(o)) return NBVH_ERR_INVALID_ARG;
  if (!eval_stageable(desc, o)) return NBVH_ERR_UNSUPPORTED;
  if (desc->mlp_prec == NBVH_FP32) {
    const int LF = desc->n_levels * desc->n_features;
    const int cs = plain_chunk_samples(desc->n_samples, LF, desc->width, desc->n_hidden, desc->n_out);
    *threads = kPlainThreads;
    *w1_streamed = cs > 0 ? 1 : 0;
    *smem_bytes = int32_t(plain_smem_bytes((cs > 0 ? cs : desc->n_samples) * LF, desc->width, desc->n_hidden,
                                           desc->n_out));
    *tmem_cols = 0;
    *pipeline = NBVH_PIPELINE_PHASES;
    return NBVH_OK;
  }
  if (use_ws(desc, o)) {
    const WsLayout L = ws_layout(desc->n_levels, desc->n_features, desc->n_samples, desc->width, desc->n_hidden);
    *threads = kWsThreads;
    *w1_streamed = 0;
    *smem_bytes = int32_t(L.total);
    *tmem_cols = 512;
    *pipeline = NBVH_PIPELINE_WARP_SPECIALISED;
    return NBVH_OK;
  }
  const TcPlan pl = tc_plan(desc, o.eval_threads, o.w1_mode);
  *threads = pl.threads;
  *w1_streamed = pl.stream ? 1 : 0;
  *smem_bytes = int32_t(pl.smem);
  *tmem_cols = int32_t(pl.ncols);
  *pipeline = NBVH_PIPELINE_PHASES;
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_eval_workspace_size(const nbvh_model_desc* desc, size_t* bytes) {
  if (!nbvh_host::desc_valid(desc) || !bytes) return NBVH_ERR_INVALID_ARG;
  *bytes = image_bytes(desc);
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_eval_segments(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                          nbvh_rays rays, const int32_t* seg_ray, const float* t0,
                                          const float* t1, int64_t n_seg, float* out,
                                          const nbvh_query_options* opt, void* workspace, size_t ws_bytes,
                                          void* stream) {
  if (!nbvh_host::desc_valid(desc) || !table || !mlp || !rays_valid(rays) || n_seg < 0)
    return NBVH_ERR_INVALID_ARG;
  const nbvh_query_options o = opt ? *opt : default_options();
  if (!options_valid(o)) return NBVH_ERR_INVALID_ARG;
  if (n_seg == 0) return NBVH_OK;
  if (!seg_ray || !t0 || !t1 || !out) return NBVH_ERR_INVALID_ARG;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return NBVH_ERR_INVALID_ARG;
  if (ws_bytes < image_bytes(desc) || (image_bytes(desc) > 0 && !workspace)) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  GridParams gp;
  if (!make_grid(desc, gp)) return NBVH_ERR_INVALID_ARG;
  if (!eval_stageable(desc, o, false)) return NBVH_ERR_UNSUPPORTED;
  EvalArgs a = base_args(desc, gp, table, mlp, rays);
  a.seg_ray = seg_ray;
  a.list_t0 = t0;
  a.list_t1 = t1;
  a.n_items = n_seg;
  a.out = out;
  cudaStream_t s = as_stream(stream);
  TcPlan plan;
  cudaError_t e = prepare_eval(desc, a, o, workspace, &plan, s);
  if (e == cudaSuccess) e = launch_eval<0>(desc, a, n_seg, plan, s);
  return status_of(e);
}

extern "C" nbvh_status nbvh_query_workspace_size(const nbvh_model_desc* desc, int64_t n_rays, int32_t max_segs,
                                                 size_t* bytes) {
  if (!nbvh_host::desc_valid(desc) || n_rays < 0 || max_segs < 1 || !bytes) return NBVH_ERR_INVALID_ARG;
  *bytes = carve_query(nullptr, n_rays, max_segs, image_bytes(desc)).bytes;
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_query_rays(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                       const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays, int32_t max_segs,
                                       nbvh_hits out, void* workspace, size_t ws_bytes, void* stream) {
  return nbvh_query_rays_opt(desc, table, mlp, nodes, n_nodes, rays, max_segs, out, workspace, ws_bytes, nullptr,
                             stream);
}

extern "C" nbvh_status nbvh_query_rays_opt(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                           const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays,
                                           int32_t max_segs, nbvh_hits out, void* workspace, size_t ws_bytes,
                                           const nbvh_query_options* opt, void* stream) {
  if (!nbvh_host::desc_valid(desc) || !table || !mlp || !nodes || n_nodes < 1 || !rays_valid(rays) ||
      max_segs < 1 || max_segs > 4096)
    return NBVH_ERR_INVALID_ARG;
  const nbvh_query_options o = opt ? *opt : default_options();
  if (!options_valid(o)) return NBVH_ERR_INVALID_ARG;
  if (rays.n == 0) return NBVH_OK;
  if (rays.n > (int64_t(1) << 31) - 1) return NBVH_ERR_INVALID_ARG;
  if (!out.hit || !out.t || !out.nx || !out.ny || !out.nz || !out.leaf || !workspace) return NBVH_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return NBVH_ERR_INVALID_ARG;
  QueryWs w = carve_query(workspace, rays.n, max_segs, image_bytes(desc));
  if (ws_bytes < w.bytes) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  GridParams gp;
  if (!make_grid(desc, gp)) return NBVH_ERR_INVALID_ARG;
  if (!eval_stageable(desc, o)) return NBVH_ERR_UNSUPPORTED;  // before anything is enqueued
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMemsetAsync(w.counters, 0, counters_bytes(max_segs), s);
  if (e != cudaSuccess) return NBVH_ERR_CUDA;
  e = launch_query_stages(desc, gp, table, mlp, nodes, rays, max_segs, out, w, false, nullptr, 0, o, s);
  return status_of(e);
}

extern "C" nbvh_status nbvh_query_stats(const void* workspace, int64_t n_rays, int32_t max_segs, int64_t* segments,
                                       int32_t* waves, void* stream) {
  if (!workspace || n_rays < 0 || max_segs < 1 || max_segs > 4096 || !segments || !waves)
    return NBVH_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return NBVH_ERR_INVALID_ARG;
  std::vector<int32_t> c(counters_bytes(max_segs) / 4);
  cudaStream_t s = as_stream(stream);
  if (cudaMemcpyAsync(c.data(), workspace, sizeof(int32_t) * c.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return NBVH_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return NBVH_ERR_CUDA;
  // persistent query (tensor-core form): one launch, items ever queued plus
  // the segments lookahead rows evaluated without queueing them
  uint64_t reserved = 0, lookahead = 0;
  std::memcpy(&reserved, c.data() + pq_base(max_segs) + 32, sizeof(reserved));
  std::memcpy(&lookahead, c.data() + pq_base(max_segs) + 98, sizeof(lookahead));
  if (reserved > 0) {
    *segments = int64_t(reserved + lookahead);
    *waves = 1;
    return NBVH_OK;
  }
  int64_t tot = 0;
  int32_t w = 0;
  for (int i = 0; i < max_segs; ++i) {
    tot += c[i];
    if (c[i] > 0) w = i + 1;
  }
  *segments = tot;
  *waves = w;
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_set_timing(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  g_timing = enable != 0;
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_get_kernel_times(double* ms, int64_t* sections, int64_t* launches, int32_t n_kinds) {
  if (!ms || !sections || !launches || n_kinds < 1) return NBVH_ERR_INVALID_ARG;
  std::vector<TimedRecord> rec;
  {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    rec.swap(g_records);
  }
  for (int32_t k = 0; k < n_kinds; ++k) {
    ms[k] = 0.0;
    sections[k] = 0;
    launches[k] = 0;
  }
  nbvh_status st = NBVH_OK;
  for (auto& r : rec) {
    float t = 0.0f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
      st = NBVH_ERR_CUDA;
    if (r.kind < n_kinds) {
      ms[r.kind] += t;
      sections[r.kind] += 1;
      launches[r.kind] += r.launches;
    }
  }
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (auto& r : rec) {
    g_free_events.push_back(r.a);
    g_free_events.push_back(r.b);
  }
  return st;
}

extern "C" int64_t nbvh_launch_count(void) { return g_launches.load(); }

extern "C" nbvh_status nbvh_bounce_rays(nbvh_rays rays, nbvh_hits hits, uint64_t seed, nbvh_rays_out out,
                                        void* stream) {
  if (!rays_valid(rays) || out.n != rays.n) return NBVH_ERR_INVALID_ARG;
  if (rays.n == 0) return NBVH_OK;
  if (!hits.hit || !hits.t || !hits.nx || !hits.ny || !hits.nz || !out.ox || !out.oy || !out.oz || !out.dx ||
      !out.dy || !out.dz || !out.tmin || !out.tmax)
    return NBVH_ERR_INVALID_ARG;
  RayOut o{out.ox, out.oy, out.oz, out.dx, out.dy, out.dz, out.tmin, out.tmax};
  TimedSection ts(NBVH_KERNEL_BOUNCE, as_stream(stream));
  bounce_kernel<<<unsigned((rays.n + 255) / 256), 256, 0, as_stream(stream)>>>(
      ray_ptrs(rays), hits, rays.n, uint32_t(seed & 0xffffffffu), uint32_t(seed >> 32), o);
  count_launches(1);
  return status_of(cudaGetLastError());
}

// ---------------------------------------------------------------- hybrid hierarchy (S9)
namespace nbvh {
namespace {
bool tri_blas_valid(const nbvh_tri_blas* b) {
  return b && b->nodes && b->n_nodes >= 1 && b->tris && b->leaf_range && b->tri_id;
}
bool hits_valid(const nbvh_hits& h) {
  return h.hit && h.t && h.nx && h.ny && h.nz && h.leaf && (!h.ar || (h.ag && h.ab));
}

TriBlasArgs tri_args(const nbvh_tri_blas& b, const nbvh_rays& rays, const nbvh_hits& h, int32_t* inst_out,
                     int32_t inst_id, int32_t merge) {
  TriBlasArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nodes = b.nodes;
  a.tris = b.tris;
  a.leaf_range = b.leaf_range;
  a.tri_id = b.tri_id;
  a.albedo = b.albedo;
  a.rays = ray_ptrs(rays);
  a.n = rays.n;
  a.hits = h;
  a.inst_out = inst_out;
  a.inst_id = inst_id;
  a.merge = merge;
  return a;
}

size_t image_bytes(const nbvh_model_desc* d);

// The largest first-layer image of the neural instances (the passes run one
// after the other on the caller's stream and share the region).
size_t hybrid_image_bytes(const nbvh_instance* inst, int32_t n_inst) {
  size_t m = 0;
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].kind == NBVH_BLAS_NEURAL) m = std::max(m, image_bytes(&inst[i].desc));
  return m;
}

int32_t hybrid_max_segs(const nbvh_instance* inst, int32_t n_inst) {
  int32_t m = 0;
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].kind == NBVH_BLAS_NEURAL) m = std::max(m, inst[i].max_segs);
  return m;
}

bool instances_valid(const nbvh_instance* inst, int32_t n_inst) {
  if (!inst || n_inst < 1 || n_inst > 64) return false;
  for (int i = 0; i < n_inst; ++i) {
    const nbvh_instance& x = inst[i];
    if (x.kind == NBVH_BLAS_TRIANGLES) {
      if (!tri_blas_valid(&x.tri)) return false;
    } else if (x.kind == NBVH_BLAS_NEURAL) {
      if (!nbvh_host::desc_valid(&x.desc) || !x.table || !x.mlp || !x.nodes || x.n_nodes < 1 ||
          x.max_segs < 1 || x.max_segs > 4096)
        return false;
    } else {
      return false;
    }
  }
  return true;
}
}  // namespace
}  // namespace nbvh

extern "C" nbvh_status nbvh_trace_triangles(const nbvh_tri_blas* blas, nbvh_rays rays, nbvh_hits hits,
                                            void* stream) {
  if (!tri_blas_valid(blas) || !rays_valid(rays)) return NBVH_ERR_INVALID_ARG;
  if (rays.n == 0) return NBVH_OK;
  if (!hits_valid(hits) || rays.n > (int64_t(1) << 31) - 1) return NBVH_ERR_INVALID_ARG;
  const TriBlasArgs a = tri_args(*blas, rays, hits, nullptr, 0, 0);
  TimedSection ts(NBVH_KERNEL_TRI_TRACE, as_stream(stream));
  tri_trace_kernel<<<unsigned((rays.n + 127) / 128), 128, 0, as_stream(stream)>>>(a);
  count_launches(1);
  return status_of(cudaGetLastError());
}

namespace nbvh {
namespace {

// Hybrid workspace: kHybridStreams query workspaces sized for the deepest
// neural instance (the sequential form uses the first), one ray list per
// neural instance (n_rays entries) and their counts, then for the concurrent
// form a per-ray instance mask and one staging hit record per neural
// instance (albedo arrays when an instance has the albedo head).
// At most two: on the 16-asset scene (3840x2160, 4 bounces) one stream takes
// 117 ms per frame, two 101, three and four 105 and 107 (the kernels contend
// for SMs and L2).
constexpr int kHybridStreams = 2;

struct HybridWs {
  QueryWs q[kHybridStreams];
  int32_t* lists;
  int32_t* counts;
  unsigned long long* mask;
  nbvh_hits stage;  // slot k of ray r at k * n + r
  size_t bytes;
};

bool hybrid_albedo(const nbvh_instance* inst, int32_t n_inst) {
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].kind == NBVH_BLAS_NEURAL && inst[i].desc.n_out >= 8) return true;
  return false;
}

HybridWs carve_hybrid(void* base, const nbvh_instance* inst, int32_t n_inst, int64_t n) {
  HybridWs h;
  std::memset(&h, 0, sizeof(h));
  int32_t n_neural = 0;
  for (int i = 0; i < n_inst; ++i) n_neural += inst[i].kind == NBVH_BLAS_NEURAL;
  const int32_t ms = std::max(hybrid_max_segs(inst, n_inst), 1);
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += align256(bytes);
    return q;
  };
  for (int j = 0; j < kHybridStreams; ++j) {
    h.q[j] = carve_query(p ? p + off : nullptr, n, ms, hybrid_image_bytes(inst, n_inst));
    off += h.q[j].bytes;
  }
  const size_t N = size_t(n), K = size_t(n_neural);
  h.lists = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * N * K));
  h.counts = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kMaxInstances));
  h.mask = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * N));
  h.stage.hit = reinterpret_cast<uint8_t*>(take(N * K));
  h.stage.t = reinterpret_cast<float*>(take(4 * N * K));
  h.stage.nx = reinterpret_cast<float*>(take(4 * N * K));
  h.stage.ny = reinterpret_cast<float*>(take(4 * N * K));
  h.stage.nz = reinterpret_cast<float*>(take(4 * N * K));
  h.stage.leaf = reinterpret_cast<int32_t*>(take(4 * N * K));
  if (hybrid_albedo(inst, n_inst)) {
    h.stage.ar = reinterpret_cast<float*>(take(4 * N * K));
    h.stage.ag = reinterpret_cast<float*>(take(4 * N * K));
    h.stage.ab = reinterpret_cast<float*>(take(4 * N * K));
  }
  h.bytes = off;
  return h;
}

// Staging record of slot k (k * n entries into every array).
nbvh_hits stage_slot(const nbvh_hits& st, int32_t k, int64_t n) {
  const size_t o = size_t(k) * size_t(n);
  nbvh_hits h = st;
  h.hit = st.hit + o;
  h.t = st.t + o;
  h.nx = st.nx + o;
  h.ny = st.ny + o;
  h.nz = st.nz + o;
  h.leaf = st.leaf + o;
  if (st.ar) {
    h.ar = st.ar + o;
    h.ag = st.ag + o;
    h.ab = st.ab + o;
  }
  return h;
}

// Per device: the side streams of the concurrent hybrid form and its fork /
// join events, created on first use and kept; one host thread at a time
// enqueues on them (their events would interleave otherwise).
struct SideStreams {
  cudaStream_t s[kHybridStreams];
  cudaEvent_t fork;
  cudaEvent_t join[kHybridStreams];
  std::mutex mu;
};

SideStreams* side_streams() {
  static std::mutex mu;
  static std::vector<std::unique_ptr<SideStreams>> per_dev;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (per_dev.size() <= size_t(dev)) per_dev.resize(size_t(dev) + 1);
  if (!per_dev[size_t(dev)]) {
    std::unique_ptr<SideStreams> x(new SideStreams());
    bool ok = cudaEventCreateWithFlags(&x->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int j = 0; j < kHybridStreams && ok; ++j)
      ok = cudaStreamCreateWithFlags(&x->s[j], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&x->join[j], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return nullptr;
    per_dev[size_t(dev)] = std::move(x);
  }
  return per_dev[size_t(dev)].get();
}

}  // namespace
}  // namespace nbvh

extern "C" nbvh_status nbvh_hybrid_workspace_size(const nbvh_instance* inst, int32_t n_inst, int64_t n_rays,
                                                  size_t* bytes) {
  if (!instances_valid(inst, n_inst) || n_rays < 0 || !bytes) return NBVH_ERR_INVALID_ARG;
  *bytes = carve_hybrid(nullptr, inst, n_inst, n_rays).bytes;
  return NBVH_OK;
}

namespace nbvh {
namespace {

// The top-level cull: for the neural instances from `from` on, the list of
// rays whose interval meets their root boxes before the record so far (the
// record only shrinks, so each list stays a superset of the rays the
// instance's traversal can give a segment); slot k = the k-th of them.
cudaError_t hybrid_cull(const nbvh_instance* inst, int32_t n_inst, int32_t from, const nbvh_rays& rays,
                        const nbvh_hits& out, const HybridWs& hw, bool with_mask, std::vector<int32_t>& cull_slot,
                        cudaStream_t s) {
  CullArgs c;
  std::memset(&c, 0, sizeof(c));
  int32_t k = 0;
  for (int j = from; j < n_inst; ++j) {
    if (inst[j].kind != NBVH_BLAS_NEURAL) continue;
    cull_slot[size_t(j)] = k;
    c.root[k] = inst[j].nodes;
    c.list[k] = hw.lists + size_t(k) * size_t(rays.n);
    ++k;
  }
  c.count = hw.counts;
  c.n_inst = k;
  c.mask = with_mask ? hw.mask : nullptr;
  TimedSection ts(NBVH_KERNEL_TLAS_CULL, s);
  cudaError_t e = cudaMemsetAsync(hw.counts, 0, sizeof(int32_t) * kMaxInstances, s);
  if (e != cudaSuccess) return e;
  tlas_cull_kernel<<<unsigned((rays.n + 255) / 256), 256, 0, s>>>(ray_ptrs(rays), rays.n, out.t, c);
  count_launches(1);
  return cudaGetLastError();
}

// One neural instance's traversal and evaluation over its ray list, on
// stream s with query workspace w: merged into `rec` (with the instance id
// into out_inst), or staged (init_t set: rec is its staging record).
cudaError_t hybrid_neural(const nbvh_instance& x, int32_t i, const GridParams& gp, const nbvh_rays& rays,
                          const nbvh_hits& rec, int32_t* out_inst, const QueryWs& w, const HybridWs& hw, int32_t k,
                          const nbvh_query_options& o, const float* init_t, const int32_t* init_inst,
                          cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(w.counters, 0, counters_bytes(x.max_segs), s);
  if (e != cudaSuccess) return e;
  nbvh_query_options oi = o;
  if (o.segments_out) oi.segments_out = o.segments_out + i;
  // beside the other stream's instances, partial tiles take the whole queue
  // by default (measured: 111 vs 114 ms per 16-asset frame with 16 items)
  if (init_t && o.partial_items == 0) oi.partial_items = int32_t(kTcM);
  return launch_query_stages(&x.desc, gp, x.table, x.mlp, x.nodes, rays, x.max_segs, rec, w, true, out_inst, i, oi,
                             s, hw.lists + size_t(k) * size_t(rays.n), hw.counts + k, init_t, init_inst);
}

}  // namespace
}  // namespace nbvh

extern "C" nbvh_status nbvh_hybrid_trace(const nbvh_instance* inst, int32_t n_inst, nbvh_rays rays,
                                         nbvh_hits out, int32_t* out_inst, void* workspace, size_t ws_bytes,
                                         const nbvh_query_options* opt, void* stream) {
  if (!instances_valid(inst, n_inst) || !rays_valid(rays)) return NBVH_ERR_INVALID_ARG;
  const nbvh_query_options o = opt ? *opt : default_options();
  if (!options_valid(o)) return NBVH_ERR_INVALID_ARG;
  if (rays.n == 0) return NBVH_OK;
  if (!hits_valid(out) || !out_inst || !workspace || rays.n > (int64_t(1) << 31) - 1) return NBVH_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return NBVH_ERR_INVALID_ARG;
  const HybridWs hw = carve_hybrid(workspace, inst, n_inst, rays.n);
  if (ws_bytes < hw.bytes) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  std::vector<GridParams> gps(static_cast<size_t>(n_inst));
  int32_t n_neural = 0;
  for (int i = 0; i < n_inst; ++i) {
    if (inst[i].kind != NBVH_BLAS_NEURAL) continue;
    ++n_neural;
    if (!make_grid(&inst[i].desc, gps[size_t(i)])) return NBVH_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_inst; ++i)  // before anything is enqueued
    if (inst[i].kind == NBVH_BLAS_NEURAL && !eval_stageable(&inst[i].desc, o)) return NBVH_ERR_UNSUPPORTED;
  const int32_t streams = std::min<int32_t>(o.instance_streams == 0 ? kHybridStreams : o.instance_streams,
                                            kHybridStreams);
  const bool concurrent = streams > 1 && n_neural > 1;
  SideStreams* side = concurrent ? side_streams() : nullptr;
  if (concurrent && !side) return NBVH_ERR_CUDA;
  cudaStream_t s = as_stream(stream);
  cudaError_t e;
  {
    TimedSection ts(NBVH_KERNEL_OTHER, s);
    hits_clear_kernel<<<unsigned((rays.n + 255) / 256), 256, 0, s>>>(out, out_inst, rays.n);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return NBVH_ERR_CUDA;
  std::vector<int32_t> cull_slot(static_cast<size_t>(n_inst), -1);
  auto tri = [&](int i) {
    const TriBlasArgs a = tri_args(inst[i].tri, rays, out, out_inst, i, 1);
    TimedSection ts(NBVH_KERNEL_TRI_TRACE, s);
    tri_trace_kernel<<<unsigned((rays.n + 127) / 128), 128, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
  };
  if (!concurrent) {
    // one instance after another in index order, each merged into the record
    int32_t culled_from = -1;  // first instance covered by the top-level cull
    for (int i = 0; i < n_inst; ++i) {
      const nbvh_instance& x = inst[i];
      if (x.kind == NBVH_BLAS_TRIANGLES) {
        e = tri(i);
        if (e != cudaSuccess) return status_of(e);
        continue;
      }
      if (culled_from < 0) {
        e = hybrid_cull(inst, n_inst, i, rays, out, hw, false, cull_slot, s);
        if (e != cudaSuccess) return NBVH_ERR_CUDA;
        culled_from = i;
      }
      e = hybrid_neural(x, i, gps[size_t(i)], rays, out, out_inst, hw.q[0], hw, cull_slot[size_t(i)], o, nullptr,
                        nullptr, s);
      if (e != cudaSuccess) return status_of(e);
    }
    return NBVH_OK;
  }
  // Concurrent form: the triangle instances first (merged in index order),
  // then every neural instance on one of the side streams, each into its own
  // staging record started at the triangles' answer, then a per-ray merge in
  // instance order. A neural instance's own closest hit does not depend on
  // where its search starts (only segments that cannot win are skipped), so
  // the record equals the sequential form's bit for bit. An instance's idle
  // persistent CTAs leave early, so the instances' evaluations overlap.
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].kind == NBVH_BLAS_TRIANGLES) {
      e = tri(i);
      if (e != cudaSuccess) return status_of(e);
    }
  e = hybrid_cull(inst, n_inst, 0, rays, out, hw, true, cull_slot, s);
  if (e != cudaSuccess) return NBVH_ERR_CUDA;
  std::lock_guard<std::mutex> lk(side->mu);
  if (cudaEventRecord(side->fork, s) != cudaSuccess) return NBVH_ERR_CUDA;
  for (int j = 0; j < streams; ++j)
    if (cudaStreamWaitEvent(side->s[j], side->fork, 0) != cudaSuccess) return NBVH_ERR_CUDA;
  StageArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  sa.st = hw.stage;
  sa.n = rays.n;
  nbvh_status st = NBVH_OK;
  for (int i = 0; i < n_inst && st == NBVH_OK; ++i) {
    if (inst[i].kind != NBVH_BLAS_NEURAL) continue;
    const int32_t k = cull_slot[size_t(i)];
    sa.inst_of[k] = i;
    const int j = k % streams;
    e = hybrid_neural(inst[i], i, gps[size_t(i)], rays, stage_slot(hw.stage, k, rays.n), nullptr, hw.q[j], hw, k, o,
                      out.t, out_inst, side->s[j]);
    if (e != cudaSuccess) st = status_of(e);
  }
  // join (also after a failure: the side streams must not outlive the caller's stream order)
  for (int j = 0; j < streams; ++j)
    if (cudaEventRecord(side->join[j], side->s[j]) != cudaSuccess ||
        cudaStreamWaitEvent(s, side->join[j], 0) != cudaSuccess)
      st = NBVH_ERR_CUDA;
  if (st != NBVH_OK) return st;
  TimedSection ts(NBVH_KERNEL_OTHER, s);
  hybrid_merge_kernel<<<unsigned((rays.n + 255) / 256), 256, 0, s>>>(out, out_inst, hw.mask, rays.n, sa);
  count_launches(1);
  return status_of(cudaGetLastError());
}

// ---------------------------------------------------------------- autotuner (S6)
extern "C" nbvh_status nbvh_autotune_query(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                           const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays,
                                           int32_t max_segs, nbvh_hits out, void* workspace, size_t ws_bytes,
                                           int32_t reps, nbvh_tune_result* best, nbvh_tune_result* all,
                                           int32_t all_cap, int32_t* n_all, void* stream) {
  if (!nbvh_host::desc_valid(desc) || !table || !mlp || !nodes || n_nodes < 1 || !rays_valid(rays) ||
      rays.n < 1 || max_segs < 1 || max_segs > 4096 || !hits_valid(out) || !workspace || reps < 1 ||
      reps > 100 || !best || (all_cap > 0 && !all) || all_cap < 0 || !n_all)
    return NBVH_ERR_INVALID_ARG;
  size_t need = 0;
  if (nbvh_query_workspace_size(desc, rays.n, max_segs, &need) != NBVH_OK) return NBVH_ERR_INVALID_ARG;
  if (ws_bytes < need) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t s = as_stream(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return NBVH_ERR_CUDA;
  }
  // one candidate: warm-up, then the median of reps timed queries
  auto time_it = [&](nbvh_tune_result& r) -> nbvh_status {
    std::vector<float> ms;
    for (int i = 0; i <= reps; ++i) {
      if (cudaEventRecord(e0, s) != cudaSuccess) return NBVH_ERR_CUDA;
      const nbvh_status st = nbvh_query_rays_opt(desc, table, mlp, nodes, n_nodes, rays, max_segs, out, workspace,
                                                 ws_bytes, &r.opt, stream);
      if (st != NBVH_OK) return st;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return NBVH_ERR_CUDA;
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return NBVH_ERR_CUDA;
      if (i > 0) ms.push_back(t);
    }
    std::sort(ms.begin(), ms.end());
    r.ms = ms[ms.size() / 2];
    return NBVH_OK;
  };
  std::vector<nbvh_tune_result> cand;
  nbvh_status st = NBVH_OK;
  nbvh_tune_result b;
  b.opt = default_options();
  b.ms = 0.0f;
  bool have = false;
  // times c (skipping shapes the kernels cannot stage) and keeps the faster
  auto consider = [&](nbvh_tune_result c) {
    if (st != NBVH_OK || !eval_stageable(desc, c.opt)) return;
    if ((st = time_it(c)) != NBVH_OK) return;
    cand.push_back(c);
    if (!have || c.ms < b.ms) {
      b = c;
      have = true;
    }
  };
  const bool tc = desc->mlp_prec != NBVH_FP32;
  {  // stage 1: schedule
    nbvh_tune_result c;
    c.opt = default_options();
    c.ms = 0.0f;
    c.opt.schedule = NBVH_SCHEDULE_WAVES;
    c.opt.patience_cycles = 0;
    consider(c);
    if (tc)
      for (int64_t p : {int64_t(0), int64_t(1000), int64_t(4000), int64_t(16000), int64_t(64000)}) {
        c.opt.schedule = NBVH_SCHEDULE_PERSISTENT;
        c.opt.patience_cycles = p;
        consider(c);
      }
  }
  if (tc && have) {  // stage 2: pipeline, evaluation CTA shape and first-layer placement
    const nbvh_tune_result base = b;
    const bool pers = base.opt.schedule == NBVH_SCHEDULE_PERSISTENT;
    const bool base_ws = use_ws(desc, base.opt);
    const TcPlan cur = tc_plan(desc, base.opt.eval_threads, base.opt.w1_mode);
    if (pers && !base_ws && ws_supported(desc)) {
      nbvh_tune_result c = base;
      c.opt.eval_pipeline = NBVH_PIPELINE_WARP_SPECIALISED;
      consider(c);
    }
    for (int32_t th : {256, 512})
      for (int32_t wm : {NBVH_W1_RESIDENT, NBVH_W1_STREAMED}) {
        if (!base_ws && th == cur.threads && (wm == NBVH_W1_STREAMED) == cur.stream) continue;  // timed in stage 1
        nbvh_tune_result c = base;
        c.opt.eval_pipeline = NBVH_PIPELINE_PHASES;
        c.opt.eval_threads = th;
        c.opt.w1_mode = wm;
        consider(c);
      }
  }
  // the fastest persistent phase-kernel candidate so far (stage 3 starts
  // from it even when waves lead: its partial tiles may change the order)
  bool have_pers = false;
  nbvh_tune_result best_pers;
  std::memset(&best_pers, 0, sizeof(best_pers));
  for (const nbvh_tune_result& c : cand)
    if (c.opt.schedule == NBVH_SCHEDULE_PERSISTENT && !use_ws(desc, c.opt) && (!have_pers || c.ms < best_pers.ms)) {
      best_pers = c;
      have_pers = true;
    }
  if (tc && have_pers) {
    // stage 3: items per partial tile (the rest of the tile: lookahead rows)
    const nbvh_tune_result base = best_pers;
    for (int32_t pi : {4, 8, 32, 128}) {
      nbvh_tune_result c = base;
      c.opt.partial_items = pi;
      consider(c);
    }
  }
  if (have) {  // stage 4: traversal CTA size
    const nbvh_tune_result base = b;
    for (int32_t tb : {64, 256}) {
      nbvh_tune_result c = base;
      c.opt.traverse_block = tb;
      consider(c);
    }
  }
  if (st == NBVH_OK && !have) st = NBVH_ERR_UNSUPPORTED;
  if (st == NBVH_OK) *best = b;
  const int32_t k = std::min<int32_t>(all_cap, int32_t(cand.size()));
  for (int32_t i = 0; i < k; ++i) all[i] = cand[size_t(i)];
  *n_all = int32_t(cand.size());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

// ---------------------------------------------------------------- measurement utility
extern "C" nbvh_status nbvh_probe_l2_gather(const void* table, int64_t n_entries, uint32_t* sink,
                                            double* gsectors_per_s, void* stream) {
  if (!table || !sink || !gsectors_per_s || n_entries < 1024 || n_entries > (int64_t(1) << 31) ||
      (n_entries & (n_entries - 1)) != 0)
    return NBVH_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const uint32_t mask = uint32_t(n_entries - 1);
  const int blocks = sm_count(), threads = 1024, iters = 100;
  const uint32_t* tab = static_cast<const uint32_t*>(table);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return NBVH_ERR_CUDA;
  }
  nbvh_status st = NBVH_OK;
  float best = 0.0f;
  for (int rep = 0; rep < 4 && st == NBVH_OK; ++rep) {  // the first launch warms the table into L2
    cudaEventRecord(e0, s);
    probe_gather_kernel<<<blocks, threads, 0, s>>>(tab, mask, iters, sink);
    count_launches(1);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      st = NBVH_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NBVH_OK) return st;
  const double loads = double(blocks) * threads * iters * kProbeLoads;
  *gsectors_per_s = loads / (double(best) * 1e-3) / 1e9;
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_probe_l2_reduce(float* grad, int64_t n_entries, double* gops_per_s, void* stream) {
  if (!grad || !gops_per_s || n_entries < 1024 || n_entries > (int64_t(1) << 30) ||
      (n_entries & (n_entries - 1)) != 0 || (reinterpret_cast<uintptr_t>(grad) & 7) != 0)
    return NBVH_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const uint32_t mask = uint32_t(n_entries - 1);
  const int blocks = sm_count(), threads = 1024, iters = 50;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return NBVH_ERR_CUDA;
  }
  nbvh_status st = NBVH_OK;
  float best = 0.0f;
  for (int rep = 0; rep < 4 && st == NBVH_OK; ++rep) {  // the first launch brings the buffer into L2
    cudaEventRecord(e0, s);
    probe_reduce_kernel<<<blocks, threads, 0, s>>>(reinterpret_cast<float2*>(grad), mask, iters);
    count_launches(1);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      st = NBVH_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NBVH_OK) return st;
  const double ops = double(blocks) * threads * iters * kProbeLoads;
  *gops_per_s = ops / (double(best) * 1e-3) / 1e9;
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_get_device_status(void* stream) {
  if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return NBVH_ERR_CUDA;
  std::vector<StatusReader> readers;
  {
    std::lock_guard<std::mutex> lk(status_mu());
    readers = status_readers();
  }
  int first = 0;
  for (StatusReader r : readers) {  // every unit's word is read and cleared
    int v = 0;
    if (r(&v) != cudaSuccess) return NBVH_ERR_CUDA;
    if (first == 0) first = v;
  }
  return static_cast<nbvh_status>(first);
}

// ---------------------------------------------------------------- built-in scratch
// Scratch of nbvh_query_rays_static: a fixed array in device memory, so that
// callers who cannot allocate still get a query. Host code must not pass the
// symbol itself to a kernel (on the host it names a stand-in, not the device
// array); the device address comes from cudaGetSymbolAddress with the device
// current, looked up once per device and context: a context created anew
// after cudaDeviceReset loads the module again, so its address is looked up
// again.
namespace nbvh {
namespace {
static __device__ __align__(256) unsigned char g_static_scratch[NBVH_STATIC_SCRATCH_BYTES];
constexpr int kMaxDevices = 64;
struct StaticAddr {
  void* ctx;   // the context the address belongs to
  void* addr;  // the array's device address in it
};
std::mutex g_static_mu;
StaticAddr g_static_addr[kMaxDevices] = {};

// The calling thread's current context (driver entry point fetched through
// the runtime, so the library does not link the driver library itself).
cudaError_t current_context(void** ctx) {
  using GetCurrent = int (*)(void**);
  static GetCurrent fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return cudaErrorSymbolNotFound;
    fn = reinterpret_cast<GetCurrent>(p);
  }
  return fn(ctx) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}
}  // namespace
}  // namespace nbvh

extern "C" nbvh_status nbvh_query_rays_static(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                              const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays,
                                              int32_t max_segs, nbvh_hits out, void* stream) {
  size_t need = 0;
  const nbvh_status st = nbvh_query_workspace_size(desc, rays.n, max_segs, &need);
  if (st != NBVH_OK) return st;
  if (need > size_t(NBVH_STATIC_SCRATCH_BYTES)) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NBVH_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NBVH_ERR_UNSUPPORTED;
  void* ctx = nullptr;  // NULL until the runtime has made a context current on this thread
  if (current_context(&ctx) != cudaSuccess) return NBVH_ERR_CUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticAddr& sa = g_static_addr[dev];
    if (!sa.addr || !ctx || sa.ctx != ctx) {
      void* p = nullptr;  // the lookup also makes the device's primary context current
      if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return NBVH_ERR_CUDA;
      if (current_context(&ctx) != cudaSuccess || !ctx) return NBVH_ERR_CUDA;
      sa.addr = p;
      sa.ctx = ctx;
    }
    base = sa.addr;
  }
  return nbvh_query_rays(desc, table, mlp, nodes, n_nodes, rays, max_segs, out, base,
                         size_t(NBVH_STATIC_SCRATCH_BYTES), stream);
}

// ---------------------------------------------------------------- training
namespace nbvh {
namespace {

// Training workspace. Per-ray arrays hold the whole batch of n rays; the
// activations the backward reads (features, hidden activations, their
// gradients) hold one chunk of `chunk` rays. chunk = n stores the whole
// batch's activations; a smaller chunk is the recompute mode: the forward
// runs chunk by chunk keeping only the per-ray outputs (raw outputs, dL/d(raw),
// loss terms), and the backward runs the forward of each chunk again to
// rebuild its activations before differentiating it.
struct TrainWs {
  int32_t* n_valid;
  float* loss;                       // the step's loss when the caller passes no loss_out
  float* partial;                    // loss reduction partial sums
  float* rays[8];
  int32_t* leaf;
  float *t0, *t1;
  uint8_t* hit;
  float *depth, *nx, *ny, *nz;
  float *ar, *ag, *ab;               // albedo labels, carved for n_out >= 8 only
  float *O, *G, *loss_seg;           // per ray (or item): raw outputs, dL/d(raw), loss terms
  int64_t chunk;                     // rays per activation chunk
  float *X, *H, *dZ;                 // FP32 path: features [c][K], H and dZ [n_hidden][c][W]
  uint16_t *X16, *H16;              // tensor-core path: 16-bit operands (X16 feature-major)
  uint16_t* HT16;                    // [n_hidden - 1][W][ld] H of the layers feeding a hidden layer, neuron-major
  uint16_t* dZT;                     // [n_hidden][W][ld] every layer's dZ, neuron-major
  int64_t ld;                        // row stride of X16, HT16 and dZT
  void* image;                       // streamed first-layer image
  uint8_t* bwd_image;                // W0^T of the streamed backward (else null)
  int32_t *counts, *cursor, *order;  // rays grouped by trained leaf (training step)
  size_t bytes;
};

constexpr int kLossBlocks = 256;

TrainWs carve_train(void* base, const nbvh_model_desc* d, int64_t n, int32_t n_leaves, int64_t chunk) {
  TrainWs w;
  std::memset(&w, 0, sizeof(w));
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += align256(bytes);
    return q;
  };
  const size_t K = size_t(d->n_samples) * d->n_levels * d->n_features;
  const size_t Wd = size_t(d->width), nh = size_t(d->n_hidden), no = size_t(d->n_out), N = size_t(n);
  const size_t C = size_t(std::min<int64_t>(std::max<int64_t>(chunk, 1), n));
  char* small = take(256);
  w.n_valid = reinterpret_cast<int32_t*>(small);
  w.loss = reinterpret_cast<float*>(small ? small + 16 : nullptr);
  w.partial = reinterpret_cast<float*>(take(4 * kLossBlocks));
  for (int k = 0; k < 8; ++k) w.rays[k] = reinterpret_cast<float*>(take(4 * N));
  w.leaf = reinterpret_cast<int32_t*>(take(4 * N));
  w.t0 = reinterpret_cast<float*>(take(4 * N));
  w.t1 = reinterpret_cast<float*>(take(4 * N));
  w.hit = reinterpret_cast<uint8_t*>(take(N));
  w.depth = reinterpret_cast<float*>(take(4 * N));
  w.nx = reinterpret_cast<float*>(take(4 * N));
  w.ny = reinterpret_cast<float*>(take(4 * N));
  w.nz = reinterpret_cast<float*>(take(4 * N));
  if (no >= 8) {
    w.ar = reinterpret_cast<float*>(take(4 * N));
    w.ag = reinterpret_cast<float*>(take(4 * N));
    w.ab = reinterpret_cast<float*>(take(4 * N));
  }
  w.O = reinterpret_cast<float*>(take(4 * N * no));
  w.G = reinterpret_cast<float*>(take(4 * N * no));
  w.loss_seg = reinterpret_cast<float*>(take(4 * N));
  w.chunk = int64_t(C);
  if (d->mlp_prec == NBVH_FP32) {
    w.X = reinterpret_cast<float*>(take(4 * C * K));
    w.H = reinterpret_cast<float*>(take(4 * nh * C * Wd));
    w.dZ = reinterpret_cast<float*>(take(4 * nh * C * Wd));
  } else {
    const size_t Kp = (K + 15) & ~size_t(15);
    w.ld = int64_t((C + 63) & ~size_t(63));
    w.X16 = reinterpret_cast<uint16_t*>(take(2 * size_t(w.ld) * Kp));
    w.dZT = reinterpret_cast<uint16_t*>(take(2 * size_t(w.ld) * Wd * nh));
    w.H16 = reinterpret_cast<uint16_t*>(take(2 * nh * C * Wd));
    if (nh > 1) w.HT16 = reinterpret_cast<uint16_t*>(take(2 * size_t(w.ld) * Wd * (nh - 1)));
    w.image = take(image_bytes(d));
    if (bwd_w0_streamed(int(K), int(Wd), int(nh))) w.bwd_image = reinterpret_cast<uint8_t*>(take(2 * Kp * Wd));
  }
  if (n_leaves > 0) {
    w.counts = reinterpret_cast<int32_t*>(take(4 * size_t(n_leaves)));
    w.cursor = reinterpret_cast<int32_t*>(take(4 * (size_t(n_leaves) + 1)));
    w.order = reinterpret_cast<int32_t*>(take(4 * N));
  }
  w.bytes = off;
  return w;
}

// Rays per activation chunk for a workspace of ws_bytes: the whole batch when
// its activations fit, else the largest multiple of 128 rays whose chunk does
// (0: not even 128 fit).
int64_t train_chunk(const nbvh_model_desc* d, int64_t n, int32_t n_leaves, size_t ws_bytes) {
  if (carve_train(nullptr, d, n, n_leaves, n).bytes <= ws_bytes) return n;
  int64_t lo = 0, hi = (n - 1) / kTcM;  // chunk = 128 k, k in [1, hi]
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (carve_train(nullptr, d, n, n_leaves, mid * kTcM).bytes <= ws_bytes)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo * kTcM;
}

// The training kernels can run this model (checked before anything is enqueued).
bool train_stageable(const nbvh_model_desc* d) {
  const int K = d->n_samples * d->n_levels * d->n_features, W = d->width;
  if (d->mlp_prec == NBVH_FP32)
    return train_fwd_smem(K, W, d->n_hidden, d->n_out) <= kSmemMax &&
           train_bwd_smem(K, W, d->n_hidden, d->n_out) <= kSmemMax;
  if (W != 32 && W != 64 && W != 128) return false;
  const TcBwdLayout bl = tc_bwd_layout(K, W, d->n_hidden, bwd_w0_streamed(K, W, d->n_hidden));
  return tc_plan(d, 0, NBVH_W1_AUTO, false).ok && bl.total <= kSmemMax && bl.ncols <= 512;
}

cudaError_t launch_train(bool bwd, const nbvh_model_desc* d, const TrainArgs& a, cudaStream_t s) {
  switch (d->table_prec) {
    case NBVH_FP32: return launch_train_t<float>(bwd, d, a, s);
    case NBVH_FP16: return launch_train_t<__half>(bwd, d, a, s);
    case NBVH_BF16: return launch_train_t<__nv_bfloat16>(bwd, d, a, s);
  }
  return cudaErrorInvalidValue;
}

bool scene_valid(const nbvh_train_scene* sc) {
  return sc && sc->nodes && sc->n_nodes >= 1 && sc->leaf_box && sc->n_leaves >= 1 && sc->tris && sc->tri_perm &&
         sc->leaf_range;
}

template <typename TZ, typename TA>
cudaError_t launch_wg_strided(const TZ* dZ, int64_t zi, int64_t zo, int n_o, const TA* A, int64_t ai, int64_t aj,
                              int n_j, int64_t n, float* dW, float* db, cudaStream_t s) {
  // split the batch so the launch has ~4 blocks per SM whatever the output size
  const int64_t gxy = int64_t((n_o + kWgT - 1) / kWgT) * ((n_j + kWgT - 1) / kWgT);
  const int64_t want = int64_t(sm_count()) * 4;
  int64_t chunk = (n * gxy + want - 1) / want;
  chunk = ((chunk + kWgRows - 1) / kWgRows) * kWgRows;
  if (chunk < 256) chunk = 256;
  dim3 grid(unsigned((n_o + kWgT - 1) / kWgT), unsigned((n_j + kWgT - 1) / kWgT), unsigned((n + chunk - 1) / chunk));
  weight_grad_tiled<TZ, TA><<<grid, 256, 0, s>>>(dZ, zi, zo, n_o, A, ai, aj, n_j, n, chunk, dW, db);
  count_launches(1);
  return cudaGetLastError();
}

template <typename TZ, typename TA>
cudaError_t launch_wg_any(const TZ* dZ, int ldz, int n_o, const TA* A, int lda, int n_j, int64_t n, float* dW,
                          float* db, cudaStream_t s) {
  return launch_wg_strided<TZ, TA>(dZ, ldz, 1, n_o, A, lda, 1, n_j, n, dW, db, s);
}

// Output-layer weight gradients (weight_grad_out) over n items: blocks of
// about n / (4 per SM) items each.
template <typename TA>
cudaError_t launch_wg_out(const float* G, int n_o, const TA* H, int W, int64_t n, float* dW, float* db,
                          cudaStream_t s) {
  if (n_o > 8 || W > 128 || W < 8 || W % 8 != 0 || (reinterpret_cast<uintptr_t>(H) & 15) != 0)
    return launch_wg_any<float, TA>(G, n_o, n_o, H, W, W, n, dW, db, s);
  const int64_t want = int64_t(sm_count()) * 4;
  const int64_t chunk = std::max<int64_t>((n + want - 1) / want, 64);
  const int64_t grid = (n + chunk - 1) / chunk;
  if (grid < 1) return cudaSuccess;
  weight_grad_out<TA, 8><<<unsigned(grid), 256, 0, s>>>(G, n_o, H, W, n, chunk, dW, db);  // n_out is 5..8
  count_launches(1);
  return cudaGetLastError();
}

// Weight gradients of the tensor-core path from its 16-bit stored operands:
// the first and hidden layers on the tensor cores (features, activations and
// pre-activation gradients stored neuron-major, the batch contiguous), the
// output layer from the FP32 dL/d(raw) and the item-major last activations.
// Shapes beyond the tensor-core kernel's TMEM/shared-memory budget use the
// CUDA-core reduction on the same operands.
template <typename T16>
cudaError_t weight_grads_16(const nbvh_model_desc* d, const TrainWs& w, const float* G, int64_t n, float* grad_mlp,
                            cudaStream_t s) {
  const int K = d->n_samples * d->n_levels * d->n_features, Kp = (K + 15) & ~15;
  const int Wd = d->width, nh = d->n_hidden, no = d->n_out;
  const bool bf16 = std::is_same<T16, __nv_bfloat16>::value;
  const T16* X = reinterpret_cast<const T16*>(w.X16);
  const T16* H = reinterpret_cast<const T16*>(w.H16);
  const T16* HT = reinterpret_cast<const T16*>(w.HT16);
  const T16* ZT = reinterpret_cast<const T16*>(w.dZT);
  const size_t lz = size_t(Wd) * size_t(w.ld);  // one layer of dZT / HT16
  size_t off = 0;
  WgTcArgs ta{w.X16, w.dZT, n, w.ld, K, Kp, grad_mlp, grad_mlp + size_t(Wd) * K};
  cudaError_t e = launch_wg_tc(bf16, Wd, ta, s);
  if (e == cudaErrorInvalidConfiguration)
    e = launch_wg_strided<T16, T16>(ZT, 1, w.ld, Wd, X, 1, w.ld, K, n, grad_mlp, grad_mlp + size_t(Wd) * K, s);
  off += size_t(Wd) * K + Wd;
  for (int h = 1; h < nh && e == cudaSuccess; ++h) {
    float* dW = grad_mlp + off;
    float* db = dW + size_t(Wd) * Wd;
    WgTcArgs th{w.HT16 + (h - 1) * lz, w.dZT + h * lz, n, w.ld, Wd, Wd, dW, db};
    e = launch_wg_tc(bf16, Wd, th, s);
    if (e == cudaErrorInvalidConfiguration)
      e = launch_wg_strided<T16, T16>(ZT + h * lz, 1, w.ld, Wd, HT + (h - 1) * lz, 1, w.ld, Wd, n, dW, db, s);
    off += size_t(Wd) * Wd + Wd;
  }
  if (e == cudaSuccess)
    e = launch_wg_out<T16>(G, no, H + size_t(nh - 1) * n * Wd, Wd, n, grad_mlp + off, grad_mlp + off + size_t(no) * Wd,
                           s);
  return e;
}

cudaError_t launch_weight_grad(const float* dZ, int n_o, const float* A, int n_j, int64_t n, float* dW, float* db,
                               cudaStream_t s) {
  return launch_wg_any<float, float>(dZ, n_o, n_o, A, n_j, n_j, n, dW, db, s);
}

// One chunk of a training batch: items [i0, i0 + c). With `order` the items
// map to rays through order[i0 ..] and the ray arrays stay whole; without it
// item i is ray i and the ray arrays are offset.
struct Chunk {
  nbvh_rays rays;
  const int32_t* leaf;
  const float *t0, *t1;
  const int32_t* order;
  int64_t i0, c;
};

Chunk chunk_of(const nbvh_rays& rays, const int32_t* leaf, const float* t0, const float* t1, const int32_t* order,
               int64_t i0, int64_t c) {
  Chunk k;
  k.rays = rays;
  k.leaf = leaf;
  k.t0 = t0;
  k.t1 = t1;
  k.order = order ? order + i0 : nullptr;
  k.i0 = i0;
  k.c = c;
  if (!order) {
    const float** f[8] = {&k.rays.ox, &k.rays.oy, &k.rays.oz, &k.rays.dx, &k.rays.dy, &k.rays.dz, &k.rays.tmin,
                          &k.rays.tmax};
    for (auto* q : f) *q += i0;
    k.leaf += i0;
    k.t0 += i0;
    k.t1 += i0;
  }
  k.rays.n = c;
  return k;
}

// The labels of a chunk's rays: indexed by ray, so offset with the ray
// arrays when the chunk's items are rays i0 .. i0 + c (no order).
Labels labels_at(const Labels& lab, const Chunk& k) {
  if (k.order || !lab.hit) return lab;
  const int64_t o = k.i0;
  auto at = [&](const float* p) { return p ? p + o : nullptr; };
  return Labels{lab.hit + o, at(lab.depth), at(lab.nx), at(lab.ny), at(lab.nz), at(lab.ar), at(lab.ag), at(lab.ab)};
}

// Forward of one chunk into the workspace's activation buffers; with labels
// (lab.hit set) also the loss terms and dL/d(raw) of its items.
cudaError_t forward_chunk(const nbvh_model_desc* d, const GridParams& gp, const void* table, const float* mlp,
                          const Chunk& k, const Labels& lab, const int32_t* n_valid, float loss_scale,
                          const float* loss_scale_dev, const TrainWs& w, const TcPlan& plan, const void* image,
                          cudaStream_t s) {
  TimedSection ts(NBVH_KERNEL_TRAIN_FORWARD, s);
  const int no = d->n_out;
  if (d->mlp_prec == NBVH_FP32) {
    TrainArgs a;
    std::memset(&a, 0, sizeof(a));
    a.gp = gp;
    a.table = table;
    a.mlp = mlp;
    a.n_hidden = d->n_hidden;
    a.width = d->width;
    a.n_out = no;
    a.rays = ray_ptrs(k.rays);
    a.leaf = k.leaf;
    a.t0 = k.t0;
    a.t1 = k.t1;
    a.n = k.c;
    a.buf = TrainBuffers{w.X, w.H, w.O + k.i0 * no, w.G + k.i0 * no, w.loss_seg + k.i0, w.dZ};
    a.lab = labels_at(lab, k);
    a.n_valid = n_valid;
    a.loss_scale = loss_scale;
    a.loss_scale_dev = loss_scale_dev;
    return launch_train(false, d, a, s);
  }
  EvalArgs a = base_args(d, gp, table, mlp, k.rays);
  a.list_t0 = k.t0;
  a.list_t1 = k.t1;
  a.n_items = k.c;
  a.w1_image = image;
  a.tr.leaf = k.leaf;
  a.tr.order = k.order;
  a.tr.X16 = w.X16;
  a.tr.ld = w.ld;
  a.tr.H16 = w.H16;
  a.tr.HT16 = w.HT16;
  a.tr.O = w.O + k.i0 * no;
  a.tr.G = w.G + k.i0 * no;
  a.tr.loss_seg = w.loss_seg + k.i0;
  a.tr.lab = labels_at(lab, k);
  a.tr.n_valid = n_valid;
  a.tr.loss_scale = loss_scale;
  a.tr.loss_scale_dev = loss_scale_dev;
  return launch_tc<2>(d, a, k.c, plan, s);
}

// Backward of one chunk whose activations are in the workspace: MLP adjoint,
// scatter into the table gradient, weight gradients (all accumulate).
cudaError_t backward_chunk(const nbvh_model_desc* d, const GridParams& gp, const void* table, const float* mlp,
                           const Chunk& k, const float* G, float* grad_table, float* grad_mlp, const TrainWs& w,
                           cudaStream_t s) {
  const int no = d->n_out;
  const float* Gk = G + k.i0 * no;
  if (d->mlp_prec != NBVH_FP32) {
    TcBwdArgs b;
    std::memset(&b, 0, sizeof(b));
    b.gp = gp;
    b.mlp = mlp;
    b.n_hidden = d->n_hidden;
    b.n_out = no;
    b.rays = ray_ptrs(k.rays);
    b.leaf = k.leaf;
    b.order = k.order;
    b.t0 = k.t0;
    b.t1 = k.t1;
    b.n = k.c;
    b.G = Gk;
    b.H16 = w.H16;
    b.dZT = w.dZT;
    b.ld = w.ld;
    b.grad_table = grad_table;
    b.w0t_image = w.bwd_image;
    cudaError_t e;
    {
      TimedSection ts(NBVH_KERNEL_TRAIN_BACKWARD, s);
      e = w.bwd_image ? launch_bwd_image(d, mlp, w.bwd_image, s) : cudaSuccess;
      if (e == cudaSuccess) e = launch_bwd_tc(d, b, s);
    }
    if (e != cudaSuccess) return e;
    TimedSection ts(NBVH_KERNEL_WEIGHT_GRAD, s);
    return d->mlp_prec == NBVH_BF16 ? weight_grads_16<__nv_bfloat16>(d, w, Gk, k.c, grad_mlp, s)
                                    : weight_grads_16<__half>(d, w, Gk, k.c, grad_mlp, s);
  }
  TrainArgs a;
  std::memset(&a, 0, sizeof(a));
  a.gp = gp;
  a.table = table;
  a.mlp = mlp;
  a.n_hidden = d->n_hidden;
  a.width = d->width;
  a.n_out = no;
  a.rays = ray_ptrs(k.rays);
  a.leaf = k.leaf;
  a.t0 = k.t0;
  a.t1 = k.t1;
  a.n = k.c;
  a.buf = TrainBuffers{w.X, w.H, nullptr, const_cast<float*>(Gk), nullptr, w.dZ};
  a.grad_table = grad_table;
  cudaError_t e;
  {
    TimedSection ts(NBVH_KERNEL_TRAIN_BACKWARD, s);
    e = launch_train(true, d, a, s);
  }
  if (e != cudaSuccess) return e;
  TimedSection ts(NBVH_KERNEL_WEIGHT_GRAD, s);
  // weight gradients, parameter order: W0 [W][K], b0, (W_h [W][W], b_h)*, Wo [n_out][W], bo
  const int K = gp.n_inputs, Wd = d->width, nh = d->n_hidden;
  const int64_t c = k.c;
  size_t off = 0;
  e = launch_weight_grad(w.dZ, Wd, w.X, K, c, grad_mlp + off, grad_mlp + off + size_t(Wd) * K, s);
  off += size_t(Wd) * K + Wd;
  for (int h = 1; h < nh && e == cudaSuccess; ++h) {
    e = launch_weight_grad(w.dZ + size_t(h) * c * Wd, Wd, w.H + size_t(h - 1) * c * Wd, Wd, c, grad_mlp + off,
                           grad_mlp + off + size_t(Wd) * Wd, s);
    off += size_t(Wd) * Wd + Wd;
  }
  if (e == cudaSuccess)
    e = launch_weight_grad(Gk, no, w.H + size_t(nh - 1) * c * Wd, Wd, c, grad_mlp + off,
                           grad_mlp + off + size_t(no) * Wd, s);
  return e;
}

// The batch loss in FP32: compensated per-thread sums, then pairwise trees
// (two launches, no atomics: the result does not depend on scheduling).
cudaError_t launch_loss(const float* term, int64_t n, const int32_t* n_valid, float* partial, float* out,
                        cudaStream_t s) {
  const int blocks = int(std::min<int64_t>(kLossBlocks, std::max<int64_t>(1, (n + 255) / 256)));
  TimedSection ts(NBVH_KERNEL_OTHER, s);
  loss_partial_kernel<<<blocks, 256, 0, s>>>(term, n, partial);
  loss_final_kernel<<<1, 256, 0, s>>>(partial, blocks, n_valid, out);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace
}  // namespace nbvh

extern "C" nbvh_status nbvh_train_rays(int32_t mode, uint64_t seed, int64_t step, const nbvh_train_scene* scene,
                                       nbvh_rays_out rays, int32_t* leaf, float* t0, float* t1, int32_t* n_valid,
                                       void* stream) {
  if ((mode != NBVH_TRAIN_PROBED_MIX && mode != NBVH_TRAIN_PAPER) || !scene_valid(scene) || rays.n < 0 ||
      step < 0)
    return NBVH_ERR_INVALID_ARG;
  if (rays.n == 0) return NBVH_OK;
  if (!rays.ox || !rays.oy || !rays.oz || !rays.dx || !rays.dy || !rays.dz || !rays.tmin || !rays.tmax || !leaf ||
      !t0 || !t1 || !n_valid || rays.n > (int64_t(1) << 31) - 1)
    return NBVH_ERR_INVALID_ARG;
  TrainRayArgs a;
  std::memset(&a, 0, sizeof(a));
  a.mode = mode;
  a.k0 = uint32_t(seed & 0xffffffffu);
  a.k1 = uint32_t(seed >> 32);
  a.step_lo = uint32_t(uint64_t(step) & 0xffffffffu);
  a.step_hi = uint32_t(uint64_t(step) >> 32);
  a.n = rays.n;
  a.nodes = scene->nodes;
  a.leaf_box = scene->leaf_box;
  a.n_leaves = scene->n_leaves;
  for (int i = 0; i < 3; ++i) {
    a.centre[i] = scene->info.centre[i];
    a.lo[i] = scene->info.lo[i];
    a.hi[i] = scene->info.hi[i];
  }
  a.radius = scene->info.sphere_radius;
  a.out = RayOut{rays.ox, rays.oy, rays.oz, rays.dx, rays.dy, rays.dz, rays.tmin, rays.tmax};
  a.leaf = leaf;
  a.t0 = t0;
  a.t1 = t1;
  a.n_valid = n_valid;
  TimedSection ts(NBVH_KERNEL_TRAIN_RAYS, as_stream(stream));
  train_rays_kernel<<<unsigned((rays.n + 127) / 128), 128, 0, as_stream(stream)>>>(a);
  count_launches(1);
  return status_of(cudaGetLastError());
}

extern "C" nbvh_status nbvh_train_labels(nbvh_rays rays, const int32_t* leaf, const float* t0, const float* t1,
                                         const nbvh_train_scene* scene, nbvh_labels out, void* stream) {
  if (!rays_valid(rays) || !scene_valid(scene)) return NBVH_ERR_INVALID_ARG;
  if (rays.n == 0) return NBVH_OK;
  if (!leaf || !t0 || !t1 || !out.hit || !out.depth || !out.nx || !out.ny || !out.nz ||
      (out.ar && (!out.ag || !out.ab)))
    return NBVH_ERR_INVALID_ARG;
  TimedSection ts(NBVH_KERNEL_LABELS, as_stream(stream));
  labels_kernel<<<unsigned((rays.n + 127) / 128), 128, 0, as_stream(stream)>>>(
      ray_ptrs(rays), leaf, t0, t1, rays.n, scene->tris, scene->tri_perm, scene->leaf_range, scene->leaf_tris,
      nullptr, out.hit, out.depth, out.nx, out.ny, out.nz, scene->tri_albedo, out.ar, out.ag, out.ab);
  count_launches(1);
  return status_of(cudaGetLastError());
}

extern "C" nbvh_status nbvh_train_workspace_size(const nbvh_model_desc* desc, int64_t n, int32_t n_leaves,
                                                 size_t* bytes) {
  if (!nbvh_host::desc_valid(desc) || n < 0 || n_leaves < 0 || !bytes) return NBVH_ERR_INVALID_ARG;
  *bytes = carve_train(nullptr, desc, n, n_leaves, n).bytes;
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_train_workspace_budget(const nbvh_model_desc* desc, int64_t n, int32_t n_leaves,
                                                   size_t max_bytes, size_t* bytes, int64_t* chunk) {
  if (!nbvh_host::desc_valid(desc) || n < 1 || n_leaves < 0 || !bytes || !chunk) return NBVH_ERR_INVALID_ARG;
  const int64_t c = train_chunk(desc, n, n_leaves, max_bytes);
  if (c <= 0) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  *chunk = c;
  *bytes = carve_train(nullptr, desc, n, n_leaves, c).bytes;
  return NBVH_OK;
}

namespace nbvh {
namespace {
nbvh_status forward_train_impl(const nbvh_model_desc* desc, const void* table, const float* mlp, nbvh_rays rays,
                               const int32_t* leaf, const float* t0, const float* t1, nbvh_labels labels,
                               const int32_t* n_valid, float loss_scale, const float* loss_scale_dev,
                               float* raw_out, float* loss_out, void* workspace, size_t ws_bytes, void* stream,
                               const int32_t* order, int32_t n_leaves) {
  if (!nbvh_host::desc_valid(desc) || !table || !mlp || !rays_valid(rays)) return NBVH_ERR_INVALID_ARG;
  if (rays.n == 0) return NBVH_OK;
  if (!leaf || !t0 || !t1 || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) ||
      (labels.hit && (!labels.depth || !labels.nx || !labels.ny || !labels.nz || !n_valid)) ||
      (labels.ar && (!labels.ag || !labels.ab)) || !(loss_scale > 0.0f) || rays.n > (int64_t(1) << 31) - 1)
    return NBVH_ERR_INVALID_ARG;
  const int64_t chunk = train_chunk(desc, rays.n, n_leaves, ws_bytes);
  if (chunk <= 0) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  TrainWs w = carve_train(workspace, desc, rays.n, n_leaves, chunk);
  GridParams gp;
  if (!make_grid(desc, gp)) return NBVH_ERR_INVALID_ARG;
  if (!train_stageable(desc)) return NBVH_ERR_UNSUPPORTED;
  cudaStream_t s = as_stream(stream);
  const Labels lab{labels.hit, labels.depth, labels.nx, labels.ny, labels.nz, labels.ar, labels.ag, labels.ab};
  EvalArgs pa = base_args(desc, gp, table, mlp, rays);
  TcPlan plan;
  cudaError_t e = prepare_eval(desc, pa, default_options(), w.image, &plan, s, false);
  for (int64_t i0 = 0; i0 < rays.n && e == cudaSuccess; i0 += chunk)
    e = forward_chunk(desc, gp, table, mlp, chunk_of(rays, leaf, t0, t1, order, i0, std::min(chunk, rays.n - i0)),
                      lab, n_valid, loss_scale, loss_scale_dev, w, plan, pa.w1_image, s);
  if (e != cudaSuccess) return status_of(e);
  if (raw_out) {
    e = cudaMemcpyAsync(raw_out, w.O, sizeof(float) * size_t(rays.n) * desc->n_out, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return NBVH_ERR_CUDA;
  }
  if (labels.hit && loss_out) e = launch_loss(w.loss_seg, rays.n, n_valid, w.partial, loss_out, s);
  return status_of(e);
}

nbvh_status backward_impl(const nbvh_model_desc* desc, const void* table, const float* mlp, nbvh_rays rays,
                          const int32_t* leaf, const float* t0, const float* t1, const float* grad_out,
                          float* grad_table, float* grad_mlp, void* workspace, size_t ws_bytes, void* stream,
                          const int32_t* order, int32_t n_leaves) {
  if (!nbvh_host::desc_valid(desc) || !table || !mlp || !rays_valid(rays)) return NBVH_ERR_INVALID_ARG;
  if (rays.n == 0) return NBVH_OK;
  if (!leaf || !t0 || !t1 || !grad_table || !grad_mlp || !workspace ||
      (reinterpret_cast<uintptr_t>(workspace) & 255) || rays.n > (int64_t(1) << 31) - 1)
    return NBVH_ERR_INVALID_ARG;
  const int64_t chunk = train_chunk(desc, rays.n, n_leaves, ws_bytes);
  if (chunk <= 0) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  TrainWs w = carve_train(workspace, desc, rays.n, n_leaves, chunk);
  GridParams gp;
  if (!make_grid(desc, gp)) return NBVH_ERR_INVALID_ARG;
  if (!train_stageable(desc)) return NBVH_ERR_UNSUPPORTED;
  cudaStream_t s = as_stream(stream);
  const float* G = grad_out ? grad_out : w.G;
  const bool recompute = chunk < rays.n;
  EvalArgs pa = base_args(desc, gp, table, mlp, rays);
  TcPlan plan;
  cudaError_t e = cudaSuccess;
  if (recompute) e = prepare_eval(desc, pa, default_options(), w.image, &plan, s, false);
  const Labels none{};
  for (int64_t i0 = 0; i0 < rays.n && e == cudaSuccess; i0 += chunk) {
    const Chunk k = chunk_of(rays, leaf, t0, t1, order, i0, std::min(chunk, rays.n - i0));
    // recompute mode: this chunk's activations again (no labels: the loss
    // terms and dL/d(raw) of the first forward stay as they are)
    if (recompute)
      e = forward_chunk(desc, gp, table, mlp, k, none, nullptr, 1.0f, nullptr, w, plan, pa.w1_image, s);
    if (e == cudaSuccess) e = backward_chunk(desc, gp, table, mlp, k, G, grad_table, grad_mlp, w, s);
  }
  return status_of(e);
}

}  // namespace
}  // namespace nbvh

extern "C" nbvh_status nbvh_forward_train(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                          nbvh_rays rays, const int32_t* leaf, const float* t0, const float* t1,
                                          nbvh_labels labels, const int32_t* n_valid, float loss_scale,
                                          const float* loss_scale_dev, float* raw_out, float* loss_out,
                                          void* workspace, size_t ws_bytes, void* stream) {
  return forward_train_impl(desc, table, mlp, rays, leaf, t0, t1, labels, n_valid, loss_scale, loss_scale_dev,
                            raw_out, loss_out, workspace, ws_bytes, stream, nullptr, 0);
}

extern "C" nbvh_status nbvh_backward(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                     nbvh_rays rays, const int32_t* leaf, const float* t0, const float* t1,
                                     const float* grad_out, float* grad_table, float* grad_mlp, void* workspace,
                                     size_t ws_bytes, void* stream) {
  return backward_impl(desc, table, mlp, rays, leaf, t0, t1, grad_out, grad_table, grad_mlp, workspace, ws_bytes,
                       stream, nullptr, 0);
}

extern "C" nbvh_status nbvh_loss_fp64(const nbvh_model_desc* desc, int64_t n, const int32_t* n_valid,
                                      const void* workspace, size_t ws_bytes, double* loss_out, void* stream) {
  if (!nbvh_host::desc_valid(desc) || n < 1 || !n_valid || !workspace || !loss_out ||
      (reinterpret_cast<uintptr_t>(workspace) & 255))
    return NBVH_ERR_INVALID_ARG;
  const int64_t chunk = train_chunk(desc, n, 0, ws_bytes);
  if (chunk <= 0) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  const TrainWs w = carve_train(const_cast<void*>(workspace), desc, n, 0, chunk);
  cudaStream_t s = as_stream(stream);
  if (cudaMemsetAsync(loss_out, 0, sizeof(double), s) != cudaSuccess) return NBVH_ERR_CUDA;
  loss_fd_fp64_kernel<<<unsigned(sm_count()), 256, 0, s>>>(w.loss_seg, n, n_valid, loss_out);
  count_launches(1);
  return status_of(cudaGetLastError());
}

extern "C" nbvh_status nbvh_adam(const nbvh_model_desc* desc, const nbvh_optim* opt, int64_t step, float lr,
                                 float beta1, float beta2, float eps, int32_t dynamic_scale, void* stream) {
  if (!nbvh_host::desc_valid(desc) || !opt || step < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return NBVH_ERR_INVALID_ARG;
  if (!opt->table_master || !opt->table_m || !opt->table_v || !opt->grad_table || !opt->mlp || !opt->mlp_m ||
      !opt->mlp_v || !opt->grad_mlp || !opt->loss_scale || !opt->counters)
    return NBVH_ERR_INVALID_ARG;
  int32_t res[NBVH_MAX_LEVELS], dense[NBVH_MAX_LEVELS];
  int64_t size[NBVH_MAX_LEVELS], offset[NBVH_MAX_LEVELS], total = 0;
  if (!nbvh_host::layout(desc, res, dense, size, offset, &total)) return NBVH_ERR_INVALID_ARG;
  const int64_t nt = total * desc->n_features;
  const int64_t nm = nbvh_host::mlp_params(desc);
  cudaStream_t s = as_stream(stream);
  AdamState st{opt->loss_scale, opt->counters, opt->counters + 1, opt->counters + 2};
  const unsigned g = unsigned(sm_count()) * 8;
  TimedSection ts(NBVH_KERNEL_ADAM, s);
  grad_check_kernel<<<g, 256, 0, s>>>(opt->grad_table, nt, st.bad);
  grad_check_kernel<<<g, 256, 0, s>>>(opt->grad_mlp, nm, st.bad);
  const double c1 = 1.0 - std::pow(double(beta1), double(step));
  const double c2 = 1.0 - std::pow(double(beta2), double(step));
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const bool vt = a16(opt->table_master) && a16(opt->grad_table) && a16(opt->table_m) && a16(opt->table_v) &&
                  (reinterpret_cast<uintptr_t>(opt->table_work) & 15) == 0;
  const bool vm = a16(opt->mlp) && a16(opt->grad_mlp) && a16(opt->mlp_m) && a16(opt->mlp_v);
  auto table_adam = [&](auto tag) {
    using T = decltype(tag);
    T* work = static_cast<T*>(opt->table_work);
    if (vt)
      adam_kernel<T, true><<<g, 256, 0, s>>>(opt->table_master, work, opt->grad_table, opt->table_m, opt->table_v, nt,
                                             lr, beta1, beta2, eps, float(c1), float(c2), st);
    else
      adam_kernel<T, false><<<g, 256, 0, s>>>(opt->table_master, work, opt->grad_table, opt->table_m, opt->table_v,
                                              nt, lr, beta1, beta2, eps, float(c1), float(c2), st);
  };
  switch (desc->table_prec) {
    case NBVH_FP16: table_adam(__half()); break;
    case NBVH_BF16: table_adam(__nv_bfloat16()); break;
    default: table_adam(float()); break;
  }
  if (vm)
    adam_kernel<float, true><<<g, 256, 0, s>>>(opt->mlp, nullptr, opt->grad_mlp, opt->mlp_m, opt->mlp_v, nm, lr, beta1,
                                               beta2, eps, float(c1), float(c2), st);
  else
    adam_kernel<float, false><<<g, 256, 0, s>>>(opt->mlp, nullptr, opt->grad_mlp, opt->mlp_m, opt->mlp_v, nm, lr,
                                                beta1, beta2, eps, float(c1), float(c2), st);
  loss_scale_update_kernel<<<1, 1, 0, s>>>(st, dynamic_scale);
  count_launches(5);
  return status_of(cudaGetLastError());
}

extern "C" nbvh_status nbvh_train_step(const nbvh_model_desc* desc, const nbvh_optim* opt,
                                       const nbvh_train_scene* scene, int32_t mode, int64_t batch, uint64_t seed,
                                       int64_t step, float lr, float* loss_out, void* workspace, size_t ws_bytes,
                                       void* stream) {
  return nbvh_train_step_weighted(desc, opt, scene, mode, batch, seed, step, lr, nullptr, nullptr, loss_out,
                                  workspace, ws_bytes, stream);
}

extern "C" nbvh_status nbvh_train_step_weighted(const nbvh_model_desc* desc, const nbvh_optim* opt,
                                                const nbvh_train_scene* scene, int32_t mode, int64_t batch,
                                                uint64_t seed, int64_t step, float lr, const float* leaf_prob,
                                                const nbvh_leaf_stats* stats, float* loss_out, void* workspace,
                                                size_t ws_bytes, void* stream) {
  if (!nbvh_host::desc_valid(desc) || !opt || !scene_valid(scene) || batch < 1 || step < 1 || !workspace ||
      (reinterpret_cast<uintptr_t>(workspace) & 255) || batch > (int64_t(1) << 31) - 1)
    return NBVH_ERR_INVALID_ARG;
  if (stats && (!stats->hits || !stats->trained || !stats->loss)) return NBVH_ERR_INVALID_ARG;
  const int64_t chunk = train_chunk(desc, batch, scene->n_leaves, ws_bytes);
  if (chunk <= 0) return NBVH_ERR_WORKSPACE_TOO_SMALL;
  if (!train_stageable(desc)) return NBVH_ERR_UNSUPPORTED;
  TrainWs w = carve_train(workspace, desc, batch, scene->n_leaves, chunk);
  cudaStream_t s = as_stream(stream);
  if (cudaMemsetAsync(w.n_valid, 0, 256, s) != cudaSuccess) return NBVH_ERR_CUDA;
  if (cudaMemsetAsync(w.counts, 0, 4 * size_t(scene->n_leaves), s) != cudaSuccess) return NBVH_ERR_CUDA;
  nbvh_rays_out ro{w.rays[0], w.rays[1], w.rays[2], w.rays[3], w.rays[4], w.rays[5], w.rays[6], w.rays[7], batch};
  nbvh_status st = nbvh_train_rays(mode, seed, step - 1, scene, ro, w.leaf, w.t0, w.t1, w.n_valid, stream);
  if (st != NBVH_OK) return st;
  if (leaf_prob || stats) {  // first-leaf hit counts; trained with the leaf's probability
    const uint64_t st0 = uint64_t(step - 1);
    TimedSection ts(NBVH_KERNEL_TRAIN_RAYS, s);
    leaf_select_kernel<<<unsigned((batch + 255) / 256), 256, 0, s>>>(
        w.leaf, batch, uint32_t(seed & 0xffffffffu), uint32_t(seed >> 32), uint32_t(st0 & 0xffffffffu),
        uint32_t(st0 >> 32), leaf_prob, stats ? stats->hits : nullptr, w.n_valid);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return NBVH_ERR_CUDA;
  }
  nbvh_rays ri{w.rays[0], w.rays[1], w.rays[2], w.rays[3], w.rays[4], w.rays[5], w.rays[6], w.rays[7], batch};
  const bool alb = desc->n_out >= 8 && scene->tri_albedo;
  nbvh_labels lab{w.hit, w.depth, w.nx, w.ny, w.nz, alb ? w.ar : nullptr, alb ? w.ag : nullptr, alb ? w.ab : nullptr};
  // group the rays by trained leaf: labels share a leaf's triangles per warp,
  // and the forward/backward tiles hold spatially close rays
  const unsigned g = unsigned((batch + 255) / 256);
  {
    TimedSection ts(NBVH_KERNEL_TRAIN_RAYS, s);
    leaf_hist_kernel<<<g, 256, 0, s>>>(w.leaf, batch, w.counts);
    leaf_scan_kernel<<<1, 1024, 0, s>>>(w.counts, scene->n_leaves, w.cursor);
    leaf_scatter_kernel<<<g, 256, 0, s>>>(w.leaf, batch, scene->n_leaves, w.cursor, w.order);
    count_launches(3);
  }
  {
    TimedSection ts(NBVH_KERNEL_LABELS, s);
    labels_kernel<<<unsigned((batch + 127) / 128), 128, 0, s>>>(
        RayPtrs{ri.ox, ri.oy, ri.oz, ri.dx, ri.dy, ri.dz, ri.tmin, ri.tmax}, w.leaf, w.t0, w.t1, batch, scene->tris,
        scene->tri_perm, scene->leaf_range, scene->leaf_tris, w.order, lab.hit, lab.depth, lab.nx, lab.ny, lab.nz,
        scene->tri_albedo, lab.ar, lab.ag, lab.ab);
    count_launches(1);
  }
  if (cudaGetLastError() != cudaSuccess) return NBVH_ERR_CUDA;
  const void* table = opt->table_work ? opt->table_work : opt->table_master;
  const int32_t* order = desc->mlp_prec != NBVH_FP32 ? w.order : nullptr;
  st = forward_train_impl(desc, table, opt->mlp, ri, w.leaf, w.t0, w.t1, lab, w.n_valid, 1.0f, opt->loss_scale,
                          nullptr, loss_out ? loss_out : w.loss, workspace, ws_bytes, stream, order,
                          scene->n_leaves);
  if (st != NBVH_OK) return st;
  if (stats) {  // per-leaf sums over each leaf's contiguous range of the grouped order
    TimedSection ts(NBVH_KERNEL_OTHER, s);
    leaf_loss_kernel<<<unsigned((scene->n_leaves + 7) / 8), 256, 0, s>>>(
        w.loss_seg, w.order, order != nullptr ? 1 : 0, w.counts, w.cursor, scene->n_leaves, stats->trained,
        stats->loss);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return NBVH_ERR_CUDA;
  }
  st = backward_impl(desc, table, opt->mlp, ri, w.leaf, w.t0, w.t1, nullptr, opt->grad_table, opt->grad_mlp,
                     workspace, ws_bytes, stream, order, scene->n_leaves);
  if (st != NBVH_OK) return st;
  return nbvh_adam(desc, opt, step, lr, 0.9f, 0.999f, 1e-8f, desc->mlp_prec != NBVH_FP32 ? 1 : 0, stream);
}

// ---------------------------------------------------------------- graphs
struct nbvh_graph_s {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

extern "C" nbvh_status nbvh_graph_begin(void* stream) {
  cudaStream_t s = as_stream(stream);
  if (!s) return NBVH_ERR_INVALID_ARG;
  return cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess ? NBVH_OK : NBVH_ERR_CUDA;
}

extern "C" nbvh_status nbvh_graph_end(void* stream, nbvh_graph* out) {
  cudaStream_t s = as_stream(stream);
  if (!s || !out) return NBVH_ERR_INVALID_ARG;
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(s, &g) != cudaSuccess || !g) return NBVH_ERR_CUDA;
  cudaGraphExec_t e = nullptr;
  if (cudaGraphInstantiate(&e, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    return NBVH_ERR_CUDA;
  }
  *out = new nbvh_graph_s{g, e};
  return NBVH_OK;
}

extern "C" nbvh_status nbvh_graph_launch(nbvh_graph graph, void* stream) {
  if (!graph) return NBVH_ERR_INVALID_ARG;
  return cudaGraphLaunch(graph->exec, as_stream(stream)) == cudaSuccess ? NBVH_OK : NBVH_ERR_CUDA;
}

extern "C" nbvh_status nbvh_graph_destroy(nbvh_graph graph) {
  if (!graph) return NBVH_ERR_INVALID_ARG;
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  delete graph;
  return NBVH_OK;
}
