// Host side of the IFNSO library: plans, workspace layout, TMA descriptors,
// the launch metadata of a batch and the pass sequence of Algorithm 1
// (Sec. 2.4) and of the Newton-Schulz baseline (Sec. 1).  Every step of the
// computation runs in this library's kernels; the host only validates,
// lays out and enqueues.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <string>
#include <vector>

#include "common.cuh"
#include "ifnso.h"

using namespace ifnso;

namespace {
// pass kinds of the tensor-core path, as ifnso_plan_autotune reports them
constexpr int kGram = 0, kSplit = 1, kPlain = 2, kApply = 3, kKinds = 4;
// stage-depth kinds: the four above and the final squaring (which reads P in its epilogue)
constexpr int kFinal = 4, kDepthKinds = 5;
}  // namespace

struct ifnso_plan {
  int64_t h = 0, w = 0;
  int dtype = IFNSO_BF16;
  int L = 0;
  int precision = IFNSO_PREC_AUTO;
  int split_squarings = -1;  // IFNSO_OPT_SPLIT_SQUARINGS (-1: max(0, L - 8))
  int scale = IFNSO_SCALE_GRAM;
  int max_ctas = 0;
  int stop_after = -1;
  int wait_ms = 0;       // limit of the kernels' pipeline waits (0: 4 s)
  int inject_stall = 0;  // testing aid: the Gram pass's first CTA loads nothing
  int cta_group = 0;     // tensor-core passes: 0 auto, 1 per-CTA MMAs, 2 MMAs of the CTA pair
  int gram_e4m3 = 0;     // Gram from a scaled E4M3 copy of A
  int small = 0;         // IFNSO_OPT_SMALL_MATRICES: 0 auto, 1 on-chip path where eligible, 2 tiled passes
  int small_tuned = 0;   // the autotuner's choice for eligible batches (0: not measured, 1 on chip, 2 tiled)
  int apply_f16 = 1;     // IFNSO_OPT_APPLY_F16
  int copy_hosts = 0;    // IFNSO_OPT_FP16_COPY_HOSTS of the last call
  bool tuned = false;    // ifnso_plan_autotune chose cg_kind
  int cg_kind[4] = {1, 2, 1, 1};  // MMA mode per pass kind (Gram, split squaring, plain squaring, product)
  int stage_lim[kDepthKinds] = {0, 0, 0, 0, 0};  // IFNSO_OPT_STAGE_LIMITS (0: the whole ring)
  int num_sms = 0;
  // metadata of the last batch (pinned host copy, uploaded into the workspace)
  uint64_t sig = 0;
  bool sig_valid = false;
  void* meta_host = nullptr;
  size_t meta_cap = 0;
  // per-pass timing (IFNSO_OPT_TIMING): events of every call since the last query
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::vector<cudaEvent_t>> ev_calls;
  std::vector<std::vector<cudaEvent_t>> ev_graph;  // recorded by the last captured call (kept for replays)
  std::vector<cudaEvent_t> ev_retired;             // events of earlier captures (graphs may still hold them)
  // ifnso_orthogonalize_host: copy streams and the events that order them
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaStream_t s_comp = nullptr;  // the second compute stream (IFNSO_OPT_HOST_STREAMS = 2)
  int host_streams = 2;
  cudaEvent_t ev_start = nullptr, ev_last = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_done;
  // timeline of the last ifnso_orthogonalize_host call (IFNSO_OPT_TIMING, eager calls):
  // tl_start, then per group uploads done, passes done, downloads done
  cudaEvent_t tl_start = nullptr;
  std::vector<cudaEvent_t> tl_ev;
  int tl_groups = 0;
  std::vector<int> tl_first;  // first matrix of each group, and the count
  int groups = 1;  // groups the item lists of the cached metadata are built for
  std::vector<size_t> sym_off, app_off;  // first work item of each group
  std::vector<int32_t> small_idx;         // matrices the on-chip path computes (ascending)
  std::mutex mu;
};

namespace {

thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};

ifnso_status fail(ifnso_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

ifnso_status cuda_fail(cudaError_t e, const char* what) {
  return fail(IFNSO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define IFNSO_CUDA(call, what)                 \
  do {                                         \
    cudaError_t e__ = (call);                  \
    if (e__ != cudaSuccess) return cuda_fail(e__, what); \
  } while (0)

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Record a timing event on `stream` if the plan times its passes.  During
// stream capture the event becomes a record node of the graph (external
// record) and stays reserved for that graph: every replay records it again.
cudaError_t mark(ifnso_plan* plan, cudaStream_t stream, bool first) {
  if (!plan->timing) return cudaSuccess;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t r = cudaStreamIsCapturing(stream, &cap);
  if (r != cudaSuccess) return r;
  const bool captured = cap == cudaStreamCaptureStatusActive;
  auto& calls = captured ? plan->ev_graph : plan->ev_calls;
  if (first && captured) {
    // a new capture: pass times follow its graph from now on; the earlier
    // graphs' events stay alive until the plan is destroyed
    for (auto& c : plan->ev_graph)
      for (cudaEvent_t ev : c) plan->ev_retired.push_back(ev);
    plan->ev_graph.clear();
  }
  if (first) calls.emplace_back();
  cudaEvent_t e;
  // a captured call takes new events (never recorded until the graph's first
  // replay, so the query can tell) and never returns them to the pool
  if (!captured && !plan->ev_pool.empty()) {
    e = plan->ev_pool.back();
    plan->ev_pool.pop_back();
  } else {
    r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
  }
  calls.back().push_back(e);
  return cudaEventRecordWithFlags(e, stream, captured ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// 2D tiled tensor map, 128-byte swizzle, zero fill outside the tensor.
// inner/outer: extents in elements, ld: row pitch in elements.
bool encode2d(CUtensorMap* map, CUtensorMapDataType dt, const void* ptr, uint64_t inner,
              uint64_t outer, uint64_t ld, uint32_t box_inner, uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld * (dt == CU_TENSOR_MAP_DATA_TYPE_UINT8 ? 1u : 2u)};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// K-major operand view: rows of `outer`, contiguous K of `inner` (box 64 x 128).
bool map_k(CUtensorMap* m, CUtensorMapDataType dt, const void* p, int64_t inner, int64_t outer, int64_t ld) {
  return encode2d(m, dt, p, inner, outer, ld, 64, 128);
}
// MN-major operand view: contiguous MN of `inner`, K rows of `outer` (box 64 x 64).
bool map_mn(CUtensorMap* m, CUtensorMapDataType dt, const void* p, int64_t inner, int64_t outer, int64_t ld) {
  return encode2d(m, dt, p, inner, outer, ld, 64, 64);
}

struct Shape {
  int64_t rows, cols, ld;
  int64_t h, w, hpad;
  int trans;
};

// ------------------------------------------------------------------ layout
// Workspace = [metadata | scalars | per-matrix buffers].  Offsets in bytes.
struct Prec {
  int ws_lo;    // the workspace keeps lo buffers
  int k_split;  // squarings 1..k_split use split operands
  int p_split;  // P = hi + lo for the final product
  int mode;     // resolved IFNSO_PREC_*
  int p_f16;    // the final product in FP16: P as one FP16 value times the FP16 copy A s
  int chip_p_split;  // P = hi + lo in the on-chip path's product (it has no FP16 form)
};

struct Layout {
  int count = 0;
  int L = 0;
  int split = 0;     // the workspace keeps lo buffers (BF16 plans)
  Prec prec{};
  int f32 = 0;
  int e4m3 = 0;      // per-matrix E4M3 copies of A for the Gram
  int ns = 0;        // Newton-Schulz layout
  int steps = 0;
  std::vector<Shape> shp;
  // metadata
  size_t off_mats = 0, off_probs = 0, off_items_sym = 0, off_items_app = 0, off_coef = 0, off_rows = 0;
  size_t off_small = 0;  // SmProblem per matrix (BF16 plans): the on-chip path for h <= 128
  size_t off_small_idx = 0;  // int32 per matrix: the matrices the on-chip path computes
  size_t off_small_ns = 0;   // SmNsProblem per matrix (BF16 Newton-Schulz layouts)
  size_t n_probs = 0, n_sym = 0, n_app = 0;
  size_t prob_bytes = 0;
  size_t meta_bytes = 0;
  size_t off_scal = 0;
  std::vector<size_t> off_buf;  // per matrix
  size_t total = 0;
  // problem slots
  size_t pi_gram = 0, pi_sqr = 0, pi_apply = 0;  // IFNSO: gram[count], sqr[2][count], apply[count]
  size_t pi_ns_gram = 0, pi_ns_sqr = 0, pi_ns_apply = 0;  // NS: gram[steps][count], sqr[count], apply[steps][count]
};

size_t a64(size_t v) { return (v + 127) & ~size_t(127); }  // 128: the alignment of CUtensorMap

constexpr int kRowSlots = 32;  // FP32 coefficient slots per matrix (K <= 31)
size_t a1k(size_t v) { return (v + 1023) & ~size_t(1023); }

ifnso_status read_batch(const ifnso_plan* plan, const ifnso_batch_desc* b, std::vector<Shape>& shp) {
  if (!b || b->count < 0 || (b->count > 0 && (!b->in || !b->rows || !b->cols)))
    return fail(IFNSO_ERR_INVALID_ARG, "batch descriptor is NULL or incomplete");
  if (b->count > 65535) return fail(IFNSO_ERR_INVALID_ARG, "batch count %d exceeds 65535", b->count);
  const int esz = plan->dtype == IFNSO_BF16 ? 2 : 4;
  shp.resize(b->count);
  for (int i = 0; i < b->count; ++i) {
    Shape s;
    s.rows = b->rows[i];
    s.cols = b->cols[i];
    s.ld = b->ld ? b->ld[i] : s.cols;
    if (s.rows <= 0 || s.cols <= 0) return fail(IFNSO_ERR_INVALID_ARG, "matrix %d: empty shape %lldx%lld", i, (long long)s.rows, (long long)s.cols);
    if (s.ld < s.cols) return fail(IFNSO_ERR_INVALID_ARG, "matrix %d: ld %lld < cols %lld", i, (long long)s.ld, (long long)s.cols);
    if (!b->in[i]) return fail(IFNSO_ERR_INVALID_ARG, "matrix %d: NULL input", i);
    const uintptr_t a = reinterpret_cast<uintptr_t>(b->in[i]);
    if (a % 16 != 0) return fail(IFNSO_ERR_INVALID_ARG, "matrix %d: input not 16-byte aligned", i);
    if (plan->dtype == IFNSO_BF16 && (s.ld * esz) % 16 != 0)
      return fail(IFNSO_ERR_INVALID_ARG, "matrix %d: BF16 leading dimension %lld not a multiple of 8", i, (long long)s.ld);
    s.trans = s.rows > s.cols ? 1 : 0;
    s.h = s.trans ? s.cols : s.rows;
    s.w = s.trans ? s.rows : s.cols;
    if (s.h > plan->h || s.w > plan->w)
      return fail(IFNSO_ERR_INVALID_ARG, "matrix %d: oriented shape %lldx%lld exceeds the plan's %lldx%lld", i,
                  (long long)s.h, (long long)s.w, (long long)plan->h, (long long)plan->w);
    s.hpad = round_up(s.h, HPAD);
    if (s.hpad / 128 > 65535 || (s.w + 255) / 256 > 65535)
      return fail(IFNSO_ERR_INVALID_ARG, "matrix %d too large", i);
    shp[i] = s;
  }
  return IFNSO_OK;
}

// Operand precision of a BF16 plan: how many of the L - 1 squarings multiply
// split (hi + lo) operands -- always the first ones: a rounding error made in
// squaring l is amplified by up to 2^(L - l) in the later ones, so the last
// seven squarings tolerate plain FP16 operands -- and whether P is split for
// the final product.
Prec resolve_prec(const ifnso_plan* p) {
  Prec r{0, 0, 0, IFNSO_PREC_PLAIN, 0, 0};
  if (p->dtype != IFNSO_BF16) return r;
  int mode = p->precision;
  const int L = p->L;
  if (mode == IFNSO_PREC_AUTO) mode = L <= 4 ? IFNSO_PREC_PLAIN : (L >= 15 ? IFNSO_PREC_SPLIT : IFNSO_PREC_MIXED);
  r.mode = mode;
  if (mode == IFNSO_PREC_SPLIT) {
    r.k_split = L - 1;
    r.p_split = 1;
  } else if (mode == IFNSO_PREC_MIXED) {
    r.k_split = p->split_squarings >= 0 ? std::min(p->split_squarings, L - 1) : std::max(0, L - 8);
    r.p_split = 1;
  }
  r.chip_p_split = r.p_split;
  // The FP16 product replaces MIXED plans' two products of P hi + lo by one.
  // (SPLIT's longer chains have larger coefficients, and P's FP16 rounding,
  // about 2^-11 of its largest entries, then exceeds the BF16 plans' budget;
  // PLAIN plans already take one BF16 product of P, and the copy of the
  // input would only add its HBM traffic.)
  if (p->apply_f16 && L >= 2 && mode == IFNSO_PREC_MIXED) {
    r.p_f16 = 1;
    r.p_split = 0;
  }
  r.ws_lo = r.p_split || r.k_split > 0;
  return r;
}

// Matrices [b[g], b[g + 1]) form group g: contiguous index ranges, at most
// `groups` of them, none empty, cut where the cumulative work (h_pad^2 w per
// matrix) crosses the targets.  Equal shares, or with `ramp` (6 groups or
// more) 1/48 and 1/16 of the work in the first two and the last two groups
// and equal shares in between: the upload before the first group's passes
// and the download after the last group's are then short, and every middle
// group's passes still outlast the next group's upload.
std::vector<int> group_bounds(const std::vector<Shape>& shp, int groups, bool ramp = false) {
  const int n = static_cast<int>(shp.size());
  std::vector<double> target;  // cumulative work fractions of the cuts
  if (ramp && groups >= 6) {
    const double e1 = 1.0 / 48.0, e2 = 1.0 / 16.0;
    const double mid = (1.0 - 2.0 * (e1 + e2)) / (groups - 4);
    double t = 0.0;
    for (int g = 0; g + 1 < groups; ++g) {
      t += (g == 0) ? e1 : (g == 1) ? e2 : (g == groups - 2) ? e2 : mid;
      target.push_back(t);
    }
  } else {
    for (int g = 1; g < groups; ++g) target.push_back(static_cast<double>(g) / groups);
  }
  std::vector<int> b{0};
  double total = 0.0;
  for (const Shape& s : shp) total += static_cast<double>(s.hpad) * s.hpad * s.w;
  double acc = 0.0;
  size_t next = 0;
  for (int i = 0; i + 1 < n && next < target.size(); ++i) {
    acc += static_cast<double>(shp[i].hpad) * shp[i].hpad * shp[i].w;
    if (acc >= total * target[next]) {
      b.push_back(i + 1);
      while (next < target.size() && acc >= total * target[next]) ++next;
    }
  }
  b.push_back(n);
  return b;
}

// Matrices of [first, last), heaviest first (longer K first for the Gram and
// the product; equal for squarings).
std::vector<int> heavy_first(const std::vector<Shape>& shp, int first, int last) {
  std::vector<int> order;
  for (int i = first; i < last; ++i) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return shp[a].hpad * shp[a].w > shp[b].hpad * shp[b].w;
  });
  return order;
}

// Work items of the symmetric passes, group after group; off[g] = first item of group g.
// skip_small: the on-chip path computes the matrices with h <= kSmallH (no items for them).
void sym_items(const std::vector<Shape>& shp, const std::vector<int>& gb, std::vector<WorkItem>& items,
               std::vector<size_t>* off = nullptr, bool skip_small = false) {
  if (off) off->clear();
  for (size_t g = 0; g + 1 < gb.size(); ++g) {
    if (off) off->push_back(items.size());
    // one item per upper 256 x 256 block (I <= J): its two 128-row halves go
    // to the two CTAs of a cluster
    for (int m : heavy_first(shp, gb[g], gb[g + 1])) {
      if (skip_small && shp[m].h <= kSmallH) continue;
      const int nb = static_cast<int>(shp[m].hpad / 256);
      for (int I = 0; I < nb; ++I)
        for (int J = I; J < nb; ++J)
          items.push_back(WorkItem{static_cast<uint16_t>(m), static_cast<uint16_t>(2 * I),
                                   static_cast<uint16_t>(J), static_cast<uint16_t>(I == J ? 1 : 0)});
    }
  }
  if (off) off->push_back(items.size());
}

void app_items(const std::vector<Shape>& shp, const std::vector<int>& gb, std::vector<WorkItem>& items,
               std::vector<size_t>* off = nullptr, bool skip_small = false) {
  if (off) off->clear();
  for (size_t g = 0; g + 1 < gb.size(); ++g) {
    if (off) off->push_back(items.size());
    // one item per pair of 128-row tiles sharing a 256-column block (rows past
    // h are computed on zero padding and not stored)
    for (int m : heavy_first(shp, gb[g], gb[g + 1])) {
      if (skip_small && shp[m].h <= kSmallH) continue;
      const int pairs = static_cast<int>((shp[m].h + 2 * BM - 1) / (2 * BM));
      const int tns = static_cast<int>((shp[m].w + BN - 1) / BN);
      for (int tn = 0; tn < tns; ++tn)
        for (int pr = 0; pr < pairs; ++pr)
          items.push_back(WorkItem{static_cast<uint16_t>(m), static_cast<uint16_t>(2 * pr),
                                   static_cast<uint16_t>(tn), 0});
    }
  }
  if (off) off->push_back(items.size());
}

Layout make_layout(const ifnso_plan* plan, const std::vector<Shape>& shp, int ns, int steps, int K) {
  Layout ly;
  ly.count = static_cast<int>(shp.size());
  ly.L = plan->L;
  ly.prec = ns ? Prec{0, 0, 0, IFNSO_PREC_PLAIN, 0, 0} : resolve_prec(plan);
  ly.split = ly.prec.ws_lo;
  ly.f32 = plan->dtype == IFNSO_F32;
  ly.e4m3 = (!ns && !ly.f32 && plan->gram_e4m3) ? 1 : 0;
  ly.ns = ns;
  ly.steps = steps;
  ly.shp = shp;
  const size_t n = shp.size();
  ly.prob_bytes = ly.f32 ? sizeof(SgProblem) : sizeof(TcProblem);
  if (!ns) {
    ly.pi_gram = 0;
    ly.pi_sqr = n;
    ly.pi_apply = 3 * n;
    ly.n_probs = 4 * n;
  } else {
    ly.pi_ns_gram = 0;
    ly.pi_ns_sqr = steps * n;
    ly.pi_ns_apply = steps * n + n;
    ly.n_probs = (2 * steps + 1) * n;
  }
  if (!ly.f32) {
    std::vector<WorkItem> a, b;
    const std::vector<int> all{0, static_cast<int>(shp.size())};
    sym_items(shp, all, a);
    app_items(shp, all, b);
    ly.n_sym = a.size();
    ly.n_app = b.size();
  }
  size_t off = 0;
  ly.off_mats = off;
  off = a64(off + n * sizeof(MatInfo));
  ly.off_probs = off;
  off = a64(off + ly.n_probs * ly.prob_bytes);
  ly.off_items_sym = off;
  off = a64(off + ly.n_sym * sizeof(WorkItem));
  ly.off_items_app = off;
  off = a64(off + ly.n_app * sizeof(WorkItem));
  ly.off_coef = off;
  off = a64(off + sizeof(double) * (K > 0 ? K : 1));
  ly.off_rows = off;  // per-matrix coefficient rows written by the proposal network
  off = a64(off + n * kRowSlots * sizeof(float));
  if (!ly.f32 && !ns) {
    ly.off_small = off;
    off = a64(off + n * sizeof(SmProblem));
    ly.off_small_idx = off;
    off = a64(off + n * sizeof(int32_t));
  }
  if (!ly.f32 && ns) {
    ly.off_small_ns = off;
    off = a64(off + n * sizeof(SmNsProblem));
  }
  ly.meta_bytes = off;
  off = a1k(off);
  ly.off_scal = off;
  off = a1k(off + n * sizeof(MatScalars));
  ly.off_buf.resize(n);
  const size_t e = ly.f32 ? 4 : 2;
  for (size_t i = 0; i < n; ++i) {
    ly.off_buf[i] = off;
    const size_t hp2 = static_cast<size_t>(shp[i].hpad) * shp[i].hpad;
    if (!ns) {
      off = a1k(off + hp2 * 4);  // T_0 / P (FP32)
      if (ly.f32) {
        off = a1k(off + hp2 * 4);  // D buffer 0
        off = a1k(off + hp2 * 4);  // D buffer 1
      } else {
        for (int b = 0; b < 4; ++b)
          if (ly.split || (b & 1) == 0) off = a1k(off + hp2 * 2);
        if (ly.e4m3) off = a1k(off + static_cast<size_t>(shp[i].h) * round_up(shp[i].w, 16));  // A s, E4M3
        if (ly.prec.p_f16) off = a1k(off + static_cast<size_t>(shp[i].rows) * round_up(shp[i].cols, 8) * 2);  // M s, FP16
      }
    } else {
      const size_t xld = static_cast<size_t>(round_up(shp[i].cols, 8));
      off = a1k(off + hp2 * e);                     // S
      off = a1k(off + hp2 * e);                     // B
      off = a1k(off + shp[i].rows * xld * e);       // X buffer 0
      off = a1k(off + shp[i].rows * xld * e);       // X buffer 1
    }
  }
  ly.total = off;
  return ly;
}

// Fill MatInfo buffer pointers for matrix i.
MatInfo mat_info(const Layout& ly, const ifnso_batch_desc* b, void* const* out, uint8_t* ws, int i) {
  const Shape& s = ly.shp[i];
  MatInfo mi;
  memset(&mi, 0, sizeof(mi));
  mi.in = b->in[i];
  mi.out = out ? out[i] : nullptr;
  mi.rows = s.rows;
  mi.cols = s.cols;
  mi.ld = s.ld;
  mi.h = static_cast<int32_t>(s.h);
  mi.w = static_cast<int32_t>(s.w);
  mi.hpad = static_cast<int32_t>(s.hpad);
  mi.trans = s.trans;
  const size_t hp2 = static_cast<size_t>(s.hpad) * s.hpad;
  uint8_t* p = ws + ly.off_buf[i];
  const size_t e = ly.f32 ? 4 : 2;
  if (!ly.ns) {
    mi.gp = reinterpret_cast<float*>(p);
    p += a1k(hp2 * 4);
    if (ly.f32) {
      mi.d[0] = p;
      p += a1k(hp2 * 4);
      mi.d[2] = p;
    } else {
      for (int bb = 0; bb < 4; ++bb) {
        if (ly.split || (bb & 1) == 0) {
          mi.d[bb] = p;
          p += a1k(hp2 * 2);
        }
      }
      if (ly.e4m3) {
        mi.a8 = static_cast<uint8_t*>(p);
        mi.a8ld = round_up(s.w, 16);
        p += a1k(static_cast<size_t>(s.h) * mi.a8ld);
      }
      if (ly.prec.p_f16) {
        mi.a16 = p;
        mi.a16ld = round_up(s.cols, 8);
      }
    }
  } else {
    const size_t xld = static_cast<size_t>(round_up(s.cols, 8));
    mi.s = p;
    p += a1k(hp2 * e);
    mi.b = p;
    p += a1k(hp2 * e);
    mi.x[0] = p;
    p += a1k(s.rows * xld * e);
    mi.x[1] = p;
    mi.xld = static_cast<int64_t>(xld);
  }
  return mi;
}

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const uint8_t* c = static_cast<const uint8_t*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t batch_sig(const ifnso_plan* plan, const ifnso_batch_desc* b, void* const* out, const void* ws,
                   const ifnso_coeffs* cf, const double* poly, int degree, int steps, int kind) {
  uint64_t h = 1469598103934665603ull;
  const Prec pr = resolve_prec(plan);
  int opts[9] = {plan->L, pr.mode, pr.k_split, pr.p_split, plan->scale, plan->dtype, kind, steps, pr.p_f16};
  h = fnv(h, opts, sizeof(opts));
  h = fnv(h, &ws, sizeof(ws));
  h = fnv(h, &b->count, sizeof(b->count));
  for (int i = 0; i < b->count; ++i) {
    h = fnv(h, &b->in[i], sizeof(void*));
    if (out) h = fnv(h, &out[i], sizeof(void*));
    h = fnv(h, &b->rows[i], 8);
    h = fnv(h, &b->cols[i], 8);
    int64_t ld = b->ld ? b->ld[i] : b->cols[i];
    h = fnv(h, &ld, 8);
  }
  if (cf) {
    h = fnv(h, &cf->K, sizeof(cf->K));
    h = fnv(h, &cf->device, sizeof(void*));
    h = fnv(h, &cf->mlp, sizeof(void*));
    if (cf->host) h = fnv(h, cf->host, sizeof(double) * cf->K);
  }
  if (poly) h = fnv(h, poly, sizeof(double) * (degree == 5 ? 3 : 2));
  return h;
}

ifnso_status ensure_meta_host(ifnso_plan* plan, size_t bytes, cudaStream_t stream) {
  if (plan->meta_cap >= bytes) {
    // the previous upload may still read the pinned buffer
    IFNSO_CUDA(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    return IFNSO_OK;
  }
  if (plan->meta_host) {
    IFNSO_CUDA(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    cudaFreeHost(plan->meta_host);
    plan->meta_host = nullptr;
    plan->meta_cap = 0;
  }
  IFNSO_CUDA(cudaMallocHost(&plan->meta_host, bytes), "cudaMallocHost (plan metadata)");
  plan->meta_cap = bytes;
  return IFNSO_OK;
}

// Largest number of two-CTA clusters a pass may use.
int grid_for(const ifnso_plan* plan, size_t items) {
  int g = plan->num_sms;
  if (plan->max_ctas > 0 && plan->max_ctas < g) g = plan->max_ctas;
  g /= 2;
  if (static_cast<size_t>(g) > items) g = static_cast<int>(items);
  return g < 1 ? 1 : g;
}

ifnso_status check_ws(const Layout& ly, void* ws, size_t ws_bytes) {
  if (!ws) return fail(IFNSO_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 1024 != 0) return fail(IFNSO_ERR_WORKSPACE, "workspace is not 1024-byte aligned");
  if (ws_bytes < ly.total)
    return fail(IFNSO_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, ly.total);
  return IFNSO_OK;
}

CUtensorMapDataType bf16_t() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
CUtensorMapDataType f16_t() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

// ---------------------------------------------------------------- IFNSO metadata
ifnso_status build_ifnso_meta(const Layout& ly, const ifnso_batch_desc* b, void* const* out, uint8_t* ws,
                              const double* host_coef, int K, const std::vector<int>& gb, uint8_t* meta,
                              bool on_chip = false) {
  memset(meta, 0, ly.meta_bytes);
  const int n = ly.count;
  MatInfo* mats = reinterpret_cast<MatInfo*>(meta + ly.off_mats);
  for (int i = 0; i < n; ++i) {
    mats[i] = mat_info(ly, b, out, ws, i);
    mats[i].on_chip = (on_chip && ly.shp[i].h <= kSmallH) ? 1 : 0;
  }
  if (host_coef) {
    double* c = reinterpret_cast<double*>(meta + ly.off_coef);
    for (int k = 0; k < K; ++k) c[k] = host_coef[k];
  }
  if (ly.f32) {
    SgProblem* pr = reinterpret_cast<SgProblem*>(meta + ly.off_probs);
    for (int i = 0; i < n; ++i) {
      const Shape& s = ly.shp[i];
      const MatInfo& mi = mats[i];
      const float* in = static_cast<const float*>(mi.in);
      const int64_t hp = s.hpad;
      // Gram: A(i,k) = in[i ld + k] (wide) or in[k ld + i] (tall)
      SgProblem g{};
      g.A = g.B = in;
      g.sa0 = g.sb0 = s.trans ? 1 : s.ld;
      g.sa1 = g.sb1 = s.trans ? s.ld : 1;
      g.a_rows = g.b_rows = static_cast<int32_t>(s.h);
      g.M = g.N = static_cast<int32_t>(hp);
      g.K = static_cast<int32_t>(s.w);
      g.mat = i;
      g.ld_aux = hp;
      g.pacc = mi.gp;
      pr[ly.pi_gram + i] = g;
      for (int par = 0; par < 2; ++par) {
        const float* src = static_cast<const float*>(mi.d[par ? 2 : 0]);
        float* dst = static_cast<float*>(mi.d[par ? 0 : 2]);
        SgProblem q{};
        q.A = q.B = src;
        q.sa0 = q.sb0 = hp;
        q.sa1 = q.sb1 = 1;
        q.a_rows = q.b_rows = static_cast<int32_t>(hp);
        q.M = q.N = q.K = static_cast<int32_t>(hp);
        q.mat = i;
        q.ld_aux = q.ld_out = hp;
        q.aux0 = src;
        q.out0 = dst;
        q.pacc = mi.gp;
        pr[ly.pi_sqr + par * n + i] = q;
      }
      SgProblem a{};
      a.A = mi.gp;  // P (FP32, symmetric)
      a.sa0 = hp;
      a.sa1 = 1;
      a.a_rows = static_cast<int32_t>(s.h);
      a.B = in;
      if (!s.trans) {  // B(n, k) = A[k][n]
        a.sb0 = 1;
        a.sb1 = s.ld;
      } else {  // B(n, k) = M[n][k]
        a.sb0 = s.ld;
        a.sb1 = 1;
      }
      a.b_rows = static_cast<int32_t>(s.w);
      a.M = static_cast<int32_t>(s.h);
      a.N = static_cast<int32_t>(s.w);
      a.K = static_cast<int32_t>(s.h);
      a.mat = i;
      a.out_trans = s.trans;
      a.rows_out = static_cast<int32_t>(s.rows);
      a.cols_out = static_cast<int32_t>(s.cols);
      a.ld_out = s.cols;
      a.out0 = static_cast<float*>(mi.out);
      pr[ly.pi_apply + i] = a;
    }
    return IFNSO_OK;
  }
  TcProblem* pr = reinterpret_cast<TcProblem*>(meta + ly.off_probs);
  for (int i = 0; i < n; ++i) {
    const Shape& s = ly.shp[i];
    const MatInfo& mi = mats[i];
    const int64_t hp = s.hpad;
    // Gram T_0 = A A^T: both operands are the input, K-major when A = M,
    // MN-major when A = M^T (the tall input is read through its own layout).
    TcProblem& g = pr[ly.pi_gram + i];
    bool ok;
    if (ly.e4m3) {
      // the E4M3 copy A s is K-major for either orientation; 128 one-byte values per K block
      ok = encode2d(&g.mapA[0], CU_TENSOR_MAP_DATA_TYPE_UINT8, mi.a8, s.w, s.h, mi.a8ld, 128, 128);
      g.a_mn = g.b_mn = 0;
      g.n_kb = static_cast<int32_t>((s.w + 2 * BK - 1) / (2 * BK));
    } else {
      if (!s.trans) ok = map_k(&g.mapA[0], bf16_t(), mi.in, s.cols, s.rows, s.ld);
      else ok = map_mn(&g.mapA[0], bf16_t(), mi.in, s.cols, s.rows, s.ld);
      g.a_mn = g.b_mn = s.trans;
      g.n_kb = static_cast<int32_t>((s.w + BK - 1) / BK);
    }
    if (!ok) return fail(IFNSO_ERR_CUDA, "cuTensorMapEncodeTiled failed (matrix %d, input)", i);
    g.mapB[0] = g.mapA[0];
    g.mat = i;
    g.ld_aux = hp;
    g.pacc = mi.gp;
    // squarings: src buffer parity par -> dst 1 - par
    for (int par = 0; par < 2; ++par) {
      TcProblem& q = pr[ly.pi_sqr + par * n + i];
      const void* shi = mi.d[2 * par];
      const void* slo = mi.d[2 * par + 1];
      // D_l is symmetric and stored on its upper blocks: A and B rows of a
      // tile read K blocks left of their diagonal block through mapT
      if (!map_k(&q.mapA[0], f16_t(), shi, hp, hp, hp) || !map_mn(&q.mapT[0], f16_t(), shi, hp, hp, hp))
        return fail(IFNSO_ERR_CUDA, "tensor map (D hi)");
      q.mapB[0] = q.mapA[0];
      if (ly.split) {
        if (!map_k(&q.mapA[1], f16_t(), slo, hp, hp, hp) || !map_mn(&q.mapT[1], f16_t(), slo, hp, hp, hp))
          return fail(IFNSO_ERR_CUDA, "tensor map (D lo)");
        q.mapB[1] = q.mapA[1];
      }
      q.sym = kSymA | kSymB;
      q.n_kb = static_cast<int32_t>(hp / BK);
      q.mat = i;
      q.ld_aux = q.ld_out = hp;
      q.aux0 = shi;
      q.aux1 = ly.split ? slo : nullptr;
      q.out0 = mi.d[2 * (1 - par)];
      q.out1 = ly.split ? mi.d[2 * (1 - par) + 1] : nullptr;
      q.pacc = mi.gp;
    }
    // apply: A operand P (BF16 hi/lo in D buffer (L-1) % 2), B operand the input
    TcProblem& a = pr[ly.pi_apply + i];
    const int fb = (ly.L - 1) % 2;
    // P is symmetric and stored on its upper blocks; the FP16 product reads P
    // as one FP16 value and, in place of the input, its FP16 copy M s
    const bool f16 = ly.prec.p_f16 != 0;
    const CUtensorMapDataType pt = f16 ? f16_t() : bf16_t();
    if (!map_k(&a.mapA[0], pt, mi.d[2 * fb], hp, hp, hp) || !map_mn(&a.mapT[0], pt, mi.d[2 * fb], hp, hp, hp))
      return fail(IFNSO_ERR_CUDA, "tensor map (P hi)");
    if (!f16 && ly.split &&
        (!map_k(&a.mapA[1], bf16_t(), mi.d[2 * fb + 1], hp, hp, hp) ||
         !map_mn(&a.mapT[1], bf16_t(), mi.d[2 * fb + 1], hp, hp, hp)))
      return fail(IFNSO_ERR_CUDA, "tensor map (P lo)");
    a.sym = kSymA;
    const void* bsrc = f16 ? mi.a16 : mi.in;
    const int64_t bld = f16 ? mi.a16ld : s.ld;
    if (!s.trans) {
      // Y = P A: B(n, k) = A[k][n], contiguous along n
      ok = map_mn(&a.mapB[0], pt, bsrc, s.cols, s.rows, bld);
      a.b_mn = 1;
      a.out_trans = 0;
    } else {
      // out = M P: computed as (P M^T)^T, B(n, k) = M[n][k], tile stored transposed
      ok = map_k(&a.mapB[0], pt, bsrc, s.cols, s.rows, bld);
      a.b_mn = 0;
      a.out_trans = 1;
    }
    if (!ok) return fail(IFNSO_ERR_CUDA, "tensor map (apply input)");
    a.a_mn = 0;
    a.n_kb = static_cast<int32_t>(hp / BK);
    a.mat = i;
    a.rows_out = static_cast<int32_t>(s.rows);
    a.cols_out = static_cast<int32_t>(s.cols);
    a.ld_out = s.cols;
    a.out0 = mi.out;
    // a Muon step reads the weights where the update goes (M's shape, contiguous)
    a.aux0 = mi.out;
    a.ld_aux = s.cols;
  }
  // the on-chip path's views of every matrix with h <= 128
  SmProblem* sp = reinterpret_cast<SmProblem*>(meta + ly.off_small);
  for (int i = 0; i < n; ++i) {
    const Shape& s = ly.shp[i];
    if (s.h > kSmallH) continue;
    SmProblem& q = sp[i];
    bool ok;
    if (!s.trans) {
      // Gram: M K-major (128 rows x 64 K); product: B(n, k) = M[k][n], MN-major chunks 64 x 64
      ok = encode2d(&q.mapG, bf16_t(), mats[i].in, s.cols, s.rows, s.ld, 64, 128) &&
           encode2d(&q.mapY, bf16_t(), mats[i].in, s.cols, s.rows, s.ld, 64, 64);
    } else {
      // Gram: A = M^T, MN-major chunks 64 x 64; product: B(n, k) = M[n][k], K-major (256 rows x 64 K)
      ok = encode2d(&q.mapG, bf16_t(), mats[i].in, s.cols, s.rows, s.ld, 64, 64) &&
           encode2d(&q.mapY, bf16_t(), mats[i].in, s.cols, s.rows, s.ld, 64, 256);
    }
    if (!ok) return fail(IFNSO_ERR_CUDA, "cuTensorMapEncodeTiled failed (matrix %d, on-chip path)", i);
    q.out = mats[i].out;
    q.ld_out = s.cols;
    q.h = static_cast<int32_t>(s.h);
    q.w = static_cast<int32_t>(s.w);
    q.trans = static_cast<int32_t>(s.trans);
  }
  int32_t* sidx = reinterpret_cast<int32_t*>(meta + ly.off_small_idx);
  for (int i = 0, k = 0; i < n; ++i)
    if (ly.shp[i].h <= kSmallH) sidx[k++] = i;
  std::vector<WorkItem> sy, ap;
  sym_items(ly.shp, gb, sy, nullptr, on_chip);
  app_items(ly.shp, gb, ap, nullptr, on_chip);
  memcpy(meta + ly.off_items_sym, sy.data(), sy.size() * sizeof(WorkItem));
  memcpy(meta + ly.off_items_app, ap.data(), ap.size() * sizeof(WorkItem));
  return IFNSO_OK;
}

// ---------------------------------------------------------------- NS metadata
ifnso_status build_ns_meta(const Layout& ly, const ifnso_batch_desc* b, void* const* out, uint8_t* ws,
                           uint8_t* meta) {
  memset(meta, 0, ly.meta_bytes);
  const int n = ly.count;
  const int steps = ly.steps;
  MatInfo* mats = reinterpret_cast<MatInfo*>(meta + ly.off_mats);
  for (int i = 0; i < n; ++i) mats[i] = mat_info(ly, b, out, ws, i);
  if (!ly.f32) {
    // the on-chip path's views (h <= 128): the input and the two X buffers, M's layout
    SmNsProblem* sp = reinterpret_cast<SmNsProblem*>(meta + ly.off_small_ns);
    for (int i = 0; i < n; ++i) {
      const Shape& s = ly.shp[i];
      if (s.h > kSmallH) continue;
      SmNsProblem& q = sp[i];
      const void* src[3] = {mats[i].in, mats[i].x[0], mats[i].x[1]};
      const int64_t ld[3] = {s.ld, mats[i].xld, mats[i].xld};
      for (int m = 0; m < 3; ++m) {
        bool ok;
        if (!s.trans)
          ok = encode2d(&q.mapG[m], bf16_t(), src[m], s.cols, s.rows, ld[m], 64, 128) &&
               encode2d(&q.mapY[m], bf16_t(), src[m], s.cols, s.rows, ld[m], 64, 64);
        else
          ok = encode2d(&q.mapG[m], bf16_t(), src[m], s.cols, s.rows, ld[m], 64, 64) &&
               encode2d(&q.mapY[m], bf16_t(), src[m], s.cols, s.rows, ld[m], 64, 256);
        if (!ok) return fail(IFNSO_ERR_CUDA, "cuTensorMapEncodeTiled failed (matrix %d, on-chip NS)", i);
      }
      q.out = mats[i].out;
      q.ld_out = s.cols;
      q.h = static_cast<int32_t>(s.h);
      q.w = static_cast<int32_t>(s.w);
      q.trans = static_cast<int32_t>(s.trans);
    }
  }
  auto xcur = [&](int i, int st) -> const void* { return st == 0 ? mats[i].in : mats[i].x[(st - 1) % 2]; };
  auto xcur_ld = [&](int i, int st) -> int64_t { return st == 0 ? ly.shp[i].ld : mats[i].xld; };
  auto xnext = [&](int i, int st) -> void* { return st == steps - 1 ? mats[i].out : mats[i].x[st % 2]; };
  auto xnext_ld = [&](int i, int st) -> int64_t { return st == steps - 1 ? ly.shp[i].cols : mats[i].xld; };
  if (ly.f32) {
    SgProblem* pr = reinterpret_cast<SgProblem*>(meta + ly.off_probs);
    for (int i = 0; i < n; ++i) {
      const Shape& s = ly.shp[i];
      const MatInfo& mi = mats[i];
      const int64_t hp = s.hpad;
      for (int st = 0; st < steps; ++st) {
        const float* X = static_cast<const float*>(xcur(i, st));
        const int64_t xl = xcur_ld(i, st);
        SgProblem g{};
        g.A = g.B = X;
        g.sa0 = g.sb0 = s.trans ? 1 : xl;
        g.sa1 = g.sb1 = s.trans ? xl : 1;
        g.a_rows = g.b_rows = static_cast<int32_t>(s.h);
        g.M = g.N = static_cast<int32_t>(hp);
        g.K = static_cast<int32_t>(s.w);
        g.mat = i;
        g.ld_out = hp;
        g.out0 = static_cast<float*>(mi.s);
        pr[ly.pi_ns_gram + st * n + i] = g;
        SgProblem a{};
        a.A = static_cast<const float*>(mi.b);  // B or S (set at launch through pi)
        a.sa0 = hp;
        a.sa1 = 1;
        a.a_rows = static_cast<int32_t>(s.h);
        a.B = X;
        if (!s.trans) {
          a.sb0 = 1;
          a.sb1 = xl;
        } else {
          a.sb0 = xl;
          a.sb1 = 1;
        }
        a.b_rows = static_cast<int32_t>(s.w);
        a.M = static_cast<int32_t>(s.h);
        a.N = static_cast<int32_t>(s.w);
        a.K = static_cast<int32_t>(s.h);
        a.mat = i;
        a.out_trans = s.trans;
        a.rows_out = static_cast<int32_t>(s.rows);
        a.cols_out = static_cast<int32_t>(s.cols);
        a.ld_out = xnext_ld(i, st);
        a.out0 = static_cast<float*>(xnext(i, st));
        a.aux0 = X;
        a.ld_aux = xl;
        pr[ly.pi_ns_apply + st * n + i] = a;
      }
      SgProblem q{};
      q.A = q.B = static_cast<const float*>(mi.s);
      q.sa0 = q.sb0 = hp;
      q.sa1 = q.sb1 = 1;
      q.a_rows = q.b_rows = static_cast<int32_t>(hp);
      q.M = q.N = q.K = static_cast<int32_t>(hp);
      q.mat = i;
      q.ld_aux = q.ld_out = hp;
      q.aux0 = static_cast<const float*>(mi.s);
      q.out0 = static_cast<float*>(mi.b);
      pr[ly.pi_ns_sqr + i] = q;
    }
    return IFNSO_OK;
  }
  TcProblem* pr = reinterpret_cast<TcProblem*>(meta + ly.off_probs);
  for (int i = 0; i < n; ++i) {
    const Shape& s = ly.shp[i];
    const MatInfo& mi = mats[i];
    const int64_t hp = s.hpad;
    for (int st = 0; st < steps; ++st) {
      const void* X = xcur(i, st);
      const int64_t xl = xcur_ld(i, st);
      TcProblem& g = pr[ly.pi_ns_gram + st * n + i];
      bool ok = !s.trans ? map_k(&g.mapA[0], bf16_t(), X, s.cols, s.rows, xl)
                         : map_mn(&g.mapA[0], bf16_t(), X, s.cols, s.rows, xl);
      if (!ok) return fail(IFNSO_ERR_CUDA, "tensor map (NS X)");
      g.mapB[0] = g.mapA[0];
      g.a_mn = g.b_mn = s.trans;
      g.n_kb = static_cast<int32_t>((s.w + BK - 1) / BK);
      g.mat = i;
      g.ld_out = hp;
      g.out0 = mi.s;
      TcProblem& a = pr[ly.pi_ns_apply + st * n + i];
      // A operand (B or S) filled below per degree; B operand X
      if (!s.trans) {
        ok = map_mn(&a.mapB[0], bf16_t(), X, s.cols, s.rows, xl);
        a.b_mn = 1;
        a.out_trans = 0;
      } else {
        ok = map_k(&a.mapB[0], bf16_t(), X, s.cols, s.rows, xl);
        a.b_mn = 0;
        a.out_trans = 1;
      }
      if (!ok) return fail(IFNSO_ERR_CUDA, "tensor map (NS apply X)");
      a.n_kb = static_cast<int32_t>(hp / BK);
      a.mat = i;
      a.rows_out = static_cast<int32_t>(s.rows);
      a.cols_out = static_cast<int32_t>(s.cols);
      a.ld_out = xnext_ld(i, st);
      a.out0 = xnext(i, st);
      a.aux0 = X;
      a.ld_aux = xl;
    }
    TcProblem& q = pr[ly.pi_ns_sqr + i];
    if (!map_k(&q.mapA[0], bf16_t(), mi.s, hp, hp, hp) || !map_mn(&q.mapT[0], bf16_t(), mi.s, hp, hp, hp))
      return fail(IFNSO_ERR_CUDA, "tensor map (NS S)");
    q.mapB[0] = q.mapA[0];
    q.sym = kSymA | kSymB;
    q.n_kb = static_cast<int32_t>(hp / BK);
    q.mat = i;
    q.ld_aux = q.ld_out = hp;
    q.aux0 = mi.s;
    q.out0 = mi.b;
  }
  std::vector<WorkItem> sy, ap;
  const std::vector<int> all{0, n};
  sym_items(ly.shp, all, sy);
  app_items(ly.shp, all, ap);
  memcpy(meta + ly.off_items_sym, sy.data(), sy.size() * sizeof(WorkItem));
  memcpy(meta + ly.off_items_app, ap.data(), ap.size() * sizeof(WorkItem));
  return IFNSO_OK;
}

// Set the A operand of every NS apply problem to B (quintic) or S (cubic).
ifnso_status ns_set_apply_source(const Layout& ly, uint8_t* meta, int use_b) {
  const int n = ly.count;
  MatInfo* mats = reinterpret_cast<MatInfo*>(meta + ly.off_mats);
  if (ly.f32) {
    SgProblem* pr = reinterpret_cast<SgProblem*>(meta + ly.off_probs);
    for (int st = 0; st < ly.steps; ++st)
      for (int i = 0; i < n; ++i)
        pr[ly.pi_ns_apply + st * n + i].A = static_cast<const float*>(use_b ? mats[i].b : mats[i].s);
    return IFNSO_OK;
  }
  TcProblem* pr = reinterpret_cast<TcProblem*>(meta + ly.off_probs);
  for (int i = 0; i < n; ++i) {
    const int64_t hp = ly.shp[i].hpad;
    CUtensorMap m, mt;
    const void* src = use_b ? mats[i].b : mats[i].s;
    if (!map_k(&m, bf16_t(), src, hp, hp, hp) || !map_mn(&mt, bf16_t(), src, hp, hp, hp))
      return fail(IFNSO_ERR_CUDA, "tensor map (NS apply operand)");
    for (int st = 0; st < ly.steps; ++st) {
      TcProblem& a = pr[ly.pi_ns_apply + st * n + i];
      a.mapA[0] = m;
      a.mapT[0] = mt;
      a.sym = kSymA;  // B and S are symmetric, stored on their upper blocks
    }
  }
  return IFNSO_OK;
}

ifnso_status init_plan_device(ifnso_plan* p) {
  if (p->num_sms > 0) return IFNSO_OK;
  int dev = 0;
  IFNSO_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  cudaDeviceProp prop;
  IFNSO_CUDA(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
  if (p->dtype == IFNSO_BF16 && prop.major * 10 + prop.minor < 100)
    return fail(IFNSO_ERR_UNSUPPORTED, "BF16 plans need a tcgen05 GPU (sm_100 family), found sm_%d%d", prop.major, prop.minor);
  p->num_sms = prop.multiProcessorCount;
  return IFNSO_OK;
}

template <class Params>
Params base_params(uint8_t* ws, const Layout& ly, const ifnso_coeffs* cf) {
  Params p{};
  p.scal = reinterpret_cast<MatScalars*>(ws + ly.off_scal);
  p.coef.K = cf ? cf->K : 0;
  if (cf && cf->device) {
    p.coef.f32 = cf->device;
    p.coef.stride = cf->K;
  } else if (cf && cf->mlp) {
    p.coef.f32 = reinterpret_cast<const float*>(ws + ly.off_rows);
    p.coef.stride = kRowSlots;
  } else {
    p.coef.d64 = reinterpret_cast<const double*>(ws + ly.off_coef);
  }
  return p;
}

// Philox4x32-10 word pair -> two N(0,1) values (Box-Muller), for the
// network's initial parameters.
void host_philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c[0];
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c[2];
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c[3] ^ k1;
    c[1] = static_cast<uint32_t>(p1);
    c[3] = static_cast<uint32_t>(p0);
    c[0] = n0;
    c[2] = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

double host_normal(uint32_t seed, uint32_t i) {
  uint32_t c[4] = {i, 0u, 0u, 0u};
  host_philox(c, seed, 0x4D4C5049u);
  const double u1 = (static_cast<double>(c[0] >> 8) + 0.5) / 16777216.0;
  const double u2 = (static_cast<double>(c[1] >> 8) + 0.5) / 16777216.0;
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

struct ifnso_mlp {
  int K = 0, L = 0, P = 0;
  float* prm = nullptr;     // device parameters
  float* mom = nullptr;     // Adam first moments
  float* vel = nullptr;     // Adam second moments
  float* wfix = nullptr;    // device w_1..w_L (FP32)
  float* wslots = nullptr;  // device (1, w_1..w_L): the fixed coefficients as a coefficient row
  float* scale = nullptr;   // device s_l
  float* stats = nullptr;   // device 6 means, 6 standard deviations
  int step = 0;
  int n = 0;
  float* xs = nullptr;
  float* raw = nullptr;
  float* z = nullptr;
  int64_t* offs = nullptr;
  int32_t* hs = nullptr;
  int cap_batch = 0;
  int32_t* idx = nullptr;
  float* grad_part = nullptr;
  float* loss_part = nullptr;
  float* grad = nullptr;
  std::mutex mu;
};

namespace {

void mlp_free_data(ifnso_mlp* m) {
  cudaFree(m->xs);
  cudaFree(m->raw);
  cudaFree(m->z);
  cudaFree(m->offs);
  cudaFree(m->hs);
  m->xs = m->raw = m->z = nullptr;
  m->offs = nullptr;
  m->hs = nullptr;
  m->n = 0;
}

ifnso_status mlp_ensure_batch(ifnso_mlp* m, int batch) {
  if (m->cap_batch >= batch) return IFNSO_OK;
  cudaFree(m->idx);
  cudaFree(m->grad_part);
  cudaFree(m->loss_part);
  const int blocks = (batch + 31) / 32;
  IFNSO_CUDA(cudaMalloc(&m->idx, sizeof(int32_t) * batch), "cudaMalloc");
  IFNSO_CUDA(cudaMalloc(&m->grad_part, sizeof(float) * static_cast<size_t>(blocks) * m->P), "cudaMalloc");
  IFNSO_CUDA(cudaMalloc(&m->loss_part, sizeof(float) * blocks), "cudaMalloc");
  m->cap_batch = batch;
  return IFNSO_OK;
}

// Arguments of an IFNSO call (shapes into shp).
ifnso_status check_call(const ifnso_plan* plan, const ifnso_batch_desc* batch, const ifnso_coeffs* coeffs,
                        void* const* out, std::vector<Shape>& shp) {
  ifnso_status st = read_batch(plan, batch, shp);
  if (st != IFNSO_OK) return st;
  if (!coeffs || coeffs->K != plan->L + 1 ||
      (coeffs->host ? 1 : 0) + (coeffs->device ? 1 : 0) + (coeffs->mlp ? 1 : 0) != 1)
    return fail(IFNSO_ERR_INVALID_ARG, "coefficients: need K = %d and exactly one of host/device/mlp", plan->L + 1);
  if (coeffs->mlp) {
    if (coeffs->mlp->K != coeffs->K) return fail(IFNSO_ERR_INVALID_ARG, "coefficient network has K = %d", coeffs->mlp->K);
    if (plan->L < 3) return fail(IFNSO_ERR_INVALID_ARG, "proposed coefficients need L >= 3");
    if (plan->dtype != IFNSO_BF16) return fail(IFNSO_ERR_UNSUPPORTED, "proposed coefficients need a BF16 plan");
    if (plan->scale == IFNSO_SCALE_GELFAND2)
      return fail(IFNSO_ERR_UNSUPPORTED, "proposed coefficients are trained on features under Gram scaling");
  }
  if (!out) return fail(IFNSO_ERR_INVALID_ARG, "out is NULL");
  for (int i = 0; i < batch->count; ++i) {
    if (!out[i]) return fail(IFNSO_ERR_INVALID_ARG, "out[%d] is NULL", i);
    if (out[i] == batch->in[i]) return fail(IFNSO_ERR_INVALID_ARG, "out[%d] aliases the input", i);
    if (reinterpret_cast<uintptr_t>(out[i]) % 16 != 0)
      return fail(IFNSO_ERR_INVALID_ARG, "out[%d] is not 16-byte aligned", i);
  }
  return IFNSO_OK;
}

// Copy streams and events of ifnso_orthogonalize_host (created on first use).
ifnso_status ensure_copy_streams(ifnso_plan* plan, int groups) {
  if (!plan->s_in) {
    IFNSO_CUDA(cudaStreamCreateWithFlags(&plan->s_in, cudaStreamNonBlocking), "cudaStreamCreate");
    IFNSO_CUDA(cudaStreamCreateWithFlags(&plan->s_out, cudaStreamNonBlocking), "cudaStreamCreate");
    IFNSO_CUDA(cudaStreamCreateWithFlags(&plan->s_comp, cudaStreamNonBlocking), "cudaStreamCreate");
    IFNSO_CUDA(cudaEventCreateWithFlags(&plan->ev_start, cudaEventDisableTiming), "cudaEventCreate");
    IFNSO_CUDA(cudaEventCreateWithFlags(&plan->ev_last, cudaEventDisableTiming), "cudaEventCreate");
  }
  for (auto* v : {&plan->ev_in, &plan->ev_done})
    while (static_cast<int>(v->size()) < groups) {
      cudaEvent_t e;
      IFNSO_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
      v->push_back(e);
    }
  if (plan->timing) {
    if (!plan->tl_start) IFNSO_CUDA(cudaEventCreate(&plan->tl_start), "cudaEventCreate");
    while (static_cast<int>(plan->tl_ev.size()) < 3 * groups) {
      cudaEvent_t e;
      IFNSO_CUDA(cudaEventCreate(&e), "cudaEventCreate");
      plan->tl_ev.push_back(e);
    }
  }
  return IFNSO_OK;
}

// Which plan last uploaded metadata into each workspace, with its signature:
// a plan re-uploads when another plan's call has used the same workspace
// since its own last upload (its cached signature alone would not show it).
std::mutex g_ws_mu;
std::unordered_map<const void*, std::pair<const ifnso_plan*, uint64_t>> g_ws_owner;

bool ws_current(const void* ws, const ifnso_plan* plan, uint64_t sig) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  auto it = g_ws_owner.find(ws);
  return it != g_ws_owner.end() && it->second.first == plan && it->second.second == sig;
}

void ws_claim(const void* ws, const ifnso_plan* plan, uint64_t sig) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  g_ws_owner[ws] = {plan, sig};
}

void ws_forget(const ifnso_plan* plan) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  for (auto it = g_ws_owner.begin(); it != g_ws_owner.end();)
    it = it->second.first == plan ? g_ws_owner.erase(it) : std::next(it);
}

// Build and upload the metadata of an IFNSO call unless the cached copy
// already describes it (item lists grouped by gb).
ifnso_status upload_ifnso_meta(ifnso_plan* plan, const Layout& ly, const ifnso_batch_desc* batch, void* const* out,
                               uint8_t* ws, const ifnso_coeffs* coeffs, const std::vector<int>& gb,
                               cudaStream_t stream, bool on_chip = false) {
  const int groups = static_cast<int>(gb.size()) - 1;
  const uint64_t sig = batch_sig(plan, batch, out, ws, coeffs, nullptr, 0, 0, (on_chip ? 2000000 : 1000) + groups);
  if (plan->sig_valid && plan->sig == sig && ws_current(ws, plan, sig)) return IFNSO_OK;
  ifnso_status st;
  if ((st = ensure_meta_host(plan, ly.meta_bytes, stream)) != IFNSO_OK) return st;
  uint8_t* meta = static_cast<uint8_t*>(plan->meta_host);
  if ((st = build_ifnso_meta(ly, batch, out, ws, coeffs->host, coeffs->K, gb, meta, on_chip)) != IFNSO_OK) return st;
  IFNSO_CUDA(cudaMemcpyAsync(ws, meta, ly.meta_bytes, cudaMemcpyHostToDevice, stream), "metadata upload");
  plan->small_idx.clear();
  for (int i = 0; i < ly.count; ++i)
    if (ly.shp[i].h <= kSmallH) plan->small_idx.push_back(i);
  std::vector<WorkItem> tmp;
  sym_items(ly.shp, gb, tmp, &plan->sym_off, on_chip);
  tmp.clear();
  app_items(ly.shp, gb, tmp, &plan->app_off, on_chip);
  plan->sig = sig;
  plan->sig_valid = true;
  plan->groups = groups;
  ws_claim(ws, plan, sig);
  return IFNSO_OK;
}

// What the passes of one IFNSO call share.
struct Run {
  ifnso_plan* plan;
  const Layout* ly;
  uint8_t* ws;
  const ifnso_coeffs* coeffs;
  int hpad_max;
  cudaStream_t stream;
  bool whole;  // the whole batch in one go: per-pass timing events and IFNSO_OPT_STOP_AFTER apply
  bool update = false;  // the product updates weights in place: W <- W - lr s Y (ifnso_muon_step)
  float lr = 0.f;
  bool on_chip = false;  // the on-chip path computes the matrices with h <= 128 (use_small)
};

// Coefficient rows of matrix `first` onwards (the SIMT kernels index a group from 0).
CoefTable shifted(CoefTable t, int first) {
  if (t.f32) t.f32 += static_cast<int64_t>(first) * t.stride;
  return t;
}

// FP32 plans: every pass of Algorithm 1 on the whole batch with the SIMT kernels.
ifnso_status run_f32(const Run& r) {
  ifnso_plan* plan = r.plan;
  const Layout& ly = *r.ly;
  uint8_t* ws = r.ws;
  cudaStream_t stream = r.stream;
  const int n = ly.count;
  const int L = ly.L;
  const int frob = plan->scale == IFNSO_SCALE_FROB;
  MatInfo* d_mats = reinterpret_cast<MatInfo*>(ws + ly.off_mats);
  IFNSO_CUDA(cudaMemsetAsync(ws + ly.off_scal, 0, n * sizeof(MatScalars), stream), "scalar reset");
  IFNSO_CUDA(mark(plan, stream, true), "timing event");
  SgParams p = base_params<SgParams>(ws, ly, r.coeffs);
  const SgProblem* probs = reinterpret_cast<const SgProblem*>(ws + ly.off_probs);
  int max_h = 0, max_w = 0;
  for (auto& s : ly.shp) {
    max_h = std::max<int>(max_h, static_cast<int>(s.h));
    max_w = std::max<int>(max_w, static_cast<int>(s.w));
  }
  // the Gram is computed over the whole padded h_pad x h_pad block (zeros beyond h)
  p.probs = probs + ly.pi_gram;
  IFNSO_CUDA(sg_launch(EPI_GRAM, p, n, r.hpad_max, r.hpad_max, stream), "FP32 Gram");
  IFNSO_CUDA(launch_scalars(d_mats, n, p.scal, p.coef, L, frob, 0, stream), "scalars");
  IFNSO_CUDA(mark(plan, stream, false), "timing event");
  if (plan->stop_after == 0) return IFNSO_OK;
  if (plan->scale == IFNSO_SCALE_GELFAND2) {
    // Gelfand's bound with q = 2: D_1 under o = ||T_0||_F (T_0 kept), the
    // FP64 sum of (D_1^2)_ij^2, and o rescaled to ||T_0^2||_F^(1/2)
    IFNSO_CUDA(launch_prep(d_mats, n, r.hpad_max, p.scal, p.coef, L, 0, 1, stream, 1), "Gelfand prep");
    p.probs = probs + ly.pi_sqr;
    IFNSO_CUDA(sg_launch(EPI_SQR_NORM, p, n, r.hpad_max, r.hpad_max, stream), "Gelfand norm pass");
    IFNSO_CUDA(launch_gelfand(n, p.scal, stream), "Gelfand scale");
  }
  IFNSO_CUDA(launch_prep(d_mats, n, r.hpad_max, p.scal, p.coef, L, 0, 1, stream), "prep");
  IFNSO_CUDA(mark(plan, stream, false), "timing event");
  if (plan->stop_after == 1) return IFNSO_OK;
  for (int j = 1; j <= L - 1; ++j) {
    const int par = (j - 1) % 2;
    p.probs = probs + ly.pi_sqr + par * n;
    p.coef_l = j + 1;
    p.final_pass = (j == L - 1);
    IFNSO_CUDA(sg_launch(EPI_SQR, p, n, r.hpad_max, r.hpad_max, stream), "FP32 squaring");
    IFNSO_CUDA(mark(plan, stream, false), "timing event");
    if (plan->stop_after == 1 + j) return IFNSO_OK;
  }
  p.probs = probs + ly.pi_apply;
  p.coef_l = 0;
  p.final_pass = 0;
  IFNSO_CUDA(sg_launch(EPI_APPLY, p, n, max_h, max_w, stream), "FP32 apply");
  IFNSO_CUDA(mark(plan, stream, false), "timing event");
  return IFNSO_OK;
}

// The on-chip path (small.cu) takes the matrices with h <= 128 of a call
// that needs nothing it does not do: the proposal network inside the call,
// Gelfand's q = 2 bound, the E4M3 Gram, the fused Muon update and the
// testing aids stay on the tiled passes.  In a batch that mixes sizes the
// tiled passes skip those matrices (no work items; the scalar and set-up
// kernels see their MatInfo flag).
bool small_applies(const ifnso_plan* plan, const Layout& ly, const ifnso_coeffs* coeffs, bool update) {
  if (ly.f32 || ly.ns || ly.e4m3 || update || plan->stop_after >= 0 || plan->inject_stall) return false;
  if (plan->scale == IFNSO_SCALE_GELFAND2 || (coeffs && coeffs->mlp)) return false;
  if (ly.L > 30) return false;
  for (const Shape& s : ly.shp)
    if (s.h <= kSmallH) return true;
  return false;
}

bool use_small(const ifnso_plan* plan, const Layout& ly, const ifnso_coeffs* coeffs, bool update) {
  if (plan->small == 2 || !small_applies(plan, ly, coeffs, update)) return false;
  if (plan->small == 1) return true;
  return plan->small_tuned != 2;
}

// The on-chip kernel over matrices first .. first + count - 1 (all with
// h <= 128), or over the n_idx matrices listed at d_idx.
cudaError_t launch_on_chip(const Run& r, int first, int count, const int32_t* d_idx) {
  const Layout& ly = *r.ly;
  const TcParams base = base_params<TcParams>(r.ws, ly, r.coeffs);
  SmParams p{};
  p.probs = reinterpret_cast<const SmProblem*>(r.ws + ly.off_small);
  p.idx = d_idx;
  p.scal = base.scal;
  p.coef = base.coef;
  p.first = first;
  p.L = ly.L;
  p.k_split = ly.prec.k_split;
  p.p_split = ly.prec.chip_p_split;
  p.frob = r.plan->scale == IFNSO_SCALE_FROB;
  p.wait_ms = static_cast<uint32_t>(r.plan->wait_ms);
  return launch_small(p, count, r.stream);
}

// A range of matrices that all have h <= 128: one launch, timed as one pass.
ifnso_status run_small(const Run& r, int first, int count) {
  ifnso_plan* plan = r.plan;
  const Layout& ly = *r.ly;
  IFNSO_CUDA(cudaMemsetAsync(r.ws + ly.off_scal + first * sizeof(MatScalars), 0, count * sizeof(MatScalars),
                             r.stream),
             "scalar reset");
  if (r.whole) IFNSO_CUDA(mark(plan, r.stream, true), "timing event");
  IFNSO_CUDA(launch_on_chip(r, first, count, nullptr), "on-chip pass");
  if (r.whole) IFNSO_CUDA(mark(plan, r.stream, false), "timing event");
  return IFNSO_OK;
}

// BF16 plans: every pass of Algorithm 1 for matrices [first, first + count),
// whose work items are [sym0, sym1) and [app0, app1) of the metadata's lists.
ifnso_status run_tc(const Run& r, int first, int count, size_t sym0, size_t sym1, size_t app0, size_t app1) {
  ifnso_plan* plan = r.plan;
  const Layout& ly = *r.ly;
  if (r.on_chip) {
    bool all = true;
    for (int i = first; i < first + count; ++i) all = all && ly.shp[i].h <= kSmallH;
    if (all) return run_small(r, first, count);
  }
  uint8_t* ws = r.ws;
  cudaStream_t stream = r.stream;
  const int L = ly.L;
  const int frob = plan->scale == IFNSO_SCALE_FROB;
  const bool whole = r.whole;
  MatInfo* d_mats = reinterpret_cast<MatInfo*>(ws + ly.off_mats) + first;
  IFNSO_CUDA(cudaMemsetAsync(ws + ly.off_scal + first * sizeof(MatScalars), 0, count * sizeof(MatScalars), stream),
             "scalar reset");
  auto mark_pass = [&](bool start) { return whole ? mark(plan, stream, start) : cudaSuccess; };
  auto stop = [&](int stage) { return whole && plan->stop_after == stage; };
  IFNSO_CUDA(mark_pass(true), "timing event");
  if (r.on_chip) {
    // the matrices with h <= 128 in this range, on chip (timed with the Gram pass)
    const auto& si = plan->small_idx;
    const auto lo = std::lower_bound(si.begin(), si.end(), first);
    const auto hi = std::lower_bound(si.begin(), si.end(), first + count);
    if (hi > lo) {
      const int32_t* d_idx = reinterpret_cast<const int32_t*>(ws + ly.off_small_idx) + (lo - si.begin());
      IFNSO_CUDA(launch_on_chip(r, 0, static_cast<int>(hi - lo), d_idx), "on-chip pass");
    }
  }
  TcParams p = base_params<TcParams>(ws, ly, r.coeffs);
  // the tensor-core passes address scalars and coefficient rows by matrix
  // index; the SIMT kernels by position in the group
  MatScalars* scal = p.scal + first;
  const CoefTable coef = shifted(p.coef, first);
  const TcProblem* probs = reinterpret_cast<const TcProblem*>(ws + ly.off_probs);
  const WorkItem* sym = reinterpret_cast<const WorkItem*>(ws + ly.off_items_sym) + sym0;
  const WorkItem* app = reinterpret_cast<const WorkItem*>(ws + ly.off_items_app) + app0;
  const size_t n_sym = sym1 - sym0, n_app = app1 - app0;
  const int n = ly.count;
  const Prec& pc = ly.prec;
  p.p_split = pc.p_split;
  p.p_f16 = pc.p_f16;
  p.wait_ms = static_cast<uint32_t>(plan->wait_ms);
  // automatic: the autotuned mode of each pass kind, else MMAs of the CTA pair
  // for the split squarings (three products per stage hide the pair's
  // handshakes) and per-CTA MMAs for every other pass
  auto cta_group = [&](int kind) {
    if (plan->cta_group) return plan->cta_group;
    if (plan->tuned) return plan->cg_kind[kind];
    return kind == kSplit ? 2 : 1;
  };
  p.cta_group = cta_group(kGram);
  p.max_stages = plan->stage_lim[kGram];
  p.probs = probs + ly.pi_gram;
  p.items = sym;
  p.n_items = static_cast<int32_t>(n_sym);
  p.inject = plan->inject_stall;
  if (ly.e4m3) {
    int max_h = 0, max_w = 0;
    for (int i = first; i < first + count; ++i) {
      max_h = std::max<int>(max_h, static_cast<int>(ly.shp[i].h));
      max_w = std::max<int>(max_w, static_cast<int>(ly.shp[i].w));
    }
    IFNSO_CUDA(launch_amax(d_mats, count, scal, std::max(1, 16 * plan->num_sms / count), stream), "max |A|");
    IFNSO_CUDA(launch_cast_e4m3(d_mats, count, max_h, max_w, scal, stream), "E4M3 copy of A");
  }
  IFNSO_CUDA(tc_launch(ly.e4m3 ? EPI_GRAM_F8 : EPI_GRAM, 1, 1, p, grid_for(plan, n_sym), stream), "Gram pass");
  p.inject = 0;
  const ifnso_mlp* net = r.coeffs->mlp;
  if (net) {
    // until the network has spoken, the scalars see the fixed coefficients
    CoefTable fixed{nullptr, net->wslots, r.coeffs->K, 0};
    IFNSO_CUDA(launch_scalars(d_mats, count, scal, fixed, L, frob, 0, stream), "scalars");
  } else {
    IFNSO_CUDA(launch_scalars(d_mats, count, scal, coef, L, frob, 0, stream), "scalars");
  }
  IFNSO_CUDA(mark_pass(false), "timing event");
  if (stop(0)) return IFNSO_OK;
  if (plan->scale == IFNSO_SCALE_GELFAND2) {
    // Gelfand's bound with q = 2: D_1 under o = ||T_0||_F (FP16 hi), then
    // ||D_1^2||_F^2 from one product of it with itself (nothing stored), and
    // o rescaled to ||T_0^2||_F^(1/2); the prep below then divides T_0 by that
    IFNSO_CUDA(launch_prep(d_mats, count, r.hpad_max, scal, coef, L, 0, 0, stream, 1), "Gelfand prep");
    p.probs = probs + ly.pi_sqr;  // squaring 1 reads D buffer 0
    p.cta_group = cta_group(kPlain);
    p.max_stages = 0;
    IFNSO_CUDA(tc_launch(EPI_SQR_NORM, 1, 1, p, grid_for(plan, n_sym), stream), "Gelfand norm pass");
    IFNSO_CUDA(launch_gelfand(count, scal, stream), "Gelfand scale");
  }
  // prep stores D_1 as hi + lo when the first squaring is split (for L = 1: P as hi + lo);
  // with fixed coefficients it also starts P = c_0 I - w_1 D_1
  const int prep_lo = L == 1 ? pc.p_split : (pc.k_split >= 1 ? 1 : 0);
  IFNSO_CUDA(launch_prep(d_mats, count, r.hpad_max, scal, coef, L, prep_lo, 0, stream, 0, net ? 0 : 1), "prep");
  // The FP16 copy M s that the final product reads (s from tr T_0) is written
  // by the side warps of the squarings that the tensor pipe bounds -- the
  // split ones, or every squaring when fewer than three are split -- each
  // writing an equal part of the copies' pieces, matrix after matrix.  Its
  // own HBM-bound kernel writes it here instead when those passes would not
  // hide it: a grid short of the GPU, a matrix of 2^31 pieces or more, or
  // passes too short for the copy (estimated from its reads at 0.5 TB/s
  // against the host passes' products at 1.6 PFLOP/s, with a margin of 0.6).
  int side_hosts = 0;
  if (pc.p_f16) {
    const int hosts = pc.k_split >= 3 ? pc.k_split : L - 1;
    double rd = 0.0, fl = 0.0;
    bool fits = 2 * grid_for(plan, n_sym) >= plan->num_sms;
    for (int i = first; i < first + count; ++i) {
      const Shape& s = ly.shp[i];
      if (r.on_chip && s.h <= kSmallH) continue;
      rd += 2.0 * static_cast<double>(s.rows) * static_cast<double>(s.cols);
      fits = fits && static_cast<uint64_t>(s.rows) * static_cast<uint64_t>((s.cols + 7) / 8) < (1ull << 31);
      const double nb = static_cast<double>(s.hpad / 256);
      fl += nb * (nb + 1.0) / 2.0 * 2.0 * 256.0 * 256.0 * static_cast<double>(s.hpad);
    }
    const int prods = pc.k_split >= 3 ? 3 : 1;
    if (fits && hosts >= 1 && rd / hosts / 0.5e12 < 0.6 * prods * fl / 1.6e15) side_hosts = hosts;
    if (!side_hosts)
      IFNSO_CUDA(launch_cast_f16(d_mats, count, scal, std::max(1, 16 * plan->num_sms / count), stream), "FP16 copy");
  }
  plan->copy_hosts = side_hosts;
  IFNSO_CUDA(mark_pass(false), "timing event");
  if (stop(1)) return IFNSO_OK;
  for (int j = 1; j <= L - 1; ++j) {
    const int par = (j - 1) % 2;
    const int split = j <= pc.k_split ? 1 : 0;
    p.probs = probs + ly.pi_sqr + par * n;
    p.items = sym;
    p.n_items = static_cast<int32_t>(n_sym);
    p.coef_l = j + 1;
    p.final_pass = (j == L - 1);
    p.read_lo = split;
    p.write_lo = (j + 1 <= pc.k_split) ? 1 : 0;
    p.cta_group = cta_group(split ? kSplit : kPlain);
    p.max_stages = plan->stage_lim[j == L - 1 ? kFinal : (split ? kSplit : kPlain)];
    if (!net) {
      // every squaring folds -2 D_j into its MMAs and adds its own term
      // -w_{j+1} D_{j+1}, from the FP32 accumulator, to P (started by prep);
      // none reads D_j in its epilogue
      p.p_mode = 3;
      p.feat = 0;
    } else {
      // proposed coefficients: squaring 1 only measures tr(D_1^4); squaring 2
      // writes P from T_0, D_2 and D_3; even squarings add D_j and D_{j+1};
      // an odd last squaring adds D_L
      p.p_mode = j == 1 ? 0 : (j == 2 ? 4 : ((j & 1) == 0 ? 2 : (j == L - 1 ? 3 : 0)));
      p.feat = j == 1 ? 1 : 0;
    }
    // passes whose P update has no D_l term take 2 D_l - D_l^2 from the MMAs
    // (the feature pass needs D_l^2 itself)
    p.fold_d = ((p.p_mode == 0 || p.p_mode == 3) && !p.feat) ? 1 : 0;
    if (j <= side_hosts) {
      // this squaring's part of the FP16 copies
      p.side_mats = d_mats;
      p.side_scal = scal;
      p.side_count = count;
      p.side_part = j - 1;
      p.side_parts = side_hosts;
    } else {
      p.side_mats = nullptr;
      p.side_scal = nullptr;
      p.side_count = 0;
    }
    IFNSO_CUDA(tc_launch(EPI_SQR, split ? 2 : 1, split ? 2 : 1, p, grid_for(plan, n_sym), stream), "squaring pass");
    if (net && j == 1) {
      IFNSO_CUDA(mlp_infer(net->prm, net->K, net->wfix, net->scale, net->stats, d_mats, scal, count,
                           reinterpret_cast<float*>(ws + ly.off_rows) + static_cast<int64_t>(first) * kRowSlots,
                           kRowSlots, stream),
                 "coefficient proposal");
    }
    IFNSO_CUDA(mark_pass(false), "timing event");
    if (stop(1 + j)) return IFNSO_OK;
  }
  p.side_mats = nullptr;
  p.side_scal = nullptr;
  p.side_count = 0;
  p.probs = probs + ly.pi_apply;
  p.items = app;
  p.n_items = static_cast<int32_t>(n_app);
  p.coef_l = 0;
  p.final_pass = 0;
  p.read_lo = p.write_lo = 0;
  p.fold_d = 0;
  p.update = r.update ? 1 : 0;
  p.lr = r.lr;
  p.cta_group = cta_group(kApply);
  p.max_stages = plan->stage_lim[kApply];
  IFNSO_CUDA(tc_launch(pc.p_f16 ? EPI_APPLY_F16 : EPI_APPLY, pc.p_split ? 2 : 1, 1, p, grid_for(plan, n_app), stream),
             "apply pass");
  IFNSO_CUDA(mark_pass(false), "timing event");
  return IFNSO_OK;
}

// ifnso_pass_times with the plan's mutex held.
ifnso_status pass_times_locked(ifnso_plan* plan, double* ms_out, int32_t max_passes, int32_t* n_passes,
                               int32_t* n_calls) {
  for (int k = 0; k < max_passes; ++k) ms_out[k] = 0.0;
  *n_passes = 0;
  int ncalls = 0;
  // eager calls since the last query, then each captured call once (its
  // events hold the durations of the graph's latest replay)
  for (auto* list : {&plan->ev_calls, &plan->ev_graph}) {
    for (auto& c : *list) {
      if (c.size() < 2) continue;
      if (list == &plan->ev_graph) {
        // a captured call whose graph has not been replayed yet has no times
        float probe = 0.f;
        cudaError_t e = cudaEventSynchronize(c.back());
        if (e == cudaSuccess) e = cudaEventElapsedTime(&probe, c.front(), c.back());
        if (e != cudaSuccess) {
          (void)cudaGetLastError();  // not sticky: clear it
          continue;
        }
      }
      IFNSO_CUDA(cudaEventSynchronize(c.back()), "cudaEventSynchronize");
      const int np = static_cast<int>(c.size()) - 1;
      *n_passes = np;
      ++ncalls;
      for (int k = 0; k < np && k < max_passes; ++k) {
        float ms = 0.f;
        IFNSO_CUDA(cudaEventElapsedTime(&ms, c[k], c[k + 1]), "cudaEventElapsedTime");
        ms_out[k] += ms;
      }
    }
  }
  if (n_calls) *n_calls = ncalls;
  for (auto& c : plan->ev_calls)
    for (cudaEvent_t e : c) plan->ev_pool.push_back(e);
  plan->ev_calls.clear();
  return IFNSO_OK;
}

// ifnso_orthogonalize with the plan's mutex held.
ifnso_status orthogonalize_locked(ifnso_plan* plan, const ifnso_batch_desc* batch, const ifnso_coeffs* coeffs,
                                  void* const* out, void* workspace, size_t workspace_bytes, cudaStream_t stream,
                                  bool update = false, float lr = 0.f) {
  std::vector<Shape> shp;
  ifnso_status st = check_call(plan, batch, coeffs, out, shp);
  if (st != IFNSO_OK || batch->count == 0) return st;
  if ((st = init_plan_device(plan)) != IFNSO_OK) return st;
  Layout ly = make_layout(plan, shp, 0, 0, plan->L + 1);
  if ((st = check_ws(ly, workspace, workspace_bytes)) != IFNSO_OK) return st;
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  const bool on_chip = use_small(plan, ly, coeffs, update);
  if ((st = upload_ifnso_meta(plan, ly, batch, out, ws, coeffs, {0, ly.count}, stream, on_chip)) != IFNSO_OK)
    return st;
  int hpad_max = 0;
  for (auto& sh : shp) hpad_max = std::max<int>(hpad_max, static_cast<int>(sh.hpad));
  Run r{plan, &ly, ws, coeffs, hpad_max, stream, true};
  r.update = update;
  r.lr = lr;
  r.on_chip = on_chip;
  if (ly.f32) return run_f32(r);
  // the item counts of the uploaded lists (without the on-chip path's matrices)
  return run_tc(r, 0, ly.count, 0, plan->sym_off.back(), 0, plan->app_off.back());
}

}  // namespace

void ifnso::count_launch(int n) { g_launches += static_cast<uint64_t>(n); }

void ifnso::set_last_error(const char* msg) { g_err = msg; }

// ====================================================================== C ABI
extern "C" {

const char* ifnso_last_error(void) { return g_err.c_str(); }

uint64_t ifnso_launch_count(void) { return g_launches.load(); }

ifnso_status ifnso_plan_create(ifnso_plan** plan, int64_t h, int64_t w, ifnso_dtype dtype,
                               const int32_t* exponents, int32_t K) {
  if (!plan) return fail(IFNSO_ERR_INVALID_ARG, "plan is NULL");
  *plan = nullptr;
  if (h <= 0 || w <= 0 || h > w)
    return fail(IFNSO_ERR_INVALID_ARG, "plan shape %lldx%lld must satisfy 0 < h <= w", (long long)h, (long long)w);
  if (dtype != IFNSO_F32 && dtype != IFNSO_BF16) return fail(IFNSO_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
  if (K < 2 || K > 31 || !exponents) return fail(IFNSO_ERR_INVALID_ARG, "K = %d must be in [2, 31]", K);
  if (exponents[0] != 0) return fail(IFNSO_ERR_INVALID_ARG, "exponents[0] must be 0");
  for (int k = 1; k < K; ++k)
    if (exponents[k] != (1 << (k - 1)))
      return fail(IFNSO_ERR_INVALID_ARG,
                  "exponents[%d] = %d: repeated squaring produces only 0, 1, 2, 4, ... (exponents[k] = 2^(k-1))", k,
                  exponents[k]);
  ifnso_plan* p = new (std::nothrow) ifnso_plan();
  if (!p) return fail(IFNSO_ERR_OOM, "out of host memory");
  p->h = h;
  p->w = w;
  p->dtype = dtype;
  p->L = K - 1;
  *plan = p;
  return IFNSO_OK;
}

ifnso_status ifnso_plan_set(ifnso_plan* plan, ifnso_option option, int64_t value) {
  if (!plan) return fail(IFNSO_ERR_INVALID_ARG, "plan is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  switch (option) {
    case IFNSO_OPT_PRECISION:
      if (value < 0 || value > 3) return fail(IFNSO_ERR_INVALID_ARG, "precision %lld", (long long)value);
      plan->precision = static_cast<int>(value);
      break;
    case IFNSO_OPT_SCALE:
      if (value < 0 || value > 2) return fail(IFNSO_ERR_INVALID_ARG, "scale %lld", (long long)value);
      plan->scale = static_cast<int>(value);
      break;
    case IFNSO_OPT_MAX_CTAS:
      if (value < 0) return fail(IFNSO_ERR_INVALID_ARG, "max ctas %lld", (long long)value);
      plan->max_ctas = static_cast<int>(value);
      break;
    case IFNSO_OPT_STOP_AFTER:
      plan->stop_after = static_cast<int>(value);
      break;
    case IFNSO_OPT_TIMING:
      plan->timing = value != 0;
      break;
    case IFNSO_OPT_WAIT_LIMIT_MS:
      if (value < 0 || value > 600000) return fail(IFNSO_ERR_INVALID_ARG, "wait limit %lld ms", (long long)value);
      plan->wait_ms = static_cast<int>(value);
      break;
    case IFNSO_OPT_INJECT_STALL:
      plan->inject_stall = value != 0;
      break;
    case IFNSO_OPT_CTA_GROUP:
      if (value < 0 || value > 2) return fail(IFNSO_ERR_INVALID_ARG, "cta group %lld", (long long)value);
      plan->cta_group = static_cast<int>(value);
      break;
    case IFNSO_OPT_GRAM_E4M3:
      if (value != 0 && plan->dtype != IFNSO_BF16)
        return fail(IFNSO_ERR_UNSUPPORTED, "the E4M3 Gram needs a BF16 plan");
      plan->gram_e4m3 = value != 0;
      break;
    case IFNSO_OPT_SPLIT_SQUARINGS:
      if (value < -1 || value > 30) return fail(IFNSO_ERR_INVALID_ARG, "split squarings %lld", (long long)value);
      plan->split_squarings = static_cast<int>(value);
      break;
    case IFNSO_OPT_HOST_STREAMS:
      if (value != 1 && value != 2) return fail(IFNSO_ERR_INVALID_ARG, "host streams %lld (1 or 2)", (long long)value);
      plan->host_streams = static_cast<int>(value);
      return IFNSO_OK;  // the metadata does not depend on it
    case IFNSO_OPT_SMALL_MATRICES:
      if (value < 0 || value > 2) return fail(IFNSO_ERR_INVALID_ARG, "small matrices %lld (0, 1 or 2)", (long long)value);
      plan->small = static_cast<int>(value);
      return IFNSO_OK;  // the metadata holds both paths' views
    case IFNSO_OPT_APPLY_F16:
      if (value != 0 && value != 1) return fail(IFNSO_ERR_INVALID_ARG, "FP16 product %lld (0 or 1)", (long long)value);
      plan->apply_f16 = static_cast<int>(value);
      plan->sig_valid = false;
      return IFNSO_OK;
    case IFNSO_OPT_STAGE_LIMITS: {
      int m[kDepthKinds];
      for (int k = 0; k < kDepthKinds; ++k) {
        m[k] = static_cast<int>((value >> (4 * k)) & 15);
        if (m[k] == 1) return fail(IFNSO_ERR_INVALID_ARG, "stage limits %lld (0 or 2..15 per kind)", (long long)value);
      }
      if (value < 0 || (value >> (4 * kDepthKinds)))
        return fail(IFNSO_ERR_INVALID_ARG, "stage limits %lld (5 kinds of 4 bits)", (long long)value);
      for (int k = 0; k < kDepthKinds; ++k) plan->stage_lim[k] = m[k];
      return IFNSO_OK;
    }
    case IFNSO_OPT_CTA_GROUP_KINDS: {
      if (value == 0) {
        plan->tuned = false;
        return IFNSO_OK;
      }
      int m[kKinds];
      for (int k = 0; k < kKinds; ++k) {
        m[k] = static_cast<int>((value >> (2 * k)) & 3);
        if (m[k] != 1 && m[k] != 2) return fail(IFNSO_ERR_INVALID_ARG, "cta group kinds %lld", (long long)value);
      }
      if (value >> (2 * kKinds)) return fail(IFNSO_ERR_INVALID_ARG, "cta group kinds %lld", (long long)value);
      for (int k = 0; k < kKinds; ++k) plan->cg_kind[k] = m[k];
      plan->tuned = true;
      return IFNSO_OK;
    }
    default:
      return fail(IFNSO_ERR_INVALID_ARG, "unknown option %d", (int)option);
  }
  plan->sig_valid = false;
  return IFNSO_OK;
}

ifnso_status ifnso_plan_get(const ifnso_plan* plan, ifnso_option option, int64_t* value) {
  if (!plan || !value) return fail(IFNSO_ERR_INVALID_ARG, "NULL argument");
  switch (option) {
    case IFNSO_OPT_PRECISION:
      *value = resolve_prec(plan).mode;
      return IFNSO_OK;
    case IFNSO_OPT_SCALE: *value = plan->scale; return IFNSO_OK;
    case IFNSO_OPT_MAX_CTAS: *value = plan->max_ctas; return IFNSO_OK;
    case IFNSO_OPT_STOP_AFTER: *value = plan->stop_after; return IFNSO_OK;
    case IFNSO_OPT_TIMING: *value = plan->timing ? 1 : 0; return IFNSO_OK;
    case IFNSO_OPT_WAIT_LIMIT_MS: *value = plan->wait_ms; return IFNSO_OK;
    case IFNSO_OPT_INJECT_STALL: *value = plan->inject_stall; return IFNSO_OK;
    case IFNSO_OPT_CTA_GROUP: *value = plan->cta_group; return IFNSO_OK;
    case IFNSO_OPT_GRAM_E4M3: *value = plan->gram_e4m3; return IFNSO_OK;
    case IFNSO_OPT_SPLIT_SQUARINGS: *value = resolve_prec(plan).k_split; return IFNSO_OK;
    case IFNSO_OPT_HOST_STREAMS: *value = plan->host_streams; return IFNSO_OK;
    case IFNSO_OPT_SMALL_MATRICES: *value = plan->small; return IFNSO_OK;
    case IFNSO_OPT_SMALL_TUNED: *value = plan->small_tuned; return IFNSO_OK;
    case IFNSO_OPT_FP16_COPY_HOSTS: *value = plan->copy_hosts; return IFNSO_OK;
    case IFNSO_OPT_STAGE_LIMITS: {
      int64_t v = 0;
      for (int k = 0; k < kDepthKinds; ++k) v |= static_cast<int64_t>(plan->stage_lim[k]) << (4 * k);
      *value = v;
      return IFNSO_OK;
    }
    case IFNSO_OPT_APPLY_F16: *value = resolve_prec(plan).p_f16; return IFNSO_OK;
    case IFNSO_OPT_CTA_GROUP_KINDS: {
      int64_t v = 0;
      if (plan->tuned)
        for (int k = 0; k < kKinds; ++k) v |= static_cast<int64_t>(plan->cg_kind[k]) << (2 * k);
      *value = v;
      return IFNSO_OK;
    }
    default: return fail(IFNSO_ERR_INVALID_ARG, "unknown option %d", (int)option);
  }
}

ifnso_status ifnso_plan_destroy(ifnso_plan* plan) {
  if (!plan) return IFNSO_OK;
  ws_forget(plan);
  for (auto* list : {&plan->ev_calls, &plan->ev_graph})
    for (auto& c : *list)
      for (cudaEvent_t e : c) cudaEventDestroy(e);
  for (cudaEvent_t e : plan->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : plan->ev_retired) cudaEventDestroy(e);
  if (plan->s_in) {
    cudaStreamSynchronize(plan->s_in);
    cudaStreamSynchronize(plan->s_out);
    cudaStreamSynchronize(plan->s_comp);
    cudaStreamDestroy(plan->s_in);
    cudaStreamDestroy(plan->s_out);
    cudaStreamDestroy(plan->s_comp);
    cudaEventDestroy(plan->ev_start);
    cudaEventDestroy(plan->ev_last);
  }
  for (auto* v : {&plan->ev_in, &plan->ev_done})
    for (cudaEvent_t e : *v) cudaEventDestroy(e);
  if (plan->meta_host) {
    cudaDeviceSynchronize();
    cudaFreeHost(plan->meta_host);
  }
  delete plan;
  return IFNSO_OK;
}

size_t ifnso_workspace_bytes(const ifnso_plan* plan, const ifnso_batch_desc* batch) {
  if (!plan) {
    fail(IFNSO_ERR_INVALID_ARG, "plan is NULL");
    return 0;
  }
  std::vector<Shape> shp;
  if (read_batch(plan, batch, shp) != IFNSO_OK) return 0;
  return make_layout(plan, shp, 0, 0, plan->L + 1).total;
}

size_t ns_workspace_bytes(const ifnso_plan* plan, const ifnso_batch_desc* batch) {
  if (!plan) {
    fail(IFNSO_ERR_INVALID_ARG, "plan is NULL");
    return 0;
  }
  std::vector<Shape> shp;
  if (read_batch(plan, batch, shp) != IFNSO_OK) return 0;
  // the step count only changes the metadata; size for up to 16 steps
  return make_layout(plan, shp, 1, 16, 1).total;
}

ifnso_status ifnso_orthogonalize(ifnso_plan* plan, const ifnso_batch_desc* batch, const ifnso_coeffs* coeffs,
                                 void* const* out, void* workspace, size_t workspace_bytes,
                                 ifnso_stream_t stream_) {
  if (!plan) return fail(IFNSO_ERR_INVALID_ARG, "plan is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  return orthogonalize_locked(plan, batch, coeffs, out, workspace, workspace_bytes,
                              reinterpret_cast<cudaStream_t>(stream_));
}

ifnso_status ifnso_muon_step(ifnso_plan* plan, const ifnso_batch_desc* grads, void* const* momentum,
                             void* const* staging, void* const* weights, const ifnso_coeffs* coeffs, double beta,
                             int32_t nesterov, double lr, void* workspace, size_t workspace_bytes,
                             ifnso_stream_t stream_) {
  if (!plan) return fail(IFNSO_ERR_INVALID_ARG, "plan is NULL");
  if (plan->dtype != IFNSO_BF16) return fail(IFNSO_ERR_UNSUPPORTED, "the Muon step needs a BF16 plan");
  if (!grads || !momentum || !staging || !weights)
    return fail(IFNSO_ERR_INVALID_ARG, "grads / momentum / staging / weights is NULL");
  if (!(beta >= 0.0 && beta < 1.0)) return fail(IFNSO_ERR_INVALID_ARG, "beta = %g must be in [0, 1)", beta);
  if (!(lr >= 0.0 && lr < 1e30)) return fail(IFNSO_ERR_INVALID_ARG, "lr = %g must be finite and >= 0", lr);
  if (nesterov != 0 && nesterov != 1) return fail(IFNSO_ERR_INVALID_ARG, "nesterov must be 0 or 1");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(plan->mu);
  std::vector<Shape> shp;
  ifnso_status st = read_batch(plan, grads, shp);
  if (st != IFNSO_OK) return st;
  std::vector<const void*> u_in(static_cast<size_t>(grads->count));
  for (int i = 0; i < grads->count; ++i) {
    const void* g = grads->in[i];
    if (!momentum[i] || !staging[i] || !weights[i])
      return fail(IFNSO_ERR_INVALID_ARG, "matrix %d: NULL momentum, staging or weights", i);
    for (const void* q : {static_cast<const void*>(momentum[i]), static_cast<const void*>(staging[i]),
                          static_cast<const void*>(weights[i])})
      if (reinterpret_cast<uintptr_t>(q) % 16 != 0)
        return fail(IFNSO_ERR_INVALID_ARG, "matrix %d: momentum, staging and weights must be 16-byte aligned", i);
    if (staging[i] == g || weights[i] == g || weights[i] == staging[i] || momentum[i] == g ||
        momentum[i] == staging[i] || momentum[i] == weights[i])
      return fail(IFNSO_ERR_INVALID_ARG, "matrix %d: grads, momentum, staging and weights must be distinct", i);
    u_in[static_cast<size_t>(i)] = staging[i];
  }
  for (int i = 0; i < grads->count; ++i) {
    const Shape& sh = shp[static_cast<size_t>(i)];
    IFNSO_CUDA(launch_muon_momentum(grads->in[i], sh.ld, static_cast<float*>(momentum[i]), staging[i], sh.rows,
                                    sh.cols, static_cast<float>(beta), nesterov, stream),
               "momentum");
  }
  // the orthogonalization of U, whose product writes W - lr s Y into the weights
  ifnso_batch_desc ub = *grads;
  ub.in = u_in.data();
  return orthogonalize_locked(plan, &ub, coeffs, weights, workspace, workspace_bytes, stream, true,
                              static_cast<float>(lr));
}

ifnso_status ifnso_plan_autotune(ifnso_plan* plan, const ifnso_batch_desc* batch, const ifnso_coeffs* coeffs,
                                 void* const* out, void* workspace, size_t workspace_bytes, int32_t reps,
                                 int32_t* chosen, ifnso_stream_t stream_) {
  if (!plan) return fail(IFNSO_ERR_INVALID_ARG, "plan is NULL");
  if (reps < 1 || reps > 100) return fail(IFNSO_ERR_INVALID_ARG, "reps %d must be in [1, 100]", reps);
  if (plan->dtype != IFNSO_BF16) return fail(IFNSO_ERR_UNSUPPORTED, "autotuning applies to BF16 plans");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(plan->mu);
  const int L = plan->L;
  const Prec pc = resolve_prec(plan);
  // pass index -> kind: 0 Gram, 1 prep (not tuned), 2.. squarings, L + 1 product
  auto kind_of = [&](int pass) {
    if (pass == 0) return kGram;
    if (pass == L + 1) return kApply;
    if (pass >= 2 && pass <= L) return (pass - 1) <= pc.k_split ? kSplit : kPlain;
    return -1;
  };
  const int saved_cg = plan->cta_group, saved_stop = plan->stop_after, saved_small = plan->small;
  const bool saved_timing = plan->timing, saved_tuned = plan->tuned;
  int saved_lim[kDepthKinds];
  for (int k = 0; k < kDepthKinds; ++k) {
    saved_lim[k] = plan->stage_lim[k];
    plan->stage_lim[k] = 0;  // the MMA modes are compared with the whole ring
  }
  plan->stop_after = -1;
  plan->timing = true;
  plan->tuned = false;
  plan->small = 2;  // the MMA modes are those of the tiled passes
  double ms[3][kKinds] = {};
  ifnso_status st = IFNSO_OK;
  std::vector<double> pt(L + 2);
  for (int cg = 1; cg <= 2 && st == IFNSO_OK; ++cg) {
    plan->cta_group = cg;
    for (int r = 0; r <= reps && st == IFNSO_OK; ++r) {
      st = orthogonalize_locked(plan, batch, coeffs, out, workspace, workspace_bytes, stream);
      if (st != IFNSO_OK) break;
      int np = 0;
      // the first call warms up (metadata upload, first touch); the others count
      st = pass_times_locked(plan, pt.data(), static_cast<int>(pt.size()), &np, nullptr);
      if (r == 0) continue;
      for (int k = 0; k < np; ++k)
        if (kind_of(k) >= 0) ms[cg][kind_of(k)] += pt[k];
    }
  }
  plan->cta_group = saved_cg;
  if (st != IFNSO_OK) {
    plan->stop_after = saved_stop;
    plan->timing = saved_timing;
    plan->tuned = saved_tuned;
    plan->small = saved_small;
    for (int k = 0; k < kDepthKinds; ++k) plan->stage_lim[k] = saved_lim[k];
    return st;
  }
  for (int k = 0; k < kKinds; ++k) plan->cg_kind[k] = ms[2][k] < ms[1][k] ? 2 : 1;
  plan->tuned = true;
  // The depth of the operand ring per pass kind, in the chosen modes: the
  // whole ring, 4 or 3 stages (fewer operand bytes in flight leave L2 to the
  // loads and stores of epilogues like the final squaring's P read).  A
  // shallower ring must win by 2%.
  {
    auto depth_of = [&](int pass) {
      if (pass == L && L >= 2) return kFinal;
      return kind_of(pass);
    };
    const int cands[3] = {0, 4, 3};
    double best[kDepthKinds] = {};
    int pick[kDepthKinds] = {};
    plan->cta_group = 0;
    for (int c = 0; c < 3 && st == IFNSO_OK; ++c) {
      for (int k = 0; k < kDepthKinds; ++k) plan->stage_lim[k] = cands[c];
      double t[kDepthKinds] = {};
      for (int r = 0; r <= reps && st == IFNSO_OK; ++r) {
        st = orthogonalize_locked(plan, batch, coeffs, out, workspace, workspace_bytes, stream);
        if (st != IFNSO_OK) break;
        int np = 0;
        st = pass_times_locked(plan, pt.data(), static_cast<int>(pt.size()), &np, nullptr);
        if (r == 0) continue;
        for (int k = 0; k < np; ++k)
          if (depth_of(k) >= 0) t[depth_of(k)] += pt[k];
      }
      for (int k = 0; k < kDepthKinds; ++k)
        if (c == 0 || t[k] < 0.98 * best[k]) {
          best[k] = t[k];
          pick[k] = cands[c];
        }
    }
    plan->cta_group = saved_cg;
    // a limit at or above the kind's ring depth is the whole ring
    const int fin_split = pc.k_split >= L - 1 ? 1 : 0;
    const int na[kDepthKinds] = {1, 2, 1, pc.p_split ? 2 : 1, fin_split ? 2 : 1};
    const int nb[kDepthKinds] = {1, 2, 1, 1, fin_split ? 2 : 1};
    for (int k = 0; k < kDepthKinds; ++k) {
      const int cg = plan->cg_kind[k == kFinal ? (fin_split ? kSplit : kPlain) : k];
      if (pick[k] >= tc_ring_stages(na[k], nb[k], cg)) pick[k] = 0;
    }
    for (int k = 0; k < kDepthKinds; ++k) plan->stage_lim[k] = st == IFNSO_OK ? pick[k] : saved_lim[k];
  }
  // the shape bucket h <= 128: the on-chip path against the tiled passes (in their tuned modes)
  {
    std::vector<Shape> shp;
    ifnso_status sb = read_batch(plan, batch, shp);
    if (sb == IFNSO_OK) {
      const Layout ly = make_layout(plan, shp, 0, 0, L + 1);
      if (small_applies(plan, ly, coeffs, false)) {
        double tot[3] = {0.0, 0.0, 0.0};
        for (int mode = 1; mode <= 2 && st == IFNSO_OK; ++mode) {
          plan->small = mode;
          for (int r = 0; r <= reps && st == IFNSO_OK; ++r) {
            st = orthogonalize_locked(plan, batch, coeffs, out, workspace, workspace_bytes, stream);
            if (st != IFNSO_OK) break;
            int np = 0;
            st = pass_times_locked(plan, pt.data(), static_cast<int>(pt.size()), &np, nullptr);
            if (r == 0) continue;
            for (int k = 0; k < np; ++k) tot[mode] += pt[k];
          }
        }
        if (st == IFNSO_OK) plan->small_tuned = tot[1] <= tot[2] ? 1 : 2;
      }
    }
  }
  plan->small = saved_small;
  plan->stop_after = saved_stop;
  plan->timing = saved_timing;
  if (st != IFNSO_OK) return st;
  plan->sig_valid = false;
  if (chosen)
    for (int k = 0; k < kKinds; ++k) chosen[k] = plan->cg_kind[k];
  return IFNSO_OK;
}

ifnso_status ifnso_orthogonalize_host(ifnso_plan* plan, const void* const* host_in,
                                      const ifnso_batch_desc* dev_batch, const ifnso_coeffs* coeffs,
                                      void* const* dev_out, void* const* host_out, void* workspace,
                                      size_t workspace_bytes, int32_t groups, ifnso_stream_t stream_) {
  if (!plan) return fail(IFNSO_ERR_INVALID_ARG, "plan is NULL");
  if (!host_in || !host_out) return fail(IFNSO_ERR_INVALID_ARG, "host_in / host_out is NULL");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(plan->mu);
  std::vector<Shape> shp;
  ifnso_status st = check_call(plan, dev_batch, coeffs, dev_out, shp);
  if (st != IFNSO_OK) return st;
  for (int i = 0; i < dev_batch->count; ++i)
    if (!host_in[i] || !host_out[i]) return fail(IFNSO_ERR_INVALID_ARG, "host buffer %d is NULL", i);
  if (dev_batch->count == 0) return IFNSO_OK;
  if ((st = init_plan_device(plan)) != IFNSO_OK) return st;
  Layout ly = make_layout(plan, shp, 0, 0, plan->L + 1);
  if ((st = check_ws(ly, workspace, workspace_bytes)) != IFNSO_OK) return st;
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  const int n = ly.count;
  const int want = ly.f32 ? 1 : std::min(groups <= 0 ? 8 : groups, n);
  const std::vector<int> gb = group_bounds(shp, want, true);
  const int ng = static_cast<int>(gb.size()) - 1;
  const bool on_chip = use_small(plan, ly, coeffs, false);
  if ((st = upload_ifnso_meta(plan, ly, dev_batch, dev_out, ws, coeffs, gb, stream, on_chip)) != IFNSO_OK) return st;
  if ((st = ensure_copy_streams(plan, ng)) != IFNSO_OK) return st;
  const size_t esz = plan->dtype == IFNSO_BF16 ? 2 : 4;
  // timeline events only for eager calls (a captured event would stay reserved for its graph)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  IFNSO_CUDA(cudaStreamIsCapturing(stream, &cap), "cudaStreamIsCapturing");
  const bool tl = plan->timing && cap == cudaStreamCaptureStatusNone;
  plan->tl_groups = tl ? ng : 0;
  if (tl) plan->tl_first = gb;
  if (tl) IFNSO_CUDA(cudaEventRecord(plan->tl_start, stream), "cudaEventRecord");
  // the copies come after everything already queued on `stream`
  IFNSO_CUDA(cudaEventRecord(plan->ev_start, stream), "cudaEventRecord");
  IFNSO_CUDA(cudaStreamWaitEvent(plan->s_in, plan->ev_start, 0), "cudaStreamWaitEvent");
  IFNSO_CUDA(cudaStreamWaitEvent(plan->s_out, plan->ev_start, 0), "cudaStreamWaitEvent");
  // odd groups on the second compute stream (which also waits for the
  // caller's earlier work, the metadata upload included)
  const bool two = plan->host_streams == 2 && ng > 1;
  if (two) IFNSO_CUDA(cudaStreamWaitEvent(plan->s_comp, plan->ev_start, 0), "cudaStreamWaitEvent");
  for (int g = 0; g < ng; ++g) {
    for (int i = gb[g]; i < gb[g + 1]; ++i) {
      const Shape& s = shp[i];
      void* dst = const_cast<void*>(dev_batch->in[i]);
      if (s.ld == s.cols)
        IFNSO_CUDA(cudaMemcpyAsync(dst, host_in[i], s.rows * s.cols * esz, cudaMemcpyHostToDevice, plan->s_in),
                   "input upload");
      else
        IFNSO_CUDA(cudaMemcpy2DAsync(dst, s.ld * esz, host_in[i], s.ld * esz, s.cols * esz, s.rows,
                                     cudaMemcpyHostToDevice, plan->s_in),
                   "input upload");
    }
    IFNSO_CUDA(cudaEventRecord(plan->ev_in[g], plan->s_in), "cudaEventRecord");
    if (tl) IFNSO_CUDA(cudaEventRecord(plan->tl_ev[3 * g], plan->s_in), "cudaEventRecord");
  }
  int hpad_max = 0;
  for (auto& sh : shp) hpad_max = std::max<int>(hpad_max, static_cast<int>(sh.hpad));
  for (int g = 0; g < ng; ++g) {
    cudaStream_t cs = (two && (g & 1)) ? plan->s_comp : stream;
    Run r{plan, &ly, ws, coeffs, hpad_max, cs, ly.f32 != 0};
    r.on_chip = on_chip;
    IFNSO_CUDA(cudaStreamWaitEvent(cs, plan->ev_in[g], 0), "cudaStreamWaitEvent");
    if (ly.f32)
      st = run_f32(r);
    else
      st = run_tc(r, gb[g], gb[g + 1] - gb[g], plan->sym_off[g], plan->sym_off[g + 1], plan->app_off[g],
                  plan->app_off[g + 1]);
    if (st != IFNSO_OK) return st;
    IFNSO_CUDA(cudaEventRecord(plan->ev_done[g], cs), "cudaEventRecord");
    if (tl) IFNSO_CUDA(cudaEventRecord(plan->tl_ev[3 * g + 1], cs), "cudaEventRecord");
    IFNSO_CUDA(cudaStreamWaitEvent(plan->s_out, plan->ev_done[g], 0), "cudaStreamWaitEvent");
    for (int i = gb[g]; i < gb[g + 1]; ++i) {
      const Shape& s = shp[i];
      IFNSO_CUDA(cudaMemcpyAsync(host_out[i], dev_out[i], s.rows * s.cols * esz, cudaMemcpyDeviceToHost,
                                 plan->s_out),
                 "output download");
    }
    if (tl) IFNSO_CUDA(cudaEventRecord(plan->tl_ev[3 * g + 2], plan->s_out), "cudaEventRecord");
  }
  // later work on `stream` comes after the last download
  IFNSO_CUDA(cudaEventRecord(plan->ev_last, plan->s_out), "cudaEventRecord");
  IFNSO_CUDA(cudaStreamWaitEvent(stream, plan->ev_last, 0), "cudaStreamWaitEvent");
  return IFNSO_OK;
}

ifnso_status ns_iterate(ifnso_plan* plan, const ifnso_batch_desc* batch, const double* poly, int32_t degree,
                        int32_t steps, void* const* out, void* workspace, size_t workspace_bytes,
                        ifnso_stream_t stream_) {
  if (!plan) return fail(IFNSO_ERR_INVALID_ARG, "plan is NULL");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(plan->mu);
  if (!poly || (degree != 3 && degree != 5)) return fail(IFNSO_ERR_INVALID_ARG, "degree must be 3 or 5 with poly given");
  if (steps < 1 || steps > 16) return fail(IFNSO_ERR_INVALID_ARG, "steps = %d must be in [1, 16]", steps);
  std::vector<Shape> shp;
  ifnso_status st = read_batch(plan, batch, shp);
  if (st != IFNSO_OK) return st;
  if (!out) return fail(IFNSO_ERR_INVALID_ARG, "out is NULL");
  for (int i = 0; i < batch->count; ++i) {
    if (!out[i]) return fail(IFNSO_ERR_INVALID_ARG, "out[%d] is NULL", i);
    if (out[i] == batch->in[i]) return fail(IFNSO_ERR_INVALID_ARG, "out[%d] aliases the input", i);
    if (reinterpret_cast<uintptr_t>(out[i]) % 16 != 0)
      return fail(IFNSO_ERR_INVALID_ARG, "out[%d] is not 16-byte aligned", i);
  }
  if (batch->count == 0) return IFNSO_OK;
  if ((st = init_plan_device(plan)) != IFNSO_OK) return st;
  Layout ly = make_layout(plan, shp, 1, steps, 1);
  Layout ly16 = make_layout(plan, shp, 1, 16, 1);
  // buffers are placed for 16 steps so that the size does not depend on `steps`
  ly.off_scal = ly16.off_scal;
  ly.off_buf = ly16.off_buf;
  ly.total = ly16.total;
  if ((st = check_ws(ly, workspace, workspace_bytes)) != IFNSO_OK) return st;
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  const uint64_t sig = batch_sig(plan, batch, out, workspace, nullptr, poly, degree, steps, 2);
  if (!plan->sig_valid || plan->sig != sig || !ws_current(ws, plan, sig)) {
    if ((st = ensure_meta_host(plan, ly.meta_bytes, stream)) != IFNSO_OK) return st;
    uint8_t* meta = static_cast<uint8_t*>(plan->meta_host);
    if ((st = build_ns_meta(ly, batch, out, ws, meta)) != IFNSO_OK) return st;
    if ((st = ns_set_apply_source(ly, meta, degree == 5)) != IFNSO_OK) return st;
    IFNSO_CUDA(cudaMemcpyAsync(ws, meta, ly.meta_bytes, cudaMemcpyHostToDevice, stream), "metadata upload");
    plan->sig = sig;
    plan->sig_valid = true;
    ws_claim(ws, plan, sig);
  }
  const int n = ly.count;
  MatInfo* d_mats = reinterpret_cast<MatInfo*>(ws + ly.off_mats);
  MatScalars* scal = reinterpret_cast<MatScalars*>(ws + ly.off_scal);
  int hpad_max = 0, max_h = 0, max_w = 0;
  for (auto& s : shp) {
    hpad_max = std::max<int>(hpad_max, static_cast<int>(s.hpad));
    max_h = std::max<int>(max_h, static_cast<int>(s.h));
    max_w = std::max<int>(max_w, static_cast<int>(s.w));
  }
  IFNSO_CUDA(cudaMemsetAsync(ws + ly.off_scal, 0, n * sizeof(MatScalars), stream), "scalar reset");
  IFNSO_CUDA(mark(plan, stream, true), "timing event");
  bool all_small = !ly.f32 && plan->small != 2 && !plan->inject_stall;
  for (auto& sh : shp) all_small = all_small && sh.h <= kSmallH;
  if (all_small) {
    // every matrix has h <= 128: the whole iteration on chip, one launch
    SmNsParams q{};
    q.probs = reinterpret_cast<const SmNsProblem*>(ws + ly.off_small_ns);
    q.scal = scal;
    q.first = 0;
    q.steps = steps;
    q.degree = degree;
    q.wait_ms = static_cast<uint32_t>(plan->wait_ms);
    q.a = static_cast<float>(poly[0]);
    q.b = static_cast<float>(poly[1]);
    q.c = degree == 5 ? static_cast<float>(poly[2]) : 0.f;
    IFNSO_CUDA(launch_small_ns(q, n, stream), "on-chip NS");
    IFNSO_CUDA(mark(plan, stream, false), "timing event");
    return IFNSO_OK;
  }
  // ||A||_F^2 into the trace slot, then the scalars with the Frobenius scale
  int gx = std::max(1, std::min(1024, 16 * plan->num_sms / std::max(1, n)));
  IFNSO_CUDA(launch_norm2(d_mats, n, plan->dtype == IFNSO_BF16, &scal[0].trace,
                          sizeof(MatScalars) / sizeof(double), gx, stream),
             "norm");
  CoefTable none{};
  IFNSO_CUDA(launch_scalars(d_mats, n, scal, none, 0, 1, 1, stream), "scalars");
  IFNSO_CUDA(mark(plan, stream, false), "timing event");
  const float a = static_cast<float>(poly[0]);
  const float b = static_cast<float>(poly[1]);
  const float c = degree == 5 ? static_cast<float>(poly[2]) : 0.f;
  if (ly.f32) {
    SgParams p{};
    p.scal = scal;
    p.ns_a = a;
    p.ns_b = b;
    p.ns_c = c;
    p.ns_bcoef = degree == 5 ? 1.f : b;
    const SgProblem* probs = reinterpret_cast<const SgProblem*>(ws + ly.off_probs);
    for (int s = 0; s < steps; ++s) {
      p.ns_step = s;
      p.probs = probs + ly.pi_ns_gram + s * n;
      IFNSO_CUDA(sg_launch(EPI_NS_GRAM, p, n, hpad_max, hpad_max, stream), "NS Gram");
      IFNSO_CUDA(mark(plan, stream, false), "timing event");
      if (degree == 5) {
        p.probs = probs + ly.pi_ns_sqr;
        IFNSO_CUDA(sg_launch(EPI_NS_SQR, p, n, hpad_max, hpad_max, stream), "NS square");
        IFNSO_CUDA(mark(plan, stream, false), "timing event");
      }
      p.probs = probs + ly.pi_ns_apply + s * n;
      IFNSO_CUDA(sg_launch(EPI_NS_APPLY, p, n, max_h, max_w, stream), "NS apply");
      IFNSO_CUDA(mark(plan, stream, false), "timing event");
    }
    return IFNSO_OK;
  }
  TcParams p{};
  p.wait_ms = static_cast<uint32_t>(plan->wait_ms);
  // MMA mode per pass: the plan's setting, else the autotuned mode of the
  // IFNSO pass of the same shape (Gram; squaring of one h x h operand;
  // product), else per-CTA MMAs
  auto ns_cg = [&](int kind) { return plan->cta_group ? plan->cta_group : (plan->tuned ? plan->cg_kind[kind] : 1); };
  p.scal = scal;
  p.ns_a = a;
  p.ns_b = b;
  p.ns_c = c;
  p.ns_bcoef = degree == 5 ? 1.f : b;
  const TcProblem* probs = reinterpret_cast<const TcProblem*>(ws + ly.off_probs);
  const WorkItem* sym = reinterpret_cast<const WorkItem*>(ws + ly.off_items_sym);
  const WorkItem* app = reinterpret_cast<const WorkItem*>(ws + ly.off_items_app);
  for (int s = 0; s < steps; ++s) {
    p.ns_step = s;
    p.probs = probs + ly.pi_ns_gram + s * n;
    p.items = sym;
    p.n_items = static_cast<int32_t>(ly.n_sym);
    p.cta_group = ns_cg(kGram);
    IFNSO_CUDA(tc_launch(EPI_NS_GRAM, 1, 1, p, grid_for(plan, ly.n_sym), stream), "NS Gram");
    IFNSO_CUDA(mark(plan, stream, false), "timing event");
    if (degree == 5) {
      p.probs = probs + ly.pi_ns_sqr;
      p.cta_group = ns_cg(kPlain);
      IFNSO_CUDA(tc_launch(EPI_NS_SQR, 1, 1, p, grid_for(plan, ly.n_sym), stream), "NS square");
      IFNSO_CUDA(mark(plan, stream, false), "timing event");
    }
    p.probs = probs + ly.pi_ns_apply + s * n;
    p.items = app;
    p.n_items = static_cast<int32_t>(ly.n_app);
    p.cta_group = ns_cg(kApply);
    IFNSO_CUDA(tc_launch(EPI_NS_APPLY, 1, 1, p, grid_for(plan, ly.n_app), stream), "NS apply");
    IFNSO_CUDA(mark(plan, stream, false), "timing event");
  }
  return IFNSO_OK;
}

ifnso_status ifnso_device_status(const ifnso_plan* plan, const void* workspace, int32_t count, int32_t* per_matrix,
                                 double* o_out, double* trace_out, ifnso_stream_t stream_) {
  if (!plan || !workspace || count < 0) return fail(IFNSO_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  IFNSO_CUDA(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
  if (count == 0) return IFNSO_OK;
  // the scalars sit right after the metadata, whose size depends on the batch:
  // find them through the MatInfo of matrix 0 (the offset of its buffers)
  std::vector<MatInfo> mats(count);
  IFNSO_CUDA(cudaMemcpy(mats.data(), workspace, count * sizeof(MatInfo), cudaMemcpyDeviceToHost), "status read");
  const uint8_t* buf0 = static_cast<const uint8_t*>(mats[0].gp ? static_cast<const void*>(mats[0].gp) : mats[0].s);
  const size_t scal_bytes = a1k(count * sizeof(MatScalars));
  const uint8_t* scal_ptr = buf0 - scal_bytes;
  std::vector<MatScalars> sc(count);
  IFNSO_CUDA(cudaMemcpy(sc.data(), scal_ptr, count * sizeof(MatScalars), cudaMemcpyDeviceToHost), "status read");
  bool timeout = false;
  for (int i = 0; i < count; ++i) {
    if (per_matrix) per_matrix[i] = sc[i].status;
    if (o_out) o_out[i] = sc[i].s2;
    if (trace_out) trace_out[i] = sc[i].trace;
    if (sc[i].status & IFNSO_DEV_TIMEOUT) timeout = true;
  }
  if (timeout) return fail(IFNSO_ERR_DEVICE_TIMEOUT, "a device wait timed out");
  return IFNSO_OK;
}

ifnso_status ifnso_pass_times(ifnso_plan* plan, double* ms_out, int32_t max_passes, int32_t* n_passes,
                              int32_t* n_calls) {
  if (!plan || !ms_out || !n_passes || max_passes < 0) return fail(IFNSO_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(plan->mu);
  return pass_times_locked(plan, ms_out, max_passes, n_passes, n_calls);
}

ifnso_status ifnso_host_timeline(ifnso_plan* plan, double* ms_out, int32_t max_groups, int32_t* n_groups,
                                 int32_t* group_first) {
  if (!plan || !ms_out || !n_groups || max_groups < 0) return fail(IFNSO_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(plan->mu);
  *n_groups = plan->tl_groups;
  if (plan->tl_groups == 0) return IFNSO_OK;
  IFNSO_CUDA(cudaEventSynchronize(plan->tl_ev[3 * plan->tl_groups - 1]), "cudaEventSynchronize");
  for (int g = 0; g < plan->tl_groups && g < max_groups; ++g)
    for (int k = 0; k < 3; ++k) {
      float ms = 0.f;
      IFNSO_CUDA(cudaEventElapsedTime(&ms, plan->tl_start, plan->tl_ev[3 * g + k]), "cudaEventElapsedTime");
      ms_out[3 * g + k] = ms;
    }
  if (group_first)
    for (int g = 0; g <= plan->tl_groups && g <= max_groups; ++g) group_first[g] = plan->tl_first[g];
  return IFNSO_OK;
}

ifnso_status ifnso_workspace_view(const ifnso_plan* plan, const ifnso_batch_desc* batch, void* workspace,
                                  int32_t index, int32_t which, void** ptr, int64_t* ld) {
  if (!plan || !ptr || !ld || !workspace) return fail(IFNSO_ERR_INVALID_ARG, "NULL argument");
  std::vector<Shape> shp;
  ifnso_status st = read_batch(plan, batch, shp);
  if (st != IFNSO_OK) return st;
  if (index < 0 || index >= batch->count) return fail(IFNSO_ERR_INVALID_ARG, "index %d", index);
  Layout ly = make_layout(plan, shp, 0, 0, plan->L + 1);
  MatInfo mi = mat_info(ly, batch, nullptr, static_cast<uint8_t*>(workspace), index);
  *ld = shp[index].hpad;
  if (which == 0) *ptr = mi.gp;
  else if (which >= 1 && which <= 4) *ptr = mi.d[which - 1];
  else if (which == 5) {
    *ptr = static_cast<uint8_t*>(workspace) + ly.off_rows + static_cast<size_t>(index) * kRowSlots * sizeof(float);
    *ld = kRowSlots;
  } else if (which == 6) {
    *ptr = static_cast<uint8_t*>(workspace) + ly.off_scal + static_cast<size_t>(index) * sizeof(MatScalars);
    *ld = sizeof(MatScalars) / sizeof(double);
  } else if (which == 7) {
    *ptr = mi.a16;
    *ld = mi.a16ld;
  }
  else return fail(IFNSO_ERR_INVALID_ARG, "which = %d", which);
  if (!*ptr) return fail(IFNSO_ERR_INVALID_ARG, "buffer %d is not used by this plan", which);
  return IFNSO_OK;
}

namespace {
// Descriptor buffers of ifnso_frobenius_norm2, one per device.
struct NormDesc {
  MatInfo* d = nullptr;
  int cap = 0;
  cudaEvent_t done = nullptr;  // recorded after the last launch that read d
};
constexpr int kNormDevices = 64;
std::mutex g_norm_mu;
NormDesc g_norm_desc[kNormDevices];
}  // namespace

ifnso_status ifnso_frobenius_norm2(const ifnso_batch_desc* batch, ifnso_dtype dtype, double* norm2_out,
                                   ifnso_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!batch || !norm2_out) return fail(IFNSO_ERR_INVALID_ARG, "NULL argument");
  if (dtype != IFNSO_BF16 && dtype != IFNSO_F32) return fail(IFNSO_ERR_INVALID_ARG, "dtype");
  ifnso_plan tmp;
  tmp.h = tmp.w = INT64_MAX / 4;
  tmp.dtype = dtype;
  std::vector<Shape> shp;
  ifnso_status st = read_batch(&tmp, batch, shp);
  if (st != IFNSO_OK) return st;
  if (batch->count == 0) return IFNSO_OK;
  int dev = 0, sms = 0;
  IFNSO_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  IFNSO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  if (dev < 0 || dev >= kNormDevices) return fail(IFNSO_ERR_UNSUPPORTED, "device %d", dev);
  IFNSO_CUDA(cudaMemsetAsync(norm2_out, 0, batch->count * sizeof(double), stream), "reset");
  // The matrices' descriptions go to a device buffer of this entry point, one
  // per device (grown on demand).  A call waits until the previous call's
  // kernel on that device has read the buffer before overwriting it, so
  // calls on different streams or host threads do not race on it.
  std::lock_guard<std::mutex> lk(g_norm_mu);
  NormDesc& nd = g_norm_desc[dev];
  if (nd.done) IFNSO_CUDA(cudaEventSynchronize(nd.done), "cudaEventSynchronize");
  if (nd.cap < batch->count) {
    if (nd.d) cudaFree(nd.d);
    nd.d = nullptr;
    nd.cap = 0;
    IFNSO_CUDA(cudaMalloc(&nd.d, batch->count * sizeof(MatInfo)), "cudaMalloc");
    nd.cap = batch->count;
  }
  if (!nd.done) IFNSO_CUDA(cudaEventCreateWithFlags(&nd.done, cudaEventDisableTiming), "cudaEventCreate");
  std::vector<MatInfo> h(batch->count);
  for (int i = 0; i < batch->count; ++i) {
    memset(&h[i], 0, sizeof(MatInfo));
    h[i].in = batch->in[i];
    h[i].rows = shp[i].rows;
    h[i].cols = shp[i].cols;
    h[i].ld = shp[i].ld;
  }
  // (a pageable source: the copy has taken the bytes when the call returns)
  IFNSO_CUDA(cudaMemcpyAsync(nd.d, h.data(), h.size() * sizeof(MatInfo), cudaMemcpyHostToDevice, stream), "upload");
  int gx = std::max(1, std::min(1024, 16 * sms / std::max(1, batch->count)));
  IFNSO_CUDA(launch_norm2(nd.d, batch->count, dtype == IFNSO_BF16, norm2_out, 1, gx, stream), "norm");
  IFNSO_CUDA(cudaEventRecord(nd.done, stream), "cudaEventRecord");
  return IFNSO_OK;
}

ifnso_status ifnso_learn_coefficients(int32_t L, int32_t iters, int32_t samples, double lr, int32_t step_size,
                                      double gamma, uint32_t seed, double* w_out) {
  if (L < 1 || L > 30 || iters < 0 || samples < 1 || samples > 4096 || !w_out)
    return fail(IFNSO_ERR_INVALID_ARG, "learn: L in [1,30], samples in [1,4096], iters >= 0");
  double* d_w = nullptr;
  IFNSO_CUDA(cudaMalloc(&d_w, sizeof(double) * L), "cudaMalloc");
  const double cL = std::exp(0.5) * (std::pow(2.0, L / 2.0) - 1.0);
  cudaError_t e = launch_learn(L, iters, samples, lr, step_size, gamma, seed, cL, d_w, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(w_out, d_w, sizeof(double) * L, cudaMemcpyDeviceToHost);
  cudaFree(d_w);
  if (e != cudaSuccess) return cuda_fail(e, "coefficient learning");
  return IFNSO_OK;
}

ifnso_status ifnso_synth_lowrank_bf16(void* out, int64_t rows, int64_t cols, int64_t ld, uint32_t seed, float alpha,
                                      float beta, ifnso_stream_t stream_) {
  if (!out || rows <= 0 || cols <= 0 || ld < cols || rows > 0xFFFFFFFFll || cols > 0xFFFFFFFFll)
    return fail(IFNSO_ERR_INVALID_ARG, "synth: bad shape or pointer");
  if ((rows + 31) / 32 > 65535) return fail(IFNSO_ERR_INVALID_ARG, "synth: too many rows");
  IFNSO_CUDA(launch_synth_lowrank(out, rows, cols, ld, seed, alpha, beta, reinterpret_cast<cudaStream_t>(stream_)),
             "synth");
  return IFNSO_OK;
}

// ------------------------------------------------------------------ coefficient proposal

int32_t ifnso_mlp_param_count(int32_t K) { return (K >= 2 && K <= 31) ? mlp_param_count(K) : 0; }

ifnso_status ifnso_mlp_create(ifnso_mlp** out, int32_t K, const double* wfix, const float* params, uint32_t seed) {
  if (!out || !wfix || K < 3 || K > 31) return fail(IFNSO_ERR_INVALID_ARG, "mlp: K must be in [3, 31] and wfix given");
  *out = nullptr;
  ifnso_mlp* m = new (std::nothrow) ifnso_mlp();
  if (!m) return fail(IFNSO_ERR_OOM, "out of host memory");
  m->K = K;
  m->L = K - 1;
  m->P = mlp_param_count(K);
  const int P = m->P, L = m->L, NO = K + 1;
  std::vector<float> init(P, 0.f);
  if (params) {
    memcpy(init.data(), params, sizeof(float) * P);
  } else {
    // W1 ~ N(0, 1/6), W2 ~ N(0, 1/64), W3 ~ 0.01 N(0, 1/64), biases 0
    const int oW1 = 0, ob1 = 64 * 6, oW2 = ob1 + 64, ob2 = oW2 + 64 * 64, oW3 = ob2 + 64;
    uint32_t i = 0;
    for (int k = 0; k < 64 * 6; ++k) init[oW1 + k] = static_cast<float>(host_normal(seed, i++) / std::sqrt(6.0));
    for (int k = 0; k < 64 * 64; ++k) init[oW2 + k] = static_cast<float>(host_normal(seed, i++) / 8.0);
    for (int k = 0; k < NO * 64; ++k) init[oW3 + k] = static_cast<float>(0.01 * host_normal(seed, i++) / 8.0);
  }
  std::vector<float> wf(L), ws(K), sc(L), st(12);
  for (int l = 0; l < L; ++l) {
    wf[l] = static_cast<float>(wfix[l]);
    ws[1 + l] = wf[l];
    sc[l] = static_cast<float>(std::max(1.0, std::fabs(wfix[l])) / 10.0);
  }
  ws[0] = 1.f;
  for (int f = 0; f < 6; ++f) {
    st[f] = 0.f;
    st[6 + f] = 1.f;
  }
  cudaError_t e = cudaSuccess;
  auto alloc = [&](float** p, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc(p, n * sizeof(float));
  };
  alloc(&m->prm, P);
  alloc(&m->mom, P);
  alloc(&m->vel, P);
  alloc(&m->grad, P);
  alloc(&m->wfix, L);
  alloc(&m->wslots, K);
  alloc(&m->scale, L);
  alloc(&m->stats, 12);
  if (e == cudaSuccess) e = cudaMemcpy(m->prm, init.data(), sizeof(float) * P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->mom, 0, sizeof(float) * P);
  if (e == cudaSuccess) e = cudaMemset(m->vel, 0, sizeof(float) * P);
  if (e == cudaSuccess) e = cudaMemcpy(m->wfix, wf.data(), sizeof(float) * L, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->wslots, ws.data(), sizeof(float) * K, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->scale, sc.data(), sizeof(float) * L, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->stats, st.data(), sizeof(float) * 12, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    ifnso_mlp_destroy(m);
    return cuda_fail(e, "mlp create");
  }
  *out = m;
  return IFNSO_OK;
}

ifnso_status ifnso_mlp_destroy(ifnso_mlp* m) {
  if (!m) return IFNSO_OK;
  cudaDeviceSynchronize();
  mlp_free_data(m);
  for (float* p : {m->prm, m->mom, m->vel, m->grad, m->wfix, m->wslots, m->scale, m->stats, m->grad_part,
                   m->loss_part})
    cudaFree(p);
  cudaFree(m->idx);
  delete m;
  return IFNSO_OK;
}

ifnso_status ifnso_mlp_get_params(const ifnso_mlp* m, float* params, float* stats) {
  if (!m) return fail(IFNSO_ERR_INVALID_ARG, "mlp is NULL");
  IFNSO_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  if (params) IFNSO_CUDA(cudaMemcpy(params, m->prm, sizeof(float) * m->P, cudaMemcpyDeviceToHost), "copy");
  if (stats) IFNSO_CUDA(cudaMemcpy(stats, m->stats, sizeof(float) * 12, cudaMemcpyDeviceToHost), "copy");
  return IFNSO_OK;
}

ifnso_status ifnso_mlp_set_params(ifnso_mlp* m, const float* params, const float* stats) {
  if (!m) return fail(IFNSO_ERR_INVALID_ARG, "mlp is NULL");
  IFNSO_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  if (params) IFNSO_CUDA(cudaMemcpy(m->prm, params, sizeof(float) * m->P, cudaMemcpyHostToDevice), "copy");
  if (stats) IFNSO_CUDA(cudaMemcpy(m->stats, stats, sizeof(float) * 12, cudaMemcpyHostToDevice), "copy");
  return IFNSO_OK;
}

ifnso_status ifnso_mlp_set_data(ifnso_mlp* m, int32_t n, const float* sigma, const int64_t* offsets,
                                const int32_t* h, const int32_t* w, int32_t fit, ifnso_stream_t stream_) {
  if (!m || n <= 0 || !sigma || !offsets || !h || !w) return fail(IFNSO_ERR_INVALID_ARG, "mlp_set_data: bad argument");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(m->mu);
  IFNSO_CUDA(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
  mlp_free_data(m);
  int64_t total = 0;
  IFNSO_CUDA(cudaMemcpy(&total, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost), "copy");
  if (total <= 0) return fail(IFNSO_ERR_INVALID_ARG, "mlp_set_data: empty data set");
  IFNSO_CUDA(cudaMalloc(&m->xs, sizeof(float) * total), "cudaMalloc");
  IFNSO_CUDA(cudaMalloc(&m->raw, sizeof(float) * 8 * n), "cudaMalloc");
  IFNSO_CUDA(cudaMalloc(&m->z, sizeof(float) * 8 * n), "cudaMalloc");
  IFNSO_CUDA(cudaMalloc(&m->offs, sizeof(int64_t) * (n + 1)), "cudaMalloc");
  IFNSO_CUDA(cudaMalloc(&m->hs, sizeof(int32_t) * n), "cudaMalloc");
  IFNSO_CUDA(cudaMemcpyAsync(m->offs, offsets, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, stream), "copy");
  IFNSO_CUDA(cudaMemcpyAsync(m->hs, h, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, stream), "copy");
  m->n = n;
  IFNSO_CUDA(mlp_prepare(n, sigma, m->offs, m->hs, w, m->xs, m->raw, m->stats, fit, m->z, stream), "mlp features");
  return IFNSO_OK;
}

ifnso_status ifnso_mlp_loss_grad(ifnso_mlp* m, const int32_t* idx, int32_t batch, float* grad, float* loss,
                                 ifnso_stream_t stream_) {
  if (!m || !idx || batch <= 0) return fail(IFNSO_ERR_INVALID_ARG, "mlp_loss_grad: bad argument");
  if (m->n == 0) return fail(IFNSO_ERR_INVALID_ARG, "mlp_loss_grad: no data set");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(m->mu);
  ifnso_status st = mlp_ensure_batch(m, batch);
  if (st != IFNSO_OK) return st;
  IFNSO_CUDA(mlp_grad(m->prm, m->K, m->wfix, m->scale, m->z, m->xs, m->offs, m->hs, idx, batch, m->grad_part,
                      m->loss_part, stream),
             "mlp forward/backward");
  IFNSO_CUDA(mlp_reduce_adam(m->K, batch, m->grad_part, m->loss_part, grad, loss, m->prm, m->mom, m->vel, 0, 0.f, 0,
                             stream),
             "mlp reduce");
  return IFNSO_OK;
}

ifnso_status ifnso_mlp_train(ifnso_mlp* m, int32_t steps, int32_t batch, float lr, uint32_t seed, float* loss_curve,
                             ifnso_stream_t stream_) {
  if (!m || steps < 0 || batch <= 0) return fail(IFNSO_ERR_INVALID_ARG, "mlp_train: bad argument");
  if (m->n == 0) return fail(IFNSO_ERR_INVALID_ARG, "mlp_train: no data set");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(m->mu);
  ifnso_status st = mlp_ensure_batch(m, batch);
  if (st != IFNSO_OK) return st;
  for (int s = 0; s < steps; ++s) {
    ++m->step;
    IFNSO_CUDA(mlp_batch_idx(batch, m->step, seed, m->n, m->idx, stream), "mlp batch");
    IFNSO_CUDA(mlp_grad(m->prm, m->K, m->wfix, m->scale, m->z, m->xs, m->offs, m->hs, m->idx, batch, m->grad_part,
                        m->loss_part, stream),
               "mlp forward/backward");
    IFNSO_CUDA(mlp_reduce_adam(m->K, batch, m->grad_part, m->loss_part, m->grad, loss_curve ? loss_curve + s : nullptr,
                               m->prm, m->mom, m->vel, m->step, lr, 1, stream),
               "mlp adam");
  }
  return IFNSO_OK;
}

ifnso_status ifnso_mlp_evaluate(const ifnso_mlp* m, const int32_t* idx, int32_t n, float* e_mlp, float* e_fix,
                                float* coeffs, int32_t* fallback, ifnso_stream_t stream_) {
  if (!m || n <= 0 || !e_mlp || !e_fix) return fail(IFNSO_ERR_INVALID_ARG, "mlp_evaluate: bad argument");
  if (m->n == 0) return fail(IFNSO_ERR_INVALID_ARG, "mlp_evaluate: no data set");
  if (!idx && n > m->n) return fail(IFNSO_ERR_INVALID_ARG, "mlp_evaluate: n exceeds the data set");
  IFNSO_CUDA(mlp_eval(m->prm, m->K, m->wfix, m->scale, m->z, m->xs, m->offs, m->hs, idx, n, e_mlp, e_fix, coeffs,
                      fallback, reinterpret_cast<cudaStream_t>(stream_)),
             "mlp evaluate");
  return IFNSO_OK;
}

}  // extern "C"
