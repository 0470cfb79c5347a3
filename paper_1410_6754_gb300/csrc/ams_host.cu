// Host side of libams: plan of the levels, scratch memory (contexts), the launch
// sequence of one sort and the C ABI declared in include/ams.h.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ams_internal.cuh"
#include "rlm.cuh"

namespace ams {

cudaError_t launch_sample_sort_ex(const LevelArgs& a, int ksize, int grid, void* raw_out,
                                  const void* sample_in, cudaStream_t s);
cudaError_t launch_splitters_ex(const LevelArgs& a, int ksize, int grid, void* sorted_out,
                                cudaStream_t s);

namespace {

// ------------------------------------------------------------------------- plan
struct LevelPlan {
  uint32_t r, B, logBp, nid, CH;
  uint64_t nseg_cap, samples_cap, items_cap, bc_cap, next_cap;
};

struct Plan {
  int L = 0;
  uint32_t b = 0, a_fixed = 0, C = 0;
  int ksize = 8;
  bool pairs = false;
  bool small = false;  // base case of half the capacity (C <= its capacity)
  uint64_t n = 0, nseg_user = 1;
  uint64_t seg1_cap = 0, bc0_cap = 0, big_cap = 0, tiny_cap = 0;
  LevelPlan lv[kMaxLevels];
};

uint32_t default_cap(ams_key_type kt, bool pairs) {
  if (pairs) return 8192;
  return (kt == AMS_U32 || kt == AMS_F32) ? 16384u : 8192u;
}

int ksize_of(ams_key_type kt) { return kt == AMS_U64 ? 8 : 4; }

ams_status make_plan(uint64_t n, uint64_t nseg_user, ams_key_type kt, bool pairs, int levels,
                     const uint32_t* r, const ams_options* opt, int sm_count, Plan* p) {
  if (levels < 1 || levels > kMaxLevels || r == nullptr) return AMS_ERR_INVALID;
  if (kt != AMS_U32 && kt != AMS_U64 && kt != AMS_F32) return AMS_ERR_INVALID;
  ams_options o{};
  if (opt) o = *opt;
  p->ksize = ksize_of(kt);
  p->pairs = pairs;
  p->n = n;
  p->nseg_user = nseg_user;
  p->b = o.overpartition_b ? o.overpartition_b : (levels == 1 ? 1u : 4u);
  p->a_fixed = o.oversample_a;
  if (p->a_fixed > 64) return AMS_ERR_INVALID;
  const uint32_t maxcap = basecase_max_cap(p->ksize, pairs);
  p->C = o.basecase_cap ? o.basecase_cap : default_cap(kt, pairs);
  if (p->C > maxcap) return AMS_ERR_UNSUPPORTED;
  std::vector<uint32_t> rr(r, r + levels);
  for (uint32_t x : rr)
    if (x < 2) return AMS_ERR_INVALID;
  uint64_t est = n;
  for (uint32_t x : rr) est = (est + x - 1) / x;
  while (est > p->C && (int)rr.size() < kMaxLevels) {
    rr.push_back(rr.back());
    est = (est + rr.back() - 1) / rr.back();
  }
  p->L = (int)rr.size();
  // a sort of one segment larger than the capacity whose leaves are expected to fit
  // the base case of half the capacity (with 25% slack for uneven groups) uses it:
  // pairs get two blocks per SM, 32-bit keys half the registers per thread (64-bit
  // keys have no such variant)
  const uint32_t small_cap = basecase_small_cap(p->ksize, pairs);
  if (small_cap && !o.basecase_cap && nseg_user == 1 && n > p->C && est * 5 / 4 <= small_cap)
    p->C = small_cap;
  p->small = small_cap && p->C <= small_cap;
  // every segment holds at most C keys: level 0 hands them all to the base case and
  // the distribution levels would find no work, so none is launched
  if (n <= p->C) p->L = 0;
  const uint64_t C = p->C;
  const uint64_t big = n / (C + 1) + 1;  // segments larger than C that fit in n
  p->seg1_cap = std::min<uint64_t>(nseg_user, big);
  p->bc0_cap = std::min<uint64_t>(nseg_user, n) + 1;
  p->tiny_cap = p->bc0_cap;
  p->big_cap = big;
  uint64_t nseg_cap = p->seg1_cap;
  const uint64_t chunk_goal = (n + (uint64_t)sm_count * 8 - 1) / ((uint64_t)sm_count * 8);
  for (int l = 0; l < p->L; ++l) {
    LevelPlan& lp = p->lv[l];
    lp.r = rr[l];
    const uint64_t B = (uint64_t)p->b * rr[l];
    if (B < 2 || B > (uint64_t)kMaxBuckets) return AMS_ERR_UNSUPPORTED;
    lp.B = (uint32_t)B;
    lp.logBp = 0;
    while ((1u << lp.logBp) < lp.B) ++lp.logBp;
    lp.nid = 2 * lp.B - 1;
    lp.CH = (uint32_t)std::max<uint64_t>(8192, (chunk_goal + 8191) / 8192 * 8192);
    lp.nseg_cap = std::max<uint64_t>(nseg_cap, 1);
    lp.samples_cap = lp.nseg_cap * B + n / 16 + 1;
    lp.items_cap = n / lp.CH + lp.nseg_cap + 1;
    lp.bc_cap = 5 * (n / C + 1) + lp.nseg_cap * lp.r + n / kCopyChunk + 16;
    lp.next_cap = std::min<uint64_t>(lp.nseg_cap * (2 * B - 1), big);
    nseg_cap = lp.next_cap;
  }
  return AMS_OK;
}

// -------------------------------------------------------------------- workspace
struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(uint64_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += (size_t)count * sizeof(T);
    return p;
  }
};

struct LevelBufs {
  Seg* segs_next;
  SegInfo* sinfo;
  void* sample;
  uint32_t* srank;
  void* spl;
  uint32_t* counts;
  uint32_t* totals;
  uint32_t* seg_L;
  uint32_t* seg_ng;
  BcItem* bc;
  void* cls_head;
  uint32_t* J2;
  uint16_t* piece_of;
  uint32_t* piece_start;
  uint32_t* npieces;
};

struct Bufs {
  void* tmp;
  uint64_t* vtmp;
  LevelCounters* ctr;  // L + 1 entries: [0] = init, [l] = level l
  uint32_t* status;
  Seg* segs1;
  BcItem* bc0;
  BcItem* tiny;
  BcItem* big;
  uint16_t* ids;  // bucket id of every key (rewritten by each level)
  LevelBufs lv[kMaxLevels];
};

size_t carve(const Plan& p, char* base, Bufs* b) {
  Carver c{base};
  b->status = c.take<uint32_t>(64);
  b->ctr = c.take<LevelCounters>(kMaxLevels + 1);
  b->tmp = c.take<char>(p.n * p.ksize);
  b->ids = c.take<uint16_t>(p.n + 8);  // the scatter copies ids in 4-byte words
  b->vtmp = p.pairs ? c.take<uint64_t>(p.n) : nullptr;
  b->segs1 = c.take<Seg>(p.seg1_cap + 1);
  b->bc0 = c.take<BcItem>(p.bc0_cap);
  b->tiny = c.take<BcItem>(p.tiny_cap);
  b->big = c.take<BcItem>(p.big_cap + 1);
  for (int l = 0; l < p.L; ++l) {
    const LevelPlan& lp = p.lv[l];
    LevelBufs& lb = b->lv[l];
    lb.sinfo = c.take<SegInfo>(lp.nseg_cap);
    lb.sample = c.take<char>(lp.samples_cap * p.ksize);
    lb.srank = c.take<uint32_t>(lp.samples_cap);
    lb.spl = c.take<char>(lp.nseg_cap * (lp.B - 1) * p.ksize);
    lb.counts = c.take<uint32_t>(lp.items_cap * lp.nid);
    lb.totals = c.take<uint32_t>(lp.nseg_cap * lp.nid);
    lb.seg_L = c.take<uint32_t>(lp.nseg_cap);
    lb.seg_ng = c.take<uint32_t>(lp.nseg_cap);
    lb.bc = c.take<BcItem>(lp.bc_cap);
    lb.segs_next = c.take<Seg>(lp.next_cap + 1);
    lb.cls_head = c.take<char>(lp.nseg_cap * 16);
    lb.J2 = c.take<uint32_t>(lp.nseg_cap * kCellTable);
    lb.piece_of = c.take<uint16_t>(lp.nseg_cap * lp.nid);
    lb.piece_start = c.take<uint32_t>(lp.nseg_cap * lp.nid);
    lb.npieces = c.take<uint32_t>(lp.nseg_cap);
  }
  return c.off + 256;
}

}  // namespace

// ---------------------------------------------------------------------- context
struct Context {
  int device = 0;
  uint64_t budget = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  uint32_t* d_status = nullptr;  // lives at the start of ws
  cudaStream_t last_stream = nullptr;
  bool has_run = false;
  int sm_count = 148;
  // statistics of the last sort
  Plan last_plan;
  Bufs last_bufs{};
  uint32_t launches = 0;
  bool timers = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  uint64_t kind_elems[AMS_K_COUNT] = {};
  // host-buffer calls
  char* stage = nullptr;
  size_t stage_bytes = 0;
  // step calls
  char* step_ws = nullptr;
  size_t step_bytes = 0;
  // graphs per size class (AMS_FLAG_GRAPH)
  struct GraphEntry {
    int kt = 0, levels = 0;
    uint32_t r[kMaxLevels] = {}, a = 0, b = 0, cap = 0, flags = 0;
    uint64_t seed = 0, n_class = 0, ws_gen = 0;
    char* buf = nullptr;  // input then output, n_class keys each
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy_in = nullptr, pad = nullptr, copy_out = nullptr;
    uint32_t launches = 0;  // kernels of the captured sort
  };
  std::vector<GraphEntry> graphs;
  size_t graph_bytes = 0;
  uint64_t ws_gen = 0;  // bumped whenever the workspace moves (captured graphs then stale)
  cudaStream_t cap_stream = nullptr;
  // RLM-sort tables (pinned staging; the event marks the end of the last copy)
  void* rlm_host = nullptr;
  size_t rlm_host_bytes = 0;
  cudaEvent_t rlm_done = nullptr;
  cudaStream_t rlm_stream = nullptr;
  bool rlm_pending = false;
  std::mutex mu;
};

static ams_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return AMS_OK;
  if (e == cudaErrorMemoryAllocation) return AMS_ERR_OOM;
  return AMS_ERR_CUDA;
}

#define AMS_TRY(expr)                           \
  do {                                          \
    cudaError_t _e = (expr);                    \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

static ams_status grow(Context* cx, char** buf, size_t* have, size_t need) {
  if (*have >= need) return AMS_OK;
  const size_t total = cx->ws_bytes + cx->stage_bytes + cx->step_bytes + cx->graph_bytes - *have + need;
  if (cx->budget && total > cx->budget) return AMS_ERR_OOM;
  if (*buf) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_status(e);
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AMS_ERR_OOM;
  }
  *buf = (char*)p;
  *have = need;
  return AMS_OK;
}

static ams_status ensure_ws(Context* cx, size_t need) {
  const bool fresh = cx->ws == nullptr || cx->ws_bytes < need;
  ams_status st = grow(cx, &cx->ws, &cx->ws_bytes, need);
  if (st != AMS_OK) return st;
  if (fresh) {
    ++cx->ws_gen;
    cx->d_status = (uint32_t*)cx->ws;
    AMS_TRY(cudaMemset(cx->d_status, 0, 256));
  }
  return AMS_OK;
}

static std::mutex g_default_mu;
static Context* g_default[64] = {};

static Context* default_context() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_default_mu);
  if (!g_default[dev]) {
    Context* cx = new (std::nothrow) Context();
    if (!cx) return nullptr;
    cx->device = dev;
    cudaDeviceGetAttribute(&cx->sm_count, cudaDevAttrMultiProcessorCount, dev);
    g_default[dev] = cx;
  }
  return g_default[dev];
}

// Kernel launch bookkeeping: count, and optional events around the launch.
struct Launcher {
  Context* cx;
  cudaStream_t s;
  int kind = 0;
  void begin(int k) {
    kind = k;
    if (!cx->timers) return;
    if (cx->ev_used + 2 > cx->ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cx->ev_pool.push_back(e);
      }
    }
    cudaEventRecord(cx->ev_pool[cx->ev_used], s);
  }
  cudaError_t end(cudaError_t e) {
    cx->launches++;
    if (cx->timers) {
      cudaEventRecord(cx->ev_pool[cx->ev_used + 1], s);
      cx->ev_kind.push_back(kind);
      cx->ev_used += 2;
    }
    return e;
  }
};

static void fill_thr(double* thr) {
  for (int a = 0; a < kThrCount; ++a) thr[a] = std::pow(10.0, a / 1.6);
}

// --------------------------------------------------------------- one whole sort
static ams_status run_sort_graph(Context* cx, const ams_request* rq, cudaStream_t s);

static ams_status run_sort(Context* cx, const ams_request* rq, cudaStream_t s) {
  if (!rq) return AMS_ERR_INVALID;
  const bool pairs = rq->vals_in != nullptr || rq->vals_out != nullptr;
  if (pairs && (rq->vals_in == nullptr || rq->vals_out == nullptr)) return AMS_ERR_INVALID;
  if (rq->n >= 0xFFFFFFFFull) return AMS_ERR_UNSUPPORTED;
  const uint64_t nseg_user = rq->d_offsets ? rq->nseg : 1;
  if (rq->n == 0 || nseg_user == 0) return AMS_OK;  // nothing to sort
  if (!rq->keys_in || !rq->keys_out) return AMS_ERR_INVALID;
  const int ks = ksize_of(rq->kt);
  if (((uintptr_t)rq->keys_in % ks) || ((uintptr_t)rq->keys_out % ks)) return AMS_ERR_INVALID;
  if ((rq->opt.flags & AMS_FLAG_GRAPH) && !pairs && !rq->d_offsets && rq->n >= 2 &&
      !(rq->opt.flags & AMS_FLAG_PHASE_TIMERS))
    return run_sort_graph(cx, rq, s);
  Plan p;
  ams_status st = make_plan(rq->n, nseg_user, rq->kt, pairs, rq->levels, rq->buckets_per_level,
                            &rq->opt, cx->sm_count, &p);
  if (st != AMS_OK) return st;
  Bufs b{};
  const size_t need = carve(p, nullptr, &b);
  if ((st = ensure_ws(cx, need)) != AMS_OK) return st;
  carve(p, cx->ws, &b);

  // launch counts and kernel events accumulate until ams_get_stats reads them
  cx->timers = (rq->opt.flags & AMS_FLAG_PHASE_TIMERS) != 0;
  cx->last_plan = p;
  cx->last_bufs = b;
  cx->last_stream = s;
  cx->has_run = true;

  const bool f32 = rq->kt == AMS_F32;
  const bool tree = (rq->opt.flags & AMS_FLAG_TREE_CLASSIFIER) != 0;
  const bool inplace = rq->keys_in == rq->keys_out;
  const int SM = cx->sm_count;
  Launcher ln{cx, s};

  AMS_TRY(cudaMemsetAsync(b.ctr, 0, sizeof(LevelCounters) * (kMaxLevels + 1), s));

  // level 0: split the user's segments
  InitArgs ia{};
  ia.offsets = rq->d_offsets;
  ia.nseg = nseg_user;
  ia.n = (uint32_t)rq->n;
  ia.C = p.C;
  ia.need_copy_small = (!inplace || f32) ? 1 : 0;
  ia.segs1 = b.segs1;
  ia.bc0 = b.bc0;
  ia.tiny = b.tiny;
  ia.ctr0 = &b.ctr[0];
  ia.status = b.status;
  ia.seg_cap = (uint32_t)p.seg1_cap;
  ia.bc_cap = (uint32_t)p.bc0_cap;
  ia.tiny_cap = (uint32_t)p.tiny_cap;
  const int init_grid = (int)std::min<uint64_t>((nseg_user + 255) / 256, (uint64_t)SM * 8);
  ln.begin(AMS_K_INIT);
  AMS_TRY(ln.end(launch_init(ia, init_grid, s)));

  // more blocks than fit at once: the block scheduler balances items of uneven size
  const uint64_t bc_grid_cap = (uint64_t)SM * 8;
  BaseArgs ba{};
  ba.out = rq->keys_out;
  ba.vout = rq->vals_out;
  auto run_basecase = [&](const void* src, const uint64_t* vsrc, const BcItem* items,
                          const uint32_t* nitems, int tf_load, uint64_t cap_items,
                          bool big) -> ams_status {
    ba.src = src;
    ba.vsrc = vsrc;
    // the merge fallback ping-pongs between the output and the temporary buffer: an
    // item sits either in the temporary buffer itself (free to overwrite once read)
    // or in the output / input, where the temporary buffer's positions are unused
    ba.scratch = b.tmp;
    ba.vscratch = b.vtmp;
    ba.items = items;
    ba.nitems = nitems;
    ba.tf_load = tf_load;
    ba.tf_store = f32 ? 1 : 0;
    ba.status = b.status;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(cap_items, bc_grid_cap));
    ln.begin(AMS_K_BASECASE);
    cudaError_t e = ln.end(launch_basecase(ba, p.ksize, p.pairs, big, grid, s, p.small));
    return cuda_status(e);
  };
  // no offsets and n above C: one segment [0, n) that level 0 hands to level 1, so
  // there is no base-case item and no tiny segment
  const bool one_big = rq->d_offsets == nullptr && rq->n > p.C;
  if (!one_big && (st = run_basecase(rq->keys_in, rq->vals_in, b.bc0, &b.ctr[0].n_bc, f32 ? 1 : 0,
                                     p.bc0_cap, false)) != AMS_OK)
    return st;
  if (!one_big) {
    // user segments of at most kTiny keys: one warp each (all-pairs ranks)
    BaseArgs ta = ba;
    ta.src = rq->keys_in;
    ta.vsrc = rq->vals_in;
    ta.items = b.tiny;
    ta.nitems = &b.ctr[0].n_tiny;
    ta.tf_load = f32 ? 1 : 0;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((p.tiny_cap + 15) / 16, (uint64_t)SM * 4));
    ln.begin(AMS_K_BASECASE);
    AMS_TRY(ln.end(launch_tiny(ta, p.ksize, p.pairs, grid, s)));
  }

  LevelArgs la{};
  fill_thr(la.a_thr);
  la.seed = rq->seed;
  la.a_fixed = p.a_fixed;
  la.C = p.C;
  la.status = b.status;
  for (int l = 1; l <= p.L; ++l) {
    const LevelPlan& lp = p.lv[l - 1];
    const LevelBufs& lb = b.lv[l - 1];
    la.level = l;
    la.B = lp.B;
    la.logBp = lp.logBp;
    la.nid = lp.nid;
    la.r = lp.r;
    la.CH = lp.CH;
    la.last = l == p.L;
    // Delivery targets alternate between the output and the temporary buffer.  An
    // out-of-place sort (keys and payloads) delivers level 1 straight into the output,
    // so that the pieces a level-1 delivery already finalises (equality buckets of
    // duplicate-heavy input) need no copy; an in-place sort must deliver level 1 into
    // the temporary buffer, since the output is its input.
    const bool out_of_place = !inplace && (!rq->vals_in || rq->vals_in != rq->vals_out);
    auto to_out = [&](int lv) { return ((lv % 2) == 1) == out_of_place; };
    la.dst = to_out(l) ? rq->keys_out : b.tmp;
    la.vdst = to_out(l) ? rq->vals_out : b.vtmp;
    if (l == 1) {
      la.src = rq->keys_in;
      la.vsrc = rq->vals_in;
      la.tf_src = f32 ? 1 : 0;
      la.segs = b.segs1;
    } else {
      la.src = to_out(l - 1) ? rq->keys_out : b.tmp;
      la.vsrc = to_out(l - 1) ? rq->vals_out : b.vtmp;
      la.tf_src = 0;
      la.segs = b.lv[l - 2].segs_next;
    }
    la.copy_final = (la.dst != rq->keys_out || f32) ? 1 : 0;
    la.in_ctr = &b.ctr[l - 1];
    la.ctr = &b.ctr[l];
    la.sinfo = lb.sinfo;
    la.sample = lb.sample;
    la.srank = lb.srank;
    la.spl = lb.spl;
    la.counts = lb.counts;
    la.totals = lb.totals;
    la.seg_L = lb.seg_L;
    la.seg_ng = lb.seg_ng;
    la.group_ends = nullptr;
    la.segs_next = lb.segs_next;
    la.bc = lb.bc;
    la.cls_head = lb.cls_head;
    la.J2 = lb.J2;
    la.piece_of = lb.piece_of;
    la.piece_start = lb.piece_start;
    la.npieces = lb.npieces;
    la.ids = b.ids;
    la.pieces_per_id = 0;
    la.nseg_cap = (uint32_t)lp.nseg_cap;
    la.samples_cap = (uint32_t)std::min<uint64_t>(lp.samples_cap, 0xFFFFFFFFull);
    la.items_cap = (uint32_t)std::min<uint64_t>(lp.items_cap, 0xFFFFFFFFull);
    la.next_cap = (uint32_t)lp.next_cap;
    la.bc_cap = (uint32_t)std::min<uint64_t>(lp.bc_cap, 0xFFFFFFFFull);
    la.big = b.big;
    la.big_cap = (uint32_t)p.big_cap;
    const int wide = SM * 4;
    const int seg_grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(lp.nseg_cap, (uint64_t)SM * 2));
    ln.begin(AMS_K_SETUP);
    AMS_TRY(ln.end(launch_setup(la, s)));
    ln.begin(AMS_K_SAMPLE_SORT);
    AMS_TRY(ln.end(launch_sample_sort(la, p.ksize, wide, s)));
    ln.begin(AMS_K_CROSS_RANK);
    AMS_TRY(ln.end(launch_cross_rank(la, p.ksize, wide, s)));
    ln.begin(AMS_K_SPLITTERS);
    AMS_TRY(ln.end(launch_splitters(la, p.ksize, wide, s)));
    ln.begin(AMS_K_TABLE);
    AMS_TRY(ln.end(launch_table(la, p.ksize, seg_grid, s)));
    ln.begin(AMS_K_CLASSIFY);
    AMS_TRY(ln.end(launch_classify(la, p.ksize, tree, SM * 6, s)));
    ln.begin(AMS_K_SCAN);
    AMS_TRY(ln.end(launch_scan(la, SM * 8, lp.nseg_cap <= 16, s)));
    ln.begin(AMS_K_BINPACK);
    AMS_TRY(ln.end(launch_binpack(la, seg_grid, s)));
    ln.begin(AMS_K_SCATTER);
    AMS_TRY(ln.end(launch_scatter(la, p.ksize, p.pairs, /*stable=*/p.pairs, SM * (p.pairs ? 2 : p.ksize == 4 ? 4 : 6), s)));
    if ((st = run_basecase(la.dst, la.vdst, lb.bc, &b.ctr[l].n_bc, 0, lp.bc_cap, false)) != AMS_OK)
      return st;
    if (la.last && (st = run_basecase(la.dst, la.vdst, b.big, &b.ctr[l].n_big, 0, p.big_cap, true)) != AMS_OK)
      return st;
  }
  return AMS_OK;
}

// ---------------------------------------------------------------- graphs per class
// Keys at or after the last position of a padded request: the largest key of the
// type in order form, stored as its bit pattern (f32: 0x7FFFFFFF, whose order map is
// the largest 32-bit value).
__global__ void k_fill_pad(void* p, uint64_t count, int ksize, uint64_t pattern) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    if (ksize == 8) ((uint64_t*)p)[i] = pattern;
    else ((uint32_t*)p)[i] = (uint32_t)pattern;
  }
}

static bool same_plan(const Context::GraphEntry& g, const ams_request* rq, uint64_t n_class) {
  if (g.kt != (int)rq->kt || g.levels != rq->levels || g.n_class != n_class || g.seed != rq->seed) return false;
  for (int l = 0; l < rq->levels; ++l)
    if (g.r[l] != rq->buckets_per_level[l]) return false;
  return g.a == rq->opt.oversample_a && g.b == rq->opt.overpartition_b && g.cap == rq->opt.basecase_cap &&
         g.flags == (rq->opt.flags & ~AMS_FLAG_GRAPH);
}

static void pad_params(cudaKernelNodeParams& kp, void** args, void*& ptr, uint64_t& cnt, int& ks, uint64_t& pat,
                       int grid) {
  kp = cudaKernelNodeParams{};
  kp.func = (void*)k_fill_pad;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(256);
  args[0] = &ptr;
  args[1] = &cnt;
  args[2] = &ks;
  args[3] = &pat;
  kp.kernelParams = args;
}

static ams_status run_sort_graph(Context* cx, const ams_request* rq, cudaStream_t s) {
  const int ks = ksize_of(rq->kt);
  uint64_t n_class = 1024;
  while (n_class < rq->n) n_class <<= 1;
  if (n_class >= 0xFFFFFFFFull) return AMS_ERR_UNSUPPORTED;
  const uint64_t pattern = rq->kt == AMS_F32 ? 0x7FFFFFFFull : ~0ull;
  Context::GraphEntry* ge = nullptr;
  for (auto& g : cx->graphs)
    if (same_plan(g, rq, n_class)) ge = &g;
  if (ge && ge->ws_gen != cx->ws_gen) {  // its workspace moved: capture again
    cudaGraphExecDestroy(ge->exec);
    cudaGraphDestroy(ge->graph);
    ge->exec = nullptr;
    ge->graph = nullptr;
  }
  int pgrid = 64;
  void* pad_ptr = nullptr;
  uint64_t pad_cnt = 0;
  int pad_ks = ks;
  uint64_t pad_pat = pattern;
  void* pargs[4];
  cudaKernelNodeParams kp;
  if (!ge || !ge->exec) {
    if (!ge) {
      cx->graphs.emplace_back();
      ge = &cx->graphs.back();
      ge->kt = (int)rq->kt;
      ge->levels = rq->levels;
      for (int l = 0; l < rq->levels; ++l) ge->r[l] = rq->buckets_per_level[l];
      ge->a = rq->opt.oversample_a;
      ge->b = rq->opt.overpartition_b;
      ge->cap = rq->opt.basecase_cap;
      ge->flags = rq->opt.flags & ~AMS_FLAG_GRAPH;
      ge->seed = rq->seed;
      ge->n_class = n_class;
      const size_t bytes = 2 * (size_t)n_class * ks;
      if (cx->budget && cx->ws_bytes + cx->stage_bytes + cx->step_bytes + cx->graph_bytes + bytes > cx->budget)
        return AMS_ERR_OOM;
      if (cudaMalloc(&ge->buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        cx->graphs.pop_back();
        return AMS_ERR_OOM;
      }
      cx->graph_bytes += bytes;
    }
    char* in = ge->buf;
    char* out = ge->buf + (size_t)n_class * ks;
    // the sort of the class size on the entry's buffers, captured on a stream of the
    // context's own (the workspace is sized first: nothing allocates during capture)
    ams_request inner = *rq;
    inner.keys_in = in;
    inner.keys_out = out;
    inner.n = n_class;
    inner.opt.flags &= ~(AMS_FLAG_GRAPH | AMS_FLAG_PHASE_TIMERS);
    const uint64_t need = ams_request_scratch_bytes(&inner);
    if (need == 0) return AMS_ERR_INVALID;
    ams_status st = ensure_ws(cx, need);
    if (st != AMS_OK) return st;
    if (!cx->cap_stream) AMS_TRY(cudaStreamCreateWithFlags(&cx->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t sort_graph = nullptr;
    const uint32_t l0 = cx->launches;
    AMS_TRY(cudaStreamBeginCapture(cx->cap_stream, cudaStreamCaptureModeThreadLocal));
    st = run_sort(cx, &inner, cx->cap_stream);
    const cudaError_t ce = cudaStreamEndCapture(cx->cap_stream, &sort_graph);
    if (st != AMS_OK || ce != cudaSuccess) {
      if (sort_graph) cudaGraphDestroy(sort_graph);
      cudaGetLastError();
      return st != AMS_OK ? st : AMS_ERR_CUDA;
    }
    ge->launches = cx->launches - l0;
    cx->launches = l0;
    ge->ws_gen = cx->ws_gen;
    // copy in -> pad fill -> the sort -> copy out
    cudaGraph_t g = nullptr;
    AMS_TRY(cudaGraphCreate(&g, 0));
    ge->graph = g;
    cudaGraphNode_t sort_node;
    AMS_TRY(cudaGraphAddMemcpyNode1D(&ge->copy_in, g, nullptr, 0, in, rq->keys_in, rq->n * ks,
                                     cudaMemcpyDeviceToDevice));
    pad_ptr = in + rq->n * ks;
    pad_cnt = n_class - rq->n;
    pad_params(kp, pargs, pad_ptr, pad_cnt, pad_ks, pad_pat, pgrid);
    AMS_TRY(cudaGraphAddKernelNode(&ge->pad, g, nullptr, 0, &kp));
    cudaGraphNode_t deps[2] = {ge->copy_in, ge->pad};
    AMS_TRY(cudaGraphAddChildGraphNode(&sort_node, g, deps, 2, sort_graph));
    cudaGraphDestroy(sort_graph);  // (the child node holds a copy)
    AMS_TRY(cudaGraphAddMemcpyNode1D(&ge->copy_out, g, &sort_node, 1, rq->keys_out, out, rq->n * ks,
                                     cudaMemcpyDeviceToDevice));
    AMS_TRY(cudaGraphInstantiate(&ge->exec, g, 0));
  } else {
    char* in = ge->buf;
    char* out = ge->buf + (size_t)n_class * ks;
    AMS_TRY(cudaGraphExecMemcpyNodeSetParams1D(ge->exec, ge->copy_in, in, rq->keys_in, rq->n * ks,
                                               cudaMemcpyDeviceToDevice));
    pad_ptr = in + rq->n * ks;
    pad_cnt = n_class - rq->n;
    pad_params(kp, pargs, pad_ptr, pad_cnt, pad_ks, pad_pat, pgrid);
    AMS_TRY(cudaGraphExecKernelNodeSetParams(ge->exec, ge->pad, &kp));
    AMS_TRY(cudaGraphExecMemcpyNodeSetParams1D(ge->exec, ge->copy_out, rq->keys_out, out, rq->n * ks,
                                               cudaMemcpyDeviceToDevice));
  }
  AMS_TRY(cudaGraphLaunch(ge->exec, s));
  cx->launches += ge->launches + 1;  // the sort's kernels and the pad fill
  cx->last_stream = s;
  return AMS_OK;
}

static ams_status read_status(Context* cx) {
  if (!cx->ws) return AMS_OK;
  uint32_t v = 0;
  AMS_TRY(cudaMemcpy(&v, cx->d_status, 4, cudaMemcpyDeviceToHost));
  if (v) AMS_TRY(cudaMemset(cx->d_status, 0, 4));
  if (v & ST_TIMEOUT) return AMS_ERR_TIMEOUT;
  if (v & ST_OVERFLOW) return AMS_ERR_INTERNAL;
  return AMS_OK;
}

// -------------------------------------------------------------------- step calls
struct StepWs {
  Seg* segs;
  LevelCounters* ctr;  // [0] input, [1] level
  SegInfo* sinfo;
  void* sample;
  uint32_t* srank;
  void* spl;
  uint32_t* counts;
  uint32_t* totals;
  uint32_t* seg_L;
  uint32_t* seg_ng;
  BcItem* bc;
  Seg* segs_next;
  void* cls_head;
  uint32_t* J2;
  uint16_t* piece_of;
  uint32_t* piece_start;
  uint32_t* npieces;
  uint16_t* ids;
};

__global__ void k_step_prepare(Seg* segs, LevelCounters* ctr, uint32_t begin, uint32_t end,
                               uint32_t* srank_iota, uint32_t iota_n) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    segs[0] = Seg{begin, end};
    ctr[0] = LevelCounters{};
    ctr[1] = LevelCounters{};
    ctr[0].nseg_next = 1;
  }
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < iota_n; i += gridDim.x * blockDim.x)
    srank_iota[i] = i;
}

__global__ void k_step_finish_binpack(const uint32_t* seg_L, const uint32_t* seg_ng, uint64_t* d_L,
                                      uint32_t* d_ng) {
  if (threadIdx.x == 0) {
    if (d_L) *d_L = seg_L[0];
    if (d_ng) *d_ng = seg_ng[0];
  }
}

__global__ void k_step_item(BcItem* items, LevelCounters* ctr, uint32_t b, uint32_t e) {
  if (threadIdx.x == 0) {
    items[0] = BcItem{b, e, BC_SORT, 0};
    *ctr = LevelCounters{};
    ctr->n_bc = 1;
  }
}

// Scratch for a one-segment level: up to `samples` sample keys, `B` buckets and
// `items` chunks.
static ams_status step_ws(Context* cx, uint64_t samples, uint32_t B, uint64_t items, int ks,
                          StepWs* w) {
  const uint32_t nid = 2 * B - 1;
  auto lay = [&](char* base) {
    Carver c{base};
    w->segs = c.take<Seg>(2);
    w->ctr = c.take<LevelCounters>(2);
    w->sinfo = c.take<SegInfo>(1);
    w->sample = c.take<char>((samples + 1) * ks);
    w->srank = c.take<uint32_t>(samples + 1);
    w->spl = c.take<char>((uint64_t)(B + 1) * ks);
    w->counts = c.take<uint32_t>(items * nid);
    w->totals = c.take<uint32_t>(nid + 1);
    w->seg_L = c.take<uint32_t>(1);
    w->seg_ng = c.take<uint32_t>(1);
    w->bc = c.take<BcItem>(2 * (uint64_t)nid + 16);
    w->segs_next = c.take<Seg>(2 * (uint64_t)nid + 16);
    w->cls_head = c.take<char>(16);
    w->J2 = c.take<uint32_t>(kCellTable);
    w->piece_of = c.take<uint16_t>(nid + 1);
    w->piece_start = c.take<uint32_t>(nid + 1);
    w->npieces = c.take<uint32_t>(1);
    w->ids = c.take<uint16_t>(items * 8192);  // covers n keys: items > n / 8192
    return c.off + 256;
  };
  const size_t need = lay(nullptr);
  ams_status st = grow(cx, &cx->step_ws, &cx->step_bytes, need);
  if (st != AMS_OK) return st;
  if (cx->ws == nullptr) {
    if ((st = ensure_ws(cx, 4096)) != AMS_OK) return st;
  }
  lay(cx->step_ws);
  return AMS_OK;
}

static LevelArgs step_level(Context* cx, const StepWs& w, uint32_t B, uint32_t a_fixed, uint32_t n) {
  LevelArgs la{};
  fill_thr(la.a_thr);
  la.level = 1;
  la.B = B;
  la.logBp = 0;
  while ((1u << la.logBp) < B) ++la.logBp;
  la.nid = 2 * B - 1;
  la.r = B;
  la.a_fixed = a_fixed;
  la.C = 0x7FFFFFFFu;
  la.CH = (uint32_t)std::max<uint64_t>(8192, ((uint64_t)n / (cx->sm_count * 4) + 8191) / 8192 * 8192);
  la.last = 1;
  la.copy_final = 0;
  la.segs = w.segs;
  la.in_ctr = &w.ctr[0];
  la.ctr = &w.ctr[1];
  la.sinfo = w.sinfo;
  la.sample = w.sample;
  la.srank = w.srank;
  la.spl = w.spl;
  la.counts = w.counts;
  la.totals = w.totals;
  la.seg_L = w.seg_L;
  la.seg_ng = w.seg_ng;
  la.segs_next = w.segs_next;
  la.bc = w.bc;
  la.cls_head = w.cls_head;
  la.J2 = w.J2;
  la.piece_of = w.piece_of;
  la.piece_start = w.piece_start;
  la.npieces = w.npieces;
  la.ids = w.ids;
  la.pieces_per_id = 0;
  la.status = cx->d_status;
  la.nseg_cap = 1;
  la.samples_cap = 0xFFFFFFFFu;
  la.items_cap = 0xFFFFFFFFu;
  la.next_cap = 2 * la.nid + 16;
  la.bc_cap = 2 * la.nid + 16;
  la.big = w.bc;   // step calls never leave a group above capacity (C is unbounded)
  la.big_cap = 0;
  return la;
}

}  // namespace ams

using namespace ams;

static Context* ctx_or_default(void* ctx) {
  return ctx ? static_cast<Context*>(ctx) : default_context();
}

static ams_status sort_common(const ams_request& rq, void* stream) {
  Context* cx = default_context();
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  return run_sort(cx, &rq, (cudaStream_t)stream);
}

static ams_request make_req(const void* in, void* out, const uint64_t* vin, uint64_t* vout,
                            uint64_t n, ams_key_type kt, int levels, const uint32_t* r,
                            uint64_t seed, const ams_options* opt) {
  ams_request rq{};
  rq.keys_in = in;
  rq.keys_out = out;
  rq.vals_in = vin;
  rq.vals_out = vout;
  rq.n = n;
  rq.kt = kt;
  rq.levels = levels;
  rq.buckets_per_level = r;
  rq.seed = seed;
  if (opt) rq.opt = *opt;
  return rq;
}

extern "C" {

ams_status ams_sort_keys(void* d_keys, uint64_t n, ams_key_type kt, int levels,
                         const uint32_t* buckets_per_level, uint64_t seed, const ams_options* opt,
                         void* stream) {
  return sort_common(make_req(d_keys, d_keys, nullptr, nullptr, n, kt, levels, buckets_per_level,
                              seed, opt),
                     stream);
}

ams_status ams_sort_pairs(void* d_keys, uint64_t* d_vals, uint64_t n, ams_key_type kt, int levels,
                          const uint32_t* buckets_per_level, uint64_t seed, const ams_options* opt,
                          void* stream) {
  if (!d_vals) return AMS_ERR_INVALID;
  return sort_common(make_req(d_keys, d_keys, d_vals, d_vals, n, kt, levels, buckets_per_level,
                              seed, opt),
                     stream);
}

ams_status ams_sort_segmented(void* d_keys, uint64_t* d_vals, const uint64_t* d_offsets,
                              uint64_t nseg, uint64_t n, ams_key_type kt, int levels,
                              const uint32_t* buckets_per_level, uint64_t seed,
                              const ams_options* opt, void* stream) {
  if (!d_offsets && nseg != 1) return AMS_ERR_INVALID;
  ams_request rq = make_req(d_keys, d_keys, d_vals, d_vals, n, kt, levels, buckets_per_level,
                            seed, opt);
  rq.d_offsets = d_offsets;
  rq.nseg = nseg;
  return sort_common(rq, stream);
}

ams_status ams_sort_keys_into(const void* d_in, void* d_out, uint64_t n, ams_key_type kt, int levels,
                              const uint32_t* buckets_per_level, uint64_t seed,
                              const ams_options* opt, void* stream) {
  return sort_common(make_req(d_in, d_out, nullptr, nullptr, n, kt, levels, buckets_per_level, seed,
                              opt),
                     stream);
}

ams_status ams_sort_pairs_into(const void* d_keys_in, void* d_keys_out, const uint64_t* d_vals_in,
                               uint64_t* d_vals_out, uint64_t n, ams_key_type kt, int levels,
                               const uint32_t* buckets_per_level, uint64_t seed,
                               const ams_options* opt, void* stream) {
  if (!d_vals_in || !d_vals_out) return AMS_ERR_INVALID;
  return sort_common(make_req(d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, kt, levels,
                              buckets_per_level, seed, opt),
                     stream);
}

// Host arrays -> the context's staging buffer, sort in place there, staging buffer ->
// host arrays, all enqueued on s (the caller holds cx->mu).  When a step fails after
// the first copy was enqueued, the stream is drained before the error is returned, so
// that no copy still reads or writes the caller's arrays once the call has returned.
static ams_status enqueue_host_sort(Context* cx, void* h_keys, uint64_t* h_vals, uint64_t n,
                                    ams_key_type kt, int levels, const uint32_t* buckets_per_level,
                                    uint64_t seed, const ams_options* opt, cudaStream_t s) {
  const size_t kb = (size_t)n * ksize_of(kt), vb = h_vals ? (size_t)n * 8 : 0;
  ams_status st = grow(cx, &cx->stage, &cx->stage_bytes, kb + vb + 512);
  if (st != AMS_OK) return st;
  void* dk = cx->stage;
  uint64_t* dv = h_vals ? (uint64_t*)(cx->stage + ((kb + 255) & ~(size_t)255)) : nullptr;
  auto fail = [&](ams_status e) {
    cudaStreamSynchronize(s);
    return e;
  };
  cudaError_t ce = cudaMemcpyAsync(dk, h_keys, kb, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess && dv) ce = cudaMemcpyAsync(dv, h_vals, vb, cudaMemcpyHostToDevice, s);
  if (ce != cudaSuccess) return fail(cuda_status(ce));
  ams_request rq = make_req(dk, dk, dv, dv, n, kt, levels, buckets_per_level, seed, opt);
  if ((st = run_sort(cx, &rq, s)) != AMS_OK) return fail(st);
  ce = cudaMemcpyAsync(h_keys, dk, kb, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess && dv) ce = cudaMemcpyAsync(h_vals, dv, vb, cudaMemcpyDeviceToHost, s);
  if (ce != cudaSuccess) return fail(cuda_status(ce));
  return AMS_OK;
}

ams_status ams_sort_host(void* h_keys, uint64_t* h_vals, uint64_t n, ams_key_type kt, int levels,
                         const uint32_t* buckets_per_level, uint64_t seed, const ams_options* opt,
                         void* stream) {
  if (!h_keys && n) return AMS_ERR_INVALID;
  if (n == 0) return AMS_OK;
  Context* cx = default_context();
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  const cudaStream_t s = (cudaStream_t)stream;
  ams_status st = enqueue_host_sort(cx, h_keys, h_vals, n, kt, levels, buckets_per_level, seed, opt, s);
  if (st != AMS_OK) return st;
  AMS_TRY(cudaStreamSynchronize(s));
  return read_status(cx);
}

ams_status ams_sort_host_async(void* ctx, void* h_keys, uint64_t* h_vals, uint64_t n, ams_key_type kt,
                               int levels, const uint32_t* buckets_per_level, uint64_t seed,
                               const ams_options* opt, void* stream) {
  if (!h_keys && n) return AMS_ERR_INVALID;
  if (n == 0) return AMS_OK;
  Context* cx = ctx_or_default(ctx);
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  return enqueue_host_sort(cx, h_keys, h_vals, n, kt, levels, buckets_per_level, seed, opt,
                           (cudaStream_t)stream);
}

ams_status ams_context_create(uint64_t hbm_budget_bytes, void** ctx) {
  if (!ctx) return AMS_ERR_INVALID;
  Context* cx = new (std::nothrow) Context();
  if (!cx) return AMS_ERR_OOM;
  cudaGetDevice(&cx->device);
  cudaDeviceGetAttribute(&cx->sm_count, cudaDevAttrMultiProcessorCount, cx->device);
  cx->budget = hbm_budget_bytes;
  *ctx = cx;
  return AMS_OK;
}

ams_status ams_context_destroy(void* ctx) {
  if (!ctx) return AMS_ERR_INVALID;
  Context* cx = static_cast<Context*>(ctx);
  if (cx->ws || cx->stage || cx->step_ws) cudaDeviceSynchronize();
  if (cx->ws) cudaFree(cx->ws);
  if (cx->stage) cudaFree(cx->stage);
  if (cx->step_ws) cudaFree(cx->step_ws);
  for (cudaEvent_t e : cx->ev_pool) cudaEventDestroy(e);
  if (cx->rlm_done) {
    cudaEventSynchronize(cx->rlm_done);
    cudaEventDestroy(cx->rlm_done);
  }
  if (cx->rlm_host) cudaFreeHost(cx->rlm_host);
  for (auto& g : cx->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    if (g.buf) cudaFree(g.buf);
  }
  if (cx->cap_stream) cudaStreamDestroy(cx->cap_stream);
  delete cx;
  return AMS_OK;
}

ams_status ams_sort_request(void* ctx, const ams_request* req, void* stream) {
  Context* cx = ctx_or_default(ctx);
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  return run_sort(cx, req, (cudaStream_t)stream);
}

ams_status ams_context_sync(void* ctx) {
  Context* cx = ctx_or_default(ctx);
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  if (cx->has_run) AMS_TRY(cudaStreamSynchronize(cx->last_stream));
  return read_status(cx);
}

uint64_t ams_request_scratch_bytes(const ams_request* rq) {
  if (!rq || rq->n == 0 || rq->n >= 0xFFFFFFFFull) return 0;
  const bool pairs = rq->vals_in != nullptr;
  const uint64_t nseg_user = rq->d_offsets ? rq->nseg : 1;
  if (nseg_user == 0) return 0;
  int sm = 148;
  Context* cx = default_context();
  if (cx) sm = cx->sm_count;
  Plan p;
  if (make_plan(rq->n, nseg_user, rq->kt, pairs, rq->levels, rq->buckets_per_level, &rq->opt, sm, &p) != AMS_OK)
    return 0;
  Bufs b{};
  return (uint64_t)carve(p, nullptr, &b);
}

ams_status ams_context_reserve(void* ctx, uint64_t bytes) {
  Context* cx = ctx_or_default(ctx);
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  return ensure_ws(cx, (size_t)bytes);
}

uint64_t ams_context_scratch_bytes(void* ctx) {
  Context* cx = ctx_or_default(ctx);
  return cx ? (uint64_t)(cx->ws_bytes + cx->stage_bytes + cx->step_bytes + cx->graph_bytes) : 0;
}

ams_status ams_get_stats(void* ctx, ams_stats* out) {
  if (!out) return AMS_ERR_INVALID;
  Context* cx = ctx_or_default(ctx);
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  std::memset(out, 0, sizeof(*out));
  if (!cx->has_run) {
    out->kernel_launches = cx->launches;
    cx->launches = 0;
    cx->ev_used = 0;
    cx->ev_kind.clear();
    return AMS_OK;
  }
  AMS_TRY(cudaStreamSynchronize(cx->last_stream));
  const Plan& p = cx->last_plan;
  LevelCounters h[kMaxLevels + 1];
  AMS_TRY(cudaMemcpy(h, cx->last_bufs.ctr, sizeof(h), cudaMemcpyDeviceToHost));
  uint32_t stw = 0;
  AMS_TRY(cudaMemcpy(&stw, cx->d_status, 4, cudaMemcpyDeviceToHost));
  out->levels_planned = (uint32_t)p.L;
  out->kernel_launches = cx->launches;
  out->device_status = stw;
  out->basecase_items[0] = h[0].n_bc;
  uint64_t elems[AMS_K_COUNT] = {};
  elems[AMS_K_BASECASE] += h[0].bc_keys;
  for (int l = 1; l <= p.L; ++l) {
    out->segments[l - 1] = h[l].nseg;
    out->basecase_items[l] = h[l].n_bc;
    elems[AMS_K_CLASSIFY] += h[l].keys;
    elems[AMS_K_SCATTER] += h[l].keys;
    elems[AMS_K_BASECASE] += h[l].bc_keys;
    elems[AMS_K_SAMPLE_SORT] += h[l].samples;
  }
  for (int k = 0; k < AMS_K_COUNT; ++k) out->kernel_elems[k] = elems[k];
  for (size_t i = 0; i < cx->ev_kind.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, cx->ev_pool[2 * i], cx->ev_pool[2 * i + 1]);
    out->kernel_ms[cx->ev_kind[i]] += ms;
    out->kernel_calls[cx->ev_kind[i]] += 1;
  }
  cx->launches = 0;
  cx->ev_used = 0;
  cx->ev_kind.clear();
  return AMS_OK;
}

// ------------------------------------------------------------------------ RLM-sort
// Section 5 on one GPU: tiles of `run` positions play the processing elements.  The
// part boundaries of every level are fixed by n and the part counts (part j of a part
// of m elements starts floor(j m / r) after it), so the host plans them, together
// with the tile lists the base-case kernel sorts: level 0 the tiles of the input,
// level l the tiles of every level-l part after its delivery (the local merge).
static ams_status run_rlm(Context* cx, const void* kin, void* kout, const uint64_t* vin, uint64_t* vout,
                          uint64_t n, ams_key_type kt, uint32_t run, int levels, const uint32_t* parts,
                          uint64_t seed, cudaStream_t s) {
  if (kt != AMS_U32 && kt != AMS_U64 && kt != AMS_F32) return AMS_ERR_INVALID;
  const bool pairs = vin != nullptr || vout != nullptr;
  if (pairs && (!vin || !vout)) return AMS_ERR_INVALID;
  if (n == 0) return AMS_OK;
  if (!kin || !kout || n >= 0xFFFFFFFFull || levels < 0 || levels > kMaxLevels) return AMS_ERR_INVALID;
  if (levels > 0 && !parts) return AMS_ERR_INVALID;
  const int ks = ksize_of(kt);
  if (((uintptr_t)kin % ks) || ((uintptr_t)kout % ks) || ((uintptr_t)vin % 8) || ((uintptr_t)vout % 8))
    return AMS_ERR_INVALID;
  if (run < 2 || run > basecase_max_cap(ks, pairs)) return AMS_ERR_UNSUPPORTED;
  // part boundaries per level (level 0: the whole input)
  std::vector<std::vector<uint32_t>> plo(levels + 1);
  plo[0] = {0u, (uint32_t)n};
  for (int l = 1; l <= levels; ++l) {
    const uint32_t r = parts[l - 1];
    if (r < 2 || r > 65536) return AMS_ERR_INVALID;
    const std::vector<uint32_t>& up = plo[l - 1];
    std::vector<uint32_t>& lo = plo[l];
    if ((up.size() - 1) * (uint64_t)r > (1u << 24)) return AMS_ERR_UNSUPPORTED;
    for (size_t q = 0; q + 1 < up.size(); ++q) {
      const uint64_t m = up[q + 1] - up[q];
      for (uint32_t j = 0; j < r; ++j) lo.push_back(up[q] + (uint32_t)((j * m) / r));
    }
    lo.push_back((uint32_t)n);
  }
  // the last level's parts must fit one tile (they are finished by its local merge)
  for (size_t q = 0; q + 1 < plo[levels].size(); ++q)
    if (plo[levels][q + 1] - plo[levels][q] > run) return AMS_ERR_UNSUPPORTED;
  // tiles of every level's parts, and the largest tile count of a part per level
  std::vector<std::vector<BcItem>> items(levels + 1);
  std::vector<uint32_t> max_tiles(levels + 1, 0);
  for (int l = 0; l <= levels; ++l) {
    for (size_t q = 0; q + 1 < plo[l].size(); ++q) {
      uint32_t t = 0;
      for (uint32_t b = plo[l][q]; b < plo[l][q + 1]; b += run, ++t)
        items[l].push_back(BcItem{b, std::min(plo[l][q + 1], b + run), BC_SORT, 0});
      max_tiles[l] = std::max(max_tiles[l], t);
    }
  }
  for (int l = 0; l < levels; ++l)
    if ((size_t)max_tiles[l] * 6 + 16 > 200u * 1024) return AMS_ERR_UNSUPPORTED;  // select windows
  // workspace: status, temporary keys (and payloads), per level part bounds, item
  // counts and items, cut table (largest level)
  size_t cut_words = 0, off_words = 0;
  for (int l = 1; l <= levels; ++l) {
    cut_words = std::max(cut_words, (plo[l - 1].size() - 1) * (size_t)(parts[l - 1] + 1) * max_tiles[l - 1]);
    off_words = std::max(off_words, (plo[l - 1].size() - 1) * (size_t)parts[l - 1] * max_tiles[l - 1]);
  }
  uint32_t* d_offs = nullptr;
  auto lay = [&](char* base, Bufs& bb, std::vector<uint32_t*>& d_plo, std::vector<uint32_t*>& d_cnt,
                 std::vector<BcItem*>& d_items, uint32_t*& d_cuts) {
    Carver c{base};
    bb.status = c.take<uint32_t>(64);
    bb.tmp = c.take<char>(n * ks);
    bb.vtmp = pairs ? c.take<uint64_t>(n) : nullptr;
    d_plo.assign(levels + 1, nullptr);
    d_cnt.assign(levels + 1, nullptr);
    d_items.assign(levels + 1, nullptr);
    for (int l = 0; l <= levels; ++l) {
      d_plo[l] = c.take<uint32_t>(plo[l].size());
      d_cnt[l] = c.take<uint32_t>(1);
      d_items[l] = c.take<BcItem>(items[l].size());
    }
    d_cuts = c.take<uint32_t>(cut_words + 1);
    d_offs = c.take<uint32_t>(off_words + 1);
    return c.off + 256;
  };
  Bufs bb{};
  std::vector<uint32_t*> d_plo, d_cnt;
  std::vector<BcItem*> d_items;
  uint32_t* d_cuts = nullptr;
  const size_t need = lay(nullptr, bb, d_plo, d_cnt, d_items, d_cuts);
  ams_status st = ensure_ws(cx, need);
  if (st != AMS_OK) return st;
  lay(cx->ws, bb, d_plo, d_cnt, d_items, d_cuts);
  cx->has_run = false;  // (the level statistics describe AMS-sort runs)
  cx->last_stream = s;
  // tables to the device through a pinned staging buffer owned by the context
  size_t hb = 0;
  for (int l = 0; l <= levels; ++l) hb += plo[l].size() * 4 + 4 + items[l].size() * sizeof(BcItem) + 16;
  if (cx->rlm_host_bytes < hb) {
    if (cx->rlm_host) {
      AMS_TRY(cudaStreamSynchronize(cx->rlm_stream ? cx->rlm_stream : s));
      cudaFreeHost(cx->rlm_host);
      cx->rlm_host = nullptr;
      cx->rlm_host_bytes = 0;
    }
    if (cudaMallocHost(&cx->rlm_host, hb) != cudaSuccess) {
      cudaGetLastError();
      return AMS_ERR_OOM;
    }
    cx->rlm_host_bytes = hb;
  } else if (cx->rlm_pending) {
    AMS_TRY(cudaEventSynchronize(cx->rlm_done));  // the previous copy out of the staging buffer
  }
  char* h = (char*)cx->rlm_host;
  for (int l = 0; l <= levels; ++l) {
    std::memcpy(h, plo[l].data(), plo[l].size() * 4);
    AMS_TRY(cudaMemcpyAsync(d_plo[l], h, plo[l].size() * 4, cudaMemcpyHostToDevice, s));
    h += plo[l].size() * 4;
    const uint32_t cnt = (uint32_t)items[l].size();
    std::memcpy(h, &cnt, 4);
    AMS_TRY(cudaMemcpyAsync(d_cnt[l], h, 4, cudaMemcpyHostToDevice, s));
    h += 4;
    std::memcpy(h, items[l].data(), items[l].size() * sizeof(BcItem));
    AMS_TRY(cudaMemcpyAsync(d_items[l], h, items[l].size() * sizeof(BcItem), cudaMemcpyHostToDevice, s));
    h += items[l].size() * sizeof(BcItem) + 16;
  }
  if (!cx->rlm_done) AMS_TRY(cudaEventCreateWithFlags(&cx->rlm_done, cudaEventDisableTiming));
  AMS_TRY(cudaEventRecord(cx->rlm_done, s));
  cx->rlm_pending = true;
  cx->rlm_stream = s;

  const bool f32 = kt == AMS_F32;
  const int SM = cx->sm_count;
  Launcher ln{cx, s};
  // buffers: level l's tiles live in X_l; X_levels is the output
  auto X = [&](int l) -> void* { return ((levels - l) % 2 == 0) ? kout : bb.tmp; };
  auto V = [&](int l) -> uint64_t* { return ((levels - l) % 2 == 0) ? vout : bb.vtmp; };
  auto sort_tiles = [&](int l, const void* src, const uint64_t* vsrc) -> ams_status {
    BaseArgs ba{};
    ba.src = src;
    ba.out = X(l);
    ba.vsrc = vsrc;
    ba.vout = pairs ? V(l) : nullptr;
    ba.items = d_items[l];
    ba.nitems = d_cnt[l];
    ba.tf_load = (l == 0 && f32) ? 1 : 0;
    ba.tf_store = (l == levels && f32) ? 1 : 0;
    ba.status = bb.status;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(items[l].size(), (uint64_t)SM * 8));
    ln.begin(AMS_K_BASECASE);
    return cuda_status(ln.end(launch_basecase(ba, ks, pairs, false, grid, s)));
  };
  if ((st = sort_tiles(0, kin, vin)) != AMS_OK) return st;
  for (int l = 1; l <= levels; ++l) {
    RlmArgs ra{};
    ra.src = X(l - 1);
    ra.dst = X(l);
    ra.vsrc = pairs ? V(l - 1) : nullptr;
    ra.vdst = pairs ? V(l) : nullptr;
    ra.part_lo = d_plo[l - 1];
    ra.nparts = (uint32_t)(plo[l - 1].size() - 1);
    ra.r = parts[l - 1];
    ra.run = run;
    ra.max_tiles = std::max<uint32_t>(1, max_tiles[l - 1]);
    ra.cuts = d_cuts;
    ra.offs = d_offs;
    ra.seed = seed;
    ra.level = l;
    ra.status = bb.status;
    ln.begin(AMS_K_SCATTER);
    AMS_TRY(ln.end(launch_rlm_level(ra, ks, pairs, SM, s)));
    if ((st = sort_tiles(l, X(l), pairs ? V(l) : nullptr)) != AMS_OK) return st;
  }
  return AMS_OK;
}

ams_status ams_rlm_sort(void* ctx, const void* d_keys_in, void* d_keys_out, const uint64_t* d_vals_in,
                        uint64_t* d_vals_out, uint64_t n, ams_key_type kt, uint32_t run, int levels,
                        const uint32_t* parts_per_level, uint64_t seed, void* stream) {
  Context* cx = ctx_or_default(ctx);
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  return run_rlm(cx, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, kt, run, levels, parts_per_level, seed,
                 (cudaStream_t)stream);
}

// ------------------------------------------------------------- level intermediates
static ams_status level_tables(Context* cx, int level, uint32_t* nseg, const Seg** segs,
                               const LevelBufs** lb) {
  if (!cx->has_run) return AMS_ERR_INVALID;
  const Plan& p = cx->last_plan;
  if (level < 1 || level > p.L) return AMS_ERR_INVALID;
  AMS_TRY(cudaStreamSynchronize(cx->last_stream));
  LevelCounters c;
  AMS_TRY(cudaMemcpy(&c, &cx->last_bufs.ctr[level], sizeof(c), cudaMemcpyDeviceToHost));
  *nseg = c.nseg;
  *segs = level == 1 ? cx->last_bufs.segs1 : cx->last_bufs.lv[level - 2].segs_next;
  *lb = &cx->last_bufs.lv[level - 1];
  return AMS_OK;
}

ams_status ams_get_level_segments(void* ctx, int level, uint32_t* nseg, ams_segment_info* h_segs,
                                  uint32_t max_seg) {
  if (!nseg) return AMS_ERR_INVALID;
  Context* cx = ctx_or_default(ctx);
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  const Seg* segs;
  const LevelBufs* lb;
  ams_status st = level_tables(cx, level, nseg, &segs, &lb);
  if (st != AMS_OK || !h_segs) return st;
  const uint32_t m = std::min(*nseg, max_seg);
  if (m == 0) return AMS_OK;
  std::vector<Seg> sg(m);
  std::vector<SegInfo> si(m);
  std::vector<uint32_t> L(m), ng(m), np(m);
  AMS_TRY(cudaMemcpy(sg.data(), segs, m * sizeof(Seg), cudaMemcpyDeviceToHost));
  AMS_TRY(cudaMemcpy(si.data(), lb->sinfo, m * sizeof(SegInfo), cudaMemcpyDeviceToHost));
  AMS_TRY(cudaMemcpy(L.data(), lb->seg_L, m * 4, cudaMemcpyDeviceToHost));
  AMS_TRY(cudaMemcpy(ng.data(), lb->seg_ng, m * 4, cudaMemcpyDeviceToHost));
  AMS_TRY(cudaMemcpy(np.data(), lb->npieces, m * 4, cudaMemcpyDeviceToHost));
  const uint32_t nid = cx->last_plan.lv[level - 1].nid;
  for (uint32_t i = 0; i < m; ++i)
    h_segs[i] = ams_segment_info{sg[i].begin, sg[i].end, si[i].a, si[i].S, L[i], ng[i], np[i], nid};
  return AMS_OK;
}

ams_status ams_get_segment_tables(void* ctx, int level, uint32_t seg, uint32_t* h_bucket_starts,
                                  uint16_t* h_piece_of, uint32_t* h_piece_starts) {
  Context* cx = ctx_or_default(ctx);
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  uint32_t nseg;
  const Seg* segs;
  const LevelBufs* lb;
  ams_status st = level_tables(cx, level, &nseg, &segs, &lb);
  if (st != AMS_OK) return st;
  if (seg >= nseg) return AMS_ERR_INVALID;
  const size_t nid = cx->last_plan.lv[level - 1].nid;
  if (h_bucket_starts)
    AMS_TRY(cudaMemcpy(h_bucket_starts, lb->totals + seg * nid, nid * 4, cudaMemcpyDeviceToHost));
  if (h_piece_of)
    AMS_TRY(cudaMemcpy(h_piece_of, lb->piece_of + seg * nid, nid * 2, cudaMemcpyDeviceToHost));
  if (h_piece_starts) {
    uint32_t np = 0;
    AMS_TRY(cudaMemcpy(&np, lb->npieces + seg, 4, cudaMemcpyDeviceToHost));
    if (np > nid) return AMS_ERR_INTERNAL;
    if (np) AMS_TRY(cudaMemcpy(h_piece_starts, lb->piece_start + seg * nid, np * 4, cudaMemcpyDeviceToHost));
  }
  return AMS_OK;
}

// ------------------------------------------------------------------ step calls
ams_status ams_step_sample(const void* d_keys, uint64_t n, ams_key_type kt, uint32_t count,
                           uint64_t seed, uint32_t level, uint64_t begin, void* d_sample,
                           void* stream) {
  if (!d_keys || !d_sample || n == 0 || n >= 0xFFFFFFFFull || count == 0 || count > (1u << 20))
    return AMS_ERR_INVALID;
  Context* cx = default_context();
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  const cudaStream_t s = (cudaStream_t)stream;
  const int ks = ksize_of(kt);
  StepWs w;
  ams_status st = step_ws(cx, count, 2, 1, ks, &w);
  if (st != AMS_OK) return st;
  LevelArgs la = step_level(cx, w, count, 1, (uint32_t)n);
  la.level = (int)level;
  la.seed = seed;
  la.rng_base = begin;
  la.src = d_keys;
  la.tf_src = kt == AMS_F32;
  la.CH = 0x7FFFFFFFu;
  k_step_prepare<<<1, 32, 0, s>>>(w.segs, w.ctr, 0, (uint32_t)n, w.srank, 0);
  AMS_TRY(cudaGetLastError());
  AMS_TRY(launch_setup(la, s));
  AMS_TRY(launch_sample_sort_ex(la, ks, cx->sm_count * 2, d_sample, nullptr, s));
  return AMS_OK;
}

ams_status ams_step_rank_sort(const void* d_sample, uint32_t count, ams_key_type kt, void* d_sorted,
                              void* stream) {
  if (!d_sample || !d_sorted || count == 0 || count > 65536) return AMS_ERR_INVALID;
  Context* cx = default_context();
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  const cudaStream_t s = (cudaStream_t)stream;
  const int ks = ksize_of(kt);
  StepWs w;
  ams_status st = step_ws(cx, count, count, 1, ks, &w);
  if (st != AMS_OK) return st;
  LevelArgs la = step_level(cx, w, count, 1, 1);
  la.CH = 0x7FFFFFFFu;
  k_step_prepare<<<1, 32, 0, s>>>(w.segs, w.ctr, 0, 1, w.srank, 0);
  AMS_TRY(cudaGetLastError());
  AMS_TRY(launch_setup(la, s));
  AMS_TRY(launch_sample_sort_ex(la, ks, cx->sm_count * 2, nullptr, d_sample, s));
  AMS_TRY(launch_cross_rank(la, ks, cx->sm_count * 4, s));
  AMS_TRY(launch_splitters_ex(la, ks, cx->sm_count * 2, d_sorted, s));
  return AMS_OK;
}

ams_status ams_step_splitters(const void* d_sorted, uint32_t a, uint32_t nbuckets, ams_key_type kt,
                              void* d_splitters, void* stream) {
  if (!d_sorted || !d_splitters || a == 0 || a > 64 || nbuckets < 2 || nbuckets > 65536)
    return AMS_ERR_INVALID;
  Context* cx = default_context();
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  const cudaStream_t s = (cudaStream_t)stream;
  const int ks = ksize_of(kt);
  const uint64_t S = (uint64_t)a * nbuckets;
  StepWs w;
  ams_status st = step_ws(cx, S, 2, 1, ks, &w);
  if (st != AMS_OK) return st;
  LevelArgs la = step_level(cx, w, nbuckets, a, 1);
  la.CH = 0x7FFFFFFFu;
  la.sample = const_cast<void*>(d_sorted);
  la.spl = d_splitters;
  // a fake segment long enough that the sample-size cap keeps a
  const uint64_t fake = std::min<uint64_t>(16ull * a * nbuckets * 16, 0xFFFFFFF0ull);
  k_step_prepare<<<64, 256, 0, s>>>(w.segs, w.ctr, 0, (uint32_t)fake, w.srank, (uint32_t)S);
  AMS_TRY(cudaGetLastError());
  AMS_TRY(launch_setup(la, s));
  AMS_TRY(launch_splitters_ex(la, ks, cx->sm_count * 2, nullptr, s));
  return AMS_OK;
}

ams_status ams_step_classify(const void* d_keys, uint64_t n, ams_key_type kt, const void* d_splitters,
                             uint32_t nbuckets, uint32_t* d_counts, uint16_t* d_ids, void* stream) {
  if (!d_keys || !d_splitters || !d_counts || n == 0 || n >= 0xFFFFFFFFull || nbuckets < 2 ||
      nbuckets > (uint32_t)kMaxBuckets)
    return AMS_ERR_INVALID;
  Context* cx = default_context();
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  const cudaStream_t s = (cudaStream_t)stream;
  const int ks = ksize_of(kt);
  StepWs w;
  const uint64_t items = n / 8192 + 2;
  ams_status st = step_ws(cx, 1, nbuckets, items, ks, &w);
  if (st != AMS_OK) return st;
  LevelArgs la = step_level(cx, w, nbuckets, 1, (uint32_t)n);
  la.src = d_keys;
  la.tf_src = kt == AMS_F32;
  la.spl = const_cast<void*>(d_splitters);
  la.items_cap = (uint32_t)items;
  k_step_prepare<<<1, 32, 0, s>>>(w.segs, w.ctr, 0, (uint32_t)n, w.srank, 0);
  AMS_TRY(cudaGetLastError());
  AMS_TRY(launch_setup(la, s));
  AMS_TRY(launch_table(la, ks, 1, s));
  if (d_ids) la.ids = d_ids;
  AMS_TRY(launch_classify(la, ks, false, cx->sm_count * 4, s));
  AMS_TRY(launch_scan(la, cx->sm_count * 8, true, s));
  AMS_TRY(cudaMemcpyAsync(d_counts, w.totals, (size_t)la.nid * 4, cudaMemcpyDeviceToDevice, s));
  return AMS_OK;
}

ams_status ams_step_bin_pack(const uint32_t* d_counts, uint32_t nbuckets, uint32_t r, uint64_t* d_L,
                             uint32_t* d_group_ends, uint32_t* d_ngroups, void* stream) {
  if (!d_counts || nbuckets < 2 || nbuckets > (uint32_t)kMaxBuckets || r == 0 || r > nbuckets)
    return AMS_ERR_INVALID;
  Context* cx = default_context();
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  const cudaStream_t s = (cudaStream_t)stream;
  StepWs w;
  ams_status st = step_ws(cx, 1, nbuckets, 1, 8, &w);
  if (st != AMS_OK) return st;
  LevelArgs la = step_level(cx, w, nbuckets, 1, 1);
  la.r = r;
  la.group_ends = d_group_ends;
  k_step_prepare<<<1, 32, 0, s>>>(w.segs, w.ctr, 0, 0x7FFFFFFFu, w.srank, 0);
  AMS_TRY(cudaGetLastError());
  AMS_TRY(launch_setup(la, s));
  AMS_TRY(cudaMemcpyAsync(w.totals, d_counts, (size_t)la.nid * 4, cudaMemcpyDeviceToDevice, s));
  AMS_TRY(launch_binpack(la, 1, s));
  k_step_finish_binpack<<<1, 32, 0, s>>>(w.seg_L, w.seg_ng, d_L, d_ngroups);
  AMS_TRY(cudaGetLastError());
  return AMS_OK;
}

static ams_status step_partition(const void* d_in, void* d_out, const uint64_t* d_vals_in,
                                 uint64_t* d_vals_out, uint64_t n, ams_key_type kt,
                                 const void* d_splitters, uint32_t nbuckets, bool stable, void* stream) {
  if (!d_in || !d_out || d_in == d_out || !d_splitters || n == 0 || n >= 0xFFFFFFFFull ||
      nbuckets < 2 || nbuckets > (uint32_t)kMaxBuckets || ((d_vals_in == nullptr) != (d_vals_out == nullptr)))
    return AMS_ERR_INVALID;
  Context* cx = default_context();
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  const cudaStream_t s = (cudaStream_t)stream;
  const int ks = ksize_of(kt);
  StepWs w;
  const uint64_t items = n / 8192 + 2;
  ams_status st = step_ws(cx, 1, nbuckets, items, ks, &w);
  if (st != AMS_OK) return st;
  LevelArgs la = step_level(cx, w, nbuckets, 1, (uint32_t)n);
  la.src = d_in;
  la.dst = d_out;
  la.vsrc = d_vals_in;
  la.vdst = d_vals_out;
  la.tf_src = kt == AMS_F32;
  la.spl = const_cast<void*>(d_splitters);
  la.items_cap = (uint32_t)items;
  k_step_prepare<<<1, 32, 0, s>>>(w.segs, w.ctr, 0, (uint32_t)n, w.srank, 0);
  AMS_TRY(cudaGetLastError());
  AMS_TRY(launch_setup(la, s));
  la.pieces_per_id = 1;  // deliver bucket by bucket
  AMS_TRY(launch_table(la, ks, 1, s));
  AMS_TRY(launch_classify(la, ks, false, cx->sm_count * 4, s));
  AMS_TRY(launch_scan(la, cx->sm_count * 8, true, s));
  AMS_TRY(launch_binpack(la, 1, s));
  const int grid = cx->sm_count * (stable ? 2 : ks == 4 ? 4 : 6);
  AMS_TRY(launch_scatter(la, ks, d_vals_in != nullptr, stable, grid, s));
  return AMS_OK;
}

ams_status ams_step_partition(const void* d_in, void* d_out, const uint64_t* d_vals_in,
                              uint64_t* d_vals_out, uint64_t n, ams_key_type kt,
                              const void* d_splitters, uint32_t nbuckets, void* stream) {
  return step_partition(d_in, d_out, d_vals_in, d_vals_out, n, kt, d_splitters, nbuckets, true, stream);
}

ams_status ams_step_partition_arrival(const void* d_in, void* d_out, uint64_t n, ams_key_type kt,
                                      const void* d_splitters, uint32_t nbuckets, void* stream) {
  return step_partition(d_in, d_out, nullptr, nullptr, n, kt, d_splitters, nbuckets, false, stream);
}

ams_status ams_step_base_case(void* d_keys, uint64_t* d_vals, uint64_t n, ams_key_type kt, void* stream) {
  const int ks = ksize_of(kt);
  if (!d_keys || n == 0 || n > basecase_max_cap(ks, d_vals != nullptr)) return AMS_ERR_INVALID;
  Context* cx = default_context();
  if (!cx) return AMS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(cx->mu);
  const cudaStream_t s = (cudaStream_t)stream;
  StepWs w;
  ams_status st = step_ws(cx, 1, 2, 1, ks, &w);
  if (st != AMS_OK) return st;
  k_step_item<<<1, 32, 0, s>>>(w.bc, &w.ctr[1], 0, (uint32_t)n);
  AMS_TRY(cudaGetLastError());
  BaseArgs ba{};
  ba.src = d_keys;
  ba.out = d_keys;
  ba.scratch = nullptr;
  ba.vsrc = d_vals;
  ba.vout = d_vals;
  ba.items = w.bc;
  ba.nitems = &w.ctr[1].n_bc;
  ba.tf_load = kt == AMS_F32;
  ba.tf_store = kt == AMS_F32;
  ba.status = cx->d_status;
  AMS_TRY(launch_basecase(ba, ks, d_vals != nullptr, false, 1, s));
  return AMS_OK;
}

const char* ams_status_string(ams_status s) {
  switch (s) {
    case AMS_OK: return "ok";
    case AMS_ERR_INVALID: return "invalid argument";
    case AMS_ERR_OOM: return "out of device memory";
    case AMS_ERR_CUDA: return "CUDA runtime error";
    case AMS_ERR_TIMEOUT: return "device wait timed out";
    case AMS_ERR_UNSUPPORTED: return "unsupported request";
    case AMS_ERR_INTERNAL: return "device table overflow";
  }
  return "unknown status";
}

uint32_t ams_default_basecase_cap(ams_key_type kt, int pairs) { return default_cap(kt, pairs != 0); }

const char* ams_version(void) { return "0.1.0"; }

}  // extern "C"
