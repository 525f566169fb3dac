// Plan, executor and C ABI of the MrDFT library (host code).
//
// A plan owns the twiddle tables (FP64 host values rounded once to FP32), the
// per-signal descriptors, the work lists of every kernel launch and the
// scratch buffers; mrdft_forward / mrdft_adjoint enqueue the fixed launch
// sequence (tile kernel, then the levels above the tile one by one), or
// replay it as a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mrdft.h"
#include "mrdft_internal.h"

namespace mrdft {
cudaError_t set_fwd_attributes();
cudaError_t set_adj_attributes();
void set_global_error(const std::string& msg);
mrdft_status noalloc_status_poll();
}  // namespace mrdft

using namespace mrdft;

namespace {

constexpr int kMaxLog = 26;

// One kernel launch (or, for two-pass levels, the cols + rows pair) over a
// contiguous range of a device work list.
enum LaunchKind { LK_TILE = 0, LK_WIN = 1, LK_PASS = 2 };
struct Launch {
  int kind;
  int level;      // level built (window / two-pass)
  int64_t off;    // first item in d_tiles or d_levels
  int count;      // items (per pass for two-pass levels)
  int64_t bytes;  // algorithmic bytes: input read once + outputs written
  // two-pass levels i, i + 1 of one chain may share one cols pass (one read of
  // x for both): dual = 1 on level i, whose cols pass is then k_fwd_cols2 over
  // the items [c2_off, c2_off + c2_count) of level i + 1, plus the plain cols
  // pass over [tail_off, tail_off + tail_count), the windows of signals (or
  // units) that end at level i; dual = 2 on level i + 1 (cols pass done)
  int dual;
  int64_t c2_off;
  int c2_count;
  int64_t tail_off;  // level-i items of units with U == i (built for every two-pass level)
  int tail_count;
};

// A segment: a group of signals or a window of one signal, at most 2^seg_log
// samples, whose levels up to seg_log run as one chain of launches on one
// stream -- small enough that x, the children spectra and the two-pass
// intermediate stay in L2 between the launches of the chain.
struct Segment {
  std::vector<Launch> chain;  // tile launch first, then levels ascending
  int parent = -1;            // forward tree: the top node over this segment, if any
};

// Forward tree of the levels above the segment size: one node per window of
// such a level (its cols and rows launches over that window's items), run as
// soon as its two children -- segments for the lowest top level, nodes above
// -- have run, on the stream of the child enqueued last, so that it overlaps
// the other chains and finds its children's spectra still in L2.
struct TopNode {
  Launch L;
  int child[2];   // >= 0: segment index; < 0: node -(c + 1)
  int parent = -1;
};

struct GraphKey {
  const void* a;
  const void* b;
  cudaStream_t s;
  const void* t;  // fused loss gradient: targets and loss accumulator
  const void* l;
  bool operator==(const GraphKey& o) const { return a == o.a && b == o.b && s == o.s && t == o.t && l == o.l; }
};

// Instantiated graphs of one direction, least recently used first out: at
// most kGraphCacheMax per direction; a new (buffers, stream) key past that
// limit re-targets the oldest executable graph with cudaGraphExecUpdate (the
// launch sequence is the same, only the pointers differ) instead of
// instantiating another one.
constexpr size_t kGraphCacheMax = 4;
struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
  uint64_t last_use;
};

std::mutex g_err_mu;
std::string g_global_err = "no error";

}  // namespace

void mrdft::set_global_error(const std::string& msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_global_err = msg;
}

struct mrdft_plan_s {
  int device = 0;
  int dtype = MRDFT_C64;
  uint32_t flags = 0;
  int num_sms = 0;
  int64_t nsig = 0;
  int max_m = 0;
  int64_t in_elems = 0, out_elems = 0, half_elems = 0;
  std::vector<SigDesc> sigs;

  // device resources
  SigDesc* d_sigs = nullptr;
  int32_t* d_tile_ids = nullptr;
  int n_tile_ids = 0;
  TileItem* d_tiles = nullptr;
  int n_tiles = 0;
  int32_t* d_tiny_ids = nullptr;
  int n_tiny = 0;
  LevelItem* d_levels = nullptr;
  int64_t n_level_items = 0;
  // MRDFT_FLAG_BITREV: items of the in-place permutation after the forward
  LevelItem* d_br = nullptr;
  int br_small = 0;                                   // {sig, block, level}, levels 2..12
  std::vector<std::pair<int, std::pair<int64_t, int>>> br_big;  // level, (first item, count), levels > 12
  std::vector<Segment> segments;
  std::vector<Launch> top;  // levels above seg_log, ascending, whole plan (adjoint; forward without the tree)
  std::vector<TopNode> top_nodes;   // forward tree (children before parents)
  bool fwd_tree = false;            // off: the forward runs `top` after every segment instead
  bool tile_first = true;           // one tile launch over every segment (before them forward, after them adjoint)
  bool tile_lean = true;            // forward tile CTAs in the 3-per-SM shape
  bool fwd_rows12 = false;          // forward C = 2^9 rows CTAs of 2^12 points
  // top_cols_early: the cols passes of the unpaired levels above the segment
  // size run on their own stream during the segment chains (they read only
  // x), each into its own scratch; their rows passes stay at the end
  bool top_cols_early = false;
  // top_overlap: those cols passes on their own stream as well (from the end
  // of the segments unless top_cols_early), each level's rows pass waiting
  // only for its own cols pass (one event per level)
  bool top_overlap = false;
  // levels_parallel: a plan of one signal of 2^5..2^12 samples runs its
  // in-tile launch as one CTA per level (k_fwd_levels); lone_m = that m, else 0
  bool levels_parallel = true;
  int lone_m = 0;
  float2* d_lone = nullptr;  // adjoint: each level's share of x_bar (lone_m x N)
  int* d_ticket = nullptr;   // adjoint: finish counter of its CTAs
  float2* d_scratch_top = nullptr;  // half_elems per early level
  std::vector<int> top_early;       // index into `top` of each early level (its scratch slot follows)
  cudaStream_t early = nullptr;
  cudaEvent_t ev_early_go = nullptr, ev_early_done = nullptr;
  std::vector<cudaEvent_t> ev_top_cols;  // top_overlap: after the cols pass of early level j
  Launch tile_all{};                // that launch (tile_first), or with tile_split > 1 ...
  int tile_split = 1;               // ... that many launches over consecutive groups of segments
  std::vector<Launch> tile_parts;   // the group launches (tile_first), in segment order
  std::vector<int> seg_part;        // group of each segment
  std::vector<cudaEvent_t> ev_tile, ev_segdone;
  std::vector<cudaEvent_t> ev_seg, ev_node;
  int seg_log = 23;
  int nstreams = 4;
  bool seg_fixed = false;      // set by mrdft_plan_opts (else the environment may override)
  bool streams_fixed = false;
  // kernel variants (mrdft_exec_opts; none changes the result)
  bool dual_cols = true;       // pair two-pass levels in one cols pass
  int adj_rows13 = 1;          // adjoint C = 2^10 rows CTAs of 2^13 points (else 2^12)
  int adj_cb_min = 10;         // adjoint two-pass levels: C = 2^max(i - 12, adj_cb_min)
  int fwd_rows14 = 1;          // forward C = 2^12 rows CTAs of 2^14 points (else 2^13; last-pass children reads only)
  int fwd_cb_min = 9;          // forward two-pass levels: C = 2^max(i - 12, fwd_cb_min)
  int fwd_rows_pf = 0;         // forward rows CTAs prefetch the children into shared memory
  std::vector<cudaStream_t> workers;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  float2* d_tw13 = nullptr;
  float2* d_twlo = nullptr;
  float2* d_twhi = nullptr;
  float2* d_scratch = nullptr;  // 2 x N/2 per signal: two-pass intermediates, level parity picks the half
  float2* d_e0 = nullptr;       // N/2 per signal
  float2* d_e1 = nullptr;       // N/2 per signal
  // the lowest top level's even-bin propagation (N/2 per signal), read by
  // the level-seg_log launches of every segment: the two segments of one
  // parent window run on different worker streams, and each writes its own
  // lower levels' propagation into d_e0 / d_e1 over the parent's range
  float2* d_etop = nullptr;
  float2* d_acc = nullptr;      // N per signal of m > 12, at 2 aux_off
  int* d_status = nullptr;
  void* d_stage_x = nullptr;
  void* d_stage_y = nullptr;
  // mrdft_forward_host: output runs copied to the host as soon as the part
  // of the forward that writes them is done -- phase 0 after the in-tile
  // levels (one tile launch), 1 after the segments, 2 at the end -- on a
  // stream of their own, forked from and joined back to the caller's
  struct HostRun {
    int64_t off, count;  // y elements
  };
  std::vector<HostRun> host_runs[3];
  bool host_runs_ready = false;
  cudaStream_t d2h = nullptr;
  cudaEvent_t ev_host[4] = {};  // phases 0..2, join
  void* host_dst = nullptr;     // set only while mrdft_forward_host enqueues


  std::vector<GraphEntry> fwd_graphs, adj_graphs;
  uint64_t graph_clock = 0;
  int64_t graph_captures = 0;   // stream captures made
  int64_t graph_updates = 0;    // of which re-targeted an existing executable graph
  // adjoint launches of mrdft_loss_grad: targets and loss accumulator (else null)
  const float2* cur_t = nullptr;
  double* cur_loss = nullptr;
  std::string err = "no error";

  // optional per-kernel timing (events around every launch, no graph replay);
  // timing_serial also runs the segments one after another on the caller's
  // stream, so that every bracketed launch has the GPU to itself
  bool timing = false;
  bool timing_serial = false;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
    int64_t bytes;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  double t_ms[MRDFT_KIND_COUNT] = {0};
  int64_t t_launches[MRDFT_KIND_COUNT] = {0};
  int64_t t_bytes[MRDFT_KIND_COUNT] = {0};
};

namespace {

mrdft_status fail(mrdft_plan_s* p, mrdft_status st, const std::string& msg) {
  if (p) {
    p->err = msg;
  } else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_global_err = msg;
  }
  return st;
}

mrdft_status cuda_fail(mrdft_plan_s* p, cudaError_t e, const char* what) {
  return fail(p, MRDFT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MRDFT_CUDA(p, call)                                  \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail((p), e_, #call); \
  } while (0)

template <class T>
cudaError_t dev_upload(T** dst, const std::vector<T>& v) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// w_L^e = exp(-j 2 pi e / L) in FP64, rounded once to FP32
float2 root32(int64_t e, int64_t L) {
  const double a = -2.0 * M_PI * (double)(e % L) / (double)L;
  return make_float2((float)std::cos(a), (float)std::sin(a));
}

cudaEvent_t pool_event(mrdft_plan_s* p) {
  if (!p->event_pool.empty()) {
    cudaEvent_t e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch `fn` bracketed by timing events when the plan's timing is on.
template <class F>
cudaError_t timed(mrdft_plan_s* p, int kind, int64_t bytes, cudaStream_t st, F&& fn) {
  if (!p->timing) return fn();
  mrdft_plan_s::Pending pd{kind, pool_event(p), pool_event(p), bytes};
  cudaEventRecord(pd.a, st);
  cudaError_t e = fn();
  cudaEventRecord(pd.b, st);
  p->pending.push_back(pd);
  return e;
}

void collect_timing(mrdft_plan_s* p) {
  for (auto& pd : p->pending) {
    cudaEventSynchronize(pd.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, pd.a, pd.b);
    p->t_ms[pd.kind] += ms;
    p->t_launches[pd.kind] += 1;
    p->t_bytes[pd.kind] += pd.bytes;
    p->event_pool.push_back(pd.a);
    p->event_pool.push_back(pd.b);
  }
  p->pending.clear();
}

void release(mrdft_plan_s* p) {
  collect_timing(p);
  for (cudaStream_t w : p->workers) cudaStreamDestroy(w);
  p->workers.clear();
  for (cudaEvent_t e : p->ev_join) cudaEventDestroy(e);
  p->ev_join.clear();
  for (cudaEvent_t e : p->ev_seg)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_tile)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_segdone)
    if (e) cudaEventDestroy(e);
  p->ev_tile.clear();
  p->ev_segdone.clear();
  for (cudaEvent_t e : p->ev_node)
    if (e) cudaEventDestroy(e);
  p->ev_seg.clear();
  p->ev_node.clear();
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  p->ev_fork = nullptr;
  if (p->early) cudaStreamDestroy(p->early);
  if (p->ev_early_go) cudaEventDestroy(p->ev_early_go);
  if (p->ev_early_done) cudaEventDestroy(p->ev_early_done);
  for (cudaEvent_t e : p->ev_top_cols)
    if (e) cudaEventDestroy(e);
  p->ev_top_cols.clear();
  p->early = nullptr;
  p->ev_early_go = p->ev_early_done = nullptr;
  for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
  p->event_pool.clear();
  if (p->d2h) cudaStreamDestroy(p->d2h);
  p->d2h = nullptr;
  for (cudaEvent_t& e : p->ev_host) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  for (auto& g : p->fwd_graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : p->adj_graphs) cudaGraphExecDestroy(g.exec);
  p->fwd_graphs.clear();
  p->adj_graphs.clear();
  void* ptrs[] = {p->d_sigs, p->d_tile_ids, p->d_tiles, p->d_tiny_ids, p->d_levels, p->d_br,
                  p->d_tw13, p->d_twlo, p->d_twhi, p->d_scratch, p->d_e0,
                  p->d_e1, p->d_etop, p->d_acc, p->d_status, p->d_stage_x, p->d_stage_y, p->d_scratch_top,
                  p->d_lone, p->d_ticket};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

mrdft_status build_plan(mrdft_plan_s* p, const int64_t* lengths, int64_t n_lengths, int64_t batch) {
  MRDFT_CUDA(p, cudaGetDevice(&p->device));
  MRDFT_CUDA(p, cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
  {
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (p->device < 64 && !done[p->device]) {
      MRDFT_CUDA(p, set_fwd_attributes());
      MRDFT_CUDA(p, set_adj_attributes());
      done[p->device] = true;
    }
  }

  // ---- signals
  p->nsig = batch;
  p->sigs.resize(batch);
  int64_t in_off = 0, out_off = 0, aux_off = 0;
  for (int64_t s = 0; s < batch; ++s) {
    const int64_t N = lengths[n_lengths == 1 ? 0 : s];
    int m = 0;
    while ((int64_t(1) << m) < N) ++m;
    SigDesc d{};
    d.in_off = in_off;
    d.out_off = out_off;
    d.m = m;
    // per-signal scratch (N/2) only for signals with levels above the tile;
    // every such block is a multiple of 2^12 elements, so vector accesses stay aligned
    d.aux_off = m > kTileLog ? aux_off : 0;
    if (m > kTileLog) aux_off += N / 2;
    p->sigs[s] = d;
    in_off += N;
    out_off += (int64_t)m * N;
    p->max_m = std::max(p->max_m, m);
  }
  p->in_elems = in_off;
  p->out_elems = out_off;
  p->half_elems = aux_off;

  // ---- segments: units of <= 2^S samples (whole signals, or windows of 2^S
  // of longer signals), signals ordered by length (longest first)
  if (!p->seg_fixed) {
    const char* env = getenv("MRDFT_SEG_LOG");
    if (env) p->seg_log = std::max(kTileLog, std::min(kMaxLog, atoi(env)));
  }
  if (!p->streams_fixed) {
    const char* env = getenv("MRDFT_STREAMS");
    if (env) p->nstreams = std::max(1, std::min(16, atoi(env)));
  }
  const int S = p->seg_log;
  const int64_t in_b = p->dtype == MRDFT_R32 ? 4 : 8;
  std::vector<int32_t> order(batch);
  for (int64_t s = 0; s < batch; ++s) order[s] = (int32_t)s;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return p->sigs[a].m > p->sigs[b].m; });
  struct Unit {
    int32_t sig;
    int32_t w;  // window index at level U
    int U;      // min(m, S)
  };
  std::vector<std::vector<Unit>> seg_units;
  std::vector<int32_t> tiny_ids;
  {
    std::vector<Unit> cur;
    int64_t cur_n = 0;
    for (int32_t s : order) {
      const int m = p->sigs[s].m;
      if (m <= 4) {
        tiny_ids.push_back(s);
        continue;
      }
      const int U = std::min(m, S);
      const int64_t nu = int64_t(1) << (m - U);
      for (int64_t w = 0; w < nu; ++w) {
        if (cur_n + (int64_t(1) << U) > (int64_t(1) << S) && !cur.empty()) {
          seg_units.push_back(cur);
          cur.clear();
          cur_n = 0;
        }
        cur.push_back(Unit{s, (int32_t)w, U});
        cur_n += int64_t(1) << U;
      }
    }
    if (!cur.empty()) seg_units.push_back(cur);
  }
  std::vector<int32_t> tile_ids;
  std::vector<TileItem> tiles;
  std::vector<Launch> seg_tiles;  // tile_first: each segment's tile items
  std::vector<LevelItem> litems;
  auto pass_blocks = [](int i) { return pass_items(i); };
  // consecutive two-pass levels (i, i + 1) of a chain, lowest first: the
  // upper level's windows, split in halves, are exactly the lower level's
  // windows of the units that go on to level i + 1 (same item count)
  auto pair_levels = [&](std::vector<Launch>& chain) {
    if (!p->dual_cols) return;
    for (size_t j = 0; j + 1 < chain.size(); ++j) {
      Launch& L = chain[j];
      Launch& M = chain[j + 1];
      if (L.kind != LK_PASS || M.kind != LK_PASS || L.dual || M.level != L.level + 1) continue;
      if (!fwd_cols2_pairable(M.level, p->fwd_cb_min) || M.count != L.count - L.tail_count) continue;
      L.dual = 1;
      L.c2_off = M.off;
      L.c2_count = M.count;
      M.dual = 2;
      ++j;
    }
  };
  auto add_level_items = [&](int i, int32_t sig, int64_t w0, int64_t nw, Launch& L) {
    const int nblk = i <= kWinMaxLog + 1 ? 1 : pass_blocks(i);
    for (int64_t w = w0; w < w0 + nw; ++w)
      for (int b = 0; b < nblk; ++b) litems.push_back(LevelItem{sig, (int32_t)w, b, 0});
    L.bytes += 8 * nw * (int64_t(1) << i);
  };
  for (const auto& units : seg_units) {
    Segment seg;
    // tile launch
    Launch T{};
    T.kind = LK_TILE;
    T.off = (int64_t)tiles.size();
    size_t q = 0;
    while (q < units.size()) {
      const Unit& u = units[q];
      const int m = p->sigs[u.sig].m;
      if (m >= kTileLog) {
        const int32_t list = (int32_t)tile_ids.size();
        tile_ids.push_back(u.sig);
        const int64_t per = int64_t(1) << (u.U - kTileLog);
        for (int64_t t = u.w * per; t < (u.w + 1) * per; ++t)
          tiles.push_back(TileItem{list, 1, (int16_t)kTileLog, (int32_t)t, 0});
        T.bytes += (int64_t(1) << u.U) * (in_b + 8 * kTileLog);
        ++q;
        continue;
      }
      // pack whole signals of equal length into one tile; the pack size is a
      // power of two (the in-tile FFT works on 2^k windows)
      const int per = 1 << (kTileLog - m);
      size_t avail = 0;
      while (q + avail < units.size() && p->sigs[units[q + avail].sig].m == m && (int)avail < per) ++avail;
      int n = 1;
      while ((size_t)(n * 2) <= avail) n *= 2;
      const int32_t list = (int32_t)tile_ids.size();
      for (int k = 0; k < n; ++k) tile_ids.push_back(units[q + k].sig);
      q += n;
      tiles.push_back(TileItem{list, (int16_t)n, (int16_t)m, 0, 0});
      T.bytes += ((int64_t)n << m) * (in_b + 8 * m);
    }
    T.count = (int)((int64_t)tiles.size() - T.off);
    if (p->tile_first) seg_tiles.push_back(T);
    if (T.count) {
      // segments append their tile items one after another: with tile_first
      // the union [0, tiles) is one launch (or one per group of segments)
      if (p->tile_first) p->tile_all.bytes += T.bytes;
      else seg.chain.push_back(T);
    }
    // levels above the tile, inside the segment
    for (int i = kTileLog + 1; i <= S; ++i) {
      Launch L{};
      L.kind = i <= kWinMaxLog + 1 ? LK_WIN : LK_PASS;
      L.level = i;
      L.off = (int64_t)litems.size();
      for (const Unit& u : units)
        if (u.U >= i) add_level_items(i, u.sig, (int64_t)u.w << (u.U - i), int64_t(1) << (u.U - i), L);
      L.count = (int)((int64_t)litems.size() - L.off);
      if (L.count && L.kind == LK_PASS) {
        Launch tail{};
        L.tail_off = (int64_t)litems.size();
        for (const Unit& u : units)
          if (u.U == i) add_level_items(i, u.sig, (int64_t)u.w, 1, tail);
        L.tail_count = (int)((int64_t)litems.size() - L.tail_off);
      }
      if (L.count) seg.chain.push_back(L);
    }
    pair_levels(seg.chain);
    p->segments.push_back(seg);
  }
  // levels above the segments, over whole signals
  for (int i = S + 1; i <= p->max_m; ++i) {
    Launch L{};
    L.kind = i <= kWinMaxLog + 1 ? LK_WIN : LK_PASS;
    L.level = i;
    L.off = (int64_t)litems.size();
    for (int32_t s : order)
      if (p->sigs[s].m >= i) add_level_items(i, s, 0, int64_t(1) << (p->sigs[s].m - i), L);
    L.count = (int)((int64_t)litems.size() - L.off);
    if (L.count && L.kind == LK_PASS) {
      Launch tail{};
      L.tail_off = (int64_t)litems.size();
      for (int32_t s : order)
        if (p->sigs[s].m == i) add_level_items(i, s, 0, 1, tail);
      L.tail_count = (int)((int64_t)litems.size() - L.tail_off);
    }
    if (L.count) p->top.push_back(L);
  }
  pair_levels(p->top);
  if ((p->top_cols_early || p->top_overlap) && !p->fwd_tree)
    for (size_t k = 0; k < p->top.size(); ++k)
      if (p->top[k].kind == LK_PASS && p->top[k].dual == 0) p->top_early.push_back((int)k);
  if (p->tile_first) {
    p->tile_all.kind = LK_TILE;
    p->tile_all.off = 0;
    p->tile_all.count = (int)tiles.size();
    // groups of consecutive segments, one tile launch each
    const int ns = (int)p->segments.size();
    const int parts = std::max(1, std::min(p->tile_split, ns));
    p->seg_part.assign(ns, 0);
    for (int g = 0; g < parts; ++g) {
      const int j0 = (int)((int64_t)ns * g / parts), j1 = (int)((int64_t)ns * (g + 1) / parts);
      Launch P{};
      P.kind = LK_TILE;
      P.off = j0 < ns ? seg_tiles[j0].off : (int64_t)tiles.size();
      for (int j = j0; j < j1; ++j) {
        P.count += seg_tiles[j].count;
        P.bytes += seg_tiles[j].bytes;
        p->seg_part[j] = g;
      }
      p->tile_parts.push_back(P);
    }
  }
  if (p->fwd_tree && !p->top.empty()) {
    // segment of each (signal, level-S window) of the signals longer than a segment
    std::map<std::pair<int32_t, int32_t>, int> seg_of;
    for (size_t j = 0; j < seg_units.size(); ++j)
      for (const Unit& u : seg_units[j])
        if (p->sigs[u.sig].m > S) seg_of[{u.sig, u.w}] = (int)j;
    for (int32_t sg : order) {
      const int m = p->sigs[sg].m;
      if (m <= S) continue;
      std::vector<int> below;  // nodes (or segments) of the level just below, by window
      for (int32_t w = 0; w < (int32_t)(int64_t(1) << (m - S)); ++w) below.push_back(seg_of.at({sg, w}));
      for (int i = S + 1; i <= m; ++i) {
        std::vector<int> here;
        for (int64_t W = 0; W < (int64_t(1) << (m - i)); ++W) {
          TopNode nd{};
          nd.L.kind = i <= kWinMaxLog + 1 ? LK_WIN : LK_PASS;
          nd.L.level = i;
          nd.L.off = (int64_t)litems.size();
          add_level_items(i, sg, W, 1, nd.L);
          nd.L.count = (int)((int64_t)litems.size() - nd.L.off);
          const int k = (int)p->top_nodes.size();
          for (int c = 0; c < 2; ++c) {
            nd.child[c] = i == S + 1 ? below[2 * W + c] : -(below[2 * W + c] + 1);
            if (i == S + 1) p->segments[below[2 * W + c]].parent = k;
            else p->top_nodes[below[2 * W + c]].parent = k;
          }
          p->top_nodes.push_back(nd);
          here.push_back(k);
        }
        below.swap(here);
      }
    }
  }
  p->n_tiles = (int)tiles.size();
  p->n_tile_ids = (int)tile_ids.size();
  p->lone_m = 0;
  if (p->levels_parallel && p->nsig == 1 && p->sigs[0].m >= 5 && p->sigs[0].m <= kTileLog && p->n_tiles == 1 &&
      !tile_ids.empty() && tile_ids[0] == 0)
    p->lone_m = p->sigs[0].m;
  p->n_level_items = (int64_t)litems.size();
  std::vector<LevelItem> br;
  if (p->flags & MRDFT_FLAG_BITREV) {
    for (int64_t sg = 0; sg < batch; ++sg) {
      const int m = p->sigs[sg].m, B = std::min(m, kTileLog);
      for (int i = 2; i <= B; ++i)
        for (int64_t b = 0; b < (int64_t(1) << (m - B)); ++b) br.push_back(LevelItem{(int32_t)sg, (int32_t)b, i, 0});
    }
    p->br_small = (int)br.size();
    for (int i = kTileLog + 1; i <= p->max_m; ++i) {
      const int64_t first = (int64_t)br.size();
      for (int64_t sg = 0; sg < batch; ++sg)
        if (p->sigs[sg].m >= i)
          for (int64_t w = 0; w < (int64_t(1) << (p->sigs[sg].m - i)); ++w)
            br.push_back(LevelItem{(int32_t)sg, (int32_t)w, i, 0});
      p->br_big.push_back({i, {first, (int)((int64_t)br.size() - first)}});
    }
  }
  p->n_tiny = (int)tiny_ids.size();

  // streams and events for the concurrent segment chains
  const int nw = std::min<int>(p->nstreams, (int)p->segments.size());
  for (int k = 0; k < std::max(0, nw); ++k) {
    cudaStream_t w = nullptr;
    cudaEvent_t e = nullptr;
    MRDFT_CUDA(p, cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking));
    p->workers.push_back(w);
    MRDFT_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    p->ev_join.push_back(e);
  }
  MRDFT_CUDA(p, cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  if (!p->top_early.empty()) {
    MRDFT_CUDA(p, cudaStreamCreateWithFlags(&p->early, cudaStreamNonBlocking));
    MRDFT_CUDA(p, cudaEventCreateWithFlags(&p->ev_early_go, cudaEventDisableTiming));
    MRDFT_CUDA(p, cudaEventCreateWithFlags(&p->ev_early_done, cudaEventDisableTiming));
    if (p->top_overlap) {
      p->ev_top_cols.assign(p->top_early.size(), nullptr);
      for (auto& e : p->ev_top_cols) MRDFT_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
  }
  if (p->tile_parts.size() > 1) {
    p->ev_tile.assign(p->tile_parts.size(), nullptr);
    p->ev_segdone.assign(p->segments.size(), nullptr);
    for (auto& e : p->ev_tile) MRDFT_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto& e : p->ev_segdone) MRDFT_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (!p->top_nodes.empty()) {
    p->ev_seg.assign(p->segments.size(), nullptr);
    p->ev_node.assign(p->top_nodes.size(), nullptr);
    for (size_t j = 0; j < p->segments.size(); ++j)
      if (p->segments[j].parent >= 0) MRDFT_CUDA(p, cudaEventCreateWithFlags(&p->ev_seg[j], cudaEventDisableTiming));
    for (size_t k = 0; k < p->top_nodes.size(); ++k)
      MRDFT_CUDA(p, cudaEventCreateWithFlags(&p->ev_node[k], cudaEventDisableTiming));
  }

  // ---- twiddles: FP64 on the host, rounded once
  std::vector<float2> tw13(1 << kTwLog), twlo(1 << kTwSplit), twhi(1 << (kTwBigLog - kTwSplit));
  for (int64_t e = 0; e < (1 << kTwLog); ++e) tw13[e] = root32(e, int64_t(1) << kTwLog);
  for (int64_t e = 0; e < (1 << kTwSplit); ++e) twlo[e] = root32(e, int64_t(1) << kTwBigLog);
  for (int64_t e = 0; e < (1 << (kTwBigLog - kTwSplit)); ++e)
    twhi[e] = root32(e << kTwSplit, int64_t(1) << kTwBigLog);

  std::vector<SigDesc> sigs = p->sigs;
  MRDFT_CUDA(p, dev_upload(&p->d_sigs, sigs));
  MRDFT_CUDA(p, dev_upload(&p->d_tile_ids, tile_ids));
  MRDFT_CUDA(p, dev_upload(&p->d_tiles, tiles));
  MRDFT_CUDA(p, dev_upload(&p->d_tiny_ids, tiny_ids));
  MRDFT_CUDA(p, dev_upload(&p->d_levels, litems));
  MRDFT_CUDA(p, dev_upload(&p->d_br, br));
  MRDFT_CUDA(p, dev_upload(&p->d_tw13, tw13));
  MRDFT_CUDA(p, dev_upload(&p->d_twlo, twlo));
  MRDFT_CUDA(p, dev_upload(&p->d_twhi, twhi));
  if (p->max_m > kTileLog) {
    const size_t half = (size_t)p->half_elems * sizeof(float2);
    cudaError_t e = cudaMalloc(&p->d_scratch, 2 * half);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_e0, half);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_e1, half);
    if (e == cudaSuccess && !p->top.empty()) e = cudaMalloc(&p->d_etop, half);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_acc, 2 * half);
    if (e == cudaSuccess && !p->top_early.empty()) e = cudaMalloc(&p->d_scratch_top, p->top_early.size() * half);
    if (e != cudaSuccess) return fail(p, MRDFT_ENOMEM, std::string("scratch allocation: ") + cudaGetErrorString(e));
  }
  if (p->lone_m) {
    cudaError_t e = cudaMalloc(&p->d_lone, (size_t)p->lone_m * ((size_t)1 << p->lone_m) * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_ticket, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_ticket, 0, sizeof(int));
    if (e != cudaSuccess) return fail(p, MRDFT_ENOMEM, std::string("lone-signal scratch: ") + cudaGetErrorString(e));
  }
  MRDFT_CUDA(p, cudaMalloc(&p->d_status, sizeof(int)));
  MRDFT_CUDA(p, cudaMemset(p->d_status, 0, sizeof(int)));

  return MRDFT_OK;
}

Twiddles twiddles(const mrdft_plan_s* p) { return Twiddles{p->d_tw13, p->d_twlo, p->d_twhi}; }

// passes: 1 the cols pass only, 2 the rows pass only, 3 both (two-pass
// levels); scr: the intermediate (nullptr: half (level & 1) of the scratch)
mrdft_status launch_fwd(mrdft_plan_s* p, FwdArgs a, const Launch& L, cudaStream_t st, int passes = 3,
                        float2* scr = nullptr) {
  a.level = L.level;
  a.nitems = L.count;
  if (L.kind == LK_TILE) {
    a.sig_ids = p->d_tile_ids;
    a.nids = p->n_tile_ids;
    a.items = p->d_tiles + L.off;
    if (p->lone_m)
      MRDFT_CUDA(p, timed(p, MRDFT_KIND_FWD_TILE, L.bytes, st, [&] { return launch_fwd_levels(a, p->lone_m, st); }));
    else
      MRDFT_CUDA(p, timed(p, MRDFT_KIND_FWD_TILE, L.bytes, st, [&] { return launch_fwd_tile(a, L.count, st); }));
  } else if (L.kind == LK_WIN) {
    a.items = p->d_levels + L.off;
    MRDFT_CUDA(p, timed(p, MRDFT_KIND_FWD_WINDOW, L.bytes, st, [&] { return launch_fwd_window(a, L.count, st); }));
  } else {
    // the two-pass intermediate of level i lives in half (i & 1) of the scratch
    a.scratch = scr ? scr : p->d_scratch + (L.level & 1) * p->half_elems;
    if (!(passes & 1)) {
      // cols pass already run
    } else if (L.dual == 1) {
      FwdArgs d = a;
      d.level = L.level + 1;
      d.nitems = L.c2_count;
      d.items = p->d_levels + L.c2_off;
      d.scratch2 = p->d_scratch + ((L.level + 1) & 1) * p->half_elems;
      MRDFT_CUDA(p, timed(p, MRDFT_KIND_FWD_COLS, 0, st, [&] { return launch_fwd_cols2(d, L.c2_count, st); }));
      if (L.tail_count) {
        FwdArgs t = a;
        t.nitems = L.tail_count;
        t.items = p->d_levels + L.tail_off;
        MRDFT_CUDA(p, timed(p, MRDFT_KIND_FWD_COLS, 0, st, [&] { return launch_fwd_cols(t, L.tail_count, st); }));
      }
    } else if (L.dual == 0) {
      a.items = p->d_levels + L.off;
      MRDFT_CUDA(p, timed(p, MRDFT_KIND_FWD_COLS, 0, st, [&] { return launch_fwd_cols(a, L.count, st); }));
    }
    a.items = p->d_levels + L.off;
    if (passes & 2)
      MRDFT_CUDA(p, timed(p, MRDFT_KIND_FWD_ROWS, L.bytes, st, [&] { return launch_fwd_rows(a, L.count, st); }));
  }
  return MRDFT_OK;
}

// Fork the segment chains over the worker streams (event fork / join on the
// caller's stream, which also works under stream capture).
struct NoAfter {
  mrdft_status operator()(size_t, cudaStream_t) const { return MRDFT_OK; }
};
struct NoFork {
  mrdft_status operator()(bool) const { return MRDFT_OK; }
};
// before(j, s) runs before segment j's chain is enqueued on s, after(j, s)
// after it; forked(parallel) runs once the worker streams have forked from
// the caller's stream (parallel) or, without workers, before the first segment
template <class F, class A = NoAfter, class B = NoAfter, class K = NoFork>
mrdft_status run_segments(mrdft_plan_s* p, cudaStream_t st, F&& chain, A&& after = NoAfter{}, B&& before = NoAfter{},
                          K&& forked = NoFork{}) {
  const int nw = p->timing_serial ? 0 : (int)p->workers.size();
  if (nw <= 1) {
    mrdft_status r0 = forked(false);
    if (r0 != MRDFT_OK) return r0;
    for (size_t j = 0; j < p->segments.size(); ++j) {
      mrdft_status r = before(j, st);
      if (r == MRDFT_OK) r = chain(p->segments[j], st);
      if (r == MRDFT_OK) r = after(j, st);
      if (r != MRDFT_OK) return r;
    }
    return MRDFT_OK;
  }
  MRDFT_CUDA(p, cudaEventRecord(p->ev_fork, st));
  for (int k = 0; k < nw; ++k) MRDFT_CUDA(p, cudaStreamWaitEvent(p->workers[k], p->ev_fork, 0));
  mrdft_status r = forked(true);
  for (size_t j = 0; j < p->segments.size() && r == MRDFT_OK; ++j) {
    r = before(j, p->workers[j % nw]);
    if (r == MRDFT_OK) r = chain(p->segments[j], p->workers[j % nw]);
    if (r == MRDFT_OK) r = after(j, p->workers[j % nw]);
  }
  // join every worker back even after a failed launch, so that the caller's
  // stream stays ordered after whatever was queued (and a capture can end)
  for (int k = 0; k < nw; ++k) {
    cudaError_t e = cudaEventRecord(p->ev_join[k], p->workers[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ev_join[k], 0);
    if (e != cudaSuccess && r == MRDFT_OK) r = cuda_fail(p, e, "joining the worker streams");
  }
  return r;
}

// The output runs of mrdft_forward_host by the phase after which they are
// final: a signal's in-tile levels (all of it when m <= 12) after the tile
// launch (phase 0, when the in-tile levels of every segment are one launch;
// tiny signals run before it), levels 13..seg_log after the segments
// (phase 1), the levels above the segment size at the end (phase 2).  The
// bit-reversed layout is written at the very end, and too many runs would
// cost more host calls than they save: then one run at the end.
void build_host_runs(mrdft_plan_s* p) {
  for (auto& v : p->host_runs) v.clear();
  const bool early_tiles = p->tile_first && p->tile_parts.size() <= 1;
  std::vector<size_t> order(p->sigs.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](size_t u, size_t v) { return p->sigs[u].out_off < p->sigs[v].out_off; });
  auto add = [&](int ph, int64_t off, int64_t cnt) {
    if (cnt <= 0) return;
    auto& v = p->host_runs[ph];
    if (!v.empty() && v.back().off + v.back().count == off) v.back().count += cnt;
    else v.push_back({off, cnt});
  };
  for (size_t k : order) {
    const SigDesc& sd = p->sigs[k];
    const int64_t N = int64_t(1) << sd.m;
    const int tile_lv = std::min(sd.m, kTileLog), seg_lv = std::max(tile_lv, std::min(sd.m, p->seg_log));
    add(early_tiles ? 0 : 1, sd.out_off, tile_lv * N);
    add(1, sd.out_off + tile_lv * N, (seg_lv - tile_lv) * N);
    add(2, sd.out_off + seg_lv * N, (sd.m - seg_lv) * N);
  }
  const size_t runs = p->host_runs[0].size() + p->host_runs[1].size() + p->host_runs[2].size();
  if ((p->flags & MRDFT_FLAG_BITREV) || runs > 64) {
    for (auto& v : p->host_runs) v.clear();
    p->host_runs[2].push_back({0, p->out_elems});
  }
  p->host_runs_ready = true;
}

// Enqueue the copies of one phase on the copy stream, after the caller's
// stream reaches this point; phase 2 also joins the copy stream back.
mrdft_status host_phase(mrdft_plan_s* p, int ph, const void* y, cudaStream_t st) {
  const auto& runs = p->host_runs[ph];
  if (runs.empty() && ph < 2) return MRDFT_OK;
  MRDFT_CUDA(p, cudaEventRecord(p->ev_host[ph], st));
  MRDFT_CUDA(p, cudaStreamWaitEvent(p->d2h, p->ev_host[ph], 0));
  for (const auto& r : runs)
    MRDFT_CUDA(p, cudaMemcpyAsync(static_cast<float2*>(p->host_dst) + r.off, static_cast<const float2*>(y) + r.off,
                                  (size_t)r.count * sizeof(float2), cudaMemcpyDeviceToHost, p->d2h));
  if (ph == 2) {
    MRDFT_CUDA(p, cudaEventRecord(p->ev_host[3], p->d2h));
    MRDFT_CUDA(p, cudaStreamWaitEvent(st, p->ev_host[3], 0));
  }
  return MRDFT_OK;
}

mrdft_status enqueue_forward(mrdft_plan_s* p, const void* x, void* y, cudaStream_t st) {
  FwdArgs a{};
  a.x = x;
  a.in_real = p->dtype == MRDFT_R32;
  a.y = reinterpret_cast<float2*>(y);
  a.sigs = p->d_sigs;
  a.nsigs = (int)p->nsig;
  a.scratch = p->d_scratch;
  a.cb_min = p->fwd_cb_min;
  a.rows14 = p->fwd_rows14;
  a.rows_pf = p->fwd_rows_pf;
  a.tile_lean = p->tile_lean;
  a.rows12 = p->fwd_rows12;
  a.tw = twiddles(p);
  a.status = p->d_status;
  if (p->n_tiny) {
    FwdArgs t = a;
    t.sig_ids = p->d_tiny_ids;
    t.nids = p->n_tiny;
    t.nitems = p->n_tiny;
    MRDFT_CUDA(p, timed(p, MRDFT_KIND_FWD_TINY, 0, st, [&] { return launch_fwd_tiny(t, p->n_tiny, st); }));
  }
  // tile_first: the first group's tile launch before the fork, the others on
  // the caller's stream after it, each segment waiting for its group's launch
  const bool parts = p->tile_first && p->tile_parts.size() > 1;
  if (p->tile_first && !parts && p->tile_all.count) {
    mrdft_status q = launch_fwd(p, a, p->tile_all, st);
    if (q != MRDFT_OK) return q;
  }
  if (p->host_dst) {
    mrdft_status q = host_phase(p, 0, y, st);
    if (q != MRDFT_OK) return q;
  }
  if (parts && p->tile_parts[0].count) {
    mrdft_status q = launch_fwd(p, a, p->tile_parts[0], st);
    if (q != MRDFT_OK) return q;
  }
  bool parallel = false;
  auto forked = [&](bool par) -> mrdft_status {
    parallel = par;
    if (!parts || !par) return MRDFT_OK;
    for (size_t g = 1; g < p->tile_parts.size(); ++g) {
      if (p->tile_parts[g].count) {
        mrdft_status q = launch_fwd(p, a, p->tile_parts[g], st);
        if (q != MRDFT_OK) return q;
      }
      MRDFT_CUDA(p, cudaEventRecord(p->ev_tile[g], st));
    }
    return MRDFT_OK;
  };
  auto before = [&](size_t j, cudaStream_t s) -> mrdft_status {
    if (!parts) return MRDFT_OK;
    const int g = p->seg_part[j];
    if (!parallel) {  // serial: the group's tiles right before its first segment
      if (g > 0 && p->seg_part[j - 1] != g && p->tile_parts[g].count) return launch_fwd(p, a, p->tile_parts[g], s);
      return MRDFT_OK;
    }
    if (g > 0) MRDFT_CUDA(p, cudaStreamWaitEvent(s, p->ev_tile[g], 0));
    return MRDFT_OK;
  };
  // the top levels' cols passes on their own stream (top_cols_early: from
  // here on; top_overlap alone: from the end of the segments)
  const bool early = !p->top_early.empty();
  const bool early_par = early && !p->timing_serial;
  const bool per_level = early_par && !p->ev_top_cols.empty();
  auto early_scr = [&](size_t j) { return p->d_scratch_top + (int64_t)j * p->half_elems; };
  bool early_forked = false;
  // an error after the fork still joins the early stream (stream capture
  // must end with every forked stream joined)
  auto join_on_error = [&](mrdft_status q) {
    if (early_forked) {
      cudaEventRecord(p->ev_early_done, p->early);
      cudaStreamWaitEvent(st, p->ev_early_done, 0);
      early_forked = false;
    }
    return q;
  };
  auto start_early = [&]() -> mrdft_status {
    cudaStream_t es = early_par ? p->early : st;
    if (early_par) {
      MRDFT_CUDA(p, cudaEventRecord(p->ev_early_go, st));
      MRDFT_CUDA(p, cudaStreamWaitEvent(es, p->ev_early_go, 0));
      early_forked = true;
    }
    // during the segments (top_cols_early) the intermediates wait for the
    // end: stored evict-first so that they do not push the segments' data
    // out of L2
    FwdArgs ea = a;
    ea.f_late = p->top_cols_early ? 1 : 0;
    for (size_t j = 0; j < p->top_early.size(); ++j) {
      mrdft_status q = launch_fwd(p, ea, p->top[p->top_early[j]], es, 1, early_scr(j));
      if (q != MRDFT_OK) return join_on_error(q);
      if (per_level) {
        const cudaError_t e = cudaEventRecord(p->ev_top_cols[j], es);
        if (e != cudaSuccess) return join_on_error(cuda_fail(p, e, "cudaEventRecord(ev_top_cols)"));
      }
    }
    if (early_par && !per_level) MRDFT_CUDA(p, cudaEventRecord(p->ev_early_done, es));
    return MRDFT_OK;
  };
  const bool early_at_start = early && p->top_cols_early;
  if (early_at_start) {
    mrdft_status q = start_early();
    if (q != MRDFT_OK) return q;
  }
  const bool tree = !p->top_nodes.empty();
  // forward tree: a node is enqueued right after the later of its two
  // children, on that child's stream, after an event of the other child
  std::vector<int> pending(p->top_nodes.size(), 2);
  std::vector<cudaStream_t> done_on(p->top_nodes.size(), nullptr);
  std::vector<cudaStream_t> seg_on(tree ? p->segments.size() : 0, nullptr);
  auto child_done = [&](int parent, cudaStream_t s) -> mrdft_status {
    while (parent >= 0 && --pending[parent] == 0) {
      const TopNode& nd = p->top_nodes[parent];
      for (int c = 0; c < 2; ++c) {  // the child on another stream: wait for its event
        const int ch = nd.child[c];
        const cudaStream_t cs = ch >= 0 ? seg_on[ch] : done_on[-ch - 1];
        const cudaEvent_t ev = ch >= 0 ? p->ev_seg[ch] : p->ev_node[-ch - 1];
        if (cs != s) MRDFT_CUDA(p, cudaStreamWaitEvent(s, ev, 0));
      }
      mrdft_status q = launch_fwd(p, a, nd.L, s);
      if (q != MRDFT_OK) return q;
      done_on[parent] = s;
      if (nd.parent >= 0) MRDFT_CUDA(p, cudaEventRecord(p->ev_node[parent], s));
      parent = nd.parent;
    }
    return MRDFT_OK;
  };
  mrdft_status r = run_segments(
      p, st,
      [&](const Segment& seg, cudaStream_t s) {
        for (const Launch& L : seg.chain) {
          mrdft_status q = launch_fwd(p, a, L, s);
          if (q != MRDFT_OK) return q;
        }
        return MRDFT_OK;
      },
      [&](size_t j, cudaStream_t s) -> mrdft_status {
        if (!tree || p->segments[j].parent < 0) return MRDFT_OK;
        seg_on[j] = s;
        MRDFT_CUDA(p, cudaEventRecord(p->ev_seg[j], s));
        return child_done(p->segments[j].parent, s);
      },
      before, forked);
  if (r != MRDFT_OK) return join_on_error(r);
  if (p->host_dst) {
    r = host_phase(p, 1, y, st);
    if (r != MRDFT_OK) return join_on_error(r);
  }
  if (early && !early_at_start) {
    r = start_early();
    if (r != MRDFT_OK) return r;
  }
  if (early_par && !per_level) MRDFT_CUDA(p, cudaStreamWaitEvent(st, p->ev_early_done, 0));
  if (!tree) {
    // with per-level events the caller's stream joins the early stream at
    // the wait for its last cols pass (nothing is enqueued there after it)
    for (size_t k = 0; k < p->top.size(); ++k) {
      size_t j = 0;
      while (j < p->top_early.size() && p->top_early[j] != (int)k) ++j;
      if (j < p->top_early.size()) {
        if (per_level) {
          const cudaError_t e = cudaStreamWaitEvent(st, p->ev_top_cols[j], 0);
          if (e != cudaSuccess) return join_on_error(cuda_fail(p, e, "cudaStreamWaitEvent(ev_top_cols)"));
        }
        r = launch_fwd(p, a, p->top[k], st, 2, early_scr(j));
      } else {
        r = launch_fwd(p, a, p->top[k], st);
      }
      if (r != MRDFT_OK) return join_on_error(r);
    }
  }
  if (p->flags & MRDFT_FLAG_BITREV) {
    // every window rewritten in place in the bit-reversed order of Sec. 3
    FwdArgs b = a;
    if (p->br_small) {
      b.items = p->d_br;
      b.nitems = p->br_small;
      MRDFT_CUDA(p, launch_bitrev_small(b, p->br_small, st));
    }
    for (const auto& lv : p->br_big) {
      b.items = p->d_br + lv.second.first;
      b.nitems = lv.second.second;
      MRDFT_CUDA(p, launch_bitrev_big(b, lv.second.second, lv.first, st));
    }
  }
  if (p->host_dst) return host_phase(p, 2, y, st);
  return MRDFT_OK;
}

// Even-bin propagation buffers: level i writes d_e[i & 1] and reads
// d_e[(i + 1) & 1], except across the boundary between the top chain and the
// segments, which goes through d_etop.
mrdft_status launch_adj(mrdft_plan_s* p, AdjArgs a, const Launch& L, cudaStream_t st, bool in_top) {
  const int S = p->seg_log;
  auto ebuf = [&](int lv) { return (lv & 1) ? p->d_e1 : p->d_e0; };
  a.level = L.level;
  a.nitems = L.count;
  if (L.kind == LK_TILE) {
    a.sig_ids = p->d_tile_ids;
    a.nids = p->n_tile_ids;
    a.items = p->d_tiles + L.off;
    a.e_in = (!in_top && S == kTileLog && p->d_etop) ? p->d_etop : ebuf(kTileLog + 1);
    if (p->lone_m && !a.t) {
      a.scratch = p->d_lone;
      a.ticket = p->d_ticket;
      MRDFT_CUDA(p, timed(p, MRDFT_KIND_ADJ_TILE, L.bytes, st, [&] { return launch_adj_levels(a, p->lone_m, st); }));
    } else {
      MRDFT_CUDA(p, timed(p, MRDFT_KIND_ADJ_TILE, L.bytes, st, [&] { return launch_adj_tile(a, L.count, st); }));
    }
    return MRDFT_OK;
  }
  a.items = p->d_levels + L.off;
  a.e_out = (in_top && L.level == S + 1) ? p->d_etop : ebuf(L.level);
  a.e_in = (!in_top && L.level == S && p->d_etop) ? p->d_etop : ebuf(L.level + 1);
  if (L.kind == LK_WIN) {
    MRDFT_CUDA(p, timed(p, MRDFT_KIND_ADJ_WINDOW, L.bytes, st, [&] { return launch_adj_window(a, L.count, st); }));
  } else {
    // the two-pass intermediate of level i lives in half (i & 1) of the scratch;
    // a paired upper level leaves its cols pass to the lower level's launch,
    // which runs it with its own after both rows passes
    a.scratch = p->d_scratch + (L.level & 1) * p->half_elems;
    MRDFT_CUDA(p, timed(p, MRDFT_KIND_ADJ_ROWS, L.bytes, st, [&] { return launch_adj_rows(a, L.count, st); }));
    if (L.dual == 1 && adj_cols2_pairable(L.level + 1, p->adj_cb_min)) {
      AdjArgs d = a;
      d.level = L.level + 1;
      d.nitems = L.c2_count;
      d.items = p->d_levels + L.c2_off;
      d.scratch2 = p->d_scratch + ((L.level + 1) & 1) * p->half_elems;
      MRDFT_CUDA(p, timed(p, MRDFT_KIND_ADJ_COLS, 0, st, [&] { return launch_adj_cols2(d, L.c2_count, st); }));
      if (L.tail_count) {
        AdjArgs t = a;
        t.nitems = L.tail_count;
        t.items = p->d_levels + L.tail_off;
        MRDFT_CUDA(p, timed(p, MRDFT_KIND_ADJ_COLS, 0, st, [&] { return launch_adj_cols(t, L.tail_count, st); }));
      }
    } else if (!(L.dual == 2 && adj_cols2_pairable(L.level, p->adj_cb_min))) {
      MRDFT_CUDA(p, timed(p, MRDFT_KIND_ADJ_COLS, 0, st, [&] { return launch_adj_cols(a, L.count, st); }));
    }
  }
  return MRDFT_OK;
}

mrdft_status enqueue_adjoint(mrdft_plan_s* p, const void* gy, void* gx, cudaStream_t st) {
  AdjArgs a{};
  a.rows13 = p->adj_rows13;
  a.cb_min = p->adj_cb_min;
  a.gy = reinterpret_cast<const float2*>(gy);
  a.gx = reinterpret_cast<float2*>(gx);
  a.sigs = p->d_sigs;
  a.nsigs = (int)p->nsig;
  a.acc = p->d_acc;
  a.scratch = p->d_scratch;
  a.tw = twiddles(p);
  a.status = p->d_status;
  a.t = p->cur_t;
  a.loss = p->cur_loss;
  for (auto it = p->top.rbegin(); it != p->top.rend(); ++it) {
    mrdft_status r = launch_adj(p, a, *it, st, true);
    if (r != MRDFT_OK) return r;
  }
  // tile_first: the tile launch after every segment, or with tile_split > 1
  // one launch per group of segments on the caller's stream, right after the
  // group's last segment is enqueued, waiting for each segment of the group
  const bool parts = p->tile_first && p->tile_parts.size() > 1;
  bool parallel = false;
  mrdft_status r = run_segments(
      p, st,
      [&](const Segment& seg, cudaStream_t s) {
        for (auto it = seg.chain.rbegin(); it != seg.chain.rend(); ++it) {
          mrdft_status q = launch_adj(p, a, *it, s, false);
          if (q != MRDFT_OK) return q;
        }
        return MRDFT_OK;
      },
      [&](size_t j, cudaStream_t s) -> mrdft_status {
        if (!parts) return MRDFT_OK;
        const int g = p->seg_part[j];
        const bool last = j + 1 == p->segments.size() || p->seg_part[j + 1] != g;
        if (!parallel) return last && p->tile_parts[g].count ? launch_adj(p, a, p->tile_parts[g], s, false) : MRDFT_OK;
        MRDFT_CUDA(p, cudaEventRecord(p->ev_segdone[j], s));
        if (!last) return MRDFT_OK;
        for (size_t k = 0; k <= j; ++k)
          if (p->seg_part[k] == g) MRDFT_CUDA(p, cudaStreamWaitEvent(st, p->ev_segdone[k], 0));
        return p->tile_parts[g].count ? launch_adj(p, a, p->tile_parts[g], st, false) : MRDFT_OK;
      },
      NoAfter{}, [&](bool par) -> mrdft_status {
        parallel = par;
        return MRDFT_OK;
      });
  if (r != MRDFT_OK) return r;
  if (p->tile_first && !parts && p->tile_all.count) {
    r = launch_adj(p, a, p->tile_all, st, false);
    if (r != MRDFT_OK) return r;
  }
  if (p->n_tiny) {
    AdjArgs t = a;
    t.sig_ids = p->d_tiny_ids;
    t.nids = p->n_tiny;
    t.nitems = p->n_tiny;
    MRDFT_CUDA(p, timed(p, MRDFT_KIND_ADJ_TINY, 0, st, [&] { return launch_adj_tiny(t, p->n_tiny, st); }));
  }
  return MRDFT_OK;
}

using Enqueue = mrdft_status (*)(mrdft_plan_s*, const void*, void*, cudaStream_t);


mrdft_status run(mrdft_plan_s* p, std::vector<GraphEntry>& cache, Enqueue fn, const void* in, void* out,
                 cudaStream_t st) {
  int dev = -1;
  MRDFT_CUDA(p, cudaGetDevice(&dev));
  if (dev != p->device) return fail(p, MRDFT_EINVAL, "plan used on a different device than it was created on");
  if (!(p->flags & MRDFT_FLAG_GRAPH) || p->timing) return fn(p, in, out, st);
  const GraphKey key{in, out, st, p->cur_t, p->cur_loss};
  for (GraphEntry& g : cache) {
    if (g.key == key) {
      g.last_use = ++p->graph_clock;
      MRDFT_CUDA(p, cudaGraphLaunch(g.exec, st));
      return MRDFT_OK;
    }
  }
  cudaStream_t cap = st;
  bool own = false;
  if (cap == nullptr) {  // the legacy stream cannot be captured
    MRDFT_CUDA(p, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    own = true;
  }
  MRDFT_CUDA(p, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  mrdft_status s = fn(p, in, out, cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cap, &graph);
  if (own) cudaStreamDestroy(cap);
  if (s != MRDFT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaStreamEndCapture");
  ++p->graph_captures;
  cudaGraphExec_t ex = nullptr;
  if (cache.size() >= kGraphCacheMax) {
    size_t old = 0;
    for (size_t j = 1; j < cache.size(); ++j)
      if (cache[j].last_use < cache[old].last_use) old = j;
    cudaGraphExecUpdateResultInfo info{};
    if (cudaGraphExecUpdate(cache[old].exec, graph, &info) == cudaSuccess) {
      ex = cache[old].exec;
      cache[old].key = key;
      cache[old].last_use = ++p->graph_clock;
      ++p->graph_updates;
    } else {
      (void)cudaGetLastError();
      cudaGraphExecDestroy(cache[old].exec);
      cache.erase(cache.begin() + (std::ptrdiff_t)old);
    }
  }
  if (!ex) {
    e = cudaGraphInstantiate(&ex, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_fail(p, e, "cudaGraphInstantiate");
    }
    cache.push_back(GraphEntry{key, ex, ++p->graph_clock});
  }
  cudaGraphDestroy(graph);
  MRDFT_CUDA(p, cudaGraphLaunch(ex, st));
  return MRDFT_OK;
}

bool misaligned(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15) != 0; }

}  // namespace

extern "C" {

mrdft_status mrdft_plan(mrdft_plan_t* out, const int64_t* lengths, int64_t n_lengths, int64_t batch,
                        int dtype, uint32_t flags) {
  return mrdft_plan_opts(out, lengths, n_lengths, batch, dtype, flags, 0, 0);
}

mrdft_status mrdft_plan_opts(mrdft_plan_t* out, const int64_t* lengths, int64_t n_lengths, int64_t batch,
                             int dtype, uint32_t flags, int32_t seg_log, int32_t streams) {
  mrdft_exec_opts o{};
  o.seg_log = seg_log;
  o.streams = streams;
  return mrdft_plan_ex(out, lengths, n_lengths, batch, dtype, flags, &o);
}

mrdft_status mrdft_plan_ex(mrdft_plan_t* out, const int64_t* lengths, int64_t n_lengths, int64_t batch, int dtype,
                           uint32_t flags, const mrdft_exec_opts* opts) {
  if (!out) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: out is NULL");
  *out = nullptr;
  mrdft_exec_opts o{};
  if (opts) o = *opts;
  auto sw = [](int32_t v) { return v == MRDFT_OPT_DEFAULT || v == MRDFT_OPT_OFF || v == MRDFT_OPT_ON; };
  if (o.seg_log != 0 && (o.seg_log < kTileLog || o.seg_log > kMaxLog))
    return fail(nullptr, MRDFT_EINVAL, "mrdft_plan_ex: seg_log must be 0 or in [12, 26]");
  if (o.streams < 0 || o.streams > 16) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan_ex: streams must be in [0, 16]");
  if (o.fwd_cb != 0 && (o.fwd_cb < 9 || o.fwd_cb > 11))
    return fail(nullptr, MRDFT_EINVAL, "mrdft_plan_ex: fwd_cb must be 0 or in [9, 11]");
  if (o.tile_split < 0 || o.tile_split > 64)
    return fail(nullptr, MRDFT_EINVAL, "mrdft_plan_ex: tile_split must be in [0, 64]");
  if (o.adj_cb != 0 && (o.adj_cb < 9 || o.adj_cb > 10))
    return fail(nullptr, MRDFT_EINVAL, "mrdft_plan_ex: adj_cb must be 0 or in [9, 10]");
  if (!sw(o.fwd_rows_prefetch) || !sw(o.fwd_rows14) || !sw(o.adj_rows13) || !sw(o.dual_cols) || !sw(o.fwd_tree) ||
      !sw(o.tile_first) || !sw(o.tile_lean) || !sw(o.fwd_rows12) || !sw(o.top_cols_early) ||
      !sw(o.top_overlap) || !sw(o.levels_parallel))
    return fail(nullptr, MRDFT_EINVAL, "mrdft_plan_ex: switches must be MRDFT_OPT_DEFAULT, _OFF or _ON");
  if (!lengths) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: lengths is NULL");
  if (batch < 1 || batch > (int64_t(1) << 30))
    return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: batch must be in [1, 2^30]");
  if (n_lengths != 1 && n_lengths != batch)
    return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: n_lengths must be 1 or batch");
  if (dtype != MRDFT_C64 && dtype != MRDFT_R32) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: unknown dtype");
  if (flags & ~(MRDFT_FLAG_GRAPH | MRDFT_FLAG_BITREV)) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: unknown flag bits");
  int64_t total = 0;
  for (int64_t s = 0; s < n_lengths; ++s) {
    const int64_t N = lengths[s];
    if (N < 2 || N > (int64_t(1) << kMaxLog) || (N & (N - 1)) != 0)
      return fail(nullptr, MRDFT_EINVAL,
                  "mrdft_plan: every length must be a power of two in [2, 2^26], got " + std::to_string(N));
    total += (n_lengths == 1) ? N * batch : N;
    if (total > (int64_t(1) << 36)) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: batch too large");
  }
  mrdft_plan_s* p = new (std::nothrow) mrdft_plan_s();
  if (!p) return fail(nullptr, MRDFT_ENOMEM, "mrdft_plan: host allocation failed");
  p->dtype = dtype;
  p->flags = flags;
  if (o.seg_log) {
    p->seg_log = o.seg_log;
    p->seg_fixed = true;
  }
  if (o.streams) {
    p->nstreams = o.streams;
    p->streams_fixed = true;
  }
  auto on = [](int32_t v, bool dflt) { return v == MRDFT_OPT_DEFAULT ? dflt : v == MRDFT_OPT_ON; };
  if (o.fwd_cb) p->fwd_cb_min = o.fwd_cb;
  if (o.adj_cb) p->adj_cb_min = o.adj_cb;
  if (o.tile_split) p->tile_split = o.tile_split;
  p->fwd_rows_pf = on(o.fwd_rows_prefetch, p->fwd_rows_pf != 0);
  p->fwd_rows14 = on(o.fwd_rows14, p->fwd_rows14 != 0);
  p->adj_rows13 = on(o.adj_rows13, p->adj_rows13 != 0);
  p->dual_cols = on(o.dual_cols, p->dual_cols);
  p->fwd_tree = on(o.fwd_tree, p->fwd_tree);
  p->tile_first = on(o.tile_first, p->tile_first);
  p->tile_lean = on(o.tile_lean, p->tile_lean);
  p->fwd_rows12 = on(o.fwd_rows12, p->fwd_rows12);
  p->top_cols_early = on(o.top_cols_early, p->top_cols_early);
  p->top_overlap = on(o.top_overlap, p->top_overlap);
  p->levels_parallel = on(o.levels_parallel, p->levels_parallel);
  mrdft_status st = build_plan(p, lengths, n_lengths, batch);
  if (st != MRDFT_OK) {
    fail(nullptr, st, p->err);
    release(p);
    delete p;
    return st;
  }
  *out = p;
  return MRDFT_OK;
}

mrdft_status mrdft_plan_get_opts(mrdft_plan_t p, mrdft_exec_opts* opts) {
  if (!p || !opts) return fail(p, MRDFT_EINVAL, "mrdft_plan_get_opts: NULL argument");
  auto sw = [](bool v) { return v ? MRDFT_OPT_ON : MRDFT_OPT_OFF; };
  opts->seg_log = p->seg_log;
  opts->streams = p->nstreams;
  opts->fwd_cb = p->fwd_cb_min;
  opts->adj_cb = p->adj_cb_min;
  opts->fwd_rows_prefetch = sw(p->fwd_rows_pf != 0);
  opts->fwd_rows14 = sw(p->fwd_rows14 != 0);
  opts->adj_rows13 = sw(p->adj_rows13 != 0);
  opts->dual_cols = sw(p->dual_cols);
  opts->fwd_tree = sw(p->fwd_tree);
  opts->tile_first = sw(p->tile_first);
  opts->tile_lean = sw(p->tile_lean);
  opts->fwd_rows12 = sw(p->fwd_rows12);
  opts->tile_split = p->tile_split;
  opts->top_cols_early = sw(p->top_cols_early);
  opts->top_overlap = sw(p->top_overlap);
  opts->levels_parallel = sw(p->levels_parallel);
  return MRDFT_OK;
}

mrdft_status mrdft_output_elems(mrdft_plan_t p, int64_t* elems) {
  if (!p || !elems) return fail(p, MRDFT_EINVAL, "mrdft_output_elems: NULL argument");
  *elems = p->out_elems;
  return MRDFT_OK;
}

mrdft_status mrdft_input_elems(mrdft_plan_t p, int64_t* elems) {
  if (!p || !elems) return fail(p, MRDFT_EINVAL, "mrdft_input_elems: NULL argument");
  *elems = p->in_elems;
  return MRDFT_OK;
}

mrdft_status mrdft_forward(mrdft_plan_t p, const void* x, void* y, mrdft_stream_t stream) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_forward: plan is NULL");
  if (!x || !y) return fail(p, MRDFT_EINVAL, "mrdft_forward: x or y is NULL");
  if (misaligned(x) || misaligned(y)) return fail(p, MRDFT_EINVAL, "mrdft_forward: x and y must be 16-byte aligned");
  return run(p, p->fwd_graphs, enqueue_forward, x, y, reinterpret_cast<cudaStream_t>(stream));
}

mrdft_status mrdft_adjoint(mrdft_plan_t p, const void* gy, void* gx, mrdft_stream_t stream) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_adjoint: plan is NULL");
  if (!gy || !gx) return fail(p, MRDFT_EINVAL, "mrdft_adjoint: gy or gx is NULL");
  if (misaligned(gy) || misaligned(gx)) return fail(p, MRDFT_EINVAL, "mrdft_adjoint: gy and gx must be 16-byte aligned");
  if (p->flags & MRDFT_FLAG_BITREV)
    return fail(p, MRDFT_EUNSUPPORTED, "mrdft_adjoint: plans with MRDFT_FLAG_BITREV are forward-only");
  return run(p, p->adj_graphs, enqueue_adjoint, gy, gx, reinterpret_cast<cudaStream_t>(stream));
}

mrdft_status mrdft_loss_grad(mrdft_plan_t p, const void* x, const void* t, void* y, void* gx, double* loss,
                             mrdft_stream_t stream) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_loss_grad: plan is NULL");
  if (!x || !t || !y || !gx) return fail(p, MRDFT_EINVAL, "mrdft_loss_grad: x, t, y or gx is NULL");
  if (misaligned(x) || misaligned(t) || misaligned(y) || misaligned(gx))
    return fail(p, MRDFT_EINVAL, "mrdft_loss_grad: buffers must be 16-byte aligned");
  if (loss && (reinterpret_cast<uintptr_t>(loss) & 7) != 0)
    return fail(p, MRDFT_EINVAL, "mrdft_loss_grad: loss must be 8-byte aligned");
  if (p->flags & MRDFT_FLAG_BITREV)
    return fail(p, MRDFT_EUNSUPPORTED, "mrdft_loss_grad: plans with MRDFT_FLAG_BITREV are forward-only");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  mrdft_status s = run(p, p->fwd_graphs, enqueue_forward, x, y, st);
  if (s != MRDFT_OK) return s;
  if (loss) MRDFT_CUDA(p, cudaMemsetAsync(loss, 0, sizeof(double), st));
  p->cur_t = reinterpret_cast<const float2*>(t);
  p->cur_loss = loss;
  s = run(p, p->adj_graphs, enqueue_adjoint, y, gx, st);
  p->cur_t = nullptr;
  p->cur_loss = nullptr;
  return s;
}

mrdft_status mrdft_forward_host(mrdft_plan_t p, const void* x_host, void* y_host, mrdft_stream_t stream) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_forward_host: plan is NULL");
  if (!x_host || !y_host) return fail(p, MRDFT_EINVAL, "mrdft_forward_host: x or y is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t xb = (size_t)p->in_elems * (p->dtype == MRDFT_R32 ? sizeof(float) : sizeof(float2));
  const size_t yb = (size_t)p->out_elems * sizeof(float2);
  if (!p->d_stage_x) {
    cudaError_t e = cudaMalloc(&p->d_stage_x, xb);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_stage_y, yb);
    if (e != cudaSuccess) return fail(p, MRDFT_ENOMEM, std::string("staging allocation: ") + cudaGetErrorString(e));
  }
  if (!p->d2h) {
    MRDFT_CUDA(p, cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking));
    for (cudaEvent_t& e : p->ev_host) MRDFT_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (!p->host_runs_ready) build_host_runs(p);
  int dev = -1;
  MRDFT_CUDA(p, cudaGetDevice(&dev));
  if (dev != p->device) return fail(p, MRDFT_EINVAL, "plan used on a different device than it was created on");
  MRDFT_CUDA(p, cudaMemcpyAsync(p->d_stage_x, x_host, xb, cudaMemcpyHostToDevice, st));
  // enqueued directly (no graph: the copies carry this call's host pointer),
  // each finished part of the output leaving while the rest is computed
  p->host_dst = y_host;
  mrdft_status s = enqueue_forward(p, p->d_stage_x, p->d_stage_y, st);
  p->host_dst = nullptr;
  if (s != MRDFT_OK) {
    cudaStreamSynchronize(p->d2h);
    return s;
  }
  MRDFT_CUDA(p, cudaStreamSynchronize(st));
  return MRDFT_OK;
}

mrdft_status mrdft_status_poll(mrdft_plan_t p) {
  if (!p) return noalloc_status_poll();
  int v = 0;
  MRDFT_CUDA(p, cudaDeviceSynchronize());
  MRDFT_CUDA(p, cudaMemcpy(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  MRDFT_CUDA(p, cudaMemset(p->d_status, 0, sizeof(int)));
  if (v == kStatusTimeout) return fail(p, MRDFT_ETIMEOUT, "a device-side wait gave up");
  if (v != 0) return fail(p, MRDFT_EDEVICE, "a kernel flagged an invalid work item (code " + std::to_string(v) + ")");
  return MRDFT_OK;
}

const char* mrdft_last_error(mrdft_plan_t p) {
  if (p) return p->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  static thread_local std::string copy;
  copy = g_global_err;
  return copy.c_str();
}

mrdft_status mrdft_plan_info(mrdft_plan_t p, int32_t* tile_log, int32_t* fwd_launches, int32_t* adj_launches) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan_info: plan is NULL");
  int n = p->n_tiny ? 1 : 0;
  int na = n;
  auto count = [&](const Launch& L) {
    if (L.kind != LK_PASS) na += 1;
    else if (L.dual == 1 && adj_cols2_pairable(L.level + 1, p->adj_cb_min)) na += 2 + (L.tail_count ? 1 : 0);
    else na += L.dual == 2 && adj_cols2_pairable(L.level, p->adj_cb_min) ? 1 : 2;
    if (L.kind != LK_PASS) n += 1;
    else if (L.dual == 1) n += 2 + (L.tail_count ? 1 : 0);
    else n += L.dual == 2 ? 1 : 2;
  };
  for (const Segment& g : p->segments)
    for (const Launch& L : g.chain) count(L);
  if (p->tile_first) {
    if (p->tile_parts.size() > 1) {
      for (const Launch& L : p->tile_parts)
        if (L.count) count(L);
    } else if (p->tile_all.count) {
      count(p->tile_all);
    }
  }
  if (p->top_nodes.empty()) {
    for (const Launch& L : p->top) count(L);
  } else {
    const int n_keep = n;
    for (const Launch& L : p->top) count(L);
    n = n_keep;
    for (const TopNode& nd : p->top_nodes) n += nd.L.kind == LK_PASS ? 2 : 1;
  }
  if (tile_log) *tile_log = kTileLog;
  if (fwd_launches) *fwd_launches = n;
  if (adj_launches) *adj_launches = na;
  return MRDFT_OK;
}

mrdft_status mrdft_timing_enable(mrdft_plan_t p, int enable) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_timing_enable: plan is NULL");
  collect_timing(p);
  p->timing = enable != 0;
  p->timing_serial = enable == 2;
  for (int k = 0; k < MRDFT_KIND_COUNT; ++k) {
    p->t_ms[k] = 0.0;
    p->t_launches[k] = 0;
    p->t_bytes[k] = 0;
  }
  return MRDFT_OK;
}

mrdft_status mrdft_timing_read(mrdft_plan_t p, int kind, double* ms, int64_t* launches, int64_t* bytes) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_timing_read: plan is NULL");
  if (kind < 0 || kind >= MRDFT_KIND_COUNT) return fail(p, MRDFT_EINVAL, "mrdft_timing_read: bad kind");
  collect_timing(p);
  if (ms) *ms = p->t_ms[kind];
  if (launches) *launches = p->t_launches[kind];
  if (bytes) *bytes = p->t_bytes[kind];
  return MRDFT_OK;
}

mrdft_status mrdft_plan_graph_stats(mrdft_plan_t p, int32_t* cached, int64_t* captures, int64_t* updates) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan_graph_stats: plan is NULL");
  if (cached) *cached = (int32_t)(p->fwd_graphs.size() + p->adj_graphs.size());
  if (captures) *captures = p->graph_captures;
  if (updates) *updates = p->graph_updates;
  return MRDFT_OK;
}

mrdft_status mrdft_debug_item(mrdft_plan_t p, int list, int64_t index, const int32_t* new_fields,
                              int32_t* old_fields) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_debug_item: plan is NULL");
  if (list != 0 && list != 1) return fail(p, MRDFT_EINVAL, "mrdft_debug_item: list must be 0 (tiles) or 1 (levels)");
  const int64_t n = list == 0 ? p->n_tiles : p->n_level_items;
  if (index < 0 || index >= n) return fail(p, MRDFT_EINVAL, "mrdft_debug_item: index out of range");
  static_assert(sizeof(TileItem) == 16 && sizeof(LevelItem) == 16, "work items are four 32-bit words");
  void* dev = list == 0 ? static_cast<void*>(p->d_tiles + index) : static_cast<void*>(p->d_levels + index);
  int32_t cur[4];
  MRDFT_CUDA(p, cudaDeviceSynchronize());
  MRDFT_CUDA(p, cudaMemcpy(cur, dev, sizeof(cur), cudaMemcpyDeviceToHost));
  if (old_fields) std::memcpy(old_fields, cur, sizeof(cur));
  if (new_fields) MRDFT_CUDA(p, cudaMemcpy(dev, new_fields, sizeof(cur), cudaMemcpyHostToDevice));
  return MRDFT_OK;
}

void mrdft_destroy(mrdft_plan_t p) {
  if (!p) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  release(p);
  if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
  delete p;
}

}  // extern "C"
