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
}  // namespace mrdft

using namespace mrdft;

namespace {

constexpr int kMaxLog = 26;

struct LevelLaunch {
  int level;
  int kind;       // 0 window, 1 two-pass (cols + rows)
  int64_t off;    // first item in the level item array
  int count;      // items of the window kernel, or of each pass
};

struct GraphKey {
  const void* a;
  const void* b;
  cudaStream_t s;
  bool operator<(const GraphKey& o) const {
    if (a != o.a) return a < o.a;
    if (b != o.b) return b < o.b;
    return s < o.s;
  }
};

std::mutex g_err_mu;
std::string g_global_err = "no error";

}  // namespace

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
  TileItem* d_tiles = nullptr;
  int n_tiles = 0;
  int32_t* d_tiny_ids = nullptr;
  int n_tiny = 0;
  LevelItem* d_levels = nullptr;
  std::vector<LevelLaunch> level_launches;  // ascending level
  float2* d_tw13 = nullptr;
  float2* d_twlo = nullptr;
  float2* d_twhi = nullptr;
  float2* d_scratch = nullptr;  // N/2 per signal
  float2* d_e0 = nullptr;       // N/2 per signal
  float2* d_e1 = nullptr;       // N/2 per signal
  float2* d_acc = nullptr;      // N per signal
  int* d_status = nullptr;
  void* d_stage_x = nullptr;
  void* d_stage_y = nullptr;


  std::map<GraphKey, cudaGraphExec_t> fwd_graphs, adj_graphs;
  std::string err = "no error";
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

void release(mrdft_plan_s* p) {
  for (auto& kv : p->fwd_graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : p->adj_graphs) cudaGraphExecDestroy(kv.second);
  p->fwd_graphs.clear();
  p->adj_graphs.clear();
  void* ptrs[] = {p->d_sigs, p->d_tile_ids, p->d_tiles, p->d_tiny_ids, p->d_levels,
                  p->d_tw13, p->d_twlo, p->d_twhi, p->d_scratch, p->d_e0,
                  p->d_e1, p->d_acc, p->d_status, p->d_stage_x, p->d_stage_y};
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

  // ---- tile work list: signals grouped by m, small ones packed per tile
  std::vector<int32_t> order(batch);
  for (int64_t s = 0; s < batch; ++s) order[s] = (int32_t)s;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return p->sigs[a].m > p->sigs[b].m; });
  std::vector<int32_t> tile_ids, tiny_ids;
  std::vector<TileItem> tiles;
  size_t q = 0;
  while (q < order.size()) {
    const int m = p->sigs[order[q]].m;
    if (m <= 4) {
      tiny_ids.push_back(order[q]);
      ++q;
      continue;
    }
    if (m >= kTileLog) {
      const int32_t list = (int32_t)tile_ids.size();
      tile_ids.push_back(order[q]);
      const int64_t ntile = int64_t(1) << (m - kTileLog);
      for (int64_t t = 0; t < ntile; ++t) tiles.push_back(TileItem{list, 1, (int16_t)kTileLog, (int32_t)t, 0});
      ++q;
      continue;
    }
    // pack whole signals of equal length into one tile; the pack size is a
    // power of two (the in-tile FFT works on 2^k windows)
    const int per = 1 << (kTileLog - m);
    size_t avail = 0;
    while (q + avail < order.size() && p->sigs[order[q + avail]].m == m && (int)avail < per) ++avail;
    int n = 1;
    while ((size_t)(n * 2) <= avail) n *= 2;
    const int32_t list = (int32_t)tile_ids.size();
    for (int k = 0; k < n; ++k) tile_ids.push_back(order[q + k]);
    q += n;
    tiles.push_back(TileItem{list, (int16_t)n, (int16_t)m, 0, 0});
  }
  p->n_tiles = (int)tiles.size();
  p->n_tiny = (int)tiny_ids.size();

  // ---- level work lists (levels above the tile)
  std::vector<LevelItem> litems;
  for (int i = kTileLog + 1; i <= p->max_m; ++i) {
    LevelLaunch L{};
    L.level = i;
    L.off = (int64_t)litems.size();
    if (i <= kWinMaxLog + 1) {
      L.kind = 0;
      for (int64_t s = 0; s < batch; ++s) {
        if (p->sigs[s].m < i) continue;
        const int64_t nw = int64_t(1) << (p->sigs[s].m - i);
        for (int64_t w = 0; w < nw; ++w) litems.push_back(LevelItem{(int32_t)s, (int32_t)w, 0, 0});
      }
    } else {
      L.kind = 1;
      const int QB = i - 1 - kColsLog;
      const int nblk = std::max(1, (1 << QB) / 4);  // cols: C / RC ; rows: Q / KC
      for (int64_t s = 0; s < batch; ++s) {
        if (p->sigs[s].m < i) continue;
        const int64_t nw = int64_t(1) << (p->sigs[s].m - i);
        for (int64_t w = 0; w < nw; ++w)
          for (int b = 0; b < nblk; ++b) litems.push_back(LevelItem{(int32_t)s, (int32_t)w, b, 0});
      }
    }
    L.count = (int)((int64_t)litems.size() - L.off);
    p->level_launches.push_back(L);
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
  MRDFT_CUDA(p, dev_upload(&p->d_tw13, tw13));
  MRDFT_CUDA(p, dev_upload(&p->d_twlo, twlo));
  MRDFT_CUDA(p, dev_upload(&p->d_twhi, twhi));
  if (p->max_m > kTileLog) {
    const size_t half = (size_t)p->half_elems * sizeof(float2);
    cudaError_t e = cudaMalloc(&p->d_scratch, half);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_e0, half);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_e1, half);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_acc, 2 * half);
    if (e != cudaSuccess) return fail(p, MRDFT_ENOMEM, std::string("scratch allocation: ") + cudaGetErrorString(e));
  }
  MRDFT_CUDA(p, cudaMalloc(&p->d_status, sizeof(int)));
  MRDFT_CUDA(p, cudaMemset(p->d_status, 0, sizeof(int)));

  return MRDFT_OK;
}

Twiddles twiddles(const mrdft_plan_s* p) { return Twiddles{p->d_tw13, p->d_twlo, p->d_twhi}; }

mrdft_status enqueue_forward(mrdft_plan_s* p, const void* x, void* y, cudaStream_t st) {
  FwdArgs a{};
  a.x = x;
  a.in_real = p->dtype == MRDFT_R32;
  a.y = reinterpret_cast<float2*>(y);
  a.sigs = p->d_sigs;
  a.scratch = p->d_scratch;
  a.tw = twiddles(p);
  a.status = p->d_status;
  if (p->n_tiles) {
    a.sig_ids = p->d_tile_ids;
    a.items = p->d_tiles;
    a.nitems = p->n_tiles;
    MRDFT_CUDA(p, launch_fwd_tile(a, p->n_tiles, st));
  }
  if (p->n_tiny) {
    a.sig_ids = p->d_tiny_ids;
    a.items = nullptr;
    a.nitems = p->n_tiny;
    MRDFT_CUDA(p, launch_fwd_tiny(a, p->n_tiny, st));
  }
  for (const LevelLaunch& L : p->level_launches) {
    a.level = L.level;
    a.items = p->d_levels + L.off;
    a.nitems = L.count;
    if (L.kind == 0) {
      MRDFT_CUDA(p, launch_fwd_window(a, L.count, st));
    } else {
      MRDFT_CUDA(p, launch_fwd_cols(a, L.count, st));
      MRDFT_CUDA(p, launch_fwd_rows(a, L.count, st));
    }
  }
  return MRDFT_OK;
}

mrdft_status enqueue_adjoint(mrdft_plan_s* p, const void* gy, void* gx, cudaStream_t st) {
  AdjArgs a{};
  a.gy = reinterpret_cast<const float2*>(gy);
  a.gx = reinterpret_cast<float2*>(gx);
  a.sigs = p->d_sigs;
  a.acc = p->d_acc;
  a.scratch = p->d_scratch;
  a.tw = twiddles(p);
  a.status = p->d_status;
  for (auto it = p->level_launches.rbegin(); it != p->level_launches.rend(); ++it) {
    const LevelLaunch& L = *it;
    a.level = L.level;
    a.items = p->d_levels + L.off;
    a.nitems = L.count;
    a.e_out = (L.level & 1) ? p->d_e1 : p->d_e0;
    a.e_in = ((L.level + 1) & 1) ? p->d_e1 : p->d_e0;
    if (L.kind == 0) {
      MRDFT_CUDA(p, launch_adj_window(a, L.count, st));
    } else {
      MRDFT_CUDA(p, launch_adj_rows(a, L.count, st));
      MRDFT_CUDA(p, launch_adj_cols(a, L.count, st));
    }
  }
  if (p->n_tiles) {
    a.sig_ids = p->d_tile_ids;
    a.items = p->d_tiles;
    a.nitems = p->n_tiles;
    a.e_in = ((kTileLog + 1) & 1) ? p->d_e1 : p->d_e0;
    MRDFT_CUDA(p, launch_adj_tile(a, p->n_tiles, st));
  }
  if (p->n_tiny) {
    a.sig_ids = p->d_tiny_ids;
    a.items = nullptr;
    a.nitems = p->n_tiny;
    MRDFT_CUDA(p, launch_adj_tiny(a, p->n_tiny, st));
  }
  return MRDFT_OK;
}

using Enqueue = mrdft_status (*)(mrdft_plan_s*, const void*, void*, cudaStream_t);

mrdft_status run(mrdft_plan_s* p, std::map<GraphKey, cudaGraphExec_t>& cache, Enqueue fn,
                 const void* in, void* out, cudaStream_t st) {
  int dev = -1;
  MRDFT_CUDA(p, cudaGetDevice(&dev));
  if (dev != p->device) return fail(p, MRDFT_EINVAL, "plan used on a different device than it was created on");
  if (!(p->flags & MRDFT_FLAG_GRAPH)) return fn(p, in, out, st);
  const GraphKey key{in, out, st};
  auto found = cache.find(key);
  if (found == cache.end()) {
    cudaStream_t cap = st;
    bool own = false;
    if (cap == nullptr) {  // the legacy stream cannot be captured
      MRDFT_CUDA(p, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      own = true;
    }
    MRDFT_CUDA(p, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    mrdft_status s = fn(p, in, out, cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (own) cudaStreamDestroy(cap);
    if (s != MRDFT_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaGraphInstantiate");
    found = cache.emplace(key, ex).first;
  }
  MRDFT_CUDA(p, cudaGraphLaunch(found->second, st));
  return MRDFT_OK;
}

bool misaligned(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15) != 0; }

}  // namespace

extern "C" {

mrdft_status mrdft_plan(mrdft_plan_t* out, const int64_t* lengths, int64_t n_lengths, int64_t batch,
                        int dtype, uint32_t flags) {
  if (!out) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: out is NULL");
  *out = nullptr;
  if (!lengths) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: lengths is NULL");
  if (batch < 1 || batch > (int64_t(1) << 30))
    return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: batch must be in [1, 2^30]");
  if (n_lengths != 1 && n_lengths != batch)
    return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: n_lengths must be 1 or batch");
  if (dtype != MRDFT_C64 && dtype != MRDFT_R32) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: unknown dtype");
  if (flags & ~MRDFT_FLAG_GRAPH) return fail(nullptr, MRDFT_EINVAL, "mrdft_plan: unknown flag bits");
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
  return run(p, p->adj_graphs, enqueue_adjoint, gy, gx, reinterpret_cast<cudaStream_t>(stream));
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
  MRDFT_CUDA(p, cudaMemcpyAsync(p->d_stage_x, x_host, xb, cudaMemcpyHostToDevice, st));
  mrdft_status s = run(p, p->fwd_graphs, enqueue_forward, p->d_stage_x, p->d_stage_y, st);
  if (s != MRDFT_OK) return s;
  MRDFT_CUDA(p, cudaMemcpyAsync(y_host, p->d_stage_y, yb, cudaMemcpyDeviceToHost, st));
  MRDFT_CUDA(p, cudaStreamSynchronize(st));
  return MRDFT_OK;
}

mrdft_status mrdft_status_poll(mrdft_plan_t p) {
  if (!p) return fail(nullptr, MRDFT_EINVAL, "mrdft_status_poll: plan is NULL");
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
  int n = (p->n_tiles ? 1 : 0) + (p->n_tiny ? 1 : 0);
  for (const LevelLaunch& L : p->level_launches) n += L.kind == 0 ? 1 : 2;
  if (tile_log) *tile_log = kTileLog;
  if (fwd_launches) *fwd_launches = n;
  if (adj_launches) *adj_launches = n;
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
