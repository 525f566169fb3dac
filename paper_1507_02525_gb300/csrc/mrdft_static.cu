// Allocation-free forward MrDFT of one signal (mrdft_forward_noalloc).
//
// Everything the transform needs besides the caller's input and output lives
// in file-scope device arrays of fixed size: the intermediate of the two-pass
// levels (15 and 16), the twiddle tables, the signal descriptors and the work
// lists for every supported length.  Host code reaches them only through
// cudaGetSymbolAddress, once per device, at the first call on that device.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mrdft.h"
#include "mrdft_internal.h"

namespace mrdft {
cudaError_t set_fwd_attributes();
void set_global_error(const std::string& msg);
mrdft_status noalloc_status_poll();
}  // namespace mrdft

using namespace mrdft;

namespace {

constexpr int kMaxLogNA = MRDFT_NOALLOC_MAX_LOG;
constexpr int kScratchElems = 1 << (kMaxLogNA - 1);  // N/2 for the largest length

// Per-length work lists, concatenated: for each m, tile items, then the
// window items of level 14, then the two-pass items of levels 15..m.
constexpr int kMaxTileItems = 1 << (kMaxLogNA - kTileLog);
constexpr int kMaxLevelItems = 64;

}  // namespace

// The fixed-size device storage (held by every device that loads the library).
static __device__ __align__(256) float2 g_noalloc_scratch[kScratchElems];
static __device__ __align__(256) float2 g_noalloc_tw13[1 << kTwLog];
static __device__ __align__(256) float2 g_noalloc_twlo[1 << kTwSplit];
static __device__ __align__(256) float2 g_noalloc_twhi[1 << (kTwBigLog - kTwSplit)];
static __device__ SigDesc g_noalloc_sigs[kMaxLogNA + 1];
static __device__ int32_t g_noalloc_ids[kMaxLogNA + 1];
static __device__ TileItem g_noalloc_tiles[(kMaxLogNA + 1) * kMaxTileItems];
static __device__ LevelItem g_noalloc_levels[(kMaxLogNA + 1) * kMaxLevelItems];
static __device__ int g_noalloc_status;

namespace {

struct DevState {
  bool ready = false;
  float2* scratch = nullptr;
  float2* tw13 = nullptr;
  float2* twlo = nullptr;
  float2* twhi = nullptr;
  SigDesc* sigs = nullptr;
  int32_t* ids = nullptr;
  TileItem* tiles = nullptr;
  LevelItem* levels = nullptr;
  int* status = nullptr;
  // per m: count of tile items; per (m, level) offset/count into levels
  int ntile[kMaxLogNA + 1] = {0};
  int lvl_off[kMaxLogNA + 1][kMaxLogNA + 1] = {{0}};
  int lvl_cnt[kMaxLogNA + 1][kMaxLogNA + 1] = {{0}};
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DevState g_dev[kMaxDevices];

float2 root(int64_t e, int64_t L) {
  const double a = -2.0 * M_PI * (double)(e % L) / (double)L;
  return make_float2((float)std::cos(a), (float)std::sin(a));
}

template <class T>
cudaError_t symbol_ptr(T** out, const void* sym) {
  return cudaGetSymbolAddress(reinterpret_cast<void**>(out), sym);
}

// One-time set-up on the current device: symbol addresses, twiddle tables
// (FP64 on the host, rounded once), descriptors and work lists.
cudaError_t setup(DevState& st) {
  cudaError_t e;
  if ((e = symbol_ptr(&st.scratch, g_noalloc_scratch)) != cudaSuccess) return e;
  if ((e = symbol_ptr(&st.tw13, g_noalloc_tw13)) != cudaSuccess) return e;
  if ((e = symbol_ptr(&st.twlo, g_noalloc_twlo)) != cudaSuccess) return e;
  if ((e = symbol_ptr(&st.twhi, g_noalloc_twhi)) != cudaSuccess) return e;
  if ((e = symbol_ptr(&st.sigs, g_noalloc_sigs)) != cudaSuccess) return e;
  if ((e = symbol_ptr(&st.ids, g_noalloc_ids)) != cudaSuccess) return e;
  if ((e = symbol_ptr(&st.tiles, g_noalloc_tiles)) != cudaSuccess) return e;
  if ((e = symbol_ptr(&st.levels, g_noalloc_levels)) != cudaSuccess) return e;
  if ((e = symbol_ptr(&st.status, &g_noalloc_status)) != cudaSuccess) return e;
  if ((e = set_fwd_attributes()) != cudaSuccess) return e;

  std::vector<float2> tw13(1 << kTwLog), twlo(1 << kTwSplit), twhi(1 << (kTwBigLog - kTwSplit));
  for (int64_t k = 0; k < (int64_t)tw13.size(); ++k) tw13[k] = root(k, int64_t(1) << kTwLog);
  for (int64_t k = 0; k < (int64_t)twlo.size(); ++k) twlo[k] = root(k, int64_t(1) << kTwBigLog);
  for (int64_t k = 0; k < (int64_t)twhi.size(); ++k) twhi[k] = root(k << kTwSplit, int64_t(1) << kTwBigLog);

  std::vector<SigDesc> sigs(kMaxLogNA + 1);
  std::vector<int32_t> ids(kMaxLogNA + 1);
  std::vector<TileItem> tiles((kMaxLogNA + 1) * kMaxTileItems);
  std::vector<LevelItem> levels((kMaxLogNA + 1) * kMaxLevelItems);
  for (int m = 1; m <= kMaxLogNA; ++m) {
    sigs[m] = SigDesc{0, 0, 0, m, 0};  // one signal at offset 0, scratch at 0
    ids[m] = m;                         // sig_ids[m] -> descriptor m
    if (m >= 5) {
      const int tl = m < kTileLog ? m : kTileLog;
      const int nt = 1 << (m - tl);
      for (int t = 0; t < nt; ++t) tiles[m * kMaxTileItems + t] = TileItem{m, 1, (int16_t)tl, t, 0};
      st.ntile[m] = nt;
    }
    int off = 0;
    for (int i = kTileLog + 1; i <= m; ++i) {
      const int nw = 1 << (m - i);
      const int nblk = i <= kWinMaxLog + 1 ? 1 : pass_items(i);
      st.lvl_off[m][i] = m * kMaxLevelItems + off;
      for (int w = 0; w < nw; ++w)
        for (int b = 0; b < nblk; ++b) levels[m * kMaxLevelItems + off++] = LevelItem{m, w, b, 0};
      st.lvl_cnt[m][i] = nw * nblk;
    }
    if (off > kMaxLevelItems) return cudaErrorInvalidValue;
  }
  if ((e = cudaMemcpyToSymbol(g_noalloc_tw13, tw13.data(), tw13.size() * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(g_noalloc_twlo, twlo.data(), twlo.size() * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(g_noalloc_twhi, twhi.data(), twhi.size() * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(g_noalloc_sigs, sigs.data(), sigs.size() * sizeof(SigDesc))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(g_noalloc_ids, ids.data(), ids.size() * sizeof(int32_t))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(g_noalloc_tiles, tiles.data(), tiles.size() * sizeof(TileItem))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(g_noalloc_levels, levels.data(), levels.size() * sizeof(LevelItem))) != cudaSuccess)
    return e;
  const int zero = 0;
  if ((e = cudaMemcpyToSymbol(g_noalloc_status, &zero, sizeof(int))) != cudaSuccess) return e;
  st.ready = true;
  return cudaSuccess;
}

mrdft_status fail_na(mrdft_status s, const std::string& msg) {
  set_global_error("mrdft_forward_noalloc: " + msg);
  return s;
}

}  // namespace

// mrdft_status_poll(NULL): read and clear the device status word of the
// allocation-free entry point on the current device (MRDFT_OK when that entry
// point has not run there).  Waits for the device.
mrdft_status mrdft::noalloc_status_poll() {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(MRDFT_ECUDA, std::string("status poll: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(MRDFT_EUNSUPPORTED, "status poll: device index out of range");
  int* status = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev[dev].ready) return MRDFT_OK;
    status = g_dev[dev].status;
  }
  int v = 0;
  if ((e = cudaDeviceSynchronize()) == cudaSuccess && (e = cudaMemcpy(&v, status, sizeof(int), cudaMemcpyDeviceToHost)) == cudaSuccess)
    e = cudaMemset(status, 0, sizeof(int));
  if (e != cudaSuccess) return fail_na(MRDFT_ECUDA, std::string("status poll: ") + cudaGetErrorString(e));
  if (v == kStatusTimeout) return fail_na(MRDFT_ETIMEOUT, "a device-side wait gave up");
  if (v != 0) return fail_na(MRDFT_EDEVICE, "a kernel flagged an invalid work item (code " + std::to_string(v) + ")");
  return MRDFT_OK;
}

extern "C" mrdft_status mrdft_forward_noalloc(const void* x, void* y, int64_t n, mrdft_stream_t stream) {
  if (!x || !y) return fail_na(MRDFT_EINVAL, "x or y is NULL");
  if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) != 0)
    return fail_na(MRDFT_EINVAL, "x and y must be 16-byte aligned");
  if (n < 2 || (n & (n - 1)) != 0) return fail_na(MRDFT_EINVAL, "n must be a power of two >= 2");
  if (n > (int64_t(1) << kMaxLogNA))
    return fail_na(MRDFT_EINVAL, "n = " + std::to_string(n) + " exceeds the fixed scratch limit 2^" +
                                     std::to_string(kMaxLogNA) + " (use mrdft_plan / mrdft_forward)");
  int m = 0;
  while ((int64_t(1) << m) < n) ++m;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(MRDFT_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(MRDFT_EUNSUPPORTED, "device index out of range");
  DevState* st = &g_dev[dev];
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!st->ready) {
      e = setup(*st);
      if (e != cudaSuccess) return fail_na(MRDFT_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FwdArgs a{};
  a.x = x;
  a.in_real = 0;
  a.y = reinterpret_cast<float2*>(y);
  a.sigs = st->sigs;
  a.nsigs = kMaxLogNA + 1;
  a.nids = kMaxLogNA + 1;
  a.scratch = st->scratch;
  a.tw = Twiddles{st->tw13, st->twlo, st->twhi};
  a.status = st->status;
  if (m <= 4) {
    a.sig_ids = st->ids + m;
    a.nitems = 1;
    e = launch_fwd_tiny(a, 1, s);
    if (e != cudaSuccess) return fail_na(MRDFT_ECUDA, cudaGetErrorString(e));
    return MRDFT_OK;
  }
  a.sig_ids = st->ids;
  a.items = st->tiles + m * kMaxTileItems;
  a.nitems = st->ntile[m];
  e = launch_fwd_tile(a, st->ntile[m], s);
  for (int i = kTileLog + 1; i <= m && e == cudaSuccess; ++i) {
    a.level = i;
    a.items = st->levels + st->lvl_off[m][i];
    a.nitems = st->lvl_cnt[m][i];
    if (i <= kWinMaxLog + 1) {
      e = launch_fwd_window(a, a.nitems, s);
    } else {
      e = launch_fwd_cols(a, a.nitems, s);
      if (e == cudaSuccess) e = launch_fwd_rows(a, a.nitems, s);
    }
  }
  if (e != cudaSuccess) return fail_na(MRDFT_ECUDA, cudaGetErrorString(e));
  return MRDFT_OK;
}
