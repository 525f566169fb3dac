// Host/device shared descriptors of the MrDFT library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mrdft_common.cuh"

namespace mrdft {

// One signal of a plan.  Offsets count complex samples (complex64 input) or
// real samples (FP32 input) for x, complex values for y; N = 2^m.
struct SigDesc {
  int64_t in_off;   // first sample of the signal in x
  int64_t out_off;  // first output of level 1 in y; level i at out_off + (i-1) N
  int64_t aux_off;  // first element of the signal in the per-signal scratch (N/2 per signal of m > 12)
  int32_t m;        // log2 N
  int32_t pad;
};

// In-tile work item: levels 1..tlog of `nsig` signals listed at
// sig_ids[sig_list ..] (each of length 2^tlog when nsig > 1), or of the
// samples [tile * 2^tlog, (tile + 1) * 2^tlog) of one longer signal.
struct TileItem {
  int32_t sig_list;
  int16_t nsig;
  int16_t tlog;
  int32_t tile;
  int32_t pad;
};

// Large-level work item: signal, window at level `level`, and a block index
// inside the window (column block or bin block for the two-pass levels).
struct LevelItem {
  int32_t sig;
  int32_t window;
  int32_t block;
  int32_t pad;
};

constexpr int kTileLog = 12;                 // in-tile levels 1..12
constexpr int kTile = 1 << kTileLog;         // 4096 samples per tile
constexpr int kTileThreads = 256;            // 16 samples per thread, 2 CTAs per SM
constexpr int kWinMaxLog = 13;               // one CTA FFT holds up to 2^13 points
constexpr int kWinThreads = 256;             // levels 13, 14: 16 or 32 points per thread
// Two-pass levels (i >= 15), h = 2^(i-1) = Q * C with C = 2^max(i - 12, cb_min),
//   so that Q <= 2^11 and every cols CTA reads chunks of at least 4
//   consecutive samples; cb_min is 9 for the forward and 10 for the adjoint
//   (FwdArgs / AdjArgs.cb_min; both directions accept 9 and 10, the forward
//   also 11).
//   cols pass: 2^12 or 2^13 points per CTA (RC chunk offsets x Q)
//   rows pass: 2^E points per CTA (KC = 2^E / C residues), E = rows_elems_log_c.
constexpr int kPassElemsLog = 13;
constexpr int kPassThreads = 256;        // 2^13-point rows / adjoint cols CTAs
constexpr int kColsThreads = 512;        // forward cols and 2^12-point adjoint rows CTAs (64 registers)
constexpr int kPassThreadsWide = 512;    // 2^14-point rows CTAs (levels 24 and 26)
// rows CTA size: 2^13 points (2^14 for C = 2^14); for the adjoint's C <= 2^10
// it gives the 2^12-point CTAs taken when AdjArgs.rows13 = 0 (2^13 otherwise)
__host__ __device__ constexpr int rows_elems_log_c(int cb, bool adj) {
  return (adj && cb <= 10) ? 12 : (cb > 13 ? cb : 13);
}
// work items of a two-pass level, per window: one per cols CTA (2^(i-14));
// a rows CTA of 2^E points takes 2^(E-13) items (E >= 13) or half an item
__host__ __device__ constexpr int pass_items(int i) { return 1 << ((i - 1) - kPassElemsLog); }

struct FwdArgs {
  const void* x;  // float2* (complex64) or float* (real FP32)
  int in_real;
  float2* y;
  const SigDesc* sigs;
  int nsigs;          // descriptors in sigs (work items are checked against it)
  int nids;           // entries in sig_ids
  const int32_t* sig_ids;
  const void* items;  // TileItem* or LevelItem*
  int nitems;
  int level;          // large-level kernels: level i being built
  float2* scratch;    // two-pass levels: intermediate, N/2 per signal
  float2* scratch2;   // dual-level cols: the upper level's intermediate
  int cb_min;         // two-pass levels: C = 2^max(i - 12, cb_min), cb_min 9..11 (0 means 10)
  int rows14;         // C = 2^12 rows CTAs of 2^14 points (4 residues, 1 per SM) instead of 2^13
  int rows_pf;        // rows CTAs that copy the children into shared memory when they start
  int rows12;         // C = 2^9 rows CTAs of 2^12 points (256 threads) instead of 2^13
  int tile_lean;      // tile CTAs in the 3-per-SM shape (work area aliasing the level buffer)
  int f_late;         // cols: the intermediate is read long after (stored evict-first in L2, not evict-last)
  Twiddles tw;
  int* status;
};

struct AdjArgs {
  const float2* gy;   // upstream gradient, same layout as y
  float2* gx;         // complex64 gradient of x
  const SigDesc* sigs;
  int nsigs;          // descriptors in sigs (work items are checked against it)
  int nids;           // entries in sig_ids
  const int32_t* sig_ids;
  const void* items;
  int nitems;
  int level;
  const float2* e_in;  // even-bin propagation from level+1 (N/2 per signal)
  float2* e_out;       // even-bin propagation to level-1 (N/2 per signal)
  float2* acc;         // x_bar contributions of the large levels (N per signal of m > 12, at 2 aux_off)
  float2* scratch;     // two-pass levels intermediate (N/2 per signal)
  float2* scratch2;    // dual-level cols: the upper level's intermediate
  int rows13;          // C = 2^10 rows CTAs of 2^13 points (8 residues) instead of 2^12
  int cb_min;          // two-pass levels: C = 2^max(i - 12, cb_min), cb_min 9 or 10 (0 means 10)
  int first;           // 1 when this is the top level (no e_in, acc written not added)
  Twiddles tw;
  int* status;
  // fused loss gradient: when t != nullptr, gy holds the forward output Y and
  // the upstream gradient of level i is 2^(1-i) (Y - T); sum_i 2^-i |Y - T|^2
  // is added to *loss (which may be nullptr)
  const float2* t;
  double* loss;
  // lone small signal (launch_adj_levels): the CTAs' finish counter, zero
  // between launches
  int* ticket;
};

// ---- work-item checks
// Kernels check every work item against the signal descriptors before using
// it; an item that does not describe a part of a planned signal (a work list
// damaged in device memory) raises kStatusBadItem in the status word and the
// block skips it, so that no access leaves the plan's buffers.
__device__ __forceinline__ bool level_item_ok(const SigDesc* sigs, int nsigs, const LevelItem& it, int level,
                                              int nblk, SigDesc& sd) {
  if (it.sig < 0 || it.sig >= nsigs) return false;
  sd = sigs[it.sig];
  if (sd.m < level || sd.m > 26 || level < 1) return false;
  if (it.window < 0 || (int64_t)it.window >= ((int64_t)1 << (sd.m - level))) return false;
  return it.block >= 0 && it.block < nblk;
}
// the header of a tile item (before any signal of it is read)
__device__ __forceinline__ bool tile_item_head_ok(const TileItem& it, int nids, int tile_log) {
  const int n = it.nsig;
  if (n < 1 || (n & (n - 1)) != 0 || it.tlog < 5 || it.tlog > tile_log) return false;
  if (((int64_t)n << it.tlog) > ((int64_t)1 << tile_log)) return false;
  if (it.tile < 0 || (n > 1 && it.tile != 0)) return false;
  return it.sig_list >= 0 && (int64_t)it.sig_list + n <= nids;
}
// one signal of a tile item: a whole signal of 2^tlog when packed, else a
// signal long enough to hold tile `tile`
__device__ __forceinline__ bool tile_sig_ok(const SigDesc* sigs, int nsigs, int id, const TileItem& it,
                                            SigDesc& sd) {
  if (id < 0 || id >= nsigs) return false;
  sd = sigs[id];
  if (sd.m > 26) return false;
  if (it.nsig > 1) return sd.m == it.tlog;
  return sd.m >= it.tlog && ((int64_t)(it.tile + 1) << it.tlog) <= ((int64_t)1 << sd.m);
}

// launchers (defined in the .cu files)
cudaError_t launch_fwd_tile(const FwdArgs& a, int grid, cudaStream_t s);
cudaError_t launch_fwd_tiny(const FwdArgs& a, int nsig_tiny, cudaStream_t s);
// one signal of 2^5 .. 2^12 samples alone in its plan: one CTA per level (grid m)
cudaError_t launch_fwd_levels(const FwdArgs& a, int m, cudaStream_t s);
cudaError_t launch_fwd_window(const FwdArgs& a, int grid, cudaStream_t s);
cudaError_t launch_fwd_cols(const FwdArgs& a, int grid, cudaStream_t s);
// cols passes of levels a.level - 1 and a.level in one read of x; grid =
// level-a.level items; both levels with the same C, Q of the lower in [2^3, 2^9]
cudaError_t launch_fwd_cols2(const FwdArgs& a, int grid, cudaStream_t s);
bool fwd_cols2_pairable(int upper_level, int cb_min);
cudaError_t launch_fwd_rows(const FwdArgs& a, int grid, cudaStream_t s);

// bit-reversed output layout (MRDFT_FLAG_BITREV), in place after the forward:
// items {sig, block, level} for levels <= 12, {sig, window, level} above
cudaError_t launch_bitrev_small(const FwdArgs& a, int grid, cudaStream_t s);
cudaError_t launch_bitrev_big(const FwdArgs& a, int grid, int level, cudaStream_t s);

cudaError_t launch_adj_tile(const AdjArgs& a, int grid, cudaStream_t s);
cudaError_t launch_adj_tiny(const AdjArgs& a, int nsig_tiny, cudaStream_t s);
// one signal of 2^5 .. 2^12 samples alone in its plan, no fused loss: one CTA
// per level (grid m), each level's x_bar share in a.scratch (m N), summed by
// the CTA that finishes last
cudaError_t launch_adj_levels(const AdjArgs& a, int m, cudaStream_t s);
cudaError_t launch_adj_window(const AdjArgs& a, int grid, cudaStream_t s);
cudaError_t launch_adj_rows(const AdjArgs& a, int grid, cudaStream_t s);
cudaError_t launch_adj_cols(const AdjArgs& a, int grid, cudaStream_t s);
// cols passes of levels a.level - 1 and a.level after both rows passes, one
// update of acc; grid = level-a.level items; both levels with the same C,
// Q of the lower in [2^4, 2^9]
cudaError_t launch_adj_cols2(const AdjArgs& a, int grid, cudaStream_t s);
bool adj_cols2_pairable(int upper_level, int cb_min);

cudaError_t set_kernel_attributes();

}  // namespace mrdft
