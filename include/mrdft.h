/*
 * mrdft.h -- C ABI of the GB300 (sm_103a) multiresolution DFT library.
 *
 * The transform (Andreatto & Cariow, "An algorithm for fast computation of
 * the multiresolution discrete Fourier transform", arXiv:1507.02525):
 * Sec. 2, Eq. 1 -- for a signal x of length N = 2^m (m >= 1) and every level
 * i = 1..m, the unnormalised spectra of the N/2^i non-overlapping rectangular
 * windows of length 2^i:
 *
 *     Y^(i)[w 2^i + k] = sum_{n=0}^{2^i - 1} x[w 2^i + n] exp(-j 2 pi n k / 2^i)
 *
 * computed with the level recursion of Sec. 3 (Eq. 4: even bins are the sum of
 * the two child spectra, odd bins a DFT of the twiddled half-difference).
 * Output order: levels ascending, windows ascending, bins natural (the
 * permutation Gamma of Sec. 3 applied).  Complex values are complex64:
 * interleaved (re, im) IEEE single precision.
 *
 * Layout of a plan's data (a batch of S signals, lengths N_s = 2^{m_s}):
 *   x : signals concatenated, signal s starting at sample sum_{t<s} N_t;
 *       complex64 (MRDFT_C64) or float32 (MRDFT_R32, promoted to complex
 *       with zero imaginary part).
 *   y : complex64, signal s starting at sum_{t<s} m_t N_t; inside a signal
 *       level i (1-based) occupies [ (i-1) N_s, i N_s ).
 *   gy: same layout as y.   gx: complex64, same layout as x.
 * All buffers are DEVICE pointers, owned by the caller, 16-byte aligned, and
 * must not alias one another.  Work is asynchronous on the given stream.
 *
 * Errors: every call returns an mrdft_status; nothing throws across the ABI.
 * A failed call leaves a message retrievable with mrdft_last_error().
 * Every kernel checks each work item it is given against the plan's signal
 * descriptors before touching memory; an item that does not describe part of
 * a planned signal (a work list damaged in device memory) is skipped and
 * raises MRDFT_EDEVICE in a device status word that mrdft_status_poll()
 * reads back.  No kernel waits on a flag or on another kernel.
 */
#ifndef MRDFT_H_
#define MRDFT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrdft_plan_s* mrdft_plan_t;
typedef struct CUstream_st* mrdft_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  MRDFT_OK = 0,
  MRDFT_EINVAL = 1,       /* bad argument: length not a power of two, null pointer, ... */
  MRDFT_ENOMEM = 2,       /* device or host allocation failed */
  MRDFT_ECUDA = 3,        /* a CUDA runtime call failed (message in mrdft_last_error) */
  MRDFT_EUNSUPPORTED = 4, /* valid request the library does not implement */
  MRDFT_ETIMEOUT = 5,     /* a device-side wait gave up (reserved: no kernel waits on a flag) */
  MRDFT_EDEVICE = 6       /* a kernel flagged an invalid work item (mrdft_status_poll) */
} mrdft_status;

typedef enum {
  MRDFT_C64 = 0, /* complex64 input */
  MRDFT_R32 = 1  /* real float32 input, complex64 output */
} mrdft_dtype;

/* Plan flags. */
#define MRDFT_FLAG_GRAPH 1u /* replay a CUDA graph of the launch sequence (captured
                               on the first call for each (input, output) pair) */
/* MRDFT_FLAG_BITREV: mrdft_forward stores every window in the order of the
 * paper's Sec. 3 before the permutation Gamma: position p of a window of
 * level i holds bin bitrev_i(p) (y_window = T_{2^i} Y_window, T the bit
 * reversal over i bits).  The bins are computed in natural order and each
 * window is then permuted in place (a read and a write of y), so this layout
 * costs more than the natural one.  Forward only: mrdft_adjoint and
 * mrdft_loss_grad return MRDFT_EUNSUPPORTED on such plans. */
#define MRDFT_FLAG_BITREV 2u

/*
 * mrdft_plan -- validate the signal lengths and allocate everything a
 * transform needs on the current CUDA device: twiddle tables (FP64 values
 * rounded once to FP32), work lists, scratch.
 *   out       : receives the plan (set to NULL on failure).
 *   lengths   : host array of n_lengths signal lengths; each a power of two
 *               in [2, 2^26] (m in 1..26).
 *   n_lengths : 1 -> `batch` signals of length lengths[0] (uniform batch);
 *               == batch -> one length per signal (ragged batch).
 *   batch     : number of signals, >= 1.
 *   dtype     : MRDFT_C64 or MRDFT_R32 input.
 *   flags     : MRDFT_FLAG_* bits.
 * Returns MRDFT_EINVAL for a bad length or count, MRDFT_ENOMEM / MRDFT_ECUDA
 * when allocation fails.  The plan is bound to the device current at the
 * call; it may be used from one stream at a time.  The execution shape and
 * kernel variants take the library defaults (see mrdft_plan_ex); the
 * environment variables MRDFT_SEG_LOG and MRDFT_STREAMS override the default
 * segment size and stream count (speed only, never the result).
 */
mrdft_status mrdft_plan(mrdft_plan_t* out, const int64_t* lengths, int64_t n_lengths,
                        int64_t batch, int dtype, uint32_t flags);

/*
 * mrdft_plan_opts -- mrdft_plan with the execution shape chosen explicitly
 * (no effect on the result, only on speed): signals are cut into segments of
 * at most 2^seg_log samples whose level chains run concurrently on `streams`
 * worker streams, so that a segment's levels find their children in L2.
 * seg_log = 0 or streams = 0 keep the default (2^23, 4 streams; the
 * environment variables MRDFT_SEG_LOG / MRDFT_STREAMS override a default).
 * EINVAL unless seg_log is 0 or in [12, 26] and streams in [0, 16].  The
 * autotuner of the Python package times candidates through this call.
 */
mrdft_status mrdft_plan_opts(mrdft_plan_t* out, const int64_t* lengths, int64_t n_lengths, int64_t batch,
                             int dtype, uint32_t flags, int32_t seg_log, int32_t streams);

/*
 * Execution options of a plan.  None of them changes the result (every
 * variant computes Eq. 1 with the same recursion, only the launch shapes
 * differ); they change the speed, and the autotuner of the Python package
 * times candidates through mrdft_plan_ex.  A field left at 0 takes the
 * library default; switches take MRDFT_OPT_OFF or MRDFT_OPT_ON.
 *   seg_log  : segments of at most 2^seg_log samples, 12..26 (default 23)
 *   streams  : worker streams the segment chains run on, 1..16 (default 4)
 *   fwd_cb   : forward two-pass split h = Q C, C = 2^max(i - 12, fwd_cb), 9..11 (default 9)
 *   adj_cb   : adjoint two-pass split, 9..10 (default 10)
 *   fwd_rows_prefetch : forward rows CTAs copy the children spectra into
 *              shared memory when they start (default off)
 *   fwd_rows14 : with prefetch off, C = 2^12 forward rows CTAs of 2^14
 *              points instead of 2^13 (default on)
 *   adj_rows13 : adjoint C = 2^10 rows CTAs of 2^13 points instead of 2^12 (default on)
 *   dual_cols : consecutive two-pass levels of a chain share one cols pass (default on)
 *   fwd_tree : the forward runs each window of a level above the segment
 *              size as soon as its two children are done; off (default):
 *              those levels run level by level after every segment
 *   tile_first : the in-tile levels of every segment run as one launch,
 *              before the segments (forward) or after them (adjoint),
 *              instead of one launch per segment (default on)
 *   tile_lean : forward tile CTAs that fit three to an SM (the FFT work
 *              area shares the level buffer, twiddles read through L1)
 *              instead of two (default on)
 *   fwd_rows12 : forward C = 2^9 rows CTAs of 2^12 points (256 threads, up
 *              to four per SM) instead of 2^13 (512 threads) (default off)
 *   tile_split : with tile_first, the in-tile levels run as this many launches
 *              over consecutive groups of segments, 1..64 (default 1): each
 *              group's segments start (forward) as soon as its own tiles are
 *              done, while the next group's tiles run; in the adjoint a
 *              group's tiles start as soon as its segments are done
 *   top_cols_early : the forward runs the cols passes of the levels above
 *              the segment size on a stream of their own while the segments
 *              run (they read only x), each into its own scratch (N/2 complex
 *              per signal and level); their rows passes stay at the end
 *              (default off)
 *   top_overlap : the forward runs the cols passes of the levels above the
 *              segment size on a stream of their own (from the end of the
 *              segments, or from the start with top_cols_early), each into
 *              its own scratch, and each level's rows pass waits only for
 *              its own cols pass: the cols pass of a level overlaps the rows
 *              pass of the level below (default off)
 *   levels_parallel : a plan of ONE signal of 2^5..2^12 samples computes
 *              each level from x in a CTA of its own (both halves of every
 *              window by FFT), all levels at once, instead of the in-tile
 *              recursion, whose chain of dependent levels sets the latency of
 *              a signal this small; its adjoint (without the fused loss) takes
 *              each level's share of x_bar in a CTA of its own and adds them
 *              in level order (default on)
 */
#define MRDFT_OPT_DEFAULT 0
#define MRDFT_OPT_OFF 1
#define MRDFT_OPT_ON 2
typedef struct {
  int32_t seg_log;
  int32_t streams;
  int32_t fwd_cb;
  int32_t adj_cb;
  int32_t fwd_rows_prefetch;
  int32_t fwd_rows14;
  int32_t adj_rows13;
  int32_t dual_cols;
  int32_t fwd_tree;
  int32_t tile_first;
  int32_t tile_lean;
  int32_t fwd_rows12;
  int32_t tile_split;
  int32_t top_cols_early;
  int32_t top_overlap;
  int32_t levels_parallel;
} mrdft_exec_opts;

/*
 * mrdft_plan_ex -- mrdft_plan with execution options (NULL: all defaults).
 * MRDFT_EINVAL for a field out of its range, otherwise as mrdft_plan.
 */
mrdft_status mrdft_plan_ex(mrdft_plan_t* out, const int64_t* lengths, int64_t n_lengths, int64_t batch,
                           int dtype, uint32_t flags, const mrdft_exec_opts* opts);

/* The execution options a plan runs with (every field filled in). */
mrdft_status mrdft_plan_get_opts(mrdft_plan_t plan, mrdft_exec_opts* opts);

/* Total complex outputs of the plan, sum_s m_s N_s (the length of y and gy). */
mrdft_status mrdft_output_elems(mrdft_plan_t plan, int64_t* elems);

/* Total input samples of the plan, sum_s N_s (the length of x and gx). */
mrdft_status mrdft_input_elems(mrdft_plan_t plan, int64_t* elems);

/*
 * mrdft_forward -- Eq. 1 for every signal of the plan (Sec. 3 recursion).
 *   x : device input (layout above), y : device output, stream : CUDA stream.
 * Asynchronous; returns MRDFT_EINVAL for null or misaligned pointers.
 */
mrdft_status mrdft_forward(mrdft_plan_t plan, const void* x, void* y, mrdft_stream_t stream);

/*
 * mrdft_adjoint -- the conjugate transpose of Eq. 1,
 *   gx = sum_i (I_{N/2^i} (x) E_{2^i})^H gy_i   (unnormalised inverse DFT per
 * window, summed over levels), the reverse of the Sec. 3 recursion.
 *   gy : device complex64 gradient with the layout of y;
 *   gx : device complex64 result with the layout of x (for MRDFT_R32 plans the
 *        gradient with respect to the real input is Re(gx)).
 */
mrdft_status mrdft_adjoint(mrdft_plan_t plan, const void* gy, void* gx, mrdft_stream_t stream);

/*
 * mrdft_forward_host -- the same transform for HOST buffers: copies x to the
 * plan's device staging buffers on `stream`, runs mrdft_forward, copies y
 * back and synchronises the stream.  x and y are host pointers (pinned
 * memory gives full copy bandwidth).  Parts of y that are final early (the
 * in-tile levels, then the levels inside the segments) start their copy to
 * the host while the rest is computed, on a copy stream of the plan joined
 * back to `stream` (up to 64 copies per call; otherwise, and with
 * MRDFT_FLAG_BITREV, one copy at the end).  This entry point never replays a
 * graph.  The first call allocates the staging buffers (MRDFT_ENOMEM on
 * failure).  y must not be read before the call returns.
 */
mrdft_status mrdft_forward_host(mrdft_plan_t plan, const void* x_host, void* y_host,
                                mrdft_stream_t stream);

/* Read and clear the plan's device status word; waits for the device.
 * Returns MRDFT_EDEVICE when a kernel skipped an invalid work item since the
 * last poll.  plan == NULL polls the status word of mrdft_forward_noalloc on
 * the current device instead (MRDFT_OK if that entry point has not run on
 * it; its error message is then read with mrdft_last_error(NULL)). */
mrdft_status mrdft_status_poll(mrdft_plan_t plan);

/* Message of the last failed call on this plan (or of the last failed
 * mrdft_plan when plan is NULL).  Never NULL. */
const char* mrdft_last_error(mrdft_plan_t plan);

/* Launch configuration the plan picked: tile log2 size and the number of
 * kernel launches one forward / adjoint issues. */
mrdft_status mrdft_plan_info(mrdft_plan_t plan, int32_t* tile_log, int32_t* fwd_launches,
                             int32_t* adj_launches);

/* Kernel kinds for per-kernel timing. */
enum {
  MRDFT_KIND_FWD_TILE = 0,   /* levels 1..12 of 4096-sample tiles (1..m for shorter signals) */
  MRDFT_KIND_FWD_TINY = 1,   /* signals of length <= 16 */
  MRDFT_KIND_FWD_WINDOW = 2, /* level 13 or 14, one window per CTA */
  MRDFT_KIND_FWD_COLS = 3,   /* two-pass levels, cross-chunk pass (one launch may serve two levels) */
  MRDFT_KIND_FWD_ROWS = 4,   /* two-pass levels, per-residue pass + even bins */
  MRDFT_KIND_ADJ_TILE = 5,
  MRDFT_KIND_ADJ_TINY = 6,
  MRDFT_KIND_ADJ_WINDOW = 7,
  MRDFT_KIND_ADJ_ROWS = 8,
  MRDFT_KIND_ADJ_COLS = 9,
  MRDFT_KIND_COUNT = 10
};

/*
 * mrdft_timing_enable -- when enable != 0, every later kernel launch of this
 * plan is bracketed by CUDA events recorded on its launch stream (graph replay
 * is bypassed meanwhile); enable == 2 also issues every launch on the
 * caller's stream, one after another, so that each bracketed launch has the
 * GPU to itself (per-kernel rooflines); resets the accumulated counters
 * either way.
 * mrdft_timing_read -- waits for the recorded events and returns, for one
 * kernel kind, the summed device milliseconds, the number of launches and the
 * summed algorithmic bytes of those launches (input read once plus the
 * outputs the kernel writes; zero for pure intermediate passes) since the
 * last enable.  Any output pointer may be NULL.
 */
mrdft_status mrdft_timing_enable(mrdft_plan_t plan, int enable);
mrdft_status mrdft_timing_read(mrdft_plan_t plan, int kind, double* ms, int64_t* launches,
                               int64_t* bytes);

/*
 * mrdft_loss_grad -- one fused loss-and-gradient step for fitting the
 * multiresolution spectra to targets T (same layout and type as y):
 *     L = sum_i 2^-i || Y^(i) - T^(i) ||^2,   Y = MrDFT(x)  (Sec. 2, Eq. 1),
 *     gx = dL/dx* = adjoint(g),  g^(i) = 2^(1-i) (Y^(i) - T^(i)),
 * where the adjoint is the conjugate transpose of Eq. 1 (as mrdft_adjoint).
 * Writes Y to y, the gradient to gx (complex64; for MRDFT_R32 plans the
 * gradient with respect to the real input is Re(gx)) and, when loss is not
 * NULL, L to the device double *loss.  The adjoint reads Y and T directly:
 * g is never materialised.  All pointers are device pointers owned by the
 * caller (x, t, y, gx 16-byte aligned, loss 8-byte aligned); asynchronous on
 * the stream.  The loss is summed with device atomics, so its last bits may
 * differ between calls; Y and gx are deterministic.
 */
mrdft_status mrdft_loss_grad(mrdft_plan_t plan, const void* x, const void* t, void* y, void* gx, double* loss,
                             mrdft_stream_t stream);

/*
 * mrdft_forward_noalloc -- forward MrDFT of ONE complex64 signal of length n
 * (a power of two, 2 <= n <= 2^MRDFT_NOALLOC_MAX_LOG) without any plan and
 * without allocating: the paper has no counterpart; this entry point exists
 * for callers that must not call cudaMalloc -- code that runs under an
 * external memory manager owning every device allocation, or inside a loop
 * where an allocation's implicit device synchronisation is not acceptable.
 *   x : device input, n complex64;  y : device output, log2(n) * n complex64
 *       (levels ascending, as for mrdft_forward);  stream : CUDA stream.
 * The intermediate of the two-pass levels (15 and 16) lives in a fixed
 * device array of 2^(MRDFT_NOALLOC_MAX_LOG - 1) complex64 (256 KiB), which
 * every GPU that loads this library keeps until the process exits, next to
 * the twiddle tables and work lists (about 350 KiB in all).  The first call
 * on a device sets that storage up (symbol addresses, tables copied from the
 * host) and synchronises with the device; make that first call before any
 * stream capture.  Every call shares the same storage, so calls whose work
 * overlaps on the GPU (different streams, or different host threads) race
 * and give wrong results; calls on one stream are ordered and safe.  Sizes
 * above the limit return MRDFT_EINVAL with a message (mrdft_last_error(NULL)).
 */
#define MRDFT_NOALLOC_MAX_LOG 16
mrdft_status mrdft_forward_noalloc(const void* x, void* y, int64_t n, mrdft_stream_t stream);

/*
 * mrdft_plan_graph_stats -- graph replay bookkeeping of a MRDFT_FLAG_GRAPH
 * plan: `cached` executable graphs held (at most 4 per direction; a new
 * (buffers, stream) combination past that re-targets the least recently
 * used one with cudaGraphExecUpdate), `captures` stream captures made and
 * `updates` of them that re-targeted an existing graph instead of
 * instantiating a new one.  Any output pointer may be NULL.
 */
mrdft_status mrdft_plan_graph_stats(mrdft_plan_t plan, int32_t* cached, int64_t* captures, int64_t* updates);

/*
 * mrdft_debug_item -- test hook of the device-side work-item checks: reads
 * (old_fields, may be NULL) and optionally overwrites (new_fields, may be
 * NULL) work item `index` of the plan's tile list (list 0) or level list
 * (list 1), four 32-bit words each, synchronously.  Level items are
 * {signal, window, block, 0}; tile items {signal-list offset,
 * count | (log2 tile length << 16), tile index, 0}.  MRDFT_EINVAL for an
 * index past the end of the list.  A kernel given an item that does not fit
 * its signal skips it and mrdft_status_poll() then returns MRDFT_EDEVICE.
 */
mrdft_status mrdft_debug_item(mrdft_plan_t plan, int list, int64_t index, const int32_t* new_fields,
                              int32_t* old_fields);

/* Release everything the plan owns.  NULL is ignored. */
void mrdft_destroy(mrdft_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* MRDFT_H_ */
