// Internal declarations shared by the FTP CUDA translation units.
// Everything here is device-side plumbing for the C ABI in include/ftp.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ftp {

// Device status word codes (mirror ftp_status values).
enum : int {
  DEV_OK = 0,
  DEV_INVALID = 1,
  DEV_ZERO_VARIANCE = 2,
  DEV_MIXED_ZERO_SIGMA = 3,
  DEV_NONFINITE = 4,
  DEV_TIMEOUT = 7,
};

// Layout of the device status block (ints).
enum : int { ST_CODE = 0, ST_DBG_SITE = 4, ST_DBG_A = 5, ST_DBG_B = 6, ST_DBG_N = 7, ST_WORDS = 8 };

// Self-checking builds (-DFTP_DEVICE_CHECKS): an index or alignment check
// that fails records (site, value, bound) in the status block once and the
// guarded access is skipped.  Release builds compile the checks away.
#ifdef FTP_DEVICE_CHECKS
#define FTP_DCHECK(status, cond, site, val, bound)                         \
  ((cond) ? true                                                           \
          : (atomicAdd(&(status)[ST_DBG_N], 1) == 0                        \
                 ? ((status)[ST_DBG_SITE] = (site), (status)[ST_DBG_A] = (int)(val), \
                    (status)[ST_DBG_B] = (int)(bound), false)              \
                 : false))
#else
#define FTP_DCHECK(status, cond, site, val, bound) true
#endif
// Solver counters of a call: iterations and items of the main pass, items
// that hit the Aberth cap there, frequencies put on the re-solve list (and
// how many of them for an item that hit the cap), and items still at the cap
// after a re-solve pass or in a call that cannot re-solve.
enum : int {
  CNT_ITERS = 0,
  CNT_ITEMS = 1,
  CNT_NONCONV = 2,
  CNT_REDO = 3,
  CNT_REDO_NC = 4,
  CNT_NC_FINAL = 5,
  CNT_WORDS = 6
};

// Re-solve marks (one int per frequency): listed, list full (the frequency
// keeps its first result), listed because an item hit the main pass's
// iteration cap, and still at the cap after the FP32 re-solve (then re-solved
// once more with FP64 Aberth iterations).
enum : int { MARK_LISTED = 1, MARK_OVERFLOW = 2, MARK_CAP = 4, MARK_FP64 = 8 };

// Default polls of a bounded mbarrier wait in the roots kernels.
constexpr int kWaitPolls = 1 << 20;

// Layout of the device moments block (doubles).
enum : int { MO_YBAR = 0, MO_YY = 1, MO_WSUM = 2, MO_UNIT = 3, MO_WORDS = 4 };

constexpr int kSpreadTile = 2048;       // grid cells owned by one spreading CTA
constexpr int kSpreadTileShift = 11;
constexpr int kMaxH = 16;

// Bound on the absolute error of one NFFT sum Z_h (relative to sum w = 1),
// used by the a-posteriori error estimate of P, and the estimated error of P
// above which a frequency is re-solved from direct FP64 sums: FP32 NFFT
// (mixed path, m = 5, sigma = 1.25: measured at most 5.0e-7 against direct
// FP64 sums on the long, bank and survey lightcurves; twice that here) and
// FP64 NFFT (FP64 path).
constexpr double kSumErrF32 = 1e-6;
// The estimate is an upper bound of |dP| for sums within that error; a
// quarter of the 1e-4 tolerance of the mixed path leaves a 4x margin.
constexpr double kRedoTolF32 = 2.5e-5;
constexpr double kSumErrF64 = 2e-13;
constexpr double kRedoTolF64 = 1e-10;

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

// ------------------------------------------------------------------ launches
// Step (a): observation preparation, binning, spreading, FFT (host), gather.
// Moments use a small scratch block (partials of at most kMomentBlocks CTAs
// and an atomic ticket that must be zero before the first use).
constexpr int kMomentBlocks = 304;
constexpr size_t kMomentScratchBytes = 64 * kMomentBlocks + 16;
void launch_moments(const double* t, const double* y, const double* dy, int64_t n,
                    double* moments, int* status, void* scratch, cudaStream_t s);

template <typename R>
void launch_points(const double* t, const double* y, const double* dy, int64_t n,
                   const double* moments, const int* status, double df, int64_t ngrid,
                   int* tile_count, int* cell, R* frac, typename C2<R>::type* coef,
                   cudaStream_t s);

void launch_scan(const int* tile_count, int64_t ntiles, int* tile_off, int* cursor,
                 const int* status, cudaStream_t s);

template <typename R>
void launch_scatter(int64_t n, const int* tile_off, int* cursor, const int* cell, const R* frac,
                    const typename C2<R>::type* coef, int* cell_s, R* frac_s,
                    typename C2<R>::type* coef_s, const int* status, cudaStream_t s);

template <typename R>
void launch_spread(const int* tile_off, const int* cell_s, const R* frac_s,
                   const typename C2<R>::type* coef_s, int64_t ngrid, int64_t ntiles, int m,
                   double beta, typename C2<R>::type* grid, const int* status, cudaStream_t s);

template <typename R>
void launch_gather(const typename C2<R>::type* X, int64_t ngrid, int64_t k0, int64_t nf,
                   int64_t nf_pad, int Hs, int m, double beta, typename C2<R>::type* sums,
                   const int* status, cudaStream_t s);

// One curve of a batched step (a): its observations in spreading-tile order,
// its NFFT grid (inside a batch's grid buffer) and its sum rows.
struct StepACurve {
  const int* tile_off;  // ntiles + 1 offsets into cell_s / frac_s / coef_s
  const int* cell_s;
  const void* frac_s;   // R[n]
  const void* coef_s;   // C2<R>[n]
  void* grid;           // C2<R>[ngrid]
  void* sums;           // C2<R>[3 Hs][nf_pad]
  int64_t ngrid, ntiles, k0, nf, nf_pad;
  int32_t Hs, pad_;
};
static_assert(sizeof(StepACurve) == 96, "StepACurve layout");

// Spreading and gather of `ncurves` curves in one launch each: spread
// tile t of the list belongs to the curve c with spread_prefix[c] <= t <
// spread_prefix[c + 1] (likewise the gather tiles); the prefixes have
// ncurves + 1 entries, the last being the total.
template <typename R>
void launch_spread_batch(const StepACurve* curves, const int64_t* spread_prefix, int ncurves,
                         int64_t total_tiles, int m, double beta, const int* status,
                         cudaStream_t s);
template <typename R>
void launch_gather_batch(const StepACurve* curves, const int64_t* gather_prefix, int ncurves,
                         int64_t total_tiles, int m, double beta, const int* status,
                         cudaStream_t s);
// Gather tiles of one curve (host side sizing of the work lists).
int64_t gather_tile_count(bool fp64, int64_t k0, int64_t nf, int Hs);

void launch_direct_sums(const double* t, const double* y, const double* dy, int64_t n,
                        const double* moments, const int* status, double df, int64_t k0,
                        const int* list, const int* count, int cap, int Hs, int64_t nf_pad,
                        double2* sums, int64_t sums_elems, int* status_rw, cudaStream_t s);

// One lightcurve of a batch, as the batched re-solve pass sees it.  Curves
// are listed in increasing redo_base (the global index of their frequency
// k = 0 in the batch's re-solve marks).
struct CurveDesc {
  const double* t;
  const double* y;
  const double* dy;
  int64_t n;
  double df;
  int64_t k0;
  int64_t redo_base;
  int64_t nf;
  int64_t out_off;  // element offset of the curve's output block [nrows][nf]
  int32_t Hs;
  int32_t nrows;
};
static_assert(sizeof(CurveDesc) == 80, "CurveDesc layout");

// One curve of a batched step (a) preparation: its observations, NFFT grid,
// and where its per-observation and per-tile scratch starts in the chunk's
// arrays (obs_base + i, tile_base + tile).
struct PrepCurve {
  const double* t;
  const double* y;
  const double* dy;
  int64_t n;
  double df;
  int64_t ngrid;
  int64_t ntiles;
  int64_t obs_base;
  int64_t tile_base;  // tile_off needs ntiles + 1 entries from here
};

// Step (a) preparation of `ncurves` curves in one launch (one CTA per curve):
// moments into moments[c * MO_WORDS ..], then the curve's observations in
// spreading-tile order (cell_s, frac_s, coef_s from obs_base) and the tile
// offsets relative to obs_base (tile_off from tile_base).  cell/frac/coef and
// tile_cnt are scratch of the same sizes.
template <typename R>
void launch_prep_batch(const PrepCurve* curves, int ncurves, double* moments, int* tile_cnt,
                       int* tile_off, int* cell, R* frac, typename C2<R>::type* coef, int* cell_s,
                       R* frac_s, typename C2<R>::type* coef_s, int* status, cudaStream_t s);
// The same for one curve (descriptor by value, obs_base = tile_base = 0);
// used for short curves, where one CTA beats six launches.
constexpr int64_t kPrepOneMaxObs = 2048;
template <typename R>
void launch_prep_one(const PrepCurve& pc, double* moments, int* tile_cnt, int* tile_off,
                     int* cell, R* frac, typename C2<R>::type* coef, int* cell_s, R* frac_s,
                     typename C2<R>::type* coef_s, int* status, cudaStream_t s);

// Direct FP64 sums for the listed global frequency indices of a batch:
// slot i of `list` (< min(*count, cap)) gets the sums of its curve at row
// stride `stride` and slot_curve[i] = the curve's index.  moments holds
// MO_WORDS doubles per curve.
// After a batched pass whose re-solve list overflowed (*count > cap): sets
// FTP_FLAG_UNRESOLVED on every output item of the frequencies marked 2.
void launch_redo_overflow(const CurveDesc* curves, int ncurves, const int* marks, int64_t nmarks,
                          const int* count, int cap, uint8_t* flags, cudaStream_t s);

// max_n bounds the curves' observation counts and Hs_max their harmonics.
void launch_direct_sums_batch(const CurveDesc* curves, int ncurves, const double* moments,
                              const int* status, const int* list, const int* count, int cap,
                              int64_t max_n, int Hs_max, int64_t stride, double2* sums,
                              int64_t sums_elems, int* slot_curve, int* status_rw,
                              cudaStream_t s);

// Steps (b)-(c): assembly, roots, candidates, polish.
//
// A batched launch covers many lightcurves: segment s is one curve's share
// (its frequencies times this launch's templates of the curve), and its work
// units are seg_units[s] .. seg_units[s+1]-1.
struct RootsSeg {
  int64_t sums_off;   // element offset of the curve's sum rows in `sums`
  int64_t nf_pad;     // row stride of those rows (elements)
  int64_t nf;         // frequencies of the curve
  int64_t out_off;    // element offset of the curve's output block [rows][nf]
  int64_t redo_base;  // global index of the curve's k = 0 in the re-solve marks
  int32_t Hs;         // harmonics the curve's sums were computed for
  int32_t curve;      // index of the curve's moments (MO_WORDS doubles each)
  int32_t tpl_first;  // first template (index into alpha) of this segment
  int32_t ntpl;       // templates of this segment
  int32_t row_first;  // output row of template j: rows[row_first + j]; -1: row 0
  int32_t pad_;
};
static_assert(sizeof(RootsSeg) == 64, "RootsSeg layout");

struct RootsArgs {
  const void* sums;        // [3*Hs][nf_pad] complex (float2 or double2, per kernel)
  int64_t sums_elems;      // elements of `sums` (bounds of the staged reads)
  int64_t out_elems;       // elements of each output array
  int64_t nf;              // items per template (host-side upper bound if nf_dev)
  const int* nf_dev;       // nullable: the item count, read on the device
  const int* kmap;         // nullable: output column of item k (else k)
  int64_t nf_pad;
  int Hs;                  // harmonics the sums were computed for
  int H;                   // template harmonics of this launch (<= Hs)
  int ntpl;                // templates in this launch
  const double2* alpha;    // [ntpl][kMaxH] alpha_n = (c_n + i s_n)/2, n = 1..H
  const int* rows;         // [ntpl] output row of each template
  const double* moments;   // ybar, YY
  double* power;           // [rows][out_stride]
  double* theta1;
  double* theta2;
  double* theta3;
  uint8_t* flags;          // nullable
  int64_t out_stride;
  int* status;
  unsigned long long* counters;  // CNT_* solver statistics
  unsigned long long* queue;     // two work-unit counters: [0] zero at launch, [1] cleared by the first roots kernel
  // re-solve list (mixed path): frequencies whose estimated error of P from
  // the FP32 sums exceeds kRedoTol; nullable (no re-solve)
  int* redo_list;
  int* redo_mark;          // [redo_marks] 0 / 1 listed / 2 list full; dedupes across templates
  int* redo_count;
  int redo_cap;            // entries of redo_list (batched re-solve pass: slots to read)
  int64_t redo_marks;      // entries of redo_mark
  double sum_err;          // error bound of one sum (kSumErr*)
  double redo_tol;         // re-solve threshold on the estimated error of P
  int maxit;
  int polish_steps;
  int wait_polls;     // polls of each bounded mbarrier wait (>= 1; kWaitPolls by default)
  int skip_copies;    // fault injection: no sum row is ever copied, so every wait runs out
  // main pass: a frequency with an item that hit the iteration cap goes on
  // the re-solve list with MARK_CAP (needs redo_list)
  int list_nonconv;
  // re-solve pass: items get FTP_FLAG_RESOLVED; resolve_pass 1: an item
  // still at the cap marks its frequency MARK_FP64 in sel_mark for a later
  // FP64 pass; resolve_pass 2: cap hits are final.  sel_mode 2 restricts
  // the pass to listed frequencies marked MARK_FP64 (0: every one).
  int resolve_pass;
  int* sel_mark;
  int sel_mode;
  // batched launches (segs != nullptr): `moments` holds MO_WORDS doubles per
  // curve, outputs are addressed through the segments, and re-solve marks and
  // list entries are global frequency indices (redo_base + k).
  const RootsSeg* segs;
  const int64_t* seg_units;  // [nseg + 1] first work unit of each segment
  int nseg;
  // batched re-solve pass (slot_curve != nullptr): one listed frequency per
  // work unit; kmap holds the global frequency indices, nf_dev their count,
  // slot_curve the curve of each slot and curve_seg[curve] its segment in
  // this launch (-1: the curve has no templates here)
  const int* slot_curve;
  const int* curve_seg;
  int ncurves;         // entries of curve_seg
  int64_t host_units;  // upper bound of the work units (grid sizing); 0: from nf
  // batched main pass on a subset of its units (screening): unit u of this
  // launch is unit unit_list[u] of the batched numbering, u < *unit_count;
  // nullable (every unit)
  const int64_t* unit_list;
  const unsigned long long* unit_count;
  // host side, nullable: events recorded on the launch stream before the
  // first roots kernel and between the two (timing of the first phase)
  cudaEvent_t ev_first_start;
  cudaEvent_t ev_first_end;
  int ctas_per_sm;  // persistent grid: CTAs per SM (0 or more than fit: as many as fit)
  int positive_only;  // only candidates with theta1 > 0; none: P = 0 (FTP_FLAG_NO_POSITIVE)
  // `sums` holds pre-assembled coefficients instead of sums: rows a_0..a_2H,
  // b_1..b_H, c_1..c_H (4H+1 rows of nf_pad, pooled multi-band assembly)
  int coef_mode;
};

// Kernel variants: float2 sums + FP32 Aberth (mixed), double2 sums + FP64
// Aberth (FP64 path), double2 sums + FP32 Aberth (mixed re-solve pass).
enum RootsKind { ROOTS_MIXED = 0, ROOTS_FP64 = 1, ROOTS_REDO = 2 };

// Launches the assembly + Aberth + candidate kernel.  Returns the number of
// kernel launches issued (1), -1 for an unsupported H, -2 on a CUDA error.
int launch_roots(RootsKind kind, const RootsArgs& a, int num_sms, cudaStream_t s);

// Frequencies per work unit (32 / lanes per item) of the kernel that
// launch_roots picks for (kind, H); 0 for an unsupported H.
int roots_items_per_unit(RootsKind kind, int H);

}  // namespace ftp
