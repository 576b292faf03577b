// C ABI of the FTP library (include/ftp.h): plans, workspaces, pointer
// staging, the step (a) pipeline and the per-H launches of steps (b)-(c).
#include <cufft.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/ftp.h"
#include "ftp_internal.cuh"
#include "ftp_screen.cuh"

namespace ftp {
void launch_shared_moments(const double* mom, const double* lam, int nbands, double* share,
                           double* dyb, double* pooled, int* status, cudaStream_t s);
void launch_shared_assembly(const void* sums, bool fp64, int64_t band_stride, int Hs, int nbands,
                            int64_t nf, int64_t nf_pad, int H, const double2* alpha,
                            const double* share, const double* dyb, double2* coef,
                            const int* status, cudaStream_t s);
int launch_roots_mixed(const RootsArgs& a, int num_sms, cudaStream_t s);
int launch_roots_fp64(const RootsArgs& a, int num_sms, cudaStream_t s);
int launch_roots_redo(const RootsArgs& a, int num_sms, cudaStream_t s);

int roots_lanes_mixed(int H);
int roots_lanes_fp64(int H);
int roots_lanes_redo(int H);

int roots_items_per_unit(RootsKind kind, int H) {
  const int g = kind == ROOTS_MIXED ? roots_lanes_mixed(H)
                : kind == ROOTS_FP64 ? roots_lanes_fp64(H)
                                     : roots_lanes_redo(H);
  return g > 0 ? 32 / g : 0;
}

int launch_roots(RootsKind kind, const RootsArgs& a, int num_sms, cudaStream_t s) {
  switch (kind) {
    case ROOTS_MIXED: return launch_roots_mixed(a, num_sms, s);
    case ROOTS_FP64: return launch_roots_fp64(a, num_sms, s);
    case ROOTS_REDO: return launch_roots_redo(a, num_sms, s);
  }
  return -1;
}
}  // namespace ftp

using namespace ftp;

namespace {

constexpr double kPi = 3.14159265358979323846;

struct FftEntry {
  cufftHandle h = 0;
  size_t work = 0;
};

// Workspace of one step (a) pipeline.  Lane 0 is the plan's own workspace
// and stream (single curves); ftp_batch runs the batched FFTs of different
// grid-size classes on the lanes' streams at once, each lane with its own
// cuFFT plans and work area (extra lanes own only a stream and an event).
struct SumLane {
  cudaStream_t s = nullptr;
  bool owned = false;  // buffers (and the stream) belong to this lane
  unsigned char* mom_scratch = nullptr;
  int* tile_count = nullptr;
  int* tile_off = nullptr;
  int* cursor = nullptr;
  int* cell = nullptr;
  int* cell_s = nullptr;
  void* frac = nullptr;
  void* frac_s = nullptr;
  void* coef = nullptr;
  void* coef_s = nullptr;
  void* grid = nullptr;
  void* fftwork = nullptr;
  size_t fftwork_bytes = 0;
  std::map<int64_t, FftEntry> ffts;
  std::map<std::pair<int64_t, int>, FftEntry> bffts;  // batched plans by (length, batch)
  cudaEvent_t done = nullptr;  // end of the lane's share of a chunk
};
constexpr int kSumLanes = 4;     // default concurrent step (a) lanes of ftp_batch
constexpr int kMaxSumLanes = 8;
// Default iteration cap of the FP64 re-solve of items whose main-pass Aberth
// iteration hit its cap (60 FP32 / 80 FP64 iterations).
constexpr int kRedoMaxit = 200;

}  // namespace

struct ftp_plan_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ftp_precision prec = FTP_MIXED;
  bool mixed = true;
  int64_t max_nobs = 0;
  int max_H = 0;
  ftp_grid grid{};
  int max_templates = 0;
  int num_sms = 0;
  // NFFT parameters
  int m = 4;
  double sigma = 2.0;
  double beta = 0.0;
  int64_t ngrid = 0, ntiles = 0, nf_pad = 0;
  size_t rsz = 4, csz = 8;  // working real / complex element sizes
  // device workspace
  double* d_in = nullptr;       // staged t, y, dy
  double* d_moments = nullptr;
  unsigned char* d_mom_scratch = nullptr;  // moment partials + ticket
  int* d_status = nullptr;
  unsigned long long* d_counters = nullptr;
  unsigned long long* d_queue = nullptr;  // work-unit counters of the two roots kernels
  int* d_redo_list = nullptr;            // frequencies to re-solve from direct FP64 sums
  int* d_redo_mark = nullptr;
  int* d_redo_count = nullptr;
  double2* d_redo_sums = nullptr;        // [3 max_H][nf_pad] direct FP64 sums
  int* d_tile_count = nullptr;
  int* d_tile_off = nullptr;
  int* d_cursor = nullptr;
  int* d_cell = nullptr;
  int* d_cell_s = nullptr;
  void* d_frac = nullptr;
  void* d_frac_s = nullptr;
  void* d_coef = nullptr;
  void* d_coef_s = nullptr;
  void* d_grid = nullptr;
  void* d_sums = nullptr;
  double2* d_alpha = nullptr;
  int* d_rows = nullptr;
  int* d_row0 = nullptr;    // a single 0: output row of one-template launches
  double* d_out = nullptr;  // staged outputs [4][max_templates][nf]
  uint8_t* d_flags = nullptr;
  SumLane l0;                     // step (a) on the plan's own workspace
  std::vector<SumLane*> xlanes;   // extra step (a) lanes of ftp_batch (grown on demand)
  cudaEvent_t fork = nullptr;     // start of a chunk's step (a), for the extra lanes
  // batch tuning knobs (ftp_batch_autotune): concurrent step (a) lanes and
  // CTAs per SM of the persistent roots launches (0: as many as fit)
  int sum_lanes = kSumLanes;
  int roots_ctas_per_sm = 0;
  bool positive_only = false;  // theta1 >= 0 constraint (ftp_set_positive_amplitude)
  // pinned host staging
  int* h_status = nullptr;
  unsigned long long* h_counters = nullptr;
  int* h_redo_count = nullptr;  // pinned: length of the re-solve list after the main pass
  double2* h_alpha = nullptr;
  int* h_rows = nullptr;
  // instrumentation
  int last_launches = 0;
  bool timing = false;
  cudaEvent_t ev[7] = {};
  float stage_ms[6] = {};
  // first roots kernel of each template group (timing only)
  cudaEvent_t fev[2 * kMaxH] = {};
  int fev_used = 0;
  float first_phase_ms = 0.f;
  int maxit = 60;
  int polish_steps = 1;
  // iteration cap of the FP64 re-solve of items that hit `maxit`, polls of
  // the roots kernels' bounded waits (0: default), fault injection (1: the
  // roots kernels never copy a sum row, so their waits run out)
  int redo_maxit = kRedoMaxit;
  int wait_polls = 0;
  int inject = 0;
  // ---- batch workspace (grown on demand by ftp_batch; never shrinks)
  bool in_batch = false;
  size_t chunk_bytes = (size_t)8 << 30;  // sum tiles of one chunk of curves
  bool use_graph = true;
  void* d_bsums = nullptr;
  size_t bsums_cap = 0;
  double* d_bmom = nullptr;
  size_t bmom_cap = 0;
  unsigned char* d_bprep = nullptr;  // step (a) preparation scratch of a chunk
  size_t bprep_cap = 0;
  double* d_bobs = nullptr;  // staged host observations [3][count]
  size_t bobs_cap = 0;
  double* d_bout = nullptr;  // staged host outputs [4][extent]
  size_t bout_cap = 0;
  uint8_t* d_bflags = nullptr;
  size_t bflags_cap = 0;
  void* d_bgrid = nullptr;  // NFFT grids of one group of a chunk's curves (batched step (a))
  size_t bgrid_cap = 0;
  int* d_bmark = nullptr;  // re-solve marks, one per frequency of a chunk
  size_t bmark_cap = 0;
  int* d_blist = nullptr;  // re-solve list [kBatchRedoCap]
  int* d_bslot_curve = nullptr;
  int* d_bcount = nullptr;
  double2* d_bredo_sums = nullptr;  // [3 max_H][kBatchRedoStride]
  unsigned char* d_bdesc = nullptr;  // segment / unit / curve descriptors
  size_t bdesc_cap = 0;
  unsigned char* h_bdesc = nullptr;  // pinned twin of d_bdesc
  size_t hbdesc_cap = 0;
  std::vector<cudaEvent_t> bev;      // batch stage events (timing only)
  int64_t last_chunks = 0;
  int last_graph = 0;                // 0 eager, 1 captured + launched, 2 replayed
  // the captured graph of the last repeated all-device batch call
  uint64_t graph_key = 0;
  uint64_t eager_key = 0;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_launches = 0;
  // screening workspace (ftp_batch_screened; grown on demand)
  float* d_bfeat = nullptr;     // [rows of a chunk][nfeat]
  size_t bfeat_cap = 0;
  float* d_bscore = nullptr;    // [rows of a chunk]
  size_t bscore_cap = 0;
  uint8_t* d_bsel = nullptr;    // [rows of a chunk]
  size_t bsel_cap = 0;
  int64_t* d_bulist = nullptr;  // listed work units of one launch
  size_t bulist_cap = 0;
  unsigned long long* d_bucount = nullptr;
  // multi-band workspace (ftp_multiband_periodogram; grown on demand)
  double* d_mb = nullptr;       // [4][bands][nf] per-band outputs, then [bands][MO_WORDS] moments
  size_t mb_cap = 0;
  uint8_t* d_mbflags = nullptr;  // [bands][nf]
  size_t mbflags_cap = 0;
  double* d_mbpow = nullptr;     // [nf] combined power
  size_t mbpow_cap = 0;
  // shared-phase multi-band workspace (ftp_shared_multiband; grown on demand)
  unsigned char* d_shsums = nullptr;  // [bands][3H][nf_pad] sums
  size_t shsums_cap = 0;
  double* d_shmisc = nullptr;  // moments [bands][MO_WORDS] | share | dyb | lambda | pooled
  size_t shmisc_cap = 0;
  double2* d_shalpha = nullptr;  // [bands][kMaxH]
  size_t shalpha_cap = 0;
  double2* d_shcoef = nullptr;   // [4H+1][nf_pad] pooled coefficients
  size_t shcoef_cap = 0;
};

namespace {

// Largest harmonic bin (k0 + nf - 1) a grid may reach.  Any grid beyond it
// needs more than the 2^31 FFT cells a 1-D cuFFT plan takes, so it is
// unsupported; the bound is checked before any grid arithmetic, where
// 2 H (k0 + nf - 1) could otherwise overflow and size a grid too small for
// the bins the kernels read.
constexpr int64_t kMaxBin = FTP_MAX_BIN;

ftp_status check_grid(const ftp_grid& g) {
  if (!(g.df > 0.0) || !isfinite(g.df) || g.k0 < 1 || g.nf < 1) return FTP_ERR_INVALID_ARG;
  if (g.k0 > kMaxBin || g.nf > kMaxBin || g.k0 + g.nf - 1 > kMaxBin) return FTP_ERR_UNSUPPORTED;
  return FTP_OK;
}

int64_t next_smooth(int64_t x) {
  if (x < 1) x = 1;
  for (int64_t v = x;; ++v) {
    int64_t r = v;
    for (int p : {2, 3, 5, 7})
      while (r % p == 0) r /= p;
    if (r == 1) return v;
  }
}

// Grid length for harmonic bins j <= J: at least 2 sigma J cells, a multiple
// of the spreading tile with a 7-smooth tile count (a cuFFT-friendly size).
int64_t grid_len(int64_t J, double sigma, int64_t* ntiles) {
  const double nmin = std::max(2.0 * sigma * (double)J, 2.0 * (double)J + 2.0);
  int64_t nt = (int64_t)ceil(nmin / (double)kSpreadTile);
  nt = next_smooth(nt);
  *ntiles = nt;
  return nt * kSpreadTile;
}

double kb_beta(int m, double sigma) {
  const double W = 2.0 * m;
  return kPi * sqrt((W / sigma) * (W / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

ftp_status cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return FTP_OK;
  return e == cudaErrorMemoryAllocation ? FTP_ERR_OOM : FTP_ERR_CUDA;
}

#define FTP_CK(x)                                   \
  do {                                              \
    const cudaError_t e_ = (x);                     \
    if (e_ != cudaSuccess) return cuda_err(e_);     \
  } while (0)

template <typename T>
ftp_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cuda_err(cudaMalloc((void**)p, count * sizeof(T)));
}

// The lane's shared cuFFT work area, grown to plan e's need (a plan being
// made may need more than the ones before it; queued transforms may still use
// the old area, so growing waits for the lane's stream), and set on e.
ftp_status lane_fft_work(SumLane& L, const FftEntry& e) {
  if (e.work > L.fftwork_bytes) {
    // queued transforms may still use the old work area
    if (L.s) cudaStreamSynchronize(L.s);
    if (L.fftwork) cudaFree(L.fftwork);
    L.fftwork = nullptr;
    L.fftwork_bytes = 0;
    if (cudaMalloc(&L.fftwork, e.work) != cudaSuccess) {
      cudaGetLastError();
      return FTP_ERR_OOM;
    }
    L.fftwork_bytes = e.work;
    for (auto& kv : L.ffts) cufftSetWorkArea(kv.second.h, L.fftwork);
    for (auto& kv : L.bffts) cufftSetWorkArea(kv.second.h, L.fftwork);
  }
  cufftSetWorkArea(e.h, L.fftwork);
  return FTP_OK;
}

ftp_status get_fft(ftp_plan_t P, SumLane& L, int64_t n, cufftHandle* out) {
  auto it = L.ffts.find(n);
  if (it != L.ffts.end()) {
    *out = it->second.h;
    return FTP_OK;
  }
  FftEntry e;
  if (cufftCreate(&e.h) != CUFFT_SUCCESS) return FTP_ERR_CUDA;
  cufftSetAutoAllocation(e.h, 0);
  const cufftType ty = P->mixed ? CUFFT_C2C : CUFFT_Z2Z;
  if (cufftMakePlan1d(e.h, (int)n, ty, 1, &e.work) != CUFFT_SUCCESS) {
    cufftDestroy(e.h);
    return FTP_ERR_CUDA;
  }
  const ftp_status st = lane_fft_work(L, e);
  if (st != FTP_OK) {
    cufftDestroy(e.h);
    return st;
  }
  L.ffts[n] = e;
  *out = e.h;
  return FTP_OK;
}

// A batched transform: `batch` grids of length n, back to back.
ftp_status get_fft_many(ftp_plan_t P, SumLane& L, int64_t n, int batch, cufftHandle* out) {
  const auto key = std::make_pair(n, batch);
  auto it = L.bffts.find(key);
  if (it != L.bffts.end()) {
    *out = it->second.h;
    return FTP_OK;
  }
  FftEntry e;
  if (cufftCreate(&e.h) != CUFFT_SUCCESS) return FTP_ERR_CUDA;
  cufftSetAutoAllocation(e.h, 0);
  const cufftType ty = P->mixed ? CUFFT_C2C : CUFFT_Z2Z;
  long long len = n;
  if (cufftMakePlanMany64(e.h, 1, &len, nullptr, 1, len, nullptr, 1, len, ty, batch, &e.work) !=
      CUFFT_SUCCESS) {
    cufftDestroy(e.h);
    return FTP_ERR_CUDA;
  }
  const ftp_status st = lane_fft_work(L, e);
  if (st != FTP_OK) {
    cufftDestroy(e.h);
    return st;
  }
  L.bffts[key] = e;
  *out = e.h;
  return FTP_OK;
}
ftp_status get_fft(ftp_plan_t P, int64_t n, cufftHandle* out) { return get_fft(P, P->l0, n, out); }

void ev_rec(ftp_plan_t P, int i) {
  if (P->timing && !P->in_batch) cudaEventRecord(P->ev[i], P->stream);
}

// Step (a) for one curve on lane L: moments, binning, spreading, FFT, gather
// into the sum tiles `sums` (layout [3 Hs][nf_pad]) and the moments block
// `moments`.  t, y, dy are device pointers; ngrid/ntiles give the NFFT grid
// (at most the plan's).
ftp_status run_sums(ftp_plan_t P, SumLane& L, const double* t, const double* y, const double* dy,
                    int64_t nobs, double df, int64_t k0, int64_t nf, int Hs, int64_t ngrid,
                    int64_t ntiles, double* moments, void* sums, int64_t nf_pad, int* launches) {
  if (ngrid > P->ngrid || ntiles > P->ntiles) return FTP_ERR_UNSUPPORTED;
  cufftHandle fft;
  ftp_status st = get_fft(P, L, ngrid, &fft);
  if (st != FTP_OK) return st;
  cudaStream_t s = L.s;
  ev_rec(P, 0);
  if (nobs <= kPrepOneMaxObs) {
    // short curve: moments, cells, tile order in one single-CTA launch
    const PrepCurve pc{t, y, dy, nobs, df, ngrid, ntiles, 0, 0};
    if (P->mixed) {
      launch_prep_one<float>(pc, moments, L.tile_count, L.tile_off, L.cell, (float*)L.frac,
                             (float2*)L.coef, L.cell_s, (float*)L.frac_s, (float2*)L.coef_s,
                             P->d_status, s);
    } else {
      launch_prep_one<double>(pc, moments, L.tile_count, L.tile_off, L.cell, (double*)L.frac,
                              (double2*)L.coef, L.cell_s, (double*)L.frac_s, (double2*)L.coef_s,
                              P->d_status, s);
    }
    *launches -= 4;  // three kernels in all, where the general path launches seven
  } else {
    FTP_CK(cudaMemsetAsync(L.tile_count, 0, sizeof(int) * ntiles, s));
    launch_moments(t, y, dy, nobs, moments, P->d_status, L.mom_scratch, s);
    if (P->mixed) {
      launch_points<float>(t, y, dy, nobs, moments, P->d_status, df, ngrid, L.tile_count, L.cell,
                           (float*)L.frac, (float2*)L.coef, s);
    } else {
      launch_points<double>(t, y, dy, nobs, moments, P->d_status, df, ngrid, L.tile_count, L.cell,
                            (double*)L.frac, (double2*)L.coef, s);
    }
    launch_scan(L.tile_count, ntiles, L.tile_off, L.cursor, P->d_status, s);
    if (P->mixed) {
      launch_scatter<float>(nobs, L.tile_off, L.cursor, L.cell, (float*)L.frac, (float2*)L.coef,
                            L.cell_s, (float*)L.frac_s, (float2*)L.coef_s, P->d_status, s);
    } else {
      launch_scatter<double>(nobs, L.tile_off, L.cursor, L.cell, (double*)L.frac, (double2*)L.coef,
                             L.cell_s, (double*)L.frac_s, (double2*)L.coef_s, P->d_status, s);
    }
  }
  ev_rec(P, 1);
  if (P->mixed) {
    launch_spread<float>(L.tile_off, L.cell_s, (float*)L.frac_s, (float2*)L.coef_s, ngrid, ntiles,
                         P->m, P->beta, (float2*)L.grid, P->d_status, s);
  } else {
    launch_spread<double>(L.tile_off, L.cell_s, (double*)L.frac_s, (double2*)L.coef_s, ngrid,
                          ntiles, P->m, P->beta, (double2*)L.grid, P->d_status, s);
  }
  ev_rec(P, 2);
  if (cufftSetStream(fft, s) != CUFFT_SUCCESS) return FTP_ERR_CUDA;
  cufftResult fr;
  if (P->mixed) {
    fr = cufftExecC2C(fft, (cufftComplex*)L.grid, (cufftComplex*)L.grid, CUFFT_INVERSE);
  } else {
    fr = cufftExecZ2Z(fft, (cufftDoubleComplex*)L.grid, (cufftDoubleComplex*)L.grid,
                      CUFFT_INVERSE);
  }
  if (fr != CUFFT_SUCCESS) return FTP_ERR_CUDA;
  ev_rec(P, 3);
  if (P->mixed) {
    launch_gather<float>((const float2*)L.grid, ngrid, k0, nf, nf_pad, Hs, P->m, P->beta,
                         (float2*)sums, P->d_status, s);
  } else {
    launch_gather<double>((const double2*)L.grid, ngrid, k0, nf, nf_pad, Hs, P->m, P->beta,
                          (double2*)sums, P->d_status, s);
  }
  ev_rec(P, 4);
  *launches += 7;
  FTP_CK(cudaGetLastError());
  return FTP_OK;
}

// Step (a) on the plan's own grid into the plan's sum tiles and moments.
ftp_status run_sums_plan(ftp_plan_t P, const double* t, const double* y, const double* dy,
                         int64_t nobs, int Hs, int* launches) {
  const int64_t J = 2 * (int64_t)Hs * (P->grid.k0 + P->grid.nf - 1);
  int64_t ntiles = 0;
  const int64_t ngrid = grid_len(J, P->sigma, &ntiles);
  return run_sums(P, P->l0, t, y, dy, nobs, P->grid.df, P->grid.k0, P->grid.nf, Hs, ngrid, ntiles,
                  P->d_moments, P->d_sums, P->nf_pad, launches);
}

ftp_status check_obs(ftp_plan_t P, const double* t, const double* y, const double* dy,
                     int64_t nobs) {
  if (!P || !t || !y || !dy) return FTP_ERR_INVALID_ARG;
  if (nobs < 2) return FTP_ERR_INVALID_ARG;
  if (nobs > P->max_nobs) return FTP_ERR_UNSUPPORTED;
  return FTP_OK;
}

// Make t, y, dy available on the device: device pointers are used in place,
// host arrays are copied into the plan's staging buffer.
ftp_status stage_obs(ftp_plan_t P, const double* t, const double* y, const double* dy,
                     int64_t nobs, const double** dt, const double** dyv, const double** ddy) {
  const double* src[3] = {t, y, dy};
  const double** dst[3] = {dt, dyv, ddy};
  for (int i = 0; i < 3; ++i) {
    if (is_device_ptr(src[i])) {
      *dst[i] = src[i];
    } else {
      double* d = P->d_in + (size_t)i * P->max_nobs;
      FTP_CK(cudaMemcpyAsync(d, src[i], sizeof(double) * nobs, cudaMemcpyHostToDevice, P->stream));
      *dst[i] = d;
    }
  }
  return FTP_OK;
}

cudaError_t reset_call(ftp_plan_t P) {
  cudaError_t e = cudaMemsetAsync(P->d_status, 0, sizeof(int) * ST_WORDS, P->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(P->d_counters, 0, sizeof(unsigned long long) * CNT_WORDS, P->stream);
  return e;
}

// Queues the read-back of the device status and the solver counters.
ftp_status read_back(ftp_plan_t P) {
  FTP_CK(cudaMemcpyAsync(P->h_status, P->d_status, sizeof(int) * ST_WORDS,
                         cudaMemcpyDeviceToHost, P->stream));
  FTP_CK(cudaMemcpyAsync(P->h_counters, P->d_counters, sizeof(unsigned long long) * CNT_WORDS,
                         cudaMemcpyDeviceToHost, P->stream));
  return FTP_OK;
}

// The call's result from the values read back (the stream has finished).
ftp_status finish_host(ftp_plan_t P) {
#ifdef FTP_DEVICE_CHECKS
  if (P->h_status[ST_DBG_N] != 0) {
    fprintf(stderr, "ftp device check failed: site %d value %d bound %d (%d failures)\n",
            P->h_status[ST_DBG_SITE], P->h_status[ST_DBG_A], P->h_status[ST_DBG_B],
            P->h_status[ST_DBG_N]);
    // a skipped access means the outputs cannot be trusted
    if (P->h_status[ST_CODE] == DEV_OK) return FTP_ERR_CUDA;
  }
#endif
  if (P->timing) {
    for (int i = 0; i < 6; ++i) P->stage_ms[i] = 0.f;
    float ms;
    for (int i = 0; i < 6; ++i)
      if (cudaEventElapsedTime(&ms, P->ev[i], P->ev[i + 1]) == cudaSuccess) P->stage_ms[i] = ms;
    P->first_phase_ms = 0.f;
    for (int g = 0; g < P->fev_used; ++g)
      if (cudaEventElapsedTime(&ms, P->fev[2 * g], P->fev[2 * g + 1]) == cudaSuccess)
        P->first_phase_ms += ms;
    P->fev_used = 0;
    cudaGetLastError();
  }
  return (ftp_status)P->h_status[ST_CODE];
}

ftp_status finish(ftp_plan_t P) {
  const ftp_status st = read_back(P);
  if (st != FTP_OK) return st;
  FTP_CK(cudaStreamSynchronize(P->stream));
  return finish_host(P);
}

ftp_status check_templates(ftp_plan_t P, const ftp_template* tpl, int ntpl) {
  if (!tpl || ntpl < 1) return FTP_ERR_INVALID_ARG;
  if (ntpl > P->max_templates) return FTP_ERR_UNSUPPORTED;
  for (int i = 0; i < ntpl; ++i) {
    if (tpl[i].H < 1 || !tpl[i].c || !tpl[i].s) return FTP_ERR_INVALID_ARG;
    if (tpl[i].H > P->max_H) return FTP_ERR_UNSUPPORTED;
    for (int n = 0; n < tpl[i].H; ++n)
      if (!isfinite(tpl[i].c[n]) || !isfinite(tpl[i].s[n])) return FTP_ERR_NONFINITE;
  }
  return FTP_OK;
}

struct HGroup {
  int H;
  int first;  // index into the grouped alpha / rows order
  int count;
};

// Uploads alpha_n = (c_n + i s_n)/2 for the templates grouped by H, and the
// output row of each; fills `groups`.
ftp_status upload_templates(ftp_plan_t P, const ftp_template* tpl, int ntpl,
                            std::vector<HGroup>* groups, std::vector<int>* pos_of) {
  std::vector<int> order(ntpl);
  for (int i = 0; i < ntpl; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return tpl[a].H < tpl[b].H; });
  groups->clear();
  pos_of->assign(ntpl, 0);
  for (int q = 0; q < ntpl; ++q) {
    const int i = order[q];
    (*pos_of)[i] = q;
    for (int n = 0; n < kMaxH; ++n) {
      double2 al = make_double2(0.0, 0.0);
      if (n < tpl[i].H) al = make_double2(0.5 * tpl[i].c[n], 0.5 * tpl[i].s[n]);
      P->h_alpha[(size_t)q * kMaxH + n] = al;
    }
    P->h_rows[q] = i;
    if (groups->empty() || groups->back().H != tpl[i].H) groups->push_back({tpl[i].H, q, 0});
    groups->back().count++;
  }
  FTP_CK(cudaMemcpyAsync(P->d_alpha, P->h_alpha, sizeof(double2) * kMaxH * ntpl,
                         cudaMemcpyHostToDevice, P->stream));
  FTP_CK(cudaMemcpyAsync(P->d_rows, P->h_rows, sizeof(int) * ntpl, cudaMemcpyHostToDevice,
                         P->stream));
  return FTP_OK;
}

// The plan's solver settings for one roots launch.
void solver_settings(ftp_plan_t P, RootsArgs& a) {
  a.maxit = P->maxit;
  a.polish_steps = P->polish_steps;
  a.ctas_per_sm = P->roots_ctas_per_sm;
  a.positive_only = P->positive_only ? 1 : 0;
  a.wait_polls = P->wait_polls > 0 ? P->wait_polls : kWaitPolls;
  a.skip_copies = P->inject == 1 ? 1 : 0;
}

// A re-solve pass over listed frequencies from direct FP64 sums.  Mixed
// path: pass 1 (FP32 iterations, rounding-level acceptance of stalled roots)
// over every listed frequency, whose items still at the cap mark their
// frequency for pass 2 (FP64 iterations, sel_mode 2: those frequencies only).
// FP64 path: pass 2 over every listed frequency (sel_mode 0).  Both passes
// iterate up to redo_maxit.
void resolve_settings(ftp_plan_t P, RootsArgs& a, int* marks, int pass, int sel_mode) {
  a.resolve_pass = pass;
  a.sel_mark = marks;
  a.sel_mode = sel_mode;
  a.maxit = P->redo_maxit;
  // re-solve lists are short (usually empty): one CTA per SM keeps an empty
  // pass cheap and still runs four warps per SM on a long list
  a.ctas_per_sm = 1;
}

ftp_status run_roots(ftp_plan_t P, RootsKind kind, const void* sums, int H, int Hs, int64_t nf,
                     const int* nf_dev, const int* kmap, bool collect_redo, const double2* alpha,
                     const int* rows, int ntpl, double* const* o, uint8_t* flags,
                     int64_t out_stride, int64_t out_elems, int* launches, bool time_first = false,
                     int resolve_pass = 0, int sel_mode = 0) {
  RootsArgs a{};
  if (time_first && P->timing && !P->in_batch && P->fev_used < kMaxH &&
      P->fev[2 * P->fev_used]) {
    a.ev_first_start = P->fev[2 * P->fev_used];
    a.ev_first_end = P->fev[2 * P->fev_used + 1];
    ++P->fev_used;
  }
  a.sums = sums;
  a.sums_elems = (int64_t)3 * P->max_H * P->nf_pad;
  a.out_elems = out_elems;
  a.nf = nf;
  a.nf_dev = nf_dev;
  a.kmap = kmap;
  a.nf_pad = P->nf_pad;
  a.Hs = Hs;
  a.H = H;
  a.ntpl = ntpl;
  a.alpha = alpha;
  a.rows = rows;
  a.moments = P->d_moments;
  a.power = o[0];
  a.theta1 = o[1];
  a.theta2 = o[2];
  a.theta3 = o[3];
  a.flags = flags;
  a.out_stride = out_stride;
  a.status = P->d_status;
  a.counters = P->d_counters;
  a.queue = P->d_queue;
  if (collect_redo) {
    a.redo_list = P->d_redo_list;
    a.redo_mark = P->d_redo_mark;
    a.redo_count = P->d_redo_count;
    a.redo_cap = (int)P->grid.nf;
    a.redo_marks = P->grid.nf;
    a.sum_err = P->mixed ? kSumErrF32 : kSumErrF64;
    a.redo_tol = P->mixed ? kRedoTolF32 : kRedoTolF64;
    a.list_nonconv = 1;
  }
  solver_settings(P, a);
  if (resolve_pass) resolve_settings(P, a, P->d_redo_mark, resolve_pass, sel_mode);
  FTP_CK(cudaMemsetAsync(P->d_queue, 0, sizeof(unsigned long long), P->stream));
  const int r = launch_roots(kind, a, P->num_sms, P->stream);
  if (r == -1) return FTP_ERR_UNSUPPORTED;
  if (r < 0) return FTP_ERR_CUDA;
  *launches += r;
  FTP_CK(cudaGetLastError());
  return FTP_OK;
}

// Steps (b)-(c) for one curve whose sums are in the plan's tiles: one launch
// per group of templates with equal H.  Frequencies whose estimated error of
// P from the NFFT sums exceeds the path's threshold (ill-conditioned ones,
// where clustered phases make MM a small difference of O(1) sums) are then
// recomputed from direct FP64 sums with the same kernel (FP32 Aberth on the
// mixed path, FP64 Aberth on the FP64 path); frequencies where an item hit
// the Aberth iteration cap are recomputed the same way with the larger cap
// redo_maxit and a rounding-level acceptance of stalled roots, and on the
// mixed path items still at the cap then once more with FP64 iterations.
//
// The main pass (solve_main) lists the frequencies to re-solve on the device;
// the caller reads the list's length back with the call's status at the sync
// the call makes anyway and runs the re-solve passes (solve_redo) only when
// the list is not empty, so a call with nothing to re-solve launches none of
// their kernels.
ftp_status solve_main(ftp_plan_t P, int64_t nf, int Hs, const std::vector<HGroup>& groups,
                      const double2* alpha, const int* rows, const int* row0, double* const* o,
                      uint8_t* flags, int64_t out_elems, int* launches) {
  FTP_CK(cudaMemsetAsync(P->d_redo_mark, 0, sizeof(int) * nf, P->stream));
  FTP_CK(cudaMemsetAsync(P->d_redo_count, 0, sizeof(int), P->stream));
  const RootsKind kind = P->mixed ? ROOTS_MIXED : ROOTS_FP64;
  for (const HGroup& g : groups) {
    ftp_status st = run_roots(P, kind, P->d_sums, g.H, Hs, nf, nullptr, nullptr, true,
                              alpha + (size_t)g.first * kMaxH, row0 ? row0 : rows + g.first,
                              g.count, o, flags, nf, out_elems, launches, true);
    if (st != FTP_OK) return st;
  }
  ev_rec(P, 5);
  return FTP_OK;
}

ftp_status solve_redo(ftp_plan_t P, const double* dt, const double* dyv, const double* ddy,
                      int64_t nobs, double df, int64_t k0, int64_t nf, int Hs,
                      const std::vector<HGroup>& groups, const double2* alpha, const int* rows,
                      const int* row0, double* const* o, uint8_t* flags, int64_t out_elems,
                      int* launches) {
  launch_direct_sums(dt, dyv, ddy, nobs, P->d_moments, P->d_status, df, k0, P->d_redo_list,
                     P->d_redo_count, (int)nf, Hs, P->nf_pad, P->d_redo_sums,
                     (int64_t)3 * P->max_H * P->nf_pad, P->d_status, P->stream);
  *launches += 2;  // zeroing + direct sums
  // mixed path: FP32 iterations for every listed frequency, then FP64
  // iterations for those still at the cap; FP64 path: FP64 for all
  const int passes = P->mixed ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    const bool fp32 = P->mixed && pass == 0;
    const RootsKind rk = fp32 ? ROOTS_REDO : ROOTS_FP64;
    for (const HGroup& g : groups) {
      ftp_status st = run_roots(P, rk, P->d_redo_sums, g.H, Hs, nf, P->d_redo_count,
                                P->d_redo_list, false, alpha + (size_t)g.first * kMaxH,
                                row0 ? row0 : rows + g.first, g.count, o, flags, nf, out_elems,
                                launches, false, fp32 ? 1 : 2, P->mixed && !fp32 ? 2 : 0);
      if (st != FTP_OK) return st;
    }
  }
  return FTP_OK;
}

}  // namespace

namespace {

// ------------------------------------------------------------------ batches
// ftp_batch runs many lightcurves through one pipeline:
//   - curves are cut into chunks whose sum tiles fit the chunk budget;
//   - step (a) runs per curve (moments .. gather, cuFFT at one of a few grid
//     size classes) into the curve's slice of the chunk's sum tiles;
//   - steps (b)-(c) run as ONE persistent roots launch per harmonic count H
//     over every (frequency, template) item of every curve in the chunk: the
//     warps' work queue walks a segment table (one segment per curve);
//   - ill-conditioned frequencies of the whole chunk go through one batched
//     direct-sums launch and one re-solve launch per H;
//   - when every array is on the device and a call repeats the previous one
//     (same pointers, sizes and templates), the device work of the call is
//     captured once into a CUDA graph and replayed afterwards.
constexpr int kBatchRedoCap = 1 << 18;                    // re-solve slots per chunk
constexpr int64_t kBatchRedoStride = kBatchRedoCap + 64;  // row stride of their sums

// Grid length for a batched curve: at least 2 sigma J cells, rounded up to
// 2048 * q with q <= 8 or q in {4, 5, 6, 7} * 2^e, so that a batch of curves
// needs only a few cuFFT plans (at most 25 % extra cells).
int64_t grid_len_class(int64_t J, double sigma, int64_t* ntiles) {
  const double nmin = std::max(2.0 * sigma * (double)J, 2.0 * (double)J + 2.0);
  const int64_t need = (int64_t)ceil(nmin / (double)kSpreadTile);
  int64_t nt = need;
  if (need > 8) {
    bool found = false;
    for (int64_t p2 = 2; !found; p2 *= 2)
      for (int m : {4, 5, 6, 7})
        if (!found && m * p2 >= need) {
          nt = m * p2;
          found = true;
        }
  }
  *ntiles = nt;
  return nt * kSpreadTile;
}

// Grow-only device buffer; dropping the old one waits for queued work.
template <typename T>
ftp_status grow_dev(T** p, size_t* cap, size_t count, bool* grew) {
  if (count == 0) count = 1;
  if (*p && *cap >= count) return FTP_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  *grew = true;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return FTP_ERR_OOM;
  }
  *cap = count;
  return FTP_OK;
}

// Multi-phase combination (Section 2.2, Eq. multibandmultiphase): per
// frequency, P = sum_b chi2_0,b P_b / sum_b chi2_0,b with chi2_0,b = YY_b W_b
// (YY is the variance under normalised weights, W the sum of the raw ones).
__global__ void __launch_bounds__(256) multiband_combine_kernel(const double* __restrict__ bp,
                                                                const double* __restrict__ mom,
                                                                int nbands, int64_t nf,
                                                                double* __restrict__ power) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  double num = 0.0, den = 0.0;
  for (int b = 0; b < nbands; ++b) {
    const double c = mom[(size_t)b * MO_WORDS + MO_YY] * mom[(size_t)b * MO_WORDS + MO_WSUM];
    num += c * bp[(size_t)b * nf + k];
    den += c;
  }
  power[k] = num / den;
}

void launch_multiband_combine(const double* bp, const double* mom, int nbands, int64_t nf,
                              double* power, cudaStream_t s) {
  multiband_combine_kernel<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(bp, mom, nbands, nf,
                                                                         power);
}

void free_lane(SumLane* L) {
  if (L->s) cudaStreamSynchronize(L->s);
  for (auto& kv : L->ffts) cufftDestroy(kv.second.h);
  L->ffts.clear();
  for (auto& kv : L->bffts) cufftDestroy(kv.second.h);
  L->bffts.clear();
  if (L->fftwork) cudaFree(L->fftwork);
  L->fftwork = nullptr;
  if (!L->owned) return;
  void* bufs[] = {L->mom_scratch, L->tile_count, L->tile_off, L->cursor, L->cell, L->cell_s,
                  L->frac, L->frac_s, L->coef, L->coef_s, L->grid};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (L->done) cudaEventDestroy(L->done);
  if (L->s) cudaStreamDestroy(L->s);
}

// Extra step (a) lanes up to `want` lanes in all (lane 0 is the plan's own),
// each sized like the plan's workspace.  *grew is set when one is created.
ftp_status ensure_lanes(ftp_plan_t P, int want, bool* grew) {
  if (!P->fork && cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming) != cudaSuccess)
    return FTP_ERR_CUDA;
  while ((int)P->xlanes.size() + 1 < want) {
    SumLane* L = new SumLane();
    L->owned = true;
    const bool ok = cudaStreamCreateWithFlags(&L->s, cudaStreamNonBlocking) == cudaSuccess &&
                    cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_lane(L);
      delete L;
      return FTP_ERR_OOM;
    }
    P->xlanes.push_back(L);
    *grew = true;
  }
  return FTP_OK;
}

struct BCurve {
  const double* t;  // device
  const double* y;
  const double* dy;
  int64_t n, nf, nf_pad, ngrid, ntiles, k0;
  int64_t sums_off;   // elements, within the chunk
  int64_t redo_base;  // within the chunk
  int64_t out_off;
  double df;
  int Hc, ntc, tpl;
  int Ht;  // template harmonics (Hc, the sums' harmonics, may be larger for features)
  int64_t obs_base, tile_base;  // within the chunk's preparation scratch
};
struct BLaunch {
  int H, ntpl, Hs;
  int64_t seg_first, units_first, cseg_first, units;
  int nseg;
};
// Batched step (a): a chunk's curves sorted by NFFT grid length and cut into
// groups whose grids fit the grid buffer; per group one spreading launch,
// one batched FFT per grid-size class, one gather launch.
struct BFftClass {
  int64_t n, goff;  // grid length; first element of the class's grids in the buffer
  int count;
};
struct BSub {
  int64_t desc_first;  // first StepACurve of the group in the descriptor blob
  int ncurves;
  int64_t pref_first;  // spread prefix at pref_first, gather prefix ncurves + 1 later
  int64_t spread_tiles = 0, gather_tiles = 0, grid_elems = 0;
  std::vector<BFftClass> classes;
};
struct BChunk {
  int64_t c0, c1, sums_elems, nf_total;
  int Hs;
  std::vector<BLaunch> launches;
  std::vector<BSub> subs;
  int64_t items;  // (template, frequency) output items of the chunk's curves
  int64_t obs_total = 0, tiles_total = 0;  // preparation scratch of the chunk
};
// The chunk's step (a) preparation scratch: observations in tile order (and
// the unsorted copies), tile offsets and counters.
struct PrepBufs {
  const PrepCurve* curves;  // device, [ncurves]
  int* cell;
  int* cell_s;
  void* frac;
  void* frac_s;
  void* coef;
  void* coef_s;
  int* tile_cnt;
  int* tile_off;
};

// Optional extra work of a batch: features only (feat_out), or screening by
// the surrogate network before the exact solve (mlp).
struct BatchScreen {
  int Hf = 0;                         // feature harmonics
  float* feat_out = nullptr;          // features-only mode: device [rows][2 Hf + 2]
  const int64_t* feat_row = nullptr;  // host: first features row of curve c
  const ftp_mlp_s* mlp = nullptr;     // screened mode
  double top_frac = 0.0;
  int nbr = 0;
  double* moments_out = nullptr;      // device [ncurves][MO_WORDS]: each curve's moments
};

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Lanes that run a group's batched FFTs (one class per lane, round-robin).
int fft_lanes_used(ftp_plan_t P, const BSub& sb) {
  return (int)std::max<int64_t>(
      1, std::min<int64_t>(std::min<int64_t>(1 + (int64_t)P->xlanes.size(), P->sum_lanes),
                           (int64_t)sb.classes.size()));
}

ftp_status enqueue_batch_device(ftp_plan_t P, const std::vector<BCurve>& cv,
                                const std::vector<BChunk>& chunks, const StepACurve* d_stepa,
                                const int64_t* d_pref, const RootsSeg* d_segs,
                                const int64_t* d_units, const CurveDesc* d_curves,
                                const int* d_cseg, double* const* o, uint8_t* of,
                                int64_t extent, const BatchScreen* scr,
                                const ScreenCurve* d_scurves, const int64_t* d_rowoff,
                                const PrepBufs& pb, int* launches) {
  cudaStream_t s = P->stream;
  const RootsKind kind = P->mixed ? ROOTS_MIXED : ROOTS_FP64;
  const RootsKind rkind = P->mixed ? ROOTS_REDO : ROOTS_FP64;
  const bool tm = P->timing;
  for (size_t q = 0; q < chunks.size(); ++q) {
    const BChunk& ch = chunks[q];
    if (tm) cudaEventRecord(P->bev[5 * q + 0], s);
    // step (a) preparation of every curve of the chunk in one launch
    // (moments, cells, tile order); then per group of curves one spreading
    // launch, one batched FFT per grid-size class (classes round-robin over
    // the lanes, fork/join through events, so a captured graph holds
    // parallel branches) and one gather launch
    if (P->mixed) {
      launch_prep_batch<float>(pb.curves + ch.c0, (int)(ch.c1 - ch.c0), P->d_bmom, pb.tile_cnt,
                               pb.tile_off, pb.cell, (float*)pb.frac, (float2*)pb.coef,
                               pb.cell_s, (float*)pb.frac_s, (float2*)pb.coef_s, P->d_status, s);
    } else {
      launch_prep_batch<double>(pb.curves + ch.c0, (int)(ch.c1 - ch.c0), P->d_bmom, pb.tile_cnt,
                                pb.tile_off, pb.cell, (double*)pb.frac, (double2*)pb.coef,
                                pb.cell_s, (double*)pb.frac_s, (double2*)pb.coef_s, P->d_status,
                                s);
    }
    *launches += 1;
    for (const BSub& sb : ch.subs) {
      const StepACurve* sc = d_stepa + sb.desc_first;
      const int64_t* spre = d_pref + sb.pref_first;
      const int64_t* gpre = spre + sb.ncurves + 1;
      if (P->mixed) {
        launch_spread_batch<float>(sc, spre, sb.ncurves, sb.spread_tiles, P->m, P->beta,
                                   P->d_status, s);
      } else {
        launch_spread_batch<double>(sc, spre, sb.ncurves, sb.spread_tiles, P->m, P->beta,
                                    P->d_status, s);
      }
      *launches += 1;
      const int used = fft_lanes_used(P, sb);
      if (used > 1) {
        FTP_CK(cudaEventRecord(P->fork, s));
        for (int l = 1; l < used; ++l) FTP_CK(cudaStreamWaitEvent(P->xlanes[l - 1]->s, P->fork, 0));
      }
      for (size_t k = 0; k < sb.classes.size(); ++k) {
        const BFftClass& fc = sb.classes[k];
        const int l = (int)(k % (size_t)used);
        SumLane& L = l == 0 ? P->l0 : *P->xlanes[l - 1];
        cufftHandle fft;
        ftp_status st = get_fft_many(P, L, fc.n, fc.count, &fft);  // made before: a lookup
        if (st != FTP_OK) return st;
        if (cufftSetStream(fft, l == 0 ? s : L.s) != CUFFT_SUCCESS) return FTP_ERR_CUDA;
        void* g = static_cast<unsigned char*>(P->d_bgrid) + (size_t)fc.goff * P->csz;
        const cufftResult fr =
            P->mixed ? cufftExecC2C(fft, (cufftComplex*)g, (cufftComplex*)g, CUFFT_INVERSE)
                     : cufftExecZ2Z(fft, (cufftDoubleComplex*)g, (cufftDoubleComplex*)g,
                                    CUFFT_INVERSE);
        if (fr != CUFFT_SUCCESS) return FTP_ERR_CUDA;
      }
      for (int l = 1; l < used; ++l) {
        SumLane& L = *P->xlanes[l - 1];
        FTP_CK(cudaEventRecord(L.done, L.s));
        FTP_CK(cudaStreamWaitEvent(s, L.done, 0));
      }
      if (P->mixed) {
        launch_gather_batch<float>(sc, gpre, sb.ncurves, sb.gather_tiles, P->m, P->beta,
                                   P->d_status, s);
      } else {
        launch_gather_batch<double>(sc, gpre, sb.ncurves, sb.gather_tiles, P->m, P->beta,
                                    P->d_status, s);
      }
      *launches += 1;
      FTP_CK(cudaGetLastError());
    }
    if (tm) cudaEventRecord(P->bev[5 * q + 1], s);
    if (scr && scr->moments_out)
      FTP_CK(cudaMemcpyAsync(scr->moments_out + (size_t)ch.c0 * MO_WORDS, P->d_bmom,
                             sizeof(double) * MO_WORDS * (size_t)(ch.c1 - ch.c0),
                             cudaMemcpyDeviceToDevice, s));
    const bool screened = scr && scr->mlp;
    if (scr && scr->Hf > 0) {
      // features of every frequency of the chunk (into the caller's array in
      // features-only mode), then the network's scores, the selection, and
      // the outputs of the frequencies that will not be evaluated
      FeatArgs fa{};
      fa.sums = P->d_bsums;
      fa.moments = P->d_bmom;
      fa.curves = d_scurves + ch.c0;
      fa.ncurves = (int)(ch.c1 - ch.c0);
      fa.Hf = scr->Hf;
      fa.nrows = ch.nf_total;
      fa.out = scr->feat_out ? scr->feat_out : P->d_bfeat;
      fa.status = P->d_status;
      const int r = launch_features(fa, !P->mixed, s);
      if (r < 0) return FTP_ERR_UNSUPPORTED;
      *launches += r;
      if (!screened) {
        if (tm) {
          cudaEventRecord(P->bev[5 * q + 2], s);
          cudaEventRecord(P->bev[5 * q + 3], s);
          cudaEventRecord(P->bev[5 * q + 4], s);
        }
        FTP_CK(cudaGetLastError());
        continue;
      }
      if (launch_mlp_forward(mlp_params_dev(scr->mlp), mlp_nfeat(scr->mlp), P->d_bfeat,
                             ch.nf_total, P->d_bscore, P->d_status, P->num_sms, s) < 0)
        return FTP_ERR_CUDA;
      SelectArgs sa{};
      sa.ncurves = (int)(ch.c1 - ch.c0);
      sa.row_off = d_rowoff + ch.c0 + q;
      sa.top_frac = scr->top_frac;
      sa.nbr = scr->nbr;
      sa.sel = P->d_bsel;
      sa.status = P->d_status;
      launch_select(sa, P->d_bscore, false, s);
      launch_fill(d_scurves + ch.c0, (int)(ch.c1 - ch.c0), ch.items, o[0], o[1], o[2], o[3], of,
                  P->d_status, s);
      *launches += 3;
    }
    if (tm) cudaEventRecord(P->bev[5 * q + 2], s);
    FTP_CK(cudaMemsetAsync(P->d_bmark, 0, sizeof(int) * (size_t)ch.nf_total, s));
    FTP_CK(cudaMemsetAsync(P->d_bcount, 0, sizeof(int), s));
    for (const BLaunch& L : ch.launches) {
      RootsArgs a{};
      a.sums = P->d_bsums;
      a.sums_elems = ch.sums_elems;
      a.out_elems = extent;
      a.Hs = L.Hs;
      a.H = L.H;
      a.ntpl = L.ntpl;
      a.alpha = P->d_alpha;
      a.rows = P->d_rows;
      a.moments = P->d_bmom;
      a.power = o[0];
      a.theta1 = o[1];
      a.theta2 = o[2];
      a.theta3 = o[3];
      a.flags = of;
      a.status = P->d_status;
      a.counters = P->d_counters;
      a.queue = P->d_queue;
      a.redo_list = P->d_blist;
      a.redo_mark = P->d_bmark;
      a.redo_count = P->d_bcount;
      a.redo_cap = kBatchRedoCap;
      a.redo_marks = ch.nf_total;
      a.sum_err = P->mixed ? kSumErrF32 : kSumErrF64;
      a.redo_tol = P->mixed ? kRedoTolF32 : kRedoTolF64;
      a.list_nonconv = 1;
      solver_settings(P, a);
      a.segs = d_segs + L.seg_first;
      a.seg_units = d_units + L.units_first;
      a.nseg = L.nseg;
      a.host_units = L.units;
      if (screened) {
        FTP_CK(cudaMemsetAsync(P->d_bucount, 0, sizeof(unsigned long long), s));
        launch_unit_list(d_segs + L.seg_first, d_units + L.units_first, L.nseg, L.units,
                         roots_items_per_unit(kind, L.H), P->d_bsel, P->d_bulist, P->d_bucount,
                         P->d_status, s);
        *launches += 1;
        a.unit_list = P->d_bulist;
        a.unit_count = P->d_bucount;
      }
      FTP_CK(cudaMemsetAsync(P->d_queue, 0, sizeof(unsigned long long), s));
      const int r = launch_roots(kind, a, P->num_sms, s);
      if (r == -1) return FTP_ERR_UNSUPPORTED;
      if (r < 0) return FTP_ERR_CUDA;
      *launches += r;
    }
    if (tm) cudaEventRecord(P->bev[5 * q + 3], s);
    const int ncc = (int)(ch.c1 - ch.c0);
    const CurveDesc* dcur = d_curves + ch.c0;
    launch_direct_sums_batch(dcur, ncc, P->d_bmom, P->d_status, P->d_blist, P->d_bcount,
                             kBatchRedoCap, P->max_nobs, P->max_H, kBatchRedoStride,
                             P->d_bredo_sums,
                             (int64_t)3 * P->max_H * kBatchRedoStride, P->d_bslot_curve,
                             P->d_status, s);
    *launches += 2;  // zeroing + direct sums
    const int passes = P->mixed ? 2 : 1;
    for (int pass = 0; pass < passes; ++pass)
    for (const BLaunch& L : ch.launches) {
      const RootsKind rk = (P->mixed && pass == 0) ? rkind : ROOTS_FP64;
      RootsArgs a{};
      a.sums = P->d_bredo_sums;
      a.sums_elems = (int64_t)3 * P->max_H * kBatchRedoStride;
      a.out_elems = extent;
      a.nf = kBatchRedoCap;
      a.nf_dev = P->d_bcount;
      a.kmap = P->d_blist;
      a.nf_pad = kBatchRedoStride;
      a.Hs = ch.Hs;
      a.H = L.H;
      a.ntpl = L.ntpl;
      a.alpha = P->d_alpha;
      a.rows = P->d_rows;
      a.moments = P->d_bmom;
      a.power = o[0];
      a.theta1 = o[1];
      a.theta2 = o[2];
      a.theta3 = o[3];
      a.flags = of;
      a.status = P->d_status;
      a.counters = P->d_counters;
      a.queue = P->d_queue;
      a.redo_cap = kBatchRedoCap;
      solver_settings(P, a);
      const bool fp32 = P->mixed && pass == 0;
      resolve_settings(P, a, P->d_bmark, fp32 ? 1 : 2, P->mixed && !fp32 ? 2 : 0);
      a.segs = d_segs + L.seg_first;
      a.seg_units = d_units + L.units_first;
      a.nseg = L.nseg;
      a.slot_curve = P->d_bslot_curve;
      a.curve_seg = d_cseg + L.cseg_first;
      a.ncurves = ncc;
      a.host_units = (int64_t)kBatchRedoCap * L.ntpl;
      FTP_CK(cudaMemsetAsync(P->d_queue, 0, sizeof(unsigned long long), s));
      const int r = launch_roots(rk, a, P->num_sms, s);
      if (r == -1) return FTP_ERR_UNSUPPORTED;
      if (r < 0) return FTP_ERR_CUDA;
      *launches += r;
    }
    if (of) {
      launch_redo_overflow(dcur, ncc, P->d_bmark, ch.nf_total, P->d_bcount, kBatchRedoCap, of, s);
      *launches += 1;
    }
    if (tm) cudaEventRecord(P->bev[5 * q + 4], s);
    FTP_CK(cudaGetLastError());
  }
  return FTP_OK;
}

ftp_status run_batch(ftp_plan_t P, int64_t ncurves, const int64_t* obs_off, const double* t,
                     const double* y, const double* dy, const ftp_grid* grids,
                     const int64_t* out_off, const ftp_template* bank, int nbank,
                     const int32_t* tpl_of_curve, double* power, double* theta1, double* theta2,
                     double* theta3, uint8_t* flags, const BatchScreen* scr) {
  const bool feat_only = scr && scr->feat_out;
  const int Hf = scr ? scr->Hf : 0;
  if (!P || ncurves < 0 || !obs_off || !t || !y || !dy || !grids)
    return FTP_ERR_INVALID_ARG;
  if (!feat_only && (!out_off || !power || !theta1 || !theta2 || !theta3))
    return FTP_ERR_INVALID_ARG;
  if (feat_only && (!scr->feat_row || !is_device_ptr(scr->feat_out))) return FTP_ERR_INVALID_ARG;
  if (scr && (scr->feat_out || scr->mlp) && (Hf < 1 || Hf > kFeatMaxH || Hf > P->max_H))
    return FTP_ERR_UNSUPPORTED;
  if (ncurves == 0) return FTP_OK;
  if (ncurves > (int64_t)1 << 30) return FTP_ERR_UNSUPPORTED;
  ftp_status st = feat_only ? FTP_OK : check_templates(P, bank, nbank);
  if (st != FTP_OK) return st;
  int Hs = Hf;
  if (!feat_only)
    for (int i = 0; i < nbank; ++i) Hs = std::max(Hs, bank[i].H);
  // ---- validate every curve on the host before any work is queued
  int64_t o_lo = obs_off[0], o_hi = obs_off[0], extent = 0;
  for (int64_t c = 0; c < ncurves; ++c) {
    const int64_t n = obs_off[c + 1] - obs_off[c];
    if (obs_off[c] < 0 || n < 2) return FTP_ERR_INVALID_ARG;
    if (n > P->max_nobs) return FTP_ERR_UNSUPPORTED;
    const ftp_grid& g = grids[c];
    const ftp_status gs = check_grid(g);
    if (gs != FTP_OK) return gs;
    if (feat_only ? scr->feat_row[c] < 0 : out_off[c] < 0) return FTP_ERR_INVALID_ARG;
    if (g.nf > P->grid.nf) return FTP_ERR_UNSUPPORTED;
    if (!feat_only && tpl_of_curve && (tpl_of_curve[c] < 0 || tpl_of_curve[c] >= nbank))
      return FTP_ERR_INVALID_ARG;
    const int H = std::max(Hf, (!feat_only && tpl_of_curve) ? bank[tpl_of_curve[c]].H : Hs);
    int64_t nt = 0;
    if (grid_len(2 * (int64_t)H * (g.k0 + g.nf - 1), P->sigma, &nt) > P->ngrid)
      return FTP_ERR_UNSUPPORTED;
    o_lo = std::min(o_lo, obs_off[c]);
    o_hi = std::max(o_hi, obs_off[c + 1]);
    if (!feat_only) extent = std::max(extent, out_off[c] + (tpl_of_curve ? 1 : nbank) * g.nf);
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  const bool in_dev = is_device_ptr(t) && is_device_ptr(y) && is_device_ptr(dy);
  const bool out_dev = feat_only ||
                       (is_device_ptr(power) && is_device_ptr(theta1) && is_device_ptr(theta2) &&
                        is_device_ptr(theta3) && (!flags || is_device_ptr(flags)));

  // ---- per-curve layout and chunks
  bool grew = false;
  const int64_t nobs_all = o_hi - o_lo;
  if (!in_dev) {
    st = grow_dev(&P->d_bobs, &P->bobs_cap, (size_t)3 * nobs_all, &grew);
    if (st != FTP_OK) return st;
  }
  std::vector<BCurve> cv((size_t)ncurves);
  std::vector<BChunk> chunks;
  {
    BChunk cur{0, 0, 0, 0, 0, {}, {}, 0};
    for (int64_t c = 0; c < ncurves; ++c) {
      BCurve& b = cv[(size_t)c];
      const ftp_grid& g = grids[c];
      const int64_t rel = obs_off[c] - o_lo;  // position in the staged copy
      b.t = in_dev ? t + obs_off[c] : P->d_bobs + rel;
      b.y = in_dev ? y + obs_off[c] : P->d_bobs + nobs_all + rel;
      b.dy = in_dev ? dy + obs_off[c] : P->d_bobs + 2 * nobs_all + rel;
      b.n = obs_off[c + 1] - obs_off[c];
      b.nf = g.nf;
      b.k0 = g.k0;
      b.df = g.df;
      b.nf_pad = (g.nf + 63) / 64 * 64;
      b.tpl = (!feat_only && tpl_of_curve) ? tpl_of_curve[c] : -1;
      b.Ht = b.tpl >= 0 ? bank[b.tpl].H : Hs;
      b.Hc = std::max(b.Ht, Hf);
      b.ntc = feat_only ? 0 : tpl_of_curve ? 1 : nbank;
      b.out_off = feat_only ? 0 : out_off[c];
      const int64_t J = 2 * (int64_t)b.Hc * (g.k0 + g.nf - 1);
      b.ngrid = grid_len_class(J, P->sigma, &b.ntiles);
      if (b.ngrid > P->ngrid) b.ngrid = grid_len(J, P->sigma, &b.ntiles);
      const int64_t elems = 3 * (int64_t)b.Hc * b.nf_pad;
      const bool full = cur.c1 > cur.c0 &&
                        ((size_t)(cur.sums_elems + elems) * P->csz > P->chunk_bytes ||
                         cur.nf_total + b.nf > ((int64_t)1 << 30));
      if (full) {
        chunks.push_back(cur);
        cur = BChunk{c, c, 0, 0, 0, {}, {}, 0};
      }
      b.sums_off = cur.sums_elems;
      b.redo_base = cur.nf_total;
      b.obs_base = cur.obs_total;
      b.tile_base = cur.tiles_total;
      cur.obs_total += b.n;
      cur.tiles_total += b.ntiles + 1;
      cur.sums_elems += elems;
      cur.nf_total += b.nf;
      cur.items += (int64_t)b.ntc * b.nf;
      cur.Hs = std::max(cur.Hs, b.Hc);
      cur.c1 = c + 1;
    }
    chunks.push_back(cur);
  }
  // ---- batched step (a): per chunk, the curves sorted by grid length and
  //      cut into groups whose grids fit the grid buffer (twice the chunk
  //      budget; a larger single curve gets a group of its own).  sa_curve /
  //      sa_goff: the curve and grid offset of each StepACurve, group after
  //      group; sa_pref: each group's spread prefix, then its gather prefix.
  std::vector<int64_t> sa_curve, sa_goff, sa_pref;
  int64_t max_group_grid = 0;
  int max_classes = 1;
  {
    const int64_t budget = (int64_t)(2 * P->chunk_bytes / P->csz);
    for (BChunk& ch : chunks) {
      std::vector<int64_t> order;
      for (int64_t c = ch.c0; c < ch.c1; ++c) order.push_back(c);
      std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return cv[(size_t)a].ngrid < cv[(size_t)b].ngrid;
      });
      BSub cur{};
      bool open = false;
      auto close = [&]() {
        cur.pref_first = (int64_t)sa_pref.size();
        int64_t acc = 0;
        sa_pref.push_back(0);
        for (int i = 0; i < cur.ncurves; ++i) {
          acc += cv[(size_t)sa_curve[(size_t)(cur.desc_first + i)]].ntiles;
          sa_pref.push_back(acc);
        }
        cur.spread_tiles = acc;
        acc = 0;
        sa_pref.push_back(0);
        for (int i = 0; i < cur.ncurves; ++i) {
          const BCurve& b = cv[(size_t)sa_curve[(size_t)(cur.desc_first + i)]];
          acc += gather_tile_count(!P->mixed, b.k0, b.nf, b.Hc);
          sa_pref.push_back(acc);
        }
        cur.gather_tiles = acc;
        max_group_grid = std::max(max_group_grid, cur.grid_elems);
        max_classes = std::max(max_classes, (int)cur.classes.size());
        ch.subs.push_back(cur);
        open = false;
      };
      for (int64_t c : order) {
        const BCurve& b = cv[(size_t)c];
        if (open && cur.grid_elems + b.ngrid > budget) close();
        if (!open) {
          cur = BSub{};
          cur.desc_first = (int64_t)sa_curve.size();
          cur.ncurves = 0;
          open = true;
        }
        if (cur.classes.empty() || cur.classes.back().n != b.ngrid)
          cur.classes.push_back(BFftClass{b.ngrid, cur.grid_elems, 0});
        cur.classes.back().count++;
        sa_curve.push_back(c);
        sa_goff.push_back(cur.grid_elems);
        cur.grid_elems += b.ngrid;
        cur.ncurves++;
      }
      if (open) close();
    }
  }

  // ---- templates (grouped by H) and the segment tables of every chunk
  std::vector<HGroup> groups;
  std::vector<int> pos_of;
  FTP_CK(reset_call(P));
  if (!feat_only) {
    st = upload_templates(P, bank, nbank, &groups, &pos_of);
    if (st != FTP_OK) return st;
  }
  const RootsKind kind = P->mixed ? ROOTS_MIXED : ROOTS_FP64;
  std::vector<RootsSeg> segs;
  std::vector<int64_t> units;
  std::vector<int> cseg;
  size_t max_chunk_curves = 0;
  int64_t max_sums_elems = 0, max_nf_total = 0, max_units = 0;
  for (BChunk& ch : chunks) {
    const int64_t ncc = ch.c1 - ch.c0;
    max_chunk_curves = std::max(max_chunk_curves, (size_t)ncc);
    max_sums_elems = std::max(max_sums_elems, ch.sums_elems);
    max_nf_total = std::max(max_nf_total, ch.nf_total);
    // (H, first, count) of each launch: one per template group (whole bank),
    // or one per distinct H of the chunk's curves (one template per curve)
    std::vector<HGroup> lg;
    if (feat_only) {
      // no exact solve
    } else if (tpl_of_curve) {
      std::vector<int> hs;
      for (int64_t c = ch.c0; c < ch.c1; ++c) hs.push_back(cv[(size_t)c].Ht);
      std::sort(hs.begin(), hs.end());
      hs.erase(std::unique(hs.begin(), hs.end()), hs.end());
      for (int h : hs) lg.push_back({h, 0, 1});
    } else {
      lg = groups;
    }
    for (const HGroup& g : lg) {
      const int ngw = roots_items_per_unit(kind, g.H);
      if (ngw <= 0) return FTP_ERR_UNSUPPORTED;
      BLaunch L{};
      L.H = g.H;
      L.ntpl = g.count;
      L.Hs = ch.Hs;
      L.seg_first = (int64_t)segs.size();
      L.units_first = (int64_t)units.size();
      L.cseg_first = (int64_t)cseg.size();
      int64_t acc = 0;
      for (int64_t c = ch.c0; c < ch.c1; ++c) {
        const BCurve& b = cv[(size_t)c];
        if (tpl_of_curve && b.Ht != g.H) {
          cseg.push_back(-1);
          continue;
        }
        RootsSeg sg{};
        sg.sums_off = b.sums_off;
        sg.nf_pad = b.nf_pad;
        sg.nf = b.nf;
        sg.out_off = b.out_off;
        sg.redo_base = b.redo_base;
        sg.Hs = b.Hc;
        sg.curve = (int32_t)(c - ch.c0);
        sg.tpl_first = tpl_of_curve ? pos_of[b.tpl] : g.first;
        sg.ntpl = tpl_of_curve ? 1 : g.count;
        sg.row_first = tpl_of_curve ? -1 : g.first;
        cseg.push_back((int)(segs.size() - L.seg_first));
        segs.push_back(sg);
        units.push_back(acc);
        acc += (b.nf + ngw - 1) / ngw * sg.ntpl;
      }
      units.push_back(acc);
      L.nseg = (int)(segs.size() - L.seg_first);
      L.units = acc;
      max_units = std::max(max_units, acc);
      ch.launches.push_back(L);
    }
  }
  std::vector<CurveDesc> curves((size_t)ncurves);
  for (int64_t c = 0; c < ncurves; ++c) {
    const BCurve& b = cv[(size_t)c];
    curves[(size_t)c] = CurveDesc{b.t, b.y, b.dy, b.n, b.df, b.k0, b.redo_base, b.nf,
                                  b.out_off, b.Hc, b.ntc};
  }
  // screening / features: per-curve descriptors and, per chunk, the row
  // offsets of its curves (chunk q's ncurves + 1 entries start at c0 + q)
  std::vector<ScreenCurve> scurves;
  std::vector<int64_t> rowoff;
  if (scr) {
    scurves.resize((size_t)ncurves);
    for (size_t q = 0; q < chunks.size(); ++q) {
      int64_t items = 0;
      for (int64_t c = chunks[q].c0; c < chunks[q].c1; ++c) {
        const BCurve& b = cv[(size_t)c];
        ScreenCurve& sc = scurves[(size_t)c];
        sc.sums_off = b.sums_off;
        sc.nf_pad = b.nf_pad;
        sc.nf = b.nf;
        sc.row_base = b.redo_base;
        sc.out_row = feat_only ? scr->feat_row[c] : b.redo_base;
        sc.nobs = b.n;
        sc.item_base = items;
        sc.out_off = b.out_off;
        sc.Hs = b.Hc;
        sc.curve = (int32_t)(c - chunks[q].c0);
        items += (int64_t)b.ntc * b.nf;
        rowoff.push_back(b.redo_base);
      }
      rowoff.push_back(chunks[q].nf_total);
    }
  }
  // one descriptor blob: segs | units | curves | curve -> segment maps |
  // screening curves | row offsets
  auto al64 = [](size_t x) { return (x + 63) / 64 * 64; };
  const size_t off_units = al64(segs.size() * sizeof(RootsSeg));
  const size_t off_curves = off_units + al64(units.size() * sizeof(int64_t));
  const size_t off_cseg = off_curves + al64(curves.size() * sizeof(CurveDesc));
  const size_t off_scur = off_cseg + al64(cseg.size() * sizeof(int));
  const size_t off_rowoff = off_scur + al64(scurves.size() * sizeof(ScreenCurve));
  std::vector<PrepCurve> prep((size_t)ncurves);
  int64_t max_obs_total = 0, max_tiles_total = 0;
  for (const BChunk& ch : chunks) {
    max_obs_total = std::max(max_obs_total, ch.obs_total);
    max_tiles_total = std::max(max_tiles_total, ch.tiles_total);
    for (int64_t c = ch.c0; c < ch.c1; ++c) {
      const BCurve& b = cv[(size_t)c];
      prep[(size_t)c] = PrepCurve{b.t, b.y, b.dy, b.n, b.df, b.ngrid, b.ntiles, b.obs_base,
                                  b.tile_base};
    }
  }
  const size_t off_prep = off_rowoff + al64(rowoff.size() * sizeof(int64_t));
  const size_t off_stepa = off_prep + al64(prep.size() * sizeof(PrepCurve));
  const size_t off_pref = off_stepa + al64(sa_curve.size() * sizeof(StepACurve));
  const size_t blob = off_pref + al64(sa_pref.size() * sizeof(int64_t));

  // ---- workspace (growing it drops a captured graph)
  st = grow_dev(reinterpret_cast<unsigned char**>(&P->d_bsums), &P->bsums_cap,
                (size_t)max_sums_elems * P->csz, &grew);
  if (st == FTP_OK) st = grow_dev(&P->d_bmom, &P->bmom_cap, max_chunk_curves * MO_WORDS, &grew);
  if (st == FTP_OK) st = grow_dev(&P->d_bmark, &P->bmark_cap, (size_t)max_nf_total, &grew);
  if (st == FTP_OK) st = grow_dev(&P->d_bdesc, &P->bdesc_cap, blob, &grew);
  if (st == FTP_OK)
    st = grow_dev(reinterpret_cast<unsigned char**>(&P->d_bgrid), &P->bgrid_cap,
                  (size_t)max_group_grid * P->csz, &grew);
  // preparation scratch: cells (unsorted, sorted), fractions, coefficients,
  // tile counters and offsets of the largest chunk
  const size_t rsz = P->csz / 2;
  const size_t mo = (size_t)std::max<int64_t>(max_obs_total, 1);
  const size_t mt = (size_t)std::max<int64_t>(max_tiles_total, 1);
  const size_t pb_cell = 0, pb_frac = al64(2 * mo * sizeof(int));
  const size_t pb_coef = pb_frac + al64(2 * mo * rsz);
  const size_t pb_tile = pb_coef + al64(2 * mo * P->csz);
  const size_t pb_end = pb_tile + al64(2 * mt * sizeof(int));
  if (st == FTP_OK) st = grow_dev(&P->d_bprep, &P->bprep_cap, pb_end, &grew);
  if (st == FTP_OK && !P->d_blist) {
    grew = true;
    if (dalloc(&P->d_blist, kBatchRedoCap) != FTP_OK ||
        dalloc(&P->d_bslot_curve, kBatchRedoCap) != FTP_OK || dalloc(&P->d_bcount, 1) != FTP_OK ||
        dalloc(&P->d_bredo_sums, (size_t)3 * P->max_H * kBatchRedoStride) != FTP_OK)
      st = FTP_ERR_OOM;
  }
  if (st == FTP_OK && scr && scr->mlp) {
    const int nfeat = 2 * Hf + 2;
    st = grow_dev(&P->d_bfeat, &P->bfeat_cap, (size_t)max_nf_total * nfeat, &grew);
    if (st == FTP_OK) st = grow_dev(&P->d_bscore, &P->bscore_cap, (size_t)max_nf_total, &grew);
    if (st == FTP_OK) st = grow_dev(&P->d_bsel, &P->bsel_cap, (size_t)max_nf_total, &grew);
    if (st == FTP_OK) st = grow_dev(&P->d_bulist, &P->bulist_cap, (size_t)max_units, &grew);
    if (st == FTP_OK && !P->d_bucount) {
      grew = true;
      st = dalloc(&P->d_bucount, 1);
    }
  }
  if (st == FTP_OK && !out_dev) {
    st = grow_dev(&P->d_bout, &P->bout_cap, (size_t)4 * extent, &grew);
    if (st == FTP_OK && flags) st = grow_dev(&P->d_bflags, &P->bflags_cap, (size_t)extent, &grew);
  }
  if (st != FTP_OK) return st;
  if (!P->h_bdesc || P->hbdesc_cap < blob) {
    if (P->h_bdesc) cudaFreeHost(P->h_bdesc);
    P->h_bdesc = nullptr;
    P->hbdesc_cap = 0;
    if (cudaMallocHost(&P->h_bdesc, blob) != cudaSuccess) return FTP_ERR_OOM;
    P->hbdesc_cap = blob;
  }
  memcpy(P->h_bdesc, segs.data(), segs.size() * sizeof(RootsSeg));
  memcpy(P->h_bdesc + off_units, units.data(), units.size() * sizeof(int64_t));
  memcpy(P->h_bdesc + off_curves, curves.data(), curves.size() * sizeof(CurveDesc));
  memcpy(P->h_bdesc + off_cseg, cseg.data(), cseg.size() * sizeof(int));
  memcpy(P->h_bdesc + off_scur, scurves.data(), scurves.size() * sizeof(ScreenCurve));
  memcpy(P->h_bdesc + off_rowoff, rowoff.data(), rowoff.size() * sizeof(int64_t));
  PrepBufs pbufs{};
  pbufs.curves = reinterpret_cast<const PrepCurve*>(P->d_bdesc + off_prep);
  pbufs.cell = reinterpret_cast<int*>(P->d_bprep + pb_cell);
  pbufs.cell_s = pbufs.cell + mo;
  pbufs.frac = P->d_bprep + pb_frac;
  pbufs.frac_s = P->d_bprep + pb_frac + mo * rsz;
  pbufs.coef = P->d_bprep + pb_coef;
  pbufs.coef_s = P->d_bprep + pb_coef + mo * P->csz;
  pbufs.tile_cnt = reinterpret_cast<int*>(P->d_bprep + pb_tile);
  pbufs.tile_off = pbufs.tile_cnt + mt;
  memcpy(P->h_bdesc + off_prep, prep.data(), prep.size() * sizeof(PrepCurve));
  {
    std::vector<StepACurve> sa(sa_curve.size());
    for (size_t i = 0; i < sa.size(); ++i) {
      const BCurve& b = cv[(size_t)sa_curve[i]];
      StepACurve& d = sa[i];
      d.tile_off = pbufs.tile_off + b.tile_base;
      d.cell_s = pbufs.cell_s + b.obs_base;
      d.frac_s = static_cast<const unsigned char*>(pbufs.frac_s) + (size_t)b.obs_base * rsz;
      d.coef_s = static_cast<const unsigned char*>(pbufs.coef_s) + (size_t)b.obs_base * P->csz;
      d.grid = static_cast<unsigned char*>(P->d_bgrid) + (size_t)sa_goff[i] * P->csz;
      d.sums = static_cast<unsigned char*>(P->d_bsums) + (size_t)b.sums_off * P->csz;
      d.ngrid = b.ngrid;
      d.ntiles = b.ntiles;
      d.k0 = b.k0;
      d.nf = b.nf;
      d.nf_pad = b.nf_pad;
      d.Hs = b.Hc;
      d.pad_ = 0;
    }
    memcpy(P->h_bdesc + off_stepa, sa.data(), sa.size() * sizeof(StepACurve));
    memcpy(P->h_bdesc + off_pref, sa_pref.data(), sa_pref.size() * sizeof(int64_t));
  }
  // step (a) lanes, then every batched FFT of every group on the lane that
  // runs it (before any capture: making a plan may resize, and so
  // synchronise, a work area)
  st = ensure_lanes(P, std::min(P->sum_lanes, max_classes), &grew);
  if (st != FTP_OK) return st;
  for (const BChunk& ch : chunks)
    for (const BSub& sb : ch.subs) {
      const int used = fft_lanes_used(P, sb);
      for (size_t k = 0; k < sb.classes.size(); ++k) {
        const int l = (int)(k % (size_t)used);
        cufftHandle h;
        st = get_fft_many(P, l == 0 ? P->l0 : *P->xlanes[l - 1], sb.classes[k].n,
                          sb.classes[k].count, &h);
        if (st != FTP_OK) return st;
      }
    }
  if (P->timing) {
    while (P->bev.size() < 5 * chunks.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return FTP_ERR_CUDA;
      P->bev.push_back(e);
    }
  }
  if (grew && P->graph_exec) {
    cudaGraphExecDestroy(P->graph_exec);
    P->graph_exec = nullptr;
    P->graph_key = 0;
  }

  // ---- eager uploads: descriptors (and host observations)
  cudaStream_t s = P->stream;
  FTP_CK(cudaMemcpyAsync(P->d_bdesc, P->h_bdesc, blob, cudaMemcpyHostToDevice, s));
  if (!in_dev) {
    FTP_CK(cudaMemcpyAsync(P->d_bobs, t + o_lo, sizeof(double) * nobs_all, cudaMemcpyHostToDevice, s));
    FTP_CK(cudaMemcpyAsync(P->d_bobs + nobs_all, y + o_lo, sizeof(double) * nobs_all,
                           cudaMemcpyHostToDevice, s));
    FTP_CK(cudaMemcpyAsync(P->d_bobs + 2 * nobs_all, dy + o_lo, sizeof(double) * nobs_all,
                           cudaMemcpyHostToDevice, s));
  }
  const RootsSeg* d_segs = reinterpret_cast<const RootsSeg*>(P->d_bdesc);
  const int64_t* d_units = reinterpret_cast<const int64_t*>(P->d_bdesc + off_units);
  const CurveDesc* d_curves = reinterpret_cast<const CurveDesc*>(P->d_bdesc + off_curves);
  const int* d_cseg = reinterpret_cast<const int*>(P->d_bdesc + off_cseg);
  const ScreenCurve* d_scur = reinterpret_cast<const ScreenCurve*>(P->d_bdesc + off_scur);
  const int64_t* d_rowoff = reinterpret_cast<const int64_t*>(P->d_bdesc + off_rowoff);
  const StepACurve* d_stepa = reinterpret_cast<const StepACurve*>(P->d_bdesc + off_stepa);
  const int64_t* d_pref = reinterpret_cast<const int64_t*>(P->d_bdesc + off_pref);
  double* o[4] = {power, theta1, theta2, theta3};
  uint8_t* of = flags;
  if (!out_dev) {
    for (int i = 0; i < 4; ++i) o[i] = P->d_bout + (size_t)i * extent;
    of = flags ? P->d_bflags : nullptr;
  }

  // ---- the device work: eager, captured, or a replay of the captured graph
  P->in_batch = true;
  struct EndBatch {
    ftp_plan_t p;
    ~EndBatch() { p->in_batch = false; }
  } end_batch{P};
  int launches = 0;
  const bool graphable = P->use_graph && !P->timing && in_dev && out_dev;
  uint64_t key = 0;
  if (graphable) {
    key = 1469598103934665603ull;
    const void* ptrs[] = {t, y, dy, power, theta1, theta2, theta3, flags};
    key = fnv(key, ptrs, sizeof(ptrs));
    key = fnv(key, &ncurves, sizeof(ncurves));
    key = fnv(key, obs_off, sizeof(int64_t) * (size_t)(ncurves + 1));
    key = fnv(key, grids, sizeof(ftp_grid) * (size_t)ncurves);
    key = fnv(key, out_off, sizeof(int64_t) * (size_t)ncurves);
    if (tpl_of_curve) key = fnv(key, tpl_of_curve, sizeof(int32_t) * (size_t)ncurves);
    key = fnv(key, &nbank, sizeof(nbank));
    key = fnv(key, P->h_alpha, sizeof(double2) * kMaxH * nbank);
    key = fnv(key, P->h_rows, sizeof(int) * nbank);
    key = fnv(key, &P->chunk_bytes, sizeof(P->chunk_bytes));
    key = fnv(key, &P->sum_lanes, sizeof(P->sum_lanes));
    key = fnv(key, &P->roots_ctas_per_sm, sizeof(P->roots_ctas_per_sm));
    key = fnv(key, &P->positive_only, sizeof(P->positive_only));
    const int solver[] = {P->maxit, P->redo_maxit, P->wait_polls, P->inject};
    key = fnv(key, solver, sizeof(solver));
    if (scr) {
      const void* sp[] = {scr->feat_out, scr->mlp, scr->moments_out};
      key = fnv(key, sp, sizeof(sp));
      key = fnv(key, &scr->Hf, sizeof(scr->Hf));
      key = fnv(key, &scr->top_frac, sizeof(scr->top_frac));
      key = fnv(key, &scr->nbr, sizeof(scr->nbr));
      if (scr->feat_row) key = fnv(key, scr->feat_row, sizeof(int64_t) * (size_t)ncurves);
    }
    if (key == 0) key = 1;
  }
  P->last_graph = 0;
  if (graphable && P->graph_exec && key == P->graph_key) {
    FTP_CK(cudaGraphLaunch(P->graph_exec, s));
    launches = P->graph_launches;
    P->last_graph = 2;
  } else if (graphable && key == P->eager_key) {
    // second identical call: capture the device work once, then launch it
    cudaGraph_t graph = nullptr;
    FTP_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    st = enqueue_batch_device(P, cv, chunks, d_stepa, d_pref, d_segs, d_units, d_curves, d_cseg,
                              o, of, extent, scr, d_scur, d_rowoff, pbufs, &launches);
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    cudaGraphExec_t exec = nullptr;
    if (st == FTP_OK && ce == cudaSuccess && graph &&
        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
      if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
      P->graph_exec = exec;
      P->graph_key = key;
      P->graph_launches = launches;
      cudaGraphDestroy(graph);
      FTP_CK(cudaGraphLaunch(P->graph_exec, s));
      P->last_graph = 1;
    } else {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      if (st != FTP_OK) return st;
      P->eager_key = 0;  // capture failed: stay eager for this call pattern
      launches = 0;
      st = enqueue_batch_device(P, cv, chunks, d_stepa, d_pref, d_segs, d_units, d_curves,
                                d_cseg, o, of, extent, scr, d_scur, d_rowoff, pbufs, &launches);
      if (st != FTP_OK) return st;
    }
  } else {
    st = enqueue_batch_device(P, cv, chunks, d_stepa, d_pref, d_segs, d_units, d_curves, d_cseg,
                              o, of, extent, scr, d_scur, d_rowoff, pbufs, &launches);
    if (st != FTP_OK) return st;
    if (graphable) P->eager_key = key;
  }

  // ---- host outputs: one copy when the curves' blocks tile [lo, extent)
  if (!out_dev) {
    std::vector<std::pair<int64_t, int64_t>> blocks((size_t)ncurves);
    for (int64_t c = 0; c < ncurves; ++c)
      blocks[(size_t)c] = {out_off[c], out_off[c] + (int64_t)cv[(size_t)c].ntc * cv[(size_t)c].nf};
    std::sort(blocks.begin(), blocks.end());
    bool tiled = true;
    for (size_t i = 1; i < blocks.size(); ++i) tiled = tiled && blocks[i].first == blocks[i - 1].second;
    double* dsto[4] = {power, theta1, theta2, theta3};
    auto copy_range = [&](int64_t a0, int64_t a1) -> cudaError_t {
      cudaError_t e = cudaSuccess;
      for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(dsto[i] + a0, o[i] + a0, sizeof(double) * (size_t)(a1 - a0),
                            cudaMemcpyDefault, s);
      if (e == cudaSuccess && flags)
        e = cudaMemcpyAsync(flags + a0, of + a0, (size_t)(a1 - a0), cudaMemcpyDefault, s);
      return e;
    };
    if (tiled) {
      FTP_CK(copy_range(blocks.front().first, blocks.back().second));
    } else {
      for (const auto& b : blocks) FTP_CK(copy_range(b.first, b.second));
    }
  }
  P->last_launches = launches;
  P->last_chunks = (int64_t)chunks.size();
  st = finish(P);
  if (P->timing) {
    for (int i = 0; i < 6; ++i) P->stage_ms[i] = 0.f;
    for (size_t q = 0; q < chunks.size(); ++q) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, P->bev[5 * q], P->bev[5 * q + 1]) == cudaSuccess)
        P->stage_ms[0] += ms;
      if (cudaEventElapsedTime(&ms, P->bev[5 * q + 1], P->bev[5 * q + 2]) == cudaSuccess)
        P->stage_ms[1] += ms;
      if (cudaEventElapsedTime(&ms, P->bev[5 * q + 2], P->bev[5 * q + 3]) == cudaSuccess)
        P->stage_ms[4] += ms;
      if (cudaEventElapsedTime(&ms, P->bev[5 * q + 3], P->bev[5 * q + 4]) == cudaSuccess)
        P->stage_ms[5] += ms;
    }
    cudaGetLastError();
  }
  return st;
}

}  // namespace

extern "C" {

const char* ftp_status_string(ftp_status s) {
  switch (s) {
    case FTP_OK: return "ok";
    case FTP_ERR_INVALID_ARG: return "invalid argument";
    case FTP_ERR_ZERO_VARIANCE: return "zero variance of y: periodogram undefined";
    case FTP_ERR_MIXED_ZERO_SIGMA: return "mixed zero and non-zero uncertainties";
    case FTP_ERR_NONFINITE: return "non-finite or negative input";
    case FTP_ERR_OOM: return "device out of memory";
    case FTP_ERR_CUDA: return "CUDA or cuFFT error";
    case FTP_ERR_TIMEOUT: return "bounded device wait timed out";
    case FTP_ERR_UNSUPPORTED: return "request exceeds the plan";
  }
  return "unknown status";
}

void ftp_destroy(ftp_plan_t P) {
  if (!P) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  for (SumLane* L : P->xlanes) {
    free_lane(L);
    delete L;
  }
  P->xlanes.clear();
  free_lane(&P->l0);
  if (P->fork) cudaEventDestroy(P->fork);
  void* dptrs[] = {P->d_in, P->d_moments, P->d_mom_scratch, P->d_status, P->d_counters, P->d_queue, P->d_redo_list,
                   P->d_redo_mark, P->d_redo_count, P->d_redo_sums, P->d_tile_count, P->d_tile_off,
                   P->d_cursor, P->d_cell, P->d_cell_s, P->d_frac, P->d_frac_s, P->d_coef,
                   P->d_coef_s, P->d_grid, P->d_sums, P->d_alpha, P->d_rows, P->d_row0, P->d_out,
                   P->d_flags};
  for (void* p : dptrs)
    if (p) cudaFree(p);
  void* bptrs[] = {P->d_bsums, P->d_bmom, P->d_bobs, P->d_bout, P->d_bflags, P->d_bmark,
                   P->d_blist, P->d_bslot_curve, P->d_bcount, P->d_bredo_sums, P->d_bdesc,
                   P->d_bfeat, P->d_bscore, P->d_bsel, P->d_bulist, P->d_bucount,
                   P->d_mb, P->d_mbflags, P->d_mbpow, P->d_shsums, P->d_shmisc,
                   P->d_shalpha, P->d_shcoef, P->d_bprep};
  for (void* p : bptrs)
    if (p) cudaFree(p);
  if (P->h_bdesc) cudaFreeHost(P->h_bdesc);
  for (auto& e : P->bev)
    if (e) cudaEventDestroy(e);
  if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
  if (P->h_status) cudaFreeHost(P->h_status);
  if (P->h_counters) cudaFreeHost(P->h_counters);
  if (P->h_redo_count) cudaFreeHost(P->h_redo_count);
  if (P->h_alpha) cudaFreeHost(P->h_alpha);
  if (P->h_rows) cudaFreeHost(P->h_rows);
  for (auto& e : P->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : P->fev)
    if (e) cudaEventDestroy(e);
  if (P->own_stream && P->stream) cudaStreamDestroy(P->stream);
  delete P;
  cudaSetDevice(prev);
}

ftp_status ftp_plan(ftp_plan_t* out, int64_t max_nobs, int max_H, ftp_grid grid, int max_templates,
                    ftp_precision prec, int device, void* cuda_stream) {
  if (!out) return FTP_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_nobs < 2 || max_H < 1 || max_templates < 1) return FTP_ERR_INVALID_ARG;
  if (max_H > FTP_MAX_H) return FTP_ERR_UNSUPPORTED;
  if (prec != FTP_FP64 && prec != FTP_MIXED) return FTP_ERR_INVALID_ARG;
  const ftp_status gs = check_grid(grid);
  if (gs != FTP_OK) return gs;
  if (max_nobs > ((int64_t)1 << 30)) return FTP_ERR_UNSUPPORTED;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return FTP_ERR_CUDA;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return FTP_ERR_CUDA;

  ftp_plan_s* P = new (std::nothrow) ftp_plan_s();
  if (!P) return FTP_ERR_OOM;
  P->device = device;
  P->prec = prec;
  P->mixed = (prec == FTP_MIXED);
  P->max_nobs = max_nobs;
  P->max_H = max_H;
  P->grid = grid;
  P->max_templates = max_templates;
  // Kaiser-Bessel half-width and oversampling.  In FP32 a wider window is
  // not better: its larger beta widens the range the deconvolution divides
  // by, and the FFT's rounding is amplified with it.  Largest error of the
  // FP32 sums against direct FP64 sums (relative to sum w = 1) over the long
  // lightcurve, the N = 1e5 bank lightcurve and survey curves: sigma 1.5,
  // m = 4: 1.1e-6 (bank); sigma 1.5, m = 5: 7.8e-7; sigma 1.25, m = 5:
  // 5.0e-7; sigma 1.25, m = 6: 1.4e-6.  The mixed path takes sigma 1.25,
  // m = 5 (the smallest worst case, and a 17 % smaller grid than sigma 1.5);
  // the FP64 path keeps sigma = 2, m = 8.
  P->m = P->mixed ? 5 : 8;
  P->sigma = P->mixed ? 1.25 : 2.0;
  P->beta = kb_beta(P->m, P->sigma);
  P->rsz = P->mixed ? sizeof(float) : sizeof(double);
  P->csz = 2 * P->rsz;
  P->maxit = P->mixed ? 60 : 80;
  P->polish_steps = 1;
  cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, device);
  const int64_t J = 2 * (int64_t)max_H * (grid.k0 + grid.nf - 1);
  P->ngrid = grid_len(J, P->sigma, &P->ntiles);
  P->nf_pad = (grid.nf + 255) / 256 * 256;

  ftp_status st = FTP_OK;
  auto fail = [&](ftp_status s) {
    ftp_destroy(P);
    cudaSetDevice(prev);
    return s;
  };
  if (P->ngrid >= ((int64_t)1 << 31)) return fail(FTP_ERR_UNSUPPORTED);
  if (cuda_stream) {
    P->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(FTP_ERR_CUDA);
    P->own_stream = true;
  }
  const size_t nobs = (size_t)max_nobs;
  const size_t nout = (size_t)max_templates * (size_t)grid.nf;
#define FTP_AL(ptr, count)                  \
  do {                                      \
    st = dalloc(&(ptr), (count));           \
    if (st != FTP_OK) return fail(st);      \
  } while (0)
  FTP_AL(P->d_in, 3 * nobs);
  FTP_AL(P->d_moments, MO_WORDS);
  FTP_AL(P->d_mom_scratch, kMomentScratchBytes);
  FTP_AL(P->d_status, ST_WORDS);
  FTP_AL(P->d_counters, CNT_WORDS);
  FTP_AL(P->d_queue, 2);  // one work counter per roots phase
  FTP_AL(P->d_redo_list, (size_t)grid.nf);
  FTP_AL(P->d_redo_mark, (size_t)grid.nf);
  FTP_AL(P->d_redo_count, 1);
  FTP_AL(P->d_redo_sums, (size_t)3 * max_H * P->nf_pad);
  FTP_AL(P->d_tile_count, (size_t)P->ntiles);
  FTP_AL(P->d_tile_off, (size_t)P->ntiles + 1);
  FTP_AL(P->d_cursor, (size_t)P->ntiles);
  FTP_AL(P->d_cell, nobs);
  FTP_AL(P->d_cell_s, nobs);
  unsigned char* tmp = nullptr;
  FTP_AL(tmp, nobs * P->rsz);
  P->d_frac = tmp;
  FTP_AL(tmp, nobs * P->rsz);
  P->d_frac_s = tmp;
  FTP_AL(tmp, nobs * P->csz);
  P->d_coef = tmp;
  FTP_AL(tmp, nobs * P->csz);
  P->d_coef_s = tmp;
  FTP_AL(tmp, (size_t)P->ngrid * P->csz);
  P->d_grid = tmp;
  const size_t sums_bytes = (size_t)3 * max_H * P->nf_pad * P->csz;
  FTP_AL(tmp, sums_bytes);
  P->d_sums = tmp;
  FTP_AL(P->d_alpha, (size_t)max_templates * kMaxH);
  FTP_AL(P->d_rows, (size_t)max_templates);
  FTP_AL(P->d_row0, 1);
  FTP_AL(P->d_out, 4 * nout);
  FTP_AL(P->d_flags, nout);
#undef FTP_AL
  if (cudaMemset(P->d_sums, 0, sums_bytes) != cudaSuccess ||
      cudaMemset(P->d_mom_scratch, 0, kMomentScratchBytes) != cudaSuccess)
    return fail(FTP_ERR_CUDA);
  if (cudaMemset(P->d_status, 0, sizeof(int) * ST_WORDS) != cudaSuccess ||
      cudaMemset(P->d_row0, 0, sizeof(int)) != cudaSuccess)
    return fail(FTP_ERR_CUDA);
  if (cudaMallocHost(&P->h_status, sizeof(int) * ST_WORDS) != cudaSuccess ||
      cudaMallocHost(&P->h_counters, sizeof(unsigned long long) * CNT_WORDS) != cudaSuccess ||
      cudaMallocHost(&P->h_redo_count, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&P->h_alpha, sizeof(double2) * kMaxH * max_templates) != cudaSuccess ||
      cudaMallocHost(&P->h_rows, sizeof(int) * max_templates) != cudaSuccess)
    return fail(FTP_ERR_OOM);
  for (auto& e : P->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(FTP_ERR_CUDA);
  P->l0.s = P->stream;
  P->l0.mom_scratch = P->d_mom_scratch;
  P->l0.tile_count = P->d_tile_count;
  P->l0.tile_off = P->d_tile_off;
  P->l0.cursor = P->d_cursor;
  P->l0.cell = P->d_cell;
  P->l0.cell_s = P->d_cell_s;
  P->l0.frac = P->d_frac;
  P->l0.frac_s = P->d_frac_s;
  P->l0.coef = P->d_coef;
  P->l0.coef_s = P->d_coef_s;
  P->l0.grid = P->d_grid;
  cufftHandle h;
  st = get_fft(P, P->ngrid, &h);
  if (st != FTP_OK) return fail(st);
  cudaSetDevice(prev);
  *out = P;
  return FTP_OK;
}

ftp_status ftp_plan_info(ftp_plan_t P, int64_t* grid_len_out, int* half_width, int64_t* ntiles,
                         int* last_launches) {
  if (!P) return FTP_ERR_INVALID_ARG;
  if (grid_len_out) *grid_len_out = P->ngrid;
  if (half_width) *half_width = P->m;
  if (ntiles) *ntiles = P->ntiles;
  if (last_launches) *last_launches = P->last_launches;
  return FTP_OK;
}

ftp_status ftp_solver_stats(ftp_plan_t P, int64_t* items, double* mean_iterations,
                            int64_t* nonconverged, int64_t* resolved,
                            int64_t* resolved_nonconverged, int64_t* still_nonconverged) {
  if (!P) return FTP_ERR_INVALID_ARG;
  const unsigned long long* c = P->h_counters;
  const unsigned long long n = c ? c[CNT_ITEMS] : 0;
  if (items) *items = (int64_t)n;
  if (mean_iterations) *mean_iterations = n ? (double)c[CNT_ITERS] / (double)n : 0.0;
  if (nonconverged) *nonconverged = n ? (int64_t)c[CNT_NONCONV] : 0;
  if (resolved) *resolved = n ? (int64_t)c[CNT_REDO] : 0;
  if (resolved_nonconverged) *resolved_nonconverged = n ? (int64_t)c[CNT_REDO_NC] : 0;
  if (still_nonconverged) *still_nonconverged = n ? (int64_t)c[CNT_NC_FINAL] : 0;
  return FTP_OK;
}

ftp_status ftp_set_solver_limits(ftp_plan_t P, int maxit, int redo_maxit, int wait_polls) {
  if (!P) return FTP_ERR_INVALID_ARG;
  if (maxit < 0 || maxit > 100000 || redo_maxit < 0 || redo_maxit > 100000 || wait_polls < 0)
    return FTP_ERR_INVALID_ARG;
  P->maxit = maxit ? maxit : (P->mixed ? 60 : 80);
  P->redo_maxit = redo_maxit ? redo_maxit : kRedoMaxit;
  P->wait_polls = wait_polls;
  return FTP_OK;
}

ftp_status ftp_set_fault_injection(ftp_plan_t P, int mode) {
  if (!P || mode < 0 || mode > 1) return FTP_ERR_INVALID_ARG;
  P->inject = mode;
  return FTP_OK;
}

ftp_status ftp_set_timing(ftp_plan_t P, int enable) {
  if (!P) return FTP_ERR_INVALID_ARG;
  P->timing = enable != 0;
  if (P->timing && !P->fev[0]) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(P->device);
    bool ok = true;
    for (auto& e : P->fev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    cudaSetDevice(prev);
    if (!ok) return FTP_ERR_CUDA;
  }
  P->fev_used = 0;
  return FTP_OK;
}

ftp_status ftp_roots_first_phase_ms(ftp_plan_t P, float* ms) {
  if (!P || !ms) return FTP_ERR_INVALID_ARG;
  *ms = P->first_phase_ms;
  return FTP_OK;
}

ftp_status ftp_stage_times(ftp_plan_t P, float* ms6) {
  if (!P || !ms6) return FTP_ERR_INVALID_ARG;
  for (int i = 0; i < 6; ++i) ms6[i] = P->stage_ms[i];
  return FTP_OK;
}

ftp_status ftp_sums(ftp_plan_t P, const double* t, const double* y, const double* dy,
                    int64_t nobs, int H_sums, void* sums_out, double* moments_out) {
  ftp_status st = check_obs(P, t, y, dy, nobs);
  if (st != FTP_OK) return st;
  if (!sums_out || H_sums < 1) return FTP_ERR_INVALID_ARG;
  if (H_sums > P->max_H) return FTP_ERR_UNSUPPORTED;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  FTP_CK(reset_call(P));
  const double *dt, *dyv, *ddy;
  st = stage_obs(P, t, y, dy, nobs, &dt, &dyv, &ddy);
  if (st != FTP_OK) return st;
  int launches = 0;
  st = run_sums_plan(P, dt, dyv, ddy, nobs, H_sums, &launches);
  if (st != FTP_OK) return st;
  ev_rec(P, 5);
  const size_t row = (size_t)P->grid.nf * P->csz;
  FTP_CK(cudaMemcpy2DAsync(sums_out, row, P->d_sums, (size_t)P->nf_pad * P->csz, row,
                           (size_t)3 * H_sums, cudaMemcpyDefault, P->stream));
  if (moments_out)
    FTP_CK(cudaMemcpyAsync(moments_out, P->d_moments, 2 * sizeof(double), cudaMemcpyDefault,
                           P->stream));
  P->last_launches = launches;
  return finish(P);
}

ftp_status ftp_periodogram(ftp_plan_t P, const double* t, const double* y, const double* dy,
                           int64_t nobs, const ftp_template* tpl, int ntemplates, double* power,
                           double* theta1, double* theta2, double* theta3, uint8_t* flags) {
  ftp_status st = check_obs(P, t, y, dy, nobs);
  if (st != FTP_OK) return st;
  if (!power || !theta1 || !theta2 || !theta3) return FTP_ERR_INVALID_ARG;
  st = check_templates(P, tpl, ntemplates);
  if (st != FTP_OK) return st;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  int Hs = 0;
  for (int i = 0; i < ntemplates; ++i) Hs = std::max(Hs, tpl[i].H);
  FTP_CK(reset_call(P));
  const double *dt, *dyv, *ddy;
  st = stage_obs(P, t, y, dy, nobs, &dt, &dyv, &ddy);
  if (st != FTP_OK) return st;
  std::vector<HGroup> groups;
  std::vector<int> pos_of;
  st = upload_templates(P, tpl, ntemplates, &groups, &pos_of);
  if (st != FTP_OK) return st;
  int launches = 0;
  st = run_sums_plan(P, dt, dyv, ddy, nobs, Hs, &launches);
  if (st != FTP_OK) return st;

  const int64_t nf = P->grid.nf;
  const size_t nout = (size_t)ntemplates * nf;
  const bool direct = is_device_ptr(power) && is_device_ptr(theta1) && is_device_ptr(theta2) &&
                      is_device_ptr(theta3) && (!flags || is_device_ptr(flags));
  double* o[4] = {power, theta1, theta2, theta3};
  uint8_t* of = flags;
  if (!direct) {
    for (int i = 0; i < 4; ++i) o[i] = P->d_out + (size_t)i * P->max_templates * nf;
    of = flags ? P->d_flags : nullptr;
  }
  const int64_t out_elems = direct ? (int64_t)nout : (int64_t)P->max_templates * nf;
  st = solve_main(P, nf, Hs, groups, P->d_alpha, P->d_rows, nullptr, o, of, out_elems, &launches);
  if (st != FTP_OK) return st;
  // status, counters and the re-solve list's length in one read-back
  st = read_back(P);
  if (st != FTP_OK) return st;
  FTP_CK(cudaMemcpyAsync(P->h_redo_count, P->d_redo_count, sizeof(int), cudaMemcpyDeviceToHost,
                         P->stream));
  ev_rec(P, 6);
  FTP_CK(cudaStreamSynchronize(P->stream));
  const bool redo = P->h_status[ST_CODE] == DEV_OK && *P->h_redo_count > 0;
  if (redo) {
    st = solve_redo(P, dt, dyv, ddy, nobs, P->grid.df, P->grid.k0, nf, Hs, groups, P->d_alpha,
                    P->d_rows, nullptr, o, of, out_elems, &launches);
    if (st != FTP_OK) return st;
    ev_rec(P, 6);
  }
  if (!direct) {
    double* dsto[4] = {power, theta1, theta2, theta3};
    for (int i = 0; i < 4; ++i)
      FTP_CK(cudaMemcpyAsync(dsto[i], o[i], sizeof(double) * nout, cudaMemcpyDefault, P->stream));
    if (flags)
      FTP_CK(cudaMemcpyAsync(flags, P->d_flags, nout, cudaMemcpyDefault, P->stream));
  }
  P->last_launches = launches;
  if (redo) return finish(P);
  if (!direct) FTP_CK(cudaStreamSynchronize(P->stream));
  return finish_host(P);
}

ftp_status ftp_batch(ftp_plan_t P, int64_t ncurves, const int64_t* obs_off, const double* t,
                     const double* y, const double* dy, const ftp_grid* grids,
                     const int64_t* out_off, const ftp_template* bank, int nbank,
                     const int32_t* tpl_of_curve, double* power, double* theta1, double* theta2,
                     double* theta3, uint8_t* flags) {
  return run_batch(P, ncurves, obs_off, t, y, dy, grids, out_off, bank, nbank, tpl_of_curve,
                   power, theta1, theta2, theta3, flags, nullptr);
}

ftp_status ftp_batch_features(ftp_plan_t P, int64_t ncurves, const int64_t* obs_off,
                              const double* t, const double* y, const double* dy,
                              const ftp_grid* grids, const int64_t* row_off, int H_feat,
                              float* features) {
  if (!features || !row_off) return FTP_ERR_INVALID_ARG;
  BatchScreen scr;
  scr.Hf = H_feat;
  scr.feat_out = features;
  scr.feat_row = row_off;
  return run_batch(P, ncurves, obs_off, t, y, dy, grids, nullptr, nullptr, 0, nullptr, nullptr,
                   nullptr, nullptr, nullptr, nullptr, &scr);
}

ftp_status ftp_batch_screened(ftp_plan_t P, int64_t ncurves, const int64_t* obs_off,
                              const double* t, const double* y, const double* dy,
                              const ftp_grid* grids, const int64_t* out_off,
                              const ftp_template* bank, int nbank, const int32_t* tpl_of_curve,
                              ftp_mlp_t mlp, double top_frac, int neighbours, double* power,
                              double* theta1, double* theta2, double* theta3, uint8_t* flags) {
  if (!P || !mlp || !(top_frac > 0.0) || !(top_frac <= 1.0) || neighbours < 0)
    return FTP_ERR_INVALID_ARG;
  const int nfeat = mlp_nfeat(mlp);
  if (nfeat % 2 != 0 || mlp_device(mlp) != P->device) return FTP_ERR_INVALID_ARG;
  BatchScreen scr;
  scr.Hf = (nfeat - 2) / 2;
  scr.mlp = mlp;
  scr.top_frac = top_frac;
  scr.nbr = neighbours;
  return run_batch(P, ncurves, obs_off, t, y, dy, grids, out_off, bank, nbank, tpl_of_curve,
                   power, theta1, theta2, theta3, flags, &scr);
}

ftp_status ftp_multiband_periodogram(ftp_plan_t P, int nbands, const int64_t* obs_off,
                                     const double* t, const double* y, const double* dy,
                                     const ftp_template* bank, int nbank,
                                     const int32_t* tpl_of_band, double* power,
                                     double* band_power, double* band_theta1,
                                     double* band_theta2, double* band_theta3,
                                     uint8_t* band_flags) {
  if (!P || nbands < 1 || !obs_off || !power || !bank || nbank < 1) return FTP_ERR_INVALID_ARG;
  if (nbands > (1 << 20)) return FTP_ERR_UNSUPPORTED;
  const int64_t nf = P->grid.nf, items = (int64_t)nbands * nf;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  bool grew = false;
  ftp_status st = grow_dev(&P->d_mb, &P->mb_cap, (size_t)4 * items + (size_t)MO_WORDS * nbands,
                           &grew);
  if (st == FTP_OK) st = grow_dev(&P->d_mbflags, &P->mbflags_cap, (size_t)items, &grew);
  if (st == FTP_OK) st = grow_dev(&P->d_mbpow, &P->mbpow_cap, (size_t)nf, &grew);
  if (st != FTP_OK) return st;
  if (grew && P->graph_exec) {
    cudaGraphExecDestroy(P->graph_exec);
    P->graph_exec = nullptr;
    P->graph_key = 0;
  }
  std::vector<ftp_grid> grids((size_t)nbands, P->grid);
  std::vector<int64_t> out_off((size_t)nbands);
  std::vector<int32_t> tob((size_t)nbands, 0);
  for (int b = 0; b < nbands; ++b) {
    out_off[(size_t)b] = (int64_t)b * nf;
    if (tpl_of_band) tob[(size_t)b] = tpl_of_band[b];
  }
  double* o[4];
  for (int i = 0; i < 4; ++i) o[i] = P->d_mb + (size_t)i * items;
  double* mom = P->d_mb + (size_t)4 * items;
  BatchScreen scr;
  scr.moments_out = mom;
  st = run_batch(P, nbands, obs_off, t, y, dy, grids.data(), out_off.data(), bank, nbank,
                 tob.data(), o[0], o[1], o[2], o[3], P->d_mbflags, &scr);
  if (st != FTP_OK) return st;
  launch_multiband_combine(o[0], mom, nbands, nf, P->d_mbpow, P->stream);
  FTP_CK(cudaGetLastError());
  FTP_CK(cudaMemcpyAsync(power, P->d_mbpow, sizeof(double) * nf, cudaMemcpyDefault, P->stream));
  double* bo[4] = {band_power, band_theta1, band_theta2, band_theta3};
  for (int i = 0; i < 4; ++i)
    if (bo[i])
      FTP_CK(cudaMemcpyAsync(bo[i], o[i], sizeof(double) * items, cudaMemcpyDefault, P->stream));
  if (band_flags)
    FTP_CK(cudaMemcpyAsync(band_flags, P->d_mbflags, (size_t)items, cudaMemcpyDefault, P->stream));
  FTP_CK(cudaStreamSynchronize(P->stream));
  return FTP_OK;
}

ftp_status ftp_shared_multiband(ftp_plan_t P, int nbands, const int64_t* obs_off,
                                const double* t, const double* y, const double* dy,
                                const double* offsets, const ftp_template* bank, int nbank,
                                const int32_t* tpl_of_band, double* power, double* theta1,
                                double* theta2, double* theta3, uint8_t* flags) {
  if (!P || nbands < 1 || !obs_off || !t || !y || !dy || !bank || nbank < 1 || !power ||
      !theta1 || !theta2 || !theta3)
    return FTP_ERR_INVALID_ARG;
  if (nbands > 4096) return FTP_ERR_UNSUPPORTED;
  ftp_status st = check_templates(P, bank, nbank);
  if (st != FTP_OK) return st;
  int H = 0;
  for (int b = 0; b < nbands; ++b) {
    const int q = tpl_of_band ? tpl_of_band[b] : 0;
    if (q < 0 || q >= nbank) return FTP_ERR_INVALID_ARG;
    const int64_t n = obs_off[b + 1] - obs_off[b];
    if (obs_off[b] < 0 || n < 2) return FTP_ERR_INVALID_ARG;
    if (n > P->max_nobs) return FTP_ERR_UNSUPPORTED;
    H = std::max(H, bank[q].H);
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  const int64_t nf = P->grid.nf, nf_pad = P->nf_pad;
  const int64_t band_elems = (int64_t)3 * H * nf_pad;
  bool grew = false;
  st = grow_dev(&P->d_shsums, &P->shsums_cap, (size_t)nbands * band_elems * P->csz, &grew);
  if (st == FTP_OK)
    st = grow_dev(&P->d_shmisc, &P->shmisc_cap, (size_t)nbands * (MO_WORDS + 3) + MO_WORDS, &grew);
  if (st == FTP_OK) st = grow_dev(&P->d_shalpha, &P->shalpha_cap, (size_t)nbands * kMaxH, &grew);
  if (st == FTP_OK)
    st = grow_dev(&P->d_shcoef, &P->shcoef_cap, (size_t)(4 * H + 1) * nf_pad, &grew);
  if (st != FTP_OK) return st;
  double* mom = P->d_shmisc;
  double* share = mom + (size_t)nbands * MO_WORDS;
  double* dyb = share + nbands;
  double* lam = dyb + nbands;
  double* pooled = lam + nbands;
  // band templates (zero-padded to H harmonics) and offsets
  std::vector<double2> al((size_t)nbands * kMaxH, make_double2(0.0, 0.0));
  for (int b = 0; b < nbands; ++b) {
    const ftp_template& tp = bank[tpl_of_band ? tpl_of_band[b] : 0];
    for (int n = 0; n < tp.H; ++n)
      al[(size_t)b * kMaxH + n] = make_double2(0.5 * tp.c[n], 0.5 * tp.s[n]);
  }
  std::vector<double> lamh((size_t)nbands, 0.0);
  if (offsets)
    for (int b = 0; b < nbands; ++b) {
      if (!isfinite(offsets[b])) return FTP_ERR_INVALID_ARG;
      lamh[(size_t)b] = offsets[b];
    }
  cudaStream_t s = P->stream;
  FTP_CK(reset_call(P));
  FTP_CK(cudaMemcpyAsync(P->d_shalpha, al.data(), sizeof(double2) * al.size(),
                         cudaMemcpyHostToDevice, s));
  FTP_CK(cudaMemcpyAsync(lam, lamh.data(), sizeof(double) * nbands, cudaMemcpyHostToDevice, s));
  FTP_CK(cudaStreamSynchronize(s));  // the host vectors go out of scope below
  int launches = 0;
  const int64_t J = 2 * (int64_t)H * (P->grid.k0 + nf - 1);
  int64_t ntiles = 0;
  const int64_t ngrid = grid_len(J, P->sigma, &ntiles);
  for (int b = 0; b < nbands; ++b) {
    const int64_t o = obs_off[b], n = obs_off[b + 1] - obs_off[b];
    const double *dt, *dyv, *ddy;
    st = stage_obs(P, t + o, y + o, dy + o, n, &dt, &dyv, &ddy);
    if (st != FTP_OK) return st;
    st = run_sums(P, P->l0, dt, dyv, ddy, n, P->grid.df, P->grid.k0, nf, H, ngrid, ntiles,
                  mom + (size_t)b * MO_WORDS, P->d_shsums + (size_t)b * band_elems * P->csz,
                  nf_pad, &launches);
    if (st != FTP_OK) return st;
  }
  launch_shared_moments(mom, lam, nbands, share, dyb, pooled, P->d_status, s);
  launch_shared_assembly(P->d_shsums, !P->mixed, band_elems, H, nbands, nf, nf_pad, H,
                         P->d_shalpha, share, dyb, P->d_shcoef, P->d_status, s);
  launches += 2;
  const bool direct = is_device_ptr(power) && is_device_ptr(theta1) && is_device_ptr(theta2) &&
                      is_device_ptr(theta3) && (!flags || is_device_ptr(flags));
  double* o[4] = {power, theta1, theta2, theta3};
  uint8_t* of = flags;
  if (!direct) {
    for (int i = 0; i < 4; ++i) o[i] = P->d_out + (size_t)i * P->max_templates * nf;
    of = flags ? P->d_flags : nullptr;
  }
  RootsArgs a{};
  a.sums = P->d_shcoef;
  a.sums_elems = (int64_t)(4 * H + 1) * nf_pad;
  a.out_elems = direct ? nf : (int64_t)P->max_templates * nf;
  a.nf = nf;
  a.nf_pad = nf_pad;
  a.Hs = H;
  a.H = H;
  a.ntpl = 1;
  a.alpha = P->d_shalpha;
  a.rows = P->d_row0;
  a.moments = pooled;
  a.power = o[0];
  a.theta1 = o[1];
  a.theta2 = o[2];
  a.theta3 = o[3];
  a.flags = of;
  a.out_stride = nf;
  a.status = P->d_status;
  a.counters = P->d_counters;
  a.queue = P->d_queue;
  solver_settings(P, a);
  a.coef_mode = 1;
  FTP_CK(cudaMemsetAsync(P->d_queue, 0, sizeof(unsigned long long), s));
  const int r = launch_roots(P->mixed ? ROOTS_REDO : ROOTS_FP64, a, P->num_sms, s);
  if (r == -1) return FTP_ERR_UNSUPPORTED;
  if (r < 0) return FTP_ERR_CUDA;
  launches += r;
  FTP_CK(cudaGetLastError());
  if (!direct) {
    double* dsto[4] = {power, theta1, theta2, theta3};
    for (int i = 0; i < 4; ++i)
      FTP_CK(cudaMemcpyAsync(dsto[i], o[i], sizeof(double) * nf, cudaMemcpyDefault, s));
    if (flags) FTP_CK(cudaMemcpyAsync(flags, P->d_flags, nf, cudaMemcpyDefault, s));
  }
  P->last_launches = launches;
  return finish(P);
}

ftp_status ftp_set_positive_amplitude(ftp_plan_t P, int enable) {
  if (!P) return FTP_ERR_INVALID_ARG;
  P->positive_only = enable != 0;
  return FTP_OK;
}

ftp_status ftp_set_batch_tuning(ftp_plan_t P, int sum_lanes, int roots_ctas_per_sm) {
  if (!P || sum_lanes < 1 || sum_lanes > kMaxSumLanes || roots_ctas_per_sm < 0)
    return FTP_ERR_INVALID_ARG;
  P->sum_lanes = sum_lanes;
  P->roots_ctas_per_sm = roots_ctas_per_sm;
  return FTP_OK;
}

ftp_status ftp_get_batch_tuning(ftp_plan_t P, int* sum_lanes, int* roots_ctas_per_sm) {
  if (!P) return FTP_ERR_INVALID_ARG;
  if (sum_lanes) *sum_lanes = P->sum_lanes;
  if (roots_ctas_per_sm) *roots_ctas_per_sm = P->roots_ctas_per_sm;
  return FTP_OK;
}

ftp_status ftp_batch_autotune(ftp_plan_t P, int64_t ncurves, const int64_t* obs_off,
                              const double* t, const double* y, const double* dy,
                              const ftp_grid* grids, const int64_t* out_off,
                              const ftp_template* bank, int nbank, const int32_t* tpl_of_curve,
                              double* power, double* theta1, double* theta2, double* theta3,
                              const char* cache_path, int* from_cache) {
  if (!P || ncurves < 1 || !obs_off || !grids || !bank || nbank < 1) return FTP_ERR_INVALID_ARG;
  // shape class of the batch: device, precision, harmonics, and log2 buckets
  // of the curve count, the median observation count and the median grid size
  std::vector<int64_t> nobs((size_t)ncurves), nfs((size_t)ncurves);
  for (int64_t c = 0; c < ncurves; ++c) {
    nobs[(size_t)c] = obs_off[c + 1] - obs_off[c];
    nfs[(size_t)c] = grids[c].nf;
  }
  std::nth_element(nobs.begin(), nobs.begin() + ncurves / 2, nobs.end());
  std::nth_element(nfs.begin(), nfs.begin() + ncurves / 2, nfs.end());
  auto lg = [](int64_t v) {
    int b = 0;
    while (v > 1) {
      v >>= 1;
      ++b;
    }
    return b;
  };
  int Hmax = 0;
  for (int i = 0; i < nbank; ++i) Hmax = std::max(Hmax, bank[i].H);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, P->device);
  std::string dev(prop.name);
  for (char& ch : dev)
    if (ch == '"' || ch == '\\' || ch == '\n') ch = '_';
  std::ostringstream ks;
  ks << dev << "/sm" << prop.multiProcessorCount << "/" << (P->mixed ? "mixed" : "fp64") << "/H"
     << Hmax << "/" << (tpl_of_curve ? "per-curve" : "bank") << "/c" << lg(ncurves) << "/n"
     << lg(nobs[(size_t)ncurves / 2]) << "/f" << lg(nfs[(size_t)ncurves / 2]);
  const std::string key = ks.str();
  if (from_cache) *from_cache = 0;
  // cache: one entry per line, "key": {"sum_lanes": L, "roots_ctas_per_sm": C, ...}
  std::vector<std::string> lines;
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      const size_t q0 = line.find('"'), q1 = q0 == std::string::npos ? q0 : line.find('"', q0 + 1);
      if (q1 == std::string::npos) continue;
      const std::string k = line.substr(q0 + 1, q1 - q0 - 1);
      int L = 0, Cc = -1;
      const size_t pl = line.find("\"sum_lanes\":"), pc = line.find("\"roots_ctas_per_sm\":");
      if (pl == std::string::npos || pc == std::string::npos) continue;
      if (sscanf(line.c_str() + pl + 12, " %d", &L) != 1 ||
          sscanf(line.c_str() + pc + 20, " %d", &Cc) != 1)
        continue;
      if (k == key && L >= 1 && L <= kMaxSumLanes && Cc >= 0) {
        P->sum_lanes = L;
        P->roots_ctas_per_sm = Cc;
        if (from_cache) *from_cache = 1;
        return FTP_OK;
      }
      if (k != key) lines.push_back(line);
    }
  }
  // time the choices on this batch (eager calls with stage events)
  const bool timing0 = P->timing;
  const int lanes0 = P->sum_lanes, ctas0 = P->roots_ctas_per_sm;
  P->timing = true;
  auto once = [&](float* sa, float* sr) -> ftp_status {
    ftp_status st = run_batch(P, ncurves, obs_off, t, y, dy, grids, out_off, bank, nbank,
                              tpl_of_curve, power, theta1, theta2, theta3, nullptr, nullptr);
    if (st == FTP_OK) {
      *sa = P->stage_ms[0];
      *sr = P->stage_ms[4];
    }
    return st;
  };
  float sa = 0.f, sr = 0.f;
  std::ostringstream rec;
  ftp_status st = FTP_OK;
  int best_l = lanes0;
  float best_a = 3e38f;
  rec << "\"step_a_ms\": {";
  for (int L : {1, 2, 4, 8}) {
    P->sum_lanes = L;
    st = once(&sa, &sr);  // warm-up: lanes and FFT plans
    if (st == FTP_OK) st = once(&sa, &sr);
    if (st != FTP_OK) break;
    rec << (L == 1 ? "" : ", ") << "\"" << L << "\": " << sa;
    if (sa < 0.97f * best_a) {
      best_a = sa;
      best_l = L;
    }
  }
  rec << "}, \"roots_ms\": {";
  int best_c = ctas0;
  float best_r = 3e38f;
  if (st == FTP_OK) {
    P->sum_lanes = best_l;
    for (int Cc : {0, 4, 3, 2}) {
      P->roots_ctas_per_sm = Cc;
      st = once(&sa, &sr);
      if (st != FTP_OK) break;
      rec << (Cc == 0 ? "" : ", ") << "\"" << Cc << "\": " << sr;
      if (sr < 0.98f * best_r) {
        best_r = sr;
        best_c = Cc;
      }
    }
  }
  rec << "}";
  P->timing = timing0;
  if (st != FTP_OK) {
    P->sum_lanes = lanes0;
    P->roots_ctas_per_sm = ctas0;
    return st;
  }
  P->sum_lanes = best_l;
  P->roots_ctas_per_sm = best_c;
  if (cache_path) {
    std::ostringstream e;
    e << "  \"" << key << "\": {\"sum_lanes\": " << best_l << ", \"roots_ctas_per_sm\": " << best_c
      << ", " << rec.str() << "}";
    std::vector<std::string> keep;
    for (const std::string& l : lines) {
      std::string x = l;
      while (!x.empty() && (x.back() == ',' || x.back() == ' ')) x.pop_back();
      if (x.find("\"sum_lanes\":") != std::string::npos) keep.push_back(x);
    }
    keep.push_back(e.str());
    std::ofstream out(cache_path, std::ios::trunc);
    if (!out) return FTP_ERR_INVALID_ARG;
    out << "{\n";
    for (size_t i = 0; i < keep.size(); ++i) out << keep[i] << (i + 1 < keep.size() ? ",\n" : "\n");
    out << "}\n";
  }
  return FTP_OK;
}

ftp_status ftp_set_batch_options(ftp_plan_t P, int64_t chunk_bytes, int use_graph) {
  if (!P || chunk_bytes < 0) return FTP_ERR_INVALID_ARG;
  if (chunk_bytes > 0) P->chunk_bytes = (size_t)chunk_bytes;
  P->use_graph = use_graph != 0;
  return FTP_OK;
}

ftp_status ftp_batch_info(ftp_plan_t P, int64_t* chunks, int* graph) {
  if (!P) return FTP_ERR_INVALID_ARG;
  if (chunks) *chunks = P->last_chunks;
  if (graph) *graph = P->last_graph;
  return FTP_OK;
}

}  // extern "C"
