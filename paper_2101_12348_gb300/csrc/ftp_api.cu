// C ABI of the FTP library (include/ftp.h): plans, workspaces, pointer
// staging, the step (a) pipeline and the per-H launches of steps (b)-(c).
#include <cufft.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "../../include/ftp.h"
#include "ftp_internal.cuh"

namespace ftp {
int launch_roots_mixed(const RootsArgs& a, int num_sms, cudaStream_t s);
int launch_roots_fp64(const RootsArgs& a, int num_sms, cudaStream_t s);
int launch_roots_redo(const RootsArgs& a, int num_sms, cudaStream_t s);

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
  unsigned long long* d_queue = nullptr;  // work-unit counter of the roots kernel
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
  void* d_fftwork = nullptr;
  size_t fftwork_bytes = 0;
  std::map<int64_t, FftEntry> ffts;
  // pinned host staging
  int* h_status = nullptr;
  unsigned long long* h_counters = nullptr;
  double2* h_alpha = nullptr;
  int* h_rows = nullptr;
  // instrumentation
  int last_launches = 0;
  bool timing = false;
  cudaEvent_t ev[7] = {};
  float stage_ms[6] = {};
  int maxit = 60;
  int polish_steps = 1;
};

namespace {

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

ftp_status get_fft(ftp_plan_t P, int64_t n, cufftHandle* out) {
  auto it = P->ffts.find(n);
  if (it != P->ffts.end()) {
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
  if (e.work > P->fftwork_bytes) {
    // queued transforms may still use the old work area
    if (P->stream) cudaStreamSynchronize(P->stream);
    if (P->d_fftwork) cudaFree(P->d_fftwork);
    P->d_fftwork = nullptr;
    P->fftwork_bytes = 0;
    if (cudaMalloc(&P->d_fftwork, e.work) != cudaSuccess) {
      cufftDestroy(e.h);
      return FTP_ERR_OOM;
    }
    P->fftwork_bytes = e.work;
    for (auto& kv : P->ffts) cufftSetWorkArea(kv.second.h, P->d_fftwork);
  }
  cufftSetWorkArea(e.h, P->d_fftwork);
  P->ffts[n] = e;
  *out = e.h;
  return FTP_OK;
}

void ev_rec(ftp_plan_t P, int i) {
  if (P->timing) cudaEventRecord(P->ev[i], P->stream);
}

// Step (a) for one curve: moments, binning, spreading, FFT, gather into the
// plan's sum tiles (layout [3 Hs][nf_pad]).  t, y, dy are device pointers.
ftp_status run_sums(ftp_plan_t P, const double* t, const double* y, const double* dy,
                    int64_t nobs, double df, int64_t k0, int64_t nf, int Hs, int* launches) {
  const int64_t J = 2 * (int64_t)Hs * (k0 + nf - 1);
  int64_t ntiles = 0;
  const int64_t ngrid = grid_len(J, P->sigma, &ntiles);
  if (ngrid > P->ngrid) return FTP_ERR_UNSUPPORTED;
  cufftHandle fft;
  ftp_status st = get_fft(P, ngrid, &fft);
  if (st != FTP_OK) return st;
  cudaStream_t s = P->stream;
  ev_rec(P, 0);
  FTP_CK(cudaMemsetAsync(P->d_tile_count, 0, sizeof(int) * ntiles, s));
  launch_moments(t, y, dy, nobs, P->d_moments, P->d_status, P->d_mom_scratch, s);
  if (P->mixed) {
    launch_points<float>(t, y, dy, nobs, P->d_moments, P->d_status, df, ngrid, P->d_tile_count,
                         P->d_cell, (float*)P->d_frac, (float2*)P->d_coef, s);
  } else {
    launch_points<double>(t, y, dy, nobs, P->d_moments, P->d_status, df, ngrid, P->d_tile_count,
                          P->d_cell, (double*)P->d_frac, (double2*)P->d_coef, s);
  }
  launch_scan(P->d_tile_count, ntiles, P->d_tile_off, P->d_cursor, P->d_status, s);
  if (P->mixed) {
    launch_scatter<float>(nobs, P->d_tile_off, P->d_cursor, P->d_cell, (float*)P->d_frac,
                          (float2*)P->d_coef, P->d_cell_s, (float*)P->d_frac_s,
                          (float2*)P->d_coef_s, P->d_status, s);
  } else {
    launch_scatter<double>(nobs, P->d_tile_off, P->d_cursor, P->d_cell, (double*)P->d_frac,
                           (double2*)P->d_coef, P->d_cell_s, (double*)P->d_frac_s,
                           (double2*)P->d_coef_s, P->d_status, s);
  }
  ev_rec(P, 1);
  if (P->mixed) {
    launch_spread<float>(P->d_tile_off, P->d_cell_s, (float*)P->d_frac_s, (float2*)P->d_coef_s,
                         ngrid, ntiles, P->m, P->beta, (float2*)P->d_grid, P->d_status, s);
  } else {
    launch_spread<double>(P->d_tile_off, P->d_cell_s, (double*)P->d_frac_s,
                          (double2*)P->d_coef_s, ngrid, ntiles, P->m, P->beta,
                          (double2*)P->d_grid, P->d_status, s);
  }
  ev_rec(P, 2);
  if (cufftSetStream(fft, s) != CUFFT_SUCCESS) return FTP_ERR_CUDA;
  cufftResult fr;
  if (P->mixed) {
    fr = cufftExecC2C(fft, (cufftComplex*)P->d_grid, (cufftComplex*)P->d_grid, CUFFT_INVERSE);
  } else {
    fr = cufftExecZ2Z(fft, (cufftDoubleComplex*)P->d_grid, (cufftDoubleComplex*)P->d_grid,
                      CUFFT_INVERSE);
  }
  if (fr != CUFFT_SUCCESS) return FTP_ERR_CUDA;
  ev_rec(P, 3);
  if (P->mixed) {
    launch_gather<float>((const float2*)P->d_grid, ngrid, k0, nf, P->nf_pad, Hs, P->m, P->beta,
                         (float2*)P->d_sums, P->d_status, s);
  } else {
    launch_gather<double>((const double2*)P->d_grid, ngrid, k0, nf, P->nf_pad, Hs, P->m,
                          P->beta, (double2*)P->d_sums, P->d_status, s);
  }
  ev_rec(P, 4);
  *launches += 7;
  FTP_CK(cudaGetLastError());
  return FTP_OK;
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

ftp_status finish(ftp_plan_t P) {
  FTP_CK(cudaMemcpyAsync(P->h_status, P->d_status, sizeof(int) * ST_WORDS,
                         cudaMemcpyDeviceToHost, P->stream));
  FTP_CK(cudaMemcpyAsync(P->h_counters, P->d_counters, sizeof(unsigned long long) * CNT_WORDS,
                         cudaMemcpyDeviceToHost, P->stream));
  FTP_CK(cudaStreamSynchronize(P->stream));
#ifdef FTP_DEVICE_CHECKS
  if (P->h_status[ST_DBG_N] != 0)
    fprintf(stderr, "ftp device check failed: site %d value %d bound %d (%d failures)\n",
            P->h_status[ST_DBG_SITE], P->h_status[ST_DBG_A], P->h_status[ST_DBG_B],
            P->h_status[ST_DBG_N]);
#endif
  if (P->timing) {
    for (int i = 0; i < 6; ++i) P->stage_ms[i] = 0.f;
    float ms;
    for (int i = 0; i < 6; ++i)
      if (cudaEventElapsedTime(&ms, P->ev[i], P->ev[i + 1]) == cudaSuccess) P->stage_ms[i] = ms;
    cudaGetLastError();
  }
  return (ftp_status)P->h_status[ST_CODE];
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

ftp_status run_roots(ftp_plan_t P, RootsKind kind, const void* sums, int H, int Hs, int64_t nf,
                     const int* nf_dev, const int* kmap, bool collect_redo, const double2* alpha,
                     const int* rows, int ntpl, double* const* o, uint8_t* flags,
                     int64_t out_stride, int64_t out_elems, int* launches) {
  RootsArgs a{};
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
    a.sum_err = P->mixed ? kSumErrF32 : kSumErrF64;
    a.redo_tol = P->mixed ? kRedoTolF32 : kRedoTolF64;
  }
  a.maxit = P->maxit;
  a.polish_steps = P->polish_steps;
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
// mixed path, FP64 Aberth on the FP64 path).
ftp_status solve(ftp_plan_t P, const double* dt, const double* dyv, const double* ddy,
                 int64_t nobs, double df, int64_t k0, int64_t nf, int Hs,
                 const std::vector<HGroup>& groups, const double2* alpha, const int* rows,
                 const int* row0, double* const* o, uint8_t* flags, int64_t out_elems,
                 int* launches) {
  const bool redo = true;
  if (redo) {
    FTP_CK(cudaMemsetAsync(P->d_redo_mark, 0, sizeof(int) * nf, P->stream));
    FTP_CK(cudaMemsetAsync(P->d_redo_count, 0, sizeof(int), P->stream));
  }
  const RootsKind kind = P->mixed ? ROOTS_MIXED : ROOTS_FP64;
  for (const HGroup& g : groups) {
    ftp_status st = run_roots(P, kind, P->d_sums, g.H, Hs, nf, nullptr, nullptr, redo,
                              alpha + (size_t)g.first * kMaxH, row0 ? row0 : rows + g.first,
                              g.count, o, flags, nf, out_elems, launches);
    if (st != FTP_OK) return st;
  }
  ev_rec(P, 5);
  if (!redo) return FTP_OK;
  launch_direct_sums(dt, dyv, ddy, nobs, P->d_moments, P->d_status, df, k0, P->d_redo_list,
                     P->d_redo_count, (int)nf, Hs, P->nf_pad, P->d_redo_sums,
                     (int64_t)3 * P->max_H * P->nf_pad, P->d_status, P->stream);
  *launches += 1;
  for (const HGroup& g : groups) {
    ftp_status st = run_roots(P, P->mixed ? ROOTS_REDO : ROOTS_FP64, P->d_redo_sums, g.H, Hs, nf,
                              P->d_redo_count,
                              P->d_redo_list, false, alpha + (size_t)g.first * kMaxH,
                              row0 ? row0 : rows + g.first, g.count, o, flags, nf, out_elems,
                              launches);
    if (st != FTP_OK) return st;
  }
  return FTP_OK;
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
  for (auto& kv : P->ffts) cufftDestroy(kv.second.h);
  void* dptrs[] = {P->d_in, P->d_moments, P->d_mom_scratch, P->d_status, P->d_counters, P->d_queue, P->d_redo_list,
                   P->d_redo_mark, P->d_redo_count, P->d_redo_sums, P->d_tile_count, P->d_tile_off,
                   P->d_cursor, P->d_cell, P->d_cell_s, P->d_frac, P->d_frac_s, P->d_coef,
                   P->d_coef_s, P->d_grid, P->d_sums, P->d_alpha, P->d_rows, P->d_row0, P->d_out,
                   P->d_flags, P->d_fftwork};
  for (void* p : dptrs)
    if (p) cudaFree(p);
  if (P->h_status) cudaFreeHost(P->h_status);
  if (P->h_counters) cudaFreeHost(P->h_counters);
  if (P->h_alpha) cudaFreeHost(P->h_alpha);
  if (P->h_rows) cudaFreeHost(P->h_rows);
  for (auto& e : P->ev)
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
  if (!(grid.df > 0.0) || !isfinite(grid.df) || grid.k0 < 1 || grid.nf < 1)
    return FTP_ERR_INVALID_ARG;
  if (prec != FTP_FP64 && prec != FTP_MIXED) return FTP_ERR_INVALID_ARG;
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
  P->m = P->mixed ? 4 : 8;
  P->sigma = 2.0;
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
  FTP_AL(P->d_queue, 1);
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
      cudaMallocHost(&P->h_alpha, sizeof(double2) * kMaxH * max_templates) != cudaSuccess ||
      cudaMallocHost(&P->h_rows, sizeof(int) * max_templates) != cudaSuccess)
    return fail(FTP_ERR_OOM);
  for (auto& e : P->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(FTP_ERR_CUDA);
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
                            int64_t* nonconverged, int64_t* resolved) {
  if (!P) return FTP_ERR_INVALID_ARG;
  const unsigned long long* c = P->h_counters;
  const unsigned long long n = c ? c[CNT_ITEMS] : 0;
  if (items) *items = (int64_t)n;
  if (mean_iterations) *mean_iterations = n ? (double)c[CNT_ITERS] / (double)n : 0.0;
  if (nonconverged) *nonconverged = n ? (int64_t)c[CNT_NONCONV] : 0;
  if (resolved) *resolved = n ? (int64_t)c[CNT_REDO] : 0;
  return FTP_OK;
}

ftp_status ftp_set_timing(ftp_plan_t P, int enable) {
  if (!P) return FTP_ERR_INVALID_ARG;
  P->timing = enable != 0;
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
  st = run_sums(P, dt, dyv, ddy, nobs, P->grid.df, P->grid.k0, P->grid.nf, H_sums, &launches);
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
  st = run_sums(P, dt, dyv, ddy, nobs, P->grid.df, P->grid.k0, P->grid.nf, Hs, &launches);
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
  st = solve(P, dt, dyv, ddy, nobs, P->grid.df, P->grid.k0, nf, Hs, groups, P->d_alpha, P->d_rows,
             nullptr, o, of, direct ? (int64_t)nout : (int64_t)P->max_templates * nf, &launches);
  if (st != FTP_OK) return st;
  ev_rec(P, 6);
  if (!direct) {
    double* dsto[4] = {power, theta1, theta2, theta3};
    for (int i = 0; i < 4; ++i)
      FTP_CK(cudaMemcpyAsync(dsto[i], o[i], sizeof(double) * nout, cudaMemcpyDefault, P->stream));
    if (flags)
      FTP_CK(cudaMemcpyAsync(flags, P->d_flags, nout, cudaMemcpyDefault, P->stream));
  }
  P->last_launches = launches;
  return finish(P);
}

ftp_status ftp_batch(ftp_plan_t P, int64_t ncurves, const int64_t* obs_off, const double* t,
                     const double* y, const double* dy, const ftp_grid* grids,
                     const int64_t* out_off, const ftp_template* bank, int nbank,
                     const int32_t* tpl_of_curve, double* power, double* theta1, double* theta2,
                     double* theta3, uint8_t* flags) {
  if (!P || ncurves < 0 || !obs_off || !t || !y || !dy || !grids || !out_off || !power ||
      !theta1 || !theta2 || !theta3)
    return FTP_ERR_INVALID_ARG;
  if (ncurves == 0) return FTP_OK;
  ftp_status st = check_templates(P, bank, nbank);
  if (st != FTP_OK) return st;
  int Hs = 0;
  for (int i = 0; i < nbank; ++i) Hs = std::max(Hs, bank[i].H);
  // validate every curve on the host before any work is queued
  for (int64_t c = 0; c < ncurves; ++c) {
    const int64_t n = obs_off[c + 1] - obs_off[c];
    if (obs_off[c] < 0 || n < 2) return FTP_ERR_INVALID_ARG;
    if (n > P->max_nobs) return FTP_ERR_UNSUPPORTED;
    const ftp_grid& g = grids[c];
    if (!(g.df > 0.0) || !isfinite(g.df) || g.k0 < 1 || g.nf < 1 || out_off[c] < 0)
      return FTP_ERR_INVALID_ARG;
    if (g.nf > P->grid.nf) return FTP_ERR_UNSUPPORTED;
    int64_t nt = 0;
    if (grid_len(2 * (int64_t)Hs * (g.k0 + g.nf - 1), P->sigma, &nt) > P->ngrid)
      return FTP_ERR_UNSUPPORTED;
    if (tpl_of_curve && (tpl_of_curve[c] < 0 || tpl_of_curve[c] >= nbank))
      return FTP_ERR_INVALID_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  FTP_CK(reset_call(P));
  std::vector<HGroup> groups;
  std::vector<int> pos_of;
  st = upload_templates(P, bank, nbank, &groups, &pos_of);
  if (st != FTP_OK) return st;
  const bool in_dev = is_device_ptr(t) && is_device_ptr(y) && is_device_ptr(dy);
  const bool out_dev = is_device_ptr(power) && is_device_ptr(theta1) && is_device_ptr(theta2) &&
                       is_device_ptr(theta3) && (!flags || is_device_ptr(flags));
  int launches = 0;
  for (int64_t c = 0; c < ncurves; ++c) {
    const int64_t a0 = obs_off[c], n = obs_off[c + 1] - obs_off[c];
    const ftp_grid& g = grids[c];
    const double *dt, *dyv, *ddy;
    if (in_dev) {
      dt = t + a0;
      dyv = y + a0;
      ddy = dy + a0;
    } else {
      st = stage_obs(P, t + a0, y + a0, dy + a0, n, &dt, &dyv, &ddy);
      if (st != FTP_OK) return st;
    }
    int Hc = Hs;
    if (tpl_of_curve) Hc = bank[tpl_of_curve[c]].H;
    st = run_sums(P, dt, dyv, ddy, n, g.df, g.k0, g.nf, Hc, &launches);
    if (st != FTP_OK) return st;
    const int ntc = tpl_of_curve ? 1 : nbank;
    const size_t nout = (size_t)ntc * g.nf;
    double* o[4] = {power + out_off[c], theta1 + out_off[c], theta2 + out_off[c],
                    theta3 + out_off[c]};
    uint8_t* of = flags ? flags + out_off[c] : nullptr;
    int64_t out_lim = (int64_t)nout;  // caller arrays: this curve's block
    if (!out_dev) {
      for (int i = 0; i < 4; ++i) o[i] = P->d_out + (size_t)i * P->max_templates * P->grid.nf;
      of = flags ? P->d_flags : nullptr;
      out_lim = (int64_t)P->max_templates * P->grid.nf;
    }
    if (tpl_of_curve) {
      const int q = pos_of[tpl_of_curve[c]];
      const std::vector<HGroup> one{{bank[tpl_of_curve[c]].H, 0, 1}};
      st = solve(P, dt, dyv, ddy, n, g.df, g.k0, g.nf, Hc, one, P->d_alpha + (size_t)q * kMaxH,
                 nullptr, P->d_row0, o, of, out_lim, &launches);
    } else {
      st = solve(P, dt, dyv, ddy, n, g.df, g.k0, g.nf, Hc, groups, P->d_alpha, P->d_rows,
                 nullptr, o, of, out_lim, &launches);
    }
    if (st != FTP_OK) return st;
    if (!out_dev) {
      double* dsto[4] = {power + out_off[c], theta1 + out_off[c], theta2 + out_off[c],
                         theta3 + out_off[c]};
      for (int i = 0; i < 4; ++i)
        FTP_CK(cudaMemcpyAsync(dsto[i], o[i], sizeof(double) * nout, cudaMemcpyDefault,
                               P->stream));
      if (flags)
        FTP_CK(cudaMemcpyAsync(flags + out_off[c], P->d_flags, nout, cudaMemcpyDefault,
                               P->stream));
    }
  }
  P->last_launches = launches;
  return finish(P);
}

}  // extern "C"
