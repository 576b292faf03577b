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
enum : int { ST_CODE = 0, ST_TIMEOUT_SITE = 1, ST_NONCONV = 2, ST_WORDS = 4 };

// Layout of the device moments block (doubles).
enum : int { MO_YBAR = 0, MO_YY = 1, MO_WSUM = 2, MO_UNIT = 3, MO_WORDS = 4 };

constexpr int kSpreadTile = 2048;       // grid cells owned by one spreading CTA
constexpr int kSpreadTileShift = 11;
constexpr int kMaxH = 16;

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

// ------------------------------------------------------------------ launches
// Step (a): observation preparation, binning, spreading, FFT (host), gather.
void launch_moments(const double* t, const double* y, const double* dy, int64_t n,
                    double* moments, int* status, cudaStream_t s);

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

// Steps (b)-(c): assembly, roots, candidates, polish.
struct RootsArgs {
  const void* sums;        // [3*Hs][nf_pad] complex (float2 mixed / double2 fp64)
  int64_t nf;
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
  int maxit;
  int polish_steps;
};

// Launches the assembly + Aberth + candidate kernel for the precision of the
// plan (mixed: float Aberth on float2 sums; otherwise all double).  Returns
// the number of kernel launches issued (1) or a negative value for an
// unsupported H.
int launch_roots(bool mixed, const RootsArgs& a, int num_sms, cudaStream_t s);

// Dynamic shared memory bytes the roots kernel needs (for tests/tuning).
size_t roots_smem_bytes(bool mixed, int H);

}  // namespace ftp
