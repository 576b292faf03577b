// Shared-phase multi-band template periodogram (Appendix A): one amplitude,
// phase and offset shared by every band, a template per band, fixed band
// offsets lambda_k subtracted from the data first.  With weights normalised
// over all observations (band shares W_k, sum_k W_k = 1) the polynomials pool
// the single-band ones:
//   <M^2>(theta) = sum_k W_k <M^(k)2>_k,   Mbar(theta) = sum_k W_k Mbar^(k)_k,
//   MM = <M^2> - Mbar^2,   YM = sum_k W_k <(y - ybar) M^(k)>_k,
// ybar the pooled mean of the offset-corrected data.  In the trigonometric
// form of the root stage (MM = a_0 + 2 Re sum a_e psi^e, YM = 2 Re sum b_n
// psi^n, Mbar = 2 Re sum c_n psi^n) the pooled coefficients are
//   c_n  = sum_k W_k alpha^(k)_n conj(Z^(k)_n)
//   b_n  = sum_k W_k alpha^(k)_n conj(Y^(k)_n + (ybar_k - ybar) Z^(k)_n)
//   a_e  = sum_k W_k conj(Z^(k)_e) K^(k)_e - (sum_{n+m=e} c_n c_m + 2 sum_{n-m=e} c_n conj(c_m))
// with Z^(k), Y^(k) the band's step (a) sums (band-normalised weights, Y
// centred on the band's own mean) and K^(k)_e the band template's
//   K_e = sum_{n+m=e} alpha_n alpha_m + 2 sum_{n-m=e} alpha_n conj(alpha_m).
// These kernels form the pooled moments and coefficients in FP64; the roots
// kernel then runs on the coefficient rows unchanged.
#include <math.h>
#include <stdint.h>

#include "ftp_internal.cuh"

namespace ftp {

namespace {

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 ca(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 cs(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Pooled moments from the bands' own ones (one thread): share[k] = W_k,
// dyb[k] = (ybar_k - lambda_k) - ybar; pooled {ybar, YY} into pooled[MO_*].
// A mix of bands with and without uncertainties is the mixed-sigma error of
// the pooled data.
__global__ void shared_moments_kernel(const double* __restrict__ mom, const double* __restrict__ lam,
                                      int nbands, double* __restrict__ share,
                                      double* __restrict__ dyb, double* __restrict__ pooled,
                                      int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (status[ST_CODE] != DEV_OK) return;
  double wtot = 0.0;
  bool any_unit = false, any_sigma = false;
  for (int k = 0; k < nbands; ++k) {
    wtot += mom[(size_t)k * MO_WORDS + MO_WSUM];
    if (mom[(size_t)k * MO_WORDS + MO_UNIT] != 0.0) any_unit = true;
    else any_sigma = true;
  }
  if (any_unit && any_sigma) {
    atomicCAS(&status[ST_CODE], DEV_OK, DEV_MIXED_ZERO_SIGMA);
    return;
  }
  double ybar = 0.0;
  for (int k = 0; k < nbands; ++k) {
    const double W = mom[(size_t)k * MO_WORDS + MO_WSUM] / wtot;
    share[k] = W;
    ybar += W * (mom[(size_t)k * MO_WORDS + MO_YBAR] - (lam ? lam[k] : 0.0));
  }
  double YY = 0.0;
  for (int k = 0; k < nbands; ++k) {
    const double d = mom[(size_t)k * MO_WORDS + MO_YBAR] - (lam ? lam[k] : 0.0) - ybar;
    dyb[k] = d;
    YY += share[k] * (mom[(size_t)k * MO_WORDS + MO_YY] + d * d);
  }
  if (!(YY > 0.0)) atomicCAS(&status[ST_CODE], DEV_OK, DEV_ZERO_VARIANCE);
  pooled[MO_YBAR] = ybar;
  pooled[MO_YY] = YY;
  pooled[MO_WSUM] = wtot;
  pooled[MO_UNIT] = any_unit ? 1.0 : 0.0;
}

// One thread per frequency: the pooled coefficient rows of the root stage,
// coef[(row) * nf_pad + k], rows a_0..a_2H, b_1..b_H, c_1..c_H; the padding
// columns [nf, nf_pad) are zero.
template <typename S2>
__global__ void __launch_bounds__(128) shared_assembly_kernel(
    const S2* __restrict__ sums, int64_t band_stride, int Hs, int nbands, int64_t nf,
    int64_t nf_pad, int H, const double2* __restrict__ alpha, const double* __restrict__ share,
    const double* __restrict__ dyb, double2* __restrict__ coef, const int* __restrict__ status) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf_pad || status[ST_CODE] != DEV_OK) return;
  if (k >= nf) {
    for (int r = 0; r <= 4 * H; ++r) coef[(int64_t)r * nf_pad + k] = make_double2(0.0, 0.0);
    return;
  }
  double2 c[kMaxH + 1], b[kMaxH + 1], raw[2 * kMaxH + 1];
  for (int n = 0; n <= H; ++n) c[n] = b[n] = make_double2(0.0, 0.0);
  for (int e = 0; e <= 2 * H; ++e) raw[e] = make_double2(0.0, 0.0);
  for (int q = 0; q < nbands; ++q) {
    const S2* sb = sums + (int64_t)q * band_stride + k;
    const double2* al = alpha + (size_t)q * kMaxH;
    const double W = share[q], d = dyb[q];
    for (int e = 0; e <= 2 * H; ++e) {
      // K_e of the band's template
      double2 Ke = make_double2(0.0, 0.0);
      for (int n = 1; n <= H; ++n) {
        if (e - n >= 1 && e - n <= H) Ke = ca(Ke, cm(al[n - 1], al[e - n - 1]));
        if (n - e >= 1) Ke = ca(Ke, cs(cm(al[n - 1], cj(al[n - e - 1])), 2.0));
      }
      double2 Ze = make_double2(1.0, 0.0);
      if (e >= 1) {
        const S2 v = sb[(int64_t)(e - 1) * nf_pad];
        Ze = make_double2((double)v.x, (double)v.y);
      }
      raw[e] = ca(raw[e], cs(cm(cj(Ze), Ke), W));
    }
    for (int n = 1; n <= H; ++n) {
      const S2 zv = sb[(int64_t)(n - 1) * nf_pad];
      const S2 yv = sb[(int64_t)(2 * Hs + n - 1) * nf_pad];
      const double2 Z = make_double2((double)zv.x, (double)zv.y);
      const double2 Y = make_double2((double)yv.x + d * (double)zv.x, (double)yv.y + d * (double)zv.y);
      c[n] = ca(c[n], cs(cm(al[n - 1], cj(Z)), W));
      b[n] = ca(b[n], cs(cm(al[n - 1], cj(Y)), W));
    }
  }
  for (int e = 0; e <= 2 * H; ++e) {
    double2 S = make_double2(0.0, 0.0);
    for (int n = 1; n <= H; ++n) {
      if (e - n >= 1 && e - n <= H) S = ca(S, cm(c[n], c[e - n]));
      if (n - e >= 1) S = ca(S, cs(cm(c[n], cj(c[n - e])), 2.0));
    }
    double2 a = make_double2(raw[e].x - S.x, raw[e].y - S.y);
    if (e == 0) a.y = 0.0;  // MM's constant coefficient is real
    coef[(int64_t)e * nf_pad + k] = a;
  }
  for (int n = 1; n <= H; ++n) {
    coef[(int64_t)(2 * H + n) * nf_pad + k] = b[n];
    coef[(int64_t)(3 * H + n) * nf_pad + k] = c[n];
  }
}

}  // namespace

void launch_shared_moments(const double* mom, const double* lam, int nbands, double* share,
                           double* dyb, double* pooled, int* status, cudaStream_t s) {
  shared_moments_kernel<<<1, 32, 0, s>>>(mom, lam, nbands, share, dyb, pooled, status);
}

void launch_shared_assembly(const void* sums, bool fp64, int64_t band_stride, int Hs, int nbands,
                            int64_t nf, int64_t nf_pad, int H, const double2* alpha,
                            const double* share, const double* dyb, double2* coef,
                            const int* status, cudaStream_t s) {
  const unsigned blocks = (unsigned)((nf_pad + 127) / 128);
  if (fp64)
    shared_assembly_kernel<double2><<<blocks, 128, 0, s>>>(
        (const double2*)sums, band_stride, Hs, nbands, nf, nf_pad, H, alpha, share, dyb, coef,
        status);
  else
    shared_assembly_kernel<float2><<<blocks, 128, 0, s>>>(
        (const float2*)sums, band_stride, Hs, nbands, nf, nf_pad, H, alpha, share, dyb, coef,
        status);
}

}  // namespace ftp
