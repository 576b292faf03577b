// Learned screening of trial frequencies (the surrogate is not part of the
// paper; its features are).
//
//  * features_kernel: per frequency, 2H+2 features read from the NFFT sums
//    Z_h, Y_h that step (a) already produced (Eqs. CCdef-YSdef):
//      P_h   floating-mean Lomb-Scargle power at h*omega (the H = 1 case of
//            the template periodogram, Section 2.1), h = 1..H
//      A_h   |Y_h|^2 / YY, h = 1..H
//      P_MH  multi-harmonic least-squares power with H harmonics
//            (Section 2.1), an upper bound of the template power
//      log10 N_obs
//    Both least-squares powers are b^T G^-1 b / YY with G the weighted
//    covariance matrix of the centred basis functions (entries from Z_0..Z_2H
//    by product-to-sum identities) and b their covariances with y (Y_h),
//    solved by a Cholesky factorisation that drops (numerically) dependent
//    columns, so a rank-deficient basis gives the projection on its span.
//  * select_kernel: per curve, the frequencies whose score is among the top
//    K = ceil(frac * nf) (radix select on order-preserving integer keys),
//    dilated by +-nbr neighbours.
//  * unit_list_kernel: the roots kernel's work units (blocks of consecutive
//    frequencies of one template) that contain a selected frequency.
//  * fill_kernel: outputs of frequencies that are not evaluated.
#include <math.h>
#include <stdint.h>

#include "ftp_internal.cuh"
#include "ftp_screen.cuh"

namespace ftp {

namespace {

template <typename R> __device__ __forceinline__ R piv_tol();
template <> __device__ __forceinline__ float piv_tol<float>() { return 1e-5f; }
template <> __device__ __forceinline__ double piv_tol<double>() { return 1e-12; }

// b^T G^-1 b for a symmetric positive semi-definite n x n matrix (lower
// triangle of G in g[i*(i+1)/2 + j], j <= i; overwritten by the factor).
template <int NMAX, typename R>
__device__ __forceinline__ R quad_form(R* g, const R* b, int n) {
  R z[NMAX];
  bool keep[NMAX];
  R acc = R(0);
  for (int j = 0; j < n; ++j) {
    const int jj = j * (j + 1) / 2;
    const R diag0 = g[jj + j];
    R d = diag0;
    for (int k = 0; k < j; ++k) d -= g[jj + k] * g[jj + k];
    keep[j] = d > piv_tol<R>() * diag0 && d > R(0);
    const R ljj = keep[j] ? sqrt(d) : R(0);
    g[jj + j] = ljj;
    const R inv = keep[j] ? R(1) / ljj : R(0);
    for (int i = j + 1; i < n; ++i) {
      const int ii = i * (i + 1) / 2;
      R v = g[ii + j];
      for (int k = 0; k < j; ++k) v -= g[ii + k] * g[jj + k];
      g[ii + j] = v * inv;
    }
    R zj = b[j];
    for (int k = 0; k < j; ++k) zj -= g[jj + k] * z[k];
    z[j] = zj * inv;
    acc += z[j] * z[j];
  }
  return acc;
}

// Features of one frequency.  zr/zi hold Z_0..Z_2H (Z_0 = 1), yr/yi Y_1..Y_H.
template <int HF, typename R>
__device__ void features_from_sums(const R* zr, const R* zi, const R* yr, const R* yi, R YY,
                                   float log10n, float* out) {
  constexpr int NF = 2 * HF + 2;
  float f[NF];
  const R invYY = R(1) / YY;
  // single harmonics
#pragma unroll
  for (int h = 1; h <= HF; ++h) {
    R g[3], b[2];
    const R C = zr[h], S = zi[h];
    g[0] = R(0.5) * (R(1) + zr[2 * h]) - C * C;  // Cov(cos, cos)
    g[1] = R(0.5) * zi[2 * h] - C * S;            // Cov(sin, cos)
    g[2] = R(0.5) * (R(1) - zr[2 * h]) - S * S;  // Cov(sin, sin)
    b[0] = yr[h];
    b[1] = yi[h];
    f[h - 1] = (float)(quad_form<2>(g, b, 2) * invYY);
    f[HF + h - 1] = (float)((yr[h] * yr[h] + yi[h] * yi[h]) * invYY);
  }
  // multi-harmonic model, basis (cos_1, sin_1, ..., cos_H, sin_H)
  constexpr int NB = 2 * HF;
  R g[NB * (NB + 1) / 2], b[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int n = i / 2 + 1, ci = i & 1;
    b[i] = ci ? yi[n] : yr[n];
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const int m = j / 2 + 1, cj = j & 1;
      const int dnm = n - m;  // >= 0 since i >= j
      const R rd = zr[dnm], id = zi[dnm];  // Z_{n-m}
      const R rs = zr[n + m], is = zi[n + m];
      R e;
      if (!ci && !cj) e = R(0.5) * (rd + rs) - zr[n] * zr[m];
      else if (ci && cj) e = R(0.5) * (rd - rs) - zi[n] * zi[m];
      else if (ci && !cj) e = R(0.5) * (is + id) - zi[n] * zr[m];  // sin_n cos_m
      else e = R(0.5) * (is - id) - zr[n] * zi[m];                 // cos_n sin_m
      g[i * (i + 1) / 2 + j] = e;
    }
  }
  f[2 * HF] = (float)(quad_form<NB>(g, b, NB) * invYY);
  f[2 * HF + 1] = log10n;
#pragma unroll
  for (int j = 0; j < NF; ++j) out[j] = f[j];
}

template <int HF, typename S2, typename R>
__global__ void __launch_bounds__(128) features_kernel(FeatArgs a) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a.status[ST_CODE] != DEV_OK || g >= a.nrows) return;
  // curve of row g: the last curve with row_base <= g
  int lo = 0, hi = a.ncurves;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.curves[mid].row_base <= g) lo = mid;
    else hi = mid;
  }
  const ScreenCurve& c = a.curves[lo];
  const int64_t k = g - c.row_base;
  if (k < 0 || k >= c.nf) return;
  const S2* base = reinterpret_cast<const S2*>(a.sums) + c.sums_off + k;
  R zr[2 * HF + 1], zi[2 * HF + 1], yr[HF + 1], yi[HF + 1];
  zr[0] = R(1);
  zi[0] = R(0);
  yr[0] = yi[0] = R(0);
#pragma unroll
  for (int h = 1; h <= 2 * HF; ++h) {
    const S2 v = base[(int64_t)(h - 1) * c.nf_pad];
    zr[h] = (R)v.x;
    zi[h] = (R)v.y;
  }
#pragma unroll
  for (int h = 1; h <= HF; ++h) {
    const S2 v = base[(int64_t)(2 * c.Hs + h - 1) * c.nf_pad];
    yr[h] = (R)v.x;
    yi[h] = (R)v.y;
  }
  const R YY = (R)a.moments[(size_t)c.curve * MO_WORDS + MO_YY];
  features_from_sums<HF, R>(zr, zi, yr, yi, YY, log10f((float)c.nobs),
                            a.out + (size_t)(c.out_row + k) * (2 * HF + 2));
}

// Order-preserving map of a float to an unsigned key (NaN lowest).
__device__ __forceinline__ uint32_t fkey(float x) {
  if (x != x) return 0u;
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
template <typename T> __device__ __forceinline__ uint32_t key_of(T v) { return fkey((float)v); }

// splitmix64: a counter-based generator (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

constexpr int kSelThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kSelThreads) select_kernel(SelectArgs a, const T* score) {
  __shared__ unsigned hist[256];
  __shared__ uint32_t s_prefix, s_rank;
  const int c = blockIdx.x;
  if (c >= a.ncurves || a.status[ST_CODE] != DEV_OK) return;
  const int64_t base = a.row_off[c], nf = a.row_off[c + 1] - base;
  const T* sc = score + base;
  uint8_t* sel = a.sel + base;
  int64_t K = (int64_t)ceil(a.top_frac * (double)nf);
  K = K < 1 ? 1 : (K > nf ? nf : K);
  // radix select of the K-th largest key, 8 bits per pass from the top
  uint32_t prefix = 0, rank = (uint32_t)K;  // rank-th largest among matching keys
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    const uint32_t hmask = pass == 0 ? 0u : (0xFFFFFFFFu << (shift + 8));
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t k = threadIdx.x; k < nf; k += blockDim.x) {
      const uint32_t key = key_of(sc[k]);
      if ((key & hmask) == (prefix & hmask)) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t acc = 0;
      int d = 255;
      for (; d > 0; --d) {
        if (acc + hist[d] >= rank) break;
        acc += hist[d];
      }
      s_prefix = prefix | ((uint32_t)d << shift);
      s_rank = rank - acc;
    }
    __syncthreads();
    prefix = s_prefix;
    rank = s_rank;
    __syncthreads();
  }
  const uint32_t thr = prefix;
  const int nbr = a.nbr;
  for (int64_t k = threadIdx.x; k < nf; k += blockDim.x) {
    const int64_t k0 = k - nbr < 0 ? 0 : k - nbr, k1 = k + nbr >= nf ? nf - 1 : k + nbr;
    bool on = false;
    for (int64_t j = k0; j <= k1 && !on; ++j) on = key_of(sc[j]) >= thr;
    if (!on && a.rand_threshold != 0)
      on = splitmix64(a.seed ^ (uint64_t)(a.row_global0 + base + k)) < a.rand_threshold;
    sel[k] = on ? 1 : 0;
  }
}

// Work units of one batched roots launch that hold a selected frequency, in
// the kernel's unit numbering (segment s: units seg_units[s] ..; within it,
// template-major blocks of ngw consecutive frequencies).
__global__ void __launch_bounds__(256) unit_list_kernel(const RootsSeg* segs,
                                                        const int64_t* seg_units, int nseg,
                                                        int64_t nunits, int ngw,
                                                        const uint8_t* sel, int64_t* list,
                                                        unsigned long long* count,
                                                        const int* status) {
  __shared__ int s_n;
  __shared__ unsigned long long s_base;
  __shared__ int64_t s_units[256];
  if (status[ST_CODE] != DEV_OK) return;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  bool on = false;
  if (u < nunits) {
    int lo = 0, hi = nseg;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (seg_units[mid] <= u) lo = mid;
      else hi = mid;
    }
    const RootsSeg& sg = segs[lo];
    const int64_t nkb = (sg.nf + ngw - 1) / ngw;
    const int64_t kb = (u - seg_units[lo]) % nkb;
    const int64_t k0 = kb * ngw, k1 = k0 + ngw < sg.nf ? k0 + ngw : sg.nf;
    for (int64_t k = k0; k < k1 && !on; ++k) on = sel[sg.redo_base + k] != 0;
  }
  int slot = -1;
  if (on) slot = atomicAdd(&s_n, 1);
  if (on) s_units[slot] = u;
  __syncthreads();
  if (threadIdx.x == 0) s_base = s_n ? atomicAdd(count, (unsigned long long)s_n) : 0ull;
  __syncthreads();
  // ascending order within the block keeps a warp's units close together
  if (threadIdx.x < s_n) {
    const int64_t mine = s_units[threadIdx.x];
    int r = 0;
    for (int i = 0; i < s_n; ++i) r += s_units[i] < mine;
    list[s_base + r] = mine;
  }
}

__global__ void __launch_bounds__(256) fill_kernel(const ScreenCurve* curves, int ncurves,
                                                   int64_t nitems, double* p, double* t1,
                                                   double* t2, double* t3, uint8_t* flags,
                                                   const int* status) {
  if (status[ST_CODE] != DEV_OK) return;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nitems) return;
  int lo = 0, hi = ncurves;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (curves[mid].item_base <= g) lo = mid;
    else hi = mid;
  }
  const int64_t o = curves[lo].out_off + (g - curves[lo].item_base);
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  p[o] = nan;
  t1[o] = nan;
  t2[o] = nan;
  t3[o] = nan;
  if (flags) flags[o] = FTP_SCREENED_OUT_FLAG;
}

// Ordered compaction of the selected rows: per-block counts, one scan, then
// each block writes its rows at its offset.
constexpr int kGatherRows = 4096;  // rows per block
constexpr int kGatherThreads = 256;

__global__ void __launch_bounds__(kGatherThreads) gather_count_kernel(const uint8_t* sel,
                                                                     int64_t rows,
                                                                     int64_t* block_counts,
                                                                     const int* status) {
  __shared__ int s_n;
  if (status[ST_CODE] != DEV_OK) return;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * kGatherRows;
  int n = 0;
  for (int i = threadIdx.x; i < kGatherRows; i += blockDim.x)
    n += (r0 + i < rows && sel[r0 + i]) ? 1 : 0;
  atomicAdd(&s_n, n);
  __syncthreads();
  if (threadIdx.x == 0) block_counts[blockIdx.x] = s_n;
}

__global__ void __launch_bounds__(1024) gather_scan_kernel(int64_t* block_counts, int64_t nblocks,
                                                           unsigned long long* count,
                                                           const int* status) {
  __shared__ int64_t part[1024];
  __shared__ int64_t s_base;
  if (status[ST_CODE] != DEV_OK) return;
  if (threadIdx.x == 0) s_base = (int64_t)*count;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nblocks; b0 += 1024) {
    const int64_t b = b0 + threadIdx.x;
    const int64_t v = b < nblocks ? block_counts[b] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
      const int64_t add = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (b < nblocks) block_counts[b] = s_base + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 0) s_base += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = (unsigned long long)s_base;
}

__global__ void __launch_bounds__(kGatherThreads) gather_write_kernel(
    const uint8_t* sel, int64_t rows, const float* X, int nfeat, const double* score,
    float* X_out, float* y_out, int64_t cap, const int64_t* block_off, const int* status) {
  __shared__ int s_warp[kGatherThreads / 32];
  if (status[ST_CODE] != DEV_OK) return;
  constexpr int PER = kGatherRows / kGatherThreads;  // consecutive rows per thread
  const int64_t r0 = (int64_t)blockIdx.x * kGatherRows + (int64_t)threadIdx.x * PER;
  int mine = 0;
  for (int i = 0; i < PER; ++i) mine += (r0 + i < rows && sel[r0 + i]) ? 1 : 0;
  // exclusive block scan of `mine`
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += s_warp[w];
  int64_t pos = block_off[blockIdx.x] + before + incl - mine;
  for (int i = 0; i < PER; ++i) {
    const int64_t r = r0 + i;
    if (r < rows && sel[r]) {
      if (pos < cap) {
        for (int j = 0; j < nfeat; ++j) X_out[pos * nfeat + j] = X[r * nfeat + j];
        y_out[pos] = (float)score[r];
      }
      ++pos;
    }
  }
}

template <int HF, typename S2, typename R>
void feat_launch(const FeatArgs& a, cudaStream_t s) {
  const int64_t blocks = (a.nrows + 127) / 128;
  features_kernel<HF, S2, R><<<(unsigned)blocks, 128, 0, s>>>(a);
}

template <typename S2, typename R>
int feat_dispatch(const FeatArgs& a, cudaStream_t s) {
  switch (a.Hf) {
    case 1: feat_launch<1, S2, R>(a, s); break;
    case 2: feat_launch<2, S2, R>(a, s); break;
    case 3: feat_launch<3, S2, R>(a, s); break;
    case 4: feat_launch<4, S2, R>(a, s); break;
    case 5: feat_launch<5, S2, R>(a, s); break;
    case 6: feat_launch<6, S2, R>(a, s); break;
    case 7: feat_launch<7, S2, R>(a, s); break;
    case 8: feat_launch<8, S2, R>(a, s); break;
    default: return -1;
  }
  return 1;
}

}  // namespace

int launch_features(const FeatArgs& a, bool fp64, cudaStream_t s) {
  if (a.nrows <= 0) return 0;
  if (a.nrows > ((int64_t)1 << 31) * 128) return -1;
  return fp64 ? feat_dispatch<double2, double>(a, s) : feat_dispatch<float2, float>(a, s);
}

void launch_select(const SelectArgs& a, const void* score, bool score_fp64, cudaStream_t s) {
  if (a.ncurves <= 0) return;
  if (score_fp64)
    select_kernel<double><<<a.ncurves, kSelThreads, 0, s>>>(a, (const double*)score);
  else
    select_kernel<float><<<a.ncurves, kSelThreads, 0, s>>>(a, (const float*)score);
}

void launch_unit_list(const RootsSeg* segs, const int64_t* seg_units, int nseg, int64_t nunits,
                      int ngw, const uint8_t* sel, int64_t* list, unsigned long long* count,
                      const int* status, cudaStream_t s) {
  if (nunits <= 0) return;
  unit_list_kernel<<<(unsigned)((nunits + 255) / 256), 256, 0, s>>>(
      segs, seg_units, nseg, nunits, ngw, sel, list, count, status);
}

void launch_fill(const ScreenCurve* curves, int ncurves, int64_t nitems, double* p, double* t1,
                 double* t2, double* t3, uint8_t* flags, const int* status, cudaStream_t s) {
  if (nitems <= 0) return;
  fill_kernel<<<(unsigned)((nitems + 255) / 256), 256, 0, s>>>(curves, ncurves, nitems, p, t1,
                                                                t2, t3, flags, status);
}

int launch_gather_rows(const uint8_t* sel, int64_t rows, const float* X, int nfeat,
                       const double* score, float* X_out, float* y_out, int64_t cap,
                       unsigned long long* count, int64_t* block_counts, const int* status,
                       cudaStream_t s) {
  if (rows <= 0) return 0;
  const int64_t nb = (rows + kGatherRows - 1) / kGatherRows;
  gather_count_kernel<<<(unsigned)nb, kGatherThreads, 0, s>>>(sel, rows, block_counts, status);
  gather_scan_kernel<<<1, 1024, 0, s>>>(block_counts, nb, count, status);
  gather_write_kernel<<<(unsigned)nb, kGatherThreads, 0, s>>>(sel, rows, X, nfeat, score, X_out,
                                                             y_out, cap, block_counts, status);
  return 3;
}

}  // namespace ftp
