// Step (a) of the Fast Template Periodogram: the weighted trigonometric sums
// (Section 2, Eqs. CCdef-YSdef) by an adjoint non-equispaced FFT.
//
// All sums the method needs are values of two adjoint transforms on the
// integer lattice of frequencies j * df:
//   Gw[j] = sum_i w_i exp(2 pi i j df t_i),  Gy[j] = sum_i w_i (y_i - ybar) exp(...)
// because h * f_k = h (k0 + k) df.  Z_h(f_k) = Gw[h (k0+k)] (h <= 2H) and
// Y_h(f_k) = Gy[h (k0+k)] (h <= H).  The two real inputs are packed into one
// complex coefficient c_i = w_i + i w_i (y_i - ybar), spread with a
// Kaiser-Bessel window onto n = TILE * ntiles cells covering one period of
// u = frac(df t), transformed with one complex FFT, and separated again with
// the Hermitian symmetry of real-input transforms in the gather kernel, which
// also divides by the window's Fourier transform.
//
// Kernels: moments (FP64 reductions, validation), points (FP64 phase
// reduction into cell + fraction, tile histogram), scan + scatter (counting
// sort of observations by spreading tile), spread (one CTA per tile, shared
// memory accumulation, TMA bulk store of the finished tile: every grid cell is
// written exactly once, no global atomics), gather (deconvolution + harmonic
// gather into the [3H][nf_pad] sum tiles).
#include <math.h>

#include "ftp_internal.cuh"

namespace ftp {

namespace {


struct OpSum {
  template <typename T> __device__ T operator()(T a, T b) const { return a + b; }
};
struct OpMin {
  __device__ double operator()(double a, double b) const { return fmin(a, b); }
};
struct OpMax {
  __device__ double operator()(double a, double b) const { return fmax(a, b); }
};

// Block-wide reduction; every thread receives the result.
template <typename T, typename Op>
__device__ T block_reduce(T v, T* sh, Op op) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    T r = sh[0];
    for (int w = 1; w < nw; ++w) r = op(r, sh[w]);
    sh[0] = r;
  }
  __syncthreads();
  const T r = sh[0];
  __syncthreads();
  return r;
}

// Weighted mean and variance in FP64 with the paper's weight rules
// (Section 2): w_i ~ sigma_i^-2, all sigma = 0 -> unit weights, mixed zero /
// non-zero sigma and Var(y) = 0 are errors.  Two passes (mean, then the sum
// of squared deviations), each a grid-wide reduction: every CTA writes its
// partial, and the CTA that takes the last ticket of an atomic counter
// combines them (no CTA waits for another).
struct MomentPartial {
  double s0, s1, sy, ymin, ymax;  // sum w (sigma > 0), sum w y, sum y, min y, max y
  long long nzero, nbad;
};

// The weight rules on the totals of pass 1: unit weights when every sigma
// is 0, errors for non-finite input, mixed zero / non-zero sigma and
// constant y; writes ybar, the weight sum and the unit flag (YY = 0 so far).
__device__ void finish_pass1(const MomentPartial& q, int64_t n, double* moments, int* status) {
  int code = DEV_OK;
  double wsum = 0, ybar = 0;
  bool unit = false;
  if (q.nbad > 0) {
    code = DEV_NONFINITE;
  } else if (q.nzero == n) {
    unit = true;
    wsum = (double)n;
    ybar = q.sy / (double)n;
  } else if (q.nzero > 0) {
    code = DEV_MIXED_ZERO_SIGMA;
  } else {
    wsum = q.s0;
    ybar = q.s1 / q.s0;
  }
  if (code == DEV_OK && !(q.ymax > q.ymin)) code = DEV_ZERO_VARIANCE;
  moments[MO_YBAR] = ybar;
  moments[MO_YY] = 0.0;
  moments[MO_WSUM] = wsum;
  moments[MO_UNIT] = unit ? 1.0 : 0.0;
  if (code != DEV_OK) atomicCAS(&status[ST_CODE], DEV_OK, code);
}

__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  return last;
}

__global__ void __launch_bounds__(256) moments_pass1(const double* __restrict__ t,
                                                     const double* __restrict__ y,
                                                     const double* __restrict__ dy, int64_t n,
                                                     MomentPartial* part, unsigned* ticket,
                                                     double* moments, int* status) {
  __shared__ double shd[32];
  __shared__ long long shl[32];
  double s0 = 0, s1 = 0, sy = 0, ymin = INFINITY, ymax = -INFINITY;
  long long nzero = 0, nbad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ti = t[i], yi = y[i], si = dy[i];
    if (!isfinite(ti) || !isfinite(yi) || !isfinite(si) || si < 0.0) {
      ++nbad;
      continue;
    }
    sy += yi;
    ymin = fmin(ymin, yi);
    ymax = fmax(ymax, yi);
    if (si == 0.0) {
      ++nzero;
    } else {
      const double w = 1.0 / (si * si);
      s0 += w;
      s1 += w * yi;
    }
  }
  MomentPartial p;
  p.s0 = block_reduce(s0, shd, OpSum());
  p.s1 = block_reduce(s1, shd, OpSum());
  p.sy = block_reduce(sy, shd, OpSum());
  p.ymin = block_reduce(ymin, shd, OpMin());
  p.ymax = block_reduce(ymax, shd, OpMax());
  p.nzero = block_reduce(nzero, shl, OpSum());
  p.nbad = block_reduce(nbad, shl, OpSum());
  if (threadIdx.x == 0) part[blockIdx.x] = p;
  if (!last_block(ticket)) return;
  // the last block reduces the partials with all its threads (L2 loads: the
  // other blocks wrote them)
  s0 = s1 = sy = 0;
  ymin = INFINITY;
  ymax = -INFINITY;
  nzero = nbad = 0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const MomentPartial* r = part + b;
    s0 += __ldcg(&r->s0);
    s1 += __ldcg(&r->s1);
    sy += __ldcg(&r->sy);
    ymin = fmin(ymin, __ldcg(&r->ymin));
    ymax = fmax(ymax, __ldcg(&r->ymax));
    nzero += __ldcg(&r->nzero);
    nbad += __ldcg(&r->nbad);
  }
  MomentPartial q;
  q.s0 = block_reduce(s0, shd, OpSum());
  q.s1 = block_reduce(s1, shd, OpSum());
  q.sy = block_reduce(sy, shd, OpSum());
  q.ymin = block_reduce(ymin, shd, OpMin());
  q.ymax = block_reduce(ymax, shd, OpMax());
  q.nzero = block_reduce(nzero, shl, OpSum());
  q.nbad = block_reduce(nbad, shl, OpSum());
  if (threadIdx.x == 0) {
    finish_pass1(q, n, moments, status);
    *ticket = 0u;  // ready for the next reduction
  }
}

__global__ void __launch_bounds__(256) moments_pass2(const double* __restrict__ y,
                                                     const double* __restrict__ dy, int64_t n,
                                                     double* part, unsigned* ticket,
                                                     double* moments, const int* status) {
  __shared__ double shd[32];
  if (status[ST_CODE] != DEV_OK) return;  // uniform: every CTA returns
  const double ybar = moments[MO_YBAR];
  const bool unit = moments[MO_UNIT] != 0.0;
  double yy = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double si = dy[i];
    const double w = unit ? 1.0 : 1.0 / (si * si);
    const double r = y[i] - ybar;
    yy += w * r * r;
  }
  yy = block_reduce(yy, shd, OpSum());
  if (threadIdx.x == 0) part[blockIdx.x] = yy;
  if (!last_block(ticket)) return;
  double tot = 0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) tot += __ldcg(part + b);
  tot = block_reduce(tot, shd, OpSum());
  if (threadIdx.x == 0) {
    moments[MO_YY] = tot / moments[MO_WSUM];
    *ticket = 0u;
  }
}

// One observation: normalised weight and packed coefficient (w, w (y - ybar)),
// and the FP64 reduction of u = frac(df t) and of its grid position
// x = ngrid u into the returned cell and the fraction (only the fraction is
// handed to the working precision).
template <typename R>
__device__ __forceinline__ int point_of(double t, double y, double dy, double ybar, double wsum,
                                        bool unit, double df, int64_t ngrid, R* frac,
                                        typename C2<R>::type* coef) {
  const double w = (unit ? 1.0 : 1.0 / (dy * dy)) / wsum;
  double u = df * t;
  u -= floor(u);
  const double x = u * (double)ngrid;
  const double fl = floor(x);
  int64_t c = (int64_t)fl;
  if (c >= ngrid) c -= ngrid;
  if (c < 0) c = 0;
  *frac = (R)(x - fl);
  typename C2<R>::type cc;
  cc.x = (R)w;
  cc.y = (R)(w * (y - ybar));
  *coef = cc;
  return (int)c;
}

// Per observation: normalised weight, packed coefficient, FP64 reduction of
// u = frac(df t) and of its grid position x = n u into an integer cell and a
// fraction (only the fraction is handed to the working precision), and the
// spreading-tile histogram.
template <typename R>
__global__ void points_kernel(const double* __restrict__ t, const double* __restrict__ y,
                              const double* __restrict__ dy, int64_t n,
                              const double* __restrict__ moments, const int* __restrict__ status,
                              double df, int64_t ngrid, int* __restrict__ tile_count,
                              int* __restrict__ cell, R* __restrict__ frac,
                              typename C2<R>::type* __restrict__ coef) {
  if (status[ST_CODE] != DEV_OK) return;
  const double ybar = moments[MO_YBAR], wsum = moments[MO_WSUM];
  const bool unit = moments[MO_UNIT] != 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = point_of<R>(t[i], y[i], dy[i], ybar, wsum, unit, df, ngrid, &frac[i], &coef[i]);
    cell[i] = c;
    atomicAdd(&tile_count[c >> kSpreadTileShift], 1);
  }
}

// Exclusive scan of a tile histogram by the whole CTA (blockDim a multiple
// of 32, at most 1024); also clears the cursors.  `sh` holds 32 ints.
__device__ void block_scan_tiles(const int* __restrict__ count, int64_t ntiles,
                                 int* __restrict__ off, int* __restrict__ cursor, int* sh,
                                 int& carry) {
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int v = (i < ntiles) ? count[i] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int nb = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += nb;
    }
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int ws = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int nb = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += nb;
      }
      sh[lane] = ws;
    }
    __syncthreads();
    const int before = carry + (warp > 0 ? sh[warp - 1] : 0) + incl - v;
    if (i < ntiles) {
      off[i] = before;
      cursor[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[ntiles] = carry;
}

// Exclusive scan of the tile histogram (one CTA); also clears the cursors.
__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ count, int64_t ntiles,
                                                     int* __restrict__ off, int* __restrict__ cursor,
                                                     const int* __restrict__ status) {
  __shared__ int sh[32];
  __shared__ int carry;
  if (status[ST_CODE] != DEV_OK) return;
  block_scan_tiles(count, ntiles, off, cursor, sh, carry);
}

template <typename R>
__global__ void scatter_kernel(int64_t n, const int* __restrict__ off, int* __restrict__ cursor,
                               const int* __restrict__ cell, const R* __restrict__ frac,
                               const typename C2<R>::type* __restrict__ coef,
                               int* __restrict__ cell_s, R* __restrict__ frac_s,
                               typename C2<R>::type* __restrict__ coef_s,
                               const int* __restrict__ status) {
  if (status[ST_CODE] != DEV_OK) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = cell[i];
    const int tile = c >> kSpreadTileShift;
    const int pos = off[tile] + atomicAdd(&cursor[tile], 1);
    cell_s[pos] = c;
    frac_s[pos] = frac[i];
    coef_s[pos] = coef[i];
  }
}

// Step (a) preparation of a chunk of curves in one launch, one CTA per
// curve: the two moment passes as block reductions, then per observation the
// weight, coefficient, cell and fraction with the tile histogram, its scan,
// and the scatter into tile order — what moments_pass1/2, points_kernel,
// scan_kernel and scatter_kernel do for one curve, without their launches.
template <typename R>
__device__ void prep_curve(const PrepCurve& pc, double* __restrict__ moments,
                           int* __restrict__ tile_cnt, int* __restrict__ tile_off,
                           int* __restrict__ cell, R* __restrict__ frac,
                           typename C2<R>::type* __restrict__ coef, int* __restrict__ cell_s,
                           R* __restrict__ frac_s, typename C2<R>::type* __restrict__ coef_s,
                           int* status) {
  __shared__ double shd[32];
  __shared__ long long shl[32];
  __shared__ int shi[32];
  __shared__ int carry;
  __shared__ int ok;
  const int64_t n = pc.n;
  // ---- pass 1: weight sums, mean, range, sigma classes
  double s0 = 0, s1 = 0, sy = 0, ymin = INFINITY, ymax = -INFINITY;
  long long nzero = 0, nbad = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double ti = pc.t[i], yi = pc.y[i], si = pc.dy[i];
    if (!isfinite(ti) || !isfinite(yi) || !isfinite(si) || si < 0.0) {
      ++nbad;
      continue;
    }
    sy += yi;
    ymin = fmin(ymin, yi);
    ymax = fmax(ymax, yi);
    if (si == 0.0) {
      ++nzero;
    } else {
      const double w = 1.0 / (si * si);
      s0 += w;
      s1 += w * yi;
    }
  }
  MomentPartial q;
  q.s0 = block_reduce(s0, shd, OpSum());
  q.s1 = block_reduce(s1, shd, OpSum());
  q.sy = block_reduce(sy, shd, OpSum());
  q.ymin = block_reduce(ymin, shd, OpMin());
  q.ymax = block_reduce(ymax, shd, OpMax());
  q.nzero = block_reduce(nzero, shl, OpSum());
  q.nbad = block_reduce(nbad, shl, OpSum());
  if (threadIdx.x == 0) {
    finish_pass1(q, n, moments, status);
    ok = status[ST_CODE] == DEV_OK;
  }
  __syncthreads();
  if (!ok) return;  // uniform
  const double ybar = moments[MO_YBAR], wsum = moments[MO_WSUM];
  const bool unit = moments[MO_UNIT] != 0.0;
  // ---- pass 2: weighted sum of squared deviations
  double yy = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double si = pc.dy[i];
    const double w = unit ? 1.0 : 1.0 / (si * si);
    const double r = pc.y[i] - ybar;
    yy += w * r * r;
  }
  yy = block_reduce(yy, shd, OpSum());
  if (threadIdx.x == 0) moments[MO_YY] = yy / wsum;
  // ---- points and tile histogram
  int* cnt = tile_cnt + pc.tile_base;
  int* off = tile_off + pc.tile_base;
  for (int64_t j = threadIdx.x; j < pc.ntiles; j += blockDim.x) cnt[j] = 0;
  __syncthreads();
  int* cl = cell + pc.obs_base;
  R* fr = frac + pc.obs_base;
  typename C2<R>::type* cf = coef + pc.obs_base;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int c = point_of<R>(pc.t[i], pc.y[i], pc.dy[i], ybar, wsum, unit, pc.df, pc.ngrid,
                              &fr[i], &cf[i]);
    cl[i] = c;
    atomicAdd(&cnt[c >> kSpreadTileShift], 1);
  }
  __syncthreads();
  // ---- scan (the counters become the cursors), scatter into tile order
  block_scan_tiles(cnt, pc.ntiles, off, cnt, shi, carry);
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int c = cl[i];
    const int tile = c >> kSpreadTileShift;
    const int64_t pos = pc.obs_base + off[tile] + atomicAdd(&cnt[tile], 1);
    cell_s[pos] = c;
    frac_s[pos] = fr[i];
    coef_s[pos] = cf[i];
  }
}

template <typename R>
__global__ void __launch_bounds__(512) prep_batch_kernel(
    const PrepCurve* __restrict__ curves, double* __restrict__ moments_all,
    int* __restrict__ tile_cnt, int* __restrict__ tile_off, int* __restrict__ cell,
    R* __restrict__ frac, typename C2<R>::type* __restrict__ coef, int* __restrict__ cell_s,
    R* __restrict__ frac_s, typename C2<R>::type* __restrict__ coef_s, int* status) {
  prep_curve<R>(curves[blockIdx.x], moments_all + (size_t)blockIdx.x * MO_WORDS, tile_cnt,
                tile_off, cell, frac, coef, cell_s, frac_s, coef_s, status);
}

// The same for one curve whose descriptor travels as a kernel parameter (a
// short single curve: one launch instead of six).
template <typename R>
__global__ void __launch_bounds__(512) prep_one_kernel(
    const PrepCurve pc, double* __restrict__ moments, int* __restrict__ tile_cnt,
    int* __restrict__ tile_off, int* __restrict__ cell, R* __restrict__ frac,
    typename C2<R>::type* __restrict__ coef, int* __restrict__ cell_s, R* __restrict__ frac_s,
    typename C2<R>::type* __restrict__ coef_s, int* status) {
  prep_curve<R>(pc, moments, tile_cnt, tile_off, cell, frac, coef, cell_s, frac_s, coef_s,
                status);
}

// Modified Bessel function I0 from its power series sum_k (x^2/4)^k / (k!)^2,
// truncated where the terms fall below the working precision for the window
// shape parameters used here (beta <= 2 pi m with m <= 8).
template <typename R> struct I0Terms;
template <> struct I0Terms<float> { static constexpr int K = 34; };
template <> struct I0Terms<double> { static constexpr int K = 64; };

template <typename R>
__device__ __forceinline__ R bessel_i0(R x) {
  const R q = x * x * R(0.25);
  R term = R(1), sum = R(1);
#pragma unroll
  for (int k = 1; k <= I0Terms<R>::K; ++k) {
    term *= q * (R(1) / R(k * k));
    sum += term;
  }
  return sum;
}

// Kaiser-Bessel window phi(x) = I0(beta sqrt(1 - (x/m)^2)) on |x| <= m.
template <typename R>
__device__ __forceinline__ R kb_window(R x, R inv_m, R beta) {
  const R r = x * inv_m;
  const R a = R(1) - r * r;
  if (a < R(0)) return R(0);
  return bessel_i0(beta * sqrt(a));
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

template <typename R>
__device__ __forceinline__ void smem_atomic_add2(typename C2<R>::type* p, R a, R b) {
  atomicAdd(&p->x, a);
  atomicAdd(&p->y, b);
}

// One CTA per tile of kSpreadTile cells.  The CTA accumulates every window
// contribution that lands in its tile into shared memory - from the points
// binned to its own tile and to its two neighbours, whose windows reach
// across the boundary - and then writes the whole tile, zeros included, with
// one TMA bulk store.  spread_tile does tile b of one curve's grid; the
// single-curve kernel runs one CTA per tile, the batched one walks a list of
// (curve, tile) pairs.
template <typename R>
__device__ __forceinline__ void spread_tile(int64_t b, const int* __restrict__ off,
                                            const int* __restrict__ cell_s,
                                            const R* __restrict__ frac_s,
                                            const typename C2<R>::type* __restrict__ coef_s,
                                            int64_t ngrid, int64_t ntiles, int m, R beta,
                                            typename C2<R>::type* __restrict__ grid,
                                            typename C2<R>::type* tile) {
  using Cx = typename C2<R>::type;
  for (int i = threadIdx.x; i < kSpreadTile; i += blockDim.x) {
    Cx z;
    z.x = R(0);
    z.y = R(0);
    tile[i] = z;
  }
  __syncthreads();
  int64_t nb[3];
  int nnb;
  if (ntiles == 1) {
    nb[0] = 0;
    nnb = 1;
  } else if (ntiles == 2) {
    nb[0] = 0;
    nb[1] = 1;
    nnb = 2;
  } else {
    nb[0] = (b == 0) ? ntiles - 1 : b - 1;
    nb[1] = b;
    nb[2] = (b + 1 == ntiles) ? 0 : b + 1;
    nnb = 3;
  }
  const int w2 = 2 * m;
  const R inv_m = R(1) / R(m);
  for (int q = 0; q < nnb; ++q) {
    const int start = off[nb[q]];
    const int cnt = off[nb[q] + 1] - start;
    const int total = cnt * w2;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int p = start + e / w2;
      const int d = e % w2 - (m - 1);
      int64_t ca = (int64_t)cell_s[p] + d;
      if (ca < 0) ca += ngrid;
      if (ca >= ngrid) ca -= ngrid;
      if ((ca >> kSpreadTileShift) != b) continue;
      const R phi = kb_window<R>((R)d - frac_s[p], inv_m, beta);
      const Cx c = coef_s[p];
      smem_atomic_add2<R>(&tile[ca & (kSpreadTile - 1)], c.x * phi, c.y * phi);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Make the generic-proxy shared-memory writes visible to the bulk copy,
    // and wait until the copy has read the tile before it is reused.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    Cx* dst = grid + b * kSpreadTile;
    asm volatile(
        "cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n\t"
        "cp.async.bulk.commit_group;\n\t"
        "cp.async.bulk.wait_group.read 0;" ::"l"(dst),
        "r"(smem_addr(tile)), "r"((unsigned)(kSpreadTile * sizeof(Cx)))
        : "memory");
  }
  __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(256) spread_kernel(const int* __restrict__ off,
                                                     const int* __restrict__ cell_s,
                                                     const R* __restrict__ frac_s,
                                                     const typename C2<R>::type* __restrict__ coef_s,
                                                     int64_t ngrid, int64_t ntiles, int m, R beta,
                                                     typename C2<R>::type* __restrict__ grid,
                                                     const int* __restrict__ status) {
  using Cx = typename C2<R>::type;
  __shared__ __align__(128) Cx tile[kSpreadTile];
  if (status[ST_CODE] != DEV_OK) return;
  spread_tile<R>(blockIdx.x, off, cell_s, frac_s, coef_s, ngrid, ntiles, m, beta, grid, tile);
}

// Index of the unit-list entry holding global tile t: the last c with
// prefix[c] <= t (prefix has n + 1 ascending entries).
__device__ __forceinline__ int find_curve(const int64_t* __restrict__ prefix, int n, int64_t t) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Spreading of many curves in one launch: global tile t of the list belongs
// to curve c with spread_prefix[c] <= t < spread_prefix[c + 1].
template <typename R>
__global__ void __launch_bounds__(256) spread_batch_kernel(const StepACurve* __restrict__ curves,
                                                           const int64_t* __restrict__ prefix,
                                                           int ncurves, int m, R beta,
                                                           const int* __restrict__ status) {
  using Cx = typename C2<R>::type;
  __shared__ __align__(128) Cx tile[kSpreadTile];
  if (status[ST_CODE] != DEV_OK) return;
  const int64_t total = prefix[ncurves];
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    const int c = find_curve(prefix, ncurves, t);
    const StepACurve cd = curves[c];
    spread_tile<R>(t - prefix[c], cd.tile_off, cd.cell_s, static_cast<const R*>(cd.frac_s),
                   static_cast<const Cx*>(cd.coef_s), cd.ngrid, cd.ntiles, m, beta,
                   static_cast<Cx*>(cd.grid), tile);
  }
}

// Deconvolution and harmonic gather: for frequency index k (K = k0 + k) and
// harmonic h, j = h K; the packed transform X gives
//   Gw[j] = (X[j] + conj X[n-j]) / 2,  Gy[j] = (X[j] - conj X[n-j]) / (2 i),
// each divided by the Kaiser-Bessel transform
//   phihat(nu) = 2 m sinh(sqrt(beta^2 - (2 pi m nu)^2)) / sqrt(...), nu = j/n.
// Tiled by grid index: a CTA reads a tile of T consecutive j (and the mirrored
// n - j) once, coalesced, deconvolves it into shared memory, then for each
// harmonic h writes Z_h(k) (and Y_h(k), h <= Hs) for the consecutive K with
// h K inside the tile - coalesced writes, strided reads from shared memory.
// Every grid value is read once instead of once per harmonic that needs it.
template <typename R> struct GatherTile;
template <> struct GatherTile<float> { static constexpr int T = 2048; };
template <> struct GatherTile<double> { static constexpr int T = 1024; };

// Number of gather tiles of one curve.
template <typename R>
__host__ __device__ __forceinline__ int64_t gather_tiles(int64_t k0, int64_t nf, int Hs) {
  return ((int64_t)2 * Hs * (k0 + nf - 1) - k0) / GatherTile<R>::T + 1;
}

// Gather tile `tile` of one curve (every thread of the CTA calls it).
template <typename R>
__device__ __forceinline__ void gather_tile(int64_t tile, const typename C2<R>::type* __restrict__ X,
                                            int64_t ngrid, int64_t k0, int64_t nf, int64_t nf_pad,
                                            int Hs, int m, R bt, typename C2<R>::type* __restrict__ sums,
                                            typename C2<R>::type* sw, typename C2<R>::type* sy,
                                            int64_t (*kb)[2]) {
  using Cx = typename C2<R>::type;
  constexpr int T = GatherTile<R>::T;
  const int H2 = 2 * Hs;
  const int64_t K1 = k0 + nf - 1;  // largest K
  const int64_t jlo = k0, jhi = (int64_t)H2 * K1;
  const R c2m = R(6.283185307179586476925286766559) * (R)m / (R)ngrid;
  const int64_t J0 = jlo + tile * T;
  const int64_t J1 = J0 + T - 1 < jhi ? J0 + T - 1 : jhi;  // inclusive
  __syncthreads();  // the previous tile's shared values are consumed
  if ((int)threadIdx.x < H2) {
    const int64_t h = threadIdx.x + 1;
    const int64_t lo = (J0 + h - 1) / h, hi = J1 / h;
    kb[threadIdx.x][0] = lo > k0 ? lo : k0;
    kb[threadIdx.x][1] = hi < K1 ? hi : K1;
  }
  for (int i = threadIdx.x; i <= (int)(J1 - J0); i += blockDim.x) {
    const int64_t j = J0 + i;
    const Cx xp = X[j];
    const Cx xm = X[ngrid - j];
    // the window transform in the working precision: its relative error is
    // at the rounding level of the sums themselves
    const R a = c2m * (R)j;
    const R z = sqrt(bt * bt - a * a);
    const R inv = z / (R(2 * m) * sinh(z));
    Cx gw, gy;
    gw.x = R(0.5) * (xp.x + xm.x) * inv;
    gw.y = R(0.5) * (xp.y - xm.y) * inv;
    gy.x = R(0.5) * (xp.y + xm.y) * inv;
    gy.y = -R(0.5) * (xp.x - xm.x) * inv;
    sw[i] = gw;
    sy[i] = gy;
  }
  __syncthreads();
  for (int h = 1; h <= H2; ++h) {
    const int64_t lo = kb[h - 1][0], hi = kb[h - 1][1];
    for (int64_t K = lo + threadIdx.x; K <= hi; K += blockDim.x) {
      const int i = (int)(h * K - J0);
      sums[(int64_t)(h - 1) * nf_pad + (K - k0)] = sw[i];
      if (h <= Hs) sums[(int64_t)(H2 + h - 1) * nf_pad + (K - k0)] = sy[i];
    }
  }
}

// Zeros in the row padding [nf, nf_pad) of one curve's sum rows (the roots
// kernels read whole work units), grid-strided over `nthreads` threads from
// thread index `first`.
template <typename R>
__device__ __forceinline__ void zero_sum_padding(typename C2<R>::type* __restrict__ sums,
                                                 int64_t nf, int64_t nf_pad, int Hs,
                                                 int64_t first, int64_t nthreads) {
  using Cx = typename C2<R>::type;
  const int64_t npad = nf_pad - nf;
  for (int64_t q = first; q < (int64_t)3 * Hs * npad; q += nthreads) {
    Cx zero;
    zero.x = R(0);
    zero.y = R(0);
    sums[(q / npad) * nf_pad + nf + q % npad] = zero;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) gather_kernel(const typename C2<R>::type* __restrict__ X,
                                                     int64_t ngrid, int64_t k0, int64_t nf,
                                                     int64_t nf_pad, int Hs, int m, double beta,
                                                     typename C2<R>::type* __restrict__ sums,
                                                     const int* __restrict__ status) {
  using Cx = typename C2<R>::type;
  constexpr int T = GatherTile<R>::T;
  __shared__ Cx sw[T], sy[T];
  __shared__ int64_t kb[2 * kMaxH][2];  // K range of each harmonic in the tile
  if (status[ST_CODE] != DEV_OK) return;
  zero_sum_padding<R>(sums, nf, nf_pad, Hs, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                      (int64_t)gridDim.x * blockDim.x);
  const int64_t ntiles = gather_tiles<R>(k0, nf, Hs);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    gather_tile<R>(tile, X, ngrid, k0, nf, nf_pad, Hs, m, (R)beta, sums, sw, sy, kb);
}

// Gather of many curves in one launch: global tile t of the list belongs to
// curve c with gather_prefix[c] <= t < gather_prefix[c + 1]; the CTA that
// takes a curve's first tile also zeros its row padding.
template <typename R>
__global__ void __launch_bounds__(256) gather_batch_kernel(const StepACurve* __restrict__ curves,
                                                           const int64_t* __restrict__ prefix,
                                                           int ncurves, int m, double beta,
                                                           const int* __restrict__ status) {
  using Cx = typename C2<R>::type;
  constexpr int T = GatherTile<R>::T;
  __shared__ Cx sw[T], sy[T];
  __shared__ int64_t kb[2 * kMaxH][2];
  if (status[ST_CODE] != DEV_OK) return;
  const int64_t total = prefix[ncurves];
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    const int c = find_curve(prefix, ncurves, t);
    const StepACurve cd = curves[c];
    Cx* sums = static_cast<Cx*>(cd.sums);
    if (t == prefix[c]) zero_sum_padding<R>(sums, cd.nf, cd.nf_pad, cd.Hs, threadIdx.x, blockDim.x);
    gather_tile<R>(t - prefix[c], static_cast<const Cx*>(cd.grid), cd.ngrid, cd.k0, cd.nf,
                   cd.nf_pad, cd.Hs, m, (R)beta, sums, sw, sy, kb);
  }
}


// Direct FP64 sums for the frequencies of a list (the re-solve pass):
// for listed frequency index k, f = (k0 + k) df,
//   Z_h = sum_i w_i e^{i h 2 pi f t_i} (h <= 2 Hs),  Y_h = sum_i w_i (y_i - ybar) e^{...} (h <= Hs),
// with the phase f t_i reduced modulo one cycle in FP64 and the harmonics
// formed by repeated multiplication.  A listed frequency's observations are
// cut into chunks of kDirectChunk; a work item is one (frequency, chunk)
// pair, so even a single listed frequency spreads over many SMs.  Each thread
// sums the terms of its kDirectPerThread observations in registers, each warp
// reduces them with shuffles into the CTA's shared accumulators, and the CTA
// adds those to the frequency's sums in global memory (FP64 atomics; the
// sums are zeroed by a first launch).
constexpr int kDirectThreads = 256;
constexpr int kDirectPerThread = 4;
constexpr int kDirectChunk = kDirectThreads * kDirectPerThread;

// The chunk of observations [i0, i0 + kDirectChunk) of one curve at frequency
// f, added into acc[3 Hs] (Z_1..Z_2Hs, then Y_1..Y_Hs); every thread of the
// CTA calls it.
__device__ void direct_sums_chunk(const double* __restrict__ t, const double* __restrict__ y,
                                  const double* __restrict__ dy, int64_t n, int64_t i0,
                                  double ybar, double wsum, bool unit, double f, int Hs,
                                  double2* acc) {
  const int lane = threadIdx.x & 31;
  double w[kDirectPerThread], r[kDirectPerThread], c1[kDirectPerThread], s1[kDirectPerThread];
  double pc[kDirectPerThread], ps[kDirectPerThread];  // e^{i h phi} of each observation
#pragma unroll
  for (int j = 0; j < kDirectPerThread; ++j) {
    const int64_t i = i0 + threadIdx.x + (int64_t)j * kDirectThreads;
    w[j] = 0.0;
    r[j] = 0.0;
    c1[j] = 1.0;
    s1[j] = 0.0;
    if (i < n) {
      const double si = dy[i];
      w[j] = (unit ? 1.0 : 1.0 / (si * si)) / wsum;
      r[j] = w[j] * (y[i] - ybar);
      double cyc = f * t[i];
      cyc -= floor(cyc);
      sincospi(2.0 * cyc, &s1[j], &c1[j]);
    }
    pc[j] = c1[j];
    ps[j] = s1[j];
  }
  for (int h = 1; h <= 2 * Hs; ++h) {
    double zx = 0.0, zy = 0.0, yx = 0.0, yy = 0.0;
#pragma unroll
    for (int j = 0; j < kDirectPerThread; ++j) {
      zx = fma(w[j], pc[j], zx);
      zy = fma(w[j], ps[j], zy);
      yx = fma(r[j], pc[j], yx);
      yy = fma(r[j], ps[j], yy);
      const double nc = pc[j] * c1[j] - ps[j] * s1[j];
      ps[j] = pc[j] * s1[j] + ps[j] * c1[j];
      pc[j] = nc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      zx += __shfl_xor_sync(0xffffffffu, zx, o);
      zy += __shfl_xor_sync(0xffffffffu, zy, o);
      if (h <= Hs) {
        yx += __shfl_xor_sync(0xffffffffu, yx, o);
        yy += __shfl_xor_sync(0xffffffffu, yy, o);
      }
    }
    if (lane == 0) {
      atomicAdd(&acc[h - 1].x, zx);
      atomicAdd(&acc[h - 1].y, zy);
      if (h <= Hs) {
        atomicAdd(&acc[2 * Hs + h - 1].x, yx);
        atomicAdd(&acc[2 * Hs + h - 1].y, yy);
      }
    }
  }
}

// Zero the sums of the listed slots (rows of `stride` elements).
__global__ void __launch_bounds__(256) zero_listed_kernel(const int* __restrict__ count, int cap,
                                                          int rows, int64_t stride,
                                                          double2* __restrict__ sums,
                                                          int64_t sums_elems) {
  const int64_t total = min(*count, cap);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total * rows;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = (q / total) * stride + q % total;
    if (e < sums_elems) sums[e] = make_double2(0.0, 0.0);
  }
}

__global__ void __launch_bounds__(kDirectThreads) direct_sums_kernel(
    const double* __restrict__ t, const double* __restrict__ y, const double* __restrict__ dy,
    int64_t n, const double* __restrict__ moments, const int* __restrict__ status, double df,
    int64_t k0, const int* __restrict__ list, const int* __restrict__ count, int cap, int Hs,
    int64_t nf_pad, double2* __restrict__ sums, int64_t sums_elems, int* status_rw) {
  __shared__ double2 acc[3 * kMaxH];
  if (status[ST_CODE] != DEV_OK) return;
  if (!FTP_DCHECK(status_rw, Hs >= 1 && Hs <= kMaxH, 31, Hs, kMaxH)) return;
  const int64_t total = min(*count, cap);
  const int64_t nchunk = (n + kDirectChunk - 1) / kDirectChunk;
  const double ybar = moments[MO_YBAR], wsum = moments[MO_WSUM];
  const bool unit = moments[MO_UNIT] != 0.0;
  for (int64_t item = blockIdx.x; item < total * nchunk; item += gridDim.x) {
    const int64_t idx = item / nchunk, chunk = item % nchunk;
    if (!FTP_DCHECK(status_rw, list[idx] >= 0 && list[idx] < nf_pad, 32, list[idx], nf_pad)) break;
    const double f = (double)(k0 + list[idx]) * df;
    for (int q = threadIdx.x; q < 3 * Hs; q += blockDim.x) acc[q] = make_double2(0.0, 0.0);
    __syncthreads();
    direct_sums_chunk(t, y, dy, n, chunk * kDirectChunk, ybar, wsum, unit, f, Hs, acc);
    __syncthreads();
    for (int q = threadIdx.x; q < 3 * Hs; q += blockDim.x)
      if (FTP_DCHECK(status_rw, (int64_t)q * nf_pad + idx < sums_elems, 33, q, idx)) {
        atomicAdd(&sums[(int64_t)q * nf_pad + idx].x, acc[q].x);
        atomicAdd(&sums[(int64_t)q * nf_pad + idx].y, acc[q].y);
      }
    __syncthreads();
  }
}

// Batched form: slot idx holds a global frequency index g of the batch; its
// curve is the last one with redo_base <= g.  Work items are (slot, chunk)
// over the chunks of the longest curve (max_n observations); chunks past a
// curve's end are skipped.
__global__ void __launch_bounds__(kDirectThreads) direct_sums_batch_kernel(
    const CurveDesc* __restrict__ curves, int ncurves, const double* __restrict__ moments,
    const int* __restrict__ status, const int* __restrict__ list, const int* __restrict__ count,
    int cap, int64_t max_n, int64_t stride, double2* __restrict__ sums, int64_t sums_elems,
    int* __restrict__ slot_curve, int* status_rw) {
  __shared__ double2 acc[3 * kMaxH];
  if (status[ST_CODE] != DEV_OK) return;
  const int64_t total = min(*count, cap);
  const int64_t nchunk = (max_n + kDirectChunk - 1) / kDirectChunk;
  for (int64_t item = blockIdx.x; item < total * nchunk; item += gridDim.x) {
    const int64_t idx = item / nchunk, chunk = item % nchunk;
    const int64_t g = list[idx];
    int lo = 0, hi = ncurves;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (curves[mid].redo_base <= g) lo = mid;
      else hi = mid;
    }
    const CurveDesc cd = curves[lo];
    if (chunk == 0 && threadIdx.x == 0) slot_curve[idx] = lo;
    if (chunk * kDirectChunk >= cd.n) continue;  // uniform over the CTA
    const int64_t k = g - cd.redo_base;
    if (!FTP_DCHECK(status_rw, k >= 0 && k < cd.nf, 34, k, cd.nf) ||
        !FTP_DCHECK(status_rw, cd.Hs >= 1 && cd.Hs <= kMaxH, 35, cd.Hs, kMaxH))
      break;
    const double* mo = moments + (size_t)lo * MO_WORDS;
    const double f = (double)(cd.k0 + k) * cd.df;
    for (int q = threadIdx.x; q < 3 * cd.Hs; q += blockDim.x) acc[q] = make_double2(0.0, 0.0);
    __syncthreads();
    direct_sums_chunk(cd.t, cd.y, cd.dy, cd.n, chunk * kDirectChunk, mo[MO_YBAR], mo[MO_WSUM],
                      mo[MO_UNIT] != 0.0, f, cd.Hs, acc);
    __syncthreads();
    for (int q = threadIdx.x; q < 3 * cd.Hs; q += blockDim.x)
      if (FTP_DCHECK(status_rw, (int64_t)q * stride + idx < sums_elems, 36, q, idx)) {
        atomicAdd(&sums[(int64_t)q * stride + idx].x, acc[q].x);
        atomicAdd(&sums[(int64_t)q * stride + idx].y, acc[q].y);
      }
    __syncthreads();
  }
}

// SM count of the current device, read once per device ordinal.
int current_sms() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }
  if (cache[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 1;
    }
    cache[dev] = n;
  }
  return cache[dev];
}

// Grid-stride launches: enough CTAs for n / threads, at most 16 per SM.
inline int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  const int64_t cap = (int64_t)current_sms() * 16;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace

void launch_moments(const double* t, const double* y, const double* dy, int64_t n,
                    double* moments, int* status, void* scratch, cudaStream_t s) {
  // scratch: [kMomentBlocks] partials + one ticket (zero between uses)
  int blocks = (int)((n + 255) / 256);
  if (blocks > kMomentBlocks) blocks = kMomentBlocks;
  if (blocks < 1) blocks = 1;
  auto* part = static_cast<MomentPartial*>(scratch);
  auto* ticket = reinterpret_cast<unsigned*>(static_cast<char*>(scratch) + kMomentScratchBytes - 16);
  moments_pass1<<<blocks, 256, 0, s>>>(t, y, dy, n, part, ticket, moments, status);
  moments_pass2<<<blocks, 256, 0, s>>>(y, dy, n, reinterpret_cast<double*>(part), ticket, moments,
                                       status);
}


void launch_direct_sums(const double* t, const double* y, const double* dy, int64_t n,
                        const double* moments, const int* status, double df, int64_t k0,
                        const int* list, const int* count, int cap, int Hs, int64_t nf_pad,
                        double2* sums, int64_t sums_elems, int* status_rw, cudaStream_t s) {
  const int sms = current_sms();
  zero_listed_kernel<<<sms, 256, 0, s>>>(count, cap, 3 * Hs, nf_pad, sums, sums_elems);
  direct_sums_kernel<<<4 * sms, kDirectThreads, 0, s>>>(t, y, dy, n, moments, status, df, k0,
                                                        list, count, cap, Hs, nf_pad, sums,
                                                        sums_elems, status_rw);
}

__global__ void __launch_bounds__(256) redo_overflow_kernel(const CurveDesc* __restrict__ curves,
                                                            int ncurves,
                                                            const int* __restrict__ marks,
                                                            int64_t nmarks,
                                                            const int* __restrict__ count,
                                                            int cap, uint8_t* __restrict__ flags) {
  if (*count <= cap) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nmarks; g += stride) {
    if ((marks[g] & MARK_OVERFLOW) == 0) continue;
    int lo = 0, hi = ncurves;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (curves[mid].redo_base <= g) lo = mid;
      else hi = mid;
    }
    const CurveDesc& cd = curves[lo];
    const int64_t k = g - cd.redo_base;
    if (k < 0 || k >= cd.nf) continue;
    for (int r = 0; r < cd.nrows; ++r) flags[cd.out_off + (int64_t)r * cd.nf + k] |= 16u;
  }
}

void launch_redo_overflow(const CurveDesc* curves, int ncurves, const int* marks, int64_t nmarks,
                          const int* count, int cap, uint8_t* flags, cudaStream_t s) {
  redo_overflow_kernel<<<2 * current_sms(), 256, 0, s>>>(curves, ncurves, marks, nmarks, count, cap,
                                                         flags);
}

void launch_direct_sums_batch(const CurveDesc* curves, int ncurves, const double* moments,
                              const int* status, const int* list, const int* count, int cap,
                              int64_t max_n, int Hs_max, int64_t stride, double2* sums,
                              int64_t sums_elems, int* slot_curve, int* status_rw,
                              cudaStream_t s) {
  const int sms = current_sms();
  zero_listed_kernel<<<sms, 256, 0, s>>>(count, cap, 3 * Hs_max, stride, sums, sums_elems);
  direct_sums_batch_kernel<<<4 * sms, kDirectThreads, 0, s>>>(curves, ncurves, moments, status,
                                                              list, count, cap, max_n, stride,
                                                              sums, sums_elems, slot_curve,
                                                              status_rw);
}

template <typename R>
void launch_points(const double* t, const double* y, const double* dy, int64_t n,
                   const double* moments, const int* status, double df, int64_t ngrid,
                   int* tile_count, int* cell, R* frac, typename C2<R>::type* coef,
                   cudaStream_t s) {
  points_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(t, y, dy, n, moments, status, df, ngrid,
                                                     tile_count, cell, frac, coef);
}

void launch_scan(const int* tile_count, int64_t ntiles, int* tile_off, int* cursor,
                 const int* status, cudaStream_t s) {
  scan_kernel<<<1, 1024, 0, s>>>(tile_count, ntiles, tile_off, cursor, status);
}

template <typename R>
void launch_scatter(int64_t n, const int* tile_off, int* cursor, const int* cell, const R* frac,
                    const typename C2<R>::type* coef, int* cell_s, R* frac_s,
                    typename C2<R>::type* coef_s, const int* status, cudaStream_t s) {
  scatter_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(n, tile_off, cursor, cell, frac, coef,
                                                      cell_s, frac_s, coef_s, status);
}

template <typename R>
void launch_spread(const int* tile_off, const int* cell_s, const R* frac_s,
                   const typename C2<R>::type* coef_s, int64_t ngrid, int64_t ntiles, int m,
                   double beta, typename C2<R>::type* grid, const int* status, cudaStream_t s) {
  spread_kernel<R><<<(unsigned)ntiles, 256, 0, s>>>(tile_off, cell_s, frac_s, coef_s, ngrid,
                                                     ntiles, m, (R)beta, grid, status);
}

template <typename R>
void launch_gather(const typename C2<R>::type* X, int64_t ngrid, int64_t k0, int64_t nf,
                   int64_t nf_pad, int Hs, int m, double beta, typename C2<R>::type* sums,
                   const int* status, cudaStream_t s) {
  const int64_t ntiles = gather_tiles<R>(k0, nf, Hs);
  const int64_t bmax = (int64_t)current_sms() * 6;
  int64_t blocks = ntiles < bmax ? ntiles : bmax;
  if (blocks < 1) blocks = 1;
  gather_kernel<R><<<(unsigned)blocks, 256, 0, s>>>(X, ngrid, k0, nf, nf_pad, Hs, m, beta, sums,
                                                    status);
}

template <typename R>
void launch_prep_batch(const PrepCurve* curves, int ncurves, double* moments, int* tile_cnt,
                       int* tile_off, int* cell, R* frac, typename C2<R>::type* coef, int* cell_s,
                       R* frac_s, typename C2<R>::type* coef_s, int* status, cudaStream_t s) {
  if (ncurves < 1) return;
  prep_batch_kernel<R><<<(unsigned)ncurves, 512, 0, s>>>(curves, moments, tile_cnt, tile_off,
                                                          cell, frac, coef, cell_s, frac_s,
                                                          coef_s, status);
}

template <typename R>
void launch_prep_one(const PrepCurve& pc, double* moments, int* tile_cnt, int* tile_off,
                     int* cell, R* frac, typename C2<R>::type* coef, int* cell_s, R* frac_s,
                     typename C2<R>::type* coef_s, int* status, cudaStream_t s) {
  prep_one_kernel<R><<<1, 512, 0, s>>>(pc, moments, tile_cnt, tile_off, cell, frac, coef, cell_s,
                                        frac_s, coef_s, status);
}

template <typename R>
void launch_spread_batch(const StepACurve* curves, const int64_t* spread_prefix, int ncurves,
                         int64_t total_tiles, int m, double beta, const int* status,
                         cudaStream_t s) {
  const int64_t bmax = (int64_t)current_sms() * 8;
  int64_t blocks = total_tiles < bmax ? total_tiles : bmax;
  if (blocks < 1) blocks = 1;
  spread_batch_kernel<R><<<(unsigned)blocks, 256, 0, s>>>(curves, spread_prefix, ncurves, m,
                                                           (R)beta, status);
}

template <typename R>
void launch_gather_batch(const StepACurve* curves, const int64_t* gather_prefix, int ncurves,
                         int64_t total_tiles, int m, double beta, const int* status,
                         cudaStream_t s) {
  const int64_t bmax = (int64_t)current_sms() * 6;
  int64_t blocks = total_tiles < bmax ? total_tiles : bmax;
  if (blocks < 1) blocks = 1;
  gather_batch_kernel<R><<<(unsigned)blocks, 256, 0, s>>>(curves, gather_prefix, ncurves, m, beta,
                                                           status);
}

int64_t gather_tile_count(bool fp64, int64_t k0, int64_t nf, int Hs) {
  return fp64 ? gather_tiles<double>(k0, nf, Hs) : gather_tiles<float>(k0, nf, Hs);
}

#define FTP_INST(R)                                                                            \
  template void launch_points<R>(const double*, const double*, const double*, int64_t,         \
                                 const double*, const int*, double, int64_t, int*, int*, R*,   \
                                 C2<R>::type*, cudaStream_t);                                  \
  template void launch_scatter<R>(int64_t, const int*, int*, const int*, const R*,             \
                                  const C2<R>::type*, int*, R*, C2<R>::type*, const int*,      \
                                  cudaStream_t);                                               \
  template void launch_spread<R>(const int*, const int*, const R*, const C2<R>::type*,         \
                                 int64_t, int64_t, int, double, C2<R>::type*, const int*,      \
                                 cudaStream_t);                                                \
  template void launch_gather<R>(const C2<R>::type*, int64_t, int64_t, int64_t, int64_t, int,  \
                                 int, double, C2<R>::type*, const int*, cudaStream_t);         \
  template void launch_prep_batch<R>(const PrepCurve*, int, double*, int*, int*, int*, R*,      \
                                     C2<R>::type*, int*, R*, C2<R>::type*, int*, cudaStream_t); \
  template void launch_prep_one<R>(const PrepCurve&, double*, int*, int*, int*, R*,             \
                                   C2<R>::type*, int*, R*, C2<R>::type*, int*, cudaStream_t);   \
  template void launch_spread_batch<R>(const StepACurve*, const int64_t*, int, int64_t, int,    \
                                       double, const int*, cudaStream_t);                       \
  template void launch_gather_batch<R>(const StepACurve*, const int64_t*, int, int64_t, int,    \
                                       double, const int*, cudaStream_t);
FTP_INST(float)
FTP_INST(double)
#undef FTP_INST

}  // namespace ftp
