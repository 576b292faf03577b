// Steps (b) and (c) of the Fast Template Periodogram, fused in one kernel:
// polynomial assembly (Section 2: MM_nm, YM_k, Eq. finalpoly), all zeros of
// the final polynomial by Aberth-Ehrlich iteration, candidates scaled onto
// the unit circle (Section 2, end), the best one chosen and polished by a
// Newton step on the phase in FP64, and (theta1, theta2, theta3, P).
//
// Work item = (frequency k, template tau).  A group of G lanes owns one item:
// it assembles the coefficients, then each lane iterates R = ceil(D/G) of the
// D = 6H-2 roots.  Each warp takes work units (32/G consecutive frequencies of
// one template) from a global queue and stages their sum tiles (3H rows in the
// [3H][nf_pad] layout) into its own shared memory with TMA bulk copies,
// double-buffered so the next unit's copy overlaps this unit's arithmetic.
// Warps never wait for each other.
//
// Notation.  Z_h = sum_i w_i e^{i h omega t_i} (Z_0 = 1, Z_{-h} = conj Z_h),
// Y_h = sum_i w_i (y_i - ybar) e^{i h omega t_i}, alpha_n = (c_n + i s_n)/2.
// The covariance sums of Eqs. CCdef-SSdef combine into
//   CCt_nm = conj(Z_{n+m} - Z_n Z_m),  CSt_nm = Z_{m-n} - conj(Z_n) Z_m
// (product-to-sum identities), and the self-inversive polynomials MM', YM'
// are kept as real trigonometric polynomials in theta = theta2:
//   MM(theta) = a_0 + 2 Re sum_{e=1..2H} a_e psi^e,  a_e = [psi^{2H+e}] MM'
//   YM(theta) = 2 Re sum_{k=1..H} b_k psi^k,         b_k = alpha_k conj(Y_k)
//   Mbar(theta) = 2 Re sum_{n=1..H} c_n psi^n,        c_n = alpha_n conj(Z_n)
// The final polynomial F = 2 MM' d(YM') - YM' d(MM') is anti-self-inversive,
// F_{D-p} = -conj(F_p), so only p = 0..3H-1 are formed and the rest mirrored.
//
// Precision.  a_e, b_k, c_n are always assembled in FP64 and the chosen phase
// is always polished and evaluated in FP64.  F, the Aberth iteration and the
// candidate screening run in the kernel's working precision R (float for the
// mixed path, double for the FP64 path).  The sum tiles are float2 (mixed,
// from the FP32 NFFT) or double2 (FP64 NFFT, or direct FP64 sums of the
// re-solve pass).
#pragma once

#include <math.h>

#include "ftp_internal.cuh"

namespace ftp {
namespace roots {

__host__ __device__ constexpr size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }
__host__ __device__ constexpr int cdiv_i(int a, int b) { return (a + b - 1) / b; }

template <typename R> struct R2T;
template <> struct R2T<float> { using type = float2; };
template <> struct R2T<double> { using type = double2; };

// S2: sum tile element; R: Aberth / screening precision; G: lanes per item.
template <typename S2, typename R, int H, int G>
struct Cfg {
  using R2 = typename R2T<R>::type;
  static constexpr bool kFast = sizeof(R) == 4;   // FP32 Aberth
  static constexpr int D = 6 * H - 2;
  static constexpr int RR = cdiv_i(D, G);         // roots per lane
  static constexpr int NGW = 32 / G;              // items per warp unit
  static constexpr int WARPS = 4;                 // warps per CTA
  static constexpr int ROWS = 3 * H;              // staged sum rows
  static constexpr int NA = 2 * H + 1;            // a_0..a_2H, Z_0..Z_2H
  static constexpr int NB = H + 1;                // b_0..b_H, c_0..c_H, Y_0..Y_H
  static constexpr int NF = 3 * H;                // F_0..F_{3H-1}
  static constexpr int NFL = cdiv_i(NF, G);
  static constexpr int NSLOT = H + 1;             // assembly slots {0}, {e, 2H+1-e}
  // per-group shared memory (bytes)
  static constexpr size_t G_Z64 = 0;
  static constexpr size_t G_Y64 = G_Z64 + NA * 16;
  static constexpr size_t G_A64 = G_Y64 + NB * 16;
  static constexpr size_t G_B64 = G_A64 + NA * 16;
  static constexpr size_t G_C64 = G_B64 + NB * 16;
  static constexpr size_t G_F = G_C64 + NB * 16;
  static constexpr size_t G_Z = G_F + rup((D + 1) * sizeof(R2), 16);
  static constexpr size_t G_AW = G_Z + rup(RR * G * sizeof(R2), 16);
  static constexpr size_t G_BW = G_AW + (kFast ? rup(NA * sizeof(R2), 16) : 0);
  static constexpr size_t G_END = G_BW + (kFast ? rup(NB * sizeof(R2), 16) : 0);
  static constexpr size_t GROUP_BYTES = rup(G_END, 16);
  // per-warp shared memory
  static constexpr size_t ROW_BYTES = NGW * sizeof(S2);
  static constexpr size_t STAGE_BYTES = ROWS * ROW_BYTES;
  static constexpr size_t W_STAGE = 0;                                   // 2 buffers
  static constexpr size_t W_MBAR = rup(2 * STAGE_BYTES, 16);             // 2 mbarriers
  static constexpr size_t W_AA = W_MBAR + 16;                            // alpha_n alpha_m
  static constexpr size_t W_AC = W_AA + H * H * 16;                      // alpha_n conj alpha_m
  static constexpr size_t W_AL = W_AC + H * H * 16;                      // alpha_n
  static constexpr size_t W_GROUPS = rup(W_AL + H * 16, 128);
  static constexpr size_t WARP_BYTES = rup(W_GROUPS + NGW * GROUP_BYTES, 128) + 16;
  static constexpr size_t SMEM = WARPS * WARP_BYTES;
};

// ------------------------------------------------------------ complex helpers
template <typename T2> __device__ __forceinline__ T2 mk(double x, double y) {
  T2 r;
  r.x = x;
  r.y = y;
  return r;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * b + c
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
template <typename T2> __device__ __forceinline__ T2 cconj(T2 a) {
  a.y = -a.y;
  return a;
}
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
template <typename T2, typename T> __device__ __forceinline__ T2 cscale(T2 a, T s) {
  a.x *= s;
  a.y *= s;
  return a;
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }
template <typename T2> __device__ __forceinline__ T2 cdiv(T2 a, T2 b) {
  const auto inv = fast_rcp(cabs2(b));
  return mk<T2>((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
template <typename T2> __device__ __forceinline__ T2 from_d2(double2 v) {
  return mk<T2>(v.x, v.y);
}
template <typename T> __device__ __forceinline__ bool finite2(T v) {
  return isfinite(v.x) && isfinite(v.y);
}

// ------------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ unsigned saddr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gaddr(const void* p) {
  unsigned long long g;
  asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(p));
  return g;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(saddr(dst)),
      "l"(gaddr(src)), "r"(bytes), "r"(saddr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after a fixed number of polls instead of spinning
// forever if a copy never lands.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (int i = 0; i < (1 << 20); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ------------------------------------------------------------ group reductions
template <int G, typename T> __device__ __forceinline__ T gsum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}
template <int G, typename T> __device__ __forceinline__ T gmax(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o, G));
  return v;
}
template <int G> __device__ __forceinline__ bool gor(bool v) {
  int x = v ? 1 : 0;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o, G);
  return x != 0;
}
// psi^(gl+1) in lane gl of each group (inclusive product scan over the group).
template <int G>
__device__ __forceinline__ double2 group_powers(double2 psi, int gl) {
  double2 pw = psi;
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    double2 v;
    v.x = __shfl_up_sync(0xffffffffu, pw.x, o, G);
    v.y = __shfl_up_sync(0xffffffffu, pw.y, o, G);
    if (gl >= o) pw = cmul(pw, v);
  }
  return pw;
}

// Real trigonometric polynomial in the working precision, |psi| = 1:
//   v0 + 2 Re sum_{e=1..n} c_e psi^e  (Horner in psi).
template <typename T2, typename T>
__device__ __forceinline__ T trig_eval(const T2* c, int n, T2 psi, T v0) {
  T2 acc = c[n];
  for (int e = n - 1; e >= 1; --e) acc = cfma(acc, psi, c[e]);
  acc = cmul(acc, psi);
  return v0 + T(2) * acc.x;
}

template <typename S2, typename R, int H, int G>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 4 : 3) roots_kernel(const RootsArgs a) {
  using C = Cfg<S2, R, H, G>;
  using R2 = typename C::R2;
  constexpr int D = C::D, RR = C::RR, NGW = C::NGW;
  constexpr bool kFast = C::kFast;
  constexpr R kTwoPi = R(6.283185307179586476925286766559);
  constexpr double kTwoPiD = 6.283185307179586476925286766559;
  constexpr R tol = kFast ? R(2e-6) : R(1e-12);
  constexpr R tie = kFast ? R(1e-6) : R(1e-12);
  // F ~ 0 relative to |a| |b| (rounding level of the working precision)
  constexpr double const_rel = kFast ? 1e-5 : 1e-13;

  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wb = smem + (size_t)warp * C::WARP_BYTES;
  S2* stage = reinterpret_cast<S2*>(wb + C::W_STAGE);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(wb + C::W_MBAR);
  double2* AA = reinterpret_cast<double2*>(wb + C::W_AA);
  double2* AC = reinterpret_cast<double2*>(wb + C::W_AC);
  double2* AL = reinterpret_cast<double2*>(wb + C::W_AL);
  const int gl = lane % G, gi = lane / G;
  unsigned char* gb = wb + C::W_GROUPS + (size_t)gi * C::GROUP_BYTES;
  double2* Z64 = reinterpret_cast<double2*>(gb + C::G_Z64);
  double2* Y64 = reinterpret_cast<double2*>(gb + C::G_Y64);
  double2* A64 = reinterpret_cast<double2*>(gb + C::G_A64);
  double2* B64 = reinterpret_cast<double2*>(gb + C::G_B64);
  double2* C64 = reinterpret_cast<double2*>(gb + C::G_C64);
  R2* Fs = reinterpret_cast<R2*>(gb + C::G_F);
  R2* Zs = reinterpret_cast<R2*>(gb + C::G_Z);
  R2* Aw = kFast ? reinterpret_cast<R2*>(gb + C::G_AW) : reinterpret_cast<R2*>(A64);
  R2* Bw = kFast ? reinterpret_cast<R2*>(gb + C::G_BW) : reinterpret_cast<R2*>(B64);

  if (a.status[ST_CODE] != DEV_OK) return;
  const int64_t nf = a.nf_dev ? (int64_t)*a.nf_dev : a.nf;
  const int64_t nkb = (nf + NGW - 1) / NGW;
  const int64_t nunits = nkb * a.ntpl;
  const double ybar = a.moments[MO_YBAR], YY = a.moments[MO_YY];

  if (lane == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_fence_init();
  }
  __syncwarp();

  auto grab = [&]() -> int64_t {
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(a.queue, 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, v, 0);
  };
  // Lane 0 stages the 3H sum rows of unit u into buffer `buf`.
  auto issue = [&](int64_t u, int buf) {
    if (lane != 0) return;
    const int64_t kb = u % nkb;
    S2* dst = stage + (size_t)buf * (C::STAGE_BYTES / sizeof(S2));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&mbar[buf], (unsigned)C::STAGE_BYTES);
    const S2* sums = reinterpret_cast<const S2*>(a.sums);
#pragma unroll 1
    for (int r = 0; r < C::ROWS; ++r) {
      const int src_row = (r < 2 * H) ? r : 2 * a.Hs + (r - 2 * H);
      const int64_t off = (int64_t)src_row * a.nf_pad + kb * NGW;
      if (!FTP_DCHECK(a.status, off >= 0 && off + NGW <= a.sums_elems, 11, off, a.sums_elems) ||
          !FTP_DCHECK(a.status, (gaddr(sums + off) & 15) == 0, 12, gaddr(sums + off) & 15, 16) ||
          !FTP_DCHECK(a.status, (saddr(dst + (size_t)r * NGW) & 15) == 0, 13, 0, 16)) {
        continue;  // the row never lands: the bounded wait reports a timeout
      }
      bulk_g2s(dst + (size_t)r * NGW, sums + off, (unsigned)C::ROW_BYTES, &mbar[buf]);
    }
  };

  unsigned long long st_iters = 0, st_items = 0, st_nonconv = 0, st_redo = 0;
  unsigned parity[2] = {0u, 0u};
  int buf = 0, cur_tau = -1;
  double sum_abs_alpha = 0.0;
  int64_t u = grab();
  if (u < nunits) issue(u, 0);
  while (u < nunits) {
    const int64_t un = grab();
    if (un < nunits) issue(un, buf ^ 1);
    const int tau = (int)(u / nkb);
    const int64_t kb = u % nkb;
    if (tau != cur_tau) {  // warp-uniform: this warp's template tables
      for (int i = lane; i < H * H; i += 32) {
        const int n = i / H, m = i % H;
        const double2 an = a.alpha[(size_t)tau * kMaxH + n];
        const double2 am = a.alpha[(size_t)tau * kMaxH + m];
        AA[i] = cmul(an, am);
        AC[i] = cmul(an, cconj(am));
      }
      if (lane < H) AL[lane] = a.alpha[(size_t)tau * kMaxH + lane];
      sum_abs_alpha = 0.0;
      for (int n = 0; n < H; ++n) sum_abs_alpha += sqrt(cabs2(a.alpha[(size_t)tau * kMaxH + n]));
      cur_tau = tau;
      __syncwarp();
    }
    const bool landed = mbar_wait(&mbar[buf], parity[buf]);
    parity[buf] ^= 1u;
    if (__any_sync(0xffffffffu, !landed)) {
      if (lane == 0) atomicCAS(&a.status[ST_CODE], DEV_OK, DEV_TIMEOUT);
      break;
    }
    const S2* st = stage + (size_t)buf * (C::STAGE_BYTES / sizeof(S2));
    const int64_t k = kb * NGW + gi;
    const bool valid = k < nf;

    // ---- sums of this item into FP64 shared memory (one conversion each)
    for (int q = gl; q < C::ROWS; q += G) {
      const double2 v = to_d2(st[q * NGW + gi]);
      if (q < 2 * H) Z64[q + 1] = v;
      else Y64[q - 2 * H + 1] = v;
    }
    if (gl == 0) {
      Z64[0] = make_double2(1.0, 0.0);
      Y64[0] = make_double2(0.0, 0.0);
    }
    __syncwarp();

    // ---- (b) FP64 assembly of a_e: slot 0 = {0}, slot s = {s, 2H+1-s}
    double amax2 = 0.0, bmax2 = 0.0;
    for (int s = gl; s < C::NSLOT; s += G) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        if (s == 0 && half == 1) break;
        const int e = (s == 0) ? 0 : (half == 0 ? s : 2 * H + 1 - s);
        double2 acc = make_double2(0.0, 0.0);
        if (e == 0) {
          for (int n = 1; n <= H; ++n)
            acc.x += 2.0 * AC[(n - 1) * H + (n - 1)].x * (1.0 - cabs2(Z64[n]));
        } else {
          const double2 Ze = Z64[e];
          // alpha_n alpha_m conj(Z_e - Z_n Z_m) over n + m = e; symmetric in (n, m)
          const int nlo = e - H > 1 ? e - H : 1;
          for (int n = nlo; 2 * n <= e; ++n) {
            const int m = e - n;
            const double2 t = cconj(csub(Ze, cmul(Z64[n], Z64[m])));
            const double2 w = AA[(n - 1) * H + (m - 1)];
            acc = cfma(n == m ? w : cscale(w, 2.0), t, acc);
          }
          // 2 alpha_n conj(alpha_m) (conj(Z_e) - conj(Z_n) Z_m) over n - m = e
          for (int n = e + 1; n <= H; ++n) {
            const int m = n - e;
            const double2 t = csub(cconj(Ze), cmul(cconj(Z64[n]), Z64[m]));
            acc = cfma(cscale(AC[(n - 1) * H + (m - 1)], 2.0), t, acc);
          }
        }
        A64[e] = acc;
        if constexpr (kFast) Aw[e] = from_d2<R2>(acc);
        amax2 = fmax(amax2, cabs2(acc));
      }
    }
    for (int kk = gl; kk <= H; kk += G) {
      double2 bv = make_double2(0.0, 0.0), cv = make_double2(0.0, 0.0);
      if (kk > 0) {
        bv = cmul(AL[kk - 1], cconj(Y64[kk]));
        cv = cmul(AL[kk - 1], cconj(Z64[kk]));
      }
      B64[kk] = bv;
      C64[kk] = cv;
      if constexpr (kFast) Bw[kk] = from_d2<R2>(bv);
      bmax2 = fmax(bmax2, cabs2(bv));
    }
    __syncwarp();
    amax2 = gmax<G>(amax2);
    bmax2 = gmax<G>(bmax2);

    // ---- final polynomial F_p, p = 0..3H-1, in the working precision:
    //      [psi^p] (2 MM' d(YM') - YM' d(MM')) = sum_{j+l=p+1} (2l - j) m_j y_l
    R2 Fl[C::NFL];
    R fmax2 = R(0);
#pragma unroll
    for (int i = 0; i < C::NFL; ++i) {
      const int p = gl + G * i;
      R2 acc = mk<R2>(0, 0);
      if (p < C::NF) {
        const int jlo = p + 1 - 2 * H > 0 ? p + 1 - 2 * H : 0;
        const int jhi = p + 1 < 4 * H ? p + 1 : 4 * H;
        for (int j = jlo; j <= jhi; ++j) {
          const int l = p + 1 - j;
          if (l == H) continue;
          const R2 mj = (j >= 2 * H) ? Aw[j - 2 * H] : cconj(Aw[2 * H - j]);
          const R2 yl = (l > H) ? Bw[l - H] : cconj(Bw[H - l]);
          acc = cfma(cscale(mj, (R)(2 * l - j)), yl, acc);
        }
        if (p == C::NF - 1) acc.x = R(0);  // F_{D/2} = -conj(F_{D/2}) is imaginary
      }
      Fl[i] = acc;
      fmax2 = fmax(fmax2, cabs2(acc));
    }
    fmax2 = gmax<G>(fmax2);
    // P independent of theta2 (or YM == 0): no roots to find.
    const bool constant = !valid || !(bmax2 > 0.0) ||
                          !((double)fmax2 > const_rel * const_rel * (double)(H * H) * amax2 * bmax2);
    const R fscale = constant ? R(0) : R(1) / sqrt(fmax2);
#pragma unroll
    for (int i = 0; i < C::NFL; ++i) {
      const int p = gl + G * i;
      if (p < C::NF) {
        const R2 f = cscale(Fl[i], fscale);
        Fs[p] = f;
        if (p < C::NF - 1) Fs[D - p] = mk<R2>(-f.x, f.y);
      }
    }

    // ---- (c) Aberth-Ehrlich on F (degree D), roots i = r*G + gl
    R2 z[RR];
    bool conv[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const int i = r * G + gl;
      R sn, cs;
      const R ang = kTwoPi * (R)i / (R)D + R(0.4);
      if constexpr (kFast) {
        __sincosf(ang, &sn, &cs);
      } else {
        sincos(ang, &sn, &cs);
      }
      const R rad = (i & 1) ? R(0.5) : R(2);
      z[r] = mk<R2>(rad * cs, rad * sn);
      conv[r] = (i >= D) || constant;
      if (i < D) Zs[i] = z[r];
    }
    __syncwarp();
    int iters = 0;
#pragma unroll 1
    for (; iters < a.maxit; ++iters) {
      bool lane_done = true;
#pragma unroll
      for (int r = 0; r < RR; ++r) lane_done = lane_done && conv[r];
      if (__all_sync(0xffffffffu, lane_done)) break;
      R2 uu[RR], p[RR], dp[RR], S[RR];
      bool outside[RR];
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const R m2 = cabs2(z[r]);
        outside[r] = m2 > R(1);
        const R inv = outside[r] ? fast_rcp(m2) : R(1);
        uu[r] = mk<R2>(z[r].x * inv, z[r].y * inv);  // 1/conj(z) outside the unit disc
        p[r] = mk<R2>(0, 0);
        dp[r] = mk<R2>(0, 0);
        S[r] = mk<R2>(0, 0);
      }
#pragma unroll 2
      for (int c = D; c >= 0; --c) {
        const R2 f = Fs[c];
#pragma unroll
        for (int r = 0; r < RR; ++r) {
          dp[r] = cfma(dp[r], uu[r], p[r]);
          p[r] = cfma(p[r], uu[r], f);
        }
      }
#pragma unroll 2
      for (int j = 0; j < D; ++j) {
        const R2 zj = Zs[j];
#pragma unroll
        for (int r = 0; r < RR; ++r) {
          const R2 d = csub(z[r], zj);
          const R inv = (j == r * G + gl) ? R(0) : fast_rcp(cabs2(d));
          S[r].x = fma(d.x, inv, S[r].x);
          S[r].y = fma(-d.y, inv, S[r].y);
        }
      }
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        // Newton ratio p/p'.  Outside the disc use the anti-self-inversive
        // identity p(z) = -z^D conj(p(u)), u = 1/conj(z):
        //   p/p' = z / (D - conj(p'(u)/p(u)) / z).
        R2 N;
        if (outside[r]) {
          const R2 q = cconj(cdiv(dp[r], p[r]));
          N = cdiv(z[r], csub(mk<R2>((R)D, 0), cdiv(q, z[r])));
        } else {
          N = cdiv(p[r], dp[r]);
        }
        R2 w = cdiv(N, csub(mk<R2>(1, 0), cmul(N, S[r])));
        if (!finite2(w)) w = mk<R2>(0, 0);
        if (!conv[r]) {
          const R zz = cabs2(z[r]);
          conv[r] = cabs2(w) <= tol * tol * (zz > R(1) ? zz : R(1));
          z[r] = csub(z[r], w);
        }
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < RR; ++r)
        if (r * G + gl < D) Zs[r * G + gl] = z[r];
      __syncwarp();
    }
    bool lane_nc = false;
#pragma unroll
    for (int r = 0; r < RR; ++r) lane_nc = lane_nc || !conv[r];
    const bool nonconv = gor<G>(lane_nc) && !constant;

    // ---- candidates: P at every root scaled onto |psi| = 1 (working precision)
    R sc[RR], th[RR];
    R2 ps[RR];
    bool pos[RR];
    R lmax = R(-1);
    const R a0w = Aw[0].x;
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const int i = r * G + gl;
      sc[r] = R(-1);
      th[r] = R(0);
      pos[r] = false;
      ps[r] = mk<R2>(1, 0);
      bool have = false;
      if (constant) {
        have = (i == 0);
      } else if (i < D) {
        const R m2 = cabs2(z[r]);
        have = m2 > R(0) && isfinite(m2);
        const R inv = have ? R(1) / sqrt(m2) : R(0);
        ps[r] = mk<R2>(z[r].x * inv, z[r].y * inv);
      }
      if (have) {
        const R mm = trig_eval(Aw, 2 * H, ps[r], a0w);
        const R ym = trig_eval(Bw, H, ps[r], R(0));
        sc[r] = (mm > R(1e-9) * a0w) ? ym * ym / mm : R(0);
        pos[r] = ym > R(0);
        R t2 = atan2(ps[r].y, ps[r].x);
        if (t2 < R(0)) t2 += kTwoPi;
        th[r] = t2;
        lmax = fmax(lmax, sc[r]);
      }
    }
    const R pmax = gmax<G>(lmax);
    const R thr = pmax - tie * (pmax > R(0) ? pmax : R(0));
    // among candidates within the tie band: theta1 > 0 first, then smallest
    // theta2; the winner's psi travels with its key
    R bkey = R(1e30);
    R2 bpsi = mk<R2>(1, 0);
#pragma unroll
    for (int r = 0; r < RR; ++r)
      if (sc[r] >= thr && sc[r] >= R(0)) {
        const R key = (pos[r] ? R(0) : R(16)) + th[r];
        if (key < bkey) {
          bkey = key;
          bpsi = ps[r];
        }
      }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const R ok = __shfl_xor_sync(0xffffffffu, bkey, o, G);
      const R ox = __shfl_xor_sync(0xffffffffu, bpsi.x, o, G);
      const R oy = __shfl_xor_sync(0xffffffffu, bpsi.y, o, G);
      if (ok < bkey || (ok == bkey && (lane ^ o) < lane)) {
        bkey = ok;
        bpsi = mk<R2>(ox, oy);
      }
    }
    double theta = (bkey < R(1e29)) ? (double)(bkey >= R(16) ? bkey - R(16) : bkey) : 0.0;
    double2 psi = make_double2((double)bpsi.x, (double)bpsi.y);
    {  // one Newton step onto |psi| = 1 in FP64
      const double s = 1.5 - 0.5 * cabs2(psi);
      psi = make_double2(psi.x * s, psi.y * s);
    }

    // ---- FP64 Newton polish of the phase on g(theta) = 2 MM YM' - YM MM'
    //      (theta-derivatives), the sums split over the group's lanes.  Every
    //      lane of the warp runs the shuffles (groups differ in `constant`);
    //      only the update is conditional.
    {
#pragma unroll 1
      for (int s = 0; s < a.polish_steps; ++s) {
        const double2 pw0 = group_powers<G>(psi, gl);  // psi^(gl+1)
        const double2 stp = make_double2(__shfl_sync(0xffffffffu, pw0.x, G - 1, G),
                                         __shfl_sync(0xffffffffu, pw0.y, G - 1, G));  // psi^G
        double ma0 = 0, ma1 = 0, ma2 = 0, mb0 = 0, mb1 = 0, mb2 = 0;
        double2 pw = pw0;
        for (int e = gl + 1; e <= 2 * H; e += G) {
          const double2 t = cmul(A64[e], pw);
          ma0 += t.x;
          ma1 = fma((double)e, t.y, ma1);
          ma2 = fma((double)(e * e), t.x, ma2);
          pw = cmul(pw, stp);
        }
        pw = pw0;
        for (int e = gl + 1; e <= H; e += G) {
          const double2 t = cmul(B64[e], pw);
          mb0 += t.x;
          mb1 = fma((double)e, t.y, mb1);
          mb2 = fma((double)(e * e), t.x, mb2);
          pw = cmul(pw, stp);
        }
        ma0 = gsum<G>(ma0);
        ma1 = gsum<G>(ma1);
        ma2 = gsum<G>(ma2);
        mb0 = gsum<G>(mb0);
        mb1 = gsum<G>(mb1);
        mb2 = gsum<G>(mb2);
        const double MM = A64[0].x + 2.0 * ma0, MMt = -2.0 * ma1, MMtt = -2.0 * ma2;
        const double YM = 2.0 * mb0, YMt = -2.0 * mb1, YMtt = -2.0 * mb2;
        const double g = 2.0 * MM * YMt - YM * MMt;
        const double gt = MMt * YMt + 2.0 * MM * YMtt - YM * MMtt;
        const double dl = g / gt;
        if (!constant && isfinite(dl) && fabs(dl) < 1e-3) {
          // psi <- psi e^{-i dl} (Taylor series, |dl| < 1e-3: error < 1e-18)
          const double d2 = dl * dl;
          const double cs = 1.0 - d2 * (0.5 - d2 * (1.0 / 24.0));
          const double sn = dl * (1.0 - d2 * (1.0 / 6.0 - d2 * (1.0 / 120.0)));
          psi = make_double2(psi.x * cs + psi.y * sn, psi.y * cs - psi.x * sn);
          theta -= dl;
        }
      }
    }
    // ---- FP64 evaluation at the chosen phase: MM, YM, Mbar
    double MM, YM, Mbar;
    {
      const double2 pw0 = group_powers<G>(psi, gl);
      const double2 stp = make_double2(__shfl_sync(0xffffffffu, pw0.x, G - 1, G),
                                       __shfl_sync(0xffffffffu, pw0.y, G - 1, G));
      double sa = 0, sb = 0, sc2 = 0;
      double2 pw = pw0;
      for (int e = gl + 1; e <= 2 * H; e += G) {
        sa += A64[e].x * pw.x - A64[e].y * pw.y;
        if (e <= H) {
          sb += B64[e].x * pw.x - B64[e].y * pw.y;
          sc2 += C64[e].x * pw.x - C64[e].y * pw.y;
        }
        pw = cmul(pw, stp);
      }
      MM = A64[0].x + 2.0 * gsum<G>(sa);
      YM = 2.0 * gsum<G>(sb);
      Mbar = 2.0 * gsum<G>(sc2);
    }
    if constexpr (!kFast) theta = atan2(psi.y, psi.x);
    const bool degenerate = !(MM > 1e-14 * (MM + Mbar * Mbar));
    double P = 0.0, th1 = 0.0;
    if (!degenerate) {
      th1 = YM / MM;
      P = YM * th1 / YY;
    }
    const double th3 = ybar - th1 * Mbar;
    theta = fmod(theta, kTwoPiD);
    if (theta < 0.0) theta += kTwoPiD;

    // ---- a-posteriori error of P from the NFFT sums: |dZ| <= e gives
    //      |dMM| <= 9 e (sum|alpha|)^2 and |dYM| <= 2 e sum|alpha| sqrt(YY);
    //      items whose P could be off by more than the threshold are
    //      re-solved from direct FP64 sums.
    bool redo = false;
    if (a.redo_list && valid) {
      if (degenerate) {
        redo = true;
      } else {
        const double dMM = 9.0 * a.sum_err * sum_abs_alpha * sum_abs_alpha;
        const double dYM = 2.0 * a.sum_err * sum_abs_alpha * sqrt(YY);
        const double err = P * dMM / MM + 2.0 * sqrt(fmax(P, 0.0) / (YY * MM)) * dYM;
        redo = !(err <= a.redo_tol);
      }
    }

    if (valid && gl == 0) {
      const int64_t col = a.kmap ? (int64_t)a.kmap[k] : k;
      const size_t o = (size_t)a.rows[tau] * a.out_stride + col;
      if (!FTP_DCHECK(a.status, col >= 0 && col < a.out_stride, 21, col, a.out_stride) ||
          !FTP_DCHECK(a.status, (int64_t)o < a.out_elems, 22, o, a.out_elems)) {
        // out of range: write nothing (self-checking builds only)
      } else {
      a.power[o] = P;
      a.theta1[o] = th1;
      a.theta2[o] = theta;
      a.theta3[o] = th3;
      if (a.flags) {
        unsigned f = 0;
        if (nonconv) f |= 1u;
        if (degenerate) f |= 2u;
        if (constant) f |= 4u;
        if (th1 < 0.0) f |= 8u;
        a.flags[o] = (uint8_t)f;
      }
      if (redo && FTP_DCHECK(a.status, col < a.redo_cap, 23, col, a.redo_cap) &&
          atomicExch(&a.redo_mark[col], 1) == 0) {
        const int slot = atomicAdd(a.redo_count, 1);
        if (slot < a.redo_cap) a.redo_list[slot] = (int)col;
        ++st_redo;
      }
      }
      st_iters += (unsigned long long)iters;
      st_items += 1;
      st_nonconv += nonconv ? 1 : 0;
    }
    __syncwarp();
    u = un;
    buf ^= 1;
  }
  // one atomic per warp for the solver statistics
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    st_iters += __shfl_xor_sync(0xffffffffu, st_iters, o);
    st_items += __shfl_xor_sync(0xffffffffu, st_items, o);
    st_nonconv += __shfl_xor_sync(0xffffffffu, st_nonconv, o);
    st_redo += __shfl_xor_sync(0xffffffffu, st_redo, o);
  }
  if (lane == 0 && st_items) {
    atomicAdd(&a.counters[CNT_ITERS], st_iters);
    atomicAdd(&a.counters[CNT_ITEMS], st_items);
    atomicAdd(&a.counters[CNT_NONCONV], st_nonconv);
    atomicAdd(&a.counters[CNT_REDO], st_redo);
  }
}

// Host side: opt in to the dynamic shared memory once, size the persistent grid.
template <typename S2, typename R, int H, int G>
int launch_h(const RootsArgs& a, int num_sms, cudaStream_t s) {
  using C = Cfg<S2, R, H, G>;
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    if (cudaFuncSetAttribute(roots_kernel<S2, R, H, G>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C::SMEM) != cudaSuccess)
      return -2;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, roots_kernel<S2, R, H, G>,
                                                      C::WARPS * 32, C::SMEM) != cudaSuccess ||
        b < 1)
      return -2;
    blocks_per_sm = b;
  }
  const int64_t nf = a.nf;  // upper bound when the count lives on the device
  const int64_t nunits = (nf + C::NGW - 1) / C::NGW * a.ntpl;
  int64_t grid = (int64_t)num_sms * blocks_per_sm;
  const int64_t need = (nunits + C::WARPS - 1) / C::WARPS;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  roots_kernel<S2, R, H, G><<<(unsigned)grid, C::WARPS * 32, C::SMEM, s>>>(a);
  return 1;
}

}  // namespace roots
}  // namespace ftp
