// Steps (b) and (c) of the Fast Template Periodogram in two kernels over the
// same work units: polynomial assembly (Section 2: MM_nm, YM_k, Eq.
// finalpoly), all zeros of the final polynomial by Aberth-Ehrlich iteration
// from Newton-polygon initial guesses, candidates scaled onto the unit circle
// (Section 2, end) and the best one chosen (first kernel); then the chosen
// phase polished by a Newton step and (theta1, theta2, theta3, P) evaluated
// at it in FP64-class arithmetic (second kernel).
//
// Work item = (frequency k, template tau).  A group of G lanes owns one item:
// it assembles the coefficients, then each lane iterates R = ceil(D/G) of the
// D = 6H-2 roots, fewer once most have converged (compaction).  Each warp
// takes work units (32/G consecutive frequencies of one template) from a
// global queue and stages their sum tiles (3H rows in the [3H][nf_pad]
// layout) into its own shared memory with TMA bulk copies, double-buffered so
// the next unit's copy overlaps this unit's arithmetic.  Warps never wait for
// each other.
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
// With c_n = alpha_n conj(Z_n) the MM' coefficients reduce to
//   a_e = conj(Z_e) K_e - ( sum_{n+m=e} c_n c_m + 2 sum_{n-m=e} c_n conj(c_m) ),
//   K_e = sum_{n+m=e} alpha_n alpha_m + 2 sum_{n-m=e} alpha_n conj(alpha_m),
// where K_e depends on the template only: one complex product per pair term.
// The final polynomial F = 2 MM' d(YM') - YM' d(MM') is anti-self-inversive,
// F_{D-p} = -conj(F_p), so only p = 0..3H-1 are formed and the rest mirrored.
//
// Precision.  a_e, b_k, c_n are assembled, and the chosen phase is polished
// and evaluated, in an FP64-class type W: native FP64 on the FP64 path and for
// FP64 sums, float-float (ftp_wide.cuh) on the mixed path.  F, the Aberth
// iteration and the candidate screening run in the kernel's working precision
// R (float for the mixed path, double for the FP64 path).  The sum tiles are
// float2 (mixed, from the FP32 NFFT) or double2 (FP64 NFFT, or direct FP64
// sums of the re-solve pass).
#pragma once

#include <math.h>

#include <type_traits>

#include "ftp_internal.cuh"
#include "ftp_wide.cuh"

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
  // Rounding-level acceptance of stalled roots during the iterations (from
  // the 12th, every 4th): every kernel except the mixed path's main one (FP32
  // sums and iterations), whose hot loop stays as it is; that kernel checks
  // its items only once they hit the cap.
  static constexpr bool kAccept = !kFast || sizeof(S2) == 16;
  // FP64-class steps: float-float on the mixed path (FP32 sums and Aberth),
  // native FP64 on the FP64 path and the re-solve pass (FP64 sums)
  static constexpr bool kDD = kFast && sizeof(S2) == 8;
  // Off-circle roots settle early (aberth_step) in that same main mixed
  // kernel only, and at H >= 8: the FP64 path and the re-solve passes iterate
  // every root to the tolerance, and below H = 8 the test costs about what
  // the iterations it saves do (measured at H = 2, 4, 6).
  static constexpr bool kSettle = kDD && H >= 8;
  using W = std::conditional_t<kDD, wide::dd, double>;
  using WC = typename wide::CT<W>::type;
  static constexpr int D = 6 * H - 2;
  static constexpr int RR = cdiv_i(D, G);         // roots per lane
  static constexpr int NGW = 32 / G;              // items per warp unit
  static constexpr int WARPS = 4;                 // warps per CTA
  static constexpr int ROWS = 3 * H;              // staged sum rows
  static constexpr int CROWS = 4 * H + 1;         // staged coefficient rows (coef_mode)
  static constexpr int NA = 2 * H + 1;            // a_0..a_2H, Z_0..Z_2H
  static constexpr int NB = H + 1;                // b_0..b_H, c_0..c_H, Y_0..Y_H
  static constexpr int NF = 3 * H;                // F_0..F_{3H-1}
  static constexpr int NFL = cdiv_i(NF, G);
  static constexpr int NSLOT = H + 1;             // assembly slots {0}, {e, 2H+1-e}
  // per-group shared memory (bytes); WC elements are 16 bytes either way
  static_assert(sizeof(WC) == 16, "wide complex layout");
  static constexpr size_t G_Z64 = 0;
  static constexpr size_t G_Y64 = G_Z64 + NA * 16;
  static constexpr size_t G_A64 = G_Y64 + NB * 16;
  static constexpr size_t G_B64 = G_A64 + NA * 16;
  static constexpr size_t G_C64 = G_B64 + NB * 16;
  static constexpr size_t G_F = G_C64 + NB * 16;
  static constexpr size_t G_Z = G_F + rup((D + 1) * sizeof(R2), 16);
  static constexpr size_t G_AW = G_Z + rup(RR * G * sizeof(R2), 16);
  static constexpr size_t G_BW = G_AW + rup(NA * sizeof(R2), 16);
  static constexpr size_t G_END = G_BW + rup(NB * sizeof(R2), 16);
  // An odd number of 16-byte words per group: the NGW (<= 8) groups of a warp
  // then start in distinct 16-byte bank slots, so the per-group broadcasts of
  // the Aberth loops (F_c, z_j) and of the assembly are free of bank conflicts.
  static constexpr size_t GROUP_BYTES = rup(G_END, 16) + ((rup(G_END, 16) / 16) % 2 == 0 ? 16 : 0);
  // per-warp shared memory
  static constexpr size_t ROW_BYTES = NGW * sizeof(S2);
  static constexpr size_t STAGE_BYTES = (ROWS > CROWS ? ROWS : CROWS) * ROW_BYTES;
  static constexpr size_t W_STAGE = 0;                                   // 2 buffers
  static constexpr size_t W_MBAR = rup(2 * STAGE_BYTES, 16);             // 2 mbarriers
  static constexpr size_t W_KE = W_MBAR + 16;                            // K_e, e = 0..2H
  static constexpr size_t W_AL = W_KE + NA * 16;                         // alpha_n
  static constexpr size_t W_KER = W_AL + H * 16;                         // K_e, working precision
  static constexpr size_t W_ALR = W_KER + rup(NA * sizeof(R2), 16);      // alpha_n, working precision
  static constexpr size_t W_GROUPS = rup(W_ALR + rup(H * sizeof(R2), 16), 128);
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
// one MUFU reciprocal (flush-to-zero approximation); the iteration corrects it
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }
// 2^x: one MUFU instruction (initial guesses only)
__device__ __forceinline__ float fast_exp2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// 1/sqrt(x): one MUFU instruction in FP32 (candidate phases only need a few ulp)
__device__ __forceinline__ float fast_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt(x); }
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
// Bounded wait: gives up after `polls` polls instead of spinning forever if
// a copy never lands.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int polls) {
  for (int i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ------------------------------------------------------------ packed FP32
// Pairs of FP32 values in one 64-bit register pair, operated on by the
// f32x2 instructions of sm_100-class GPUs: one instruction does the work of
// two FP32 ones, and each element is rounded exactly as the scalar
// instruction would round it.
using f2p = unsigned long long;
__device__ __forceinline__ f2p pk2(float lo, float hi) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(f2p v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
  f2p d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
  f2p d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// A root whose correction has stalled is accepted when F's value there is
// at the rounding level of its evaluation: |F(z)| <= 8 D eps
// sum_k |F_k| |z|^k (a backward error of a few units of the working
// precision in the coefficients), so that no further digits are obtainable in
// that precision - the case of clustered and multiple roots, whose Newton
// corrections stall at about sqrt(eps) instead of meeting the tolerance.
// Outside the unit disc F is evaluated at u = 1/conj(z): F is
// anti-self-inversive, so |F(z)| = |z|^D |F(u)| and the sum of |F_k||z|^k
// scales alike.  Out of line: it runs only for roots still unconverged after
// many iterations, and the hot loops keep their registers.
template <int D, typename R, typename R2>
__device__ __noinline__ bool pseudo_zero(R2 z, const R2* Fs) {
  const R m2 = cabs2(z);
  const R inv = m2 > R(1) ? R(1) / m2 : R(1);
  const R2 u = mk<R2>(z.x * inv, z.y * inv);
  const R au = sqrt(cabs2(u));
  R2 p = mk<R2>(0, 0);
  R pa = R(0);
#pragma unroll 1
  for (int c = D; c >= 0; --c) {
    const R2 f = Fs[c];
    p = cfma(p, u, f);
    pa = fma(pa, au, sqrt(cabs2(f)));
  }
  const R eps = sizeof(R) == 4 ? R(5.9604645e-8) : R(1.1102230246251565e-16);
  const R bound = R(8 * D) * eps * pa;
  return isfinite(pa) && cabs2(p) <= bound * bound;
}

// ------------------------------------------------------------ Aberth step
// Only the zeros of F on the unit circle are stationary points of P (Section
// 2, end); the others come in pairs z, 1/conj(z) and serve the candidate
// list only through their projections onto the circle, which cannot beat the
// best stationary value.  So a root may stop iterating (be "settled") before
// it meets the tolerance once it is known to lie off the circle: its
// correction w is
//   - small:            |w| < kSettleStep max(1, |z|),
//   - a Newton step:    the repulsion term of the Aberth denominator is at
//                       most kSettleDom of the Newton term (|p S| <= 0.1
//                       |p'|), so w ~ p/p' and the root is within ~|w| of z
//                       (and no other approximation lies within ~10 |w| of z,
//                       whose 1/(z - z_j) would dominate S),
//   - far from the circle: | |z| - 1 | > kSettleDist |w| + kSettleGap.
// The settled root keeps its position in the pair sums of the others, which
// still converge to the tolerance (the fixed points of the iteration are the
// zeros of F whatever the other approximations are).
constexpr float kSettleStep = 1e-2f, kSettleDom = 0.1f, kSettleDist = 50.0f,
                kSettleGap = 1e-3f;
// Candidate roots: | |z|^2 - 1 | below this (|z| within about 0.05 of 1).
constexpr float kNearCircle = 0.1f;

// One Aberth-Ehrlich iteration for the NS root slots of a lane.  Slot r holds
// root idx[r] of the item (idx < 0: an empty slot, marked converged), z[r] its
// position; Fs holds F's D + 1 coefficients and Zs the positions of all D
// roots of the item (read for the pair sums, written back at the end).
// kSettle: roots known to lie off the unit circle stop early (above) and are
// marked in settled[] (one byte per root of the item).
template <int NS, int D, bool kFast, bool kSettle, typename R, typename R2>
__device__ __forceinline__ void aberth_step(R2 (&z)[NS], bool (&conv)[NS], const int (&idx)[NS],
                                            const R2* Fs, R2* Zs, R tol,
                                            unsigned char* settled) {
  // unroll factors of the Horner and pair loops (measured per H on the
  // long lightcurve): 4 for Horner, 5 where D + 1 is a multiple of 5 (H = 6,
  // 11); 2 for the pair loop at five or more slots per lane or low degree,
  // where 4 costs registers and scheduling, else 4
  constexpr int kUH = (D + 1) % 5 == 0 && D <= 64 ? 5 : 4;
  constexpr int kUP = NS >= 5 || D < 16 ? 2 : 4;
  R2 uu[NS], p[NS], dp[NS], S[NS];
  bool outside[NS];
#pragma unroll
  for (int r = 0; r < NS; ++r) {
    const R m2 = cabs2(z[r]);
    outside[r] = m2 > R(1);
    const R inv = outside[r] ? fast_rcp(m2) : R(1);
    uu[r] = mk<R2>(z[r].x * inv, z[r].y * inv);  // 1/conj(z) outside the unit disc
    p[r] = mk<R2>(0, 0);
    dp[r] = mk<R2>(0, 0);
    S[r] = mk<R2>(0, 0);
  }
  if constexpr (kFast && NS >= 2) {
    // FP32: slots 2q and 2q+1 travel as packed pairs (real parts in one,
    // imaginary parts in the other), the same FMAs in the same order as
    // the scalar loops below, in half the instructions
    constexpr int NP = NS / 2;
    f2p UX[NP], UY[NP], UYn[NP], PX[NP], PY[NP], DX[NP], DY[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      UX[q] = pk2(uu[2 * q].x, uu[2 * q + 1].x);
      UY[q] = pk2(uu[2 * q].y, uu[2 * q + 1].y);
      UYn[q] = pk2(-uu[2 * q].y, -uu[2 * q + 1].y);
      PX[q] = PY[q] = DX[q] = DY[q] = 0ull;
    }
#pragma unroll (kUH)
    for (int c = D; c >= 0; --c) {
      const R2 f = Fs[c];
      const f2p FX = pk2(f.x, f.x), FY = pk2(f.y, f.y);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        // dp = dp u + p, then p = p u + f (complex)
        const f2p ndx = fma2(DX[q], UX[q], fma2(DY[q], UYn[q], PX[q]));
        const f2p ndy = fma2(DX[q], UY[q], fma2(DY[q], UX[q], PY[q]));
        const f2p npx = fma2(PX[q], UX[q], fma2(PY[q], UYn[q], FX));
        const f2p npy = fma2(PX[q], UY[q], fma2(PY[q], UX[q], FY));
        DX[q] = ndx;
        DY[q] = ndy;
        PX[q] = npx;
        PY[q] = npy;
      }
      if constexpr (NS % 2 != 0) {
        dp[NS - 1] = cfma(dp[NS - 1], uu[NS - 1], p[NS - 1]);
        p[NS - 1] = cfma(p[NS - 1], uu[NS - 1], f);
      }
    }
    f2p ZX[NP], ZY[NP], SX[NP], SYn[NP];  // SYn accumulates -Im S
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      ZX[q] = pk2(z[2 * q].x, z[2 * q + 1].x);
      ZY[q] = pk2(z[2 * q].y, z[2 * q + 1].y);
      SX[q] = SYn[q] = 0ull;
    }
    const f2p tiny2 = pk2(1e-30f, 1e-30f);
#pragma unroll (kUP)
    for (int j = 0; j < D; ++j) {
      const R2 zj = Zs[j];
      const f2p JX = pk2(zj.x, zj.x), JY = pk2(zj.y, zj.y);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const f2p dx = sub2(ZX[q], JX), dy = sub2(ZY[q], JY);
        float ma, mb;
        upk2(fma2(dx, dx, fma2(dy, dy, tiny2)), ma, mb);
        const f2p inv = pk2(fast_rcp(ma), fast_rcp(mb));
        SX[q] = fma2(dx, inv, SX[q]);
        SYn[q] = fma2(dy, inv, SYn[q]);
      }
      if constexpr (NS % 2 != 0) {
        const R2 d = csub(z[NS - 1], zj);
        const R inv = fast_rcp(fma(d.x, d.x, fma(d.y, d.y, R(1e-30))));
        S[NS - 1].x = fma(d.x, inv, S[NS - 1].x);
        S[NS - 1].y = fma(-d.y, inv, S[NS - 1].y);
      }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      upk2(PX[q], p[2 * q].x, p[2 * q + 1].x);
      upk2(PY[q], p[2 * q].y, p[2 * q + 1].y);
      upk2(DX[q], dp[2 * q].x, dp[2 * q + 1].x);
      upk2(DY[q], dp[2 * q].y, dp[2 * q + 1].y);
      upk2(SX[q], S[2 * q].x, S[2 * q + 1].x);
      float sa, sb;
      upk2(SYn[q], sa, sb);
      S[2 * q].y = -sa;
      S[2 * q + 1].y = -sb;
    }
  } else {
#pragma unroll 2
  for (int c = D; c >= 0; --c) {
    const R2 f = Fs[c];
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      dp[r] = cfma(dp[r], uu[r], p[r]);
      p[r] = cfma(p[r], uu[r], f);
    }
  }
  // sum_{j != i} 1/(z_i - z_j): the j = i term has d = 0 and contributes
  // conj(0) / (0 + tiny) = 0, so no branch is needed
#pragma unroll 2
  for (int j = 0; j < D; ++j) {
    const R2 zj = Zs[j];
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      const R2 d = csub(z[r], zj);
      const R inv = fast_rcp(fma(d.x, d.x, fma(d.y, d.y, kFast ? R(1e-30) : R(1e-300))));
      S[r].x = fma(d.x, inv, S[r].x);
      S[r].y = fma(-d.y, inv, S[r].y);
    }
  }
  }
#pragma unroll
  for (int r = 0; r < NS; ++r) {
    // Aberth correction w = N / (1 - N S) = 1 / (p'/p - S), N = p/p' the
    // Newton ratio, formed as one quotient.  Outside the disc the
    // anti-self-inversive identity p(z) = -z^D conj(p(u)), u = 1/conj(z),
    // gives p'/p = (D z - conj(p'(u)/p(u))) / z^2:
    //   inside:  w = p / (p' - p S);
    //   outside: w = z^2 / (D z - conj(p'(u)/p(u)) - S z^2).
    // den = newt - rep: the Newton term (z^2 p'/p outside, p' inside) and
    // the repulsion term of the other roots (S z^2 outside, p S inside)
    R2 num, den, newt, rep;
    if (outside[r]) {
      const R2 q = cconj(cdiv(dp[r], p[r]));
      const R2 z2 = cmul(z[r], z[r]);
      num = z2;
      if constexpr (kSettle) {
        newt = csub(mk<R2>(R(D) * z[r].x, R(D) * z[r].y), q);
        rep = cmul(S[r], z2);
        den = csub(newt, rep);
      } else {
        den = csub(csub(mk<R2>(R(D) * z[r].x, R(D) * z[r].y), q), cmul(S[r], z2));
      }
    } else {
      num = p[r];
      if constexpr (kSettle) {
        newt = dp[r];
        rep = cmul(p[r], S[r]);
        den = csub(newt, rep);
      } else {
        den = csub(dp[r], cmul(p[r], S[r]));
      }
    }
    R2 w = cdiv(num, den);
    if (!finite2(w)) w = mk<R2>(0, 0);
    if (!conv[r]) {
      const R zz = cabs2(z[r]);
      if constexpr (kSettle) {
        const R sc = zz > R(1) ? zz : R(1);
        const R w2 = cabs2(w);
        bool done = w2 <= tol * tol * sc;
        if (!done && w2 < R(kSettleStep * kSettleStep) * sc &&
            cabs2(rep) <= R(kSettleDom * kSettleDom) * cabs2(newt)) {
          const R az = zz * fast_rsqrt(zz), aw = w2 * fast_rsqrt(w2);  // w2 > 0 here
          done = fabs(az - R(1)) > R(kSettleDist) * aw + R(kSettleGap);
          if (done) settled[idx[r]] = 1;
        }
        conv[r] = done;
      } else {
        conv[r] = cabs2(w) <= tol * tol * (zz > R(1) ? zz : R(1));
      }
      z[r] = csub(z[r], w);
    }
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < NS; ++r)
    if (idx[r] >= 0) Zs[idx[r]] = z[r];
  __syncwarp();
}

// Iterations over NS slots per lane until every root converged (false) or,
// if NT < NS, until every group of the warp has at most NT * G unconverged
// roots (true: time to compact).
template <int G, int NS, int NT, int D, bool kAccept, bool kSettle, typename R, typename R2>
__device__ __forceinline__ bool aberth_run(R2 (&z)[NS], bool (&conv)[NS], const int (&idx)[NS],
                                           const R2* Fs, R2* Zs, R tol, int& iters, int maxit,
                                           unsigned char* settled) {
#pragma unroll 1
  for (; iters < maxit; ++iters) {
    if constexpr (kAccept) {
      // from the 12th iteration on, every 4th, a root that is a zero of F to
      // the working precision is accepted - the corrections of clustered and
      // multiple roots stall near sqrt(eps) and would otherwise run to the
      // cap (well-separated roots converge in ~11)
      if (iters >= 12 && (iters & 3) == 0) {
#pragma unroll  // static indices keep z and conv in registers
        for (int r = 0; r < NS; ++r)
          if (!conv[r] && idx[r] >= 0 && pseudo_zero<D, R>(z[r], Fs)) conv[r] = true;
      }
    }
    int nact = 0;
#pragma unroll
    for (int r = 0; r < NS; ++r) nact += conv[r] ? 0 : 1;
    if (__all_sync(0xffffffffu, nact == 0)) return false;
    if constexpr (NT < NS) {
      int wmax = 0;
      {
        int v = nact;
#pragma unroll
        for (int sh = G / 2; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh, G);
        wmax = v;
      }
#pragma unroll
      for (int sh = G; sh < 32; sh <<= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, sh));
      if (wmax <= NT * G) return true;
    }
    aberth_step<NS, D, sizeof(R) == 4, kSettle>(z, conv, idx, Fs, Zs, tol, settled);
  }
  return false;
}
// Moves a group's unconverged roots from NS slots per lane into NT slots per
// lane: the roots are listed in `act` (prefix over the lanes' counts), lane
// gl takes list entries gl, gl + G, ...; positions come from Zs.
template <int G, int NS, int NT, typename R2>
__device__ __forceinline__ void compact_roots(const bool (&conv)[NS], const int (&idx)[NS],
                                              short* act, const R2* Zs, int gl, R2 (&z2)[NT],
                                              bool (&c2)[NT], int (&i2)[NT]) {
  int nact = 0;
#pragma unroll
  for (int r = 0; r < NS; ++r) nact += conv[r] ? 0 : 1;
  int incl = nact;
#pragma unroll
  for (int sh = 1; sh < G; sh <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, sh, G);
    if (gl >= sh) incl += t;
  }
  const int gact = __shfl_sync(0xffffffffu, incl, G - 1, G);
  int pos = incl - nact;
  __syncwarp();
#pragma unroll
  for (int r = 0; r < NS; ++r)
    if (!conv[r]) act[pos++] = (short)idx[r];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    const int q = gl + k * G;
    i2[k] = q < gact ? (int)act[q] : -1;
    z2[k] = i2[k] >= 0 ? Zs[i2[k]] : mk<R2>(0, 0);
    c2[k] = i2[k] < 0;
  }
  __syncwarp();
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
template <int G, typename W>
__device__ __forceinline__ typename wide::CT<W>::type group_powers(
    typename wide::CT<W>::type psi, int gl) {
  using namespace wide;
  auto pw = psi;
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    const auto v = mkc(w_shfl_up(re(pw), o, G), w_shfl_up(im(pw), o, G));
    if (gl >= o) pw = c_mul<W>(pw, v);
  }
  return pw;
}
template <int G, typename W> __device__ __forceinline__ W wsum(W v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = wide::w_add(v, wide::w_shfl_xor(v, o, G));
  return v;
}
// Sums of eight wide values over the group, every lane getting all eight:
// a butterfly reduce-scatter (at offset o a lane keeps the half of its
// values picked by bit o of its index and adds the partner's copy of it),
// then a gather of the eight totals.  7 wide additions instead of 8 log2 G.
template <int G, typename W> __device__ __forceinline__ void wsum8(W* v, int gl) {
  constexpr int L = G < 8 ? G : 8;  // lanes that end up with distinct totals
  constexpr int S = 8 / L;          // totals per lane
  W cur[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) cur[i] = v[i];
#pragma unroll
  for (int o = L / 2, n = 4; o >= 1; o >>= 1, n >>= 1) {
    const bool upper = (gl & o) != 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const W keep = upper ? cur[i + n] : cur[i];
      const W send = upper ? cur[i] : cur[i + n];
      cur[i] = wide::w_add(keep, wide::w_shfl_xor(send, o, G));
    }
  }
#pragma unroll
  for (int o = L; o < G; o <<= 1)
#pragma unroll
    for (int i = 0; i < S; ++i) cur[i] = wide::w_add(cur[i], wide::w_shfl_xor(cur[i], o, G));
  // total j sits in slot j % S of lane j / S
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = wide::w_shfl(cur[j % S], j / S, G);
}

// An increasing function of arg(p) on [0, 2 pi) for |p| = 1 (values in [0, 4)):
// orders candidate phases without an arctangent.
template <typename T2>
__device__ __forceinline__ auto pseudo_angle(T2 p) -> decltype(p.x) {
  using T = decltype(p.x);
  const T ax = p.x < T(0) ? -p.x : p.x, ay = p.y < T(0) ? -p.y : p.y;
  const T q = ay * fast_rcp(ax + ay + T(1e-30));  // in [0, 1]
  // quadrants I..IV map to [0,1), [1,2), [2,3), [3,4)
  if (p.y >= T(0)) return p.x >= T(0) ? q : T(2) - q;
  return p.x < T(0) ? T(2) + q : T(4) - q;
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

// The work of one item runs in two kernels over the same work units:
//   PH = 1  assembly, final polynomial, Aberth iterations and candidate
//           choice; it leaves the chosen phase psi and three flag bits in the
//           item's output slots (power <- Re psi, theta1 <- Im psi,
//           theta2 <- bits);
//   PH = 2  assembly again (FP64-class), polish and evaluation at psi, the
//           a-posteriori error and the outputs.
// Each kernel's code is a fraction of the whole, so the warps of an SM, which
// are at different points of their items, share far fewer instructions in the
// instruction caches than one fused kernel would make them fetch.
// Resident CTAs per SM the launch bounds ask for: FP32 kernels 5 (94-96
// registers), the first kernel at H >= 8 six (80 registers; measured at
// H = 10: -2.6 %, at H = 6: +1 %), FP64 kernels 3.
template <typename R, int H, int PH>
constexpr int roots_min_blocks() {
  return sizeof(R) == 4 ? ((PH == 1 && H >= 8) ? 6 : 5) : 3;
}

template <typename S2, typename R, int H, int G, int PH>
__global__ void __launch_bounds__(128, roots_min_blocks<R, H, PH>()) roots_kernel(const RootsArgs a) {
  using namespace wide;
  using C = Cfg<S2, R, H, G>;
  using R2 = typename C::R2;
  using W = typename C::W;
  using WC = typename C::WC;
  constexpr int D = C::D, RR = C::RR, NGW = C::NGW;
  constexpr bool kFast = C::kFast;
  constexpr R kTwoPi = R(6.283185307179586476925286766559);
  constexpr R tol = kFast ? R(2e-6) : R(1e-12);
  constexpr R tie = kFast ? R(1e-6) : R(1e-12);
  // F ~ 0 relative to |a| |b| (rounding level of the working precision)
  constexpr R const_rel = kFast ? R(1e-5) : R(1e-13);

  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wb = smem + (size_t)warp * C::WARP_BYTES;
  S2* stage = reinterpret_cast<S2*>(wb + C::W_STAGE);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(wb + C::W_MBAR);
  WC* KE = reinterpret_cast<WC*>(wb + C::W_KE);
  WC* AL = reinterpret_cast<WC*>(wb + C::W_AL);
  R2* KER = reinterpret_cast<R2*>(wb + C::W_KER);
  R2* ALR = reinterpret_cast<R2*>(wb + C::W_ALR);
  const int gl = lane % G, gi = lane / G;
  unsigned char* gb = wb + C::W_GROUPS + (size_t)gi * C::GROUP_BYTES;
  WC* Z64 = reinterpret_cast<WC*>(gb + C::G_Z64);
  WC* Y64 = reinterpret_cast<WC*>(gb + C::G_Y64);
  WC* A64 = reinterpret_cast<WC*>(gb + C::G_A64);
  WC* B64 = reinterpret_cast<WC*>(gb + C::G_B64);
  WC* C64 = reinterpret_cast<WC*>(gb + C::G_C64);
  R2* Fs = reinterpret_cast<R2*>(gb + C::G_F);
  R2* Zs = reinterpret_cast<R2*>(gb + C::G_Z);
  R2* Aw = reinterpret_cast<R2*>(gb + C::G_AW);  // working-precision copies
  R2* Bw = reinterpret_cast<R2*>(gb + C::G_BW);

  // one work counter per phase; the first kernel clears the second's (the
  // second runs after it on the same stream)
  unsigned long long* const queue = PH == 1 ? a.queue : a.queue + 1;
  if (PH == 1 && blockIdx.x == 0 && threadIdx.x == 0) a.queue[1] = 0ull;
  if (a.status[ST_CODE] != DEV_OK) return;
  // Three ways to number the work units:
  //   one curve      (segs == nullptr): unit = tau * nkb + kb over a.ntpl
  //                  templates, NGW consecutive frequencies per unit;
  //   batched        (segs, no slot_curve): the units of segment s follow
  //                  those of segment s-1 (seg_units), numbered as above
  //                  within the segment;
  //   batched redo   (segs and slot_curve): unit = tau * count + slot, one
  //                  listed frequency per unit (group 0; the others idle).
  const bool batched = a.segs != nullptr;
  const bool redo_pass = batched && a.slot_curve != nullptr;
  const int64_t nf = a.nf_dev ? (int64_t)min(*a.nf_dev, a.redo_cap > 0 ? a.redo_cap : *a.nf_dev)
                              : a.nf;
  const int64_t nkb = (nf + NGW - 1) / NGW;
  const bool listed = batched && !redo_pass && a.unit_list != nullptr;
  const int64_t nunits = redo_pass ? nf * a.ntpl
                         : listed  ? (int64_t)*a.unit_count
                         : batched ? a.seg_units[a.nseg]
                                   : nkb * a.ntpl;
  const double* mom = a.moments;
  W ybar = w_of<W>(mom[MO_YBAR]), YY = w_of<W>(mom[MO_YY]);
  R YYr = (R)mom[MO_YY];
  int cur_curve = 0;
  const W twopi = w_of<W>(6.283185307179586476925286766559);

  if (lane == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_fence_init();
  }
  __syncwarp();

  auto grab = [&]() -> int64_t {
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(queue, 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, v, 0);
  };
  // Segment of unit u (batched main pass): the last s >= lo with
  // seg_units[s] <= u.  Units only grow along a warp's queue, so `lo` is the
  // previous answer and the first probe usually settles it.
  auto find_seg = [&](int64_t u, int lo) -> int {
    if (u < a.seg_units[lo]) lo = 0;  // listed units need not ascend
    if (u < a.seg_units[lo + 1]) return lo;
    int hi = a.nseg;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.seg_units[mid] <= u) lo = mid;
      else hi = mid;
    }
    return lo;
  };
  struct URef {
    int seg;         // segment (-1: none), 0 for one curve
    int tl;          // template within the segment / launch
    int64_t kfirst;  // first frequency (slot in the redo pass) of the unit
  };
  auto resolve = [&](int64_t u, int hint) -> URef {
    URef r;
    if (!batched) {
      r.seg = 0;
      r.tl = (int)(u / nkb);
      r.kfirst = (u % nkb) * NGW;
    } else if (!redo_pass) {
      if (listed) u = a.unit_list[u];
      r.seg = find_seg(u, hint);
      const int64_t local = u - a.seg_units[r.seg];
      const int64_t nkb_s = (a.segs[r.seg].nf + NGW - 1) / NGW;
      r.tl = (int)(local / nkb_s);
      r.kfirst = (local % nkb_s) * NGW;
    } else {
      r.kfirst = u % nf;
      r.tl = (int)(u / nf);
      const int c = a.slot_curve[r.kfirst];
      r.seg = (c >= 0 && c < a.ncurves) ? a.curve_seg[c] : -1;
    }
    return r;
  };
  // The warp stages the sum rows of unit r into buffer `buf`: lane 0 arms the
  // mbarrier with the unit's byte count, then the lanes issue one row copy
  // each (one lane issuing all 3H copies was a sixth of the second kernel's
  // time).  Called by the whole warp.
  auto issue = [&](const URef& r, int buf) {
    int64_t base = r.kfirst, stride = a.nf_pad;
    int Hs = a.Hs;
    if (batched && r.seg >= 0) {
      Hs = a.segs[r.seg].Hs;
      if (!redo_pass) {
        base += a.segs[r.seg].sums_off;
        stride = a.segs[r.seg].nf_pad;
      }
    }
    S2* dst = stage + (size_t)buf * (C::STAGE_BYTES / sizeof(S2));
    const int nrows = a.coef_mode ? C::CROWS : C::ROWS;
    if (lane == 0) mbar_expect_tx(&mbar[buf], (unsigned)(nrows * C::ROW_BYTES));
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const S2* sums = reinterpret_cast<const S2*>(a.sums);
#pragma unroll 1
    for (int r2 = lane; r2 < nrows; r2 += 32) {
      const int src_row = a.coef_mode ? r2 : (r2 < 2 * H) ? r2 : 2 * Hs + (r2 - 2 * H);
      const int64_t off = (int64_t)src_row * stride + base;
      if (a.skip_copies) continue;  // fault injection: the row never lands
      if (!FTP_DCHECK(a.status, off >= 0 && off + NGW <= a.sums_elems, 11, off, a.sums_elems) ||
          !FTP_DCHECK(a.status, (gaddr(sums + off) & 15) == 0, 12, gaddr(sums + off) & 15, 16) ||
          !FTP_DCHECK(a.status, (saddr(dst + (size_t)r2 * NGW) & 15) == 0, 13, 0, 16)) {
        continue;  // the row never lands: the bounded wait reports a timeout
      }
      bulk_g2s(dst + (size_t)r2 * NGW, sums + off, (unsigned)C::ROW_BYTES, &mbar[buf]);
    }
  };

  unsigned long long st_iters = 0;
  unsigned st_items = 0, st_nonconv = 0, st_redo = 0, st_redo_nc = 0, st_final = 0;
  const int polls = a.wait_polls;  // resolved by the host (kWaitPolls by default)
  unsigned parity[2] = {0u, 0u};
  int buf = 0, cur_tau = -1;
  R sum_abs_alpha = R(0);
  int64_t u = grab();
  int seg_hint = 0;
  if (u < nunits) {
    const URef r0 = resolve(u, 0);
    seg_hint = batched && !redo_pass ? r0.seg : 0;
    issue(r0, 0);
  }
  while (u < nunits) {
    const URef cu = resolve(u, seg_hint);
    const int64_t un = grab();
    if (un < nunits) {
      const URef rn = resolve(un, batched && !redo_pass ? cu.seg : 0);
      issue(rn, buf ^ 1);
    }
    if (batched && !redo_pass) seg_hint = cu.seg;
    // template (index into alpha) and validity of this unit
    int tau = cu.tl;
    bool unit_ok = true;
    int64_t seg_nf = nf;
    if (batched) {
      if (cu.seg < 0) {
        unit_ok = false;
        tau = cur_tau < 0 ? 0 : cur_tau;
      } else {
        const RootsSeg& sg = a.segs[cu.seg];
        unit_ok = cu.tl < sg.ntpl;
        tau = sg.tpl_first + (unit_ok ? cu.tl : 0);
        seg_nf = sg.nf;
        if (sg.curve != cur_curve) {  // warp-uniform: this curve's moments
          mom = a.moments + (size_t)sg.curve * MO_WORDS;
          ybar = w_of<W>(mom[MO_YBAR]);
          YY = w_of<W>(mom[MO_YY]);
          YYr = (R)mom[MO_YY];
          cur_curve = sg.curve;
        }
      }
    }
    if (tau != cur_tau) {  // warp-uniform: this warp's template tables (FP64, then wide)
      const double2* al = a.alpha + (size_t)tau * kMaxH;
      for (int e = lane; e <= 2 * H; e += 32) {
        double2 k = make_double2(0.0, 0.0);
        for (int n = 1; n <= H; ++n) {
          if (e - n >= 1 && e - n <= H) k = cfma(al[n - 1], al[e - n - 1], k);
          if (n - e >= 1) k = cfma(cscale(al[n - 1], 2.0), cconj(al[n - e - 1]), k);
        }
        KE[e] = mkc(w_of<W>(k.x), w_of<W>(k.y));
        KER[e] = mk<R2>(k.x, k.y);
      }
      if (lane < H) {
        AL[lane] = mkc(w_of<W>(al[lane].x), w_of<W>(al[lane].y));
        ALR[lane] = mk<R2>(al[lane].x, al[lane].y);
      }
      double sa = 0.0;
      for (int n = 0; n < H; ++n) sa += sqrt(cabs2(al[n]));
      sum_abs_alpha = (R)sa;
      cur_tau = tau;
      __syncwarp();
    }
    const bool landed = mbar_wait(&mbar[buf], parity[buf], polls);
    parity[buf] ^= 1u;
    if (__any_sync(0xffffffffu, !landed)) {
      // give up: report the timeout, then let this warp's copies in flight
      // (the late unit's and the next unit's, each waited on once more with
      // the same bound) land before the CTA's shared memory is released
      if (lane == 0) atomicCAS(&a.status[ST_CODE], DEV_OK, DEV_TIMEOUT);
      mbar_wait(&mbar[buf], parity[buf] ^ 1u, polls);
      if (un < nunits) mbar_wait(&mbar[buf ^ 1], parity[buf ^ 1], polls);
      break;
    }
    const S2* st = stage + (size_t)buf * (C::STAGE_BYTES / sizeof(S2));
    const int64_t k = redo_pass ? cu.kfirst : cu.kfirst + gi;
    bool valid = unit_ok && (redo_pass ? gi == 0 : k < seg_nf);
    if (valid && a.sel_mode == 2)  // FP64 re-solve: only frequencies still at the cap
      valid = (a.sel_mark[a.kmap[k]] & MARK_FP64) != 0;

    R amax2 = R(0), bmax2 = R(0);
    if (a.coef_mode) {
      // pre-assembled coefficients (a_0..a_2H, b_1..b_H, c_1..c_H) of this item
      for (int q = gl; q < C::CROWS; q += G) {
        const S2 v = st[q * NGW + gi];
        WC wv;
        if constexpr (C::kDD) {
          wv = mkc(w_off<W>((float)v.x), w_off<W>((float)v.y));
        } else {
          wv = mkc((double)v.x, (double)v.y);
        }
        const R2 rw = mk<R2>((R)v.x, (R)v.y);
        if (q <= 2 * H) {
          A64[q] = wv;
          if constexpr (PH == 1) {
            Aw[q] = rw;
            amax2 = fmax(amax2, cabs2(rw));
          }
        } else if (q <= 3 * H) {
          B64[q - 2 * H] = wv;
          if constexpr (PH == 1) {
            Bw[q - 2 * H] = rw;
            bmax2 = fmax(bmax2, cabs2(rw));
          }
        } else {
          C64[q - 3 * H] = wv;
        }
      }
      if (gl == 0) {
        B64[0] = c_zero<W>();
        C64[0] = c_zero<W>();
        Bw[0] = mk<R2>(0, 0);
      }
      if constexpr (PH == 2) {
        // the second kernel evaluates <M^2> - Mbar^2: a_e + S_e from the rows
        __syncwarp();
        for (int e = gl; e <= 2 * H; e += G) {
          WC S = c_zero<W>();
          if (e == 0) {
            W q = w_zero<W>();
            for (int n = 1; n <= H; ++n) q = w_add(q, c_abs2<W>(C64[n]));
            S = mkc(w_mulf(q, 2.0f), w_zero<W>());
          } else {
            const int nlo = e - H > 1 ? e - H : 1;
            for (int n = nlo; 2 * n <= e; ++n) {
              const WC t = c_mul<W>(C64[n], C64[e - n]);
              S = c_add<W>(S, (2 * n == e) ? t : c_mulf<W>(t, 2.0f));
            }
            for (int n = e + 1; n <= H; ++n)
              S = c_add<W>(S, c_mulf<W>(c_mul<W>(C64[n], c_conj<W>(C64[n - e])), 2.0f));
          }
          A64[e] = c_add<W>(A64[e], S);
        }
      }
    } else if constexpr (PH == 1 && C::kDD) {
      // ---- (b) assembly in FP32 for the mixed path's first kernel.  Its final
      //      polynomial, root search and candidate screening run in FP32, and
      //      an FP32 assembly errs by ~6e-8 of its terms, below the ~4e-7
      //      error of the FP32 NFFT sums it starts from; the second kernel
      //      assembles again in float-float for the polish and the outputs.
      R2* Zr = reinterpret_cast<R2*>(Z64);
      R2* Yr = reinterpret_cast<R2*>(Y64);
      R2* Cr = reinterpret_cast<R2*>(C64);
      for (int q = gl; q < C::ROWS; q += G) {
        const S2 v = st[q * NGW + gi];
        const R2 rv = mk<R2>((R)v.x, (R)v.y);
        if (q < 2 * H) Zr[q + 1] = rv;
        else Yr[q - 2 * H + 1] = rv;
      }
      if (gl == 0) {
        Zr[0] = mk<R2>(1, 0);
        Yr[0] = mk<R2>(0, 0);
      }
      __syncwarp();
      for (int kk = gl; kk <= H; kk += G) {
        R2 bv = mk<R2>(0, 0), cv = mk<R2>(0, 0);
        if (kk > 0) {
          const R2 al = ALR[kk - 1];
          bv = cmul(al, cconj(Yr[kk]));
          cv = cmul(al, cconj(Zr[kk]));
        }
        Bw[kk] = bv;
        Cr[kk] = cv;
        bmax2 = fmax(bmax2, cabs2(bv));
      }
      __syncwarp();
      for (int s = gl; s < C::NSLOT; s += G) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          if (s == 0 && half == 1) break;
          const int e = (s == 0) ? 0 : (half == 0 ? s : 2 * H + 1 - s);
          R2 acc;
          if (e == 0) {
            R q = R(0);
            for (int n = 1; n <= H; ++n) q += cabs2(Cr[n]);
            acc = mk<R2>(KER[0].x - R(2) * q, 0);
          } else {
            R2 S = mk<R2>(0, 0);
            const int nlo = e - H > 1 ? e - H : 1;
            for (int n = nlo; 2 * n <= e; ++n) {  // sum_{n+m=e} c_n c_m, symmetric
              const R2 t = cmul(Cr[n], Cr[e - n]);
              S = (2 * n == e) ? mk<R2>(S.x + t.x, S.y + t.y)
                               : mk<R2>(fma(R(2), t.x, S.x), fma(R(2), t.y, S.y));
            }
            for (int n = e + 1; n <= H; ++n) {  // 2 sum_{n-m=e} c_n conj(c_m)
              const R2 t = cmul(Cr[n], cconj(Cr[n - e]));
              S = mk<R2>(fma(R(2), t.x, S.x), fma(R(2), t.y, S.y));
            }
            acc = csub(cmul(cconj(Zr[e]), KER[e]), S);
          }
          Aw[e] = acc;
          amax2 = fmax(amax2, cabs2(acc));
        }
      }
    } else {
      // ---- sums of this item into wide shared memory (one conversion each)
      for (int q = gl; q < C::ROWS; q += G) {
        const S2 v = st[q * NGW + gi];
        WC wv;
        if constexpr (C::kDD) {
          wv = mkc(w_off<W>((float)v.x), w_off<W>((float)v.y));
        } else {
          wv = mkc((double)v.x, (double)v.y);
        }
        if (q < 2 * H) Z64[q + 1] = wv;
        else Y64[q - 2 * H + 1] = wv;
      }
      if (gl == 0) {
        Z64[0] = mkc(w_of<W>(1.0), w_zero<W>());
        Y64[0] = c_zero<W>();
      }
      __syncwarp();

      // ---- (b) assembly (FP64-class).  b_k = alpha_k conj(Y_k), c_n = alpha_n conj(Z_n)
      for (int kk = gl; kk <= H; kk += G) {
        WC bv = c_zero<W>(), cv = c_zero<W>();
        if (kk > 0) {
          bv = c_mul<W>(AL[kk - 1], c_conj<W>(Y64[kk]));
          cv = c_mul<W>(AL[kk - 1], c_conj<W>(Z64[kk]));
        }
        B64[kk] = bv;
        C64[kk] = cv;
        if constexpr (PH == 1) {  // working-precision copy for the root search
          const R2 bw = mk<R2>((R)w_f(re(bv)), (R)w_f(im(bv)));
          Bw[kk] = bw;
          bmax2 = fmax(bmax2, cabs2(bw));
        }
      }
      __syncwarp();
      // a_e = conj(Z_e) K_e - S_e over slots {0}, {e, 2H+1-e}.  The second
      // kernel keeps the raw part conj(Z_e) K_e (the coefficients of <M^2>)
      // and subtracts Mbar^2 at the evaluation point instead of S_e (the
      // coefficients of Mbar^2): O(H) products per item instead of O(H^2).
      for (int s = gl; s < C::NSLOT; s += G) {
  #pragma unroll
        for (int half = 0; half < 2; ++half) {
          if (s == 0 && half == 1) break;
          const int e = (s == 0) ? 0 : (half == 0 ? s : 2 * H + 1 - s);
          WC acc;
          if constexpr (PH == 2) {
            acc = (e == 0) ? mkc(re(KE[0]), w_zero<W>()) : c_mul<W>(c_conj<W>(Z64[e]), KE[e]);
          } else if (e == 0) {
            W q = w_zero<W>();
            for (int n = 1; n <= H; ++n) q = w_add(q, c_abs2<W>(C64[n]));
            acc = mkc(w_sub(re(KE[0]), w_mulf(q, 2.0f)), w_zero<W>());
          } else {
            WC S = c_zero<W>();
            const int nlo = e - H > 1 ? e - H : 1;
            for (int n = nlo; 2 * n <= e; ++n) {  // sum_{n+m=e} c_n c_m, symmetric
              const WC t = c_mul<W>(C64[n], C64[e - n]);
              S = c_add<W>(S, (2 * n == e) ? t : c_mulf<W>(t, 2.0f));
            }
            for (int n = e + 1; n <= H; ++n)  // 2 sum_{n-m=e} c_n conj(c_m)
              S = c_add<W>(S, c_mulf<W>(c_mul<W>(C64[n], c_conj<W>(C64[n - e])), 2.0f));
            acc = c_sub<W>(c_mul<W>(c_conj<W>(Z64[e]), KE[e]), S);
          }
          A64[e] = acc;
          if constexpr (PH == 1) {
            const R2 aw = mk<R2>((R)w_f(re(acc)), (R)w_f(im(acc)));
            Aw[e] = aw;
            amax2 = fmax(amax2, cabs2(aw));
          }
        }
      }
    }
    __syncwarp();
    if constexpr (PH == 1) {
      amax2 = gmax<G>(amax2);
      bmax2 = gmax<G>(bmax2);
    }

    // ---- this item's output slot (both phases)
    int64_t col = 0, ridx = 0, ostride = a.out_stride;
    size_t o = 0;
    if (valid) {
      if (!batched) {
        col = a.kmap ? (int64_t)a.kmap[k] : k;
        o = (size_t)a.rows[tau] * a.out_stride + col;
        ridx = col;
      } else {
        const RootsSeg& sg = a.segs[cu.seg];
        col = redo_pass ? (int64_t)a.kmap[k] - sg.redo_base : k;
        const int row = sg.row_first < 0 ? 0 : a.rows[sg.row_first + cu.tl];
        o = (size_t)(sg.out_off + (int64_t)row * sg.nf + col);
        ostride = sg.nf;
        ridx = sg.redo_base + col;
      }
    }
    const bool in_range =
        FTP_DCHECK(a.status, !valid || (col >= 0 && col < ostride), 21, col, ostride) &&
        FTP_DCHECK(a.status, !valid || (int64_t)o < a.out_elems, 22, o, a.out_elems);

    if constexpr (PH == 1) {
    // ---- final polynomial F_p, p = 0..3H-1, in the working precision:
    //      [psi^p] (2 MM' d(YM') - YM' d(MM')) = sum_{j+l=p+1} (2l - j) m_j y_l
    //      with m_j = [psi^j] MM' (j = 0..4H) and y_l = [psi^l] YM' (l = 0..2H,
    //      y_H = 0), laid out once in the sums' shared memory (dead after the
    //      assembly) so that the sum is a branch-free convolution.
    R2* Mx = reinterpret_cast<R2*>(Z64);
    R2* Yx = Mx + (4 * H + 1);
    static_assert((6 * H + 2) * sizeof(R2) <= C::G_F - C::G_Z64, "convolution arrays fit");
    for (int j = gl; j <= 4 * H; j += G) Mx[j] = (j >= 2 * H) ? Aw[j - 2 * H] : cconj(Aw[2 * H - j]);
    for (int l = gl; l <= 2 * H; l += G)
      Yx[l] = (l == H) ? mk<R2>(0, 0) : (l > H) ? Bw[l - H] : cconj(Bw[H - l]);
    __syncwarp();
    R2 Fl[C::NFL];
    R fmax2 = R(0);
#pragma unroll
    for (int i = 0; i < C::NFL; ++i) {
      const int p = gl + G * i;
      R2 acc = mk<R2>(0, 0);
      if (p < C::NF) {
        const int jlo = p + 1 - 2 * H > 0 ? p + 1 - 2 * H : 0;
        const int jhi = p + 1 < 4 * H ? p + 1 : 4 * H;
        R cf = (R)(2 * (p + 1) - 3 * jlo);  // 2l - j = 2(p + 1) - 3j, exact
#pragma unroll 4
        for (int j = jlo; j <= jhi; ++j) {
          const R2 t = cmul(Mx[j], Yx[p + 1 - j]);
          acc = mk<R2>(fma(cf, t.x, acc.x), fma(cf, t.y, acc.y));
          cf -= R(3);
        }
        if (p == C::NF - 1) acc.x = R(0);  // F_{D/2} = -conj(F_{D/2}) is imaginary
      }
      Fl[i] = acc;
      fmax2 = fmax(fmax2, cabs2(acc));
    }
    fmax2 = gmax<G>(fmax2);
    // P independent of theta2 (or YM == 0): no roots to find.
    const bool constant = !valid || !(bmax2 > R(0)) ||
                          !(fmax2 > const_rel * const_rel * (R)(H * H) * amax2 * bmax2);
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

    // ---- initial guesses from the Newton polygon of F (Bini's rule): the
    //      upper convex hull of the points (k, log2|F_k|^2), k = 0..D.  An
    //      edge from vertex a to vertex b stands for b - a roots of modulus
    //      about 2^(-slope/2).  F is anti-self-inversive (|F_k| = |F_{D-k}|),
    //      so the hull is symmetric about D/2: only k <= D/2 matter, slot
    //      m < D/2 takes the m-th root counted from the innermost circle and
    //      slot D/2 + m its mirror 1/conj(z), half a step further round.  The
    //      circles' angles are offset by golden-ratio multiples of their first
    //      vertex, so that no two circles start aligned.  FP32 for either
    //      precision.
    constexpr int HD = D / 2;
    __syncwarp();
    float* Lg = reinterpret_cast<float*>(Z64);  // the sums are dead after the assembly
    for (int q = gl; q <= HD; q += G) {
      const float fx = (float)Fs[q].x, fy = (float)Fs[q].y;
      Lg[q] = __log2f(fmaf(fx, fx, fmaf(fy, fy, 1.17549435e-38f)));
    }
    __syncwarp();
    // Vertices of the upper hull of the left half k = 0..D/2 that it reaches
    // while still rising — by symmetry the rest of the hull lies under the
    // horizontal edge to the mirror vertex.  Point q is a hull vertex iff it
    // lies strictly above every chord from a point left of it to a point
    // right of it, i.e. iff L(q) = min over o < q of the slope o -> q exceeds
    // R(q) = max over k > q of the slope q -> k; L(q) is then the slope of
    // the hull edge into q, so the hull still rises into q iff L(q) > 0
    // (collinear points are not vertices; k = 0 always is).  The lanes of a
    // group test their points in parallel, O(D^2 / G) independent slopes per
    // lane, where a monotone chain would be a serial O(D) walk on one lane.
    unsigned long long vmask = 0ull;
    for (int q = gl; q <= HD; q += G) {
      if (q == 0) continue;
      const float Lq = Lg[q];
      float lo = 3.0e38f, hi = -3.0e38f;
#pragma unroll 4
      for (int j = 0; j <= HD; ++j) {
        const float sl = (Lq - Lg[j]) * fast_rcp((float)(q - j));  // slope j -> q (q -> j)
        if (j < q) lo = fminf(lo, sl);
        if (j > q) hi = fmaxf(hi, sl);
      }
      if (lo > hi && lo > 0.0f && Lq == Lq) vmask |= 1ull << q;  // (a NaN point is none)
    }
#pragma unroll
    for (int sh = G / 2; sh > 0; sh >>= 1) vmask |= __shfl_xor_sync(0xffffffffu, vmask, sh, G);
    vmask |= 1ull;

    // ---- (c) Aberth-Ehrlich on F (degree D), roots i = r*G + gl.  The
    //      settled-root marks follow the compaction lists (D shorts) in the
    //      sums' shared memory, clear of the hull's D/2 + 1 floats.
    unsigned char* const settled = reinterpret_cast<unsigned char*>(Z64) + rup(2 * D + 4, 16);
    static_assert(rup(2 * D + 4, 16) + D <= C::NA * 16, "settled-root marks fit");
    R2 z[RR];
    bool conv[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const int i = r * G + gl;
      z[r] = mk<R2>(0, 0);
      if (i < D) {
        const bool outer = i >= HD;
        const int m = outer ? i - HD : i;
        const unsigned long long below = (2ull << m) - 1ull;  // bits 0..m
        const int va = 63 - __clzll(vmask & below);           // last vertex <= m
        const unsigned long long above = vmask & ~below;
        const int vb = above ? __ffsll(above) - 1 : D - va;  // next vertex (or the mirror of va)
        const int cnt = min(vb, HD) - va;                     // roots of this circle in slots < D/2
        const float slope = (Lg[vb <= HD ? vb : D - vb] - Lg[va]) * fast_rcp((float)(2 * (vb - va)));
        const float lr = fminf(fmaxf(-slope, -12.0f), 12.0f);  // log2 of the inner modulus
        const float ang = 6.2831853f * ((float)(m - va) + (outer ? 0.5f : 0.0f)) * fast_rcp((float)cnt) +
                          0.4f + 3.8832221f * (float)va;       // 2 pi (golden ratio - 1) per vertex
        float sn, cs;
        __sincosf(ang, &sn, &cs);
        const float rad = fast_exp2(outer ? -lr : lr);
        z[r] = mk<R2>((R)(rad * cs), (R)(rad * sn));
      }
      conv[r] = (i >= D) || constant;
      if (i < D) {
        Zs[i] = z[r];
        if constexpr (C::kSettle) settled[i] = 0;
      }
    }
    __syncwarp();
    // Iterations over all RR slots per lane until every group of the warp has
    // at most RS * G unconverged roots, then over RS slots per lane holding
    // the unconverged roots only (listed per group in shared memory;
    // converged ones stay in Zs for the pair sums), then likewise over RT.
    constexpr int RS = (RR + 1) / 2;
    constexpr int RT = (RR + 3) / 4;
    int iters = 0;
    bool lane_nc = false;
    {
      short* act = reinterpret_cast<short*>(Z64);  // free after the Newton polygon
      int idx[RR];
#pragma unroll
      for (int r = 0; r < RR; ++r) idx[r] = r * G + gl < D ? r * G + gl : -1;
      if (aberth_run<G, RR, RS, D, C::kAccept, C::kSettle>(z, conv, idx, Fs, Zs, tol, iters, a.maxit, settled)) {
        if constexpr (RS < RR) {
          R2 z2[RS];
          bool c2[RS];
          int i2[RS];
          compact_roots<G, RR, RS>(conv, idx, act, Zs, gl, z2, c2, i2);
          if (aberth_run<G, RS, RT, D, C::kAccept, C::kSettle>(z2, c2, i2, Fs, Zs, tol, iters, a.maxit, settled)) {
            if constexpr (RT < RS) {
              R2 z3[RT];
              bool c3[RT];
              int i3[RT];
              compact_roots<G, RS, RT>(c2, i2, act, Zs, gl, z3, c3, i3);
              aberth_run<G, RT, RT, D, C::kAccept, C::kSettle>(z3, c3, i3, Fs, Zs, tol, iters, a.maxit, settled);
#pragma unroll
              for (int k = 0; k < RT; ++k) lane_nc = lane_nc || !c3[k];
            }
          } else {
#pragma unroll
            for (int k = 0; k < RS; ++k) lane_nc = lane_nc || !c2[k];
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < RR; ++r) lane_nc = lane_nc || !conv[r];
      }
    }
    bool nonconv = gor<G>(lane_nc) && !constant;
    if (__any_sync(0xffffffffu, nonconv)) {
      // at the cap keep the flag only if some root of the item is not a zero
      // of F to the working precision (the lanes split the roots): stalled
      // clusters are accepted here and need no re-solve
      bool bad = false;
      // (settled roots lie off the circle by construction and are not
      // zeros of F to the working precision)
      if (nonconv)
        for (int i = gl; i < D; i += G)
          bad = bad || (!(C::kSettle && settled[i]) && !pseudo_zero<D, R>(Zs[i], Fs));
      nonconv = gor<G>(bad);
    }

    // ---- candidates: P at the roots near the unit circle, scaled onto
    //      |psi| = 1 (working precision).  Only zeros of F on the circle are
    //      stationary points of P; the others (pairs z, 1/conj(z)) add
    //      candidates that cannot beat the best stationary value.  The group
    //      lists its roots with | |z|^2 - 1 | < kNearCircle (|z| within about
    //      0.05 of 1, far beyond the working-precision error of a root on the
    //      circle) in the compaction array, which is free now, and scores the
    //      list: one round of the loop in nearly every item instead of RR.  A
    //      group with no such root scores every root.  Rolled loops (roots
    //      read back from shared memory): this phase runs once per item.
    short* const cand = reinterpret_cast<short*>(Z64);
    int ncand = 1;
    bool every_root = true;
    {
      bool near[RR];
      int mine = 0;
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const int i = r * G + gl;
        near[r] = !constant && i < D && fabs(cabs2(Zs[i]) - R(1)) < R(kNearCircle);  // NaN: no
        mine += near[r] ? 1 : 0;
      }
      int incl = mine;  // every lane runs the shuffles (groups differ in `constant`)
#pragma unroll
      for (int sh = 1; sh < G; sh <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, sh, G);
        if (gl >= sh) incl += t;
      }
      const int total = __shfl_sync(0xffffffffu, incl, G - 1, G);
      int pos = incl - mine;
#pragma unroll
      for (int r = 0; r < RR; ++r)
        if (near[r]) cand[pos++] = (short)(r * G + gl);
      if (!constant) {
        every_root = total == 0;
        ncand = every_root ? D : total;
      }
    }
    __syncwarp();
    int nround = (ncand + G - 1) / G;  // rounds: the warp's longest list
#pragma unroll
    for (int sh = G; sh < 32; sh <<= 1) nround = max(nround, __shfl_xor_sync(0xffffffffu, nround, sh));
    R sc[RR], key[RR];
    int rix[RR];
    R lmax = R(-1);
    const R a0w = Aw[0].x;
#pragma unroll 1
    for (int r = 0; r < nround; ++r) {
      const int q = r * G + gl;
      const int i = q < ncand ? (every_root ? q : (int)cand[q]) : -1;
      R s = R(-1), kk = R(0);
      bool have = false;
      R2 p = mk<R2>(1, 0);
      if (constant) {
        have = (i == 0);
      } else if (i >= 0) {
        const R2 zi = Zs[i];
        const R m2 = cabs2(zi);
        have = m2 > R(0) && isfinite(m2);
        const R inv = have ? fast_rsqrt(m2) : R(0);
        p = mk<R2>(zi.x * inv, zi.y * inv);
      }
      if (have) {
        const R mm = trig_eval(Aw, 2 * H, p, a0w);
        const R ym = trig_eval(Bw, H, p, R(0));
        s = (mm > R(1e-9) * a0w) ? ym * ym * fast_rcp(mm) : R(0);
        const bool pos = ym > R(0);
        // positive-amplitude mode: only candidates with theta1 = YM/MM > 0
        if (a.positive_only && !pos) s = R(-1);
        kk = (pos ? R(0) : R(16)) + pseudo_angle(p);
        lmax = fmax(lmax, s);
      }
      sc[r] = s;
      key[r] = kk;
      rix[r] = i;
    }
    const R pmax = gmax<G>(lmax);
    const R thr = pmax - tie * (pmax > R(0) ? pmax : R(0));
    // among candidates within the tie band: theta1 > 0 first, then smallest
    // theta2; the winner's psi travels with its key
    R bkey = R(1e30);
    int bslot = -1;
#pragma unroll 1
    for (int r = 0; r < nround; ++r)
      if (sc[r] >= thr && sc[r] >= R(0) && key[r] < bkey) {
        bkey = key[r];
        bslot = rix[r];
      }
    R2 bpsi = mk<R2>(1, 0);
    if (bslot >= 0 && !constant) {
      const R2 zi = Zs[bslot];
      const R inv = fast_rsqrt(cabs2(zi));
      bpsi = mk<R2>(zi.x * inv, zi.y * inv);
    }
#pragma unroll
    for (int sh = G / 2; sh > 0; sh >>= 1) {
      const R ok = __shfl_xor_sync(0xffffffffu, bkey, sh, G);
      const R ox = __shfl_xor_sync(0xffffffffu, bpsi.x, sh, G);
      const R oy = __shfl_xor_sync(0xffffffffu, bpsi.y, sh, G);
      if (ok < bkey || (ok == bkey && (lane ^ sh) < lane)) {
        bkey = ok;
        bpsi = mk<R2>(ox, oy);
      }
    }
    const bool no_candidate = !(bkey < R(1e29));
    // the chosen phase and the flags for the second kernel
    {
      const unsigned bits = (constant ? 1u : 0u) | (nonconv ? 2u : 0u) | (no_candidate ? 4u : 0u);
      const double rv = gl == 0 ? (double)bpsi.x : gl == 1 ? (double)bpsi.y : (double)bits;
      if (valid && in_range && gl < 3) (gl == 0 ? a.power : gl == 1 ? a.theta1 : a.theta2)[o] = rv;
    }
    if (valid && in_range && gl == 0 && !a.resolve_pass) {
      st_iters += (unsigned long long)iters;
      st_items += 1;
      st_nonconv += nonconv ? 1 : 0;
    }
    } else {
    bool constant = true, nonconv = false, no_candidate = false;
    R2 bpsi = mk<R2>(1, 0);
    if (valid && in_range) {
      bpsi = mk<R2>((R)a.power[o], (R)a.theta1[o]);
      const unsigned bits = (unsigned)a.theta2[o];
      constant = (bits & 1u) != 0;
      nonconv = (bits & 2u) != 0;
      no_candidate = (bits & 4u) != 0;
    }
    R theta_w = atan2(bpsi.y, bpsi.x);
    if (theta_w < R(0)) theta_w += kTwoPi;
    // psi in wide precision, one Newton step onto |psi| = 1
    WC psi;
    if constexpr (C::kDD) {
      psi = mkc(w_off<W>((float)bpsi.x), w_off<W>((float)bpsi.y));
    } else {
      psi = mkc((double)bpsi.x, (double)bpsi.y);
    }
    {
      const W sfac = w_sub(w_of<W>(1.5), w_mulf(c_abs2<W>(psi), 0.5f));
      psi = mkc(w_mul(re(psi), sfac), w_mul(im(psi), sfac));
    }

    // ---- polish and evaluation in one FP64-class pass.  At psi (the chosen
    //      root) MM, YM, Mbar and their theta-derivatives come from
    //      trigonometric sums split over the group's lanes; one Newton step on
    //      g(theta) = 2 MM YM' - YM MM' gives the correction dl.  P is
    //      stationary, so P at psi differs from P at the corrected phase by
    //      O(dl^2); theta1 and Mbar are carried to it to first order.  Every
    //      lane runs the shuffles (groups differ in `constant`).
    // Trigonometric sums at phase psi over the group's lanes: returns
    // {Re S_a, Im S'_a, Re S''_a, Re S_b, Im S'_b, Re S''_b, Re S_c, Im S'_c}
    // with S_x = sum_e x_e psi^e, S'_x = sum_e e x_e psi^e, S''_x = sum e^2 ...
    auto trig_sums = [&](WC ps0, W* v) {
      const WC pw0 = group_powers<G, W>(ps0, gl);  // psi^(gl+1)
      const WC stp = mkc(w_shfl(re(pw0), G - 1, G), w_shfl(im(pw0), G - 1, G));  // psi^G
#pragma unroll
      for (int i = 0; i < 9; ++i) v[i] = w_zero<W>();
      WC pw = pw0;
#pragma unroll 1
      for (int e = gl + 1; e <= 2 * H; e += G) {
        const WC t = c_mul<W>(A64[e], pw);
        v[0] = w_add(v[0], re(t));
        v[1] = w_add(v[1], w_mulf(im(t), (float)e));
        v[2] = w_add(v[2], w_mulf(re(t), (float)(e * e)));
        if (e <= H) {
          const WC tb = c_mul<W>(B64[e], pw);
          v[3] = w_add(v[3], re(tb));
          v[4] = w_add(v[4], w_mulf(im(tb), (float)e));
          v[5] = w_add(v[5], w_mulf(re(tb), (float)(e * e)));
          const WC tc = c_mul<W>(C64[e], pw);
          v[6] = w_add(v[6], re(tc));
          v[7] = w_add(v[7], w_mulf(im(tc), (float)e));
          v[8] = w_add(v[8], w_mulf(re(tc), (float)(e * e)));
        }
        pw = c_mul<W>(pw, stp);
      }
      wsum8<G, W>(v, gl);
      v[8] = wsum<G>(v[8]);
    };
    W MM, YM, Mbar, dl = w_zero<W>(), th1 = w_zero<W>();
    {
      // pass 0 at psi; pass 1 (only when some item needs it) at the
      // corrected phase.  One loop keeps a single copy of the sums' code.
      WC pe = psi;
      bool again = false;
      W MM0 = w_zero<W>(), YM0 = w_zero<W>(), Mb0 = w_zero<W>();
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        W v[9];
        trig_sums(pe, v);
        // <M^2> = Q, Mbar and their theta-derivatives; MM = Q - Mbar^2
        const W Mb = w_mulf(v[6], 2.0f);
        const W Q = w_add(re(A64[0]), w_mulf(v[0], 2.0f));
        if (pass == 1) {
          if (again) {
            const W MM1 = w_sub(Q, w_mul(Mb, Mb));
            const W YM1 = w_mulf(v[3], 2.0f);
            // keep the corrected phase unless it lowers P (a step that left
            // the maximum's basin): P0 = YM0^2 / MM0 against P1
            const double m0 = w_d(MM0), m1 = w_d(MM1), y0 = w_d(YM0), y1 = w_d(YM1);
            if (m1 > 0.0 && y1 * y1 * m0 >= y0 * y0 * m1 * (1.0 - 1e-11)) {
              MM = MM1;
              YM = YM1;
              Mbar = Mb;
              th1 = w_div(YM, MM);
            } else {
              dl = w_zero<W>();
              MM = MM0;
              YM = YM0;
              Mbar = Mb0;
              th1 = (w_f(MM) > 0.0f) ? w_div(YM, MM) : w_zero<W>();
            }
          }
          break;
        }
        Mbar = Mb;
        const W Mbart = w_mulf(v[7], -2.0f), Mbartt = w_mulf(v[8], -2.0f);
        MM = w_sub(Q, w_mul(Mbar, Mbar));
        const W MMt = w_sub(w_mulf(v[1], -2.0f), w_mulf(w_mul(Mbar, Mbart), 2.0f));
        const W MMtt = w_sub(w_mulf(v[2], -2.0f),
                             w_mulf(w_add(w_mul(Mbart, Mbart), w_mul(Mbar, Mbartt)), 2.0f));
        YM = w_mulf(v[3], 2.0f);
        const W YMt = w_mulf(v[4], -2.0f), YMtt = w_mulf(v[5], -2.0f);
        MM0 = MM;
        YM0 = YM;
        Mb0 = Mbar;
        // The residual g is formed in the wide type; on the float-float path
        // the correction itself only needs FP32 (|dl| < 0.05, so its
        // relative error of ~1e-7 is below 5e-9 absolute, and a Newton step
        // from an FP32 root leaves an error of order dl^2).  A root of F near
        // a flat maximum can be off by more than 1e-3 rad in FP32; larger
        // steps are checked against P below.
        if (a.polish_steps > 0 && !constant) {
          const W g = w_sub(w_mulf(w_mul(MM, YMt), 2.0f), w_mul(YM, MMt));
          const W gt = w_sub(w_add(w_mul(MMt, YMt), w_mulf(w_mul(MM, YMtt), 2.0f)), w_mul(YM, MMtt));
          W d;
          if constexpr (C::kDD) {
            d = w_off<W>(w_f(g) * fast_rcp(w_f(gt)));
          } else {
            d = w_div(g, gt);
          }
          const float df = w_f(d);
          if (isfinite(df) && fabsf(df) < 0.05f) dl = d;
        }
        if (w_f(MM) > 0.0f) {
          const W q = w_div(YM, MM);
          if constexpr (C::kDD) {
            const float mf = w_f(MM);
            const float dq = (w_f(YMt) * mf - w_f(YM) * w_f(MMt)) * fast_rcp(mf * mf);
            th1 = w_sub(q, w_off<W>(w_f(dl) * dq));
          } else {
            const W dq = w_div(w_sub(w_mul(YMt, MM), w_mul(YM, MMt)), w_mul(MM, MM));
            th1 = w_sub(q, w_mul(dl, dq));
          }
        }
        Mbar = w_sub(Mbar, w_mul(dl, Mbart));
        // A correction that is not tiny (an ill-conditioned item) makes the
        // O(dl^2) shortcut too coarse: evaluate again at the corrected phase
        // psi e^{-i dl} (Taylor series of cos, sin to dl^5: truncation below
        // 3e-11 for |dl| < 0.05).
        again = fabsf(w_f(dl)) > (kFast ? 1e-5f : 1e-9f);
        if (!__any_sync(0xffffffffu, again)) break;
        const W d2 = w_mul(dl, dl);
        const W cs = w_sub(w_of<W>(1.0), w_mul(d2, w_sub(w_of<W>(0.5), w_mul(d2, w_of<W>(1.0 / 24.0)))));
        const W sn = w_mul(dl, w_sub(w_of<W>(1.0), w_mul(d2, w_sub(w_of<W>(1.0 / 6.0),
                                                                  w_mul(d2, w_of<W>(1.0 / 120.0))))));
        pe = mkc(w_add(w_mul(re(psi), cs), w_mul(im(psi), sn)),
                 w_sub(w_mul(im(psi), cs), w_mul(re(psi), sn)));
        {  // back onto |psi| = 1 (the truncated series leaves ~dl^6/720)
          const W sfac = w_sub(w_of<W>(1.5), w_mulf(c_abs2<W>(pe), 0.5f));
          pe = mkc(w_mul(re(pe), sfac), w_mul(im(pe), sfac));
        }
      }
    }
    W theta;
    if constexpr (kFast) {
      theta = w_sub(w_off<W>((float)theta_w), dl);
    } else {
      theta = w_sub(atan2(w_d(im(psi)), w_d(re(psi))), dl);
    }
    if (w_f(theta) < 0.0f) theta = w_add(theta, twopi);
    if (w_f(theta) >= w_f(twopi)) theta = w_sub(theta, twopi);
    const float MMf = w_f(MM), Mbf = w_f(Mbar);
    const bool degenerate = !(MMf > 1e-14f * (MMf + Mbf * Mbf)) || !(MMf > 0.0f);
    W P = w_zero<W>();
    if (!degenerate) {
      P = w_div(w_mul(YM, YM), w_mul(YY, MM));
    } else {
      th1 = w_zero<W>();
    }
    // positive-amplitude mode without an admissible candidate: the best
    // theta1 >= 0 is 0 at every phase, so P = 0 (theta2 = 0, theta3 = ybar)
    const bool no_positive =
        a.positive_only && (no_candidate || degenerate || !(w_f(th1) > 0.0f));
    if (no_positive) {
      P = w_zero<W>();
      th1 = w_zero<W>();
      theta = w_zero<W>();
    }
    const W th3 = w_sub(ybar, w_mul(th1, Mbar));

    // ---- a-posteriori error of P from the NFFT sums: |dZ| <= e gives
    //      |dMM| <= 9 e (sum|alpha|)^2 and |dYM| <= 2 e sum|alpha| sqrt(YY);
    //      items whose P could be off by more than the threshold are
    //      re-solved from direct FP64 sums.
    bool redo = false;
    if (a.sum_err > 0.0 && valid) {
      if (degenerate) {
        redo = true;
      } else {
        const R Pf = (R)w_f(P), Mf = (R)MMf;
        const R dMM = R(9) * (R)a.sum_err * sum_abs_alpha * sum_abs_alpha;
        // an estimate with margin: MUFU reciprocal and square root suffice
        const R dYM = R(2) * (R)a.sum_err * sum_abs_alpha * (YYr * fast_rsqrt(YYr));
        const R q = fmax(Pf, R(0)) * fast_rcp(YYr * Mf);
        const R sq = q > R(0) ? q * fast_rsqrt(q) : R(0);
        const R err = Pf * dMM * fast_rcp(Mf) + R(2) * sq * dYM;
        redo = !(err <= (R)a.redo_tol);
      }
    }

    // ---- outputs: lanes 0..3 of the group convert one value each (one
    //      conversion instruction for the whole warp), then write it
    {
      const W v = gl == 0 ? P : gl == 1 ? th1 : gl == 2 ? theta : th3;
      const double dv = w_d(v);
      if (valid && in_range && gl < 4) {
        double* dst = gl == 0 ? a.power : gl == 1 ? a.theta1 : gl == 2 ? a.theta2 : a.theta3;
        dst[o] = dv;
      }
    }
    if (valid && in_range && gl == 0) {
      // A frequency goes on the re-solve list once (mark 0 -> MARK_LISTED),
      // with MARK_FP64 added when one of its items hit the iteration cap
      // (re-solved with FP64 Aberth iterations); if the list is full the
      // mark gets MARK_OVERFLOW and a later pass flags its items.  Without a
      // list (a call that cannot re-solve) an item over the error threshold
      // is flagged unresolved.
      const bool cap = nonconv && a.list_nonconv;
      // a cap hit is final in the last re-solve pass and where no re-solve
      // follows; in the FP32 re-solve pass it sends its frequency on to the
      // FP64 one
      st_final += (nonconv && (a.resolve_pass == 2 ||
                               (!a.resolve_pass && !(a.list_nonconv && a.redo_list)))) ? 1 : 0;
      if (nonconv && a.resolve_pass == 1 && a.sel_mark)
        atomicOr(&a.sel_mark[a.kmap[k]], MARK_FP64);
      bool unresolved = false;
      if ((redo || cap) && a.redo_list) {
        if (FTP_DCHECK(a.status, ridx < a.redo_marks, 23, ridx, a.redo_marks)) {
          if (atomicCAS(&a.redo_mark[ridx], 0, MARK_LISTED) == 0) {
            const int slot = atomicAdd(a.redo_count, 1);
            if (slot < a.redo_cap) {
              a.redo_list[slot] = (int)ridx;
              ++st_redo;
            } else {
              atomicOr(&a.redo_mark[ridx], MARK_OVERFLOW);
            }
          }
          // counted once per frequency: by the item that sets the bit
          if (cap && (atomicOr(&a.redo_mark[ridx], MARK_CAP) & MARK_CAP) == 0) ++st_redo_nc;
        }
      } else if (redo && !a.resolve_pass) {
        unresolved = true;
      }
      if (a.flags) {
        unsigned f = 0;
        if (nonconv) f |= 1u;
        if (degenerate) f |= 2u;
        if (constant) f |= 4u;
        if (w_f(th1) < 0.0f) f |= 8u;
        if (unresolved) f |= 16u;
        if (no_positive) f |= 64u;
        if (a.resolve_pass) f |= 128u;
        a.flags[o] = (uint8_t)f;
      }
    }
    }  // phase 2
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
    st_redo_nc += __shfl_xor_sync(0xffffffffu, st_redo_nc, o);
    st_final += __shfl_xor_sync(0xffffffffu, st_final, o);
  }
  if (lane == 0 && (st_items || st_redo || st_final)) {
    atomicAdd(&a.counters[CNT_ITERS], st_iters);
    atomicAdd(&a.counters[CNT_ITEMS], (unsigned long long)st_items);
    atomicAdd(&a.counters[CNT_NONCONV], (unsigned long long)st_nonconv);
    atomicAdd(&a.counters[CNT_REDO], (unsigned long long)st_redo);
    atomicAdd(&a.counters[CNT_REDO_NC], (unsigned long long)st_redo_nc);
    atomicAdd(&a.counters[CNT_NC_FINAL], (unsigned long long)st_final);
  }
}

// Host side: opt in to the dynamic shared memory once per phase kernel, size
// the persistent grids, launch the two phases back to back.
template <typename S2, typename R, int H, int G, int PH>
int launch_phase(const RootsArgs& a, int num_sms, cudaStream_t s) {
  using C = Cfg<S2, R, H, G>;
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    if (cudaFuncSetAttribute(roots_kernel<S2, R, H, G, PH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C::SMEM) != cudaSuccess)
      return -2;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, roots_kernel<S2, R, H, G, PH>,
                                                      C::WARPS * 32, C::SMEM) != cudaSuccess ||
        b < 1)
      return -2;
    blocks_per_sm = b;
  }
  const int64_t nf = a.nf;  // upper bound when the count lives on the device
  const int64_t nunits = a.host_units > 0 ? a.host_units : (nf + C::NGW - 1) / C::NGW * a.ntpl;
  const int bps = (a.ctas_per_sm > 0 && a.ctas_per_sm < blocks_per_sm) ? a.ctas_per_sm
                                                                       : blocks_per_sm;
  int64_t grid = (int64_t)num_sms * bps;
  const int64_t need = (nunits + C::WARPS - 1) / C::WARPS;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  roots_kernel<S2, R, H, G, PH><<<(unsigned)grid, C::WARPS * 32, C::SMEM, s>>>(a);
  return 1;
}
template <typename S2, typename R, int H, int G>
int launch_h(const RootsArgs& a, int num_sms, cudaStream_t s) {
  if (a.ev_first_start) cudaEventRecord(a.ev_first_start, s);
  const int r = launch_phase<S2, R, H, G, 1>(a, num_sms, s);
  if (r < 0) return r;
  if (a.ev_first_end) cudaEventRecord(a.ev_first_end, s);
  const int r2 = launch_phase<S2, R, H, G, 2>(a, num_sms, s);
  return r2 < 0 ? r2 : r + r2;
}

}  // namespace roots
}  // namespace ftp
