// Steps (b) and (c) of the Fast Template Periodogram, fused in one kernel:
// polynomial assembly (Section 2: MM_nm, YM_k, Eq. finalpoly), all zeros of
// the final polynomial by Aberth-Ehrlich iteration, candidates scaled onto
// the unit circle (Section 2, end), the best one chosen and polished by a
// Newton step on the phase in FP64, and (theta1, theta2, theta3, P).
//
// Work item = (frequency k, template tau).  A group of G lanes owns one item:
// it assembles the coefficients, then each lane iterates R = ceil(D/G) of
// the D = 6H-2 roots.  A CTA processes NG consecutive frequencies of one
// template per work unit; their sum tiles (3H rows of NG complex values in the
// [3H][nf_pad] layout) are staged into shared memory by TMA bulk copies,
// double-buffered so the next unit's copy overlaps this unit's arithmetic.
//
// Notation.  Z_h = sum_i w_i e^{i h omega t_i} (Z_0 = 1, Z_{-h} = conj Z_h),
// Y_h = sum_i w_i (y_i - ybar) e^{i h omega t_i}, alpha_n = (c_n + i s_n)/2.
// With these, the covariance sums of Eqs. CCdef-SSdef combine into
//   CCt_nm = conj(Z_{n+m} - Z_n Z_m),  CSt_nm = Z_{m-n} - conj(Z_n) Z_m
// (product-to-sum identities), and the self-inversive polynomials are kept
// as real trigonometric polynomials in theta = theta2:
//   MM(theta) = a_0 + 2 Re sum_{e=1..2H} a_e psi^e,  a_e = [psi^{2H+e}] MM'
//   YM(theta) = 2 Re sum_{k=1..H} b_k psi^k,         b_k = alpha_k conj(Y_k)
//   Mbar(theta) = 2 Re sum_{n=1..H} c_n psi^n,        c_n = alpha_n conj(Z_n)
// The final polynomial F = 2 MM' d(YM') - YM' d(MM') is anti-self-inversive,
// F_{D-p} = -conj(F_p), so only p = 0..3H-1 are formed and the rest mirrored.
#pragma once

#include <math.h>

#include "ftp_internal.cuh"

namespace ftp {
namespace roots {

template <bool MIXED> struct PT;
template <> struct PT<true> {
  using S2 = float2;   // sum tile element
  using R = float;     // Aberth / screening precision
  using R2 = float2;
};
template <> struct PT<false> {
  using S2 = double2;
  using R = double;
  using R2 = double2;
};

__host__ __device__ constexpr size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <bool MIXED, int H>
struct Cfg {
  using P = PT<MIXED>;
  static constexpr int D = 6 * H - 2;
  static constexpr int G = MIXED ? (D <= 40 ? 4 : 8) : (D <= 24 ? 4 : (D <= 48 ? 8 : 16));
  static constexpr int R = (D + G - 1) / G;
  static constexpr int WARPS = 8;
  static constexpr int GPW = 32 / G;          // groups per warp
  static constexpr int NG = WARPS * GPW;      // frequencies per work unit
  static constexpr int ROWS = 3 * H;          // staged sum rows
  static constexpr int NA = 2 * H + 1;        // a_0..a_2H
  static constexpr int NB = H + 1;            // b_0..b_H, c_0..c_H
  static constexpr int NF = 3 * H;            // F_0..F_{3H-1}
  static constexpr int NFL = (NF + G - 1) / G;
  // per-group shared memory
  static constexpr size_t O_A64 = 0;
  static constexpr size_t O_B64 = O_A64 + NA * sizeof(double2);
  static constexpr size_t O_C64 = O_B64 + NB * sizeof(double2);
  static constexpr size_t O_F = O_C64 + NB * sizeof(double2);
  static constexpr size_t O_Z = O_F + rup((D + 1) * sizeof(typename P::R2), 16);
  static constexpr size_t O_A32 = O_Z + rup(R * G * sizeof(typename P::R2), 16);
  static constexpr size_t O_B32 = O_A32 + (MIXED ? rup(NA * sizeof(float2), 16) : 0);
  static constexpr size_t O_END = O_B32 + (MIXED ? rup(NB * sizeof(float2), 16) : 0);
  // stride = 16 (mod 128) bytes keeps the groups of a warp on distinct banks
  static constexpr size_t GROUP_BYTES = rup(O_END, 128) + 16;
  // per-CTA shared memory
  static constexpr size_t O_AA = 0;                                   // alpha_n alpha_m
  static constexpr size_t O_AC = O_AA + H * H * sizeof(double2);      // alpha_n conj(alpha_m)
  static constexpr size_t O_AL = O_AC + H * H * sizeof(double2);      // alpha_n
  static constexpr size_t O_MBAR = rup(O_AL + H * sizeof(double2), 16);
  static constexpr size_t O_STAGE = rup(O_MBAR + 16, 128);
  static constexpr size_t STAGE_BYTES = (size_t)ROWS * NG * sizeof(typename P::S2);
  static constexpr size_t O_GROUPS = rup(O_STAGE + 2 * STAGE_BYTES, 128);
  static constexpr size_t SMEM = O_GROUPS + (size_t)NG * GROUP_BYTES;
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
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) {
  a.x += b.x;
  a.y += b.y;
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
// a / b (plain formula; callers guard non-finite results)
__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  const float inv = __fdividef(1.0f, cabs2(b));
  return make_float2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double inv = 1.0 / cabs2(b);
  return make_double2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float2 to_r2(float2 v, float2*) { return v; }
__device__ __forceinline__ float2 to_r2(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_r2(double2 v, double2*) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
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

// Real trigonometric polynomial evaluation at psi (|psi| = 1):
//   v0 + 2 Re sum_{e=1..n} c_e psi^e, by Horner in psi.
template <typename T2>
__device__ __forceinline__ auto trig_eval(const T2* c, int n, T2 psi, decltype(T2().x) v0) {
  T2 acc = c[n];
  for (int e = n - 1; e >= 1; --e) acc = cfma(acc, psi, c[e]);
  acc = cmul(acc, psi);
  return v0 + 2 * acc.x;
}

template <bool MIXED, int H>
__global__ void __launch_bounds__(Cfg<MIXED, H>::WARPS * 32) roots_kernel(const RootsArgs a) {
  using C = Cfg<MIXED, H>;
  using S2 = typename C::P::S2;
  using R = typename C::P::R;
  using R2 = typename C::P::R2;
  constexpr int D = C::D, G = C::G, RR = C::R, NG = C::NG;
  constexpr R kTwoPi = R(6.283185307179586476925286766559);
  constexpr R tol = MIXED ? R(2e-6) : R(1e-12);
  constexpr R tie = MIXED ? R(1e-6) : R(1e-12);

  extern __shared__ __align__(128) unsigned char smem[];
  double2* AA = reinterpret_cast<double2*>(smem + C::O_AA);
  double2* AC = reinterpret_cast<double2*>(smem + C::O_AC);
  double2* AL = reinterpret_cast<double2*>(smem + C::O_AL);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + C::O_MBAR);
  S2* stage0 = reinterpret_cast<S2*>(smem + C::O_STAGE);

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane % G;
  const int grp = warp * C::GPW + lane / G;
  unsigned char* gb = smem + C::O_GROUPS + (size_t)grp * C::GROUP_BYTES;
  double2* A64 = reinterpret_cast<double2*>(gb + C::O_A64);
  double2* B64 = reinterpret_cast<double2*>(gb + C::O_B64);
  double2* C64 = reinterpret_cast<double2*>(gb + C::O_C64);
  R2* Fs = reinterpret_cast<R2*>(gb + C::O_F);
  R2* Zs = reinterpret_cast<R2*>(gb + C::O_Z);
  // screening coefficients in the working precision
  R2* Aw = MIXED ? reinterpret_cast<R2*>(gb + C::O_A32) : reinterpret_cast<R2*>(A64);
  R2* Bw = MIXED ? reinterpret_cast<R2*>(gb + C::O_B32) : reinterpret_cast<R2*>(B64);

  if (a.status[ST_CODE] != DEV_OK) return;
  const int64_t nkb = (a.nf + NG - 1) / NG;
  const int64_t nunits = nkb * a.ntpl;
  const double ybar = a.moments[MO_YBAR], YY = a.moments[MO_YY];

  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();

  // Thread 0 stages the 3H sum rows of unit u into buffer `buf`.
  auto issue = [&](int64_t u, int buf) {
    const int64_t kb = u % nkb;
    constexpr unsigned row_bytes = NG * sizeof(S2);
    S2* dst = stage0 + (size_t)buf * (C::STAGE_BYTES / sizeof(S2));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&mbar[buf], C::ROWS * row_bytes);
    const S2* sums = reinterpret_cast<const S2*>(a.sums);
#pragma unroll 1
    for (int r = 0; r < C::ROWS; ++r) {
      const int src_row = (r < 2 * H) ? r : 2 * a.Hs + (r - 2 * H);
      bulk_g2s(dst + (size_t)r * NG, sums + (size_t)src_row * a.nf_pad + kb * NG, row_bytes,
               &mbar[buf]);
    }
  };

  int64_t u = blockIdx.x;
  if (u < nunits && threadIdx.x == 0) issue(u, 0);
  int cur_tau = -1;
  for (int it = 0; u < nunits; u += gridDim.x, ++it) {
    const int buf = it & 1;
    const int64_t un = u + gridDim.x;
    if (un < nunits && threadIdx.x == 0) issue(un, buf ^ 1);
    const int tau = (int)(u / nkb);
    const int64_t kb = u % nkb;
    if (tau != cur_tau) {  // CTA-uniform
      for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
        const int n = i / H, m = i % H;
        const double2 an = a.alpha[(size_t)tau * kMaxH + n];
        const double2 am = a.alpha[(size_t)tau * kMaxH + m];
        AA[i] = cmul(an, am);
        AC[i] = cmul(an, cconj(am));
      }
      for (int i = threadIdx.x; i < H; i += blockDim.x) AL[i] = a.alpha[(size_t)tau * kMaxH + i];
      cur_tau = tau;
      __syncthreads();
    }
    const bool landed = mbar_wait(&mbar[buf], (unsigned)((it >> 1) & 1));
    if (__syncthreads_or(!landed)) {
      if (threadIdx.x == 0) atomicCAS(&a.status[ST_CODE], DEV_OK, DEV_TIMEOUT);
      return;
    }
    const S2* st = stage0 + (size_t)buf * (C::STAGE_BYTES / sizeof(S2));
    const int64_t k = kb * NG + grp;
    const bool valid = k < a.nf;

    auto Zv = [&](int h) -> double2 {  // Z_h, h in [-2H, 2H]
      if (h == 0) return make_double2(1.0, 0.0);
      const int hh = h < 0 ? -h : h;
      const double2 v = to_d2(st[(hh - 1) * NG + grp]);
      return h < 0 ? cconj(v) : v;
    };

    // ---- (b) assembly in FP64: a_e, b_k, c_n
    double amax2 = 0.0, bmax2 = 0.0;
    for (int e = gl; e <= 2 * H; e += G) {
      double2 acc = make_double2(0.0, 0.0);
      if (e == 0) {
        for (int n = 1; n <= H; ++n) acc.x += 2.0 * AC[(n - 1) * H + (n - 1)].x * (1.0 - cabs2(Zv(n)));
      } else {
        const double2 Ze = Zv(e);
        const int nlo = e - H > 1 ? e - H : 1, nhi = e - 1 < H ? e - 1 : H;
        for (int n = nlo; n <= nhi; ++n) {
          const double2 t = csub(Ze, cmul(Zv(n), Zv(e - n)));
          acc = cfma(AA[(n - 1) * H + (e - n - 1)], cconj(t), acc);
        }
        for (int n = e + 1; n <= H; ++n) {
          const double2 t = csub(cconj(Ze), cmul(cconj(Zv(n)), Zv(n - e)));
          acc = cfma(cscale(AC[(n - 1) * H + (n - e - 1)], 2.0), t, acc);
        }
      }
      A64[e] = acc;
      if constexpr (MIXED) Aw[e] = to_r2(acc, (R2*)nullptr);
      amax2 = fmax(amax2, cabs2(acc));
    }
    for (int kk = gl; kk <= H; kk += G) {
      double2 bv = make_double2(0.0, 0.0), cv = make_double2(0.0, 0.0);
      if (kk > 0) {
        const double2 Yk = to_d2(st[(2 * H + kk - 1) * NG + grp]);
        bv = cmul(AL[kk - 1], cconj(Yk));
        cv = cmul(AL[kk - 1], cconj(Zv(kk)));
      }
      B64[kk] = bv;
      C64[kk] = cv;
      if constexpr (MIXED) Bw[kk] = to_r2(bv, (R2*)nullptr);
      bmax2 = fmax(bmax2, cabs2(bv));
    }
    __syncwarp();

    // ---- final polynomial F_p, p = 0..3H-1 (FP64), coefficient of psi^p in
    //      2 MM' d(YM') - YM' d(MM'):  sum_{j+l=p+1} (2l - j) m_j y_l
    double2 Fl[C::NFL];
    double fmax2 = 0.0;
#pragma unroll
    for (int i = 0; i < C::NFL; ++i) {
      const int p = gl + G * i;
      double2 acc = make_double2(0.0, 0.0);
      if (p < C::NF) {
        const int jlo = p + 1 - 2 * H > 0 ? p + 1 - 2 * H : 0;
        const int jhi = p + 1 < 4 * H ? p + 1 : 4 * H;
        for (int j = jlo; j <= jhi; ++j) {
          const int l = p + 1 - j;
          if (l == H) continue;
          const double2 mj = (j >= 2 * H) ? A64[j - 2 * H] : cconj(A64[2 * H - j]);
          const double2 yl = (l > H) ? B64[l - H] : cconj(B64[H - l]);
          acc = cfma(cscale(mj, (double)(2 * l - j)), yl, acc);
        }
        if (p == C::NF - 1) acc.x = 0.0;  // F_{D/2} = -conj(F_{D/2}) is imaginary
      }
      Fl[i] = acc;
      fmax2 = fmax(fmax2, cabs2(acc));
    }
    fmax2 = gmax<G>(fmax2);
    amax2 = gmax<G>(amax2);
    bmax2 = gmax<G>(bmax2);
    // P independent of theta2 (or YM == 0): no roots to find.
    const bool constant =
        !valid || !(fmax2 > 1e-26 * (double)(H * H) * amax2 * bmax2) || !(bmax2 > 0.0);
    const double fscale = constant ? 0.0 : 1.0 / sqrt(fmax2);
#pragma unroll
    for (int i = 0; i < C::NFL; ++i) {
      const int p = gl + G * i;
      if (p < C::NF) {
        const R2 f = to_r2(cscale(Fl[i], fscale), (R2*)nullptr);
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
      if constexpr (MIXED) {
        __sincosf(ang, &sn, &cs);
      } else {
        sincos(ang, &sn, &cs);
      }
      const R rad = (i & 1) ? R(0.5) : R(2);
      z[r] = mk<R2>(rad * cs, rad * sn);
      conv[r] = (i >= D) || constant || !valid;
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
    const bool nonconv = gor<G>(lane_nc) && valid && !constant;

    // ---- candidates: P at every root scaled onto |psi| = 1 (working precision)
    R sc[RR], th[RR];
    bool pos[RR];
    R lmax = R(-1);
    const R a0w = Aw[0].x;
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const int i = r * G + gl;
      sc[r] = R(-1);
      th[r] = R(0);
      pos[r] = false;
      R2 psi;
      bool have = false;
      if (constant) {
        have = (i == 0);
        psi = mk<R2>(1, 0);
      } else if (i < D) {
        const R m2 = cabs2(z[r]);
        have = m2 > R(0) && isfinite(m2);
        const R inv = have ? R(1) / sqrt(m2) : R(0);
        psi = mk<R2>(z[r].x * inv, z[r].y * inv);
      }
      if (have) {
        const R mm = trig_eval(Aw, 2 * H, psi, a0w);
        const R ym = trig_eval(Bw, H, psi, R(0));
        sc[r] = (mm > R(1e-9) * a0w) ? ym * ym / mm : R(0);
        pos[r] = ym > R(0);
        R t2 = atan2(psi.y, psi.x);
        if (t2 < R(0)) t2 += kTwoPi;
        th[r] = t2;
        lmax = fmax(lmax, sc[r]);
      }
    }
    const R pmax = gmax<G>(lmax);
    const R thr = pmax - tie * (pmax > R(0) ? pmax : R(0));
    // among candidates within the tie band: theta1 > 0 first, then smallest theta2
    R bkey = R(1e30);
#pragma unroll
    for (int r = 0; r < RR; ++r)
      if (sc[r] >= thr && sc[r] >= R(0)) {
        const R key = (pos[r] ? R(0) : R(16)) + th[r];
        bkey = fmin(bkey, key);
      }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) bkey = fmin(bkey, __shfl_xor_sync(0xffffffffu, bkey, o, G));
    double theta = (double)(bkey >= R(16) ? bkey - R(16) : bkey);
    if (!(bkey < R(1e29))) theta = 0.0;

    // ---- FP64 Newton polish of the chosen phase on the real function
    //      g(theta) = 2 MM YM' - YM MM' (theta-derivatives), then P, theta1, theta3.
    auto trig3 = [&](const double2* cf, int n, double2 psi, double2& s0, double2& s1,
                     double2& s2) {
      s0 = s1 = s2 = make_double2(0.0, 0.0);
      double2 pw = psi;
      for (int e = 1; e <= n; ++e) {
        const double2 t = cmul(cf[e], pw);
        s0 = cadd(s0, t);
        s1 = cadd(s1, cscale(t, (double)e));
        s2 = cadd(s2, cscale(t, (double)(e * e)));
        pw = cmul(pw, psi);
      }
    };
    if (!constant) {
#pragma unroll 1
      for (int s = 0; s < a.polish_steps; ++s) {
        double sn, cs;
        sincos(theta, &sn, &cs);
        const double2 psi = make_double2(cs, sn);
        double2 a0, a1, a2, b0, b1, b2;
        trig3(A64, 2 * H, psi, a0, a1, a2);
        trig3(B64, H, psi, b0, b1, b2);
        const double MM = A64[0].x + 2.0 * a0.x, MMt = -2.0 * a1.y, MMtt = -2.0 * a2.x;
        const double YM = 2.0 * b0.x, YMt = -2.0 * b1.y, YMtt = -2.0 * b2.x;
        const double g = 2.0 * MM * YMt - YM * MMt;
        const double gt = MMt * YMt + 2.0 * MM * YMtt - YM * MMtt;
        const double step = g / gt;
        if (isfinite(step) && fabs(step) < 1e-3) theta -= step;
      }
    }
    double sn, cs;
    sincos(theta, &sn, &cs);
    const double2 psi = make_double2(cs, sn);
    double2 s0, s1, s2;
    trig3(A64, 2 * H, psi, s0, s1, s2);
    const double MM = A64[0].x + 2.0 * s0.x;
    trig3(B64, H, psi, s0, s1, s2);
    const double YM = 2.0 * s0.x;
    trig3(C64, H, psi, s0, s1, s2);
    const double Mbar = 2.0 * s0.x;
    const bool degenerate = !(MM > 1e-14 * (MM + Mbar * Mbar));
    double P = 0.0, th1 = 0.0;
    if (!degenerate) {
      th1 = YM / MM;
      P = YM * th1 / YY;
    }
    const double th3 = ybar - th1 * Mbar;
    theta = fmod(theta, 6.283185307179586476925286766559);
    if (theta < 0.0) theta += 6.283185307179586476925286766559;

    if (valid && gl == 0) {
      const size_t o = (size_t)a.rows[tau] * a.out_stride + k;
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
      if (nonconv) atomicAdd(&a.status[ST_NONCONV], 1);
    }
    __syncthreads();
  }
}

// Host side: opt in to the dynamic shared memory once, size the persistent grid.
template <bool MIXED, int H>
int launch_h(const RootsArgs& a, int num_sms, cudaStream_t s) {
  using C = Cfg<MIXED, H>;
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    if (cudaFuncSetAttribute(roots_kernel<MIXED, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C::SMEM) != cudaSuccess)
      return -2;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, roots_kernel<MIXED, H>, C::WARPS * 32,
                                                      C::SMEM) != cudaSuccess ||
        b < 1)
      return -2;
    blocks_per_sm = b;
  }
  const int64_t nunits = (a.nf + C::NG - 1) / C::NG * a.ntpl;
  int64_t grid = (int64_t)num_sms * blocks_per_sm;
  if (grid > nunits) grid = nunits;
  if (grid < 1) grid = 1;
  roots_kernel<MIXED, H><<<(unsigned)grid, C::WARPS * 32, C::SMEM, s>>>(a);
  return 1;
}

}  // namespace roots
}  // namespace ftp
