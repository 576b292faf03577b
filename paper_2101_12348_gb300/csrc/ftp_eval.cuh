// Second root-stage kernel of the mixed path's main pass, one lane per item:
// at the phase psi chosen by the first kernel, one float-float Newton step
// on g(theta) = 2 MM YM' - YM MM' and the evaluation of P, theta1, theta2,
// theta3 (Section 2: MM = Var M, YM = Cov(M, y), P = YM^2 / (YY MM),
// theta1 = YM / MM, theta3 = ybar - theta1 <M>), the a-posteriori error of P
// from the NFFT sums and the re-solve list.
//
// The first kernel's groups of G lanes per item suit the root search, whose
// D roots spread over the lanes.  Evaluation at one phase is O(H) per item
// and mostly scalar float-float arithmetic, which a group would repeat on
// every lane, with float-float shuffles to combine its partial sums; here
// each lane owns its item, forms the coefficients a_e = conj(Z_e) K_e,
// b_e = alpha_e conj(Y_e), c_e = alpha_e conj(Z_e) on the fly from the sums
// (read with plain loads: the items of a warp are consecutive frequencies,
// so each row read is one contiguous 256-byte segment) and sums them in
// order.  Work units are those of the first kernel (NGW1 consecutive
// frequencies of one template); a warp takes 32 / NGW1 consecutive units.
// The template table K_e, alpha_n (float-float) sits in the warp's shared
// memory and is rebuilt when the template changes; lanes whose items belong
// to another template than the warp's first (at template and curve
// boundaries) run in a second round.
#pragma once

#include "ftp_roots.cuh"

namespace ftp {
namespace roots {

template <int H>
struct EvalCfg {
  static constexpr int WARPS = 4;
  static constexpr int NA = 2 * H + 1;
  // K_e (e = 0..2H) and alpha_n (n = 1..H), 16 bytes each, and sum |alpha_n|
  static constexpr size_t WARP_BYTES = (size_t)(NA + H) * 16 + 16;
  static constexpr size_t SMEM = WARPS * WARP_BYTES;
};

// Sums of one item at phase ps (|ps| = 1), in order over e:
//   v0 = Re S_a, v1 = Im S'_a, v2 = Re S''_a, v3..v5 the same for b,
//   v6, v7, v8 for c, with S_x = sum_e x_e ps^e, S'_x = sum_e e x_e ps^e,
//   S''_x = sum_e e^2 x_e ps^e (a_e for e = 1..2H, b_e and c_e for e <= H).
// Z(e) and Y(e) return the item's sums Z_e, Y_e.
template <int H, typename ZF, typename YF>
__device__ __forceinline__ void eval_sums(wide::ddc ps, const wide::ddc* KE, const wide::ddc* AL,
                                          ZF Z, YF Y, wide::dd (&v)[9]) {
  using namespace wide;
  using W = dd;
#pragma unroll
  for (int i = 0; i < 9; ++i) v[i] = w_zero<W>();
  ddc pw = ps;
  // the next e's sums are loaded one iteration ahead
  float2 zn = Z(1), yn = Y(1);
#pragma unroll 1
  for (int e = 1; e <= 2 * H; ++e) {
    const float2 z = zn;
    const float2 y = yn;
    if (e < 2 * H) zn = Z(e + 1);
    if (e < H) yn = Y(e + 1);
    const ddc zc = mkc(w_off<W>(z.x), w_off<W>(-z.y));  // conj(Z_e)
    const ddc t = c_mul<W>(c_mul<W>(zc, KE[e]), pw);
    v[0] = w_add(v[0], re(t));
    v[1] = w_add(v[1], w_mulf(im(t), (float)e));
    v[2] = w_add(v[2], w_mulf(re(t), (float)(e * e)));
    if (e <= H) {
      const ddc al = AL[e - 1];
      const ddc tb = c_mul<W>(c_mul<W>(al, mkc(w_off<W>(y.x), w_off<W>(-y.y))), pw);
      v[3] = w_add(v[3], re(tb));
      v[4] = w_add(v[4], w_mulf(im(tb), (float)e));
      v[5] = w_add(v[5], w_mulf(re(tb), (float)(e * e)));
      const ddc tc = c_mul<W>(c_mul<W>(al, zc), pw);
      v[6] = w_add(v[6], re(tc));
      v[7] = w_add(v[7], w_mulf(im(tc), (float)e));
      v[8] = w_add(v[8], w_mulf(re(tc), (float)(e * e)));
    }
    pw = c_mul<W>(pw, ps);
  }
}

template <int H, int NGW1>
__global__ void __launch_bounds__(128, 4) eval_kernel(const RootsArgs a) {
  using namespace wide;
  using W = dd;
  using WC = ddc;
  using EC = EvalCfg<H>;
  constexpr int UPW = 32 / NGW1;  // first-kernel work units per warp step
  constexpr float kTwoPiF = 6.283185307179586f;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WC* const KE = reinterpret_cast<WC*>(smem + (size_t)warp * EC::WARP_BYTES);
  WC* const AL = KE + EC::NA;
  float* const SA = reinterpret_cast<float*>(AL + H);  // sum |alpha_n|
  if (a.status[ST_CODE] != DEV_OK) return;

  const bool batched = a.segs != nullptr;
  const int64_t nf = a.nf_dev ? (int64_t)min(*a.nf_dev, a.redo_cap > 0 ? a.redo_cap : *a.nf_dev)
                              : a.nf;
  const int64_t nkb = (nf + NGW1 - 1) / NGW1;
  const bool listed = batched && a.unit_list != nullptr;
  const int64_t nunits = listed ? (int64_t)*a.unit_count : batched ? a.seg_units[a.nseg] : nkb * a.ntpl;
  const int64_t nsteps = (nunits + UPW - 1) / UPW;
  const int64_t nwarps = (int64_t)gridDim.x * EC::WARPS;
  const W twopi = w_of<W>(6.283185307179586476925286766559);

  // segment of unit u (batched): the last s with seg_units[s] <= u
  auto find_seg = [&](int64_t u, int lo) -> int {
    if (u < a.seg_units[lo]) lo = 0;
    if (u < a.seg_units[lo + 1]) return lo;
    int hi = a.nseg;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.seg_units[mid] <= u) lo = mid;
      else hi = mid;
    }
    return lo;
  };

  // the a-posteriori error test's constants
  const bool check_err = a.sum_err > 0.0;
  const float se = (float)a.sum_err, rtol = (float)a.redo_tol;
  unsigned st_redo = 0, st_redo_nc = 0, st_final = 0;
  int cur_tau = -1, seg_hint = 0;
  const double* cur_mom = nullptr;
  W ybar = w_zero<W>(), YY = w_zero<W>();
  float YYr = 0.0f;
#pragma unroll 1
  for (int64_t step = (int64_t)blockIdx.x * EC::WARPS + warp; step < nsteps; step += nwarps) {
    // ---- this lane's item: unit, template, frequency, output slot
    const int64_t uu = step * UPW + lane / NGW1;
    const int j = lane % NGW1;
    bool valid = uu < nunits;
    int seg = 0, tl = 0;
    int64_t kfirst = 0, seg_nf = nf;
    if (valid) {
      if (!batched) {
        tl = (int)(uu / nkb);
        kfirst = (uu % nkb) * NGW1;
      } else {
        const int64_t u = listed ? a.unit_list[uu] : uu;
        seg = find_seg(u, seg_hint);
        seg_hint = seg;
        const int64_t local = u - a.seg_units[seg];
        const int64_t nkb_s = (a.segs[seg].nf + NGW1 - 1) / NGW1;
        tl = (int)(local / nkb_s);
        kfirst = (local % nkb_s) * NGW1;
      }
    }
    const int64_t k = kfirst + j;
    int tau = tl;
    const double* mom = a.moments;
    int64_t base = k, stride = a.nf_pad;
    int Hs = a.Hs;
    if (batched && valid) {
      const RootsSeg& sg = a.segs[seg];
      valid = tl < sg.ntpl;
      tau = sg.tpl_first + (valid ? tl : 0);
      seg_nf = sg.nf;
      mom = a.moments + (size_t)sg.curve * MO_WORDS;
      base = sg.sums_off + k;
      stride = sg.nf_pad;
      Hs = sg.Hs;
    }
    valid = valid && k < seg_nf;
    int64_t col = 0, ridx = 0, ostride = a.out_stride;
    size_t o = 0;
    if (valid) {
      if (!batched) {
        col = a.kmap ? (int64_t)a.kmap[k] : k;
        o = (size_t)a.rows[tau] * a.out_stride + col;
        ridx = col;
      } else {
        const RootsSeg& sg = a.segs[seg];
        col = k;
        const int row = sg.row_first < 0 ? 0 : a.rows[sg.row_first + tl];
        o = (size_t)(sg.out_off + (int64_t)row * sg.nf + col);
        ostride = sg.nf;
        ridx = sg.redo_base + col;
      }
      valid = FTP_DCHECK(a.status, col >= 0 && col < ostride, 21, col, ostride) &&
              FTP_DCHECK(a.status, (int64_t)o < a.out_elems, 22, o, a.out_elems);
    }
    const float2* const sums = reinterpret_cast<const float2*>(a.sums);
    // Z_e (rows 0..2H-1) and Y_e (rows 2 Hs .. 2 Hs + H - 1) of this item
    auto Zl = [&](int e) -> float2 {
      const int64_t off = (int64_t)(e - 1) * stride + base;
      if (!FTP_DCHECK(a.status, off >= 0 && off < a.sums_elems, 11, off, a.sums_elems))
        return make_float2(0.f, 0.f);
      return __ldg(sums + off);
    };
    auto Yl = [&](int e) -> float2 {
      const int64_t off = (int64_t)(2 * Hs + e - 1) * stride + base;
      if (!FTP_DCHECK(a.status, off >= 0 && off < a.sums_elems, 11, off, a.sums_elems))
        return make_float2(0.f, 0.f);
      return __ldg(sums + off);
    };

    // ---- one round per distinct template among the warp's items (normally one)
    unsigned pending = __ballot_sync(0xffffffffu, valid);
#pragma unroll 1
    while (pending) {
      const int t0 = __shfl_sync(0xffffffffu, tau, __ffs(pending) - 1);
      if (t0 != cur_tau) {  // warp-uniform: alpha_n, K_e and sum |alpha_n| of template t0
        // (float-float from the FP64 alpha_n, one conversion each: the FP64 pipe
        // of this GPU is ~75x slower than the FP32 one)
        __syncwarp();
        const double2* al = a.alpha + (size_t)t0 * kMaxH;
        if (lane < H) AL[lane] = mkc(w_of<W>(al[lane].x), w_of<W>(al[lane].y));
        __syncwarp();
        for (int e = lane; e <= 2 * H; e += 32) {
          WC kk = c_zero<W>();
          for (int n = 1; n <= H; ++n) {
            if (e - n >= 1 && e - n <= H) kk = c_add<W>(kk, c_mul<W>(AL[n - 1], AL[e - n - 1]));
            if (n - e >= 1)
              kk = c_add<W>(kk, c_mulf<W>(c_mul<W>(AL[n - 1], c_conj<W>(AL[n - e - 1])), 2.0f));
          }
          KE[e] = kk;
        }
        if (lane == 0) {
          float sa = 0.0f;
          for (int n = 0; n < H; ++n) sa += sqrtf(w_f(c_abs2<W>(AL[n])));
          *SA = sa;
        }
        cur_tau = t0;
        __syncwarp();
      }
      const bool mine = ((pending >> lane) & 1u) && tau == t0;
      pending &= ~__ballot_sync(0xffffffffu, mine);
      if (!mine) continue;

      if (mom != cur_mom) {  // this item's curve: ybar, YY
        ybar = w_of<W>(mom[MO_YBAR]);
        YY = w_of<W>(mom[MO_YY]);
        YYr = (float)mom[MO_YY];
        cur_mom = mom;
      }
      // the first kernel's chosen phase and flag bits
      const float2 bpsi = make_float2((float)a.power[o], (float)a.theta1[o]);
      const unsigned bits = (unsigned)a.theta2[o];
      const bool constant = (bits & 1u) != 0;
      const bool nonconv = (bits & 2u) != 0;
      const bool no_candidate = (bits & 4u) != 0;
      float theta_w = atan2f(bpsi.y, bpsi.x);
      if (theta_w < 0.0f) theta_w += kTwoPiF;
      // psi in float-float, one Newton step onto |psi| = 1
      WC psi = mkc(w_off<W>(bpsi.x), w_off<W>(bpsi.y));
      {
        const W sfac = w_sub(w_of<W>(1.5), w_mulf(c_abs2<W>(psi), 0.5f));
        psi = mkc(w_mul(re(psi), sfac), w_mul(im(psi), sfac));
      }
      // ---- polish and evaluation: MM, YM, Mbar and their theta-derivatives
      //      at psi; one Newton step on g = 2 MM YM' - YM MM' gives dl; P is
      //      stationary, so P at psi differs from P at the corrected phase by
      //      O(dl^2), and theta1, Mbar are carried to it to first order.  A
      //      correction that is not tiny evaluates again at the corrected
      //      phase (pass 1), kept unless it lowers P.
      W MM, YM, Mbar, dl = w_zero<W>(), th1 = w_zero<W>();
      {
        WC pe = psi;
        bool again = false;
        W MM0 = w_zero<W>(), YM0 = w_zero<W>(), Mb0 = w_zero<W>();
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
          W v[9];
          eval_sums<H>(pe, KE, AL, Zl, Yl, v);
          // <M^2> = Q, Mbar and their theta-derivatives; MM = Q - Mbar^2
          const W Mb = w_mulf(v[6], 2.0f);
          const W Q = w_add(re(KE[0]), w_mulf(v[0], 2.0f));
          if (pass == 1) {
            const W MM1 = w_sub(Q, w_mul(Mb, Mb));
            const W YM1 = w_mulf(v[3], 2.0f);
            // P1 >= P0 (1 - 1e-11): YM1^2 MM0 >= YM0^2 MM1 (1 - 1e-11), float-float
            const W lhs = w_mul(w_mul(YM1, YM1), MM0);
            const W rhs = w_mul(w_mul(w_mul(YM0, YM0), MM1), w_of<W>(1.0 - 1e-11));
            if (w_f(MM1) > 0.0f && w_f(w_sub(lhs, rhs)) >= 0.0f) {
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
          // the residual in float-float, the correction in FP32 (|dl| < 0.05)
          if (a.polish_steps > 0 && !constant) {
            const W g = w_sub(w_mulf(w_mul(MM, YMt), 2.0f), w_mul(YM, MMt));
            const W gt =
                w_sub(w_add(w_mul(MMt, YMt), w_mulf(w_mul(MM, YMtt), 2.0f)), w_mul(YM, MMtt));
            const W d = w_off<W>(w_f(g) * fast_rcp(w_f(gt)));
            const float df = w_f(d);
            if (isfinite(df) && fabsf(df) < 0.05f) dl = d;
          }
          if (w_f(MM) > 0.0f) {
            const W q = w_div(YM, MM);
            const float mf = w_f(MM);
            const float dq = (w_f(YMt) * mf - w_f(YM) * w_f(MMt)) * fast_rcp(mf * mf);
            th1 = w_sub(q, w_off<W>(w_f(dl) * dq));
          }
          Mbar = w_sub(Mbar, w_mul(dl, Mbart));
          again = fabsf(w_f(dl)) > 1e-5f;
          if (!again) break;
          // psi e^{-i dl} (cos, sin to dl^5), back onto |psi| = 1
          const W d2 = w_mul(dl, dl);
          const W cs =
              w_sub(w_of<W>(1.0), w_mul(d2, w_sub(w_of<W>(0.5), w_mul(d2, w_of<W>(1.0 / 24.0)))));
          const W sn = w_mul(dl, w_sub(w_of<W>(1.0), w_mul(d2, w_sub(w_of<W>(1.0 / 6.0),
                                                                    w_mul(d2, w_of<W>(1.0 / 120.0))))));
          pe = mkc(w_add(w_mul(re(psi), cs), w_mul(im(psi), sn)),
                   w_sub(w_mul(im(psi), cs), w_mul(re(psi), sn)));
          const W sfac = w_sub(w_of<W>(1.5), w_mulf(c_abs2<W>(pe), 0.5f));
          pe = mkc(w_mul(re(pe), sfac), w_mul(im(pe), sfac));
        }
      }
      W theta = w_sub(w_off<W>(theta_w), dl);
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
      // positive-amplitude mode without an admissible candidate: P = 0
      // (theta2 = 0, theta3 = ybar)
      const bool no_positive =
          a.positive_only && (no_candidate || degenerate || !(w_f(th1) > 0.0f));
      if (no_positive) {
        P = w_zero<W>();
        th1 = w_zero<W>();
        theta = w_zero<W>();
      }
      const W th3 = w_sub(ybar, w_mul(th1, Mbar));

      // ---- a-posteriori error of P from the NFFT sums: |dZ| <= e gives
      //      |dMM| <= 9 e (sum|alpha|)^2 and |dYM| <= 2 e sum|alpha| sqrt(YY)
      bool redo = false;
      if (check_err) {
        if (degenerate) {
          redo = true;
        } else {
          const float sa = *SA;
          const float Pf = w_f(P), Mf = MMf;
          const float dMM = 9.0f * se * sa * sa;
          const float dYM = 2.0f * se * sa * (YYr * fast_rsqrt(YYr));
          const float q = fmaxf(Pf, 0.0f) * fast_rcp(YYr * Mf);
          const float sq = q > 0.0f ? q * fast_rsqrt(q) : 0.0f;
          const float err = Pf * dMM * fast_rcp(Mf) + 2.0f * sq * dYM;
          redo = !(err <= rtol);
        }
      }

      // ---- outputs, flags and the re-solve list
      a.power[o] = w_d(P);
      a.theta1[o] = w_d(th1);
      a.theta2[o] = w_d(theta);
      a.theta3[o] = w_d(th3);
      // a cap hit is final where no re-solve follows
      const bool cap = nonconv && a.list_nonconv;
      st_final += (nonconv && !(a.list_nonconv && a.redo_list)) ? 1 : 0;
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
      } else if (redo) {
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
        a.flags[o] = (uint8_t)f;
      }
    }
  }
  // one atomic per warp for the solver statistics
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    st_redo += __shfl_xor_sync(0xffffffffu, st_redo, off);
    st_redo_nc += __shfl_xor_sync(0xffffffffu, st_redo_nc, off);
    st_final += __shfl_xor_sync(0xffffffffu, st_final, off);
  }
  if (lane == 0 && (st_redo || st_redo_nc || st_final)) {
    atomicAdd(&a.counters[CNT_REDO], (unsigned long long)st_redo);
    atomicAdd(&a.counters[CNT_REDO_NC], (unsigned long long)st_redo_nc);
    atomicAdd(&a.counters[CNT_NC_FINAL], (unsigned long long)st_final);
  }
}

// Host side: the persistent grid of the evaluation kernel (as many CTAs as fit
// on every SM, no more than the work needs).
template <int H, int NGW1>
int launch_eval(const RootsArgs& a, int num_sms, cudaStream_t s) {
  using EC = EvalCfg<H>;
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, eval_kernel<H, NGW1>, EC::WARPS * 32,
                                                      EC::SMEM) != cudaSuccess ||
        b < 1)
      return -2;
    blocks_per_sm = b;
  }
  constexpr int UPW = 32 / NGW1;
  const int64_t nunits =
      a.host_units > 0 ? a.host_units : (a.nf + NGW1 - 1) / NGW1 * a.ntpl;
  const int64_t need = ((nunits + UPW - 1) / UPW + EC::WARPS - 1) / EC::WARPS;
  int64_t grid = (int64_t)num_sms * blocks_per_sm;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  eval_kernel<H, NGW1><<<(unsigned)grid, EC::WARPS * 32, EC::SMEM, s>>>(a);
  return 1;
}

// Both root-stage kernels of the mixed path: the first kernel (groups of G
// lanes per item), then the one-lane-per-item evaluation for the main pass;
// pre-assembled coefficients and the re-solve passes keep the group-wise
// second kernel.
template <int H, int G>
int launch_h_mixed(const RootsArgs& a, int num_sms, cudaStream_t s) {
  if (a.coef_mode || a.resolve_pass || a.slot_curve) return launch_h<float2, float, H, G>(a, num_sms, s);
  if (a.ev_first_start) cudaEventRecord(a.ev_first_start, s);
  const int r = launch_phase<float2, float, H, G, 1>(a, num_sms, s);
  if (r < 0) return r;
  if (a.ev_first_end) cudaEventRecord(a.ev_first_end, s);
  const int r2 = launch_eval<H, 32 / G>(a, num_sms, s);
  return r2 < 0 ? r2 : r + r2;
}

}  // namespace roots
}  // namespace ftp
