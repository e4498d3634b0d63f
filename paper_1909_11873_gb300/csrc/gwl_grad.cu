// gwl_grad.cu -- log-likelihood and its gradient by adjoint accumulation.
//
// With lnL = sum_d Re[K_d Z_d] - <h|h>/2,  Z_d = sum_j G_d,j e^{-2 pi i r_d,j},
// r_d,j = sum_m c_m B_m(f_j) + tau_d f_j, the derivative along a sampled
// coordinate theta_k is
//   d lnL = sum_d Re[dK_d Z_d] + 2 pi [sum_m dc_m A_m + sum_d dtau_d T_d] - d<h|h>/2,
//   y_d,j = Im(K_d G_d,j e^{-2 pi i r_d,j}),
//   A_m = sum_j B_m(f_j) sum_d y_d,j,   T_d = sum_j f_j y_d,j
// (d/dc_m of the phasor is -2 pi i B_m times it, and Re(-i z) = Im z).  K_d is
// known before the bin loop, so the detectors are combined per bin: the loop
// accumulates Z_d (complex), T_d and A_m -- 3 NDET + 8 real sums, one pass
// over the bins with the likelihood's phase arithmetic.  The per-proposal
// derivatives dc_m, dtau_d,
// dK_d, d<h|h> come from the prologue evaluated on a forward-mode tangent type
// whose value is FP64 (GWL_FP64) or a float pair (GWL_MIXED, the likelihood
// prologue's arithmetic) while the tangents are carried in FP64 or FP32.  A
// proposal whose cut falls in its first window is finished in the bin loop;
// the combination kernel takes the others.  The ISCO cut index is held at its
// value: the gradient of the piecewise-smooth lnL.
#include <cmath>
#include <map>
#include <mutex>

#include "gwl_bins.cuh"
#include "gwl_ff.cuh"
#include "gwl_sched.cuh"

namespace gwl {

// The window sums of a proposal: [2d] U_d, [2d + 1] V_d (Z_d = U_d + i V_d),
// [2 NDET + d] T_d, [3 NDET + m] A_m; padded to a multiple of four (16-byte
// vector loads in the combination).
template <int NDET>
struct GradSums {
  static constexpr int n = (3 * NDET + kNBasis + 3) / 4 * 4;
};
static int grad_sums_per_row(int n_det) { return (3 * n_det + kNBasis + 3) / 4 * 4; }

template <class G>
struct PropGrad {
  G dc[kNBasis][11];
  G dtau[kMaxDet][11];
  G dKr[kMaxDet][11], dKi[kMaxDet][11];
  G dhh[11];
};

// ---------------------------------------------------------------- tangent prologue
// The sampled directions are split into groups of tan_group tangents; thread
// t takes row t / ngrp and directions [tan_group g, tan_group (g + 1)),
// g = t % ngrp.  Every thread of a row runs the value path -- FP64 (GWL_FP64)
// or float pairs on the FP32 pipe (GWL_MIXED, as the likelihood's prologue) --
// and the group-0 thread writes the values.  The FP64 path takes four tangents
// per thread (each copy of the value path occupies the narrow FP64 pipe); the
// mixed path's value path is cheap, so it takes one tangent per thread: eleven
// short threads per row instead of three long ones hide the latency of the
// float-pair chains (measured 75 us against 88 us per call on 4096 proposals).
template <bool MIXED>
constexpr int tan_group() { return MIXED ? 1 : 4; }

template <bool MIXED>
__global__ void __launch_bounds__(64) k_prologue_grad(SegInfo s, const double* __restrict__ theta, int64_t B,
                                                       int ngrp, PropMixed* __restrict__ pm, PropF64* __restrict__ pf,
                                                       PropCommon* __restrict__ pc,
                                                       PropGrad<typename std::conditional<MIXED, float, double>::type>* __restrict__ pg,
                                                       int* __restrict__ work, int* __restrict__ hist, int CH) {
  // let the bin loop launch now: its CTAs stage table rows, then wait for this grid to complete
  cudaTriggerProgrammaticLaunchCompletion();
  using G = typename std::conditional<MIXED, float, double>::type;
  using V = typename std::conditional<MIXED, FF, double>::type;
  constexpr int kTanGroup = tan_group<MIXED>();
  using T = Tan<kTanGroup, G, V>;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = t / ngrp;
  const int i0 = (int)(t % ngrp) * kTanGroup;
  const bool lead = i0 == 0;
  int ncut = 0;
  if (p < B) {
    double th[11];
    expand_theta(s, theta + p * s.stride, th);
    const bool ok = physical(th);
    if (!ok) {
      th[0] = 10.0; th[1] = 0.5; th[2] = th[3] = 0.0; th[4] = 100.0;
#pragma unroll
      for (int k = 5; k < 11; ++k) th[k] = 0.0;
    }
    T x[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) x[k] = tan_const<kTanGroup, G, V>(th[k]);
#pragma unroll
    for (int k = 0; k < 11; ++k) {
      const int j = s.param_pos[k] - i0;  // this thread's tangent slot of parameter k, if any
#pragma unroll
      for (int jj = 0; jj < kTanGroup; ++jj)
        if (j == jj) x[k].d[jj] = (G)1;
    }

    const PNCoeffs<T> P = pn_coeffs(x[1], x[2], x[3]);
    const Scale<T> S = mass_scale(x[0], P.eta, x[4], s.amp_scale);
    T c[kNBasis], ccyc;
    basis_coeffs(P, S, c, ccyc);
    ncut = (int)s.M;
    if (s.fcut_mode == 0) ncut = count_bins_le(s, vval(1.0 / (kSix32 * (S.a13.v * S.a13.v * S.a13.v))));
    if (!ok) ncut = 0;
    const Sky<T> k = sky_trig(x[7], x[8], s.gmst);
    T sp, cp;
    sincos(x[6], &sp, &cp);
    const T ci = cos(x[5]);
    T sa, ca;
    k_angle(x[10], ccyc, sa, ca);

    PropGrad<G>& g = pg[p];
    PropCommon cm;
#pragma unroll
    for (int m = 0; m < kNBasis; ++m) {
#pragma unroll
      for (int j = 0; j < kTanGroup; ++j)
        if (i0 + j < 11) g.dc[m][i0 + j] = ok ? c[m].d[j] : (G)0;
      if (lead) {
        if constexpr (MIXED) {
          pm[p].ch[m] = ok ? c[m].v.hi : 0.0f;
          pm[p].cl[m] = ok ? c[m].v.lo : 0.0f;
        } else {
          pf[p].c[m] = ok ? c[m].v : 0.0;
        }
      }
    }
    T hh = tan_const<kTanGroup, G, V>(0.0);
#pragma unroll 1
    for (int d = 0; d < kMaxDet; ++d) {  // rolled: the per-detector tangent code is long
      T tau = tan_const<kTanGroup, G, V>(0.0), Kr = tau, Ki = tau;
      if (d < s.n_det && ok) {
        T Pr, Pi;
        if constexpr (MIXED) {
          tau = delay_vc(x[9], k, s.vtx_c_ff[d]);
          response(k, sp, cp, ci, s.geom_ff[d], Pr, Pi);
        } else {
          const double* gd = s.geom + 9 * d;
          tau = delay(x[9], k, gd);
          response(k, sp, cp, ci, gd, Pr, Pi);
        }
        Kr = S.amp * (Pr * ca - Pi * sa);
        Ki = S.amp * (Pr * sa + Pi * ca);
        if (ncut > 0) {
          const double Hd = s.H[(int64_t)d * s.M + ncut - 1];
          if constexpr (MIXED) hh = hh + (S.amp * S.amp) * (Pr * Pr + Pi * Pi) * ff_from(Hd);
          else hh = hh + (S.amp * S.amp) * (Pr * Pr + Pi * Pi) * Hd;
        }
      }
#pragma unroll
      for (int j = 0; j < kTanGroup; ++j)
        if (i0 + j < 11) {
          g.dtau[d][i0 + j] = tau.d[j];
          g.dKr[d][i0 + j] = Kr.d[j];
          g.dKi[d][i0 + j] = Ki.d[j];
        }
      if (lead) {
        if constexpr (MIXED) {
          pm[p].th[d] = tau.v.hi;
          pm[p].tl[d] = tau.v.lo;
        } else {
          pf[p].tau[d] = tau.v;
        }
      }
      cm.Kr[d] = vval(Kr.v);
      cm.Ki[d] = vval(Ki.v);
    }
#pragma unroll
    for (int j = 0; j < kTanGroup; ++j)
      if (i0 + j < 11) g.dhh[i0 + j] = hh.d[j];
    cm.hh = vval(hh.v);
    cm.ncut = ncut;
    cm.flag = ok ? 0 : 1;
    if (lead) pc[p] = cm;
  }
  hist_last_window(lead ? ncut : 0, CH, hist);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) ncut = max(ncut, __shfl_xor_sync(0xffffffffu, ncut, off));
  if ((threadIdx.x & 31) == 0 && ncut > 0) atomicMax(&work[0], ncut);
}

// The mixed path's tangent prologue in the shape of the likelihood's: a CTA of
// four warps takes 32 rows along N sampled directions (N blockIdx.y, ...,
// N blockIdx.y + N - 1), and its warps play the likelihood prologue's roles on
// tangent values (float-pair value, FP32 tangents along those directions),
// exchanging them through shared memory, so that each warp's chain is one
// role's instead of the whole model's.
//   phase 1: ln(pi Mc T_sun) and the amplitude (warp 0); the PN coefficients
//            and ln eta (warp 1); the sky angles and the delays tau_d (warp 2);
//            psi and iota (warp 3)
//   phase 2: the basis coefficients c_m (warp 0); the antenna patterns
//            (warp 1); K's phase angle (warp 2); the cut and H_d there (warp 3)
//   phase 3: K_d and its <h|h> term on warp d, then <h|h> on warp 0.
// The direction-0 CTAs also write the rows' values (coefficients, delays, K_d,
// <h|h>, cut) and count them in the work counters.
template <int N>
struct ProSmemTan {
  using T = Tan<N, float, FF>;
  T lmc[32], leta[32], amp[32], eta[32];
  T phi[6][32];
  T sky[4][32];
  T ori[3][32];
  T P[2 * kMaxDet][32];
  T ang[2][32];           // sin, cos of K's phase angle
  T hh[kMaxDet][32];      // per-detector <h|h> terms
  double Hc[kMaxDet][32]; // H_d at the cut bin
  int ncut[32];
};

template <int N>
__global__ void __launch_bounds__(128) k_prologue_grad_roles(SegInfo s, const double* __restrict__ theta, int64_t B,
                                                              PropMixed* __restrict__ pm, PropCommon* __restrict__ pc,
                                                              PropGrad<float>* __restrict__ pg, int* __restrict__ work,
                                                              int* __restrict__ hist, int CH) {
  // let the bin loop launch now: its CTAs stage table rows, then wait for this grid to complete
  cudaTriggerProgrammaticLaunchCompletion();
  using T = Tan<N, float, FF>;
  __shared__ ProSmemTan<N> sm;
  const int role = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dir = blockIdx.y * N;  // the first sampled direction whose tangents this CTA carries
  const bool values = dir == 0;
  // tangent j goes to slot dir + j of the row's derivative arrays (slots past
  // the eleventh are not written; those past n_dim carry zero tangents)
  auto slot_ok = [&](int j) { return dir + j < 11; };
  const int64_t p = (int64_t)blockIdx.x * 32 + lane;
  const bool valid = p < B;
  double th[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) th[k] = 1.0;
  if (valid) expand_theta(s, theta + p * s.stride, th);
  const bool ok = valid && physical(th);
  if (!ok) {  // keep every function below on a harmless argument
    th[0] = 10.0; th[1] = 0.5; th[2] = th[3] = 0.0; th[4] = 100.0;
#pragma unroll
    for (int k = 5; k < 11; ++k) th[k] = 0.0;
  }
  auto tan_of = [&](int k) {
    T x = tan_const<N, float, FF>(th[k]);
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (s.param_pos[k] == dir + j) x.d[j] = 1.0f;
    return x;
  };
  PropGrad<float>* g = valid ? pg + p : nullptr;

  // ---- phase 1
  if (role == 0) {
    const T lmc = log(tan_of(0) * (kPi * kTsun));  // ln(pi Mc T_sun)
    sm.lmc[lane] = lmc;
    sm.amp[lane] = exp((lmc - kLnPi) * (5.0 / 6.0)) * (kAmpConst * kC / kMpc * s.amp_scale) / tan_of(4);
  } else if (role == 1) {
    const PNCoeffs<T> P = pn_coeffs(tan_of(1), tan_of(2), tan_of(3));
    sm.leta[lane] = log(P.eta);
    sm.eta[lane] = P.eta;
    sm.phi[0][lane] = P.p2;
    sm.phi[1][lane] = P.p3;
    sm.phi[2][lane] = P.p4;
    sm.phi[3][lane] = P.p5c;
    sm.phi[4][lane] = P.p6c;
    sm.phi[5][lane] = P.p7;
  } else if (role == 2) {
    const Sky<T> k = sky_trig(tan_of(7), tan_of(8), s.gmst);
    sm.sky[0][lane] = k.sl;
    sm.sky[1][lane] = k.cl;
    sm.sky[2][lane] = k.sd;
    sm.sky[3][lane] = k.cd;
    const T tc = tan_of(9);
#pragma unroll 1
    for (int d = 0; d < kMaxDet; ++d) {
      T tau = tan_const<N, float, FF>(0.0);
      if (d < s.n_det && ok) tau = delay_vc(tc, k, s.vtx_c_ff[d]);
      if (valid) {
#pragma unroll
        for (int j = 0; j < N; ++j)
          if (slot_ok(j)) g->dtau[d][dir + j] = tau.d[j];
        if (values) {
          pm[p].th[d] = tau.v.hi;
          pm[p].tl[d] = tau.v.lo;
        }
      }
    }
  } else {
    if (valid && values) prefetch_cut_H(s, th[0], th[1]);  // read on warp 3 in phase 2
    T sp, cp;
    sincos(tan_of(6), &sp, &cp);
    sm.ori[0][lane] = sp;
    sm.ori[1][lane] = cp;
    sm.ori[2][lane] = cos(tan_of(5));
  }
  __syncthreads();

  // ---- phase 2
  if (role == 0) {
    Scale<T> S;
    S.la = sm.lmc[lane] - 0.6 * sm.leta[lane];
    S.a13 = exp(S.la * (1.0 / 3.0));
    S.amp = sm.amp[lane];
    PNCoeffs<T> P;
    P.eta = sm.eta[lane];
    P.p2 = sm.phi[0][lane];
    P.p3 = sm.phi[1][lane];
    P.p4 = sm.phi[2][lane];
    P.p5c = sm.phi[3][lane];
    P.p6c = sm.phi[4][lane];
    P.p7 = sm.phi[5][lane];
    T c[kNBasis], ccyc;
    basis_coeffs(P, S, c, ccyc);
    if (valid) {
#pragma unroll
      for (int m = 0; m < kNBasis; ++m) {
#pragma unroll
        for (int j = 0; j < N; ++j)
          if (slot_ok(j)) g->dc[m][dir + j] = ok ? c[m].d[j] : 0.0f;
        if (values) {
          pm[p].ch[m] = ok ? c[m].v.hi : 0.0f;
          pm[p].cl[m] = ok ? c[m].v.lo : 0.0f;
        }
      }
    }
  } else if (role == 1) {
    Sky<T> k;
    k.sl = sm.sky[0][lane];
    k.cl = sm.sky[1][lane];
    k.sd = sm.sky[2][lane];
    k.cd = sm.sky[3][lane];
    const T sp = sm.ori[0][lane], cp = sm.ori[1][lane], ci = sm.ori[2][lane];
#pragma unroll 1
    for (int d = 0; d < kMaxDet; ++d) {
      T Pr = tan_const<N, float, FF>(0.0), Pi = Pr;
      if (d < s.n_det) response(k, sp, cp, ci, s.geom_ff[d], Pr, Pi);
      sm.P[2 * d][lane] = Pr;
      sm.P[2 * d + 1][lane] = Pi;
    }
  } else if (role == 2) {
    // the same constant-phase cycles as basis_coeffs forms on warp 0
    const T la = sm.lmc[lane] - 0.6 * sm.leta[lane];
    const T ccyc = const_cycles(cycles_pref(sm.eta[lane]), sm.phi[3][lane], la);
    T sa, ca;
    k_angle(tan_of(10), ccyc, sa, ca);
    sm.ang[0][lane] = sa;
    sm.ang[1][lane] = ca;
  } else {
    const T la = sm.lmc[lane] - 0.6 * sm.leta[lane];
    const T a13 = exp(la * (1.0 / 3.0));
    int ncut = (int)s.M;
    if (s.fcut_mode == 0) ncut = count_bins_le(s, vval(1.0 / (kSix32 * (a13.v * a13.v * a13.v))));
    if (!ok) ncut = 0;
    sm.ncut[lane] = ncut;
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) sm.Hc[d][lane] = (d < s.n_det && ncut > 0) ? s.H[(int64_t)d * s.M + ncut - 1] : 0.0;
  }
  __syncthreads();

  // ---- phase 3: detector d on warp d
  const int ncut = sm.ncut[lane];
  if (role < s.n_det) {
    const int d = role;
    T Kr = tan_const<N, float, FF>(0.0), Ki = Kr, hd = Kr;
    if (ok) {
      const T amp = sm.amp[lane], Pr = sm.P[2 * d][lane], Pi = sm.P[2 * d + 1][lane];
      const T sa = sm.ang[0][lane], ca = sm.ang[1][lane];
      Kr = amp * (Pr * ca - Pi * sa);
      Ki = amp * (Pr * sa + Pi * ca);
      if (ncut > 0) hd = (amp * amp) * (Pr * Pr + Pi * Pi) * ff_from(sm.Hc[d][lane]);
    }
    sm.hh[d][lane] = hd;
    if (valid) {
#pragma unroll
      for (int j = 0; j < N; ++j)
        if (slot_ok(j)) {
          g->dKr[d][dir + j] = Kr.d[j];
          g->dKi[d][dir + j] = Ki.d[j];
        }
      if (values) {
        pc[p].Kr[d] = vval(Kr.v);
        pc[p].Ki[d] = vval(Ki.v);
      }
    }
  } else if (role < kMaxDet && valid) {
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (slot_ok(j)) {
        g->dKr[role][dir + j] = 0.0f;
        g->dKi[role][dir + j] = 0.0f;
      }
    if (values) pc[p].Kr[role] = pc[p].Ki[role] = 0.0;
  }
  __syncthreads();
  if (role == 0) {
    T hh = tan_const<N, float, FF>(0.0);
    for (int d = 0; d < s.n_det; ++d) hh = hh + sm.hh[d][lane];  // detector order, as the single-thread form
    if (valid) {
#pragma unroll
      for (int j = 0; j < N; ++j)
        if (slot_ok(j)) g->dhh[dir + j] = hh.d[j];
      if (values) {
        pc[p].hh = vval(hh.v);
        pc[p].ncut = ncut;
        pc[p].flag = ok ? 0 : 1;
      }
    }
    if (values) {
      hist_last_window(valid ? ncut : 0, CH, hist);
      int nm = valid ? ncut : 0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) nm = max(nm, __shfl_xor_sync(0xffffffffu, nm, off));
      if (lane == 0 && nm > 0) atomicMax(&work[0], nm);
    }
  }
}

// ---------------------------------------------------------------- bin loop
struct GradArgs {
  SinCosTab sct;  // the mixed phase's sine/cosine table
  const void* tab;
  int row_elems;
  int64_t M;
  int CH;
  int64_t B;
  int nw_total;
  const PropCommon* pc;
  const void* prop;
  void* partials;  // [B][nw_total][GradSums<NDET>::n]
  int* work;
  const int* hist;    // [w] proposals whose last window is w
  int* status;
  // a proposal whose cut falls in its first window is finished in the bin loop
  const void* pg;     // PropGrad<G>[B]
  double* lnl;        // [B]
  double* grad;       // [B][gstride]: the n_dim source directions first
  int n_dim;
  int gstride;        // doubles per row of grad (and theta)
  // calibration model (instances with CAL only): the window's calibration rows
  // follow its table rows in shared memory (cal_smem elements in)
  const void* cal;
  int cal_row;
  int cal_smem;
  const double* theta;
  int cal_par;        // first calibration parameter of a row of theta
  int nn;             // calibration nodes
  const void* calQ;   // [nn][nn] natural-spline matrix, float (mixed) or double
  void* xpart;        // [B][nw_total][NDET] per-window <h|h> corrections X_d
};

// lnL = sum_d [Re K_d Z_d] - <h|h>/2 and d lnL / d theta_i from the window
// sums: Z(d, 0..1) the data-template sums (U, V), S(k) the sums T_d
// (k = 2 NDET + d) and A_m (k = 3 NDET + m) in working precision.
template <int NDET, class ZF>
__device__ __forceinline__ double grad_lnl(const PropCommon* c, ZF Z) {
  double l = -0.5 * c->hh;
#pragma unroll
  for (int d = 0; d < NDET; ++d) l += c->Kr[d] * Z(d, 0) - c->Ki[d] * Z(d, 1);
  return l;
}
template <int NDET, class G, class ZF, class SF>
__device__ __forceinline__ G grad_dir(const PropCommon* c, const PropGrad<G>& g, int i, ZF Z, SF S) {
  G ph = (G)0;  // the phase part: sum_m dc_m A_m + sum_d dtau_d T_d
#pragma unroll
  for (int m = 0; m < kNBasis; ++m) ph += g.dc[m][i] * S(3 * NDET + m);
  G acc = (G)(-0.5) * g.dhh[i];
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    ph += g.dtau[d][i] * S(2 * NDET + d);
    acc += g.dKr[d][i] * (G)Z(d, 0) - g.dKi[d][i] * (G)Z(d, 1);
  }
  return acc + (G)(2.0 * kPi) * ph;
}

// With CAL, bin j's term of detector d is (1 + dA) G_d,j e^{-2 pi i (r_d,j - dphi)}
// (calibration rows staged at cal_smem, the proposal's node data in nodes)
// and X_d collects the <h|h> correction sum_j dA (2 + dA) dH_d,j.
template <int NDET, bool MIXED, bool CAL, typename Node>
__device__ __forceinline__ void grad_sums(const GradArgs& a, const void* __restrict__ smv, const Node* nodes,
                                          const float2* __restrict__ sct, int64_t p, int j0, int jend, int lane,
                                          typename std::conditional<MIXED, float, double>::type (&S)[GradSums<NDET>::n],
                                          typename std::conditional<MIXED, float, double>::type (&X)[NDET]) {
  using Acc = typename std::conditional<MIXED, float, double>::type;
  constexpr int T0 = 2 * NDET, A0 = 3 * NDET;
#pragma unroll
  for (int k = 0; k < GradSums<NDET>::n; ++k) S[k] = (Acc)0;
#pragma unroll
  for (int d = 0; d < NDET; ++d) X[d] = (Acc)0;
  // the proposal's amplitudes K_d in working precision
  const PropCommon* pcp = a.pc + p;
  Acc kr[NDET], ki[NDET];
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    kr[d] = (Acc)pcp->Kr[d];
    ki[d] = (Acc)pcp->Ki[d];
  }
  if constexpr (MIXED) {
    const float* sm = reinterpret_cast<const float*>(smv);
    const PropMixed* P = reinterpret_cast<const PropMixed*>(a.prop) + p;
    float ch[kNBasis], cl[kNBasis], th[NDET], tl[NDET];
#pragma unroll
    for (int m = 0; m < kNBasis; ++m) {
      ch[m] = P->ch[m];
      cl[m] = P->cl[m];
    }
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      th[d] = P->th[d];
      tl[d] = P->tl[d];
    }
    for (int j = j0 + lane; j < jend; j += 32) {
      float v[RowM<NDET>::n];
      load_row<NDET>(sm + (int64_t)(j - j0) * a.row_elems, v);
      float sn[NDET], cs[NDET];
      CalBin<NDET, float> cb;
      if constexpr (CAL) {
        cal_eval<NDET>(sm + a.cal_smem + (int64_t)(j - j0) * a.cal_row, reinterpret_cast<const float4*>(nodes), cb);
        phase_mixed<NDET, true>(v, ch, cl, th, tl, sn, cs, cb.P, sct);
      } else {
        phase_mixed<NDET, true>(v, ch, cl, th, tl, sn, cs, nullptr, sct);
      }
      float Y = 0.0f;
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        float gr = v[18 + 2 * d], gi = v[19 + 2 * d];
        if constexpr (CAL) {
          const float a1 = 1.0f + cb.A[d];
          gr *= a1;
          gi *= a1;
          X[d] = fmaf(cb.A[d] * (2.0f + cb.A[d]), cb.H[d], X[d]);
        }
        const float uw = fmaf(gr, cs[d], gi * sn[d]);
        const float vw = fmaf(gi, cs[d], -gr * sn[d]);
        S[2 * d] += uw;
        S[2 * d + 1] += vw;
        const float y = fmaf(kr[d], vw, ki[d] * uw);  // Im(K_d (uw + i vw))
        S[T0 + d] = fmaf(y, v[16], S[T0 + d]);
        Y += y;
      }
#pragma unroll
      for (int m = 0; m < kNBasis; ++m) S[A0 + m] = fmaf(Y, v[m], S[A0 + m]);
    }
  } else {
    const double* sm = reinterpret_cast<const double*>(smv);
    const PropF64* P = reinterpret_cast<const PropF64*>(a.prop) + p;
    double c[kNBasis], tau[NDET];
#pragma unroll
    for (int m = 0; m < kNBasis; ++m) c[m] = P->c[m];
#pragma unroll
    for (int d = 0; d < NDET; ++d) tau[d] = P->tau[d];
    for (int j = j0 + lane; j < jend; j += 32) {
      double v[RowD<NDET>::n];
      load_row<NDET>(sm + (int64_t)(j - j0) * a.row_elems, v);
      double sn[NDET], cs[NDET];
      CalBin<NDET, double> cb;
      if constexpr (CAL) {
        cal_eval<NDET>(sm + a.cal_smem + (int64_t)(j - j0) * a.cal_row, reinterpret_cast<const CalNodeD*>(nodes), cb);
        phase_f64<NDET>(v, c, tau, sn, cs, cb.P);
      } else {
        phase_f64<NDET>(v, c, tau, sn, cs);
      }
      double Y = 0.0;
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        double gr = v[9 + 2 * d], gi = v[10 + 2 * d];
        if constexpr (CAL) {
          const double a1 = 1.0 + cb.A[d];
          gr *= a1;
          gi *= a1;
          X[d] = fma(cb.A[d] * (2.0 + cb.A[d]), cb.H[d], X[d]);
        }
        const double uw = fma(gr, cs[d], gi * sn[d]);
        const double vw = fma(gi, cs[d], -gr * sn[d]);
        S[2 * d] += uw;
        S[2 * d + 1] += vw;
        const double y = fma(kr[d], vw, ki[d] * uw);
        S[T0 + d] = fma(y, v[8], S[T0 + d]);
        Y += y;
      }
#pragma unroll
      for (int m = 0; m < kNBasis; ++m) S[A0 + m] = fma(Y, v[m], S[A0 + m]);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < A0 + kNBasis; ++k) S[k] += __shfl_xor_sync(0xffffffffu, S[k], off);
#pragma unroll
    for (int d = 0; d < NDET; ++d)
      if constexpr (CAL) X[d] += __shfl_xor_sync(0xffffffffu, X[d], off);
  }
}

// The calibration model's terms of lnL and of the source directions' derivatives:
// -1/2 sum_d |K_d|^2 X_d and its derivative -sum_d (Kr_d dKr_d + Ki_d dKi_d) X_d.
template <int NDET, class XF>
__device__ __forceinline__ double cal_lnl_term(const PropCommon* c, XF X) {
  double t = 0.0;
#pragma unroll
  for (int d = 0; d < NDET; ++d) t -= 0.5 * (c->Kr[d] * c->Kr[d] + c->Ki[d] * c->Ki[d]) * (double)X(d);
  return t;
}
template <int NDET, class G, class XF>
__device__ __forceinline__ G cal_grad_term(const PropCommon* c, const PropGrad<G>& g, int i, XF X) {
  G t = (G)0;
#pragma unroll
  for (int d = 0; d < NDET; ++d) t -= ((G)c->Kr[d] * g.dKr[d][i] + (G)c->Ki[d] * g.dKi[d][i]) * (G)X(d);
  return t;
}

// One thread: bins [j0, j1) of the table into shared memory (bulk copy
// completing on bar); with CAL the window's calibration rows follow at element
// offset cal_smem, in pairs (a bulk copy moves whole 16-byte units; the table
// has a zero row past the last bin).
template <bool MIXED, bool CAL>
__device__ __forceinline__ void grad_stage(const GradArgs& a, void* sm, int j0, int j1, uint64_t* bar) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  const Elem* tab = reinterpret_cast<const Elem*>(a.tab);
  const uint32_t bytes = (uint32_t)(j1 - j0) * (uint32_t)a.row_elems * (uint32_t)sizeof(Elem);
  uint32_t cbytes = 0;
  if constexpr (CAL) cbytes = (uint32_t)((j1 - j0 + 1) & ~1) * (uint32_t)a.cal_row * (uint32_t)sizeof(Elem);
  mbar_arrive_expect_tx(bar, bytes + cbytes);
  bulk_g2s(sm, tab + (int64_t)j0 * a.row_elems, bytes, bar);
  if constexpr (CAL)
    bulk_g2s(reinterpret_cast<Elem*>(sm) + a.cal_smem, reinterpret_cast<const Elem*>(a.cal) + (int64_t)j0 * a.cal_row,
             cbytes, bar);
}

template <int NDET, bool MIXED, bool CAL>
__global__ void __launch_bounds__(256, 2) k_window_grad(GradArgs a) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  using Node = typename std::conditional<MIXED, float4, CalNodeD>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ __align__(32) Node s_nodes[CAL ? 8 * NDET * kMaxCalNodes : 1];
  Elem* sm = reinterpret_cast<Elem*>(smem_raw);
  const int lane = threadIdx.x & 31;
  Node* nodes = s_nodes + (CAL ? (threadIdx.x >> 5) * NDET * kMaxCalNodes : 0);
  // the mixed phase's sine/cosine table
  __shared__ float2 s_sct[64];
  if (MIXED && threadIdx.x < 64) s_sct[threadIdx.x] = a.sct.v[threadIdx.x];
  // window 0 of the table is copied while the prologue finishes (see k_window)
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    grad_stage<MIXED, CAL>(a, sm, 0, a.CH < a.M ? (int)a.CH : (int)a.M, &bar);
  }
  __syncthreads();
  bool w0_pending = true;
  uint32_t parity = 0;
  cudaGridDependencySynchronize();
  const int maxn = a.work[0];
  int nw = (maxn + a.CH - 1) / a.CH;
  if (nw > a.nw_total) nw = a.nw_total;
  int n_w = 0;
  int w = nw < 1 ? 0 : start_window(a.hist, 0, nw, blockIdx.x, gridDim.x, &n_w);
  for (; w < nw; ++w) {
    const int j0 = w * a.CH;
    int64_t j1l = (int64_t)j0 + a.CH;
    if (j1l > a.M) j1l = a.M;
    if (j1l > maxn) j1l = maxn;
    const int j1 = (int)j1l;  // > j0 because w < nw
    int* ctr = a.work + 1 + w;
    // every warp is done with the previous window; a window whose proposals are all taken is skipped
    const bool drained = __syncthreads_or(threadIdx.x == 0 && __ldcg(ctr) >= a.B);
    if (!drained) {
      if (w0_pending) {
        if (!mbar_wait_bounded(&bar, parity, a.status)) return;
        parity ^= 1u;
        w0_pending = false;
        if (w != 0) __syncthreads();  // every thread has seen the copy land before the barrier is armed again
      }
      if (w != 0) {
        if (threadIdx.x == 0) {
          fence_proxy_async_smem();
          grad_stage<MIXED, CAL>(a, sm, j0, j1, &bar);
        }
        if (!mbar_wait_bounded(&bar, parity, a.status)) return;
        parity ^= 1u;
      }
      drain_window(ctr, a.B, claim_size(a.B, n_w), a.pc, j0, lane, [&](int64_t p, int ncut) {
        Elem S[GradSums<NDET>::n], X[NDET];
        if constexpr (CAL) cal_nodes_fill<NDET, MIXED>(a.theta + p * a.gstride + a.cal_par, a.nn, a.calQ, lane, nodes);
        grad_sums<NDET, MIXED, CAL>(a, sm, nodes, s_sct, p, j0, ncut < j1 ? ncut : j1, lane, S, X);
        if (ncut <= a.CH) {  // the proposal's only window (every lane holds the sums): finish it here
          const PropCommon* c = a.pc + p;
          auto Z = [&](int d, int k) { return (double)S[2 * d + k]; };
          auto Sf = [&](int k) { return S[k]; };
          auto Xf = [&](int d) { return X[d]; };
          if (lane == 0) a.lnl[p] = grad_lnl<NDET>(c, Z) + (CAL ? cal_lnl_term<NDET>(c, Xf) : 0.0);
          if (lane < a.n_dim) {
            const PropGrad<Elem>& g = reinterpret_cast<const PropGrad<Elem>*>(a.pg)[p];
            Elem d = grad_dir<NDET>(c, g, lane, Z, Sf);
            if constexpr (CAL) d += cal_grad_term<NDET>(c, g, lane, Xf);
            a.grad[p * a.gstride + lane] = (double)d;
          }
          return;
        }
        // lanes write the per-window sums cooperatively
        Elem* o = reinterpret_cast<Elem*>(a.partials) + (p * a.nw_total + w) * GradSums<NDET>::n;
#pragma unroll
        for (int k2 = 0; k2 < GradSums<NDET>::n; ++k2)
          if (lane == k2) o[k2] = S[k2];
        if constexpr (CAL) {
          Elem* ox = reinterpret_cast<Elem*>(a.xpart) + (p * a.nw_total + w) * NDET;
#pragma unroll
          for (int d = 0; d < NDET; ++d)
            if (lane == d) ox[d] = X[d];
        }
      });
    }
    n_w -= __ldcg(&a.hist[w]);
  }
  if (w0_pending) mbar_wait_bounded(&bar, parity, a.status);  // no copy may outlive the CTA
}

// ---------------------------------------------------------------- combination
// One window's sums of a proposal, read as 16-byte vectors (each window's
// block starts on a 16-byte boundary: GradSums<NDET>::n is a multiple of four).
template <int N, class G>
__device__ __forceinline__ void load_sums(const G* __restrict__ qw, G (&v)[N]) {
  if constexpr (sizeof(G) == 4) {
    static_assert(N % 4 == 0, "float sums in float4 units");
    const float4* src = reinterpret_cast<const float4*>(qw);
#pragma unroll
    for (int k = 0; k < N / 4; ++k) {
      const float4 x = src[k];
      v[4 * k] = x.x;
      v[4 * k + 1] = x.y;
      v[4 * k + 2] = x.z;
      v[4 * k + 3] = x.w;
    }
  } else {
    static_assert(N % 2 == 0, "double sums in double2 units");
    const double2* src = reinterpret_cast<const double2*>(qw);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const double2 x = src[k];
      v[2 * k] = x.x;
      v[2 * k + 1] = x.y;
    }
  }
}

// Multi-window proposals: a thread per (proposal, direction of the row).  The
// source directions add the windows' sums (Z in FP64, T_d and A_m in working
// precision; with CAL also the X_d corrections); the calibration
// directions add the windows' derivatives of k_cal_moments in window order.
template <int NDET, bool MIXED, bool CAL>
__global__ void k_finalize_grad(const PropCommon* __restrict__ pc,
                                const PropGrad<typename std::conditional<MIXED, float, double>::type>* __restrict__ pg,
                                const void* __restrict__ partials_v, const void* __restrict__ xpart_v,
                                const void* __restrict__ cpart_v, int64_t B, int CH, int nw_total, int n_dim,
                                int gstride, int nq, double* __restrict__ lnl, double* __restrict__ grad) {
  cudaGridDependencySynchronize();
  using G = typename std::conditional<MIXED, float, double>::type;
  // the directions of a proposal are adjacent threads, so their loads of its window sums coincide
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = t / gstride;
  const int i = (int)(t % gstride);
  if (p >= B) return;
  const PropCommon c = pc[p];
  if (c.flag) {
    if (i == 0) lnl[p] = -INFINITY;
    grad[p * gstride + i] = 0.0;
    return;
  }
  const int nwp = (c.ncut + CH - 1) / CH;
  if (nwp == 1) return;  // finished in the bin loops
  if (CAL && i >= n_dim) {  // a calibration direction
    const G* q = reinterpret_cast<const G*>(cpart_v) + (int64_t)p * nw_total * (NDET * nq) + (i - n_dim);
    double s = 0.0;
    for (int w = 0; w < nwp; ++w) s += (double)q[(int64_t)w * (NDET * nq)];
    grad[p * gstride + i] = s;
    return;
  }
  constexpr int N = GradSums<NDET>::n;
  const G* q = reinterpret_cast<const G*>(partials_v) + (int64_t)p * nw_total * N;
  double Z[NDET][2], X[NDET];
  G S[N];
#pragma unroll
  for (int d = 0; d < NDET; ++d) Z[d][0] = Z[d][1] = X[d] = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) S[k] = (G)0;
  for (int w = 0; w < nwp; ++w) {
    G v[N];
    load_sums(q + (int64_t)w * N, v);
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      Z[d][0] += (double)v[2 * d];
      Z[d][1] += (double)v[2 * d + 1];
      if constexpr (CAL) X[d] += (double)reinterpret_cast<const G*>(xpart_v)[((int64_t)p * nw_total + w) * NDET + d];
    }
#pragma unroll
    for (int k = 2 * NDET; k < N; ++k) S[k] += v[k];
  }
  auto Zf = [&](int d, int k) { return Z[d][k]; };
  auto Sf = [&](int k) { return S[k]; };
  auto Xf = [&](int d) { return X[d]; };
  if (i == 0) lnl[p] = grad_lnl<NDET>(&c, Zf) + (CAL ? cal_lnl_term<NDET>(&c, Xf) : 0.0);
  G g = grad_dir<NDET>(&c, pg[p], i, Zf, Sf);
  if constexpr (CAL) g += cal_grad_term<NDET>(&c, pg[p], i, Xf);
  grad[p * gstride + i] = (double)g;
}

// ---------------------------------------------------------------- launchers
// Per-window sums of the bin loop, then (calibration model) the X_d
// corrections and the calibration directions' per-window derivatives.
int64_t calgrad_part_elems(const gwl_ctx* c, int64_t B);
cudaError_t launch_cal_moments(gwl_ctx* c, int64_t B, int* ctr, const int* hist, void* cpart, double* grad,
                               const double* theta, cudaStream_t st);

static int grad_window_of(const gwl_ctx* c) { return c->grad_window > c->M ? (int)c->M : c->grad_window; }
static int64_t grad_sums_bytes(const gwl_ctx* c, int64_t B) {
  const int CH = grad_window_of(c);
  const int64_t nw = (c->M + CH - 1) / CH;
  return B * nw * grad_sums_per_row(c->n_det) *
         (int64_t)(c->opt.precision == GWL_MIXED ? sizeof(float) : sizeof(double));
}
static int64_t grad_x_bytes(const gwl_ctx* c, int64_t B) {
  if (!c->n_cal_nodes) return 0;
  const int CH = grad_window_of(c);
  return B * ((c->M + CH - 1) / CH) * c->n_det * (int64_t)(c->opt.precision == GWL_MIXED ? sizeof(float) : sizeof(double));
}
int64_t grad_partials_bytes(const gwl_ctx* c, int64_t B) {
  const int64_t el = c->opt.precision == GWL_MIXED ? sizeof(float) : sizeof(double);
  const int64_t cp = c->n_cal_nodes ? calgrad_part_elems(c, B) * el : 0;
  return ((grad_sums_bytes(c, B) + 255) & ~255ll) + ((grad_x_bytes(c, B) + 255) & ~255ll) + cp;
}
int64_t prop_grad_bytes(const gwl_ctx* c) {
  return c->opt.precision == GWL_MIXED ? (int64_t)sizeof(PropGrad<float>) : (int64_t)sizeof(PropGrad<double>);
}
int64_t work_needed(const gwl_ctx* c, int64_t B);
int* window_hist(const gwl_ctx* c);
int* calgrad_counters(const gwl_ctx* c, int64_t B);

// Directions per CTA of the role-form tangent prologue, and how many of its
// CTAs an SM holds (from the kernel's registers and shared memory).
constexpr int kRoleTangents = 3;
// resident CTAs of the role form per SM on the context's device (asked once per
// device; the current device is the context's while a call runs)
static int role_ctas_per_sm(int device) {
  static std::mutex mu;
  static std::map<int, int> per_device;
  std::lock_guard<std::mutex> lk(mu);
  auto it = per_device.find(device);
  if (it != per_device.end()) return it->second;
  int k = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_prologue_grad_roles<kRoleTangents>, 128, 0) != cudaSuccess) {
    cudaGetLastError();
    k = 0;
  }
  per_device[device] = k;
  return k;
}

template <int NDET, bool MIXED, bool CAL>
static cudaError_t run_grad(gwl_ctx* c, const double* theta, int64_t B, double* lnl, double* grad, cudaStream_t st) {
  using G = typename std::conditional<MIXED, float, double>::type;
  const int CH = grad_window_of(c);
  const int nw_total = (int)((c->M + CH - 1) / CH);
  cudaError_t e = cudaMemsetAsync(c->d_work, 0, sizeof(int) * (size_t)work_needed(c, B), st);
  if (e != cudaSuccess) return e;
  {
    ProfScope ps(c, GWL_KERNEL_PROLOGUE, st);
    // the role form, three directions per CTA, while its CTAs fit one wave
    // (measured on the 8 s workload, 11-D, gradient call: 27.5 / 35.2 / 37.3 /
    // 48.6 us at B = 256 / 1024 / 2048 / 4096 against 29.3 / 35.0 / 38.5 us
    // with one direction per CTA and 52.2 us with one thread per row and
    // direction at B = 4096); beyond one wave, the one-thread form
    const int64_t role_ctas = (B + 31) / 32 * ((c->opt.n_dim + kRoleTangents - 1) / kRoleTangents);
    if (MIXED && role_ctas <= (int64_t)role_ctas_per_sm(c->device) * c->num_sms) {
      const dim3 grid((unsigned)((B + 31) / 32), (unsigned)((c->opt.n_dim + kRoleTangents - 1) / kRoleTangents));
      k_prologue_grad_roles<kRoleTangents><<<grid, 128, 0, st>>>(c->seg, theta, B, c->d_pm, c->d_pc,
                                                                 reinterpret_cast<PropGrad<float>*>(c->d_pgrad),
                                                                 c->d_work, window_hist(c), CH);
    } else {
      constexpr int kTanGroup = tan_group<MIXED>();
      const int ngrp = (c->opt.n_dim + kTanGroup - 1) / kTanGroup;
      const int64_t nt = B * ngrp;
      k_prologue_grad<MIXED><<<(unsigned)((nt + 63) / 64), 64, 0, st>>>(c->seg, theta, B, ngrp, c->d_pm, c->d_pf,
                                                                            c->d_pc,
                                                                            reinterpret_cast<PropGrad<G>*>(c->d_pgrad),
                                                                            c->d_work, window_hist(c), CH);
    }
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  char* gp = reinterpret_cast<char*>(c->d_gpartials);
  void* xpart = gp + ((grad_sums_bytes(c, B) + 255) & ~255ll);
  void* cpart = reinterpret_cast<char*>(xpart) + ((grad_x_bytes(c, B) + 255) & ~255ll);
  static const SinCosTab sct = make_sincos_tab();
  GradArgs a;
  a.sct = sct;
  a.tab = MIXED ? (const void*)c->d_tab_mixed : (const void*)c->d_tab_f64;
  a.row_elems = MIXED ? c->row_floats : c->row_doubles;
  a.M = c->M;
  a.CH = CH;
  a.B = B;
  a.nw_total = nw_total;
  a.pc = c->d_pc;
  a.prop = MIXED ? (const void*)c->d_pm : (const void*)c->d_pf;
  a.partials = c->d_gpartials;
  a.work = c->d_work;
  a.hist = window_hist(c);
  a.status = c->d_status;
  a.pg = c->d_pgrad;
  a.lnl = lnl;
  a.grad = grad;
  a.n_dim = c->opt.n_dim;
  a.gstride = (int)theta_stride(c);
  int64_t elems = (int64_t)CH * a.row_elems;
  a.cal = nullptr;
  a.cal_row = 0;
  a.cal_smem = (int)elems;
  a.theta = theta;
  a.cal_par = c->opt.n_dim;
  a.nn = c->n_cal_nodes;
  a.calQ = nullptr;
  a.xpart = xpart;
  if (CAL) {
    a.cal = MIXED ? (const void*)c->d_cal_f : (const void*)c->d_cal_d;
    a.cal_row = MIXED ? c->row_cal_f : c->row_cal_d;
    a.calQ = MIXED ? (const void*)c->d_calQ_f : (const void*)c->d_calQ_d;
    elems += (int64_t)(CH + 1) * a.cal_row;  // staged in pairs
  }
  const size_t smem = (size_t)elems * sizeof(G);
  if ((e = raise_smem_limit((const void*)k_window_grad<NDET, MIXED, CAL>, c->device, smem)) != cudaSuccess) return e;
  {
    ProfScope ps(c, GWL_KERNEL_GRAD, st);
    int64_t want = ((B + 7) / 8) * nw_total;
    int grid = c->num_sms * 2;
    if (want < grid) grid = (int)(want > 0 ? want : 1);
    e = launch_pdl(k_window_grad<NDET, MIXED, CAL>, dim3(grid), dim3(256), smem, st, a);
    c->launches++;
    if (e != cudaSuccess) return e;
  }
  if (CAL) {
    e = launch_cal_moments(c, B, calgrad_counters(c, B), window_hist(c), cpart, grad, theta, st);
    if (e != cudaSuccess) return e;
  }
  {
    ProfScope ps(c, GWL_KERNEL_COMBINE, st);
    const int64_t nt = B * a.gstride;
    e = launch_pdl(k_finalize_grad<NDET, MIXED, CAL>, dim3((unsigned)((nt + 63) / 64)), dim3(64), 0, st,
                   (const PropCommon*)c->d_pc, (const PropGrad<G>*)c->d_pgrad, (const void*)c->d_gpartials,
                   (const void*)xpart, (const void*)cpart, B, CH, nw_total, c->opt.n_dim, a.gstride,
                   2 * c->n_cal_nodes, lnl, grad);
    c->launches++;
  }
  return e;
}

template <int NDET>
static cudaError_t run_grad_any(gwl_ctx* c, const double* theta, int64_t B, double* lnl, double* grad,
                                cudaStream_t st) {
  const bool mixed = c->opt.precision == GWL_MIXED;
  if (c->n_cal_nodes)
    return mixed ? run_grad<NDET, true, true>(c, theta, B, lnl, grad, st)
                 : run_grad<NDET, false, true>(c, theta, B, lnl, grad, st);
  return mixed ? run_grad<NDET, true, false>(c, theta, B, lnl, grad, st)
               : run_grad<NDET, false, false>(c, theta, B, lnl, grad, st);
}

cudaError_t launch_grad(gwl_ctx* c, const double* theta, int64_t B, double* lnl, double* grad, cudaStream_t st) {
  switch (c->n_det) {
    case 1: return run_grad_any<1>(c, theta, B, lnl, grad, st);
    case 2: return run_grad_any<2>(c, theta, B, lnl, grad, st);
    case 3: return run_grad_any<3>(c, theta, B, lnl, grad, st);
    default: return run_grad_any<4>(c, theta, B, lnl, grad, st);
  }
}

}  // namespace gwl
