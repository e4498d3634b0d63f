// gwl_lnl.cu -- batched log-likelihood: prologue, windowed bin loop, combination.
//
//   lnL_p = sum_d [ Re K_d,p U_d,p - Im K_d,p V_d,p - 1/2 |K_d,p|^2 H_d[ncut_p - 1] ]
//   U_d,p + i V_d,p = sum_{j < ncut_p} G_d,j e^{-2 pi i r_d,j,p}
//   r_d,j,p = sum_m c_m,p B_m(f_j) + tau_d,p f_j      (cycles)
// which is Eq. 2 of the paper (as the log-likelihood ratio) for the TaylorF2
// template, regrouped so that per bin and detector only the phase, one
// sincos and four multiply-adds remain.
//
// Work decomposition: a clearing kernel zeroes the work counters; a prologue
// kernel turns each parameter row into its coefficients (four warps per 32
// rows); the bins are cut into windows of W bins, and each CTA of the
// persistent bin-loop kernel starts in the window holding its share of the
// work, stages the window's table rows in shared memory with one bulk
// asynchronous copy (cp.async.bulk, completion on an mbarrier, bounded wait),
// and its warps take proposals from the window's atomic counter in claims of
// 1-32, the 32 lanes striding over the window's bins two blocks per iteration.
// Per-lane sums are reduced with warp shuffles.  A proposal whose cut falls in
// its only window is queued in the CTA's shared memory and combined there in
// FP64 at the next window boundary; otherwise each window's warp publishes a
// partial, and the warp that closes the proposal's last window adds them in
// window order (FP64).  The counters only schedule work: no atomics touch the
// sums, so results are deterministic.  The three kernels are chained with
// programmatic dependent launch.
//
// Precision modes:
//   GWL_FP64  -- phase as an FP64 FMA chain, FP64 sincospi, FP64 sums.
//   GWL_MIXED -- phase in float-float arithmetic (about 48-bit significand,
//                built from error-free TwoProduct/TwoSum on the FP32 pipe) at
//                an anchor bin every 32 bins, FP32 basis deltas within the
//                block where its phase excursion is small, exact reduction of
//                the anchor term, FP32 sincos, FP32 per-lane sums over at most
//                W/32 bins, FP32 warp tree, FP64 across windows and for the
//                combination; the prologue too runs in float-float arithmetic
//                (gwl_ff.cuh).  On GB300 the FP64 pipe issues about 2 FMAs per
//                SM per clock against about 128 FP32 FMAs, so float-float is
//                several times cheaper than FP64 at the same precision.
#include <cmath>
#include <type_traits>

#include "gwl_bins.cuh"
#include "gwl_ff.cuh"
#include "gwl_sched.cuh"

namespace gwl {

// ---------------------------------------------------------------- prologue
// 128 threads per CTA, 32 rows.  The FP64 path's work of a row is spread over
// four warps so that more warps keep the (narrow) FP64 pipe busy:
//   phase 1  warp 0: ln(pi Mc T), ln(eta) -> a^{1/3}, amplitude, frequency cut
//            warp 1: PN phase coefficients phi_k (polynomials in eta, spins)
//            warp 2: sky direction -> per-detector delays tau_d
//            warp 3: sin/cos of psi, cos of iota
//   phase 2  warp 0: basis coefficients c_m and the constant PN phase
//            warp 1: antenna patterns -> complex responses P_d
//   phase 3  warp 2: K_d, <h|h>, cut; the batch's largest cut
struct ProSmem {
  double la[32], a13[32], amp[32], ccyc[32];
  double phi[6][32];
  double sky[4][32];  // sin/cos of (ra - gmst), sin/cos of dec
  double ori[3][32];  // sin psi, cos psi, cos iota
  double P[2 * kMaxDet][32];
  int ncut[32];
};

// The FP64 coefficients of rows row0 .. row0+31, computed by four warps (role
// 0..3); `sync` synchronises exactly those four warps.
template <class Sync>
__device__ __forceinline__ void prologue_rows(const SegInfo& s, const double* __restrict__ theta, int64_t B,
                                              int64_t row0, int role, int lane, ProSmem& sm, Sync sync,
                                              PropF64* __restrict__ pf, PropCommon* __restrict__ pc,
                                              int* __restrict__ work, int* __restrict__ hist, int CH,
                                              double* __restrict__ lnl) {
  double (&sh_la)[32] = sm.la;
  double (&sh_a13)[32] = sm.a13;
  double (&sh_amp)[32] = sm.amp;
  double (&sh_ccyc)[32] = sm.ccyc;
  double (&sh_phi)[6][32] = sm.phi;
  double (&sh_sky)[4][32] = sm.sky;
  double (&sh_ori)[3][32] = sm.ori;
  double (&sh_P)[2 * kMaxDet][32] = sm.P;
  int (&sh_ncut)[32] = sm.ncut;
  const int64_t p = row0 + lane;
  const bool valid = p < B;
  double th[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) th[k] = 1.0;
  if (valid) expand_theta(s, theta + p * s.stride, th);
  const bool ok = valid && physical(th);
  if (!ok) {  // keep every transcendental below on a harmless argument
    th[0] = 10.0; th[1] = 0.5; th[2] = th[3] = 0.0; th[4] = 100.0;
#pragma unroll
    for (int k = 5; k < 11; ++k) th[k] = 0.0;
  }
  const double opq = th[1] + 1.0;
  const double eta = th[1] / (opq * opq);

  // ---- phase 1
  if (role == 0) {
    const Scale<double> S = mass_scale(th[0], eta, th[4], s.amp_scale);
    sh_la[lane] = S.la;
    sh_a13[lane] = S.a13;
    sh_amp[lane] = S.amp;
    int ncut = (int)s.M;
    if (s.fcut_mode == 0) ncut = count_bins_le(s, 1.0 / (kSix32 * S.a13 * S.a13 * S.a13));
    sh_ncut[lane] = ok ? ncut : 0;
  } else if (role == 1) {
    const PNCoeffs<double> P = pn_coeffs(th[1], th[2], th[3]);
    sh_phi[0][lane] = P.p2;
    sh_phi[1][lane] = P.p3;
    sh_phi[2][lane] = P.p4;
    sh_phi[3][lane] = P.p5c;
    sh_phi[4][lane] = P.p6c;
    sh_phi[5][lane] = P.p7;
  } else if (role == 2) {
    const Sky<double> k = sky_trig(th[7], th[8], s.gmst);
    sh_sky[0][lane] = k.sl;
    sh_sky[1][lane] = k.cl;
    sh_sky[2][lane] = k.sd;
    sh_sky[3][lane] = k.cd;
    if (valid) {
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        pf[p].tau[d] = (d < s.n_det && ok) ? delay(th[9], k, s.geom + 9 * d) : 0.0;
      }
    }
  } else {
    double sp, cp;
    sincos(th[6], &sp, &cp);
    sh_ori[0][lane] = sp;
    sh_ori[1][lane] = cp;
    sh_ori[2][lane] = cos(th[5]);
  }
  sync();

  // ---- phase 2
  if (role == 0) {
    PNCoeffs<double> P;
    P.eta = eta;
    P.p2 = sh_phi[0][lane];
    P.p3 = sh_phi[1][lane];
    P.p4 = sh_phi[2][lane];
    P.p5c = sh_phi[3][lane];
    P.p6c = sh_phi[4][lane];
    P.p7 = sh_phi[5][lane];
    Scale<double> S;
    S.la = sh_la[lane];
    S.a13 = sh_a13[lane];
    S.amp = sh_amp[lane];
    double c[kNBasis], ccyc;
    basis_coeffs(P, S, c, ccyc);
    sh_ccyc[lane] = ccyc;
    if (valid) {
#pragma unroll
      for (int m = 0; m < kNBasis; ++m) pf[p].c[m] = ok ? c[m] : 0.0;
    }
  } else if (role == 1) {
    Sky<double> k;
    k.sl = sh_sky[0][lane];
    k.cl = sh_sky[1][lane];
    k.sd = sh_sky[2][lane];
    k.cd = sh_sky[3][lane];
    const double sp = sh_ori[0][lane], cp = sh_ori[1][lane], ci = sh_ori[2][lane];
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) {
      double Pr = 0.0, Pi = 0.0;
      if (d < s.n_det) response(k, sp, cp, ci, s.geom + 9 * d, Pr, Pi);
      sh_P[2 * d][lane] = Pr;
      sh_P[2 * d + 1][lane] = Pi;
    }
  }
  sync();
  // the work counters (cleared by the preceding kernel) are touched from here on
  cudaGridDependencySynchronize();

  // ---- phase 3
  if (role == 2) {
    const int ncut = sh_ncut[lane];
    if (valid) {
      PropCommon cm;
      double hh = 0.0;
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) cm.Kr[d] = cm.Ki[d] = 0.0;
      if (ok) {
        const double amp = sh_amp[lane];
        double sa, ca;
        k_angle(th[10], sh_ccyc[lane], sa, ca);
        for (int d = 0; d < s.n_det; ++d) {
          const double Pr = sh_P[2 * d][lane], Pi = sh_P[2 * d + 1][lane];
          cm.Kr[d] = amp * (Pr * ca - Pi * sa);
          cm.Ki[d] = amp * (Pr * sa + Pi * ca);
          if (ncut > 0) hh += amp * amp * (Pr * Pr + Pi * Pi) * s.H[(int64_t)d * s.M + ncut - 1];
        }
      }
      cm.hh = hh;
      cm.ncut = ncut;
      cm.flag = ok ? 0 : 1;
      pc[p] = cm;
      // rows that no bin loop visits: unphysical (-inf) or without an in-band bin (lnL = 0)
      if (lnl && ncut == 0) lnl[p] = ok ? 0.0 : -INFINITY;
    }
    // largest cut of the batch: one atomic per warp
    int nm = valid ? ncut : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nm = max(nm, __shfl_xor_sync(0xffffffffu, nm, off));
    if (lane == 0 && nm > 0) atomicMax(&work[0], nm);
    hist_last_window(valid ? ncut : 0, CH, hist);
  }
}

struct CtaSync {
  __device__ void operator()() const { __syncthreads(); }
};

// The mixed path's prologue: the same quantities, roles and phases in
// float-float arithmetic on the FP32 pipe (gwl_ff.cuh, ~1e-14 relative), so
// that FP64 is left only for reading theta, the cut frequency's bin count and
// the double outputs K_d, <h|h>.  The phase of K_d also gets the float-float
// sine and cosine.
struct ProSmemFF {
  FF lmc[32], leta[32], amp[32], eta[32];
  FF phi[6][32];
  FF sky[4][32];
  FF ori[3][32];
  FF P[2 * kMaxDet][32];
  double Hc[kMaxDet][32];  // H_d at the cut bin
  int ncut[32];
};

__device__ __forceinline__ void prologue_rows_ff(const SegInfo& s, const double* __restrict__ theta, int64_t B,
                                                 int64_t row0, int role, int lane, ProSmemFF& sm,
                                                 PropMixed* __restrict__ pm, PropCommon* __restrict__ pc,
                                                 int* __restrict__ work, int* __restrict__ hist, int CH,
                                                 double* __restrict__ lnl, const Buckets& bk) {
  const int64_t p = row0 + lane;
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

  // ---- phase 1 (the mass scale is split over two warps: ln(pi Mc T_sun) and
  // the amplitude on warp 0, ln eta beside the PN coefficients on warp 1)
  if (role == 0) {
    const FF lmc = log(ff_from(th[0]) * (kPi * kTsun));  // ln(pi Mc T_sun)
    sm.lmc[lane] = lmc;
    sm.amp[lane] = exp((lmc - kLnPi) * (5.0 / 6.0)) * s.amp_c_ff / ff_from(th[4]);
  } else if (role == 1) {
    const PNCoeffs<FF> P = pn_coeffs(ff_from(th[1]), ff_from(th[2]), ff_from(th[3]));
    sm.leta[lane] = log(P.eta);
    sm.eta[lane] = P.eta;
    sm.phi[0][lane] = P.p2;
    sm.phi[1][lane] = P.p3;
    sm.phi[2][lane] = P.p4;
    sm.phi[3][lane] = P.p5c;
    sm.phi[4][lane] = P.p6c;
    sm.phi[5][lane] = P.p7;
  } else if (role == 2) {
    const Sky<FF> k = sky_trig(ff_from(th[7]), ff_from(th[8]), s.gmst);
    sm.sky[0][lane] = k.sl;
    sm.sky[1][lane] = k.cl;
    sm.sky[2][lane] = k.sd;
    sm.sky[3][lane] = k.cd;
    if (valid) {
      const FF tc = ff_from(th[9]);
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        const FF tau = (d < s.n_det && ok) ? delay_vc(tc, k, s.vtx_c_ff[d]) : ff(0.0f);
        pm[p].th[d] = tau.hi;
        pm[p].tl[d] = tau.lo;
      }
    }
  } else {
    if (valid) prefetch_cut_H(s, th[0], th[1]);  // read on warp 3 in phase 2
    FF sp, cp;
    sincos(ff_from(th[6]), &sp, &cp);
    sm.ori[0][lane] = sp;
    sm.ori[1][lane] = cp;
    sm.ori[2][lane] = cos(ff_from(th[5]));
  }
  __syncthreads();

  // ---- phase 2: the basis coefficients (warp 0), the antenna patterns (warp 1),
  // K's phase angle (warp 2, which keeps it for phase 3) and the cut bin with the
  // <h|h> prefix entries there (warp 3: its global loads leave phase 3 free of them)
  FF sa, ca;
  if (role == 0) {
    Scale<FF> S;
    S.la = sm.lmc[lane] - 0.6 * sm.leta[lane];
    S.a13 = exp(S.la * (1.0 / 3.0));
    S.amp = sm.amp[lane];
    PNCoeffs<FF> P;
    P.eta = sm.eta[lane];
    P.p2 = sm.phi[0][lane];
    P.p3 = sm.phi[1][lane];
    P.p4 = sm.phi[2][lane];
    P.p5c = sm.phi[3][lane];
    P.p6c = sm.phi[4][lane];
    P.p7 = sm.phi[5][lane];
    FF c[kNBasis], ccyc;
    basis_coeffs(P, S, c, ccyc);
    if (valid) {
#pragma unroll
      for (int m = 0; m < kNBasis; ++m) {
        pm[p].ch[m] = ok ? c[m].hi : 0.0f;
        pm[p].cl[m] = ok ? c[m].lo : 0.0f;
      }
    }
  } else if (role == 1) {
    Sky<FF> k;
    k.sl = sm.sky[0][lane];
    k.cl = sm.sky[1][lane];
    k.sd = sm.sky[2][lane];
    k.cd = sm.sky[3][lane];
    const FF sp = sm.ori[0][lane], cp = sm.ori[1][lane], ci = sm.ori[2][lane];
#pragma unroll 1
    for (int d = 0; d < kMaxDet; ++d) {
      FF Pr = ff(0.0f), Pi = ff(0.0f);
      if (d < s.n_det) response(k, sp, cp, ci, s.geom_ff[d], Pr, Pi);
      sm.P[2 * d][lane] = Pr;
      sm.P[2 * d + 1][lane] = Pi;
    }
  } else if (role == 2) {
    // the same constant-phase cycles as basis_coeffs forms on warp 0
    const FF la = sm.lmc[lane] - 0.6 * sm.leta[lane];
    const FF ccyc = const_cycles(cycles_pref(sm.eta[lane]), sm.phi[3][lane], la);
    sincos(ff_from(th[10]) + 0.25 * kPi - (2.0 * kPi) * frac_near(ccyc), &sa, &ca);
  } else {
    const FF la = sm.lmc[lane] - 0.6 * sm.leta[lane];
    const FF a13 = exp(la * (1.0 / 3.0));
    int ncut = (int)s.M;
    if (s.fcut_mode == 0) ncut = count_bins_le(s, ff_to_double(1.0 / (kSix32 * (a13 * a13 * a13))));
    if (!ok) ncut = 0;
    sm.ncut[lane] = ncut;
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) sm.Hc[d][lane] = (d < s.n_det && ncut > 0) ? s.H[(int64_t)d * s.M + ncut - 1] : 0.0;
  }
  __syncthreads();
  // the work counters (cleared by the preceding kernel) are touched from here on
  cudaGridDependencySynchronize();

  // ---- phase 3
  if (role == 2) {
    const int ncut = sm.ncut[lane];
    if (valid) {
      PropCommon cm;
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) cm.Kr[d] = cm.Ki[d] = 0.0;
      FF hh = ff(0.0f);
      if (ok) {
        const FF amp = sm.amp[lane];
        for (int d = 0; d < s.n_det; ++d) {
          const FF Pr = sm.P[2 * d][lane], Pi = sm.P[2 * d + 1][lane];
          const FF kr = amp * (Pr * ca - Pi * sa), ki = amp * (Pr * sa + Pi * ca);
          cm.Kr[d] = ff_to_double(kr);
          cm.Ki[d] = ff_to_double(ki);
          hh = hh + (kr * kr + ki * ki) * ff_from(sm.Hc[d][lane]);
        }
      }
      cm.hh = ff_to_double(hh);
      cm.ncut = ncut;
      cm.flag = ok ? 0 : 1;
      pc[p] = cm;
      // rows that no bin loop visits: unphysical (-inf) or without an in-band bin (lnL = 0)
      if (lnl && ncut == 0) lnl[p] = ok ? 0.0 : -INFINITY;
    }
    // largest cut of the batch: one atomic per warp
    int nm = valid ? ncut : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nm = max(nm, __shfl_xor_sync(0xffffffffu, nm, off));
    if (lane == 0 && nm > 0) atomicMax(&work[0], nm);
    hist_last_window(valid ? ncut : 0, CH, hist);
    if (bk.count) bucket_push(valid ? ncut : 0, p, bk, B);
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(128) k_prologue(SegInfo s, const double* __restrict__ theta, int64_t B,
                                                  PropMixed* __restrict__ pm, PropF64* __restrict__ pf,
                                                  PropCommon* __restrict__ pc, int* __restrict__ work,
                                                  int* __restrict__ hist, int CH, double* __restrict__ lnl,
                                                  Buckets bk) {
  // let the bin loop launch now: its CTAs stage table rows, then wait for this grid to complete
  cudaTriggerProgrammaticLaunchCompletion();
  if constexpr (MIXED) {
    __shared__ ProSmemFF sm;
    prologue_rows_ff(s, theta, B, (int64_t)blockIdx.x * 32, threadIdx.x >> 5, threadIdx.x & 31, sm, pm, pc, work,
                     hist, CH, lnl, bk);
  } else {
    __shared__ ProSmem sm;
    prologue_rows(s, theta, B, (int64_t)blockIdx.x * 32, threadIdx.x >> 5, threadIdx.x & 31, sm, CtaSync(), pf, pc,
                  work, hist, CH, lnl);
  }
}

// ---------------------------------------------------------------- windowed bin loop
struct WinArgs {
  const void* tab;
  int row_elems;  // floats (mixed) or doubles (fp64) per row, padded
  int64_t M;
  int CH;         // bins per window
  int64_t B;
  int nw_total;   // ceil(M / CH)
  const PropCommon* pc;
  const void* prop;  // PropMixed* or PropF64*
  void* partials;    // [B][nw_total][S NDET] float (mixed) or double (fp64), S = 2 (3 with calibration)
  int* work;         // [0] largest cut, [1 + w] proposal counter of window w
  const int* hist;   // [w] proposals whose last window is w
  const float* anchor;  // mixed: anchor rows, one per kAnchor bins
  float df;          // bin spacing [Hz]
  int* pdone;        // [p] windows of proposal p already summed
  double* lnl;       // [B] output
  int* status;       // latched error bits
  // calibration model (instances with CAL only)
  const void* cal;       // [M][cal_row] calibration rows, float (mixed) or double
  int cal_row;           // elements per calibration row
  int cal_smem;          // offset of the window's calibration rows in shared memory (elements)
  const double* theta;   // [B][stride] parameter rows
  int64_t stride;        // doubles per row of theta
  int cal_par;           // first calibration parameter of a row
  int nn;                // calibration nodes
  const void* calQ;      // [nn][nn] natural-spline matrix m = Q y, float (mixed) or double
  unsigned long long* ffc;  // diagnostic counter of float-float-delta blocks, or null
};

// lnL_p = sum_d [Re K_d U_d - Im K_d V_d - |K_d|^2 X_d / 2] - <h|h>/2 (FP64),
// U_d + i V_d the proposal's data-template sums over all its windows and X_d
// the calibration's <h|h> correction (CAL only).  Warp-level: lane d
// (d < NDET) forms detector d's term and a fixed shuffle tree adds them, so
// the FP64 pipe sees a handful of warp instructions per proposal; the result
// is valid on lane 0.
template <int NDET, bool CAL, typename T>
__device__ __forceinline__ double combine_lnl(const PropCommon* __restrict__ c, const T (&U)[NDET],
                                              const T (&V)[NDET], const T (&X)[NDET], int lane) {
  static_assert(NDET <= 4, "at most four detectors");
  T u = (T)0, v = (T)0, x = (T)0;
#pragma unroll
  for (int d = 0; d < NDET; ++d)
    if (lane == d) {
      u = U[d];
      v = V[d];
      if (CAL) x = X[d];
    }
  double t = 0.0;
  if (lane < NDET) {
    const double kr = c->Kr[lane], ki = c->Ki[lane];
    t = kr * (double)u - ki * (double)v;
    if (CAL) t -= 0.5 * (kr * kr + ki * ki) * (double)x;
  }
  t += __shfl_down_sync(0xffffffffu, t, 2);
  t += __shfl_down_sync(0xffffffffu, t, 1);
  return t - 0.5 * c->hh;
}

// Node data of proposal p for the warp's calibration splines (cal_nodes_fill).
template <int NDET, bool MIXED, typename Node>
__device__ __forceinline__ void cal_nodes(const WinArgs& a, int64_t p, int lane, Node* __restrict__ nd) {
  cal_nodes_fill<NDET, MIXED>(a.theta + p * a.stride + a.cal_par, a.nn, a.calQ, lane, nd);
}

// The FP64-phase mixed mode (GWL_MIXED_F64PHASE): per bin the FP64 phase
// r_d = sum_m c_m B_m(f_j) + tau_d f_j, reduced exactly modulo one cycle in
// FP64 (r - rint r), narrowed to FP32 for the hardware sine and cosine, and
// FP32 sums.  The window's FP64 rows carry G_d as floats (narrowed once per
// staged window, in place of the FP64 values).
template <int NDET>
__device__ __forceinline__ void f64phase_sums(const double* __restrict__ sm, int row_elems,
                                              const PropF64* __restrict__ P, int j0, int jend, int lane,
                                              float (&U)[NDET], float (&V)[NDET]) {
  double c[kNBasis], tau[NDET];
#pragma unroll
  for (int m = 0; m < kNBasis; ++m) c[m] = P->c[m];
#pragma unroll
  for (int d = 0; d < NDET; ++d) tau[d] = P->tau[d];
#pragma unroll
  for (int d = 0; d < NDET; ++d) U[d] = V[d] = 0.0f;
  for (int j = j0 + lane; j < jend; j += 32) {
    const double* row = sm + (int64_t)(j - j0) * row_elems;
    double v[kNBasis + 1];
#pragma unroll
    for (int m = 0; m < kNBasis + 1; ++m) v[m] = row[m];
    const float* g = reinterpret_cast<const float*>(row + kNBasis + 1);
    double r = c[0] * v[0];
#pragma unroll
    for (int m = 1; m < kNBasis; ++m) r = fma(c[m], v[m], r);
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      double ph = fma(tau[d], v[kNBasis], r);
      ph -= rint(ph);  // exact: |ph - rint ph| <= 1/2
      float sn, cs;
      __sincosf(6.283185307179586f * (float)ph, &sn, &cs);
      const float gr = g[2 * d], gi = g[2 * d + 1];
      U[d] = fmaf(gr, cs, fmaf(gi, sn, U[d]));
      V[d] = fmaf(gi, cs, fmaf(-gr, sn, V[d]));
    }
  }
}

// In place: the staged FP64 rows' G_d (2 NDET doubles after the basis and f)
// narrowed to floats at the start of the same space (all threads of the CTA;
// each row by one thread).
template <int NDET>
__device__ __forceinline__ void narrow_window_g(double* sm, int row_elems, int nrows) {
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
    double* g = sm + (int64_t)r * row_elems + kNBasis + 1;
    float t[2 * NDET];
#pragma unroll
    for (int k = 0; k < 2 * NDET; ++k) t[k] = (float)g[k];
    float* gf = reinterpret_cast<float*>(g);
#pragma unroll
    for (int k = 0; k < 2 * NDET; ++k) gf[k] = t[k];
  }
}

template <int NDET, bool MIXED, bool CAL, bool F64PH, typename Acc, typename Node>
__device__ __forceinline__ void window_sums(const WinArgs& a, const void* __restrict__ smv, const Node* nodes,
                                            int64_t p, int j0, int jend, int lane, Acc (&Ud)[NDET],
                                            Acc (&Vd)[NDET], Acc (&Xd)[NDET]) {
  if constexpr (F64PH) {
    float U[NDET], V[NDET];
    f64phase_sums<NDET>(reinterpret_cast<const double*>(smv), a.row_elems,
                        reinterpret_cast<const PropF64*>(a.prop) + p, j0, jend, lane, U, V);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        U[d] += __shfl_xor_sync(0xffffffffu, U[d], off);
        V[d] += __shfl_xor_sync(0xffffffffu, V[d], off);
      }
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      Ud[d] = U[d];
      Vd[d] = V[d];
      Xd[d] = (Acc)0;
    }
  } else if constexpr (MIXED) {
    float U[NDET], V[NDET], X[NDET];
    // the window's anchor rows follow its delta rows in shared memory, its
    // calibration rows follow the anchor rows
    const float* smf = reinterpret_cast<const float*>(smv);
    const float* sa = smf + (int64_t)a.CH * a.row_elems;
    anchored_sums_cal<NDET, CAL>(smf, a.row_elems, sa, a.df, reinterpret_cast<const PropMixed*>(a.prop) + p, j0,
                                 jend, lane, U, V, smf + a.cal_smem, a.cal_row,
                                 reinterpret_cast<const float4*>(nodes), X, a.ffc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        U[d] += __shfl_xor_sync(0xffffffffu, U[d], off);
        V[d] += __shfl_xor_sync(0xffffffffu, V[d], off);
        if (CAL) X[d] += __shfl_xor_sync(0xffffffffu, X[d], off);
      }
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      Ud[d] = U[d];
      Vd[d] = V[d];
      Xd[d] = CAL ? X[d] : 0.0f;
    }
  } else {
    const double* sm = reinterpret_cast<const double*>(smv);
    const PropF64* P = reinterpret_cast<const PropF64*>(a.prop) + p;
    double c[kNBasis], tau[NDET];
#pragma unroll
    for (int m = 0; m < kNBasis; ++m) c[m] = P->c[m];
#pragma unroll
    for (int d = 0; d < NDET; ++d) tau[d] = P->tau[d];
#pragma unroll
    for (int d = 0; d < NDET; ++d) Ud[d] = Vd[d] = Xd[d] = 0.0;
    for (int j = j0 + lane; j < jend; j += 32) {
      double v[RowD<NDET>::n];
      load_row<NDET>(sm + (int64_t)(j - j0) * a.row_elems, v);
      if constexpr (CAL) {
        CalBin<NDET, double> cb;
        cal_eval<NDET>(sm + a.cal_smem + (int64_t)(j - j0) * a.cal_row, reinterpret_cast<const CalNodeD*>(nodes),
                       cb);
        bin_f64_cal<NDET>(v, c, tau, cb, Ud, Vd, Xd);
      } else {
        bin_f64<NDET>(v, c, tau, Ud, Vd);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        Ud[d] += __shfl_xor_sync(0xffffffffu, Ud[d], off);
        Vd[d] += __shfl_xor_sync(0xffffffffu, Vd[d], off);
        if (CAL) Xd[d] += __shfl_xor_sync(0xffffffffu, Xd[d], off);
      }
  }
}

// Proposals whose only window a CTA has summed wait in shared memory and are
// combined by all the CTA's threads together at the next window boundary: an
// FP64 warp instruction costs the pipe the same whether one lane or 32 are
// active, so one proposal per lane keeps the FP64 work off the bin loop.
template <int NDET, typename Acc, bool CAL>
struct Pending {
  int64_t p;
  Acc U[NDET], V[NDET], X[CAL ? NDET : 1];
};
constexpr int kPendCap = 128;

// All threads of the CTA, after a CTA barrier: lnL of the waiting proposals.
template <int NDET, typename Acc, bool CAL>
__device__ __forceinline__ void flush_pending(const Pending<NDET, Acc, CAL>* pend, int* npend,
                                              const PropCommon* __restrict__ pc, double* __restrict__ lnl) {
  const int n = *npend < kPendCap ? *npend : kPendCap;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const Pending<NDET, Acc, CAL>& q = pend[e];
    const PropCommon* c = pc + q.p;
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      const double kr = c->Kr[d], ki = c->Ki[d];
      acc += kr * (double)q.U[d] - ki * (double)q.V[d];
      if constexpr (CAL) acc -= 0.5 * (kr * kr + ki * ki) * (double)q.X[d];
    }
    lnl[q.p] = acc - 0.5 * c->hh;
  }
  __syncthreads();
  if (threadIdx.x == 0) *npend = 0;
  __syncthreads();
}

// One thread: copy bins [j0, j1) of the table into shared memory (bulk copy
// completing on bar); in the mixed path the window's anchor rows follow the
// delta rows (after CH rows); with calibration the window's calibration rows
// follow at element offset cal_smem.
template <bool MIXED, bool CAL>
__device__ __forceinline__ void stage_window(const WinArgs& a, void* sm, int j0, int j1, uint64_t* bar) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  const Elem* tab = reinterpret_cast<const Elem*>(a.tab);
  const uint32_t bytes = (uint32_t)(j1 - j0) * (uint32_t)a.row_elems * (uint32_t)sizeof(Elem);
  uint32_t abytes = 0, cbytes = 0;
  int a0 = 0;
  if constexpr (MIXED) {
    a0 = j0 / kAnchor;
    const int a1 = (j1 + kAnchor - 1) / kAnchor;
    abytes = (uint32_t)(a1 - a0) * (uint32_t)(kAnchorRowFloats * sizeof(float));
  }
  // calibration rows in pairs: a bulk copy moves whole 16-byte units (the table has a row past the last bin)
  if constexpr (CAL) cbytes = (uint32_t)((j1 - j0 + 1) & ~1) * (uint32_t)a.cal_row * (uint32_t)sizeof(Elem);
  mbar_arrive_expect_tx(bar, bytes + abytes + cbytes);
  bulk_g2s(sm, tab + (int64_t)j0 * a.row_elems, bytes, bar);
  if constexpr (MIXED)
    bulk_g2s(reinterpret_cast<float*>(sm) + (int64_t)a.CH * a.row_elems, a.anchor + (int64_t)a0 * kAnchorRowFloats,
             abytes, bar);
  if constexpr (CAL)
    bulk_g2s(reinterpret_cast<Elem*>(sm) + a.cal_smem,
             reinterpret_cast<const Elem*>(a.cal) + (int64_t)j0 * a.cal_row, cbytes, bar);
}

template <int NDET, bool MIXED, bool CAL, bool F64PH = false>
__global__ void __launch_bounds__(256, 2) k_window(WinArgs a) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  using Node = typename std::conditional<MIXED, float4, CalNodeD>::type;
  constexpr int S = CAL ? 3 : 2;  // sums per detector in a partial
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  Elem* sm = reinterpret_cast<Elem*>(smem_raw);
  const int lane = threadIdx.x & 31;
  // per-window partial sums: FP32 (mixed, FP64-phase mixed) or FP64
  using Acc = typename std::conditional<MIXED || F64PH, float, double>::type;
  __shared__ Pending<NDET, Acc, CAL> s_pend[kPendCap];
  __shared__ int s_npend;
  __shared__ __align__(32) Node s_nodes[CAL ? 8 * NDET * kMaxCalNodes : 1];
  Node* nodes = s_nodes + (CAL ? (threadIdx.x >> 5) * NDET * kMaxCalNodes : 0);

  // Window 0 of the table does not depend on the prologue: its copy starts
  // before the wait (the prologue lets this grid launch early), and most CTAs
  // start there.  A CTA that starts elsewhere retires the copy first.
  if (threadIdx.x == 0) {
    s_npend = 0;
    mbar_init(&bar, 1);
    fence_mbar_init();
    stage_window<MIXED, CAL>(a, sm, 0, a.CH < a.M ? (int)a.CH : (int)a.M, &bar);
  }
  bool w0_pending = true;  // the copy of window 0 (phase 0 of the barrier) is in flight
  uint32_t parity = 0;
  cudaGridDependencySynchronize();  // the prologue's outputs are visible past this point

  // Each warp takes its first claim in window 0 at once (the window's rows are
  // being staged already), so that the claim's round trip overlaps the reads
  // that place the CTA among the windows instead of following them.  That
  // claim takes two proposals where the window holds more than two per warp;
  // the later claims hold about one active proposal each, which shortens the
  // tail of the last claims.
  const int64_t b_cap = a.B < 0x7fffffff ? a.B : 0x7fffffff;
  const int chunk0 = claim_size(a.B, (int)b_cap);
  int first = 0;
  if (lane == 0) first = atomicAdd(a.work + 1, chunk0);
  const int maxn = a.work[0];
  int nw = (maxn + a.CH - 1) / a.CH;
  if (nw > a.nw_total) nw = a.nw_total;
  // one window: every CTA works in it, on all the proposals
  int n_w = (int)b_cap;
  int w = nw > 1 ? start_window(a.hist, 0, nw, blockIdx.x, gridDim.x, &n_w) : 0;
  auto window_end = [&](int ww) {
    int64_t e = (int64_t)ww * a.CH + a.CH;
    if (e > a.M) e = a.M;
    if (e > maxn) e = maxn;
    return (int)e;
  };

  // the proposal body of the drain: sums over [j0, j1) of window ww, then the
  // combination (a proposal with one window) or the window's partial sums
  auto body = [&](int ww, int j0, int j1, int64_t p, int ncut) {
    Acc U[NDET], V[NDET], X[NDET];
    if constexpr (CAL) cal_nodes<NDET, MIXED>(a, p, lane, nodes);
    window_sums<NDET, MIXED, CAL, F64PH>(a, sm, nodes, p, j0, ncut < j1 ? ncut : j1, lane, U, V, X);
    const int nwp = (ncut + a.CH - 1) / a.CH;
    if (nwp == 1) {  // the proposal's only window: queue it for the CTA's next combination
      int slot = 0;
      if (lane == 0) slot = atomicAdd(&s_npend, 1);
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (slot < kPendCap) {
        if (lane == 0) {
          s_pend[slot].p = p;
#pragma unroll
          for (int d = 0; d < NDET; ++d) {
            s_pend[slot].U[d] = U[d];
            s_pend[slot].V[d] = V[d];
            if constexpr (CAL) s_pend[slot].X[d] = X[d];
          }
        }
      } else {  // queue full: combine here
        const double l = combine_lnl<NDET, CAL>(a.pc + p, U, V, X, lane);
        if (lane == 0) a.lnl[p] = l;
      }
      return;
    }
    // several windows: publish this one; the warp that closes the last one combines
    int done = 0;
    if (lane == 0) {
      Acc* o = reinterpret_cast<Acc*>(a.partials) + (p * a.nw_total + ww) * (S * NDET);
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        o[S * d] = U[d];
        o[S * d + 1] = V[d];
        if constexpr (CAL) o[S * d + 2] = X[d];
      }
      __threadfence();
      done = atomicAdd(&a.pdone[p], 1);
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done != nwp - 1) return;
    __threadfence();
    // lanes take windows lane, lane + 32, ...; a fixed shuffle tree then sums
    // the lanes (FP64, the same order whichever warp closes the proposal)
    const Acc* q = reinterpret_cast<const Acc*>(a.partials) + p * a.nw_total * (S * NDET);
    double Ud[NDET], Vd[NDET], Xd[NDET];
#pragma unroll
    for (int d = 0; d < NDET; ++d) Ud[d] = Vd[d] = Xd[d] = 0.0;
    for (int v = lane; v < nwp; v += 32)
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        Ud[d] += (double)__ldcg(&q[v * (S * NDET) + S * d]);
        Vd[d] += (double)__ldcg(&q[v * (S * NDET) + S * d + 1]);
        if constexpr (CAL) Xd[d] += (double)__ldcg(&q[v * (S * NDET) + S * d + 2]);
      }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        Ud[d] += __shfl_xor_sync(0xffffffffu, Ud[d], off);
        Vd[d] += __shfl_xor_sync(0xffffffffu, Vd[d], off);
        if constexpr (CAL) Xd[d] += __shfl_xor_sync(0xffffffffu, Xd[d], off);
      }
    const double l = combine_lnl<NDET, CAL>(a.pc + p, Ud, Vd, Xd, lane);
    if (lane == 0) a.lnl[p] = l;
  };

  // window 0's copy: let it land (and, on the FP64-phase arm, narrow its G)
  auto window0_ready = [&](int j1) {
    if (!mbar_wait_bounded(&bar, parity, a.status)) return false;
    parity ^= 1u;
    w0_pending = false;
    if constexpr (F64PH) {
      narrow_window_g<NDET>(reinterpret_cast<double*>(sm), a.row_elems, j1);
      __syncthreads();
    }
    return true;
  };

  bool have_first = nw >= 1;
  if (have_first && w != 0) {
    // this CTA starts in a later window: its first claims (window 0) are summed first
    const int j1 = window_end(0);
    if (!window0_ready(j1)) return;
    drain_window(a.work + 1, a.B, chunk0, a.pc, 0, lane,
                 [&](int64_t p, int ncut) { body(0, 0, j1, p, ncut); }, first, chunk0, true);
    have_first = false;
  }

  for (; w < nw; ++w) {
    const int j0 = w * a.CH;
    const int j1 = window_end(w);  // > j0 because w < nw
    int* ctr = a.work + 1 + w;
    const bool use_first = have_first && w == 0;  // the same in every thread of the CTA
    // every warp is done with the previous window; a window whose proposals are
    // all taken is skipped (not checked where the warps hold a claim in it)
    const bool drained = use_first ? false : __syncthreads_or(threadIdx.x == 0 && __ldcg(ctr) >= a.B);
    if (s_npend > 0) flush_pending<NDET, Acc, CAL>(s_pend, &s_npend, a.pc, a.lnl);
    if (!drained) {
      if (w0_pending) {  // window 0's copy: use it, or let it land before staging another window
        if (!window0_ready(w == 0 ? j1 - j0 : window_end(0))) return;
        if (w != 0) __syncthreads();  // every thread has seen the copy land before the barrier is armed again
      }
      if (w != 0) {
        if (threadIdx.x == 0) {
          fence_proxy_async_smem();
          stage_window<MIXED, CAL>(a, sm, j0, j1, &bar);
        }
        if (!mbar_wait_bounded(&bar, parity, a.status)) return;
        parity ^= 1u;
        if constexpr (F64PH) {
          narrow_window_g<NDET>(reinterpret_cast<double*>(sm), a.row_elems, j1 - j0);
          __syncthreads();
        }
      }
      drain_window(ctr, a.B, claim_size(a.B, n_w, false), a.pc, j0, lane,
                   [&](int64_t p, int ncut) { body(w, j0, j1, p, ncut); }, first, use_first ? chunk0 : 0);
    }
    have_first = false;
    n_w -= __ldcg(&a.hist[w]);
  }
  __syncthreads();
  if (s_npend > 0) flush_pending<NDET, Acc, CAL>(s_pend, &s_npend, a.pc, a.lnl);
  if (w0_pending) mbar_wait_bounded(&bar, parity, a.status);  // no copy may outlive the CTA
}


// ---------------------------------------------------------------- waveform (FP64)
__global__ void k_waveform(SegInfo s, const PropF64* __restrict__ pf, const PropCommon* __restrict__ pc,
                           const double* __restrict__ tab, int row_d, double* __restrict__ h) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = blockIdx.y;
  if (j >= s.M) return;
  const PropCommon c = pc[p];
  double* out = h + (int64_t)p * s.n_det * s.M * 2;
  if (c.flag || j >= c.ncut) {
    for (int d = 0; d < s.n_det; ++d) out[2 * ((int64_t)d * s.M + j)] = out[2 * ((int64_t)d * s.M + j) + 1] = 0.0;
    return;
  }
  const double* row = tab + j * row_d;
  const double f = row[8];
  double r = 0.0;
  for (int m = 0; m < kNBasis; ++m) r = fma(pf[p].c[m], row[m], r);
  const double x = f * s.t_ref;
  const double fref = x - floor(x);
  const double f76 = pow(f, -7.0 / 6.0) / s.amp_scale;  // K carries the table normalisation
  for (int d = 0; d < s.n_det; ++d) {
    double ph = fma(pf[p].tau[d], f, r);
    ph -= rint(ph);
    ph += fref;
    double sn, cs;
    sincospi(2.0 * ph, &sn, &cs);
    // K_d f^{-7/6} e^{-2 pi i ph}
    out[2 * ((int64_t)d * s.M + j)] = f76 * (c.Kr[d] * cs + c.Ki[d] * sn);
    out[2 * ((int64_t)d * s.M + j) + 1] = f76 * (c.Ki[d] * cs - c.Kr[d] * sn);
  }
}

// ---------------------------------------------------------------- launchers
static int window_of(const gwl_ctx* c, int precision) {
  (void)precision;
  return c->window > c->M ? (int)c->M : c->window;
}

// Partial sums of either bin loop (in doubles): per (proposal, window) of the
// warp kernel, per (proposal, chunk) of the lane kernel (floats).
int64_t partials_needed(const gwl_ctx* c, int64_t B) {
  const int CH = window_of(c, c->opt.precision);
  const int64_t nw = (c->M + CH - 1) / CH;
  const int64_t warp = B * nw * sums_per_det(c) * c->n_det;
  const int64_t lane = (lanes_slot_floats(c, B) + 1) / 2;
  return warp > lane ? warp : lane;
}

// Windows of the likelihood or the gradient bin loop, whichever has more.
static int64_t nw_max(const gwl_ctx* c) {
  int CH = window_of(c, c->opt.precision);
  const int CHg = c->grad_window > c->M ? (int)c->M : c->grad_window;
  if (CHg < CH) CH = CHg;
  return (c->M + CH - 1) / CH;
}
// [0] largest cut, [1 + w] proposal (or item) counter of window w,
// [1 + nw_max + w] histogram of last windows, [1 + 2 nw_max + p] windows (or
// chunks) of proposal p summed, [1 + 2 nw_max + B + K] bucket counts of the
// lane kernel (chunks of at least 32 bins), then the window counters of the
// calibrated gradient's second bin loop.
int64_t work_needed(const gwl_ctx* c, int64_t B) { return 1 + 3 * nw_max(c) + B + (c->M + 31) / 32; }
int* window_hist(const gwl_ctx* c) { return c->d_work + 1 + nw_max(c); }
int* calgrad_counters(const gwl_ctx* c, int64_t B) { return c->d_work + 1 + 2 * nw_max(c) + B + (c->M + 31) / 32; }

template <int NDET, bool MIXED, bool CAL, bool F64PH = false>
static cudaError_t run_window(gwl_ctx* c, const WinArgs& a, int grid, size_t smem, bool pdl, cudaStream_t st) {
  {
    const cudaError_t e = raise_smem_limit((const void*)k_window<NDET, MIXED, CAL, F64PH>, c->device, smem);
    if (e != cudaSuccess) return e;
  }
  ProfScope ps(c, GWL_KERNEL_BINS, st);
  cudaError_t e;
  if (pdl) {
    e = launch_pdl(k_window<NDET, MIXED, CAL, F64PH>, dim3(grid), dim3(256), smem, st, a);
  } else {
    k_window<NDET, MIXED, CAL, F64PH><<<grid, 256, smem, st>>>(a);
    e = cudaGetLastError();
  }
  c->launches++;
  return e;
}

// Clears the work counters; lets the prologue launch at once (it waits for
// this grid only before its first counter update, in its last phase).  It
// also asks L2 for the batch's parameter rows (one prefetch per 128-byte
// line), so that their fetch from memory is under way while the prologue is
// being launched.
__global__ void k_clear_work(int* __restrict__ work, int64_t n, const double* __restrict__ theta, int64_t lines) {
  cudaTriggerProgrammaticLaunchCompletion();
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  const char* base = reinterpret_cast<const char*>(theta);
  for (int64_t i = t0; i < lines; i += nt) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + 128 * i));
  for (int64_t i = t0; i < n; i += nt) work[i] = 0;
}

static cudaError_t launch_clear_work(gwl_ctx* c, int* work, int64_t n, cudaStream_t st, const double* theta = nullptr,
                                     int64_t theta_bytes = 0) {
  // the rows' 128-byte lines (the first from the line holding theta[0])
  const uintptr_t t = reinterpret_cast<uintptr_t>(theta), tl = t & ~(uintptr_t)127;
  const int64_t lines = theta ? (int64_t)((t + theta_bytes - tl + 127) / 128) : 0;
  const int64_t need = n > lines ? n : lines;
  const unsigned nb = (unsigned)((need + 255) / 256);
  k_clear_work<<<nb < 64 ? nb : 64, 256, 0, st>>>(work, n, reinterpret_cast<const double*>(tl), lines);
  c->launches++;
  return cudaGetLastError();
}

// Prologue of rows [0, B) of theta into the coefficient arrays at row offset
// `off`, with `work` the counter region (cleared just before, by a memset or
// k_clear_work; launched as a programmatic dependent of the latter).
// pdl: a programmatic dependent launch of the clearing kernel before it;
// otherwise an ordinary launch (after a kernel that wrote theta).
static cudaError_t launch_prologue(gwl_ctx* c, const double* theta, int64_t B, int64_t off, int precision,
                                   double* lnl, int* work, cudaStream_t st, Buckets bk = Buckets{nullptr, nullptr, 32},
                                   bool pdl = true) {
  ProfScope ps(c, GWL_KERNEL_PROLOGUE, st);
  const unsigned nb = (unsigned)((B + 31) / 32);
  int* hist = work + 1 + nw_max(c);
  const int CH = window_of(c, precision);
  cudaError_t e;
  if (!pdl) {
    if (precision == GWL_MIXED)
      k_prologue<true><<<nb, 128, 0, st>>>(c->seg, theta, B, c->d_pm + off, c->d_pf + off, c->d_pc + off, work, hist,
                                           CH, lnl, bk);
    else
      k_prologue<false><<<nb, 128, 0, st>>>(c->seg, theta, B, c->d_pm + off, c->d_pf + off, c->d_pc + off, work,
                                            hist, CH, lnl, bk);
    e = cudaGetLastError();
  } else if (precision == GWL_MIXED) {
    e = launch_pdl(k_prologue<true>, dim3(nb), dim3(128), 0, st, c->seg, theta, B, c->d_pm + off, c->d_pf + off,
                   c->d_pc + off, work, hist, CH, lnl, bk);
  } else {
    e = launch_pdl(k_prologue<false>, dim3(nb), dim3(128), 0, st, c->seg, theta, B, c->d_pm + off, c->d_pf + off,
                   c->d_pc + off, work, hist, CH, lnl, bk);
  }
  c->launches++;
  return e;
}

// The bin loop (which also forms lnL) of rows [off, off + B) of the batch.
template <int NDET>
static cudaError_t launch_bins(gwl_ctx* c, const double* theta, int64_t B, int64_t off, double* lnl, int* work,
                               bool pdl, cudaStream_t st) {
  const bool mixed = c->opt.precision == GWL_MIXED;
  const int CH = window_of(c, c->opt.precision);
  const int nw_total = (int)((c->M + CH - 1) / CH);
  WinArgs a;
  a.tab = mixed ? (const void*)c->d_tab_delta : (const void*)c->d_tab_f64;
  a.row_elems = mixed ? c->row_delta : c->row_doubles;
  a.anchor = c->d_anchor;
  a.df = (float)c->df;
  a.M = c->M;
  a.CH = CH;
  a.B = B;
  a.nw_total = nw_total;
  a.pc = c->d_pc + off;
  a.prop = mixed ? (const void*)(c->d_pm + off) : (const void*)(c->d_pf + off);
  const bool cal = c->n_cal_nodes > 0;
  const bool f64ph = c->opt.precision == GWL_MIXED_F64PHASE;
  a.partials = reinterpret_cast<char*>(c->d_partials) +
               off * nw_total * sums_per_det(c) * NDET * (int64_t)(mixed || f64ph ? sizeof(float) : sizeof(double));
  a.work = work;
  a.hist = work + 1 + nw_max(c);
  a.pdone = work + 1 + 2 * nw_max(c);
  a.lnl = lnl;
  a.status = c->d_status;
  a.ffc = c->count_ff ? c->d_ffc : nullptr;
  // shared memory (elements): the window's rows, [mixed] its anchor rows, [calibration] its calibration rows
  int64_t elems = (int64_t)CH * a.row_elems;
  if (mixed) elems += (int64_t)((CH + kAnchor - 1) / kAnchor) * kAnchorRowFloats;
  a.cal = nullptr;
  a.cal_row = 0;
  a.cal_smem = (int)elems;
  a.theta = nullptr;
  a.stride = theta_stride(c);
  a.cal_par = c->opt.n_dim;
  a.nn = c->n_cal_nodes;
  a.calQ = nullptr;
  if (cal) {
    a.cal = mixed ? (const void*)c->d_cal_f : (const void*)c->d_cal_d;
    a.cal_row = mixed ? c->row_cal_f : c->row_cal_d;
    a.theta = theta;
    a.calQ = mixed ? (const void*)c->d_calQ_f : (const void*)c->d_calQ_d;
    elems += (int64_t)(CH + 1) * a.cal_row;  // rows are staged in pairs
  }
  const size_t smem = (size_t)elems * (mixed ? sizeof(float) : sizeof(double));
  // enough CTAs for every warp of a window to find a proposal, at most a full wave
  const int64_t want = ((B + 7) / 8) * nw_total;
  int grid = c->num_sms * c->ctas_per_sm;
  if (want < grid) grid = (int)(want > 0 ? want : 1);
  if (cal)
    return mixed ? run_window<NDET, true, true>(c, a, grid, smem, pdl, st)
                 : run_window<NDET, false, true>(c, a, grid, smem, pdl, st);
  if (f64ph) return run_window<NDET, false, false, true>(c, a, grid, smem, pdl, st);
  return mixed ? run_window<NDET, true, false>(c, a, grid, smem, pdl, st)
               : run_window<NDET, false, false>(c, a, grid, smem, pdl, st);
}

// Prologue (per-proposal coefficients, FP64) then the windowed bin loop, which
// also forms lnL (programmatic dependent launch: its CTAs start while the
// prologue drains and wait for its results).
// With the lane kernel the prologue also files every proposal in the bucket
// of its last chunk.
// cleared: the work counters were cleared by the kernel just before (which
// also wrote theta), so no clearing kernel runs and the prologue is an
// ordinary launch after it.
template <int NDET>
static cudaError_t run_pipeline(gwl_ctx* c, const double* theta, int64_t B, double* lnl, cudaStream_t st,
                                bool cleared = false) {
  const int seg = lanes_seg(c, B);
  int* pdone = c->d_work + 1 + 2 * nw_max(c);
  int* bcount = pdone + B;
  const Buckets bk = seg ? Buckets{bcount, c->d_blist, seg} : Buckets{nullptr, nullptr, 32};
  cudaError_t e = cleared ? cudaSuccess
                          : launch_clear_work(c, c->d_work, work_needed(c, B), st, theta,
                                              B * theta_stride(c) * (int64_t)sizeof(double));
  if (e == cudaSuccess) e = launch_prologue(c, theta, B, 0, c->opt.precision, lnl, c->d_work, st, bk, !cleared);
  if (e != cudaSuccess) return e;
  if (seg) return launch_lanes(c, B, lnl, c->d_work, c->d_work + 1 + nw_max(c), pdone, bcount, seg, st);
  return launch_bins<NDET>(c, theta, B, 0, lnl, c->d_work, true, st);
}

cudaError_t launch_loglike(gwl_ctx* c, const double* theta, int64_t B, double* lnl, cudaStream_t st) {
  switch (c->n_det) {
    case 1: return run_pipeline<1>(c, theta, B, lnl, st);
    case 2: return run_pipeline<2>(c, theta, B, lnl, st);
    case 3: return run_pipeline<3>(c, theta, B, lnl, st);
    default: return run_pipeline<4>(c, theta, B, lnl, st);
  }
}

cudaError_t launch_loglike_cleared(gwl_ctx* c, const double* theta, int64_t B, double* lnl, cudaStream_t st) {
  switch (c->n_det) {
    case 1: return run_pipeline<1>(c, theta, B, lnl, st, true);
    case 2: return run_pipeline<2>(c, theta, B, lnl, st, true);
    case 3: return run_pipeline<3>(c, theta, B, lnl, st, true);
    default: return run_pipeline<4>(c, theta, B, lnl, st, true);
  }
}

cudaError_t launch_waveform(gwl_ctx* c, const double* theta, int64_t B, double* h, cudaStream_t st) {
  // the waveform is always produced in FP64
  cudaError_t e = cudaMemsetAsync(c->d_work, 0, sizeof(int) * (size_t)work_needed(c, B), st);
  if (e == cudaSuccess) e = launch_prologue(c, theta, B, 0, GWL_FP64, nullptr, c->d_work, st);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((c->M + 255) / 256), (unsigned)B);
  k_waveform<<<grid, 256, 0, st>>>(c->seg, c->d_pf, c->d_pc, c->d_tab_f64, c->row_doubles, h);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace gwl
