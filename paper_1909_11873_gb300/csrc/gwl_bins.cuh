// gwl_bins.cuh -- per-bin arithmetic shared by the likelihood and gradient bin loops.
#pragma once

#include <cmath>
#include <type_traits>

#include "gwl_internal.h"

namespace gwl {

// ---------------------------------------------------------------- launch helper
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// ---------------------------------------------------------------- per-bin bodies
// Row element counts actually read (without the trailing pad unit).
template <int NDET> struct RowM { static constexpr int n = (18 + 2 * NDET + 3) / 4 * 4; };
template <int NDET> struct RowD { static constexpr int n = (9 + 2 * NDET + 1) / 2 * 2; };

template <int NDET>
__device__ __forceinline__ void load_row(const float* __restrict__ row, float (&v)[RowM<NDET>::n]) {
#pragma unroll
  for (int k = 0; k < RowM<NDET>::n / 4; ++k)
    *reinterpret_cast<float4*>(&v[4 * k]) = reinterpret_cast<const float4*>(row)[k];
}
template <int NDET>
__device__ __forceinline__ void load_row(const double* __restrict__ row, double (&v)[RowD<NDET>::n]) {
#pragma unroll
  for (int k = 0; k < RowD<NDET>::n / 2; ++k)
    *reinterpret_cast<double2*>(&v[2 * k]) = reinterpret_cast<const double2*>(row)[k];
}

// Nearest integer of x by the 1.5 * 2^23 shift (exact for |x| < 2^22).  The
// shift runs on the FMA pipe, whereas a rounding instruction would occupy the
// narrow conversion pipe.
__device__ __forceinline__ float nearest_int(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}

// Sine and cosine of the 64th-cycle points 2 pi k / 64, k = 0 .. 63, for the
// gradient bin loop's sine and cosine (kernel argument, copied to shared
// memory).  The first quadrant comes from the FP64 library functions, the
// others by symmetry, so that the quarter-turn points are exactly 0 and +-1.
struct SinCosTab {
  float2 v[64];
};
inline SinCosTab make_sincos_tab() {
  SinCosTab t;
  for (int k = 0; k < 64; ++k) {
    const int q = k / 16, m = k % 16;  // k = 16 q + m: angle q pi/2 + m pi/32
    const double sm = m ? std::sin(kPi * m / 32.0) : 0.0, cm = m ? std::cos(kPi * m / 32.0) : 1.0;
    const double s = q == 0 ? sm : q == 1 ? cm : q == 2 ? -sm : -cm;
    const double c = q == 0 ? cm : q == 1 ? -sm : q == 2 ? -cm : sm;
    t.v[k] = make_float2((float)s, (float)c);
  }
  return t;
}

// sin and cos of 2 pi fr (|fr| below about 0.6 cycles) from a table of the
// 64th-cycle points: k the nearest integer to 64 fr (by the 1.5 * 2^23 shift,
// whose low mantissa bits are k mod 64), rho = fr - k/64 (|rho| <= 1/128,
// exact), (sin, cos)(2 pi k/64) = tab[k mod 64], and sin and cos of
// u = 2 pi rho from their Taylor series through u^3 and u^4 (truncation below
// 3e-9 for |u| <= pi/64), then the rotation by the table's angle.
__device__ __forceinline__ void sincos_cycles_tab(float fr, const float2* __restrict__ tab, float* s, float* c) {
  const float t = __fadd_rn(64.0f * fr, 12582912.0f);
  const int k = __float_as_int(t) & 63;
  const float rho = __fmaf_rn(__fsub_rn(t, 12582912.0f), -0.015625f, fr);
  const float u = 6.283185307179586f * rho;
  const float u2 = u * u;
  const float sr = __fmaf_rn(u * u2, -0.16666666666666666f, u);
  const float cr = __fmaf_rn(u2, __fmaf_rn(u2, 0.041666666666666664f, -0.5f), 1.0f);
  const float2 e = tab[k];
  *s = __fmaf_rn(e.x, cr, e.y * sr);
  *c = __fmaf_rn(e.y, cr, -(e.x * sr));
}

// Phase of one bin in float-float arithmetic, reduced modulo one cycle, and its
// sine and cosine: (sn_d, cs_d) = sin/cos 2 pi r_d, r_d = S + tau_d f.
// S = sum_m c_m B_m is summed as an unevaluated float pair (s, lo); tau_d f is
// formed exactly as p + e (p = fl(tau_hi f_hi), e its error plus the cross
// terms).  Two reductions:
//   EXACT_SUM (gradient): t + q = s + p exactly (TwoSum), then
//     r_d mod 1 = (t - rint t) + (lo + e + q): one final rounding of at most
//     2^-25 cycles.
//   otherwise (likelihood): S mod 1 = (s - rint s) + lo once per bin, and per
//     detector r_d mod 1 = (S mod 1) + (p - rint p) + e (s - rint s and
//     p - rint p are exact): two roundings of at most 2^-24 cycles each, and
//     seven fewer FP32 operations per detector.
// With shift (may be null) the phase of detector d is r_d - shift[d] (the
// calibration model's phase correction, in cycles).  EXACT_SUM takes the
// sine/cosine table sct (make_sincos_tab's values, in shared memory).
template <int NDET, bool EXACT_SUM>
__device__ __forceinline__ void phase_mixed(const float (&v)[RowM<NDET>::n], const float (&ch)[kNBasis],
                                            const float (&cl)[kNBasis], const float (&th)[NDET],
                                            const float (&tl)[NDET], float (&sn)[NDET], float (&cs)[NDET],
                                            const float* shift = nullptr, const float2* __restrict__ sct = nullptr) {
  float s, lo;
  if constexpr (EXACT_SUM) {
    // the eight products' high parts summed pairwise (three levels of TwoSum
    // instead of a chain of seven), their errors and the low-part terms in two
    // running sums
    static_assert(kNBasis == 8, "pairwise sum written for eight basis functions");
    float p[kNBasis], l2[2] = {0.0f, 0.0f};
#pragma unroll
    for (int m = 0; m < kNBasis; ++m) {
      float e;
      two_prod(ch[m], v[m], p[m], e);
      l2[m & 1] = __fmaf_rn(ch[m], v[kNBasis + m], __fmaf_rn(cl[m], v[m], l2[m & 1] + e));
    }
    float a[4], qa = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float q;
      two_sum(p[2 * k], p[2 * k + 1], a[k], q);
      qa += q;
    }
    float b0, b1, q0, q1, qc;
    two_sum(a[0], a[1], b0, q0);
    two_sum(a[2], a[3], b1, q1);
    two_sum(b0, b1, s, qc);
    lo = (l2[0] + l2[1]) + (qa + ((q0 + q1) + qc));
  } else {
    {
      float e;
      two_prod(ch[0], v[0], s, e);
      lo = __fmaf_rn(cl[0], v[0], __fmaf_rn(ch[0], v[kNBasis], e));
    }
#pragma unroll
    for (int m = 1; m < kNBasis; ++m) {
      const float bh = v[m], bl = v[kNBasis + m];
      float p, e, t, q;
      two_prod(ch[m], bh, p, e);
      two_sum(s, p, t, q);
      s = t;
      lo = __fmaf_rn(ch[m], bl, __fmaf_rn(cl[m], bh, lo + (q + e)));
    }
  }
  const float fh = v[16], fl = v[17];
  if constexpr (EXACT_SUM) {
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      float p, e, t, q;
      two_prod(th[d], fh, p, e);
      e = __fmaf_rn(th[d], fl, __fmaf_rn(tl[d], fh, e));
      two_sum(s, p, t, q);
      const float l = lo + (e + q);
      float fr = __fadd_rn(__fsub_rn(t, nearest_int(t)), l);  // t - rint t is exact
      if (shift) fr = fr - shift[d];
      // the gradient's basis-weighted sums amplify the absolute error of the
      // hardware sine and cosine (~4e-7, a smooth function of the argument, so
      // it adds up across bins): the table of 64th-cycle points and short
      // series instead (sct, in shared memory)
      sincos_cycles_tab(fr, sct, &sn[d], &cs[d]);
    }
  } else {
    const float sf = __fadd_rn(__fsub_rn(s, nearest_int(s)), lo);
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      float p, e;
      two_prod(th[d], fh, p, e);
      e = __fmaf_rn(th[d], fl, __fmaf_rn(tl[d], fh, e));
      float fr = __fadd_rn(__fadd_rn(sf, __fsub_rn(p, nearest_int(p))), e);
      if (shift) fr = fr - shift[d];
      __sincosf(6.283185307179586f * fr, &sn[d], &cs[d]);
    }
  }
}

template <int NDET>
__device__ __forceinline__ void bin_mixed(const float (&v)[RowM<NDET>::n], const float (&ch)[kNBasis],
                                          const float (&cl)[kNBasis], const float (&th)[NDET],
                                          const float (&tl)[NDET], float (&U)[NDET], float (&V)[NDET]) {
  float sn[NDET], cs[NDET];
  phase_mixed<NDET, false>(v, ch, cl, th, tl, sn, cs);
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    const float gr = v[18 + 2 * d], gi = v[19 + 2 * d];
    // (gr + i gi)(cs - i sn)
    U[d] = fmaf(gr, cs[d], fmaf(gi, sn[d], U[d]));
    V[d] = fmaf(gi, cs[d], fmaf(-gr, sn[d], V[d]));
  }
}

// ---------------------------------------------------------------- calibration model (Section 2.2)
// With calibration the template of detector d at bin j is multiplied by
// (1 + dA_d,j) e^{i dphi_d,j}: with dphi in cycles the bin's term becomes
//   (1 + dA) G_d,j e^{-2 pi i (r_d,j - dphi)},
// and <h|h>_d = |K_d|^2 (H_d[ncut - 1] + X_d) with X_d = sum_j dA (2 + dA) dH_d,j.
// dA and dphi come from the bin's calibration row (spline weights, interval k)
// and the warp's node data of the proposal (see gwl_device.cuh).
template <int NDET, typename T>
struct CalBin {
  T A[NDET], P[NDET], H[NDET];
};

// Spline weights of a bin from its row [t, h^2/6, k, dH_d ...]:
//   (1 - t, t, h^2/6 (1 - t)((1 - t)^2 - 1), h^2/6 t (t^2 - 1)).
template <int NDET, typename T>
__device__ __forceinline__ void cal_weights(const T (&r)[2 * ((3 + NDET + 1) / 2)], T (&w)[4]) {
  const T t = r[0], h6 = r[1], a = (T)1 - t;
  w[0] = a;
  w[1] = t;
  w[2] = h6 * a * fma(a, a, (T)-1);
  w[3] = h6 * t * fma(t, t, (T)-1);
}

template <int NDET>
__device__ __forceinline__ void cal_eval(const float* __restrict__ crow, const float4* __restrict__ nodes,
                                         CalBin<NDET, float>& cb) {
  constexpr int NP = (3 + NDET + 1) / 2;  // 8-byte pairs per row
  float r[2 * NP], w[4];
#pragma unroll
  for (int i = 0; i < NP; ++i) *reinterpret_cast<float2*>(&r[2 * i]) = reinterpret_cast<const float2*>(crow)[i];
  cal_weights<NDET>(r, w);
  const int k = __float_as_int(r[2]);
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    const float4 n0 = nodes[d * kMaxCalNodes + k], n1 = nodes[d * kMaxCalNodes + k + 1];
    cb.A[d] = fmaf(w[0], n0.x, fmaf(w[1], n1.x, fmaf(w[2], n0.y, w[3] * n1.y)));
    cb.P[d] = fmaf(w[0], n0.z, fmaf(w[1], n1.z, fmaf(w[2], n0.w, w[3] * n1.w)));
    cb.H[d] = r[3 + d];
  }
}

template <int NDET>
__device__ __forceinline__ void cal_eval(const double* __restrict__ crow, const CalNodeD* __restrict__ nodes,
                                         CalBin<NDET, double>& cb) {
  constexpr int NP = (3 + NDET + 1) / 2;
  double r[2 * NP], w[4];
#pragma unroll
  for (int i = 0; i < NP; ++i) *reinterpret_cast<double2*>(&r[2 * i]) = reinterpret_cast<const double2*>(crow)[i];
  cal_weights<NDET>(r, w);
  const int k = (int)r[2];
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    const CalNodeD& n0 = nodes[d * kMaxCalNodes + k];
    const CalNodeD& n1 = nodes[d * kMaxCalNodes + k + 1];
    cb.A[d] = fma(w[0], n0.v[0], fma(w[1], n1.v[0], fma(w[2], n0.v[1], w[3] * n1.v[1])));
    cb.P[d] = fma(w[0], n0.v[2], fma(w[1], n1.v[2], fma(w[2], n0.v[3], w[3] * n1.v[3])));
    cb.H[d] = r[3 + d];
  }
}

// One detector's term of a bin: reduced phase fr [cycles], data weight (gr, gi).
template <bool CAL, typename T>
__device__ __forceinline__ void cal_apply(T& fr, T& gr, T& gi, T A, T P, T H, T& X) {
  if constexpr (CAL) {
    fr = fr - P;
    const T a1 = (T)1 + A;
    gr *= a1;
    gi *= a1;
    X = fma(A * ((T)2 + A), H, X);
  }
}

// ---------------------------------------------------------------- anchored phase (likelihood, mixed path)
// For the block of kAnchor bins starting at anchor bin a, the phase is
//   r_d,j = [S(f_a) + tau_d f_a] + dS_j + tau_d (f_j - f_a),  dS_j = sum_m c_m dB_m(f_j).
// The anchor term is formed once per block in float-float arithmetic and
// reduced modulo one cycle.  |dS_j| is at most sum_m |c_m| max|dB_m| over the
// block (the chirp's duration times the block's width in frequency): where
// that bound is below kFastBound cycles, dS_j runs in plain FP32 (8 FMA), is
// reduced exactly (dS - rint dS), and the small anchor and lane-offset terms
// are added (three roundings of at most 2^-24 cycles plus the FP32 error of
// dS, at most ~8 2^-24 kFastBound and ~1e-7 cycles rms on the workloads here,
// about the error of the hardware sine); otherwise dS_j runs in float-float
// arithmetic like the unanchored phase.  The choice is made per block, so it
// is uniform over the warp.
constexpr float kFastBound = 16.0f;

// Anchor term of one block: (S(f_a) + tau_d f_a) mod 1 per detector, from the
// anchor row (B_m(f_a), f_a as float pairs); returns whether the block may use
// the FP32 delta.
template <int NDET>
__device__ __forceinline__ bool anchor_terms(const float* __restrict__ ra, const float (&ch)[kNBasis],
                                             const float (&cl)[kNBasis], const float (&th)[NDET],
                                             const float (&tl)[NDET], float (&an)[NDET]) {
  float v[kAnchorRowFloats];
#pragma unroll
  for (int k = 0; k < kAnchorRowFloats / 4; ++k)
    *reinterpret_cast<float4*>(&v[4 * k]) = reinterpret_cast<const float4*>(ra)[k];
  float bound = 0.0f;
#pragma unroll
  for (int m = 0; m < kNBasis; ++m) bound = fmaf(fabsf(ch[m]), v[18 + m], bound);
  float s, lo;
  {
    float e;
    two_prod(ch[0], v[0], s, e);
    lo = __fmaf_rn(cl[0], v[0], __fmaf_rn(ch[0], v[kNBasis], e));
  }
#pragma unroll
  for (int m = 1; m < kNBasis; ++m) {
    const float bh = v[m], bl = v[kNBasis + m];
    float p, e, t, q;
    two_prod(ch[m], bh, p, e);
    two_sum(s, p, t, q);
    s = t;
    lo = __fmaf_rn(ch[m], bl, __fmaf_rn(cl[m], bh, lo + (q + e)));
  }
  const float sf = __fadd_rn(__fsub_rn(s, nearest_int(s)), lo);
  const float fh = v[16], fl = v[17];
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    float p, e;
    two_prod(th[d], fh, p, e);
    e = __fmaf_rn(th[d], fl, __fmaf_rn(tl[d], fh, e));
    const float x = __fadd_rn(__fadd_rn(sf, __fsub_rn(p, nearest_int(p))), e);
    an[d] = __fsub_rn(x, nearest_int(x));
  }
  return bound < kFastBound;
}

// One bin of the anchored path with an FP32 delta: v = the first part of the
// delta row (dB_m high parts, G_d), ad[d] = the block's anchor term plus this
// lane's tau_d (f_j - f_a).
template <int NDET, bool CAL>
__device__ __forceinline__ void bin_anchor(const float (&v)[4 * ((kNBasis + 2 * NDET + 3) / 4)],
                                           const float (&ch)[kNBasis], const float (&ad)[NDET], float (&U)[NDET],
                                           float (&V)[NDET], const CalBin<NDET, float>& cb, float (&X)[NDET]) {
  float ds = __fmul_rn(ch[0], v[0]);
#pragma unroll
  for (int m = 1; m < kNBasis; ++m) ds = __fmaf_rn(ch[m], v[m], ds);
  ds = __fsub_rn(ds, nearest_int(ds));  // exact
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    // |ds + ad| < 1.5 cycles: the hardware sine and cosine take it unreduced
    float fr = __fadd_rn(ds, ad[d]);
    float gr = v[kNBasis + 2 * d], gi = v[kNBasis + 2 * d + 1];
    cal_apply<CAL>(fr, gr, gi, cb.A[d], cb.P[d], cb.H[d], X[d]);
    float sn, cs;
    __sincosf(6.283185307179586f * fr, &sn, &cs);
    U[d] = fmaf(gr, cs, fmaf(gi, sn, U[d]));
    V[d] = fmaf(gi, cs, fmaf(-gr, sn, V[d]));
  }
}

// One bin of the anchored path with a float-float delta: v = the whole delta
// row, dB_m = (v[m], v[kNBasis + 2 NDET + m]).
template <int NDET, bool CAL>
__device__ __forceinline__ void bin_anchor_exact(const float (&v)[4 * ((2 * kNBasis + 2 * NDET + 3) / 4)],
                                                 const float (&ch)[kNBasis], const float (&cl)[kNBasis],
                                                 const float (&ad)[NDET], float (&U)[NDET], float (&V)[NDET],
                                                 const CalBin<NDET, float>& cb, float (&X)[NDET]) {
  constexpr int LO = kNBasis + 2 * NDET;
  float s, lo;
  {
    float e;
    two_prod(ch[0], v[0], s, e);
    lo = __fmaf_rn(cl[0], v[0], __fmaf_rn(ch[0], v[LO], e));
  }
#pragma unroll
  for (int m = 1; m < kNBasis; ++m) {
    const float bh = v[m], bl = v[LO + m];
    float p, e, t, q;
    two_prod(ch[m], bh, p, e);
    two_sum(s, p, t, q);
    s = t;
    lo = __fmaf_rn(ch[m], bl, __fmaf_rn(cl[m], bh, lo + (q + e)));
  }
  const float ds = __fadd_rn(__fsub_rn(s, nearest_int(s)), lo);
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    // |ds + ad| < 1.5 cycles: the hardware sine and cosine take it unreduced
    float fr = __fadd_rn(ds, ad[d]);
    float gr = v[kNBasis + 2 * d], gi = v[kNBasis + 2 * d + 1];
    cal_apply<CAL>(fr, gr, gi, cb.A[d], cb.P[d], cb.H[d], X[d]);
    float sn, cs;
    __sincosf(6.283185307179586f * fr, &sn, &cs);
    U[d] = fmaf(gr, cs, fmaf(gi, sn, U[d]));
    V[d] = fmaf(gi, cs, fmaf(-gr, sn, V[d]));
  }
}

// Window sums U_d + i V_d of one proposal over bins [j0, jend) of a staged
// window of delta rows (sm, row_elems floats per row; j0 on an anchor), by the
// anchored phase; anc0 = the anchor row of bin j0 (shared or global memory).
// With CAL, cal_sm holds the window's calibration rows (cal_row floats each),
// nodes the proposal's node data, and X_d collects the <h|h> correction.
// ffc (may be null) counts the blocks that take the float-float delta.
// The result is per lane (the caller reduces over the warp).
template <int NDET, bool CAL>
__device__ __forceinline__ void anchored_sums_cal(const float* __restrict__ sm, int row_elems,
                                                  const float* __restrict__ anc0, float df,
                                                  const PropMixed* __restrict__ P, int j0, int jend, int lane,
                                                  float (&U)[NDET], float (&V)[NDET],
                                                  const float* __restrict__ cal_sm, int cal_row,
                                                  const float4* __restrict__ nodes, float (&X)[NDET],
                                                  unsigned long long* __restrict__ ffc) {
  // anchored phase: the window starts on an anchor (windows are multiples of
  // kAnchor bins); lane l forms the anchor terms of block l of each batch of
  // 32 blocks and the warp shares them by shuffles
  constexpr int RX = 4 * ((kNBasis + 2 * NDET + 3) / 4);       // floats the FP32-delta bin reads
  constexpr int RXF = 4 * ((2 * kNBasis + 2 * NDET + 3) / 4);  // floats the float-float-delta bin reads
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
  // tau_d (f_j - f_a) = tau_d lane df (|.| < 1 cycle)
  float dtl[NDET];
  const float lane_df = (float)lane * df;
#pragma unroll
  for (int d = 0; d < NDET; ++d) dtl[d] = __fmul_rn(th[d], lane_df);
#pragma unroll
  for (int d = 0; d < NDET; ++d) U[d] = V[d] = X[d] = 0.0f;
  CalBin<NDET, float> cb0, cb1;
  const int nblk = (jend - j0 + kAnchor - 1) / kAnchor;
  for (int b0 = 0; b0 < nblk; b0 += 32) {
    float an[NDET];
#pragma unroll
    for (int d = 0; d < NDET; ++d) an[d] = 0.0f;
    bool fast = false;
    if (b0 + lane < nblk)
      fast = anchor_terms<NDET>(anc0 + (int64_t)(b0 + lane) * kAnchorRowFloats, ch, cl, th, tl, an);
    const unsigned fast_mask = __ballot_sync(0xffffffffu, fast);
    const int nb = nblk - b0 < 32 ? nblk - b0 : 32;
    for (int it = 0; it < nb; it += 2) {
      float ad0[NDET], ad1[NDET];
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        ad0[d] = __fadd_rn(__shfl_sync(0xffffffffu, an[d], it), dtl[d]);
        ad1[d] = __fadd_rn(__shfl_sync(0xffffffffu, an[d], (it + 1) & 31), dtl[d]);
      }
      const int j = j0 + (b0 + it) * kAnchor + lane;
      const int jb = j - lane;  // first bin of block it
      if (it + 1 < nb && ((fast_mask >> it) & 3u) == 3u && jb + 2 * kAnchor <= jend) {
        // the common case, two complete blocks with FP32 deltas: straight-line
        // code so that the two bins' chains interleave
        float v0[RX], v1[RX];
        const float* r0 = sm + (int64_t)(j - j0) * row_elems;
        const float* r1 = r0 + (int64_t)kAnchor * row_elems;
#pragma unroll
        for (int k = 0; k < RX / 4; ++k) {
          *reinterpret_cast<float4*>(&v0[4 * k]) = reinterpret_cast<const float4*>(r0)[k];
          *reinterpret_cast<float4*>(&v1[4 * k]) = reinterpret_cast<const float4*>(r1)[k];
        }
        if constexpr (CAL) {
          const float* c0 = cal_sm + (int64_t)(j - j0) * cal_row;
          cal_eval<NDET>(c0, nodes, cb0);
          cal_eval<NDET>(c0 + (int64_t)kAnchor * cal_row, nodes, cb1);
        }
        bin_anchor<NDET, CAL>(v0, ch, ad0, U, V, cb0, X);
        bin_anchor<NDET, CAL>(v1, ch, ad1, U, V, cb1, X);
        continue;
      }
      // otherwise block by block: each takes the FP32 or the float-float delta,
      // uniformly over the warp, and lanes past the cut sit out
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (it + h >= nb) break;
        const int jj = j + h * kAnchor;
        const float* row = sm + (int64_t)(jj - j0) * row_elems;
        if (jj < jend) {
          if constexpr (CAL) cal_eval<NDET>(cal_sm + (int64_t)(jj - j0) * cal_row, nodes, cb0);
        }
        if ((fast_mask >> (it + h)) & 1u) {
          if (jj < jend) {
            float v[RX];
#pragma unroll
            for (int k = 0; k < RX / 4; ++k) *reinterpret_cast<float4*>(&v[4 * k]) = reinterpret_cast<const float4*>(row)[k];
            bin_anchor<NDET, CAL>(v, ch, h ? ad1 : ad0, U, V, cb0, X);
          }
        } else if (jj < jend) {
          if (ffc && lane == 0) atomicAdd(ffc, 1ull);  // lane 0 holds the block's first bin
          float v[RXF];
#pragma unroll
          for (int k = 0; k < RXF / 4; ++k) *reinterpret_cast<float4*>(&v[4 * k]) = reinterpret_cast<const float4*>(row)[k];
          bin_anchor_exact<NDET, CAL>(v, ch, cl, h ? ad1 : ad0, U, V, cb0, X);
        }
      }
    }
  }
}

// The same without calibration.
template <int NDET>
__device__ __forceinline__ void anchored_sums(const float* __restrict__ sm, int row_elems,
                                              const float* __restrict__ anc0, float df,
                                              const PropMixed* __restrict__ P, int j0, int jend, int lane,
                                              float (&U)[NDET], float (&V)[NDET],
                                              unsigned long long* __restrict__ ffc = nullptr) {
  float X[NDET];
  anchored_sums_cal<NDET, false>(sm, row_elems, anc0, df, P, j0, jend, lane, U, V, nullptr, 0, nullptr, X, ffc);
}

template <int NDET>
__device__ __forceinline__ void phase_f64(const double (&v)[RowD<NDET>::n], const double (&c)[kNBasis],
                                          const double (&tau)[NDET], double (&sn)[NDET], double (&cs)[NDET],
                                          const double* shift = nullptr) {
  double r = c[0] * v[0];
#pragma unroll
  for (int m = 1; m < kNBasis; ++m) r = fma(c[m], v[m], r);
  const double f = v[8];
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    double ph = fma(tau[d], f, r);
    if (shift) ph -= shift[d];
    sincospi(2.0 * ph, &sn[d], &cs[d]);
  }
}

template <int NDET>
__device__ __forceinline__ void bin_f64(const double (&v)[RowD<NDET>::n], const double (&c)[kNBasis],
                                        const double (&tau)[NDET], double (&U)[NDET], double (&V)[NDET]) {
  double sn[NDET], cs[NDET];
  phase_f64<NDET>(v, c, tau, sn, cs);
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    const double gr = v[9 + 2 * d], gi = v[10 + 2 * d];
    U[d] = fma(gr, cs[d], fma(gi, sn[d], U[d]));
    V[d] = fma(gi, cs[d], fma(-gr, sn[d], V[d]));
  }
}

// FP64 bin with the calibration factor (phase correction in cycles).
template <int NDET>
__device__ __forceinline__ void bin_f64_cal(const double (&v)[RowD<NDET>::n], const double (&c)[kNBasis],
                                            const double (&tau)[NDET], const CalBin<NDET, double>& cb,
                                            double (&U)[NDET], double (&V)[NDET], double (&X)[NDET]) {
  double r = c[0] * v[0];
#pragma unroll
  for (int m = 1; m < kNBasis; ++m) r = fma(c[m], v[m], r);
  const double f = v[8];
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    double ph = fma(tau[d], f, r);
    double gr = v[9 + 2 * d], gi = v[10 + 2 * d];
    cal_apply<true>(ph, gr, gi, cb.A[d], cb.P[d], cb.H[d], X[d]);
    double sn, cs;
    sincospi(2.0 * ph, &sn, &cs);
    U[d] = fma(gr, cs, fma(gi, sn, U[d]));
    V[d] = fma(gi, cs, fma(-gr, sn, V[d]));
  }
}

}  // namespace gwl
