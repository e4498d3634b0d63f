// gwl_ff.cuh -- float-float arithmetic and elementary functions on the FP32 pipe.
//
// GB300 issues FP64 instructions at about 1/60 of its FP32 rate (measured:
// 1.9 DFMA against 116 FFMA per clock per SM), so the mixed prologue keeps
// FP64-class precision (~48 significant bits, relative error ~1e-14) with
// unevaluated float pairs built from error-free transformations (Dekker 1971;
// Knuth's TwoSum; FMA-based TwoProduct).  A float-float add or multiply costs
// 7-11 FP32 instructions, several times less pipe time than one FP64
// instruction, and the elementary functions below are written from their
// series:
//   exp x   = 2^k e^r, k = rint(x / ln 2), |r| <= ln 2 / 2, e^r by its Taylor
//             series to r^13 / 13! (truncation < 4e-18), the orders from r^8 on
//             (below 6e-9) summed in FP32 and the rest in float pairs;
//   ln x    = y0 + ln(1 + t), y0 = the FP32 logarithm of the high part,
//             1 + t = x e^{-y0} (|t| ~ 1e-7), ln(1 + t) = t - t^2/2 (+ O(t^3));
//   sin/cos = reduction x = k pi/2 + r with |r| <= pi/4, the Taylor series of
//             sin r to r^15 / 15! and cos r to r^16 / 16! (truncation < 5e-17),
//             the orders from r^11 (sin) and r^12 (cos) on in FP32, the
//             quadrant k mod 4 selecting and signing them.
// The series coefficients are the reciprocal factorials.  The reductions
// subtract k c with c = ln 2 or pi/2 split into three floats (Cody & Waite
// 1980): c1 with 12 significant bits (k c1 exact for |k| < 2^12), c2 and c3
// the next 24 bits each (derived here from 50-digit values; the remainder is
// below 1e-19).  Inputs of the elementary functions are small (|x| < 2^11).
#pragma once

#include "gwl_bins.cuh"

namespace gwl {

// A double constant as a float pair (folded at compile time for literals).
__host__ __device__ constexpr FF ffc(double x) { return FF{(float)x, (float)(x - (double)(float)x)}; }
__device__ __forceinline__ FF ff(float x) { return FF{x, 0.0f}; }
// A run-time double as a float pair, and back, with integer operations: on
// GB300 an f32<->f64 conversion instruction occupies the narrow FP64 unit.
// hi = x truncated to 24 significant bits (an exact float), lo = the
// remaining 29 mantissa bits rounded to a float (integer-valued floats built
// by the 2^23 bias trick, then scaled by a power of two): hi + lo = x to about
// 2^-48.  Zero and subnormal doubles give zero; |x| outside [2^-70, 2^100]
// (not met by the prologues' inputs) takes the conversion instructions.
__device__ __forceinline__ FF ff_from(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return FF{0.0f, 0.0f};
  if (e < 1023 - 70 || e > 1023 + 100) {
    FF r;
    split_f64(x, r.hi, r.lo);
    return r;
  }
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(m >> 29));
  const unsigned ml = (unsigned)(m & 0x1FFFFFFFu);
  const float a = __fsub_rn(__uint_as_float(0x4B000000u | (ml >> 23)), 8388608.0f);       // top 6 bits
  const float c = __fsub_rn(__uint_as_float(0x4B000000u | (ml & 0x7FFFFFu)), 8388608.0f);  // low 23 bits
  const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);                   // 2^(e - 1075)
  const float lo = __fmul_rn(__fmaf_rn(a, 8388608.0f, c), scale);
  return FF{hi, sign ? -lo : lo};
}
// A float widened to double exactly (normal floats and zero; subnormal floats give zero).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)s);
  return __longlong_as_double((long long)(s | ((unsigned long long)(e - 127 + 1023) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double ff_to_double(const FF& a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

// s + e renormalised, for |e| <= |s| or s == 0 (Fast2Sum).
__device__ __forceinline__ FF ff_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return FF{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ FF operator+(const FF& a, const FF& b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return ff_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ FF operator-(const FF& a) { return FF{-a.hi, -a.lo}; }
__device__ __forceinline__ FF operator-(const FF& a, const FF& b) { return a + (-b); }
__device__ __forceinline__ FF operator*(const FF& a, const FF& b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  return ff_norm(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
// a / b: the FP32 quotient of the high parts, corrected by the quotient of the remainder.
__device__ __forceinline__ FF operator/(const FF& a, const FF& b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const FF r = a - b * ff(q1);
  return ff_norm(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ FF operator+(const FF& a, double c) { return a + ffc(c); }
__device__ __forceinline__ FF operator+(double c, const FF& a) { return a + ffc(c); }
__device__ __forceinline__ FF operator-(const FF& a, double c) { return a + ffc(-c); }
__device__ __forceinline__ FF operator-(double c, const FF& a) { return ffc(c) - a; }
__device__ __forceinline__ FF operator*(const FF& a, double c) { return a * ffc(c); }
__device__ __forceinline__ FF operator*(double c, const FF& a) { return a * ffc(c); }
__device__ __forceinline__ FF operator/(const FF& a, double c) { return a / ffc(c); }
__device__ __forceinline__ FF operator/(double c, const FF& a) { return ffc(c) / a; }

// a - rint(a) for |a| < 2^22 (the high part's nearest integer; hi - r is exact).
__device__ __forceinline__ FF frac_near(const FF& a) {
  const float r = nearest_int(a.hi);
  float s, e;
  two_sum(__fsub_rn(a.hi, r), a.lo, s, e);
  return FF{s, e};
}

// Series coefficients as float pairs (constant memory):
//   exp:  1/n!                    n = 0..13
//   sin:  (-1)^n / (2n+1)!        n = 0..7   (sin r = r sum_n c_n r^{2n})
//   cos:  (-1)^n / (2n)!          n = 0..8
static __constant__ FF kExpCoef[14] = {ffc(1.0), ffc(1.0), ffc(1.0 / 2.0), ffc(1.0 / 6.0), ffc(1.0 / 24.0),
                                       ffc(1.0 / 120.0), ffc(1.0 / 720.0), ffc(1.0 / 5040.0), ffc(1.0 / 40320.0),
                                       ffc(1.0 / 362880.0), ffc(1.0 / 3628800.0), ffc(1.0 / 39916800.0),
                                       ffc(1.0 / 479001600.0), ffc(1.0 / 6227020800.0)};
static __constant__ FF kSinCoef[8] = {ffc(1.0), ffc(-1.0 / 6.0), ffc(1.0 / 120.0), ffc(-1.0 / 5040.0),
                                      ffc(1.0 / 362880.0), ffc(-1.0 / 39916800.0), ffc(1.0 / 6227020800.0),
                                      ffc(-1.0 / 1307674368000.0)};
static __constant__ FF kCosCoef[9] = {ffc(1.0), ffc(-1.0 / 2.0), ffc(1.0 / 24.0), ffc(-1.0 / 720.0),
                                      ffc(1.0 / 40320.0), ffc(-1.0 / 3628800.0), ffc(1.0 / 479001600.0),
                                      ffc(-1.0 / 87178291200.0), ffc(1.0 / 20922789888000.0)};
// x - k (c1 + c2 + c3): k c1 exact, k c2 exact as a float pair (TwoProduct),
// k c3 below the float-float rounding.
__device__ __forceinline__ FF ff_reduce(const FF& x, float k, float c1, float c2, float c3) {
  FF t = x - ff(__fmul_rn(k, c1));
  float p, e;
  two_prod(k, c2, p, e);
  t = t - FF{p, e};
  return t - ff(__fmul_rn(k, c3));
}

// The elementary functions are out of line: each is a few hundred
// instructions, called from several places, and one copy of each keeps the
// prologues' code within the instruction cache.  In each series only the
// orders whose FP32 rounding would show at the float-pair level are summed
// as float pairs: the high orders of a Taylor series are small enough for
// plain FP32, which takes about a fifth of the instructions.
static __device__ __noinline__ FF ff_exp(const FF& x) {
  const float k = nearest_int(__fmul_rn(x.hi, 1.44269504088896341f));
  const FF r = ff_reduce(x, k, 0x1.62e000p-1f, 0x1.0bfbe8p-15f, 0x1.cf79acp-40f);  // ln 2
  // orders 8..13 in FP32 (r^8 / 8! < 6e-9, so their rounding stays below 1e-15 relative)
  const float rh = r.hi;
  float q = kExpCoef[13].hi;
#pragma unroll
  for (int n = 12; n >= 8; --n) q = __fmaf_rn(q, rh, kExpCoef[n].hi);
  FF p = ff(q);
#pragma unroll 1
  for (int n = 7; n >= 0; --n) p = p * r + kExpCoef[n];
  const float s = __int_as_float((127 + (int)k) << 23);  // 2^k (|k| < 127 for these inputs)
  return FF{__fmul_rn(p.hi, s), __fmul_rn(p.lo, s)};
}

static __device__ __noinline__ FF ff_log(const FF& x) {
  const float y0 = logf(x.hi);
  const FF t = x * ff_exp(ff(-y0)) - 1.0;
  return ff(y0) + (t - t * t * 0.5);
}

static __device__ __noinline__ void ff_sincos(const FF& x, FF* sn, FF* cs) {
  const float k = nearest_int(__fmul_rn(x.hi, 0.636619772367581343f));
  const FF r = ff_reduce(x, k, 0x1.920000p+0f, 0x1.fb5444p-12f, 0x1.68c234p-39f);  // pi / 2
  const FF r2 = r * r;
  // sin: orders r^11.. and cos: orders r^12.. in FP32 (below 2e-9 and 2e-10), the rest as float pairs
  const float h = r2.hi;
  float qs = kSinCoef[7].hi, qc = kCosCoef[8].hi;
  qs = __fmaf_rn(qs, h, kSinCoef[6].hi);
  qs = __fmaf_rn(qs, h, kSinCoef[5].hi);
  qc = __fmaf_rn(qc, h, kCosCoef[7].hi);
  qc = __fmaf_rn(qc, h, kCosCoef[6].hi);
  FF ps = ff(qs), pc = ff(qc);
  pc = pc * r2 + kCosCoef[5];
#pragma unroll 1
  for (int n = 4; n >= 0; --n) {  // the two series interleaved
    ps = ps * r2 + kSinCoef[n];
    pc = pc * r2 + kCosCoef[n];
  }
  const FF s = r * ps, c = pc;
  switch ((int)k & 3) {
    case 0: *sn = s; *cs = c; break;
    case 1: *sn = c; *cs = -s; break;
    case 2: *sn = -s; *cs = -c; break;
    default: *sn = -c; *cs = s; break;
  }
}

// Overloads used by the templated model code (gwl_device.cuh).
// K's phase angle: the float-pair sine and cosine reduce by pi/2 themselves, so
// the 2 pi reduction (an FP64 rint) of the generic version is not needed.
template <int N, class G>
__device__ __forceinline__ void k_angle(const Tan<N, G, FF>& phic, const Tan<N, G, FF>& ccyc, Tan<N, G, FF>& sa,
                                        Tan<N, G, FF>& ca) {
  sincos(phic + (0.25 * kPi) - (2.0 * kPi) * frac_near(ccyc), &sa, &ca);
}
template <>
__device__ __forceinline__ FF make_value<FF>(double x) { return ff_from(x); }
__device__ __forceinline__ double vval(const FF& x) { return ff_to_double(x); }
template <class G>
__device__ __forceinline__ G vshadow(const FF& x) { return (G)x.hi; }
__device__ __forceinline__ FF vexp(const FF& x) { return ff_exp(x); }
__device__ __forceinline__ FF vlog(const FF& x) { return ff_log(x); }
__device__ __forceinline__ void vsincos(const FF& x, FF* s, FF* c) { ff_sincos(x, s, c); }
__device__ __forceinline__ FF vfrac(const FF& x) { return frac_near(x); }
// tangent values times float-pair constants (the pre-split detector geometry)
template <int N, class G>
__device__ __forceinline__ Tan<N, G, FF> operator*(const Tan<N, G, FF>& a, const FF& b) {
  Tan<N, G, FF> r;
  r.v = a.v * b;
  const G bt = (G)b.hi;
  r.vt = a.vt * bt;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * bt;
  return r;
}
template <int N, class G>
__device__ __forceinline__ Tan<N, G, FF> operator*(const FF& b, const Tan<N, G, FF>& a) { return a * b; }
__device__ __forceinline__ FF exp(const FF& x) { return ff_exp(x); }
__device__ __forceinline__ FF log(const FF& x) { return ff_log(x); }
__device__ __forceinline__ void sincos(const FF& x, FF* s, FF* c) { ff_sincos(x, s, c); }
__device__ __forceinline__ FF cos(const FF& x) {
  FF s, c;
  ff_sincos(x, &s, &c);
  return c;
}

// Node data of one proposal for the warp's calibration splines (spline
// s = 2 d + q, q = 0 amplitude, 1 phase; node k): the lanes first store the
// node values y_k from the proposal's row of theta, y = [NDET][2][nn] (the
// phase scaled to cycles; in the mixed path each is narrowed once, by integer
// operations), then form the curvatures m_k = sum_i Q_ki y_i from the stored
// values.  Nodes: (dA_k, m^A_k, dphi_k, m^phi_k) per detector and node.
template <int NDET, bool MIXED, typename Node>
__device__ __forceinline__ void cal_nodes_fill(const double* __restrict__ y, int nn, const void* __restrict__ calQ,
                                               int lane, Node* __restrict__ nd) {
  using T = typename std::conditional<MIXED, float, double>::type;
  const T* Q = reinterpret_cast<const T*>(calQ);
  __syncwarp();  // the warp is done with the previous proposal's node data
  for (int o = lane; o < 2 * NDET * nn; o += 32) {
    const int sp = o / nn, k = o - sp * nn;
    const double yd = __ldg(y + o);
    T yv;
    if constexpr (MIXED) yv = ff_from(yd).hi;
    else yv = yd;
    reinterpret_cast<T*>(&nd[(sp >> 1) * kMaxCalNodes + k])[2 * (sp & 1)] = (sp & 1) ? yv * (T)(0.5 / kPi) : yv;
  }
  __syncwarp();
  for (int o = lane; o < 2 * NDET * nn; o += 32) {
    const int sp = o / nn, k = o - sp * nn;
    const T* ys = reinterpret_cast<const T*>(&nd[(sp >> 1) * kMaxCalNodes]) + 2 * (sp & 1);  // stride 4 T
    T m = (T)0;
    for (int i = 0; i < nn; ++i) m = fma(Q[k * nn + i], ys[4 * i], m);
    reinterpret_cast<T*>(&nd[(sp >> 1) * kMaxCalNodes + k])[2 * (sp & 1) + 1] = m;
  }
  __syncwarp();
}

}  // namespace gwl
