// gwl_device.cuh -- device-side building blocks shared by the library's kernels.
//
// Model (the paper fixes only Eq. 2; the template is an aligned-spin
// TaylorF2 inspiral):
//   h_d(f) = A f^{-7/6} [F+_d (1 + cos^2 i)/2 - i Fx_d cos i] e^{-i Psi_d(f)},
//   Psi_d(f) = 2 pi f (t_ref + tc + dt_d) - phic - pi/4
//              + 3/(128 eta v^5) sum_k phi_k v^k,   v = (pi M f)^{1/3},
//   A = sqrt(5/24) pi^{-2/3} (Mc T_sun)^{5/6} c / dL,  h = 0 above the cut.
// The PN phase is linear in nine functions of f (f^{-5/3}, f^{-1}, f^{-2/3},
// f^{-1/3}, ln f, f^{1/3}, f^{1/3} ln f, f^{2/3}, f) plus a constant, so per
// proposal it reduces to eight coefficients c_m (in cycles), a per-detector
// time tau_d = tc + dt_d and a complex constant K_d that also carries the
// amplitude, the antenna response, phic, pi/4 and the constant PN term.
// The data side (conj(d) f^{-7/6} 4 df / S and the t_ref phase) is folded into
// per-bin tables G_d, and <h|h> into prefix sums H_d of 4 df f^{-7/3} / S.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gwl {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTsun = 4.925490947e-6;       // G M_sun / c^3 [s]
constexpr double kC = 299792458.0;             // [m/s]
constexpr double kMpc = 3.085677581491367e22;  // [m]
constexpr double kGammaE = 0.5772156649015329;

constexpr int kMaxDet = 4;
constexpr int kNBasis = 8;  // basis functions besides f itself

// Status bits latched by kernels.
constexpr int kStatusTimeout = 1;

// Per-bin table rows.
//  mixed: float [bh 0..7 | bl 0..7 | fh fl | G_d (re, im) x n_det | pad]
//  fp64 : double [b 0..7 | f | G_d (re, im) x n_det | pad]
// Rows are padded to an odd number of 16-byte units: when the 32 lanes of a
// warp read 32 consecutive rows with 16-byte vector loads, the 8 lanes of each
// shared-memory phase then hit 8 different 16-byte bank groups (no conflicts).
__host__ __device__ constexpr int odd_units(int units) { return (units % 2) ? units : units + 1; }
__host__ __device__ constexpr int mixed_row_floats(int ndet) { return 4 * odd_units((18 + 2 * ndet + 3) / 4); }
__host__ __device__ constexpr int f64_row_doubles(int ndet) { return 2 * odd_units((9 + 2 * ndet + 1) / 2); }
// Anchored phase (likelihood, mixed path): bins are grouped in blocks of
// kAnchor; a delta row holds dB_m(f_j) = B_m(f_j) - B_m(f_a) (a = the block's
// first bin) as a float pair and G_d,j, laid out [dB_hi 0..7][G_d][dB_lo 0..7];
// an anchor row holds B_m(f_a) and f_a as float pairs and the block's largest
// |dB_m|: [bh 0..7][bl 0..7][fh, fl][dmax 0..7][pad 2] (seven 16-byte units).
constexpr int kAnchor = 32;
__host__ __device__ constexpr int delta_row_floats(int ndet) { return 4 * odd_units((16 + 2 * ndet + 3) / 4); }
constexpr int kAnchorRowFloats = 28;

// Calibration model (Section 2.2 of the paper): per detector, amplitude and
// phase corrections at n_nodes frequency nodes, natural cubic splines in
// x = ln f.  On interval [x_k, x_{k+1}] (h = x_{k+1} - x_k, t = (x - x_k)/h,
// the end intervals continued beyond the nodes) a spline with node values y
// and second derivatives m is
//   S(x) = (1 - t) y_k + t y_{k+1} + w_c m_k + w_e m_{k+1},
//   w_c = h^2/6 ((1 - t)^3 - (1 - t)),  w_e = h^2/6 (t^3 - t),
// so a bin needs t, h^2/6 and k, shared by every spline, and a proposal
// needs (y, m) per node, with m = Q y for a fixed n_nodes x n_nodes matrix Q
// of the node layout.  Calibration rows: [t, h^2/6, k, dH_d x n_det]
// (dH_d,j = H_d[j] - H_d[j-1], the bin's <h|h> weight), float rows in whole
// 8-byte pairs (24 bytes for 2-3 detectors: three 64-bit loads per bin without
// bank conflicts), double rows padded to an odd number of 16-byte units.  A
// table holds one zero row past the last bin, because float rows are staged in
// pairs (a bulk copy moves whole 16-byte units).
constexpr int kMaxCalNodes = 16;
__host__ __device__ constexpr int cal_row_floats(int ndet) { return 2 * ((3 + ndet + 1) / 2); }
__host__ __device__ constexpr int cal_row_doubles(int ndet) { return 2 * odd_units((3 + ndet + 1) / 2); }
// Per-warp node data of the proposal being summed: (dA_k, m^A_k, dphi_k,
// m^phi_k) per detector and node, the phase values in cycles.
struct alignas(32) CalNodeD {
  double v[4];
};

// Per-proposal coefficients read warp-uniformly by the bin loop.
struct alignas(16) PropMixed {
  float ch[kNBasis], cl[kNBasis];  // c_m as float pairs [cycles per basis unit]
  float th[kMaxDet], tl[kMaxDet];  // tau_d as float pairs [s]
};
struct alignas(16) PropF64 {
  double c[kNBasis];
  double tau[kMaxDet];
};
// Per-proposal values used once, at the combination step.
struct alignas(16) PropCommon {
  double Kr[kMaxDet], Ki[kMaxDet];  // K_d
  double hh;                        // sum_d |K_d|^2 H_d[ncut - 1]  (= <h|h>)
  int ncut;                         // bins with f_j <= f_cut (0 .. M)
  int flag;                         // 1: unphysical row, lnL = -inf
};

// Everything the prologue needs about the data segment.
// An unevaluated float pair x = hi + lo with |lo| <= ulp(hi)/2: about 48
// significant bits, computed on the FP32 pipe (arithmetic in gwl_ff.cuh).
struct FF {
  float hi, lo;
};

struct SegInfo {
  const double* freqs;  // [M]
  const double* H;      // [n_det][M] inclusive prefix of 4 df f^{-7/3} / S
  const double* geom;   // [n_det][9]
  int64_t M;
  int n_det;
  int fcut_mode;
  double f0, df, gmst, t_ref;
  // Exact power of two close to sqrt(<h|h> weight of the whole band): the
  // tables hold G / amp_scale and H / amp_scale^2 and the prologue multiplies
  // the amplitude by amp_scale, so that every quantity is O(1) -- well inside
  // the FP32 range used by the mixed path and the FP32 tangents.
  double amp_scale;
  // sampled-parameter map; rows of theta hold n_dim sampled coordinates, then
  // (with calibration) 2 n_nodes n_det calibration parameters: stride doubles
  int n_dim;
  int stride;
  int param_map[11];
  int param_pos[11];  // inverse of param_map: the row position of parameter k, -1 when fixed
  double fixed[11];
  double inv_df;      // 1 / df
  // float-float copies for the mixed prologue: the detector geometry, the
  // vertex over c (delays) and the amplitude constant
  // sqrt(5/24) pi^{-2/3} c / Mpc * amp_scale
  FF geom_ff[kMaxDet][9];
  FF vtx_c_ff[kMaxDet][3];
  FF amp_c_ff;
};

// ------------------------------------------------------------- float-float
// Error-free transformations (Knuth TwoSum, FMA-based TwoProduct).  The
// explicit _rn intrinsics keep the compiler from contracting a product into a
// following addition, which would break exactness.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__host__ __device__ inline void split_f64(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// ------------------------------------------------------------- TMA / mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Bulk (non-tensor) asynchronous copy global -> shared, completing on an
// mbarrier.  Both addresses and the size must be multiples of 16 bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for an mbarrier phase for at most `limit` SM clocks (default ~1 s);
// on timeout latch kStatusTimeout and return false (the caller then leaves
// the kernel).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status,
                                                  long long limit = 2000000000LL) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      atomicOr(status, kStatusTimeout);
      return false;
    }
  }
  return true;
}

// ------------------------------------------------------------- prologue
// Constants of the model evaluated at compile time.
constexpr double kLnPi = 1.1447298858494002;            // ln(pi)
constexpr double kLn4 = 1.3862943611198906;             // ln(4)
constexpr double kLn6 = 1.791759469228055;              // ln(6)
constexpr double kSix32 = 14.696938456699069;           // 6^{3/2}
constexpr double kAmpConst = 0.21278751013966343;       // sqrt(5/24) pi^{-2/3}

// Full 11-D parameter vector from the sampled coordinates of one row.
// One compile-time index per parameter: th stays in registers and the row's
// loads are all issued before the first is used.
__device__ __forceinline__ void expand_theta(const SegInfo& s, const double* row, double th[11]) {
#pragma unroll
  for (int k = 0; k < 11; ++k) th[k] = s.param_pos[k] >= 0 ? row[s.param_pos[k]] : s.fixed[k];
}

__device__ __forceinline__ bool physical(const double th[11]) {
  bool ok = th[1] > 0.0 && th[1] <= 1.0 && th[0] > 0.0 && th[4] > 0.0;
#pragma unroll
  for (int k = 0; k < 11; ++k) ok = ok && isfinite(th[k]);
  return ok;
}

// Pull the lines of H_d[j-1 .. j+1] (all detectors) into L2, j an FP32
// estimate of the last bin at or below the cut frequency 1 / (6^{3/2} pi M
// T_sun): the exact count that is read later differs from it by at most a bin.
__device__ __forceinline__ void prefetch_cut_H(const SegInfo& s, double mc, double q) {
  int64_t j = s.M - 1;
  if (s.fcut_mode == 0) {
    const float qf = (float)q, opq = 1.0f + qf;
    const float M = (float)mc * __powf(qf / (opq * opq), -0.6f);
    const float fc = 1.0f / ((float)(kSix32 * kPi * kTsun) * M);
    const float x = fminf(fmaxf(floorf((fc - (float)s.f0) * (float)s.inv_df), 0.0f), (float)(s.M - 1));
    j = (int64_t)x;
  }
  const int64_t a = j > 0 ? j - 1 : 0, b = j + 1 < s.M ? j + 1 : s.M - 1;
  for (int d = 0; d < s.n_det; ++d) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(s.H + d * s.M + a));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(s.H + d * s.M + b));
  }
}

// Number of bins with freqs[j] <= fc (bins ascend).  The stored frequencies
// lie within 1e-9 df of f0 + j df (checked when the context is made), so when
// x = (fc - f0) / df is more than 1e-7 from an integer the count follows from
// x alone; otherwise it is settled against the stored FP64 frequencies.  Either
// way the decision matches a per-bin comparison exactly.
__device__ __forceinline__ int count_bins_le(const SegInfo& s, double fc) {
  const double x = (fc - s.f0) * s.inv_df;
  const double jf = floor(x), r = x - jf;
  if (r > 1e-7 && r < 1.0 - 1e-7) {
    if (jf < 0.0) return 0;
    if (jf >= (double)(s.M - 1)) return (int)s.M;
    return (int)jf + 1;
  }
  if (!(fc >= s.freqs[0])) return 0;
  if (fc >= s.freqs[s.M - 1]) return (int)s.M;
  int64_t j = (int64_t)floor((fc - s.f0) / s.df);
  if (j < 0) j = 0;
  if (j > s.M - 1) j = s.M - 1;
  while (j + 1 < s.M && s.freqs[j + 1] <= fc) ++j;
  while (j >= 0 && s.freqs[j] > fc) --j;
  return (int)(j + 1);
}

// ------------------------------------------------------------- model formulas
// Written once as templates over the scalar type: T = double for the FP64
// likelihood, T = FF (a float pair, gwl_ff.cuh) for the mixed one, and
// T = Tan<...> (value with tangents) for the gradient.

// Value-type helpers: V = double here; gwl_ff.cuh adds the float-pair versions.
template <class V>
__device__ __forceinline__ V make_value(double x);
template <>
__device__ __forceinline__ double make_value<double>(double x) { return x; }
__device__ __forceinline__ double vval(double x) { return x; }
template <class G>
__device__ __forceinline__ G vshadow(double x) { return (G)x; }
__device__ __forceinline__ double vexp(double x) { return ::exp(x); }
__device__ __forceinline__ double vlog(double x) { return ::log(x); }
__device__ __forceinline__ void vsincos(double x, double* s, double* c) { ::sincos(x, s, c); }
__device__ __forceinline__ double vfrac(double x) { return x - rint(x); }

// Forward-mode tangent type: the value V is FP64 (bit-identical arithmetic to
// the FP64 path) or a float pair (the mixed path's arithmetic); the N
// tangents, and a shadow copy of the value used for the tangent arithmetic,
// are kept in G (float on the fast pipe, or double).
template <int N, class G, class V = double>
struct Tan {
  V v;
  G vt;
  G d[N];
};

template <int N, class G, class V = double>
__device__ __forceinline__ Tan<N, G, V> tan_const(double x) {
  Tan<N, G, V> r;
  r.v = make_value<V>(x);
  r.vt = vshadow<G>(r.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (G)0;
  return r;
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator+(const Tan<N, G, V>& a, const Tan<N, G, V>& b) {
  Tan<N, G, V> r;
  r.v = a.v + b.v;
  r.vt = a.vt + b.vt;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator-(const Tan<N, G, V>& a, const Tan<N, G, V>& b) {
  Tan<N, G, V> r;
  r.v = a.v - b.v;
  r.vt = a.vt - b.vt;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator-(const Tan<N, G, V>& a) {
  Tan<N, G, V> r;
  r.v = -a.v;
  r.vt = -a.vt;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator*(const Tan<N, G, V>& a, const Tan<N, G, V>& b) {
  Tan<N, G, V> r;
  r.v = a.v * b.v;
  r.vt = a.vt * b.vt;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.vt + a.vt * b.d[i];
  return r;
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator/(const Tan<N, G, V>& a, const Tan<N, G, V>& b) {
  Tan<N, G, V> r;
  r.v = a.v / b.v;
  r.vt = a.vt / b.vt;
  const G ib = (G)1 / b.vt;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.vt * b.d[i]) * ib;
  return r;
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator+(const Tan<N, G, V>& a, double b) {
  Tan<N, G, V> r = a;
  r.v = a.v + b;
  r.vt += (G)b;
  return r;
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator+(double b, const Tan<N, G, V>& a) { return a + b; }
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator-(const Tan<N, G, V>& a, double b) { return a + (-b); }
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator-(double b, const Tan<N, G, V>& a) { return (-a) + b; }
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator*(const Tan<N, G, V>& a, double b) {
  Tan<N, G, V> r;
  r.v = a.v * b;
  r.vt = a.vt * (G)b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * (G)b;
  return r;
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator*(double b, const Tan<N, G, V>& a) { return a * b; }
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator/(const Tan<N, G, V>& a, double b) { return a * (1.0 / b); }
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> operator/(double a, const Tan<N, G, V>& b) {
  return tan_const<N, G, V>(a) / b;
}

template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> tan_lift(const Tan<N, G, V>& a, const V& fv, G ft, G dft) {
  Tan<N, G, V> r;
  r.v = fv;
  r.vt = ft;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = dft * a.d[i];
  return r;
}
// double overloads visible next to the tangent-type templates in this namespace
__device__ __forceinline__ double exp(double x) { return ::exp(x); }
__device__ __forceinline__ double log(double x) { return ::log(x); }
__device__ __forceinline__ double cos(double x) { return ::cos(x); }
__device__ __forceinline__ void sincos(double x, double* s, double* c) { ::sincos(x, s, c); }

// For the transcendental functions the shadow values are taken from the
// full-precision results: an argument whose shadow has drifted (a phase of
// many cycles, say) would otherwise spoil the derivative.
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> exp(const Tan<N, G, V>& a) {
  const V fv = vexp(a.v);
  const G ft = vshadow<G>(fv);
  return tan_lift(a, fv, ft, ft);
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> log(const Tan<N, G, V>& a) {
  const V fv = vlog(a.v);
  return tan_lift(a, fv, vshadow<G>(fv), (G)1 / vshadow<G>(a.v));
}
template <int N, class G, class V>
__device__ __forceinline__ void sincos(const Tan<N, G, V>& a, Tan<N, G, V>* s, Tan<N, G, V>* c) {
  V sv, cv;
  vsincos(a.v, &sv, &cv);
  const G st = vshadow<G>(sv), ct = vshadow<G>(cv);
  *s = tan_lift(a, sv, st, ct);
  *c = tan_lift(a, cv, ct, -st);
}
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> cos(const Tan<N, G, V>& a) {
  Tan<N, G, V> s, c;
  sincos(a, &s, &c);
  return c;
}
// x - nearest integer: the integer shift carries no derivative.
__device__ __forceinline__ double frac_near(double x) { return x - rint(x); }
template <int N, class G, class V>
__device__ __forceinline__ Tan<N, G, V> frac_near(const Tan<N, G, V>& a) {
  Tan<N, G, V> r = a;
  r.v = vfrac(a.v);
  r.vt = vshadow<G>(r.v);  // the reduced value, not the drifted shadow of a large one
  return r;
}
__device__ __forceinline__ double val(double x) { return x; }
template <int N, class G, class V>
__device__ __forceinline__ double val(const Tan<N, G, V>& a) { return vval(a.v); }

// TaylorF2 phase coefficients phi_k (aligned spins; the 2.5PN and 3PN terms
// carry the ln v parts separately).
template <class T>
struct PNCoeffs {
  T eta, p2, p3, p4, p5c, p6c, p7;
};

template <class T>
__device__ __forceinline__ PNCoeffs<T> pn_coeffs(const T& q, const T& chi1, const T& chi2) {
  PNCoeffs<T> P;
  const T opq = q + 1.0;
  const T eta = q / (opq * opq);
  const T delta = (1.0 - q) / opq;  // sqrt(1 - 4 eta) for q <= 1
  const T x1 = 1.0 / opq, x2 = q * x1;
  const T chis = (chi1 + chi2) * 0.5, chia = (chi1 - chi2) * 0.5;
  const T eta2 = eta * eta;
  const T beta = ((113.0 / 12.0) * x1 * x1 + 6.25 * eta) * chi1 + ((113.0 / 12.0) * x2 * x2 + 6.25 * eta) * chi2;
  const T gam = (732985.0 / 2268.0 - (24260.0 / 81.0) * eta - (340.0 / 9.0) * eta2) * chis +
                ((140.0 / 9.0) * eta + 732985.0 / 2268.0) * delta * chia;
  P.eta = eta;
  P.p2 = (743.0 / 336.0 + (11.0 / 4.0) * eta) * (20.0 / 9.0);
  P.p3 = 4.0 * beta - 16.0 * kPi;
  P.p4 = (3058673.0 / 1016064.0 + (5429.0 / 1008.0) * eta + (617.0 / 144.0) * eta2) * 10.0 -
         (10.0 * 79.0 / 8.0) * eta * chi1 * chi2;
  P.p5c = kPi * (38645.0 / 756.0 - (65.0 / 9.0) * eta) - gam;
  P.p6c = (11583231236531.0 / 4694215680.0 - (640.0 / 3.0) * kPi * kPi - (6848.0 / 21.0) * kGammaE) +
          eta * (-15737765635.0 / 3048192.0 + (2255.0 / 12.0) * kPi * kPi) + (76055.0 / 1728.0) * eta2 -
          (127825.0 / 1296.0) * eta2 * eta +
          kPi * ((2270.0 / 3.0) * delta * chia + ((2270.0 / 3.0) - 520.0 * eta) * chis);
  P.p7 = kPi * (77096675.0 / 254016.0 + (378515.0 / 1512.0) * eta - (74045.0 / 756.0) * eta2) +
         ((-25150083775.0 / 3048192.0) + (10566655595.0 / 762048.0) * eta - (1042165.0 / 3024.0) * eta2 +
          (5345.0 / 36.0) * eta2 * eta) * chis +
         delta * ((-25150083775.0 / 3048192.0) + (26804935.0 / 6048.0) * eta - (1985.0 / 48.0) * eta2) * chia;
  return P;
}

// Mass scale: ln a and a^{1/3} with a = pi M = pi Mc eta^{-3/5} T_sun, and the
// amplitude A = sqrt(5/24) pi^{-2/3} (Mc T_sun)^{5/6} c / dL.
template <class T>
struct Scale {
  T la, a13, amp;
};
template <class T>
__device__ __forceinline__ Scale<T> mass_scale(const T& mc, const T& eta, const T& dl, double amp_scale) {
  Scale<T> o;
  const T lmc = log(mc * (kPi * kTsun));  // ln(pi Mc T_sun)
  o.la = lmc - 0.6 * log(eta);
  o.a13 = exp(o.la * (1.0 / 3.0));
  o.amp = exp((lmc - kLnPi) * (5.0 / 6.0)) * (kAmpConst * kC / kMpc * amp_scale) / dl;
  return o;
}

// The 2.5PN term's constant phase phi5 (1 + ln a - 3 ln v_lso) in cycles,
// v_lso = 6^{-1/2}, given pref = 3 / (128 eta) / (2 pi).
template <class T>
__device__ __forceinline__ T const_cycles(const T& pref, const T& p5c, const T& la) {
  return pref * p5c * (la + (1.0 + 1.5 * kLn6));
}
template <class T>
__device__ __forceinline__ T cycles_pref(const T& eta) { return (3.0 / (128.0 * 2.0 * kPi)) / eta; }

// Basis coefficients c_m [cycles] and the constant PN phase [cycles]:
// v^k = (a f)^{k/3}, so a^{k/3} folds into c_m; 3 ln v = ln a + ln f.
template <class T>
__device__ __forceinline__ void basis_coeffs(const PNCoeffs<T>& P, const Scale<T>& S, T (&c)[kNBasis], T& ccyc) {
  const T am13 = 1.0 / S.a13, am23 = am13 * am13;
  const T pref = cycles_pref(P.eta);  // radians -> cycles
  c[0] = pref * am23 * am23 * am13;                                                // f^{-5/3}
  c[1] = pref * P.p2 * am23 * am13;                                                // f^{-1}
  c[2] = pref * P.p3 * am23;                                                       // f^{-2/3}
  c[3] = pref * P.p4 * am13;                                                       // f^{-1/3}
  c[4] = pref * P.p5c;                                                             // ln f
  c[5] = pref * S.a13 * (P.p6c - (6848.0 / 21.0) * kLn4 - (6848.0 / 63.0) * S.la);  // f^{1/3}
  c[6] = pref * S.a13 * (-6848.0 / 63.0);                                          // f^{1/3} ln f
  c[7] = pref * P.p7 * S.a13 * S.a13;                                              // f^{2/3}
  ccyc = const_cycles(pref, P.p5c, S.la);
}

// Sky direction n = (cos dec cos lam, cos dec sin lam, sin dec), lam = ra - gmst.
template <class T>
struct Sky {
  T sl, cl, sd, cd;
};
template <class T>
__device__ __forceinline__ Sky<T> sky_trig(const T& ra, const T& dec, double gmst) {
  Sky<T> k;
  sincos(ra - gmst, &k.sl, &k.cl);
  sincos(dec, &k.sd, &k.cd);
  return k;
}

// tau_d = tc - (r_d / c . n), the vertex over c given (double or float pairs)
template <class T, class Gc>
__device__ __forceinline__ T delay_vc(const T& tc, const Sky<T>& k, const Gc* vc) {
  return tc - ((k.cd * k.cl) * vc[0] + (k.cd * k.sl) * vc[1] + k.sd * vc[2]);
}

// tau_d = tc - (r_d . n)/c
template <class T>
__device__ __forceinline__ T delay(const T& tc, const Sky<T>& k, const double* g) {
  return tc - ((k.cd * k.cl) * (g[0] / kC) + (k.cd * k.sl) * (g[1] / kC) + k.sd * (g[2] / kC));
}

// P_d = F+ (1 + cos^2 i)/2 - i Fx cos i for one detector, with the wave-frame
// axes X = cos psi e_E + sin psi e_N, Y = -sin psi e_E + cos psi e_N,
// e_E = (-sin lam, cos lam, 0), e_N = (-sin dec cos lam, -sin dec sin lam, cos dec),
// F+ = D:(XX - YY), Fx = D:(XY + YX), D = (xx - yy)/2.
template <class T, class G>
__device__ __forceinline__ void response(const Sky<T>& k, const T& sp, const T& cp, const T& ci, const G* g,
                                         T& Pr, T& Pi) {
  const T X0 = -(cp * k.sl) - sp * k.sd * k.cl, X1 = cp * k.cl - sp * k.sd * k.sl, X2 = sp * k.cd;
  const T Y0 = sp * k.sl - cp * k.sd * k.cl, Y1 = -(sp * k.cl) - cp * k.sd * k.sl, Y2 = cp * k.cd;
  const T xX = X0 * g[3] + X1 * g[4] + X2 * g[5], xY = Y0 * g[3] + Y1 * g[4] + Y2 * g[5];
  const T yX = X0 * g[6] + X1 * g[7] + X2 * g[8], yY = Y0 * g[6] + Y1 * g[7] + Y2 * g[8];
  const T Fp = ((xX * xX - xY * xY) - (yX * yX - yY * yY)) * 0.5;
  const T Fx = xX * xY - yX * yY;
  Pr = Fp * ((ci * ci + 1.0) * 0.5);
  Pi = -(Fx * ci);
}

// K_d = A P_d e^{i (phic + pi/4 - 2 pi ccyc)} and <h|h>_d = |K_d|^2 H_d[ncut - 1].
template <class T>
__device__ __forceinline__ void k_angle(const T& phic, const T& ccyc, T& sa, T& ca) {
  T ang = phic + (0.25 * kPi) - (2.0 * kPi) * frac_near(ccyc);
  ang = ang - (2.0 * kPi) * rint(val(ang) * (0.5 / kPi));
  sincos(ang, &sa, &ca);
}

}  // namespace gwl
