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
struct SegInfo {
  const double* freqs;  // [M]
  const double* H;      // [n_det][M] inclusive prefix of 4 df f^{-7/3} / S
  const double* geom;   // [n_det][9]
  int64_t M;
  int n_det;
  int fcut_mode;
  double f0, df, gmst, t_ref;
  // sampled-parameter map
  int n_dim;
  int param_map[11];
  double fixed[11];
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
// Wait for an mbarrier phase for at most ~1 s of SM clock; on timeout latch
// kStatusTimeout and return false (the caller then leaves the kernel).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > 2000000000LL) {
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
__device__ __forceinline__ void expand_theta(const SegInfo& s, const double* row, double th[11]) {
#pragma unroll
  for (int k = 0; k < 11; ++k) th[k] = s.fixed[k];
  for (int i = 0; i < s.n_dim; ++i) th[s.param_map[i]] = row[i];
}

__device__ __forceinline__ bool physical(const double th[11]) {
  bool ok = th[1] > 0.0 && th[1] <= 1.0 && th[0] > 0.0 && th[4] > 0.0;
#pragma unroll
  for (int k = 0; k < 11; ++k) ok = ok && isfinite(th[k]);
  return ok;
}

// Number of bins with freqs[j] <= fc (bins ascend): estimate from the grid,
// then settle against the stored FP64 frequencies so the decision matches a
// per-bin comparison exactly.
__device__ __forceinline__ int count_bins_le(const SegInfo& s, double fc) {
  if (!(fc >= s.freqs[0])) return 0;
  if (fc >= s.freqs[s.M - 1]) return (int)s.M;
  int64_t j = (int64_t)floor((fc - s.f0) / s.df);
  if (j < 0) j = 0;
  if (j > s.M - 1) j = s.M - 1;
  while (j + 1 < s.M && s.freqs[j + 1] <= fc) ++j;
  while (j >= 0 && s.freqs[j] > fc) --j;
  return (int)(j + 1);
}

// Intrinsic part: masses and spins -> basis coefficients c_m [cycles], the
// constant PN phase [cycles], the frequency cut and the amplitude A.  FP64.
struct Intrinsic {
  double c[kNBasis];
  double ccyc;
  double amp;
  int ncut;
};

__device__ inline void prologue_intrinsic(const SegInfo& s, const double th[11], Intrinsic& o) {
  const double mc = th[0], q = th[1], chi1 = th[2], chi2 = th[3], dl = th[4];
  const double opq = 1.0 + q;
  const double eta = q / (opq * opq);
  const double delta = (1.0 - q) / opq;  // sqrt(1 - 4 eta) for q <= 1
  const double x1 = 1.0 / opq, x2 = q * x1;
  const double chis = 0.5 * (chi1 + chi2), chia = 0.5 * (chi1 - chi2);
  const double eta2 = eta * eta;

  // PN phase coefficients phi_k
  const double p2 = (20.0 / 9.0) * (743.0 / 336.0 + (11.0 / 4.0) * eta);
  const double beta = ((113.0 / 12.0) * x1 * x1 + 6.25 * eta) * chi1 + ((113.0 / 12.0) * x2 * x2 + 6.25 * eta) * chi2;
  const double p3 = -16.0 * kPi + 4.0 * beta;
  const double p4 = 10.0 * (3058673.0 / 1016064.0 + (5429.0 / 1008.0) * eta + (617.0 / 144.0) * eta2) -
                    10.0 * (79.0 / 8.0) * eta * chi1 * chi2;
  const double gam = (732985.0 / 2268.0 - (24260.0 / 81.0) * eta - (340.0 / 9.0) * eta2) * chis +
                     (732985.0 / 2268.0 + (140.0 / 9.0) * eta) * delta * chia;
  const double p5c = kPi * (38645.0 / 756.0 - (65.0 / 9.0) * eta) - gam;
  const double p6c = 11583231236531.0 / 4694215680.0 - (640.0 / 3.0) * kPi * kPi - (6848.0 / 21.0) * kGammaE +
                     eta * (-15737765635.0 / 3048192.0 + (2255.0 / 12.0) * kPi * kPi) + (76055.0 / 1728.0) * eta2 -
                     (127825.0 / 1296.0) * eta2 * eta +
                     kPi * ((2270.0 / 3.0) * delta * chia + (2270.0 / 3.0 - 520.0 * eta) * chis);
  const double p7 = kPi * (77096675.0 / 254016.0 + (378515.0 / 1512.0) * eta - (74045.0 / 756.0) * eta2) +
                    (-25150083775.0 / 3048192.0 + (10566655595.0 / 762048.0) * eta - (1042165.0 / 3024.0) * eta2 +
                     (5345.0 / 36.0) * eta2 * eta) * chis +
                    delta * (-25150083775.0 / 3048192.0 + (26804935.0 / 6048.0) * eta - (1985.0 / 48.0) * eta2) * chia;

  // a = pi M [s], M = Mc eta^{-3/5}; v^k = (a f)^{k/3}: fold a^{k/3} into c_m.
  const double lmc = log(kPi * kTsun * mc);  // ln(pi Mc T_sun)
  const double la = lmc - 0.6 * log(eta);    // ln a
  const double a13 = exp(la * (1.0 / 3.0));
  const double am13 = 1.0 / a13;
  const double am23 = am13 * am13;
  const double pref = 3.0 / (128.0 * eta) / (2.0 * kPi);  // radians -> cycles
  o.c[0] = pref * am23 * am23 * am13;  // f^{-5/3}
  o.c[1] = pref * p2 * am23 * am13;     // f^{-1}
  o.c[2] = pref * p3 * am23;            // f^{-2/3}
  o.c[3] = pref * p4 * am13;            // f^{-1/3}
  o.c[4] = pref * p5c;                  // ln f    (3 ln v = ln a + ln f)
  o.c[5] = pref * a13 * (p6c - (6848.0 / 21.0) * kLn4 - (6848.0 / 63.0) * la);  // f^{1/3}
  o.c[6] = pref * a13 * (-6848.0 / 63.0);                                     // f^{1/3} ln f
  o.c[7] = pref * p7 * a13 * a13;                                             // f^{2/3}
  // constant PN phase [cycles]: phi5 (1 + ln a - 3 ln v_lso), v_lso = 6^{-1/2}
  o.ccyc = pref * p5c * (1.0 + la + 1.5 * kLn6);
  if (s.fcut_mode == 0) {
    const double a3 = a13 * a13 * a13;  // = pi M
    o.ncut = count_bins_le(s, 1.0 / (kSix32 * a3));
  } else {
    o.ncut = (int)s.M;
  }
  // A = sqrt(5/24) pi^{-2/3} (Mc T_sun)^{5/6} c / dL
  o.amp = kAmpConst * exp((5.0 / 6.0) * (lmc - kLnPi)) * kC / (dl * kMpc);
}

// Extrinsic part: sky position, polarisation angle and inclination ->
// per-detector delay tau_d = tc + dt_d and complex response
// P_d = F+_d (1 + cos^2 i)/2 - i Fx_d cos i.  FP64.
struct Extrinsic {
  double tau[kMaxDet];
  double Pr[kMaxDet], Pi[kMaxDet];
};

__device__ inline void prologue_extrinsic(const SegInfo& s, const double th[11], Extrinsic& o) {
  const double iota = th[5], psi = th[6], ra = th[7], dec = th[8], tc = th[9];
  double sl, cl, sd, cd, sp, cp;
  sincos(ra - s.gmst, &sl, &cl);
  sincos(dec, &sd, &cd);
  sincos(psi, &sp, &cp);
  const double ci = cos(iota);
  const double n0 = cd * cl, n1 = cd * sl, n2 = sd;
  // wave-frame axes X = cos psi e_E + sin psi e_N, Y = -sin psi e_E + cos psi e_N
  const double X0 = -cp * sl - sp * sd * cl, X1 = cp * cl - sp * sd * sl, X2 = sp * cd;
  const double Y0 = sp * sl - cp * sd * cl, Y1 = -sp * cl - cp * sd * sl, Y2 = cp * cd;
  const double hp = 0.5 * (1.0 + ci * ci);
#pragma unroll
  for (int d = 0; d < kMaxDet; ++d) {
    if (d >= s.n_det) {
      o.tau[d] = o.Pr[d] = o.Pi[d] = 0.0;
      continue;
    }
    const double* g = s.geom + 9 * d;
    const double xX = g[3] * X0 + g[4] * X1 + g[5] * X2, xY = g[3] * Y0 + g[4] * Y1 + g[5] * Y2;
    const double yX = g[6] * X0 + g[7] * X1 + g[8] * X2, yY = g[6] * Y0 + g[7] * Y1 + g[8] * Y2;
    // F+ = D:(XX - YY), Fx = D:(XY + YX), D = (xx - yy)/2
    const double Fp = 0.5 * ((xX * xX - xY * xY) - (yX * yX - yY * yY));
    const double Fx = xX * xY - yX * yY;
    o.tau[d] = tc - (g[0] * n0 + g[1] * n1 + g[2] * n2) / kC;
    o.Pr[d] = Fp * hp;
    o.Pi[d] = -Fx * ci;
  }
}

}  // namespace gwl
