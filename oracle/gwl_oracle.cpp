// gwl_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, FP64 CPU oracle for the batched frequency-domain Gaussian-noise
// gravitational-wave log-likelihood and for static parallel nested sampling
// (Smith, Ashton, Vajpeyi & Talbot 2020, "Massively parallel Bayesian
// inference for transient gravitational-wave astronomy").  Only the test
// suite, the smoke check and the CPU-baseline leg of the benchmark may load
// this library; the product path never does.
//
// Everything here is written from the plain definitions, one bin at a time:
//   * Eq. 2 of the paper, read as the log-likelihood ratio
//       lnL = sum_det [ <d|h> - 1/2 <h|h> ],  <a|b> = 4 df Re sum_j conj(a_j) b_j / S_j
//     (the Gaussian exponent -(2/T)|d-h|^2/S equals -1/2 <d-h|d-h> since
//     4 df / 2 = 2/T; the theta-independent -1/2<d|d> and the normalisation
//     are dropped);
//   * an aligned-spin TaylorF2 inspiral (Newtonian amplitude, 3.5PN phase)
//     evaluated directly per bin: cbrt, log, pow, FP64 sin/cos of the FULL
//     phase, complex FP64 arithmetic -- no basis tables, no prefix sums, no
//     factorisation of the inner product, no cycle reduction;
//   * the gradient: the same templated code run on forward-mode dual numbers;
//   * the calibration model of Section 2.2: per-detector amplitude and phase
//     corrections at frequency nodes, natural cubic splines in ln f applied
//     to the template bin by bin (pinned against scipy's natural spline, a
//     brute-force inner product and two closed forms);
//   * static nested sampling with parallel (batched) constrained random walks,
//     Section 3 and Algorithm 1 of the paper;
//   * the gradient-informed constrained walk (Galilean Monte Carlo), driven by
//     dual-number derivatives in the unit cube.
//
// Parity status of the waveform: the Newtonian amplitude and phase, the
// antenna patterns, the inner product and the time/phase structure are pinned
// by closed forms and invariants in the tests; the non-spinning phase through
// 3.5PN and the 2PN spin-spin term by their published coefficients; the
// spin-orbit terms at 1.5, 2.5, 3 and 3.5PN by a stationary-phase derivation
// from the published spin-orbit binding energy and energy flux.
//
// Sums run in bin order with Neumaier compensation.  Built with -O3 and
// without -ffast-math.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTsun = 4.925490947e-6;       // G M_sun / c^3 [s]
constexpr double kC = 299792458.0;             // speed of light [m/s]
constexpr double kMpc = 3.085677581491367e22;  // [m]
constexpr double kGammaE = 0.5772156649015329; // Euler-Mascheroni constant

// ---------------------------------------------------------------------------
// Forward-mode dual numbers with N tangent directions.
// ---------------------------------------------------------------------------
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }  // NOLINT
};

inline double val(double x) { return x; }
template <int N> inline double val(const Dual<N>& x) { return x.v; }

template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r;
}
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r;
}
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
template <int N> Dual<N> operator+(const Dual<N>& a, double b) { Dual<N> r = a; r.v += b; return r; }
template <int N> Dual<N> operator+(double a, const Dual<N>& b) { return b + a; }
template <int N> Dual<N> operator-(const Dual<N>& a, double b) { Dual<N> r = a; r.v -= b; return r; }
template <int N> Dual<N> operator-(double a, const Dual<N>& b) { return (-b) + a; }
template <int N> Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r; r.v = a.v * b; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b; return r;
}
template <int N> Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N> Dual<N> operator/(const Dual<N>& a, double b) {
  Dual<N> r; r.v = a.v / b; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / b; return r;
}
template <int N> Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }

// f(a) with derivative df: value fv, derivative dfv.
template <int N> Dual<N> lift(const Dual<N>& a, double fv, double dfv) {
  Dual<N> r; r.v = fv; for (int i = 0; i < N; ++i) r.d[i] = dfv * a.d[i]; return r;
}
template <int N> Dual<N> sqrt(const Dual<N>& a) { double f = std::sqrt(a.v); return lift(a, f, 0.5 / f); }
template <int N> Dual<N> cbrt(const Dual<N>& a) { double f = std::cbrt(a.v); return lift(a, f, f / (3.0 * a.v)); }
template <int N> Dual<N> log(const Dual<N>& a) { return lift(a, std::log(a.v), 1.0 / a.v); }
template <int N> Dual<N> exp(const Dual<N>& a) { double f = std::exp(a.v); return lift(a, f, f); }
template <int N> Dual<N> sin(const Dual<N>& a) { return lift(a, std::sin(a.v), std::cos(a.v)); }
template <int N> Dual<N> cos(const Dual<N>& a) { return lift(a, std::cos(a.v), -std::sin(a.v)); }
template <int N> Dual<N> pow(const Dual<N>& a, double p) {
  return lift(a, std::pow(a.v, p), p * std::pow(a.v, p - 1.0));
}
template <int N> Dual<N> acos(const Dual<N>& a) { return lift(a, std::acos(a.v), -1.0 / std::sqrt(1.0 - a.v * a.v)); }
template <int N> Dual<N> asin(const Dual<N>& a) { return lift(a, std::asin(a.v), 1.0 / std::sqrt(1.0 - a.v * a.v)); }

using std::acos; using std::asin;
using std::cbrt; using std::cos; using std::exp; using std::log; using std::pow; using std::sin; using std::sqrt;

// ---------------------------------------------------------------------------
// Neumaier-compensated running sum (bin order).
// ---------------------------------------------------------------------------
template <class T>
struct NeumaierSum {
  T s{0.0}, c{0.0};
  void add(const T& x) {
    T t = s + x;
    if (std::fabs(val(s)) >= std::fabs(val(x))) c = c + ((s - t) + x);
    else c = c + ((x - t) + s);
    s = t;
  }
  T result() const { return s + c; }
};

// ---------------------------------------------------------------------------
// Event description (all host arrays, not owned).
// ---------------------------------------------------------------------------
struct Event {
  const double* freqs;   // [M] uniformly spaced, ascending
  int64_t M;
  const double* strain;  // [n_det][M][2] (re, im)
  const double* psd;     // [n_det][M] one-sided PSD
  const double* geom;    // [n_det][9]: vertex xyz [m], x-arm unit, y-arm unit
  int n_det;
  double gmst;           // [rad], Earth rotation ignored over the segment
  double t_ref;          // [s] from segment start; t_c is relative to it
  int fcut_mode;         // 0: h = 0 above f_ISCO; 1: no cut below f_high
};

inline double event_df(const Event& ev) {
  return (ev.freqs[ev.M - 1] - ev.freqs[0]) / double(ev.M - 1);
}

// Parameter order (11-D): Mc [Msun], q in (0,1], chi1z, chi2z, dL [Mpc],
// iota, psi, ra, dec [rad], tc [s rel. t_ref], phic [rad].
enum { P_MC, P_Q, P_CHI1, P_CHI2, P_DL, P_IOTA, P_PSI, P_RA, P_DEC, P_TC, P_PHIC, P_N };

// Antenna patterns and arrival delay for one detector (model reading):
// n = (cos dec cos lam, cos dec sin lam, sin dec), lam = ra - gmst;
// e_E = (-sin lam, cos lam, 0), e_N = (-sin dec cos lam, -sin dec sin lam, cos dec);
// X = cos psi e_E + sin psi e_N, Y = -sin psi e_E + cos psi e_N;
// e+ = XX - YY, ex = XY + YX; D = (xx - yy)/2; F+ = D:e+, Fx = D:ex;
// dt = -(r . n)/c.
template <class T>
void antenna(const double* g, const T& psi, const T& ra, const T& dec, double gmst,
             T* Fp, T* Fx, T* dt) {
  T lam = ra - gmst;
  T cl = cos(lam), sl = sin(lam), cd = cos(dec), sd = sin(dec);
  T cp = cos(psi), sp = sin(psi);
  T n[3] = {cd * cl, cd * sl, sd};
  T eE[3] = {-sl, cl, T(0.0)};
  T eN[3] = {-sd * cl, -sd * sl, cd};
  T X[3], Y[3];
  for (int i = 0; i < 3; ++i) { X[i] = cp * eE[i] + sp * eN[i]; Y[i] = -sp * eE[i] + cp * eN[i]; }
  const double* x = g + 3;
  const double* y = g + 6;
  T fp(0.0), fx(0.0);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      double Dik = 0.5 * (x[i] * x[k] - y[i] * y[k]);
      fp = fp + Dik * (X[i] * X[k] - Y[i] * Y[k]);
      fx = fx + Dik * (X[i] * Y[k] + Y[i] * X[k]);
    }
  *Fp = fp; *Fx = fx;
  *dt = -(g[0] * n[0] + g[1] * n[1] + g[2] * n[2]) / kC;
}

// TaylorF2 PN phase coefficients (aligned spins; Buonanno et al. 2009 Eq. 3.18
// non-spinning terms, leading spin-orbit and aligned spin-spin terms).
template <class T>
struct PNPhase {
  T eta, Ms;  // symmetric mass ratio, total mass [s]
  T p2, p3, p4, p5c, p6c, p7;
};

template <class T>
PNPhase<T> pn_phase(const T& Mc, const T& q, const T& chi1, const T& chi2) {
  PNPhase<T> P;
  T eta = q / ((1.0 + q) * (1.0 + q));
  T Mtot = Mc * pow(eta, -0.6);
  T delta = (1.0 - q) / (1.0 + q);            // = sqrt(1 - 4 eta) for q <= 1
  T m1 = 1.0 / (1.0 + q), m2 = q / (1.0 + q);  // component masses / M
  T chis = 0.5 * (chi1 + chi2), chia = 0.5 * (chi1 - chi2);
  P.eta = eta;
  P.Ms = Mtot * kTsun;
  P.p2 = (20.0 / 9.0) * (743.0 / 336.0 + 11.0 / 4.0 * eta);
  // 1.5PN: tail + spin-orbit beta = sum_i [(113/12)(m_i/M)^2 + (25/4) eta] chi_i
  T beta = ((113.0 / 12.0) * m1 * m1 + 25.0 / 4.0 * eta) * chi1 +
           ((113.0 / 12.0) * m2 * m2 + 25.0 / 4.0 * eta) * chi2;
  P.p3 = -16.0 * kPi + 4.0 * beta;
  // 2PN: point-particle + aligned spin-spin sigma = (79/8) eta chi1 chi2
  T sigma = (79.0 / 8.0) * eta * chi1 * chi2;
  P.p4 = 10.0 * (3058673.0 / 1016064.0 + 5429.0 / 1008.0 * eta + 617.0 / 144.0 * eta * eta) -
         10.0 * sigma;
  // 2.5PN: [pi(38645/756 - 65 eta/9) - gamma] (1 + 3 ln(v/v_lso))
  T gam = (732985.0 / 2268.0 - 24260.0 / 81.0 * eta - 340.0 / 9.0 * eta * eta) * chis +
          (732985.0 / 2268.0 + 140.0 / 9.0 * eta) * delta * chia;
  P.p5c = kPi * (38645.0 / 756.0 - 65.0 / 9.0 * eta) - gam;
  // 3PN: constant part; the -(6848/21) ln(4v) part is added per bin.
  P.p6c = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * kPi * kPi - 6848.0 / 21.0 * kGammaE +
          eta * (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * kPi * kPi) +
          76055.0 / 1728.0 * eta * eta - 127825.0 / 1296.0 * eta * eta * eta +
          kPi * (2270.0 / 3.0 * delta * chia + (2270.0 / 3.0 - 520.0 * eta) * chis);
  // 3.5PN: point-particle + spin-orbit
  P.p7 = kPi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta * eta) +
         (-25150083775.0 / 3048192.0 + 10566655595.0 / 762048.0 * eta -
          1042165.0 / 3024.0 * eta * eta + 5345.0 / 36.0 * eta * eta * eta) * chis +
         delta * (-25150083775.0 / 3048192.0 + 26804935.0 / 6048.0 * eta - 1985.0 / 48.0 * eta * eta) * chia;
  return P;
}

// Psi_PN(f) = 3/(128 eta v^5) sum_k phi_k v^k, v = (pi M f)^(1/3).
template <class T>
T pn_psi(const PNPhase<T>& P, double f) {
  const double vlso = 1.0 / std::sqrt(6.0);
  T v = cbrt(kPi * P.Ms * f);
  T v2 = v * v, v3 = v2 * v, v4 = v3 * v, v5 = v4 * v;
  T p5 = P.p5c * (1.0 + 3.0 * log(v / vlso));
  T p6 = P.p6c - 6848.0 / 21.0 * log(4.0 * v);
  T series = 1.0 + P.p2 * v2 + P.p3 * v3 + P.p4 * v4 + p5 * v5 + p6 * v5 * v + P.p7 * v5 * v2;
  return 3.0 / (128.0 * P.eta * v5) * series;
}

// Rows outside the physical domain (q not in (0,1], Mc <= 0, dL <= 0) or with a
// non-finite entry have lnL = -inf by definition of the interface.
template <class T>
bool physical(const T* th) {
  double q = val(th[P_Q]), mc = val(th[P_MC]), dl = val(th[P_DL]);
  bool ok = q > 0.0 && q <= 1.0 && mc > 0.0 && dl > 0.0;
  for (int k = 0; k < P_N; ++k) ok = ok && std::isfinite(val(th[k]));
  return ok;
}

// Upper frequency cut: f_ISCO = 1/(6^{3/2} pi M) in ISCO mode, otherwise +inf.
template <class T>
double f_cut(const Event& ev, const PNPhase<T>& P) {
  if (ev.fcut_mode != 0) return std::numeric_limits<double>::infinity();
  return 1.0 / (std::pow(6.0, 1.5) * kPi * val(P.Ms));
}

// Detector-projected strain h_d(f_j) at one bin, evaluated from the definition.
template <class T>
void strain_bin(const T* th, const PNPhase<T>& P, const T& amp, const T& Fp, const T& Fx,
                const T& dt, double t_ref, double f, T* hr, T* hi) {
  T ci = cos(th[P_IOTA]);
  T psi_full = 2.0 * kPi * f * (t_ref + th[P_TC] + dt) - th[P_PHIC] - kPi / 4.0 + pn_psi(P, f);
  T a = amp * pow(T(f), -7.0 / 6.0);  // A f^{-7/6}
  // h_d = a [F+ (1+cos^2 i)/2 - i Fx cos i] (cos Psi - i sin Psi)
  T pr = Fp * (1.0 + ci * ci) * 0.5;
  T pi = -(Fx * ci);
  T c = cos(psi_full), s = sin(psi_full);
  *hr = a * (pr * c + pi * s);
  *hi = a * (pi * c - pr * s);
}

template <class T>
T amplitude(const T* th) {
  // A = sqrt(5/24) pi^{-2/3} (Mc Tsun)^{5/6} c / dL
  return std::sqrt(5.0 / 24.0) * std::pow(kPi, -2.0 / 3.0) * pow(th[P_MC] * kTsun, 5.0 / 6.0) * kC /
         (th[P_DL] * kMpc);
}

template <class T>
T loglike_one(const Event& ev, const T* th) {
  if (!physical(th)) return T(-std::numeric_limits<double>::infinity());
  const double df = event_df(ev);
  PNPhase<T> P = pn_phase(th[P_MC], th[P_Q], th[P_CHI1], th[P_CHI2]);
  const double fc = f_cut(ev, P);
  T amp = amplitude(th);
  NeumaierSum<T> acc;
  for (int d = 0; d < ev.n_det; ++d) {
    T Fp, Fx, dt;
    antenna(ev.geom + 9 * d, th[P_PSI], th[P_RA], th[P_DEC], ev.gmst, &Fp, &Fx, &dt);
    const double* dd = ev.strain + 2 * ev.M * d;
    const double* S = ev.psd + ev.M * d;
    for (int64_t j = 0; j < ev.M; ++j) {
      const double f = ev.freqs[j];
      if (f > fc) break;  // h = 0 above the cut; bins ascend
      T hr, hi;
      strain_bin(th, P, amp, Fp, Fx, dt, ev.t_ref, f, &hr, &hi);
      const double w = 4.0 * df / S[j];
      // w [Re(conj(d) h) - |h|^2 / 2]
      T term = w * ((dd[2 * j] * hr + dd[2 * j + 1] * hi) - 0.5 * (hr * hr + hi * hi));
      acc.add(term);
    }
  }
  return acc.result();
}

// ---------------------------------------------------------------------------
// Calibration model (Section 2.2 of the paper: uncertainty in the calibration
// of each interferometer's data is modelled by amplitude and phase corrections
// at a set of frequency nodes, typically ten per interferometer, i.e. twenty
// parameters per detector).  The paper gives no functional form; the reading
// used here: the template seen by detector d is C_d(f) h_d(f) with
//   C_d(f) = (1 + dA_d(f)) exp(i dphi_d(f)),
// where dA_d and dphi_d (radians) are natural cubic splines in x = ln f
// through the node values (x_k = ln f_k, shared by all detectors); outside
// [x_0, x_{n-1}] the end cubics are continued.  Parameter layout after the 11
// source parameters: per detector d, dA at the n nodes, then dphi at the n nodes.
// ---------------------------------------------------------------------------

// Second derivatives m_k of the natural cubic spline through (x_k, y_k): the
// cubic pieces match in value, slope and curvature at the interior nodes and
// have zero curvature at both ends, which for k = 1 .. n-2 reads
//   h_{k-1} m_{k-1} + 2 (h_{k-1} + h_k) m_k + h_k m_{k+1}
//     = 6 [ (y_{k+1} - y_k) / h_k - (y_k - y_{k-1}) / h_{k-1} ],  h_k = x_{k+1} - x_k,
// with m_0 = m_{n-1} = 0.  The tridiagonal system is strictly diagonally
// dominant and is solved by forward elimination and back substitution.
template <class T>
void natural_spline(int n, const double* x, const T* y, T* m) {
  for (int k = 0; k < n; ++k) m[k] = T(0.0);
  if (n < 3) return;
  const int ni = n - 2;  // unknowns m_1 .. m_{n-2}
  std::vector<double> sub(ni), dia(ni), sup(ni);
  std::vector<T> rhs(ni);
  for (int i = 0; i < ni; ++i) {
    const int k = i + 1;
    const double hl = x[k] - x[k - 1], hr = x[k + 1] - x[k];
    sub[i] = hl;
    dia[i] = 2.0 * (hl + hr);
    sup[i] = hr;
    rhs[i] = 6.0 * ((y[k + 1] - y[k]) / hr - (y[k] - y[k - 1]) / hl);
  }
  for (int i = 1; i < ni; ++i) {
    const double w = sub[i] / dia[i - 1];
    dia[i] -= w * sup[i - 1];
    rhs[i] = rhs[i] - w * rhs[i - 1];
  }
  m[ni] = rhs[ni - 1] / dia[ni - 1];
  for (int i = ni - 2; i >= 0; --i) m[i + 1] = (rhs[i] - sup[i] * m[i + 2]) / dia[i];
}

// Value of the spline at xq: the piece of the interval [x_k, x_{k+1}] holding
// xq (the first or last piece outside the node range), in the standard form
// with A = (x_{k+1} - xq)/h, B = (xq - x_k)/h:
//   S = A y_k + B y_{k+1} + [(A^3 - A) m_k + (B^3 - B) m_{k+1}] h^2 / 6.
template <class T>
T spline_eval(int n, const double* x, const T* y, const T* m, double xq) {
  int k = 0;
  while (k < n - 2 && xq >= x[k + 1]) ++k;
  const double h = x[k + 1] - x[k];
  const double A = (x[k + 1] - xq) / h, B = (xq - x[k]) / h;
  return A * y[k] + B * y[k + 1] + ((A * A * A - A) * m[k] + (B * B * B - B) * m[k + 1]) * (h * h / 6.0);
}

// lnL of one parameter vector (11 source parameters, then the calibration
// node values) with the calibration factor applied per bin:
// lnL = sum_d sum_j 4 df / S_d,j [ Re(conj(d_j) C_j h_j) - |C_j h_j|^2 / 2 ].
// Templated like loglike_one: T = double for lnL, dual numbers for its
// gradient (the spline is linear in the node values, the factor C is not).
template <class T>
T loglike_cal_T(const Event& ev, const T* th, int nn, const double* xn) {
  using std::cos;
  using std::sin;
  if (!physical(th)) return T(-std::numeric_limits<double>::infinity());
  const double df = event_df(ev);
  PNPhase<T> P = pn_phase(th[P_MC], th[P_Q], th[P_CHI1], th[P_CHI2]);
  const double fc = f_cut(ev, P);
  const T amp = amplitude(th);
  std::vector<T> ma(nn), mp(nn);
  NeumaierSum<T> acc;
  for (int d = 0; d < ev.n_det; ++d) {
    const T* ya = th + P_N + 2 * nn * d;
    const T* yp = ya + nn;
    natural_spline(nn, xn, ya, ma.data());
    natural_spline(nn, xn, yp, mp.data());
    T Fp, Fx, dt;
    antenna(ev.geom + 9 * d, th[P_PSI], th[P_RA], th[P_DEC], ev.gmst, &Fp, &Fx, &dt);
    const double* dd = ev.strain + 2 * ev.M * d;
    const double* S = ev.psd + ev.M * d;
    for (int64_t j = 0; j < ev.M; ++j) {
      const double f = ev.freqs[j];
      if (f > fc) break;
      T hr, hi;
      strain_bin(th, P, amp, Fp, Fx, dt, ev.t_ref, f, &hr, &hi);
      const double x = std::log(f);
      const T dA = spline_eval(nn, xn, ya, ma.data(), x);
      const T dphi = spline_eval(nn, xn, yp, mp.data(), x);
      const T cr = (1.0 + dA) * cos(dphi), ci = (1.0 + dA) * sin(dphi);
      const T gr = cr * hr - ci * hi, gi = cr * hi + ci * hr;  // C h
      const double w = 4.0 * df / S[j];
      acc.add(w * ((dd[2 * j] * gr + dd[2 * j + 1] * gi) - 0.5 * (gr * gr + gi * gi)));
    }
  }
  return acc.result();
}

double loglike_cal_one(const Event& ev, const double* th, int nn, const double* xn) {
  return loglike_cal_T<double>(ev, th, nn, xn);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw 2011),
// written from its published definition: 10 rounds of the 4x32 S-P network
// with multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments
// 0x9E3779B9, 0xBB67AE85.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x[4]; };

U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = uint64_t(0xD2511F53u) * c.x[0];
    uint64_t p1 = uint64_t(0xCD9E8D57u) * c.x[2];
    uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
    U4 n;
    n.x[0] = hi1 ^ c.x[1] ^ k0;
    n.x[1] = lo1;
    n.x[2] = hi0 ^ c.x[3] ^ k1;
    n.x[3] = lo0;
    c = n;
  }
  return c;
}

// Random-walk stream layout shared by definition with the device sampler:
// key = (seed low word, seed high word); counter = (block, step, chain,
// call counter low word).  step 0 block 0 word 0 picks the start point; for
// step s >= 1, block b gives normals z[4b..4b+3] by Box-Muller on word pairs
// (w0,w1), (w2,w3): u1 = (w0 + 1) 2^-32 in (0,1], u2 = w1 2^-32,
// z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
void walk_normals(uint64_t seed, uint64_t counter, uint32_t chain, uint32_t step, int D, double* z) {
  const uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
  for (int b = 0; 4 * b < D; ++b) {
    U4 c{{uint32_t(b), step, chain, uint32_t(counter)}};
    U4 w = philox4x32_10(c, k0, k1);
    for (int h = 0; h < 2; ++h) {
      double u1 = (double(w.x[2 * h]) + 1.0) * 0x1p-32;
      double u2 = double(w.x[2 * h + 1]) * 0x1p-32;
      double r = std::sqrt(-2.0 * std::log(u1));
      int i0 = 4 * b + 2 * h;
      if (i0 < D) z[i0] = r * std::cos(2.0 * kPi * u2);
      if (i0 + 1 < D) z[i0 + 1] = r * std::sin(2.0 * kPi * u2);
    }
  }
}

uint32_t walk_start_word(uint64_t seed, uint64_t counter, uint32_t chain) {
  U4 c{{0u, 0u, chain, uint32_t(counter)}};
  return philox4x32_10(c, uint32_t(seed), uint32_t(seed >> 32)).x[0];
}

// ---------------------------------------------------------------------------
// Prior transform from the unit cube.
//   kind 0: uniform lo + u (hi - lo)
//   kind 1: uniform in volume [lo^3 + u (hi^3 - lo^3)]^{1/3}
//   kind 2: sine prior on [0, pi]: arccos(1 - 2u)
//   kind 3: cosine prior on [-pi/2, pi/2]: arcsin(2u - 1)
// ---------------------------------------------------------------------------
struct Sampling {
  int D;
  const int* param_map;   // [D] -> index into the 11-D theta
  const double* fixed;    // [11] values of the unsampled parameters
  const int* kind;        // [D]
  const double* lo;       // [D]
  const double* hi;       // [D]
  const int* periodic;    // [D]
};

template <typename T>
T prior_map(int kind, double lo, double hi, const T& u) {
  switch (kind) {
    case 1: return cbrt(lo * lo * lo + u * (hi * hi * hi - lo * lo * lo));
    case 2: return acos(1.0 - 2.0 * u);
    case 3: return asin(2.0 * u - 1.0);
    default: return lo + u * (hi - lo);
  }
}

template <typename T>
void unit_to_theta(const Sampling& s, const T* u, T* th) {
  for (int k = 0; k < P_N; ++k) th[k] = T(s.fixed[k]);
  for (int i = 0; i < s.D; ++i) th[s.param_map[i]] = prior_map(s.kind[i], s.lo[i], s.hi[i], u[i]);
}

double loglike_unit(const Event& ev, const Sampling& s, const double* u) {
  double th[P_N];
  unit_to_theta(s, u, th);
  return loglike_one<double>(ev, th);
}

// One constrained random walk (Algorithm 1's worker step with the fixed-length
// random-walk proposal): start at live point `start`, walk_len Gaussian steps
// u' = u + scale * L z in the unit cube; periodic coordinates wrap, any other
// coordinate outside [0,1] rejects the step; a step is accepted iff
// lnL(u') >= lnl_star.
using UnitLike = std::function<double(const double*)>;

void random_walk(const UnitLike& like, const int* periodic, int D, const double* u0, double l0,
                 double lnl_star, uint64_t seed, uint64_t counter, uint32_t chain, int walk_len,
                 double scale, const double* chol, double* u_out, double* l_out, int32_t* nacc_out) {
  std::vector<double> u(u0, u0 + D), up(D), z(D);
  double l = l0;
  int32_t nacc = 0;
  for (int st = 1; st <= walk_len; ++st) {
    walk_normals(seed, counter, chain, uint32_t(st), D, z.data());
    bool inside = true;
    for (int i = 0; i < D; ++i) {
      double dz = 0.0;
      for (int k = 0; k <= i; ++k) dz += chol[i * D + k] * z[k];
      double x = u[i] + scale * dz;
      if (periodic[i]) x -= std::floor(x);
      else if (x < 0.0 || x > 1.0) inside = false;
      up[i] = x;
    }
    if (!inside) continue;
    double lp = like(up.data());
    if (lp >= lnl_star) { u = up; l = lp; ++nacc; }
  }
  std::copy(u.begin(), u.end(), u_out);
  *l_out = l;
  *nacc_out = nacc;
}

// Gradient-informed constrained walk: Galilean Monte Carlo (Skilling 2012),
// with the velocity drawn from the random walk's proposal distribution and
// reflections taken in that distribution's own metric.  The chain carries a
// velocity, initially v = scale * L z (z: the normals of step word
// 0x40000000), and from step 2 on partly refreshed before the step,
//   v <- rho v + sqrt(1 - rho^2) scale L z  (z: the normals of the step's word),
// an autoregressive move that keeps N(0, scale^2 L L^T).  With Sigma = L L^T,
// a reflection of v off a surface of normal g is
//   v' = v - 2 (v.g) / (g.Sigma g) Sigma g,
// which keeps v^T Sigma^-1 v (so the velocity distribution) and undoes itself.
// Each step tries x1 = u + v (periodic coordinates wrap):
//   * x1 inside the cube with lnL(x1) >= L*: move to x1, keep v;
//   * otherwise reflect at x1 -- off the likelihood contour (g = d lnL / du at
//     x1) when x1 is inside the cube, off the walls it crossed when it is not
//     (g = the outward unit normals of those walls summed) -- and try
//     x2 = x1 + v'; inside the cube with lnL(x2) >= L*: move to x2 with v';
//   * otherwise stay and reverse the velocity, v <- -v.
// The normal depends on x1 alone, so the map (u, v) -> (u', -v') is an
// involution and preserves volume: the uniform distribution inside the
// contour times the velocity distribution is left invariant.
using UnitLikeGrad = std::function<double(const double*, double*)>;  // lnL(u), writes d lnL / du

void galilean_walk(const UnitLike& like, const UnitLikeGrad& like_grad, const int* periodic, int D,
                   const double* u0, double l0, double lnl_star, uint64_t seed, uint64_t counter,
                   uint32_t chain, int walk_len, double scale, double rho, const double* chol, double* u_out,
                   double* l_out, int32_t* nacc_out) {
  std::vector<double> u(u0, u0 + D), v(D), z(D), x1(D), x2(D), g(D), sg(D), v2(D), sigma(D * D, 0.0);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j)
      for (int k = 0; k < D; ++k) sigma[i * D + j] += chol[i * D + k] * chol[j * D + k];
  walk_normals(seed, counter, chain, 0x40000000u, D, z.data());
  for (int i = 0; i < D; ++i) {
    double dz = 0.0;
    for (int k = 0; k <= i; ++k) dz += chol[i * D + k] * z[k];
    v[i] = scale * dz;
  }
  auto step_to = [&](const std::vector<double>& from, const std::vector<double>& vel, std::vector<double>& to) {
    bool inside = true;
    for (int i = 0; i < D; ++i) {
      double x = from[i] + vel[i];
      if (periodic[i]) x -= std::floor(x);
      else if (x < 0.0 || x > 1.0) inside = false;
      to[i] = x;
    }
    return inside;
  };
  double l = l0;
  int32_t nacc = 0;
  for (int st = 1; st <= walk_len; ++st) {
    if (st > 1 && rho < 1.0) {
      walk_normals(seed, counter, chain, uint32_t(st), D, z.data());
      for (int i = 0; i < D; ++i) {
        double dz = 0.0;
        for (int k = 0; k <= i; ++k) dz += chol[i * D + k] * z[k];
        v[i] = rho * v[i] + std::sqrt(1.0 - rho * rho) * scale * dz;
      }
    }
    if (step_to(u, v, x1)) {
      const double l1 = like_grad(x1.data(), g.data());
      if (l1 >= lnl_star) { u = x1; l = l1; ++nacc; continue; }
    } else {
      for (int i = 0; i < D; ++i) g[i] = (!periodic[i] && x1[i] > 1.0) ? 1.0 : (!periodic[i] && x1[i] < 0.0) ? -1.0 : 0.0;
    }
    double gsg = 0.0, vg = 0.0;
    for (int i = 0; i < D; ++i) {
      sg[i] = 0.0;
      for (int j = 0; j < D; ++j) sg[i] += sigma[i * D + j] * g[j];
      gsg += g[i] * sg[i];
      vg += v[i] * g[i];
    }
    bool moved = false;
    if (gsg > 0.0 && std::isfinite(gsg) && std::isfinite(vg)) {
      for (int i = 0; i < D; ++i) v2[i] = v[i] - 2.0 * vg / gsg * sg[i];
      if (step_to(x1, v2, x2)) {
        const double l2 = like(x2.data());
        if (l2 >= lnl_star) { u = x2; l = l2; v = v2; ++nacc; moved = true; }
      }
    }
    if (!moved)
      for (int i = 0; i < D; ++i) v[i] = -v[i];
  }
  std::copy(u.begin(), u.end(), u_out);
  *l_out = l;
  *nacc_out = nacc;
}

int pick_start(uint64_t seed, uint64_t counter, uint32_t chain, int64_t K, int64_t worst) {
  // Uniform over the K-1 live points other than the worst (exact integer map).
  uint32_t w = walk_start_word(seed, counter, chain);
  int64_t idx = int64_t((uint64_t(w) * uint64_t(K - 1)) >> 32);
  return int(idx < worst ? idx : idx + 1);
}

double logaddexp(double a, double b) {
  if (a == -std::numeric_limits<double>::infinity()) return b;
  if (b == -std::numeric_limits<double>::infinity()) return a;
  double m = std::max(a, b);
  return m + std::log(std::exp(a - m) + std::exp(b - m));
}

// Plain Cholesky of a symmetric positive-definite D x D matrix (row-major,
// lower triangle written; upper zeroed).  Returns false if not SPD.
bool cholesky(std::vector<double>& A, int D) {
  for (int j = 0; j < D; ++j) {
    double s = A[j * D + j];
    for (int k = 0; k < j; ++k) s -= A[j * D + k] * A[j * D + k];
    if (!(s > 0.0)) return false;
    A[j * D + j] = std::sqrt(s);
    for (int i = j + 1; i < D; ++i) {
      double t = A[i * D + j];
      for (int k = 0; k < j; ++k) t -= A[i * D + k] * A[j * D + k];
      A[i * D + j] = t / A[j * D + j];
    }
    for (int k = j + 1; k < D; ++k) A[j * D + k] = 0.0;
  }
  return true;
}

}  // namespace

// ===========================================================================
// C interface (ctypes).
// ===========================================================================
extern "C" {

// Per-bin strain h_d(f_j) of one 11-D parameter vector -> h[n_det][M][2].
int oracle_waveform(const double* freqs, int64_t M, const double* geom, int n_det, double gmst,
                    double t_ref, int fcut_mode, const double* theta, double* h) {
  Event ev{freqs, M, nullptr, nullptr, geom, n_det, gmst, t_ref, fcut_mode};
  std::memset(h, 0, sizeof(double) * 2 * M * n_det);
  if (!physical(theta)) return -1;
  PNPhase<double> P = pn_phase(theta[P_MC], theta[P_Q], theta[P_CHI1], theta[P_CHI2]);
  const double fc = f_cut(ev, P);
  double amp = amplitude(theta);
  for (int d = 0; d < n_det; ++d) {
    double Fp, Fx, dt;
    antenna(geom + 9 * d, theta[P_PSI], theta[P_RA], theta[P_DEC], gmst, &Fp, &Fx, &dt);
    for (int64_t j = 0; j < M; ++j) {
      if (freqs[j] > fc) break;
      strain_bin(theta, P, amp, Fp, Fx, dt, t_ref, freqs[j], &h[2 * (M * d + j)],
                 &h[2 * (M * d + j) + 1]);
    }
  }
  return 0;
}

// Antenna patterns F+, Fx and delay dt for each detector -> out[n_det][3].
void oracle_antenna(const double* geom, int n_det, double gmst, double psi, double ra, double dec,
                    double* out) {
  for (int d = 0; d < n_det; ++d) antenna(geom + 9 * d, psi, ra, dec, gmst, &out[3 * d], &out[3 * d + 1], &out[3 * d + 2]);
}

// PN phase Psi_PN(f) [rad] and f_ISCO for one intrinsic point (test hook).
double oracle_pn_psi(double Mc, double q, double chi1, double chi2, double f) {
  return pn_psi(pn_phase(Mc, q, chi1, chi2), f);
}

// Batched lnL of B full 11-D parameter vectors theta[B][11] -> lnl[B].
int oracle_loglike(const double* freqs, int64_t M, const double* strain, const double* psd,
                   const double* geom, int n_det, double gmst, double t_ref, int fcut_mode,
                   const double* theta, int64_t B, double* lnl, int n_threads) {
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t b = 0; b < B; ++b) lnl[b] = loglike_one<double>(ev, theta + P_N * b);
  return 0;
}

// Batched lnL with the calibration model: theta[B][11 + 2 n_nodes n_det]
// (source parameters, then per detector dA and dphi at the nodes), node
// frequencies node_f[n_nodes] ascending -> lnl[B].
int oracle_loglike_cal(const double* freqs, int64_t M, const double* strain, const double* psd,
                       const double* geom, int n_det, double gmst, double t_ref, int fcut_mode, int n_nodes,
                       const double* node_f, const double* theta, int64_t B, double* lnl, int n_threads) {
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
  if (n_nodes < 2) return -1;
  std::vector<double> xn(n_nodes);
  for (int k = 0; k < n_nodes; ++k) xn[k] = std::log(node_f[k]);
  const int64_t D = P_N + 2 * (int64_t)n_nodes * n_det;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t b = 0; b < B; ++b) lnl[b] = loglike_cal_one(ev, theta + D * b, n_nodes, xn.data());
  return 0;
}

// Natural cubic spline through (x[n], y[n]) evaluated at xq[nq] -> out[nq] (test hook).
void oracle_cal_spline(int n, const double* x, const double* y, int64_t nq, const double* xq, double* out) {
  std::vector<double> m(n);
  natural_spline(n, x, y, m.data());
  for (int64_t i = 0; i < nq; ++i) out[i] = spline_eval(n, x, y, m.data(), xq[i]);
}

// Batched lnL and its gradient with respect to all 11 parameters by
// forward-mode dual numbers -> lnl[B], grad[B][11].
int oracle_grad(const double* freqs, int64_t M, const double* strain, const double* psd,
                const double* geom, int n_det, double gmst, double t_ref, int fcut_mode,
                const double* theta, int64_t B, double* lnl, double* grad, int n_threads) {
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t b = 0; b < B; ++b) {
    Dual<P_N> th[P_N];
    for (int k = 0; k < P_N; ++k) { th[k] = Dual<P_N>(theta[P_N * b + k]); th[k].d[k] = 1.0; }
    Dual<P_N> r = loglike_one<Dual<P_N>>(ev, th);
    lnl[b] = r.v;
    for (int k = 0; k < P_N; ++k) grad[P_N * b + k] = std::isfinite(r.v) ? r.d[k] : 0.0;
  }
  return 0;
}

// Batched lnL with the calibration model and its gradient with respect to all
// D = 11 + 2 n_nodes n_det parameters (theta's layout) by forward-mode dual
// numbers, sixteen directions per pass -> lnl[B], grad[B][D].
int oracle_grad_cal(const double* freqs, int64_t M, const double* strain, const double* psd,
                    const double* geom, int n_det, double gmst, double t_ref, int fcut_mode, int n_nodes,
                    const double* node_f, const double* theta, int64_t B, double* lnl, double* grad,
                    int n_threads) {
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
  if (n_nodes < 2) return -1;
  std::vector<double> xn(n_nodes);
  for (int k = 0; k < n_nodes; ++k) xn[k] = std::log(node_f[k]);
  const int64_t D = P_N + 2 * (int64_t)n_nodes * n_det;
  constexpr int NT = 16;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t b = 0; b < B; ++b) {
    std::vector<Dual<NT>> th(D);
    for (int64_t c0 = 0; c0 < D; c0 += NT) {
      for (int64_t k = 0; k < D; ++k) {
        th[k] = Dual<NT>(theta[D * b + k]);
        if (k >= c0 && k < c0 + NT) th[k].d[k - c0] = 1.0;
      }
      const Dual<NT> r = loglike_cal_T<Dual<NT>>(ev, th.data(), n_nodes, xn.data());
      lnl[b] = r.v;
      for (int64_t k = c0; k < D && k < c0 + NT; ++k) grad[D * b + k] = std::isfinite(r.v) ? r.d[k - c0] : 0.0;
    }
  }
  return 0;
}

// Philox4x32-10 block (test hook).
void oracle_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  U4 c{{ctr[0], ctr[1], ctr[2], ctr[3]}};
  U4 r = philox4x32_10(c, key[0], key[1]);
  for (int i = 0; i < 4; ++i) out[i] = r.x[i];
}

// Unit-cube -> parameter transform of n points u[n][D] -> theta[n][11].
void oracle_prior_transform(int D, const int* param_map, const double* fixed, const int* kind,
                            const double* lo, const double* hi, const int* periodic,
                            const double* u, int64_t n, double* theta) {
  Sampling s{D, param_map, fixed, kind, lo, hi, periodic};
  for (int64_t i = 0; i < n; ++i) unit_to_theta(s, u + D * i, theta + P_N * i);
}

}  // extern "C"

namespace {

void ns_replace_impl(const UnitLike& like, int D, const int* periodic, const double* live_u,
                     const double* live_lnl, int64_t K, int64_t worst, double lnl_star, uint64_t seed,
                     uint64_t counter, int64_t n_chains, int walk_len, double scale,
                     const double* chol, double* out_u, double* out_lnl, int32_t* out_nacc,
                     int32_t* out_start, int n_threads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t b = 0; b < n_chains; ++b) {
    int st = pick_start(seed, counter, uint32_t(b), K, worst);
    if (out_start) out_start[b] = st;
    random_walk(like, periodic, D, live_u + D * st, live_lnl[st], lnl_star, seed, counter,
                uint32_t(b), walk_len, scale, chol, out_u + D * b, &out_lnl[b], &out_nacc[b]);
  }
}

// Static parallel nested sampling (Section 3, Algorithm 1), written plainly.
//   init: K prior draws (uniform in the unit cube; Philox words with step
//     word 0xFFFFFFFF, chain word = live index, call word 0xFFFFFFFF);
//   each round r: L* = min live lnL; Cholesky factor of the live-set
//     covariance in the unit cube; n_chains constrained random walks
//     (ns_replace semantics, call counter r); consumption: repeatedly take the
//     current worst live point, find the next unused candidate (generation
//     order) with lnL > that worst value -- candidates that fail are
//     discarded -- move the worst to the dead list and put the candidate in
//     its place; the round ends when candidates run out;
//   prior volume ln X_i = -i/K, weights dX_i = X_{i-1} - X_i, lnZ by
//     logaddexp; scale <- scale exp(acceptance - 1/2) clamped to [1e-3, 1];
//   stop when ln(Z + Lmax X) - ln Z < dlogz or after max_rounds rounds;
//   the final K live points are added in ascending order with equal prior
//   volume X_N / (K+1) each.
// res[0]=lnZ, res[1]=sqrt(H/K), res[2]=H, res[3]=n_dead, res[4]=n_proposals,
// res[5]=rounds, res[6]=last scale, res[7]=mean acceptance,
// res[8]=mean candidates consumed per round.
void ns_run_impl(const UnitLike& like, int D, const int* periodic, int64_t K, int64_t n_chains,
                 int walk_len, uint64_t seed, double dlogz, int64_t max_rounds, double scale0,
                 double* res, double* dead_lnl, double* dead_logwt, double* dead_u, int64_t max_dead,
                 int n_threads) {
  const double ninf = -std::numeric_limits<double>::infinity();
  std::vector<double> lu(K * D), ll(K);
  for (int64_t k = 0; k < K; ++k)
    for (int b = 0; 4 * b < D; ++b) {
      U4 c{{uint32_t(b), 0xFFFFFFFFu, uint32_t(k), 0xFFFFFFFFu}};
      U4 w = philox4x32_10(c, uint32_t(seed), uint32_t(seed >> 32));
      for (int i = 0; i < 4 && 4 * b + i < D; ++i)
        lu[k * D + 4 * b + i] = (double(w.x[i]) + 0.5) * 0x1p-32;
    }
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t k = 0; k < K; ++k) ll[k] = like(&lu[k * D]);
  int64_t n_prop = K;

  std::vector<double> dl, dw, du;
  double lnZ = ninf;
  int64_t it = 0;
  double scale = scale0, acc_sum = 0.0;
  int64_t rounds = 0, consumed = 0;
  std::vector<double> cu(n_chains * D), cl(n_chains), chol(D * D);
  std::vector<int32_t> cn(n_chains);
  const double log1m = std::log1p(-std::exp(-1.0 / double(K)));
  while (rounds < max_rounds) {
    int64_t worst = int64_t(std::min_element(ll.begin(), ll.end()) - ll.begin());
    double lstar = ll[worst];
    std::vector<double> mean(D, 0.0), cov(D * D, 0.0);
    for (int64_t k = 0; k < K; ++k)
      for (int i = 0; i < D; ++i) mean[i] += lu[k * D + i] / double(K);
    for (int64_t k = 0; k < K; ++k)
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j)
          cov[i * D + j] += (lu[k * D + i] - mean[i]) * (lu[k * D + j] - mean[j]) / double(K - 1);
    chol = cov;
    if (!cholesky(chol, D)) {
      std::fill(chol.begin(), chol.end(), 0.0);
      for (int i = 0; i < D; ++i) chol[i * D + i] = std::sqrt(std::max(cov[i * D + i], 1e-300));
    }
    ns_replace_impl(like, D, periodic, lu.data(), ll.data(), K, worst, lstar, seed,
                    uint64_t(rounds), n_chains, walk_len, scale, chol.data(), cu.data(), cl.data(),
                    cn.data(), nullptr, n_threads);
    ++rounds;
    n_prop += n_chains * walk_len;
    int64_t tot_acc = 0;
    for (int64_t b = 0; b < n_chains; ++b) tot_acc += cn[b];
    double acc = double(tot_acc) / double(n_chains * walk_len);
    acc_sum += acc;
    int64_t ptr = 0;
    while (true) {
      int64_t w = int64_t(std::min_element(ll.begin(), ll.end()) - ll.begin());
      double lmin = ll[w];
      while (ptr < n_chains && !(cl[ptr] > lmin)) ++ptr;
      if (ptr >= n_chains) break;
      ++it;
      double lw = -double(it - 1) / double(K) + log1m;  // ln(X_{i-1} - X_i)
      dl.push_back(lmin); dw.push_back(lw);
      du.insert(du.end(), &lu[w * D], &lu[w * D] + D);
      lnZ = logaddexp(lnZ, lmin + lw);
      std::copy(&cu[ptr * D], &cu[ptr * D] + D, &lu[w * D]);
      ll[w] = cl[ptr];
      ++ptr;
      ++consumed;
    }
    scale = std::min(1.0, std::max(1e-3, scale * std::exp(acc - 0.5)));
    double lmax = *std::max_element(ll.begin(), ll.end());
    double lnX = -double(it) / double(K);
    if (logaddexp(lnZ, lmax + lnX) - lnZ < dlogz) break;
  }
  std::vector<int64_t> order(K);
  for (int64_t k = 0; k < K; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return ll[a] < ll[b]; });
  double lw_final = -double(it) / double(K) - std::log(double(K + 1));
  for (int64_t k = 0; k < K; ++k) {
    dl.push_back(ll[order[k]]); dw.push_back(lw_final);
    du.insert(du.end(), &lu[order[k] * D], &lu[order[k] * D] + D);
    lnZ = logaddexp(lnZ, ll[order[k]] + lw_final);
  }
  double H = 0.0;
  for (size_t i = 0; i < dl.size(); ++i) {
    double p = std::exp(dl[i] + dw[i] - lnZ);
    if (p > 0.0) H += p * (dl[i] - lnZ);
  }
  res[0] = lnZ; res[1] = std::sqrt(std::max(H, 0.0) / double(K)); res[2] = H;
  res[3] = double(dl.size()); res[4] = double(n_prop); res[5] = double(rounds); res[6] = scale;
  res[7] = rounds > 0 ? acc_sum / double(rounds) : 0.0;
  res[8] = rounds > 0 ? double(consumed) / double(rounds) : 0.0;
  int64_t nd = std::min<int64_t>(max_dead, int64_t(dl.size()));
  for (int64_t i = 0; i < nd; ++i) {
    if (dead_lnl) dead_lnl[i] = dl[i];
    if (dead_logwt) dead_logwt[i] = dw[i];
    if (dead_u) std::copy(&du[i * D], &du[i * D] + D, dead_u + i * D);
  }
}

// Analytic test likelihood: isotropic Gaussian N(mu, sigma^2 I) on the unit
// cube with a uniform prior, lnL = -1/2 |u - mu|^2 / sigma^2 - D ln(sigma sqrt(2 pi)).
UnitLike gauss_like(int D, const double* mu, double sigma) {
  std::vector<double> m(mu, mu + D);
  return [m, D, sigma](const double* u) {
    double s = 0.0;
    for (int i = 0; i < D; ++i) { double t = (u[i] - m[i]) / sigma; s += t * t; }
    return -0.5 * s - D * std::log(sigma * std::sqrt(2.0 * kPi));
  };
}

// Phi^{-1}(u) for the standard normal: the root of Phi(x) = u, bracketed by
// bisection and polished by Newton steps x <- x - F(x) / phi(x) until they
// stop shrinking.  u > 1/2 uses Phi^{-1}(u) = -Phi^{-1}(1 - u) (1 - u is exact
// there), so the root is negative; F is written so that it has no rounding
// floor near the root: F(x) = erfc(-x / sqrt 2) / 2 - p in the tail (p < 1/4),
// and F(x) = erf(x / sqrt 2) / 2 - (p - 1/2) near the centre (p - 1/2 is
// exact for p >= 1/4, and erf is accurate relative to its small values).
double inv_normal_cdf(double u) {
  if (!(u > 0.0)) return -std::numeric_limits<double>::infinity();
  if (!(u < 1.0)) return std::numeric_limits<double>::infinity();
  if (u == 0.5) return 0.0;
  const bool upper = u > 0.5;
  const double p = upper ? 1.0 - u : u;  // in (0, 1/2): the root is negative
  const bool centre = p >= 0.25;
  const double pc = p - 0.5;
  auto F = [centre, p, pc](double x) {
    return centre ? 0.5 * std::erf(x / std::sqrt(2.0)) - pc : 0.5 * std::erfc(-x / std::sqrt(2.0)) - p;
  };
  double a = -40.0, b = 0.0;
  for (int i = 0; i < 40; ++i) {
    const double m = 0.5 * (a + b);
    if (F(m) < 0.0) a = m;
    else b = m;
  }
  double x = 0.5 * (a + b), step = 1.0;
  for (int i = 0; i < 50; ++i) {
    const double phi = std::exp(-0.5 * x * x) / std::sqrt(2.0 * kPi);
    const double nx = x - F(x) / phi;
    const double ns = std::fabs(nx - x);
    if (!(ns < step)) break;  // no longer converging: at the rounding floor
    step = ns;
    x = nx;
    if (ns == 0.0) break;
  }
  return upper ? -x : x;
}

// The calibrated likelihood of unit-cube points: the first s.D coordinates
// through the source prior, the next 2 nn n_det through zero-mean Gaussian
// priors of width sig[0] (amplitude) and sig[1] (phase), per detector nn
// amplitude then nn phase corrections.
UnitLike cal_like(const Event& ev, const Sampling& s, int nn, const double* node_f, const double* sig) {
  std::vector<double> xn(nn);
  for (int k = 0; k < nn; ++k) xn[k] = std::log(node_f[k]);
  const int nc = 2 * nn * ev.n_det;
  const double sa = sig[0], sp = sig[1];
  return [ev, s, nn, xn, nc, sa, sp](const double* u) {
    std::vector<double> th(P_N + nc);
    unit_to_theta(s, u, th.data());
    for (int c = 0; c < nc; ++c) th[P_N + c] = ((c / nn) % 2 ? sp : sa) * inv_normal_cdf(u[s.D + c]);
    return loglike_cal_one(ev, th.data(), nn, xn.data());
  };
}

UnitLike gw_like(const Event& ev, const Sampling& s) {
  return [ev, s](const double* u) { return loglike_unit(ev, s, u); };
}

// lnL of a unit-cube point and its derivatives with respect to the unit-cube
// coordinates: dual numbers seeded on u and carried through the prior maps
// (and, with the calibration model, through theta = sigma Phi^{-1}(u), whose
// derivative is sigma / phi(Phi^{-1}(u))), sixteen directions per pass.
UnitLikeGrad gw_like_grad(const Event& ev, const Sampling& s) {
  return [ev, s](const double* u, double* g) {
    using DT = Dual<P_N>;
    DT uu[P_N], th[P_N];
    for (int i = 0; i < s.D; ++i) {
      uu[i] = DT(u[i]);
      uu[i].d[i] = 1.0;
    }
    unit_to_theta(s, uu, th);
    const DT r = loglike_one<DT>(ev, th);
    for (int i = 0; i < s.D; ++i) g[i] = r.d[i];
    return r.v;
  };
}

UnitLikeGrad cal_like_grad(const Event& ev, const Sampling& s, int nn, const double* node_f, const double* sig) {
  std::vector<double> xn(nn);
  for (int k = 0; k < nn; ++k) xn[k] = std::log(node_f[k]);
  const int nc = 2 * nn * ev.n_det;
  const double sa = sig[0], sp = sig[1];
  return [ev, s, nn, xn, nc, sa, sp](const double* u, double* g) {
    constexpr int NT = 16;
    using DT = Dual<NT>;
    const int Dw = s.D + nc;
    std::vector<DT> uu(s.D), th(P_N + nc);
    double val = 0.0;
    for (int c0 = 0; c0 < Dw; c0 += NT) {
      auto seeded = [&](int k, double x) {
        DT t(x);
        if (k >= c0 && k < c0 + NT) t.d[k - c0] = 1.0;
        return t;
      };
      for (int i = 0; i < s.D; ++i) uu[i] = seeded(i, u[i]);
      unit_to_theta(s, uu.data(), th.data());
      for (int c = 0; c < nc; ++c) {
        const double sg = (c / nn) % 2 ? sp : sa, z = inv_normal_cdf(u[s.D + c]);
        th[P_N + c] = lift(seeded(s.D + c, u[s.D + c]), sg * z, sg * std::sqrt(2.0 * kPi) * std::exp(0.5 * z * z));
      }
      const DT r = loglike_cal_T<DT>(ev, th.data(), nn, xn.data());
      val = r.v;
      for (int k = c0; k < Dw && k < c0 + NT; ++k) g[k] = r.d[k - c0];
    }
    return val;
  };
}

UnitLikeGrad gauss_like_grad(int D, const double* mu, double sigma) {
  std::vector<double> m(mu, mu + D);
  const UnitLike f = gauss_like(D, mu, sigma);
  return [m, D, sigma, f](const double* u, double* g) {
    for (int i = 0; i < D; ++i) g[i] = -(u[i] - m[i]) / (sigma * sigma);
    return f(u);
  };
}

void gmc_replace_impl(const UnitLike& like, const UnitLikeGrad& like_grad, int D, const int* periodic,
                      const double* live_u, const double* live_lnl, int64_t K, int64_t worst, double lnl_star,
                      uint64_t seed, uint64_t counter, int64_t n_chains, int walk_len, double scale, double rho,
                      const double* chol, double* out_u, double* out_lnl, int32_t* out_nacc, int32_t* out_start,
                      int n_threads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t b = 0; b < n_chains; ++b) {
    int st = pick_start(seed, counter, uint32_t(b), K, worst);
    if (out_start) out_start[b] = st;
    galilean_walk(like, like_grad, periodic, D, live_u + D * st, live_lnl[st], lnl_star, seed, counter,
                  uint32_t(b), walk_len, scale, rho, chol, out_u + D * b, &out_lnl[b], &out_nacc[b]);
  }
}

}  // namespace

extern "C" {

// Batched constrained random walks with the same semantics and random stream
// as the device sampler: n_chains chains, each started at a live point other
// than `worst`, walk_len steps, accept iff lnL >= lnl_star.
int oracle_ns_replace(const double* freqs, int64_t M, const double* strain, const double* psd,
                      const double* geom, int n_det, double gmst, double t_ref, int fcut_mode,
                      int D, const int* param_map, const double* fixed, const int* kind,
                      const double* lo, const double* hi, const int* periodic,
                      const double* live_u, const double* live_lnl, int64_t K, int64_t worst,
                      double lnl_star, uint64_t seed, uint64_t counter, int64_t n_chains,
                      int walk_len, double scale, const double* chol, double* out_u,
                      double* out_lnl, int32_t* out_nacc, int32_t* out_start, int n_threads) {
  if (K < 2 || worst < 0 || worst >= K) return -1;
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
  Sampling s{D, param_map, fixed, kind, lo, hi, periodic};
  ns_replace_impl(gw_like(ev, s), D, periodic, live_u, live_lnl, K, worst, lnl_star, seed, counter,
                  n_chains, walk_len, scale, chol, out_u, out_lnl, out_nacc, out_start, n_threads);
  return 0;
}

int oracle_ns_run(const double* freqs, int64_t M, const double* strain, const double* psd,
                  const double* geom, int n_det, double gmst, double t_ref, int fcut_mode, int D,
                  const int* param_map, const double* fixed, const int* kind, const double* lo,
                  const double* hi, const int* periodic, int64_t K, int64_t n_chains, int walk_len,
                  uint64_t seed, double dlogz, int64_t max_rounds, double scale0, double* res,
                  double* dead_lnl, double* dead_logwt, double* dead_u, int64_t max_dead,
                  int n_threads) {
  if (K < 2 || D < 1) return -1;
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
  Sampling s{D, param_map, fixed, kind, lo, hi, periodic};
  ns_run_impl(gw_like(ev, s), D, periodic, K, n_chains, walk_len, seed, dlogz, max_rounds, scale0,
              res, dead_lnl, dead_logwt, dead_u, max_dead, n_threads);
  return 0;
}

// ns_replace / ns_run with the calibration model: the walk coordinates are the
// D sampled source coordinates followed by 2 n_nodes n_det calibration
// coordinates (Gaussian priors of widths sig[2]); live_u, chol and out_u use
// that dimension.
int oracle_ns_replace_cal(const double* freqs, int64_t M, const double* strain, const double* psd,
                          const double* geom, int n_det, double gmst, double t_ref, int fcut_mode,
                          int D, const int* param_map, const double* fixed, const int* kind,
                          const double* lo, const double* hi, const int* periodic, int n_nodes,
                          const double* node_f, const double* sig, const double* live_u,
                          const double* live_lnl, int64_t K, int64_t worst, double lnl_star,
                          uint64_t seed, uint64_t counter, int64_t n_chains, int walk_len,
                          double scale, const double* chol, double* out_u, double* out_lnl,
                          int32_t* out_nacc, int32_t* out_start, int n_threads) {
  if (K < 2 || worst < 0 || worst >= K || n_nodes < 2) return -1;
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
  Sampling s{D, param_map, fixed, kind, lo, hi, periodic};
  const int Dw = D + 2 * n_nodes * n_det;
  std::vector<int> per(Dw, 0);
  for (int i = 0; i < D; ++i) per[i] = periodic[i];
  ns_replace_impl(cal_like(ev, s, n_nodes, node_f, sig), Dw, per.data(), live_u, live_lnl, K, worst,
                  lnl_star, seed, counter, n_chains, walk_len, scale, chol, out_u, out_lnl, out_nacc,
                  out_start, n_threads);
  return 0;
}

int oracle_ns_run_cal(const double* freqs, int64_t M, const double* strain, const double* psd,
                      const double* geom, int n_det, double gmst, double t_ref, int fcut_mode, int D,
                      const int* param_map, const double* fixed, const int* kind, const double* lo,
                      const double* hi, const int* periodic, int n_nodes, const double* node_f,
                      const double* sig, int64_t K, int64_t n_chains, int walk_len, uint64_t seed,
                      double dlogz, int64_t max_rounds, double scale0, double* res, int n_threads) {
  if (K < 2 || D < 1 || n_nodes < 2) return -1;
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
  Sampling s{D, param_map, fixed, kind, lo, hi, periodic};
  const int Dw = D + 2 * n_nodes * n_det;
  std::vector<int> per(Dw, 0);
  for (int i = 0; i < D; ++i) per[i] = periodic[i];
  ns_run_impl(cal_like(ev, s, n_nodes, node_f, sig), Dw, per.data(), K, n_chains, walk_len, seed, dlogz,
              max_rounds, scale0, res, nullptr, nullptr, nullptr, 0, n_threads);
  return 0;
}

// Galilean (gradient-informed) constrained walks on the device sampler's
// stream: chains pick their start as in oracle_ns_replace and walk as in
// galilean_walk.  n_nodes = 0: no calibration model; otherwise the walk
// coordinates are those of oracle_ns_replace_cal.
int oracle_gmc_replace(const double* freqs, int64_t M, const double* strain, const double* psd,
                       const double* geom, int n_det, double gmst, double t_ref, int fcut_mode,
                       int D, const int* param_map, const double* fixed, const int* kind,
                       const double* lo, const double* hi, const int* periodic, int n_nodes,
                       const double* node_f, const double* sig, const double* live_u,
                       const double* live_lnl, int64_t K, int64_t worst, double lnl_star,
                       uint64_t seed, uint64_t counter, int64_t n_chains, int walk_len,
                       double scale, double rho, const double* chol, double* out_u, double* out_lnl,
                       int32_t* out_nacc, int32_t* out_start, int n_threads) {
  if (K < 2 || worst < 0 || worst >= K || n_nodes == 1 || n_nodes < 0 || !(rho >= 0.0 && rho <= 1.0)) return -1;
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
  Sampling s{D, param_map, fixed, kind, lo, hi, periodic};
  const int Dw = D + 2 * n_nodes * n_det;
  std::vector<int> per(Dw, 0);
  for (int i = 0; i < D; ++i) per[i] = periodic[i];
  if (n_nodes)
    gmc_replace_impl(cal_like(ev, s, n_nodes, node_f, sig), cal_like_grad(ev, s, n_nodes, node_f, sig), Dw,
                     per.data(), live_u, live_lnl, K, worst, lnl_star, seed, counter, n_chains, walk_len, scale,
                     rho, chol, out_u, out_lnl, out_nacc, out_start, n_threads);
  else
    gmc_replace_impl(gw_like(ev, s), gw_like_grad(ev, s), D, per.data(), live_u, live_lnl, K, worst, lnl_star,
                     seed, counter, n_chains, walk_len, scale, rho, chol, out_u, out_lnl, out_nacc, out_start,
                     n_threads);
  return 0;
}

// lnL and d lnL / du at n unit-cube points u[n][Dw] (test hook; n_nodes as in
// oracle_gmc_replace) -> lnl[n], grad[n][Dw].
int oracle_unit_grad(const double* freqs, int64_t M, const double* strain, const double* psd,
                     const double* geom, int n_det, double gmst, double t_ref, int fcut_mode, int D,
                     const int* param_map, const double* fixed, const int* kind, const double* lo,
                     const double* hi, const int* periodic, int n_nodes, const double* node_f,
                     const double* sig, const double* u, int64_t n, double* lnl, double* grad, int n_threads) {
  if (n_nodes == 1 || n_nodes < 0) return -1;
  Event ev{freqs, M, strain, psd, geom, n_det, gmst, t_ref, fcut_mode};
  Sampling s{D, param_map, fixed, kind, lo, hi, periodic};
  const int Dw = D + 2 * n_nodes * n_det;
  const UnitLikeGrad f = n_nodes ? cal_like_grad(ev, s, n_nodes, node_f, sig) : gw_like_grad(ev, s);
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t i = 0; i < n; ++i) lnl[i] = f(u + Dw * i, grad + Dw * i);
  return 0;
}

// Galilean walks on the analytic Gaussian-in-a-box likelihood from given
// start points u0[n][D] (test pin of the walk itself): chain b uses chain
// word b of the stream.
int oracle_gmc_gauss(int D, const double* mu, double sigma, const int* periodic, const double* u0, int64_t n,
                     double lnl_star, uint64_t seed, uint64_t counter, int walk_len, double scale, double rho,
                     const double* chol, double* out_u, double* out_lnl, int32_t* out_nacc, int n_threads) {
  if (D < 1 || n < 0 || !(rho >= 0.0 && rho <= 1.0)) return -1;
  const UnitLike f = gauss_like(D, mu, sigma);
  const UnitLikeGrad fg = gauss_like_grad(D, mu, sigma);
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t b = 0; b < n; ++b)
    galilean_walk(f, fg, periodic, D, u0 + D * b, f(u0 + D * b), lnl_star, seed, counter, uint32_t(b), walk_len,
                  scale, rho, chol, out_u + D * b, &out_lnl[b], &out_nacc[b]);
  return 0;
}

// Phi^{-1} of n values (test hook).
void oracle_inv_normal_cdf(int64_t n, const double* u, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = inv_normal_cdf(u[i]);
}

// Nested sampling of the analytic Gaussian-in-a-box likelihood (test pin).
int oracle_ns_run_gauss(int D, const double* mu, double sigma, int64_t K, int64_t n_chains,
                        int walk_len, uint64_t seed, double dlogz, int64_t max_rounds,
                        double scale0, double* res, double* dead_lnl, double* dead_logwt,
                        double* dead_u, int64_t max_dead, int n_threads) {
  if (K < 2 || D < 1) return -1;
  std::vector<int> per(D, 0);
  ns_run_impl(gauss_like(D, mu, sigma), D, per.data(), K, n_chains, walk_len, seed, dlogz,
              max_rounds, scale0, res, dead_lnl, dead_logwt, dead_u, max_dead, n_threads);
  return 0;
}

}  // extern "C"
