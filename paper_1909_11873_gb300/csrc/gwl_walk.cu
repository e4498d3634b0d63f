// gwl_walk.cu -- constrained random walks (ns_replace) and nested-sampling
// bookkeeping on the device (Section 3 and Algorithm 1 of the paper).
//
// Parallel sampling step: n_chains chains each start at a live point other
// than the current worst and make walk_len steps u' = u + scale * L z in the
// unit cube (z standard normal, L a lower-triangular matrix from the live
// set's covariance); periodic coordinates wrap, a step leaving the cube in any
// other coordinate is rejected, and a step is accepted iff lnL(theta(u')) >=
// L* (the worst live value).  Every step of all chains is one batched
// likelihood evaluation, so the walk is: init, then walk_len times {propose,
// batched lnL, accept}.
//
// Consumption (the replacement loop of Algorithm 1): candidates, in chain
// order, replace successive worst live points; a candidate whose lnL does not
// exceed the current worst is discarded (it was drawn above the round's first
// threshold only), and the round ends when candidates run out.  Dead point i
// gets the prior-volume weight dX_i = X_{i-1} - X_i with X_i = e^{-i/K}, so
// lnZ is a log-sum-exp that needs no sequential accumulation.  The final live
// points enter with equal weights X_N/(K+1).
#include <cmath>
#include <vector>

#include "gwl_internal.h"

namespace gwl {

// ---------------------------------------------------------------- random numbers
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011): 10 rounds of the 4x32
// S-P network, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments
// 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Normals of walk step `step` of chain `chain` (Box-Muller on word pairs).
__device__ __forceinline__ void walk_normals(uint64_t seed, uint64_t counter, uint32_t chain, uint32_t step, int D,
                                             double* z) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int b = 0; 4 * b < D; ++b) {
    const uint4 w = philox(make_uint4((uint32_t)b, step, chain, (uint32_t)counter), k0, k1);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double u1 = ((double)ws[2 * h] + 1.0) * 0x1p-32;
      const double u2 = (double)ws[2 * h + 1] * 0x1p-32;
      const double r = sqrt(-2.0 * ::log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      const int i0 = 4 * b + 2 * h;
      if (i0 < D) z[i0] = r * cs;
      if (i0 + 1 < D) z[i0 + 1] = r * sn;
    }
  }
}

// Unit cube -> parameter.  A walk coordinate is one of the n_src sampled
// source coordinates (the context's prior of each) or, with the calibration
// model, one of the 2 nn n_det calibration parameters that follow them (per
// detector nn amplitude then nn phase corrections), each with a zero-mean
// Gaussian prior: theta = sigma Phi^{-1}(u).
constexpr int kMaxWalkDim = GWL_N_PARAM + 2 * kMaxCalNodes * kMaxDet;
struct PriorInfo {
  int D;      // walk dimension
  int n_src;  // sampled source coordinates
  int kind[11];
  double lo[11], hi[11];
  int periodic[11];
  int nn;               // calibration nodes (0: none)
  double cal_sigma[2];  // prior widths of the amplitude and the phase [rad] corrections
};

__device__ __forceinline__ double prior_map(int kind, double lo, double hi, double u) {
  switch (kind) {
    case GWL_PRIOR_VOLUME: return cbrt(lo * lo * lo + u * (hi * hi * hi - lo * lo * lo));
    case GWL_PRIOR_SINE: return acos(1.0 - 2.0 * u);
    case GWL_PRIOR_COSINE: return asin(2.0 * u - 1.0);
    default: return lo + u * (hi - lo);
  }
}

__device__ __forceinline__ bool coord_periodic(const PriorInfo& pr, int i) { return i < pr.n_src && pr.periodic[i]; }

__device__ __forceinline__ double coord_map(const PriorInfo& pr, int i, double u) {
  if (i < pr.n_src) return prior_map(pr.kind[i], pr.lo[i], pr.hi[i], u);
  const int c = i - pr.n_src;
  return pr.cal_sigma[(c / pr.nn) & 1] * normcdfinv(u);
}

// ---------------------------------------------------------------- walk kernels
// Device-resident scalars of one walk (written by the host for ns_replace, by
// the preparation kernel inside ns_run).
struct WalkScalars {
  double lstar;
  double scale;
  long long worst;
  unsigned long long counter;
};

__global__ void k_walk_init(const double* __restrict__ live_u, const double* __restrict__ live_lnl, int64_t K,
                            int D, const WalkScalars* __restrict__ sc, uint64_t seed, int64_t n_chains,
                            double* __restrict__ cu, double* __restrict__ cl, int32_t* __restrict__ cn,
                            int32_t* __restrict__ cstart) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_chains) return;
  const uint4 w = philox(make_uint4(0u, 0u, (uint32_t)b, (uint32_t)sc->counter), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
  const int64_t idx = (int64_t)(((uint64_t)w.x * (uint64_t)(K - 1)) >> 32);
  const int64_t st = idx < sc->worst ? idx : idx + 1;
  for (int i = 0; i < D; ++i) cu[b * D + i] = live_u[st * D + i];
  cl[b] = live_lnl[st];
  cn[b] = 0;
  if (cstart) cstart[b] = (int32_t)st;
}

__device__ __forceinline__ void walk_propose_row(const PriorInfo& pr, const WalkScalars* __restrict__ sc,
                                                 const double* __restrict__ chol, uint64_t seed, uint32_t step,
                                                 int64_t b, const double* __restrict__ cu, double* __restrict__ pu,
                                                 double* __restrict__ ptheta) {
  const int D = pr.D;
  double z[kMaxWalkDim];
  walk_normals(seed, sc->counter, (uint32_t)b, step, D, z);
  const double scale = sc->scale;
  bool inside = true;
  for (int i = 0; i < D; ++i) {
    double dz = 0.0;
    for (int k = 0; k <= i; ++k) dz += chol[i * D + k] * z[k];
    double x = cu[b * D + i] + scale * dz;
    if (coord_periodic(pr, i)) x -= floor(x);
    else if (x < 0.0 || x > 1.0) inside = false;
    pu[b * D + i] = x;
  }
  for (int i = 0; i < D; ++i) ptheta[b * D + i] = inside ? coord_map(pr, i, pu[b * D + i]) : NAN;
}

__device__ __forceinline__ void walk_accept_row(const WalkScalars* __restrict__ sc, int D, int64_t b,
                                                const double* __restrict__ pu, const double* __restrict__ plnl,
                                                double* __restrict__ cu, double* __restrict__ cl,
                                                int32_t* __restrict__ cn) {
  const double l = plnl[b];
  if (l >= sc->lstar) {  // NaN rows (steps outside the cube) give -inf and fail
    for (int i = 0; i < D; ++i) cu[b * D + i] = pu[b * D + i];
    cl[b] = l;
    cn[b] += 1;
  }
}

__global__ void k_walk_accept(const WalkScalars* __restrict__ sc, int D, int64_t n_chains,
                              const double* __restrict__ pu, const double* __restrict__ plnl, double* __restrict__ cu,
                              double* __restrict__ cl, int32_t* __restrict__ cn) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n_chains) walk_accept_row(sc, D, b, pu, plnl, cu, cl, cn);
}

// One launch per walk step: the previous step's accept/reject (step > 1),
// this step's proposals, and the work counters of the likelihood call that
// follows cleared (that call then launches no clearing kernel of its own).
__global__ void k_walk_step(PriorInfo pr, const WalkScalars* __restrict__ sc, const double* __restrict__ chol,
                            uint64_t seed, uint32_t step, int64_t n_chains, const double* __restrict__ plnl,
                            double* __restrict__ cu, double* __restrict__ cl, int32_t* __restrict__ cn,
                            double* __restrict__ pu, double* __restrict__ ptheta, int* __restrict__ work,
                            int64_t nwork) {
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = t0; i < nwork; i += nt) work[i] = 0;
  if (t0 >= n_chains) return;
  if (step > 1) walk_accept_row(sc, pr.D, t0, pu, plnl, cu, cl, cn);
  walk_propose_row(pr, sc, chol, seed, step, t0, cu, pu, ptheta);
}

// ---------------------------------------------------------------- Galilean walk
// Gradient-informed constrained walk (Galilean Monte Carlo, Skilling 2012):
// each chain carries a velocity v (initially scale * L z).  A step tries
// x1 = u + v; if x1 is inside the cube and lnL(x1) >= L* the chain moves.
// Otherwise, if x1 left the cube, the offending velocity components are
// reversed and the chain stays; if x1 violated the likelihood constraint, v is
// reflected off the contour, v' = v - 2 (v.n) n with n the unit gradient of
// lnL at x1 in the unit cube, and x2 = x1 + v' is tried: the chain moves to x2
// (keeping v') if it satisfies the constraint, else it stays and v <- -v.
// Normals for the initial velocity come from step word 0x40000000.
__device__ __forceinline__ double prior_jac(int kind, double lo, double hi, double th) {
  switch (kind) {
    case GWL_PRIOR_VOLUME: return (hi * hi * hi - lo * lo * lo) / (3.0 * th * th);
    case GWL_PRIOR_SINE: return 2.0 / fmax(sin(th), 1e-300);
    case GWL_PRIOR_COSINE: return 2.0 / fmax(cos(th), 1e-300);
    default: return hi - lo;
  }
}

// d theta / d u of walk coordinate i at theta: the source priors above, or for
// a calibration parameter theta = sigma Phi^{-1}(u): sigma sqrt(2 pi) e^{z^2/2}, z = theta / sigma.
__device__ __forceinline__ double coord_jac(const PriorInfo& pr, int i, double th) {
  if (i < pr.n_src) return prior_jac(pr.kind[i], pr.lo[i], pr.hi[i], th);
  const double sg = pr.cal_sigma[((i - pr.n_src) / pr.nn) & 1], z = th / sg;
  return sg * 2.5066282746310002 * exp(0.5 * z * z);
}

__global__ void k_gmc_init(PriorInfo pr, const double* __restrict__ live_u, const double* __restrict__ live_lnl,
                           int64_t K, const WalkScalars* __restrict__ sc, const double* __restrict__ chol,
                           uint64_t seed, int64_t n_chains, double* __restrict__ cu, double* __restrict__ cl,
                           int32_t* __restrict__ cn, int32_t* __restrict__ cstart, double* __restrict__ vel) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_chains) return;
  const int D = pr.D;
  const uint4 w = philox(make_uint4(0u, 0u, (uint32_t)b, (uint32_t)sc->counter), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
  const int64_t idx = (int64_t)(((uint64_t)w.x * (uint64_t)(K - 1)) >> 32);
  const int64_t st = idx < sc->worst ? idx : idx + 1;
  for (int i = 0; i < D; ++i) cu[b * D + i] = live_u[st * D + i];
  cl[b] = live_lnl[st];
  cn[b] = 0;
  if (cstart) cstart[b] = (int32_t)st;
  double z[kMaxWalkDim];
  walk_normals(seed, sc->counter, (uint32_t)b, 0x40000000u, D, z);
  for (int i = 0; i < D; ++i) {
    double dz = 0.0;
    for (int k = 0; k <= i; ++k) dz += chol[i * D + k] * z[k];
    vel[b * D + i] = sc->scale * dz;
  }
}

// From the second step on, the velocity is partly refreshed,
//   v <- rho v + sqrt(1 - rho^2) scale L z  (z: the normals of this step's word),
// which keeps its distribution N(0, scale^2 L L^T); then x1 = u + v and
// theta1 (NaN rows outside the cube).
__global__ void k_gmc_step1(PriorInfo pr, const WalkScalars* __restrict__ sc, const double* __restrict__ chol,
                            uint64_t seed, uint32_t step, double rho, int64_t n_chains,
                            const double* __restrict__ cu, double* __restrict__ vel, double* __restrict__ x1,
                            double* __restrict__ th1) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_chains) return;
  const int D = pr.D;
  if (step > 1 && rho < 1.0) {
    double z[kMaxWalkDim];
    walk_normals(seed, sc->counter, (uint32_t)b, step, D, z);
    const double a = sqrt(1.0 - rho * rho) * sc->scale;
    for (int i = 0; i < D; ++i) {
      double dz = 0.0;
      for (int k = 0; k <= i; ++k) dz += chol[i * D + k] * z[k];
      vel[b * D + i] = rho * vel[b * D + i] + a * dz;
    }
  }
  bool inside = true;
  for (int i = 0; i < D; ++i) {
    double x = cu[b * D + i] + vel[b * D + i];
    if (coord_periodic(pr, i)) x -= floor(x);
    else if (x < 0.0 || x > 1.0) inside = false;
    x1[b * D + i] = x;
  }
  for (int i = 0; i < D; ++i) th1[b * D + i] = inside ? coord_map(pr, i, x1[b * D + i]) : NAN;
}

// Accept x1, or reflect off the surface at x1 and set up the second trial.
// The surface is the likelihood contour when x1 is inside the cube (normal g:
// the gradient of lnL in the unit cube, chain rule through the coordinate
// maps) and the walls x1 crossed when it is not (g: their outward unit
// normals summed) -- either way a function of x1 alone.  The reflection is
// taken in the metric of the step covariance Sigma = L L^T,
//   v' = v - 2 (v.g) / (g.Sigma g) Sigma g,  Sigma g = L (L^T g),
// so that it keeps the velocity distribution and undoes itself.  v' goes to
// vel2 and theta2 = theta(x1 + v') is written for the chains that try x2.
// mode: 0 moved to x1; 1 try x2; 2 stay and reverse v.
__global__ void k_gmc_reflect(PriorInfo pr, const WalkScalars* __restrict__ sc, int64_t n_chains,
                              const double* __restrict__ chol, const double* __restrict__ x1,
                              const double* __restrict__ th1, const double* __restrict__ l1,
                              const double* __restrict__ g1, double* __restrict__ cu, double* __restrict__ cl,
                              int32_t* __restrict__ cn, const double* __restrict__ vel, double* __restrict__ vel2,
                              double* __restrict__ x2, double* __restrict__ th2, int32_t* __restrict__ mode) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_chains) return;
  const int D = pr.D;
  bool inside = true;
  for (int i = 0; i < D; ++i) inside = inside && !isnan(th1[b * D + i]);
  for (int i = 0; i < D; ++i) th2[b * D + i] = NAN;
  if (inside && l1[b] >= sc->lstar) {  // move
    for (int i = 0; i < D; ++i) cu[b * D + i] = x1[b * D + i];
    cl[b] = l1[b];
    cn[b] += 1;
    mode[b] = 0;
    return;
  }
  double g[kMaxWalkDim], m[kMaxWalkDim];
  for (int i = 0; i < D; ++i) {
    const double x = x1[b * D + i];
    g[i] = inside ? g1[b * D + i] * coord_jac(pr, i, th1[b * D + i])
                  : (coord_periodic(pr, i) ? 0.0 : (x > 1.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0)));
  }
  double gsg = 0.0, vg = 0.0;
  for (int k = 0; k < D; ++k) {  // m = L^T g
    double t = 0.0;
    for (int i = k; i < D; ++i) t += chol[i * D + k] * g[i];
    m[k] = t;
    gsg += t * t;
    vg += vel[b * D + k] * g[k];
  }
  if (!(gsg > 0.0) || !isfinite(gsg) || !isfinite(vg)) {
    mode[b] = 2;
    return;
  }
  const double f = 2.0 * vg / gsg;
  bool in2 = true;
  for (int i = 0; i < D; ++i) {
    double sgi = 0.0;  // (Sigma g)_i = (L m)_i
    for (int k = 0; k <= i; ++k) sgi += chol[i * D + k] * m[k];
    const double v2 = vel[b * D + i] - f * sgi;
    double x = x1[b * D + i] + v2;
    if (coord_periodic(pr, i)) x -= floor(x);
    else if (x < 0.0 || x > 1.0) in2 = false;
    x2[b * D + i] = x;
    vel2[b * D + i] = v2;
  }
  if (!in2) {
    mode[b] = 2;
    return;
  }
  for (int i = 0; i < D; ++i) th2[b * D + i] = coord_map(pr, i, x2[b * D + i]);
  mode[b] = 1;
}

// Move to x2 with v' (mode 1, lnL(x2) >= L*), or stay and reverse v (mode 1
// below L*, mode 2).
__global__ void k_gmc_step2(int D, const WalkScalars* __restrict__ sc, int64_t n_chains, const double* __restrict__ x2,
                            const double* __restrict__ l2, const int32_t* __restrict__ mode,
                            const double* __restrict__ vel2, double* __restrict__ cu, double* __restrict__ cl,
                            int32_t* __restrict__ cn, double* __restrict__ vel) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_chains || mode[b] == 0) return;
  if (mode[b] == 1 && l2[b] >= sc->lstar) {
    for (int i = 0; i < D; ++i) {
      cu[b * D + i] = x2[b * D + i];
      vel[b * D + i] = vel2[b * D + i];
    }
    cl[b] = l2[b];
    cn[b] += 1;
  } else {
    for (int i = 0; i < D; ++i) vel[b * D + i] = -vel[b * D + i];
  }
}

// ---------------------------------------------------------------- nested-sampling state kernels
struct NsDev {
  // live set
  double* lu;   // [K][D]
  double* ll;   // [K]
  int64_t K;
  int D;
  // candidates of the current round (the walk's outputs)
  double* cu;
  double* cl;
  int32_t* cn;
  int64_t n_chains;
  // this round's dead points: lnL + ln dX, one per consumed candidate
  double* rx;   // [n_chains]
  double* rl;   // [n_chains] lnL
  // dead points (kept up to cap for posterior samples)
  double* dl;   // [cap]
  double* dw;   // [cap] ln dX
  double* du;   // [cap][D]
  int64_t cap;
  // scalars
  WalkScalars* ws;
  double* chol;   // [D][D]
  double* stats;  // see NS_* below
};

// stats layout
enum {
  NS_LNZ = 0,        // ln Z of the dead points so far (m + ln ZS)
  NS_NDEAD = 1,      // dead points so far (as double)
  NS_LMAX = 2,       // largest live lnL
  NS_ROUND = 3,      // rounds done
  NS_DONE = 4,       // 1 once the stopping rule holds
  NS_ACC_SUM = 5,    // sum over rounds of the acceptance fraction
  NS_CONSUMED = 6,   // candidates consumed in total
  NS_DLOGZ = 7,      // ln(Z + Lmax X) - ln Z after the last round
  NS_NDEAD_ROUND0 = 8,  // dead count at the start of the round
  NS_M = 9,          // reference maximum of lnL + ln dX
  NS_ZS = 10,        // sum exp(lnL + ln dX - m)
  NS_AS = 11,        // sum exp(lnL + ln dX - m) lnL   (for the information H)
  NS_H = 12,         // information H = AS/ZS - ln Z
  NS_NSTATS = 16
};

__device__ __forceinline__ double logaddexp_d(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  const double m = a > b ? a : b;
  return m + ::log(::exp(a - m) + ::exp(b - m));
}

// Round preparation: worst live point and L*, Cholesky factor of the live-set
// covariance in the unit cube (plain, FP64, one CTA).
__device__ void ns_prep_body(const NsDev& s) {
  if (s.stats[NS_DONE] > 0.5) return;  // rounds replayed after the stopping rule held change nothing
  __shared__ double red_v[256];
  __shared__ long long red_i[256];
  const int t = threadIdx.x;
  // argmin of the live lnL
  double bv = INFINITY;
  long long bi = 0;
  for (int64_t k = t; k < s.K; k += blockDim.x) {
    const double v = s.ll[k];
    if (v < bv || (v == bv && k < bi)) {
      bv = v;
      bi = k;
    }
  }
  red_v[t] = bv;
  red_i[t] = bi;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (t < off) {
      const double v = red_v[t + off];
      const long long i = red_i[t + off];
      if (v < red_v[t] || (v == red_v[t] && i < red_i[t])) {
        red_v[t] = v;
        red_i[t] = i;
      }
    }
    __syncthreads();
  }
  const int D = s.D;
  // mean and covariance of the live set: thread t handles one (dimension or
  // pair) and one slice of the points; slices are reduced through shared
  // memory (with more pairs than threads, each thread takes whole pairs)
  __shared__ double part[256];
  __shared__ double mean[kMaxWalkDim], diag[kMaxWalkDim];
  {
    const int S = blockDim.x / D;  // D <= kMaxWalkDim < blockDim
    const int i = t % D, sl = t / D;
    double m = 0.0;
    if (sl < S)
      for (int64_t k = sl; k < s.K; k += S) m += s.lu[k * D + i];
    part[t] = sl < S ? m : 0.0;
    __syncthreads();
    if (t < D) {
      double a = 0.0;
      for (int q = 0; q < S; ++q) a += part[q * D + t];
      mean[t] = a / (double)s.K;
    }
    __syncthreads();
  }
  double* A = s.chol;  // the covariance, then (in place) its Cholesky factor
  {
    const int P = D * (D + 1) / 2;
    auto pair = [D](int pr, int& i, int& j) {  // pair index -> (i, j), i <= j
      i = 0;
      j = pr;
      while (j >= D - i) {
        j -= D - i;
        ++i;
      }
      j += i;
    };
    if (P <= (int)blockDim.x) {
      const int S = blockDim.x / P;
      const int pr = t % P, sl = t / P;
      int i, j;
      pair(pr, i, j);
      double c = 0.0;
      if (sl < S)
        for (int64_t k = sl; k < s.K; k += S) c += (s.lu[k * D + i] - mean[i]) * (s.lu[k * D + j] - mean[j]);
      part[t] = sl < S ? c : 0.0;
      __syncthreads();
      if (t < P) {
        double a = 0.0;
        for (int q = 0; q < S; ++q) a += part[q * P + t];
        int ii, jj;
        pair(t, ii, jj);
        A[ii * D + jj] = A[jj * D + ii] = a / (double)(s.K - 1);
      }
    } else {
      for (int pr = t; pr < P; pr += blockDim.x) {
        int i, j;
        pair(pr, i, j);
        double c = 0.0;
        for (int64_t k = 0; k < s.K; ++k) c += (s.lu[k * D + i] - mean[i]) * (s.lu[k * D + j] - mean[j]);
        A[i * D + j] = A[j * D + i] = c / (double)(s.K - 1);
      }
    }
    __syncthreads();
  }
  // Cholesky factor (lower), left-looking, in place: column j's diagonal on
  // thread 0, its rows below in parallel, one barrier per column; a diagonal
  // factor of the covariance if it is not positive definite
  __shared__ int s_ok;
  for (int i = t; i < D; i += blockDim.x) diag[i] = A[i * D + i];
  if (t == 0) s_ok = 1;
  __syncthreads();
  for (int j = 0; j < D; ++j) {
    if (t == 0) {
      double d = A[j * D + j];
      for (int k = 0; k < j; ++k) d -= A[j * D + k] * A[j * D + k];
      if (d > 0.0) A[j * D + j] = sqrt(d);
      else s_ok = 0;
    }
    __syncthreads();
    if (!s_ok) break;
    const double ljj = A[j * D + j];
    for (int i = j + 1 + t; i < D; i += blockDim.x) {
      double x = A[i * D + j];
      for (int k = 0; k < j; ++k) x -= A[i * D + k] * A[j * D + k];
      A[i * D + j] = x / ljj;
    }
    __syncthreads();
  }
  const bool okc = s_ok != 0;
  for (int x = t; x < D * D; x += blockDim.x) {
    const int i = x / D, j = x % D;
    if (!okc) A[x] = i == j ? sqrt(fmax(diag[i], 1e-300)) : 0.0;
    else if (j > i) A[x] = 0.0;
  }
  if (t == 0) {
    s.ws->lstar = red_v[0];
    s.ws->worst = red_i[0];
    s.ws->counter = (unsigned long long)s.stats[NS_ROUND];
    s.stats[NS_NDEAD_ROUND0] = s.stats[NS_NDEAD];
  }
}

// Order key of a log-likelihood: a signed 64-bit integer whose order is the
// values' order (IEEE bits; negative values with all bits but the sign
// flipped), so that the replacement loop compares on the integer pipe instead
// of the narrow FP64 one.  -0 takes +0's key, so the two tie as they compare
// equal; log-likelihoods are never NaN (rows the likelihood cannot evaluate
// give -inf), and a NaN takes -inf's key.
__device__ __forceinline__ long long lnl_key(double x) {
  if (x != x) x = -INFINITY;
  long long i = __double_as_longlong(x);
  if (i == (long long)0x8000000000000000ull) i = 0;
  return i < 0 ? i ^ 0x7fffffffffffffffll : i;
}
__device__ __forceinline__ double key_lnl(long long k) {
  return __longlong_as_double(k < 0 ? k ^ 0x7fffffffffffffffll : k);
}

// Consumption of the round's candidates.  The sequential replacement loop
// (warp 0) touches only shared memory: the order keys of the live lnL and of
// the candidates' lnL and, per live slot, where its point currently comes from
// (an original live point or a candidate); it records each dead point's lnL
// and slot.  The dead points' prior weights, the unit-cube coordinates of
// dead points and of the replaced slots are then written by the whole CTA.
__device__ void ns_consume_body(const NsDev& s) {
  if (s.stats[NS_DONE] > 0.5) return;
  extern __shared__ __align__(16) unsigned char smc[];
  long long* ll = reinterpret_cast<long long*>(smc);  // [K]   keys of the live lnL
  long long* cl = ll + s.K;                           // [n_chains] keys of the candidates' lnL
  int* src = reinterpret_cast<int*>(cl + s.n_chains);  // [K]   -1: original, else candidate index
  int* rslot = src + s.K;                          // [n_chains] slot replaced at step r
  int* rsrc = rslot + s.n_chains;                  // [n_chains] source of the dead point at step r
  __shared__ int sh_nrep;
  __shared__ double sh_lw1;
  const int t = threadIdx.x, lane = t & 31;
  const int D = s.D;
  for (int64_t k = t; k < s.K; k += blockDim.x) {
    ll[k] = lnl_key(s.ll[k]);
    src[k] = -1;
  }
  for (int64_t b = t; b < s.n_chains; b += blockDim.x) cl[b] = lnl_key(s.cl[b]);
  __syncthreads();
  const int64_t nd0 = (int64_t)s.stats[NS_NDEAD];
  if (t < 32) {
    int64_t ptr = 0;
    int nrep = 0;
    while (true) {
      long long bv = 0x7fffffffffffffffll;
      int bi = 0;
      for (int k = lane; k < s.K; k += 32) {
        const long long v = ll[k];
        if (v < bv || (v == bv && k < bi)) {
          bv = v;
          bi = k;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const long long v = __shfl_xor_sync(0xffffffffu, bv, off);
        const int i = __shfl_xor_sync(0xffffffffu, bi, off);
        if (v < bv || (v == bv && i < bi)) {
          bv = v;
          bi = i;
        }
      }
      while (ptr < s.n_chains && !(cl[ptr] > bv)) ++ptr;
      if (ptr >= s.n_chains) break;
      if (lane == 0) {
        s.rl[nrep] = key_lnl(bv);
        rslot[nrep] = bi;
        rsrc[nrep] = src[bi];
        src[bi] = (int)ptr;
        ll[bi] = cl[ptr];
      }
      __syncwarp();
      ++ptr;
      ++nrep;
    }
    if (lane == 0) sh_nrep = nrep;
  } else if (t == 32) {  // beside the loop: ln(1 - e^{-1/K})
    sh_lw1 = log1p(-::exp(-1.0 / (double)s.K));
  }
  __syncthreads();
  const int nrep = sh_nrep;
  // the dead points' prior weights ln(X_{i-1} - X_i) and weighted values
  const double lw1 = sh_lw1;
  for (int r = t; r < nrep; r += blockDim.x) {
    const int64_t nd = nd0 + r + 1;
    const double lw = -(double)(nd - 1) / (double)s.K + lw1;
    const double l = s.rl[r];
    s.rx[r] = l + lw;
    if (nd <= s.cap) {
      s.dl[nd - 1] = l;
      s.dw[nd - 1] = lw;
    }
  }
  // dead points' coordinates (before any live slot is overwritten)
  for (int64_t x = t; x < (int64_t)nrep * D; x += blockDim.x) {
    const int r = (int)(x / D), i = (int)(x % D);
    const int64_t nd = nd0 + r + 1;
    if (nd <= s.cap) {
      const int sr = rsrc[r];
      s.du[(nd - 1) * D + i] = sr < 0 ? s.lu[(int64_t)rslot[r] * D + i] : s.cu[(int64_t)sr * D + i];
    }
  }
  __syncthreads();
  // live slots that now hold a candidate
  for (int64_t x = t; x < s.K * D; x += blockDim.x) {
    const int64_t k = x / D;
    const int i = (int)(x % D);
    const int sr = src[k];
    if (sr >= 0) s.lu[x] = s.cu[(int64_t)sr * D + i];
  }
  for (int64_t k = t; k < s.K; k += blockDim.x) {
    const int sr = src[k];
    if (sr >= 0) s.ll[k] = s.cl[sr];
  }
  if (t == 0) {
    s.stats[NS_NDEAD] = (double)(nd0 + nrep);
    s.stats[NS_CONSUMED] += (double)nrep;
  }
}

size_t consume_smem_bytes(int64_t K, int64_t n_chains) {
  return sizeof(long long) * (size_t)(K + n_chains) + sizeof(int) * (size_t)(K + 2 * n_chains);
}

// Fold n weighted points x_i = lnL_i + ln dX_i (with lnL_i) into the running
// sums (m, ZS, AS) of stats; one CTA.
__device__ void fold_points(double* stats, const double* x, const double* l, int64_t n, double* red) {
  const int t = threadIdx.x;
  double m = -INFINITY;
  for (int64_t i = t; i < n; i += blockDim.x) m = fmax(m, x[i]);
  red[t] = m;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (t < off) red[t] = fmax(red[t], red[t + off]);
    __syncthreads();
  }
  const double mr = red[0];
  __syncthreads();
  const double mref = fmax(stats[NS_M], mr);
  double zs = 0.0, as = 0.0;
  if (mref > -INFINITY)
    for (int64_t i = t; i < n; i += blockDim.x) {
      const double e = ::exp(x[i] - mref);
      zs += e;
      as += e * l[i];
    }
  red[t] = zs;
  red[blockDim.x + t] = as;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (t < off) {
      red[t] += red[t + off];
      red[blockDim.x + t] += red[blockDim.x + t + off];
    }
    __syncthreads();
  }
  if (t == 0 && mref > -INFINITY) {
    const double r = stats[NS_M] > -INFINITY ? ::exp(stats[NS_M] - mref) : 0.0;
    stats[NS_ZS] = stats[NS_ZS] * r + red[0];
    stats[NS_AS] = stats[NS_AS] * r + red[blockDim.x];
    stats[NS_M] = mref;
    stats[NS_LNZ] = mref + ::log(stats[NS_ZS]);
    stats[NS_H] = stats[NS_AS] / stats[NS_ZS] - stats[NS_LNZ];
  }
  __syncthreads();
}

// End of round: ln Z update from the round's dead points, largest live lnL,
// stopping rule ln(Z + Lmax X) - ln Z < dlogz, acceptance and scale
// adaptation scale <- scale exp(acc - 1/2) clamped to [1e-3, 1].
__device__ void ns_stats_body(const NsDev& s, int walk_len, double dlogz) {
  if (s.stats[NS_DONE] > 0.5) return;
  __shared__ double red[512];
  const int t = threadIdx.x;
  const int64_t nr = (int64_t)(s.stats[NS_NDEAD] - s.stats[NS_NDEAD_ROUND0]);
  fold_points(s.stats, s.rx, s.rl, nr, red);
  double lm = -INFINITY;
  for (int64_t k = t; k < s.K; k += blockDim.x) lm = fmax(lm, s.ll[k]);
  red[t] = lm;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (t < off) red[t] = fmax(red[t], red[t + off]);
    __syncthreads();
  }
  const double lmax = red[0];
  __syncthreads();
  double na = 0.0;
  for (int64_t b = t; b < s.n_chains; b += blockDim.x) na += (double)s.cn[b];
  red[t] = na;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (t < off) red[t] += red[t + off];
    __syncthreads();
  }
  if (t == 0) {
    const double lnZ = s.stats[NS_LNZ];
    s.stats[NS_LMAX] = lmax;
    const double lnX = -s.stats[NS_NDEAD] / (double)s.K;
    const double dz = logaddexp_d(lnZ, lmax + lnX) - lnZ;
    s.stats[NS_DLOGZ] = dz;
    if (dz < dlogz) s.stats[NS_DONE] = 1.0;
    const double accf = red[0] / ((double)s.n_chains * (double)walk_len);
    s.stats[NS_ACC_SUM] += accf;
    s.ws->scale = fmin(1.0, fmax(1e-3, s.ws->scale * ::exp(accf - 0.5)));
    s.stats[NS_ROUND] += 1.0;
  }
}

// The final live points, each with prior volume X_N / (K + 1).
__device__ void ns_final_body(const NsDev& s) {
  __shared__ double red[512];
  const double lw = -s.stats[NS_NDEAD] / (double)s.K - ::log((double)(s.K + 1));
  const int64_t nd = (int64_t)s.stats[NS_NDEAD];
  for (int64_t k = threadIdx.x; k < s.K; k += blockDim.x) {
    s.rx[k] = s.ll[k] + lw;
    if (nd + k < s.cap) {  // the final live points close the dead list
      s.dl[nd + k] = s.ll[k];
      s.dw[nd + k] = lw;
      for (int i = 0; i < s.D; ++i) s.du[(nd + k) * s.D + i] = s.lu[k * s.D + i];
    }
  }
  __syncthreads();
  fold_points(s.stats, s.rx, s.ll, s.K, red);
}

// One event (parameters by value) or E events (one CTA per event).
__global__ void __launch_bounds__(256) k_ns_prep(NsDev s) { ns_prep_body(s); }
__global__ void __launch_bounds__(256) k_ns_consume(NsDev s) { ns_consume_body(s); }
__global__ void __launch_bounds__(256) k_ns_stats(NsDev s, int walk_len, double dlogz) { ns_stats_body(s, walk_len, dlogz); }
__global__ void __launch_bounds__(256) k_ns_final(NsDev s) { ns_final_body(s); }
__global__ void __launch_bounds__(256) k_mns_prep(const NsDev* a) { ns_prep_body(a[blockIdx.x]); }
__global__ void __launch_bounds__(256) k_mns_consume(const NsDev* a) { ns_consume_body(a[blockIdx.x]); }
__global__ void __launch_bounds__(256) k_mns_stats(const NsDev* a, int walk_len, double dlogz) {
  ns_stats_body(a[blockIdx.x], walk_len, dlogz);
}
__global__ void __launch_bounds__(256) k_mns_final(const NsDev* a) { ns_final_body(a[blockIdx.x]); }

// Walk kernels over E events x n chains: chain b belongs to event b / n; each
// event has its own live set, walk scalars, step matrix, prior and Philox key
// (seed + event * 0x9E3779B97F4A7C15).  Events whose run has stopped propose
// nothing (NaN rows, which the likelihood flags without bin work).
__host__ __device__ __forceinline__ uint64_t event_key(uint64_t seed, int e) {
  return seed + (uint64_t)e * 0x9E3779B97F4A7C15ull;
}

__global__ void k_mwalk_init(const NsDev* __restrict__ a, int64_t n, int E, uint64_t seed) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * E) return;
  const int e = (int)(g / n);
  const int64_t b = g - (int64_t)e * n;
  const NsDev& s = a[e];
  const uint64_t key = event_key(seed, e);
  const uint4 w = philox(make_uint4(0u, 0u, (uint32_t)b, (uint32_t)s.ws->counter), (uint32_t)key,
                         (uint32_t)(key >> 32));
  const int64_t idx = (int64_t)(((uint64_t)w.x * (uint64_t)(s.K - 1)) >> 32);
  const int64_t st = idx < s.ws->worst ? idx : idx + 1;
  for (int i = 0; i < s.D; ++i) s.cu[b * s.D + i] = s.lu[st * s.D + i];
  s.cl[b] = s.ll[st];
  s.cn[b] = 0;
}

__global__ void k_mwalk_propose(const NsDev* __restrict__ a, const PriorInfo* __restrict__ prs, int64_t n, int E,
                                uint64_t seed, uint32_t step, double* __restrict__ pu, double* __restrict__ ptheta) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * E) return;
  const int e = (int)(g / n);
  const int64_t b = g - (int64_t)e * n;
  const NsDev& s = a[e];
  const PriorInfo& pr = prs[e];
  const int D = pr.D;
  if (s.stats[NS_DONE] > 0.5) {
    for (int i = 0; i < D; ++i) ptheta[g * D + i] = NAN;
    return;
  }
  double z[kMaxWalkDim];
  walk_normals(event_key(seed, e), s.ws->counter, (uint32_t)b, step, D, z);
  const double scale = s.ws->scale;
  bool inside = true;
  for (int i = 0; i < D; ++i) {
    double dz = 0.0;
    for (int k = 0; k <= i; ++k) dz += s.chol[i * D + k] * z[k];
    double x = s.cu[b * D + i] + scale * dz;
    if (coord_periodic(pr, i)) x -= floor(x);
    else if (x < 0.0 || x > 1.0) inside = false;
    pu[g * D + i] = x;
  }
  for (int i = 0; i < D; ++i) ptheta[g * D + i] = inside ? coord_map(pr, i, pu[g * D + i]) : NAN;
}

__global__ void k_mwalk_accept(const NsDev* __restrict__ a, int64_t n, int E, const double* __restrict__ pu,
                               const double* __restrict__ plnl) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * E) return;
  const int e = (int)(g / n);
  const int64_t b = g - (int64_t)e * n;
  const NsDev& s = a[e];
  const double l = plnl[g];
  if (l >= s.ws->lstar) {
    for (int i = 0; i < s.D; ++i) s.cu[b * s.D + i] = pu[g * s.D + i];
    s.cl[b] = l;
    s.cn[b] += 1;
  }
}

// Initial live points: uniform in the unit cube, Philox words (block, step
// 0xFFFFFFFF, point k, 0xFFFFFFFF), u = (w + 1/2) 2^-32; theta by the prior map.
__global__ void k_ns_init(PriorInfo pr, uint64_t seed, int64_t K, double* __restrict__ lu,
                          double* __restrict__ theta) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int D = pr.D;
  for (int b = 0; 4 * b < D; ++b) {
    const uint4 w = philox(make_uint4((uint32_t)b, 0xFFFFFFFFu, (uint32_t)k, 0xFFFFFFFFu), (uint32_t)seed,
                           (uint32_t)(seed >> 32));
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    for (int i = 0; i < 4 && 4 * b + i < D; ++i) {
      const double u = ((double)ws[i] + 0.5) * 0x1p-32;
      lu[k * D + 4 * b + i] = u;
      theta[k * D + 4 * b + i] = coord_map(pr, 4 * b + i, u);
    }
  }
}

// ---------------------------------------------------------------- host side
static PriorInfo prior_info(const gwl_ctx* c) {
  PriorInfo p;
  p.D = (int)theta_stride(c);
  p.n_src = c->opt.n_dim;
  for (int i = 0; i < 11; ++i) {
    p.kind[i] = c->opt.prior_kind[i];
    p.lo[i] = c->opt.prior_lo[i];
    p.hi[i] = c->opt.prior_hi[i];
    p.periodic[i] = c->opt.periodic[i];
  }
  p.nn = c->n_cal_nodes > 0 ? c->n_cal_nodes : 1;
  p.cal_sigma[0] = c->cal_sigma[0];
  p.cal_sigma[1] = c->cal_sigma[1];
  return p;
}

// The walk proper: chains start from live points and take walk_len steps.
static cudaError_t launch_gmc(gwl_ctx* c, const double* live_u, const double* live_lnl, int64_t K,
                              const WalkScalars* sc, uint64_t seed, int64_t n_chains, int walk_len, const double* chol,
                              double* out_u, double* out_lnl, int32_t* out_nacc, int32_t* out_start, double* pu,
                              double* pth, double* plnl, cudaStream_t st) {
  const int D = (int)theta_stride(c);
  const unsigned nb = (unsigned)((n_chains + 127) / 128);
  const PriorInfo pr = prior_info(c);
  // scratch after the random-walk proposal buffers: velocity, reflected velocity, x2, theta2, gradient,
  // l2, mode
  double* vel = c->d_gmc;
  double* vel2 = vel + n_chains * D;
  double* x2 = vel2 + n_chains * D;
  double* th2 = x2 + n_chains * D;
  double* g1 = th2 + n_chains * D;
  double* l2 = g1 + n_chains * D;
  int32_t* mode = reinterpret_cast<int32_t*>(l2 + n_chains);
  {
    ProfScope ps(c, GWL_KERNEL_WALK, st);
    k_gmc_init<<<nb, 128, 0, st>>>(pr, live_u, live_lnl, K, sc, chol, seed, n_chains, out_u, out_lnl, out_nacc,
                                   out_start, vel);
    c->launches++;
  }
  cudaError_t e = cudaGetLastError();
  for (int s = 1; s <= walk_len && e == cudaSuccess; ++s) {
    k_gmc_step1<<<nb, 128, 0, st>>>(pr, sc, chol, seed, (uint32_t)s, c->gmc_persistence, n_chains, out_u, vel, pu,
                                    pth);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = launch_grad(c, pth, n_chains, plnl, g1, st)) != cudaSuccess) break;
    k_gmc_reflect<<<nb, 128, 0, st>>>(pr, sc, n_chains, chol, pu, pth, plnl, g1, out_u, out_lnl, out_nacc, vel,
                                      vel2, x2, th2, mode);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = launch_loglike(c, th2, n_chains, l2, st)) != cudaSuccess) break;
    k_gmc_step2<<<nb, 128, 0, st>>>(D, sc, n_chains, x2, l2, mode, vel2, out_u, out_lnl, out_nacc, vel);
    c->launches++;
    e = cudaGetLastError();
  }
  return e;
}

size_t gmc_scratch_doubles(int64_t n_chains, int D) { return (size_t)n_chains * (5 * D + 2); }

cudaError_t launch_walk(gwl_ctx* c, const double* live_u, const double* live_lnl, int64_t K, const void* scalars,
                        uint64_t seed, int64_t n_chains, int walk_len, const double* chol, double* out_u,
                        double* out_lnl, int32_t* out_nacc, int32_t* out_start, double* pu, double* pth,
                        double* plnl, cudaStream_t st) {
  const WalkScalars* sc = static_cast<const WalkScalars*>(scalars);
  if (c->walk_kind == GWL_WALK_GALILEAN)
    return launch_gmc(c, live_u, live_lnl, K, sc, seed, n_chains, walk_len, chol, out_u, out_lnl, out_nacc,
                      out_start, pu, pth, plnl, st);
  const int D = (int)theta_stride(c);
  const unsigned nb = (unsigned)((n_chains + 127) / 128);
  const PriorInfo pr = prior_info(c);
  {
    ProfScope ps(c, GWL_KERNEL_WALK, st);
    k_walk_init<<<nb, 128, 0, st>>>(live_u, live_lnl, K, D, sc, seed, n_chains, out_u, out_lnl, out_nacc, out_start);
    c->launches++;
  }
  cudaError_t e = cudaGetLastError();
  const int64_t nwork = work_needed(c, n_chains);
  for (int s = 1; s <= walk_len && e == cudaSuccess; ++s) {
    {
      ProfScope ps(c, GWL_KERNEL_WALK, st);
      k_walk_step<<<nb, 128, 0, st>>>(pr, sc, chol, seed, (uint32_t)s, n_chains, plnl, out_u, out_lnl, out_nacc, pu,
                                      pth, c->d_work, nwork);
      c->launches++;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    e = launch_loglike_cleared(c, pth, n_chains, plnl, st);
  }
  if (e == cudaSuccess && walk_len > 0) {  // the last step's accept/reject
    ProfScope ps(c, GWL_KERNEL_WALK, st);
    k_walk_accept<<<nb, 128, 0, st>>>(sc, D, n_chains, pu, plnl, out_u, out_lnl, out_nacc);
    c->launches++;
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_ns_init(gwl_ctx* c, uint64_t seed, int64_t K, double* lu, double* theta, cudaStream_t st) {
  k_ns_init<<<(unsigned)((K + 127) / 128), 128, 0, st>>>(prior_info(c), seed, K, lu, theta);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_ns_round(gwl_ctx* c, const NsDev& s, uint64_t seed, int walk_len, double dlogz, double* pu,
                            double* pth, double* plnl, cudaStream_t st) {
  k_ns_prep<<<1, 256, 0, st>>>(s);
  c->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_walk(c, s.lu, s.ll, s.K, s.ws, seed, s.n_chains, walk_len, s.chol, s.cu, s.cl, s.cn, nullptr, pu, pth,
                  plnl, st);
  if (e != cudaSuccess) return e;
  const size_t csm = consume_smem_bytes(s.K, s.n_chains);
  if (csm > 48 * 1024 && (e = raise_smem_limit((const void*)k_ns_consume, c->device, csm)) != cudaSuccess) return e;
  k_ns_consume<<<1, 256, csm, st>>>(s);
  k_ns_stats<<<1, 256, 0, st>>>(s, walk_len, dlogz);
  c->launches += 2;
  return cudaGetLastError();
}

size_t walk_scalars_bytes() { return sizeof(WalkScalars); }

void set_walk_scalars(void* host_buf, double lstar, double scale, int64_t worst, uint64_t counter) {
  WalkScalars* w = static_cast<WalkScalars*>(host_buf);
  w->lstar = lstar;
  w->scale = scale;
  w->worst = worst;
  w->counter = counter;
}

// Static nested sampling run with all state on the device.
static int ns_run_on(gwl_ctx* c, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                     int64_t max_rounds, double scale0, int64_t max_dead, double* dead_lnl, double* dead_logwt,
                     double* dead_u, double* res, cudaStream_t st, int use_graph, const double* resume,
                     double* checkpoint);

// ---------------------------------------------------------------- checkpoint / resume
// The state of a run between rounds, in host doubles (ns_state_doubles):
//   [0] kStateMagic, [1] format version, [2] K, [3] D, [4] dead points stored
//   n, [5] the dead-list capacity of the run that wrote it, [6] L*, [7] walk
//   scale, [8] worst index, [9] round counter, [10, 10 + NS_NSTATS) the
//   accumulators, then live u [K][D], live lnL [K], dead lnL [n], dead
//   ln dX [n], dead u [n][D].
// The walk draws its normals from a counter-based generator keyed by the round
// counter, so a run restored from this state continues bit for bit.
constexpr double kStateMagic = 5.4217e15;
constexpr double kStateVersion = 1.0;
constexpr int kStateHeader = 10 + NS_NSTATS;

// max_dead: the caller's dead-point capacity (the device list holds at least one slot)
static cudaError_t state_save(const NsDev& s, int64_t max_dead, double* out, cudaStream_t st) {
  double stats[NS_NSTATS];
  WalkScalars w;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(stats, s.stats, sizeof(stats), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(&w, s.ws, sizeof(w), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  const int64_t nd = (int64_t)stats[NS_NDEAD];
  const int64_t n = nd < max_dead ? nd : max_dead;
  out[0] = kStateMagic;
  out[1] = kStateVersion;
  out[2] = (double)s.K;
  out[3] = (double)s.D;
  out[4] = (double)n;
  out[5] = (double)max_dead;
  out[6] = w.lstar;
  out[7] = w.scale;
  out[8] = (double)w.worst;
  out[9] = (double)w.counter;
  for (int i = 0; i < NS_NSTATS; ++i) out[10 + i] = stats[i];
  double* p = out + kStateHeader;
  if ((e = cudaMemcpy(p, s.lu, sizeof(double) * s.K * s.D, cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
  p += s.K * s.D;
  if ((e = cudaMemcpy(p, s.ll, sizeof(double) * s.K, cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
  p += s.K;
  if (n > 0) {
    if ((e = cudaMemcpy(p, s.dl, sizeof(double) * n, cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(p + n, s.dw, sizeof(double) * n, cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(p + 2 * n, s.du, sizeof(double) * n * s.D, cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t state_restore(const NsDev& s, const double* in, cudaStream_t st) {
  double stats[NS_NSTATS];
  for (int i = 0; i < NS_NSTATS; ++i) stats[i] = in[10 + i];
  WalkScalars w;
  w.lstar = in[6];
  w.scale = in[7];
  w.worst = (long long)in[8];
  w.counter = (unsigned long long)in[9];
  const int64_t stored = (int64_t)in[4];
  const int64_t n = stored < s.cap ? stored : s.cap;
  const double* p = in + kStateHeader;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(s.stats, stats, sizeof(stats), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(s.ws, &w, sizeof(w), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(s.lu, p, sizeof(double) * s.K * s.D, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(s.ll, p + s.K * s.D, sizeof(double) * s.K, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  p += s.K * (s.D + 1);
  if (n > 0) {
    if ((e = cudaMemcpyAsync(s.dl, p, sizeof(double) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(s.dw, p + stored, sizeof(double) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(s.du, p + 2 * stored, sizeof(double) * n * s.D, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return e;
  }
  return cudaStreamSynchronize(st);  // the host buffer may be released after the call
}

int64_t state_doubles(int64_t K, int64_t D, int64_t max_dead) {
  return kStateHeader + K * (D + 1) + max_dead * (D + 2);
}

// A resume buffer's header against this run's sizes: 0 when it matches.
int state_check(const double* in, int64_t K, int64_t D) {
  if (in[0] != kStateMagic || in[1] != kStateVersion) return 1;
  if (in[2] != (double)K || in[3] != (double)D) return 2;
  if (!(in[4] >= 0.0) || !(in[4] <= in[5])) return 3;
  return 0;
}

// The run is captured into a CUDA graph, which needs a capturable stream: it
// runs on a private non-blocking stream after the caller's stream drains.
int ns_run_impl(gwl_ctx* c, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                int64_t max_rounds, double scale0, int64_t max_dead, double* dead_lnl, double* dead_logwt,
                double* dead_u, double* res, cudaStream_t caller, int use_graph, const double* resume,
                double* checkpoint) {
  if (cudaStreamSynchronize(caller) != cudaSuccess) return -2;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return -2;
  const int rc = ns_run_on(c, K, n_chains, walk_len, seed, dlogz, max_rounds, scale0, max_dead, dead_lnl, dead_logwt,
                           dead_u, res, st, use_graph, resume, checkpoint);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  return rc;
}

static int ns_run_on(gwl_ctx* c, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                     int64_t max_rounds, double scale0, int64_t max_dead, double* dead_lnl, double* dead_logwt,
                     double* dead_u, double* res, cudaStream_t st, int use_graph, const double* resume,
                     double* checkpoint) {
  const int D = (int)theta_stride(c);
  const int64_t cap = max_dead > 0 ? max_dead : 1;
  const int64_t rbuf = n_chains > K ? n_chains : K;
  NsDev s;
  s.K = K;
  s.D = D;
  s.n_chains = n_chains;
  s.cap = cap;
  double* pu = nullptr;
  double* pth = nullptr;
  double* plnl = nullptr;
  void* blocks[16] = {nullptr};
  int nblk = 0;
  auto alloc = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 8);
    if (e == cudaSuccess) blocks[nblk++] = *p;
    return e;
  };
  cudaError_t e = cudaSuccess;
  do {
    if ((e = alloc((void**)&s.lu, sizeof(double) * K * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.ll, sizeof(double) * K)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.cu, sizeof(double) * n_chains * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.cl, sizeof(double) * n_chains)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.cn, sizeof(int32_t) * n_chains)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.rx, sizeof(double) * rbuf)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.rl, sizeof(double) * rbuf)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.dl, sizeof(double) * cap)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.dw, sizeof(double) * cap)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.du, sizeof(double) * cap * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.ws, sizeof(WalkScalars))) != cudaSuccess) break;
    if ((e = alloc((void**)&s.chol, sizeof(double) * D * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&s.stats, sizeof(double) * NS_NSTATS)) != cudaSuccess) break;
    if ((e = alloc((void**)&pu, sizeof(double) * rbuf * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&pth, sizeof(double) * rbuf * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&plnl, sizeof(double) * rbuf)) != cudaSuccess) break;
  } while (false);
  if (e != cudaSuccess) {
    for (int i = 0; i < nblk; ++i) cudaFree(blocks[i]);
    return -2;
  }
  double st0[NS_NSTATS] = {0};
  st0[NS_LNZ] = -INFINITY;
  st0[NS_M] = -INFINITY;
  st0[NS_LMAX] = -INFINITY;
  WalkScalars w0;
  w0.lstar = -INFINITY;
  w0.scale = scale0;
  w0.worst = 0;
  w0.counter = 0;
  int rc = 0;
  do {
    if ((e = cudaMemcpyAsync(s.stats, st0, sizeof(st0), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(s.ws, &w0, sizeof(w0), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = launch_ns_init(c, seed, K, s.lu, pth, st)) != cudaSuccess) break;
    if (resume) {  // continue a checkpointed run: its state replaces the initial draw
      if ((e = state_restore(s, resume, st)) != cudaSuccess) break;
    } else if ((e = launch_loglike(c, pth, K, s.ll, st)) != cudaSuccess) {
      break;
    }
    if (c->walk_kind == GWL_WALK_GALILEAN) {  // warm the gradient path (kernel attributes) before capture
      const int64_t nw = K < n_chains ? K : n_chains;
      if ((e = launch_grad(c, pth, nw, plnl, c->d_gmc, st)) != cudaSuccess) break;
    }
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    const bool prof = c->profiling;
    int64_t per_round = 0;  // kernels in one round's graph
    if (use_graph) {
      c->profiling = false;
      if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
      const int64_t l0 = c->launches;
      cudaError_t er = launch_ns_round(c, s, seed, walk_len, dlogz, pu, pth, plnl, st);
      per_round = c->launches - l0;
      c->launches = l0;
      e = cudaStreamEndCapture(st, &graph);
      c->profiling = prof;
      if (er != cudaSuccess) e = er;
      if (e != cudaSuccess) break;
      if ((e = cudaGraphInstantiate(&gexec, graph, 0)) != cudaSuccess) break;
    }
    double stats[NS_NSTATS];
    int64_t r = 0;
    const int check = 4;
    while (r < max_rounds) {
      const int64_t todo = (max_rounds - r) < check ? (max_rounds - r) : check;
      for (int64_t i = 0; i < todo && e == cudaSuccess; ++i) {
        e = use_graph ? cudaGraphLaunch(gexec, st) : launch_ns_round(c, s, seed, walk_len, dlogz, pu, pth, plnl, st);
        if (e == cudaSuccess) c->launches += use_graph ? per_round : 0;
      }
      if (e != cudaSuccess) break;
      r += todo;
      if ((e = cudaMemcpyAsync(stats, s.stats, sizeof(stats), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
      if (stats[NS_DONE] > 0.5) break;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) break;
    // the state after the last round, before the final live points join the dead list
    if (checkpoint && (e = state_save(s, max_dead, checkpoint, st)) != cudaSuccess) break;
    // rounds after the stopping rule held are no-ops only if none ran: the
    // loop checks every `check` rounds, so report the rounds actually run
    k_ns_final<<<1, 256, 0, st>>>(s);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(stats, s.stats, sizeof(stats), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    const int64_t nd = (int64_t)stats[NS_NDEAD] + K;  // dead points and the final live set
    const int64_t nk = nd < cap ? nd : cap;
    if (dead_lnl && max_dead > 0)
      if ((e = cudaMemcpy(dead_lnl, s.dl, sizeof(double) * nk, cudaMemcpyDeviceToHost)) != cudaSuccess) break;
    if (dead_logwt && max_dead > 0)
      if ((e = cudaMemcpy(dead_logwt, s.dw, sizeof(double) * nk, cudaMemcpyDeviceToHost)) != cudaSuccess) break;
    if (dead_u && max_dead > 0)
      if ((e = cudaMemcpy(dead_u, s.du, sizeof(double) * nk * D, cudaMemcpyDeviceToHost)) != cudaSuccess) break;
    const double rounds = stats[NS_ROUND];
    res[0] = stats[NS_LNZ];
    res[1] = sqrt(fmax(stats[NS_H], 0.0) / (double)K);
    res[2] = stats[NS_H];
    res[3] = (double)nd;
    res[4] = (double)K + rounds * (double)n_chains * (double)walk_len;
    res[5] = rounds;
    WalkScalars wl;
    if ((e = cudaMemcpy(&wl, s.ws, sizeof(wl), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
    res[6] = wl.scale;
    res[7] = rounds > 0 ? stats[NS_ACC_SUM] / rounds : 0.0;
    res[8] = rounds > 0 ? stats[NS_CONSUMED] / rounds : 0.0;
    res[9] = stats[NS_DLOGZ];
    res[10] = (double)nk;
  } while (false);
  if (e != cudaSuccess) rc = -2;
  cudaStreamSynchronize(st);
  for (int i = 0; i < nblk; ++i) cudaFree(blocks[i]);
  return rc;
}

}  // namespace gwl

namespace gwl {
int multi_events(const Multi* m);
int multi_dim(const Multi* m);
gwl_ctx* multi_ctx(const Multi* m, int e);
void multi_count(Multi* m, int64_t n);

// Nested sampling of E events at once: every round is one sequence of
// launches covering all events (per-event kernels run one CTA per event; the
// walk steps evaluate all events' chains in one multi-event batch).
// A multi-event run's state between rounds: [0] kMultiStateMagic, [1] format
// version, [2] events E, [3] K, [4] D, then each event's state in the
// single-event format without dead points (state_doubles(K, D, 0) doubles).
constexpr double kMultiStateMagic = 5.4218e15;
constexpr int kMultiStateHeader = 5;

int64_t multi_state_doubles(int E, int64_t K, int64_t D) { return kMultiStateHeader + E * state_doubles(K, D, 0); }

int multi_state_check(const double* in, int E, int64_t K, int64_t D) {
  if (in[0] != kMultiStateMagic || in[1] != kStateVersion) return 1;
  if (in[2] != (double)E || in[3] != (double)K || in[4] != (double)D) return 2;
  for (int i = 0; i < E; ++i) {
    const double* b = in + kMultiStateHeader + i * state_doubles(K, D, 0);
    if (state_check(b, K, D) != 0 || b[4] != 0.0) return 3;
  }
  return 0;
}

static int multi_ns_run_on(Multi* m, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                           int64_t max_rounds, double scale0, double* res, cudaStream_t st, const double* resume,
                           double* checkpoint) {
  const int E = multi_events(m);
  const int D = multi_dim(m);
  const int64_t rbuf = n_chains > K ? n_chains : K;
  std::vector<void*> blocks;
  auto alloc = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 8);
    if (e == cudaSuccess) blocks.push_back(*p);
    return e;
  };
  double *lu, *ll, *cu, *cl, *rx, *rl, *dl, *dw, *du, *chol, *stats, *pu, *pth, *plnl;
  int32_t* cn;
  WalkScalars* ws;
  NsDev* d_ns;
  PriorInfo* d_pr;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = alloc((void**)&lu, sizeof(double) * E * K * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&ll, sizeof(double) * E * K)) != cudaSuccess) break;
    if ((e = alloc((void**)&cu, sizeof(double) * E * n_chains * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&cl, sizeof(double) * E * n_chains)) != cudaSuccess) break;
    if ((e = alloc((void**)&cn, sizeof(int32_t) * E * n_chains)) != cudaSuccess) break;
    if ((e = alloc((void**)&rx, sizeof(double) * E * rbuf)) != cudaSuccess) break;
    if ((e = alloc((void**)&rl, sizeof(double) * E * rbuf)) != cudaSuccess) break;
    if ((e = alloc((void**)&dl, sizeof(double) * E)) != cudaSuccess) break;
    if ((e = alloc((void**)&dw, sizeof(double) * E)) != cudaSuccess) break;
    if ((e = alloc((void**)&du, sizeof(double) * E * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&chol, sizeof(double) * E * D * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&stats, sizeof(double) * E * NS_NSTATS)) != cudaSuccess) break;
    if ((e = alloc((void**)&ws, sizeof(WalkScalars) * E)) != cudaSuccess) break;
    if ((e = alloc((void**)&d_ns, sizeof(NsDev) * E)) != cudaSuccess) break;
    if ((e = alloc((void**)&d_pr, sizeof(PriorInfo) * E)) != cudaSuccess) break;
    if ((e = alloc((void**)&pu, sizeof(double) * E * rbuf * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&pth, sizeof(double) * E * rbuf * D)) != cudaSuccess) break;
    if ((e = alloc((void**)&plnl, sizeof(double) * E * rbuf)) != cudaSuccess) break;
  } while (false);
  int rc = 0;
  if (e == cudaSuccess) do {
    if ((e = multi_prepare(m, rbuf)) != cudaSuccess) break;
    std::vector<NsDev> hns(E);
    std::vector<PriorInfo> hpr(E);
    std::vector<double> st0((size_t)E * NS_NSTATS, 0.0);
    std::vector<WalkScalars> w0(E);
    for (int i = 0; i < E; ++i) {
      NsDev& s = hns[i];
      s.lu = lu + (int64_t)i * K * D;
      s.ll = ll + (int64_t)i * K;
      s.K = K;
      s.D = D;
      s.cu = cu + (int64_t)i * n_chains * D;
      s.cl = cl + (int64_t)i * n_chains;
      s.cn = cn + (int64_t)i * n_chains;
      s.n_chains = n_chains;
      s.rx = rx + (int64_t)i * rbuf;
      s.rl = rl + (int64_t)i * rbuf;
      s.dl = dl + i;
      s.dw = dw + i;
      s.du = du + (int64_t)i * D;
      s.cap = 0;  // no dead-point list kept for multi-event runs (lnZ and H are accumulated)
      s.ws = ws + i;
      s.chol = chol + (int64_t)i * D * D;
      s.stats = stats + (int64_t)i * NS_NSTATS;
      hpr[i] = prior_info(multi_ctx(m, i));
      st0[(size_t)i * NS_NSTATS + NS_LNZ] = -INFINITY;
      st0[(size_t)i * NS_NSTATS + NS_M] = -INFINITY;
      st0[(size_t)i * NS_NSTATS + NS_LMAX] = -INFINITY;
      w0[i].lstar = -INFINITY;
      w0[i].scale = scale0;
      w0[i].worst = 0;
      w0[i].counter = 0;
    }
    if ((e = cudaMemcpyAsync(d_ns, hns.data(), sizeof(NsDev) * E, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(d_pr, hpr.data(), sizeof(PriorInfo) * E, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(stats, st0.data(), sizeof(double) * st0.size(), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(ws, w0.data(), sizeof(WalkScalars) * E, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      break;
    const int64_t per = state_doubles(K, D, 0);
    if (resume) {  // every event's live set, accumulators and walk state from the checkpoint
      for (int i = 0; i < E && e == cudaSuccess; ++i) e = state_restore(hns[i], resume + kMultiStateHeader + i * per, st);
      if (e != cudaSuccess) break;
    } else {  // initial live points of every event, one batched likelihood call
      for (int i = 0; i < E && e == cudaSuccess; ++i) {
        k_ns_init<<<(unsigned)((K + 127) / 128), 128, 0, st>>>(hpr[i], event_key(seed, i), K, hns[i].lu,
                                                               pth + (int64_t)i * K * D);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) break;
      if ((e = multi_loglike(m, pth, K, ll, st)) != cudaSuccess) break;
    }
    // one round, captured
    const size_t csm = consume_smem_bytes(K, n_chains);
    if (csm > 48 * 1024) {
      if ((e = cudaFuncSetAttribute(k_mns_consume, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm)) !=
          cudaSuccess)
        break;
    }
    const int64_t NC = n_chains * E;
    const unsigned nb = (unsigned)((NC + 127) / 128);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
    {
      cudaError_t er = cudaSuccess;
      k_mns_prep<<<E, 256, 0, st>>>(d_ns);
      k_mwalk_init<<<nb, 128, 0, st>>>(d_ns, n_chains, E, seed);
      for (int s2 = 1; s2 <= walk_len && er == cudaSuccess; ++s2) {
        k_mwalk_propose<<<nb, 128, 0, st>>>(d_ns, d_pr, n_chains, E, seed, (uint32_t)s2, pu, pth);
        er = multi_loglike(m, pth, n_chains, plnl, st);
        k_mwalk_accept<<<nb, 128, 0, st>>>(d_ns, n_chains, E, pu, plnl);
      }
      k_mns_consume<<<E, 256, csm, st>>>(d_ns);
      k_mns_stats<<<E, 256, 0, st>>>(d_ns, walk_len, dlogz);
      cudaError_t ec = cudaStreamEndCapture(st, &graph);
      e = er != cudaSuccess ? er : ec;
    }
    if (e != cudaSuccess) break;
    if ((e = cudaGraphInstantiate(&gexec, graph, 0)) != cudaSuccess) break;
    std::vector<double> hst((size_t)E * NS_NSTATS);
    int64_t r = 0;
    const int check = 4;
    while (r < max_rounds && e == cudaSuccess) {
      const int64_t todo = (max_rounds - r) < check ? (max_rounds - r) : check;
      for (int64_t i = 0; i < todo && e == cudaSuccess; ++i) {
        e = cudaGraphLaunch(gexec, st);
        multi_count(m, 5 + 5 * (int64_t)walk_len);
      }
      if (e != cudaSuccess) break;
      r += todo;
      if ((e = cudaMemcpyAsync(hst.data(), stats, sizeof(double) * hst.size(), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess)
        break;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
      bool all = true;
      for (int i = 0; i < E; ++i) all = all && hst[(size_t)i * NS_NSTATS + NS_DONE] > 0.5;
      if (all) break;
    }
    cudaGraphExecDestroy(gexec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) break;
    if (checkpoint) {  // the state after this call's rounds, before the live points join the evidence
      checkpoint[0] = kMultiStateMagic;
      checkpoint[1] = kStateVersion;
      checkpoint[2] = (double)E;
      checkpoint[3] = (double)K;
      checkpoint[4] = (double)D;
      for (int i = 0; i < E && e == cudaSuccess; ++i) e = state_save(hns[i], 0, checkpoint + kMultiStateHeader + i * per, st);
      if (e != cudaSuccess) break;
    }
    k_mns_final<<<E, 256, 0, st>>>(d_ns);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(hst.data(), stats, sizeof(double) * hst.size(), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      break;
    std::vector<WalkScalars> wl(E);
    if ((e = cudaMemcpyAsync(wl.data(), ws, sizeof(WalkScalars) * E, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    for (int i = 0; i < E; ++i) {
      const double* x = hst.data() + (size_t)i * NS_NSTATS;
      double* o = res + 11 * i;
      const double rounds = x[NS_ROUND];
      o[0] = x[NS_LNZ];
      o[1] = sqrt(fmax(x[NS_H], 0.0) / (double)K);
      o[2] = x[NS_H];
      o[3] = x[NS_NDEAD] + (double)K;
      o[4] = (double)K + rounds * (double)n_chains * (double)walk_len;
      o[5] = rounds;
      o[6] = wl[i].scale;
      o[7] = rounds > 0 ? x[NS_ACC_SUM] / rounds : 0.0;
      o[8] = rounds > 0 ? x[NS_CONSUMED] / rounds : 0.0;
      o[9] = x[NS_DLOGZ];
      o[10] = 0.0;
    }
  } while (false);
  if (e != cudaSuccess) rc = -2;
  cudaStreamSynchronize(st);
  for (void* b : blocks) cudaFree(b);
  return rc;
}

int multi_ns_run(Multi* m, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                 int64_t max_rounds, double scale0, double* res, cudaStream_t caller, const double* resume,
                 double* checkpoint) {
  if (cudaStreamSynchronize(caller) != cudaSuccess) return -2;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return -2;
  const int rc = multi_ns_run_on(m, K, n_chains, walk_len, seed, dlogz, max_rounds, scale0, res, st, resume,
                                 checkpoint);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  return rc;
}

}  // namespace gwl

// ---------------------------------------------------------------- generator check
namespace gwl {
int set_error(int code, const char* fmt, ...);

// One Philox4x32-10 block per record: in = [n][6] words (counter c0..c3, key
// k0, k1), out = [n][4] words -- the device generator of the walks, exposed so
// that it can be checked against the generator's published known answers.
__global__ void k_philox_eval(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* r = in + 6 * i;
  const uint4 w = philox(make_uint4(r[0], r[1], r[2], r[3]), r[4], r[5]);
  out[4 * i] = w.x;
  out[4 * i + 1] = w.y;
  out[4 * i + 2] = w.z;
  out[4 * i + 3] = w.w;
}
}  // namespace gwl

extern "C" int gwl_test_philox(const uint32_t* in_dev, int64_t n, uint32_t* out_dev, void* stream) {
  if (n < 0 || (n > 0 && (!in_dev || !out_dev))) return gwl::set_error(GWL_ERR_ARG, "gwl_test_philox: bad arguments");
  if (n == 0) return GWL_OK;
  gwl::k_philox_eval<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(in_dev, n, out_dev);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gwl::set_error(GWL_ERR_CUDA, "gwl_test_philox: %s", cudaGetErrorString(e));
  return GWL_OK;
}
