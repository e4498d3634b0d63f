// gwl_bins.cuh -- per-bin arithmetic shared by the likelihood and gradient bin loops.
#pragma once

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
template <int NDET, bool EXACT_SUM>
__device__ __forceinline__ void phase_mixed(const float (&v)[RowM<NDET>::n], const float (&ch)[kNBasis],
                                            const float (&cl)[kNBasis], const float (&th)[NDET],
                                            const float (&tl)[NDET], float (&sn)[NDET], float (&cs)[NDET]) {
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
  const float fh = v[16], fl = v[17];
  if constexpr (EXACT_SUM) {
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      float p, e, t, q;
      two_prod(th[d], fh, p, e);
      e = __fmaf_rn(th[d], fl, __fmaf_rn(tl[d], fh, e));
      two_sum(s, p, t, q);
      const float l = lo + (e + q);
      const float fr = __fadd_rn(__fsub_rn(t, nearest_int(t)), l);  // t - rint t is exact
      __sincosf(6.283185307179586f * fr, &sn[d], &cs[d]);
    }
  } else {
    const float sf = __fadd_rn(__fsub_rn(s, nearest_int(s)), lo);
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      float p, e;
      two_prod(th[d], fh, p, e);
      e = __fmaf_rn(th[d], fl, __fmaf_rn(tl[d], fh, e));
      const float fr = __fadd_rn(__fadd_rn(sf, __fsub_rn(p, nearest_int(p))), e);
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

template <int NDET>
__device__ __forceinline__ void phase_f64(const double (&v)[RowD<NDET>::n], const double (&c)[kNBasis],
                                          const double (&tau)[NDET], double (&sn)[NDET], double (&cs)[NDET]) {
  double r = c[0] * v[0];
#pragma unroll
  for (int m = 1; m < kNBasis; ++m) r = fma(c[m], v[m], r);
  const double f = v[8];
#pragma unroll
  for (int d = 0; d < NDET; ++d) sincospi(2.0 * fma(tau[d], f, r), &sn[d], &cs[d]);
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

}  // namespace gwl
