// gwl_lnl.cu -- batched log-likelihood: prologue, windowed bin loop, combination.
//
//   lnL_p = sum_d [ Re K_d,p U_d,p - Im K_d,p V_d,p - 1/2 |K_d,p|^2 H_d[ncut_p - 1] ]
//   U_d,p + i V_d,p = sum_{j < ncut_p} G_d,j e^{-2 pi i r_d,j,p}
//   r_d,j,p = sum_m c_m,p B_m(f_j) + tau_d,p f_j      (cycles)
// which is Eq. 2 of the paper (as the log-likelihood ratio) for the TaylorF2
// template, regrouped so that per bin and detector only the phase, one
// sincos and four multiply-adds remain.
//
// Work decomposition: the bins are cut into windows of W bins; a work item is
// (window, slice of proposals).  A CTA stages its window's table rows in
// shared memory with one bulk asynchronous copy (cp.async.bulk, completion on
// an mbarrier, bounded wait), then each warp takes one proposal at a time with
// its 32 lanes striding over the window's bins; the per-lane sums are reduced
// with warp shuffles and written as one partial per (proposal, window).  A
// final kernel adds the partials of each proposal in window order (FP64) and
// forms lnL.  No atomics touch the sums, so results are deterministic.
//
// Precision modes:
//   GWL_FP64  -- phase as an FP64 FMA chain, FP64 sincospi, FP64 sums.
//   GWL_MIXED -- phase in float-float arithmetic (about 48-bit significand,
//                built from error-free TwoProduct/TwoSum on the FP32 pipe),
//                exact reduction to [-1/2, 1/2] cycles, FP32 sincos, FP32
//                per-lane sums over at most W/32 bins, FP32 warp tree, FP64
//                across windows and for the combination.  On GB300 the FP64
//                pipe issues about 2 FMAs per SM per clock against about 128
//                FP32 FMAs, so the float-float phase is several times cheaper
//                than an FP64 one at the same phase precision.
#include <cmath>
#include <type_traits>

#include "gwl_internal.h"

namespace gwl {

// ---------------------------------------------------------------- prologue
__global__ void k_prologue(SegInfo s, const double* __restrict__ theta, int64_t B, int precision,
                           PropMixed* __restrict__ pm, PropF64* __restrict__ pf, PropCommon* __restrict__ pc,
                           int* __restrict__ status) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int ncut = 0;
  if (p < B) {
    double th[11];
    expand_theta(s, theta + p * s.n_dim, th);
    Prologue o;
    prologue(s, th, o);
    PropCommon cm;
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) {
      cm.Kr[d] = o.Kr[d];
      cm.Ki[d] = o.Ki[d];
    }
    cm.hh = o.hh;
    cm.ncut = o.flag ? 0 : o.ncut;
    cm.flag = o.flag;
    pc[p] = cm;
    if (precision == GWL_MIXED) {
      PropMixed q;
#pragma unroll
      for (int m = 0; m < kNBasis; ++m) split_f64(o.c[m], q.ch[m], q.cl[m]);
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) split_f64(o.tau[d], q.th[d], q.tl[d]);
      pm[p] = q;
    } else {
      PropF64 q;
#pragma unroll
      for (int m = 0; m < kNBasis; ++m) q.c[m] = o.c[m];
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) q.tau[d] = o.tau[d];
      pf[p] = q;
    }
    ncut = cm.ncut;
  }
  // largest cut of the batch: one atomic per warp
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) ncut = max(ncut, __shfl_xor_sync(0xffffffffu, ncut, off));
  if ((threadIdx.x & 31) == 0 && ncut > 0) atomicMax(&status[1], ncut);
}

// ---------------------------------------------------------------- per-bin bodies
template <int NDET>
__device__ __forceinline__ void bin_mixed(const float* __restrict__ row, const float (&ch)[kNBasis],
                                          const float (&cl)[kNBasis], const float (&th)[NDET],
                                          const float (&tl)[NDET], float (&U)[NDET], float (&V)[NDET]) {
  // common phase S = sum_m c_m B_m as an unevaluated float pair (s, lo)
  float s, lo;
  {
    float e;
    two_prod(ch[0], row[0], s, e);
    lo = __fmaf_rn(cl[0], row[0], __fmaf_rn(ch[0], row[kNBasis], e));
  }
#pragma unroll
  for (int m = 1; m < kNBasis; ++m) {
    const float bh = row[m], bl = row[kNBasis + m];
    float p, e, t, q;
    two_prod(ch[m], bh, p, e);
    two_sum(s, p, t, q);
    s = t;
    lo = __fmaf_rn(ch[m], bl, __fmaf_rn(cl[m], bh, lo + (q + e)));
  }
  const float fh = row[16], fl = row[17];
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    // r_d = S + tau_d f, then its fractional part in [-1/2, 1/2]
    float p, e, t, q;
    two_prod(th[d], fh, p, e);
    e = __fmaf_rn(th[d], fl, __fmaf_rn(tl[d], fh, e));
    two_sum(s, p, t, q);
    const float l = lo + (e + q);
    const float n = rintf(t);
    const float fr = __fadd_rn(__fsub_rn(t, n), l);  // t - n is exact
    float sn, cs;
    __sincosf(6.283185307179586f * fr, &sn, &cs);
    const float gr = row[18 + 2 * d], gi = row[19 + 2 * d];
    // (gr + i gi)(cs - i sn)
    U[d] = fmaf(gr, cs, fmaf(gi, sn, U[d]));
    V[d] = fmaf(gi, cs, fmaf(-gr, sn, V[d]));
  }
}

template <int NDET>
__device__ __forceinline__ void bin_f64(const double* __restrict__ row, const double (&c)[kNBasis],
                                        const double (&tau)[NDET], double (&U)[NDET], double (&V)[NDET]) {
  double r = c[0] * row[0];
#pragma unroll
  for (int m = 1; m < kNBasis; ++m) r = fma(c[m], row[m], r);
  const double f = row[8];
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    const double rd = fma(tau[d], f, r);
    double sn, cs;
    sincospi(2.0 * rd, &sn, &cs);
    const double gr = row[9 + 2 * d], gi = row[10 + 2 * d];
    U[d] = fma(gr, cs, fma(gi, sn, U[d]));
    V[d] = fma(gi, cs, fma(-gr, sn, V[d]));
  }
}

// ---------------------------------------------------------------- windowed bin loop
struct WinArgs {
  const void* tab;
  int row_elems;  // floats (mixed) or doubles (fp64) per row
  int64_t M;
  int CH;         // bins per window
  int64_t B;
  int slice;      // proposals per work item
  int nw_total;   // ceil(M / CH)
  const PropCommon* pc;
  const void* prop;  // PropMixed* or PropF64*
  double* partials;  // [B][nw_total][2 NDET]
  int* status;
};

template <int NDET, bool MIXED>
__global__ void __launch_bounds__(256) k_window(WinArgs a) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  Elem* sm = reinterpret_cast<Elem*>(smem_raw);
  const Elem* tab = reinterpret_cast<const Elem*>(a.tab);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  const int maxn = a.status[1];
  int nw = (maxn + a.CH - 1) / a.CH;
  if (nw > a.nw_total) nw = a.nw_total;
  const int64_t nsl = (a.B + a.slice - 1) / a.slice;
  const int64_t nitems = (int64_t)nw * nsl;
  if ((int64_t)blockIdx.x >= nitems) return;  // uniform across the CTA

  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();

  int loaded = -1;
  uint32_t parity = 0;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int w = (int)(item / nsl);
    const int64_t sl = item - (int64_t)w * nsl;
    const int j0 = w * a.CH;
    int64_t j1l = (int64_t)j0 + a.CH;
    if (j1l > a.M) j1l = a.M;
    if (j1l > maxn) j1l = maxn;
    const int j1 = (int)j1l;
    if (w != loaded) {
      __syncthreads();  // every warp is done with the previous window
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        const uint32_t bytes = (uint32_t)(j1 - j0) * (uint32_t)a.row_elems * (uint32_t)sizeof(Elem);
        mbar_arrive_expect_tx(&bar, bytes);
        bulk_g2s(sm, tab + (int64_t)j0 * a.row_elems, bytes, &bar);
      }
      if (!mbar_wait_bounded(&bar, parity, a.status)) return;
      parity ^= 1u;
      loaded = w;
    }
    const int64_t pbeg = sl * a.slice;
    const int64_t pend = pbeg + a.slice < a.B ? pbeg + a.slice : a.B;
    for (int64_t p = pbeg + warp; p < pend; p += nwarps) {
      const int ncut = a.pc[p].ncut;
      if (ncut <= j0) continue;
      const int jend = ncut < j1 ? ncut : j1;
      if constexpr (MIXED) {
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
        float U[NDET], V[NDET];
#pragma unroll
        for (int d = 0; d < NDET; ++d) U[d] = V[d] = 0.0f;
        for (int j = j0 + lane; j < jend; j += 32)
          bin_mixed<NDET>(sm + (int64_t)(j - j0) * a.row_elems, ch, cl, th, tl, U, V);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
          for (int d = 0; d < NDET; ++d) {
            U[d] += __shfl_xor_sync(0xffffffffu, U[d], off);
            V[d] += __shfl_xor_sync(0xffffffffu, V[d], off);
          }
        if (lane == 0) {
          double* o = a.partials + ((int64_t)p * a.nw_total + w) * (2 * NDET);
#pragma unroll
          for (int d = 0; d < NDET; ++d) {
            o[2 * d] = (double)U[d];
            o[2 * d + 1] = (double)V[d];
          }
        }
      } else {
        const PropF64* P = reinterpret_cast<const PropF64*>(a.prop) + p;
        double c[kNBasis], tau[NDET];
#pragma unroll
        for (int m = 0; m < kNBasis; ++m) c[m] = P->c[m];
#pragma unroll
        for (int d = 0; d < NDET; ++d) tau[d] = P->tau[d];
        double U[NDET], V[NDET];
#pragma unroll
        for (int d = 0; d < NDET; ++d) U[d] = V[d] = 0.0;
        for (int j = j0 + lane; j < jend; j += 32)
          bin_f64<NDET>(sm + (int64_t)(j - j0) * a.row_elems, c, tau, U, V);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
          for (int d = 0; d < NDET; ++d) {
            U[d] += __shfl_xor_sync(0xffffffffu, U[d], off);
            V[d] += __shfl_xor_sync(0xffffffffu, V[d], off);
          }
        if (lane == 0) {
          double* o = a.partials + ((int64_t)p * a.nw_total + w) * (2 * NDET);
#pragma unroll
          for (int d = 0; d < NDET; ++d) {
            o[2 * d] = U[d];
            o[2 * d + 1] = V[d];
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- combination
template <int NDET>
__global__ void k_finalize(const PropCommon* __restrict__ pc, const double* __restrict__ partials, int64_t B,
                           int CH, int nw_total, double* __restrict__ lnl) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B) return;
  const PropCommon c = pc[p];
  if (c.flag) {
    lnl[p] = -INFINITY;
    return;
  }
  const int nwp = (c.ncut + CH - 1) / CH;
  const double* q = partials + (int64_t)p * nw_total * (2 * NDET);
  double acc = 0.0;
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    double U = 0.0, V = 0.0;
    for (int w = 0; w < nwp; ++w) {
      U += q[w * (2 * NDET) + 2 * d];
      V += q[w * (2 * NDET) + 2 * d + 1];
    }
    acc += c.Kr[d] * U - c.Ki[d] * V;
  }
  lnl[p] = acc - 0.5 * c.hh;
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
  const double f76 = pow(f, -7.0 / 6.0);
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
template <int NDET, bool MIXED>
static cudaError_t run_window(gwl_ctx* c, const WinArgs& a, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_window<NDET, MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  {
    ProfScope ps(c, GWL_KERNEL_BINS, st);
    k_window<NDET, MIXED><<<grid, 256, smem, st>>>(a);
  }
  c->launches++;
  return cudaGetLastError();
}

template <int NDET>
static cudaError_t run_pipeline(gwl_ctx* c, int64_t B, double* lnl, cudaStream_t st) {
  const bool mixed = c->opt.precision == GWL_MIXED;
  int CH = mixed ? c->window_mixed : c->window_f64;
  if (CH > c->M) CH = (int)c->M;
  const int nw_total = (int)((c->M + CH - 1) / CH);
  WinArgs a;
  a.tab = mixed ? (const void*)c->d_tab_mixed : (const void*)c->d_tab_f64;
  a.row_elems = mixed ? c->row_floats : c->row_doubles;
  a.M = c->M;
  a.CH = CH;
  a.B = B;
  a.slice = c->slice;
  a.nw_total = nw_total;
  a.pc = c->d_pc;
  a.prop = mixed ? (const void*)c->d_pm : (const void*)c->d_pf;
  a.partials = c->d_partials;
  a.status = c->d_status;
  const size_t smem = (size_t)CH * a.row_elems * (mixed ? sizeof(float) : sizeof(double));
  const int64_t nsl = (B + c->slice - 1) / c->slice;
  int64_t items = nsl * nw_total;
  int64_t grid = (int64_t)c->num_sms * c->ctas_per_sm;
  if (grid > items) grid = items;
  if (grid < 1) grid = 1;
  cudaError_t e = mixed ? run_window<NDET, true>(c, a, (int)grid, smem, st)
                        : run_window<NDET, false>(c, a, (int)grid, smem, st);
  if (e != cudaSuccess) return e;
  {
    ProfScope ps(c, GWL_KERNEL_COMBINE, st);
    k_finalize<NDET><<<(unsigned)((B + 255) / 256), 256, 0, st>>>(c->d_pc, c->d_partials, B, CH, nw_total, lnl);
  }
  c->launches++;
  return cudaGetLastError();
}

int64_t partials_needed(const gwl_ctx* c, int64_t B) {
  const int CHm = c->window_mixed < c->M ? c->window_mixed : (int)c->M;
  const int CHf = c->window_f64 < c->M ? c->window_f64 : (int)c->M;
  const int CH = c->opt.precision == GWL_MIXED ? CHm : CHf;
  const int64_t nw = (c->M + CH - 1) / CH;
  return B * nw * 2 * c->n_det;
}

cudaError_t launch_prologue(gwl_ctx* c, const double* theta, int64_t B, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(c->d_status + 1, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  {
    ProfScope ps(c, GWL_KERNEL_PROLOGUE, st);
    k_prologue<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(c->seg, theta, B, c->opt.precision, c->d_pm, c->d_pf,
                                                             c->d_pc, c->d_status);
  }
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_loglike(gwl_ctx* c, const double* theta, int64_t B, double* lnl, cudaStream_t st) {
  cudaError_t e = launch_prologue(c, theta, B, st);
  if (e != cudaSuccess) return e;
  switch (c->n_det) {
    case 1: return run_pipeline<1>(c, B, lnl, st);
    case 2: return run_pipeline<2>(c, B, lnl, st);
    case 3: return run_pipeline<3>(c, B, lnl, st);
    default: return run_pipeline<4>(c, B, lnl, st);
  }
}

cudaError_t launch_waveform(gwl_ctx* c, const double* theta, int64_t B, double* h, cudaStream_t st) {
  // the waveform is always produced in FP64: run the FP64 prologue
  const int saved = c->opt.precision;
  c->opt.precision = GWL_FP64;
  cudaError_t e = launch_prologue(c, theta, B, st);
  c->opt.precision = saved;
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((c->M + 255) / 256), (unsigned)B);
  k_waveform<<<grid, 256, 0, st>>>(c->seg, c->d_pf, c->d_pc, c->d_tab_f64, c->row_doubles, h);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace gwl
