// gwl_multi.cu -- many events of uneven durations in one batched evaluation.
//
// A multi-event context groups E single-event contexts (each with its own
// tables, built by gwl_create) that share the detector count, precision and
// sampled dimension.  One batched call evaluates n_per proposals of every
// event: proposal p belongs to event p / n_per.  The bin-loop kernel is
// persistent: its CTAs take (event, window) tasks from one atomic queue,
// stage that event's window of table rows in shared memory (cp.async.bulk on
// an mbarrier, bounded wait) and drain that event's per-window proposal
// counter; events with 4 s and 128 s segments thus share one launch.  With
// the calibration model (every context of the batch with the same number of
// nodes, each with its own node frequencies and tables) the window's
// calibration rows are staged beside its table rows and each proposal's
// spline node values beside the warp, as in the single-event bin loop.  The
// nested-sampling rounds of all events likewise run as one sequence of
// launches (one CTA or warp per event where the work is per event), captured
// once in a CUDA graph and replayed.
#include <cmath>
#include <vector>

#include "gwl_bins.cuh"
#include "gwl_ff.cuh"

namespace gwl {

struct EvDesc {
  SegInfo seg;
  const void* tab;     // delta table (mixed) or FP64 table of this event
  const float* anchor; // anchor rows (mixed)
  float df;
  int row_elems;
  int CH;              // window (bins)
  int nw_total;        // ceil(M / CH)
  int64_t part_off;    // offset of this event's partials block (elements)
  int64_t work_off;    // offset of this event's work block (ints): [0] max cut, [1 + w] counters
  // calibration model (null cal: off)
  const void* cal;     // [M][cal_row] calibration rows, float (mixed) or double
  const void* calQ;    // [nn][nn] natural-spline matrix, float (mixed) or double
  int cal_row;         // elements per calibration row
  int nn;              // nodes
};

// ---------------------------------------------------------------- prologue (one thread per row)
template <bool MIXED>
__global__ void __launch_bounds__(128) k_mprologue(const EvDesc* __restrict__ ev, int64_t n_per, int64_t B,
                                                   const double* __restrict__ theta, PropMixed* __restrict__ pm,
                                                   PropF64* __restrict__ pf, PropCommon* __restrict__ pc,
                                                   int* __restrict__ work) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B) return;
  const int e = (int)(p / n_per);
  const SegInfo& s = ev[e].seg;
  double th[11];
  expand_theta(s, theta + p * s.stride, th);
  const bool ok = physical(th);
  if (!ok) {
    th[0] = 10.0; th[1] = 0.5; th[2] = th[3] = 0.0; th[4] = 100.0;
#pragma unroll
    for (int k = 5; k < 11; ++k) th[k] = 0.0;
  }
  const PNCoeffs<double> P = pn_coeffs(th[1], th[2], th[3]);
  const Scale<double> S = mass_scale(th[0], P.eta, th[4], s.amp_scale);
  double c[kNBasis], ccyc;
  basis_coeffs(P, S, c, ccyc);
  int ncut = (int)s.M;
  if (s.fcut_mode == 0) ncut = count_bins_le(s, 1.0 / (kSix32 * S.a13 * S.a13 * S.a13));
  if (!ok) ncut = 0;
  const Sky<double> k = sky_trig(th[7], th[8], s.gmst);
  double sp, cp;
  sincos(th[6], &sp, &cp);
  const double ci = cos(th[5]);
  double sa, ca;
  if (MIXED) {
    double ang = th[10] + 0.25 * kPi - 2.0 * kPi * frac_near(ccyc);
    ang -= 2.0 * kPi * rint(ang * (0.5 / kPi));
    float sf, cf;
    sincosf((float)ang, &sf, &cf);
    sa = sf;
    ca = cf;
  } else {
    k_angle(th[10], ccyc, sa, ca);
  }
  PropCommon cm;
  double hh = 0.0;
#pragma unroll
  for (int d = 0; d < kMaxDet; ++d) {
    double tau = 0.0;
    cm.Kr[d] = cm.Ki[d] = 0.0;
    if (d < s.n_det && ok) {
      const double* g = s.geom + 9 * d;
      tau = delay(th[9], k, g);
      double Pr, Pi;
      response(k, sp, cp, ci, g, Pr, Pi);
      cm.Kr[d] = S.amp * (Pr * ca - Pi * sa);
      cm.Ki[d] = S.amp * (Pr * sa + Pi * ca);
      if (ncut > 0) hh += S.amp * S.amp * (Pr * Pr + Pi * Pi) * s.H[(int64_t)d * s.M + ncut - 1];
    }
    if (MIXED) split_f64(tau, pm[p].th[d], pm[p].tl[d]);
    else pf[p].tau[d] = tau;
  }
#pragma unroll
  for (int m = 0; m < kNBasis; ++m) {
    if (MIXED) split_f64(ok ? c[m] : 0.0, pm[p].ch[m], pm[p].cl[m]);
    else pf[p].c[m] = ok ? c[m] : 0.0;
  }
  cm.hh = hh;
  cm.ncut = ncut;
  cm.flag = ok ? 0 : 1;
  pc[p] = cm;
  if (ncut > 0) atomicMax(&work[ev[e].work_off], ncut);
}

// ---------------------------------------------------------------- persistent bin loop
struct MultiArgs {
  const EvDesc* ev;
  int E;
  int64_t n_per;
  const PropCommon* pc;
  const void* prop;
  void* partials;
  int* work;
  int* task_counter;
  int* status;
  // calibration model
  const double* theta;  // [B][stride] parameter rows (the node values follow the n_dim sampled coordinates)
  int64_t stride;
  int cal_par;          // first calibration parameter of a row (= n_dim)
  int cal_smem;         // element offset of the window's calibration rows in shared memory
};

template <int NDET, bool MIXED, bool CAL>
__global__ void __launch_bounds__(256, 2) k_mwindow(MultiArgs a) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  using Node = typename std::conditional<MIXED, float4, CalNodeD>::type;
  constexpr int S = CAL ? 3 : 2;  // sums per detector in a partial
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int sh_task;
  __shared__ __align__(32) Node s_nodes[CAL ? 8 * NDET * kMaxCalNodes : 1];
  Node* nodes = s_nodes + (CAL ? (threadIdx.x >> 5) * NDET * kMaxCalNodes : 0);
  Elem* sm = reinterpret_cast<Elem*>(smem_raw);
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity = 0;
  while (true) {
    if (threadIdx.x == 0) sh_task = atomicAdd(a.task_counter, 1);
    __syncthreads();
    int t = sh_task;
    __syncthreads();
    // task t -> (event e, window w): events in order, each with its needed windows
    int e = 0, w = -1;
    for (; e < a.E; ++e) {
      const EvDesc& d = a.ev[e];
      int nw = (a.work[d.work_off] + d.CH - 1) / d.CH;
      if (nw > d.nw_total) nw = d.nw_total;
      if (t < nw) {
        w = t;
        break;
      }
      t -= nw;
    }
    if (w < 0) break;  // no task left (uniform across the CTA)
    const EvDesc& d = a.ev[e];
    const int maxn = a.work[d.work_off];
    const int j0 = w * d.CH;
    int64_t j1l = (int64_t)j0 + d.CH;
    if (j1l > d.seg.M) j1l = d.seg.M;
    if (j1l > maxn) j1l = maxn;
    const int j1 = (int)j1l;
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      const uint32_t bytes = (uint32_t)(j1 - j0) * (uint32_t)d.row_elems * (uint32_t)sizeof(Elem);
      // calibration rows in pairs: a bulk copy moves whole 16-byte units (the table has a row past the last bin)
      const uint32_t cbytes = CAL ? (uint32_t)((j1 - j0 + 1) & ~1) * (uint32_t)d.cal_row * (uint32_t)sizeof(Elem) : 0u;
      mbar_arrive_expect_tx(&bar, bytes + cbytes);
      bulk_g2s(sm, reinterpret_cast<const Elem*>(d.tab) + (int64_t)j0 * d.row_elems, bytes, &bar);
      if constexpr (CAL)
        bulk_g2s(sm + a.cal_smem, reinterpret_cast<const Elem*>(d.cal) + (int64_t)j0 * d.cal_row, cbytes, &bar);
    }
    if (!mbar_wait_bounded(&bar, parity, a.status)) return;
    parity ^= 1u;
    int* ctr = a.work + d.work_off + 1 + w;
    while (true) {
      int pi = 0;
      if (lane == 0) pi = atomicAdd(ctr, 1);
      pi = __shfl_sync(0xffffffffu, pi, 0);
      if (pi >= a.n_per) break;
      const int64_t p = (int64_t)e * a.n_per + pi;
      const int ncut = a.pc[p].ncut;
      if (ncut <= j0) continue;
      const int jend = ncut < j1 ? ncut : j1;
      Elem U[NDET], V[NDET], X[NDET];
#pragma unroll
      for (int q = 0; q < NDET; ++q) U[q] = V[q] = X[q] = (Elem)0;
      if constexpr (CAL) {
        cal_nodes_fill<NDET, MIXED>(a.theta + p * a.stride + a.cal_par, d.nn, d.calQ, lane, nodes);
        __syncwarp();
      }
      if constexpr (MIXED) {
        anchored_sums_cal<NDET, CAL>(sm, d.row_elems, d.anchor + (int64_t)(j0 / kAnchor) * kAnchorRowFloats, d.df,
                                     reinterpret_cast<const PropMixed*>(a.prop) + p, j0, jend, lane, U, V,
                                     sm + a.cal_smem, d.cal_row, reinterpret_cast<const float4*>(nodes), X, nullptr);
      } else {
        const PropF64* P = reinterpret_cast<const PropF64*>(a.prop) + p;
        double c[kNBasis], tau[NDET];
#pragma unroll
        for (int m = 0; m < kNBasis; ++m) c[m] = P->c[m];
#pragma unroll
        for (int q = 0; q < NDET; ++q) tau[q] = P->tau[q];
        for (int j = j0 + lane; j < jend; j += 32) {
          double v[RowD<NDET>::n];
          load_row<NDET>(sm + (int64_t)(j - j0) * d.row_elems, v);
          if constexpr (CAL) {
            CalBin<NDET, double> cb;
            cal_eval<NDET>(reinterpret_cast<const double*>(sm) + a.cal_smem + (int64_t)(j - j0) * d.cal_row,
                           reinterpret_cast<const CalNodeD*>(nodes), cb);
            bin_f64_cal<NDET>(v, c, tau, cb, U, V, X);
          } else {
            bin_f64<NDET>(v, c, tau, U, V);
          }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int q = 0; q < NDET; ++q) {
          U[q] += __shfl_xor_sync(0xffffffffu, U[q], off);
          V[q] += __shfl_xor_sync(0xffffffffu, V[q], off);
          if (CAL) X[q] += __shfl_xor_sync(0xffffffffu, X[q], off);
        }
      if (lane == 0) {
        Elem* o = reinterpret_cast<Elem*>(a.partials) + d.part_off + ((int64_t)pi * d.nw_total + w) * (S * NDET);
#pragma unroll
        for (int q = 0; q < NDET; ++q) {
          o[S * q] = U[q];
          o[S * q + 1] = V[q];
          if constexpr (CAL) o[S * q + 2] = X[q];
        }
      }
      if constexpr (CAL) __syncwarp();  // the warp's node data is replaced by its next proposal's
    }
    __syncthreads();  // all warps done with this window before the next task overwrites it
  }
}

template <int NDET, typename Acc, bool CAL>
__global__ void k_mfinalize(const EvDesc* __restrict__ ev, int64_t n_per, int64_t B, const PropCommon* __restrict__ pc,
                            const Acc* __restrict__ partials, double* __restrict__ lnl) {
  constexpr int S = CAL ? 3 : 2;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B) return;
  const int e = (int)(p / n_per);
  const int64_t pi = p - (int64_t)e * n_per;
  const EvDesc& d = ev[e];
  const PropCommon c = pc[p];
  if (c.flag) {
    lnl[p] = -INFINITY;
    return;
  }
  const int nwp = (c.ncut + d.CH - 1) / d.CH;
  const Acc* q = partials + d.part_off + pi * d.nw_total * (S * NDET);
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < NDET; ++k) {
    double U = 0.0, V = 0.0, X = 0.0;
    for (int w = 0; w < nwp; ++w) {
      U += (double)q[w * (S * NDET) + S * k];
      V += (double)q[w * (S * NDET) + S * k + 1];
      if constexpr (CAL) X += (double)q[w * (S * NDET) + S * k + 2];
    }
    acc += c.Kr[k] * U - c.Ki[k] * V;
    if constexpr (CAL) acc -= 0.5 * (c.Kr[k] * c.Kr[k] + c.Ki[k] * c.Ki[k]) * X;
  }
  lnl[p] = acc - 0.5 * c.hh;
}

// ---------------------------------------------------------------- host side
struct Multi {
  int E = 0;
  int n_det = 0, precision = 0, D = 0;
  int n_dim = 0;
  bool cal = false;
  std::vector<int64_t> cal_gen;  // the contexts' calibration generations the descriptors were built from
  int64_t n_per = 0;
  std::vector<gwl_ctx*> ctxs;
  std::vector<EvDesc> host_ev;
  EvDesc* d_ev = nullptr;
  // scratch for n_per proposals per event
  PropMixed* pm = nullptr;
  PropF64* pf = nullptr;
  PropCommon* pc = nullptr;
  void* partials = nullptr;
  int* work = nullptr;  // event work blocks + task counter at the end
  int64_t work_len = 0;
  int64_t cap_per = 0;
  int num_sms = 0;
  int64_t launches = 0;
  int* status = nullptr;
};

static void multi_free_scratch(Multi* m) {
  cudaFree(m->pm);
  cudaFree(m->pf);
  cudaFree(m->pc);
  cudaFree(m->partials);
  cudaFree(m->work);
  cudaFree(m->d_ev);
  m->pm = nullptr;
  m->pf = nullptr;
  m->pc = nullptr;
  m->partials = nullptr;
  m->work = nullptr;
  m->d_ev = nullptr;
  m->cap_per = 0;
}

// (Re)build the descriptors and scratch for n_per proposals per event.
cudaError_t multi_prepare(Multi* m, int64_t n_per) {
  bool fresh = true;  // no context's calibration changed since the descriptors were built
  for (int e = 0; e < m->E; ++e) fresh = fresh && m->cal_gen[e] == m->ctxs[e]->cal_gen;
  if (fresh && n_per <= m->cap_per && m->d_ev) {
    m->n_per = n_per;
    return cudaSuccess;
  }
  multi_free_scratch(m);
  m->D = (int)theta_stride(m->ctxs[0]);
  m->cal = m->ctxs[0]->n_cal_nodes > 0;
  for (int e = 0; e < m->E; ++e) m->cal_gen[e] = m->ctxs[e]->cal_gen;
  const bool mixed = m->precision == GWL_MIXED;
  m->host_ev.resize(m->E);
  int64_t part = 0, work = 0;
  for (int e = 0; e < m->E; ++e) {
    gwl_ctx* c = m->ctxs[e];
    EvDesc& d = m->host_ev[e];
    d.seg = c->seg;
    d.tab = mixed ? (const void*)c->d_tab_delta : (const void*)c->d_tab_f64;
    d.anchor = c->d_anchor;
    d.df = (float)c->df;
    d.row_elems = mixed ? c->row_delta : c->row_doubles;
    int CH = c->window;
    if (CH > c->M) CH = (int)c->M;
    d.CH = CH;
    d.nw_total = (int)((c->M + CH - 1) / CH);
    d.part_off = part;
    d.work_off = work;
    d.cal = nullptr;
    d.calQ = nullptr;
    d.cal_row = 0;
    d.nn = c->n_cal_nodes;
    if (c->n_cal_nodes) {
      d.cal = mixed ? (const void*)c->d_cal_f : (const void*)c->d_cal_d;
      d.calQ = mixed ? (const void*)c->d_calQ_f : (const void*)c->d_calQ_d;
      d.cal_row = mixed ? c->row_cal_f : c->row_cal_d;
    }
    part += n_per * d.nw_total * (m->cal ? 3 : 2) * m->n_det;
    work += 1 + d.nw_total;
  }
  m->work_len = work + 1;  // + task counter
  const int64_t B = n_per * m->E;
  cudaError_t e;
  if ((e = cudaMalloc(&m->d_ev, sizeof(EvDesc) * m->E)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(m->d_ev, m->host_ev.data(), sizeof(EvDesc) * m->E, cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if ((e = cudaMalloc(&m->pm, sizeof(PropMixed) * B)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->pf, sizeof(PropF64) * B)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->pc, sizeof(PropCommon) * B)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->partials, (mixed ? sizeof(float) : sizeof(double)) * (size_t)(part > 0 ? part : 1))) !=
      cudaSuccess)
    return e;
  if ((e = cudaMalloc(&m->work, sizeof(int) * m->work_len)) != cudaSuccess) return e;
  m->cap_per = n_per;
  m->n_per = n_per;
  return cudaSuccess;
}

template <int NDET, bool MIXED, bool CAL>
static cudaError_t multi_run(Multi* m, const double* theta, int64_t n_per, double* lnl, cudaStream_t st) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  const int64_t B = n_per * m->E;
  cudaError_t e = cudaMemsetAsync(m->work, 0, sizeof(int) * m->work_len, st);
  if (e != cudaSuccess) return e;
  k_mprologue<MIXED><<<(unsigned)((B + 127) / 128), 128, 0, st>>>(m->d_ev, n_per, B, theta, m->pm, m->pf, m->pc,
                                                                   m->work);
  m->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int CHmax = 0, rowmax = 0, calmax = 0;
  for (const EvDesc& d : m->host_ev) {
    CHmax = d.CH > CHmax ? d.CH : CHmax;
    rowmax = d.row_elems > rowmax ? d.row_elems : rowmax;
    calmax = d.cal_row > calmax ? d.cal_row : calmax;
  }
  // the window's table rows, then (calibration) its calibration rows, staged in pairs
  const int64_t cal_smem = (int64_t)CHmax * rowmax;
  const size_t smem = (size_t)(cal_smem + (CAL ? (int64_t)(CHmax + 1) * calmax : 0)) * sizeof(Elem);
  if ((e = raise_smem_limit((const void*)k_mwindow<NDET, MIXED, CAL>, m->ctxs[0]->device, smem)) != cudaSuccess)
    return e;
  MultiArgs a;
  a.ev = m->d_ev;
  a.E = m->E;
  a.n_per = n_per;
  a.pc = m->pc;
  a.prop = MIXED ? (const void*)m->pm : (const void*)m->pf;
  a.partials = m->partials;
  a.work = m->work;
  a.task_counter = m->work + m->work_len - 1;
  a.status = m->status;
  a.theta = theta;
  a.stride = m->D;
  a.cal_par = m->n_dim;
  a.cal_smem = (int)cal_smem;
  k_mwindow<NDET, MIXED, CAL><<<m->num_sms * 2, 256, smem, st>>>(a);
  m->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_mfinalize<NDET, Elem, CAL><<<(unsigned)((B + 63) / 64), 64, 0, st>>>(m->d_ev, n_per, B, m->pc,
                                                                           (const Elem*)m->partials, lnl);
  m->launches++;
  return cudaGetLastError();
}

template <int NDET>
static cudaError_t multi_dispatch(Multi* m, const double* theta, int64_t n_per, double* lnl, cudaStream_t st) {
  const bool mixed = m->precision == GWL_MIXED;
  if (m->cal)
    return mixed ? multi_run<NDET, true, true>(m, theta, n_per, lnl, st)
                 : multi_run<NDET, false, true>(m, theta, n_per, lnl, st);
  return mixed ? multi_run<NDET, true, false>(m, theta, n_per, lnl, st)
               : multi_run<NDET, false, false>(m, theta, n_per, lnl, st);
}

cudaError_t multi_loglike(Multi* m, const double* theta, int64_t n_per, double* lnl, cudaStream_t st) {
  switch (m->n_det) {
    case 1: return multi_dispatch<1>(m, theta, n_per, lnl, st);
    case 2: return multi_dispatch<2>(m, theta, n_per, lnl, st);
    case 3: return multi_dispatch<3>(m, theta, n_per, lnl, st);
    default: return multi_dispatch<4>(m, theta, n_per, lnl, st);
  }
}

Multi* multi_new(gwl_ctx* const* ctxs, int E) {
  Multi* m = new Multi();
  m->E = E;
  m->ctxs.assign(ctxs, ctxs + E);
  m->n_det = ctxs[0]->n_det;
  m->precision = ctxs[0]->opt.precision;
  m->n_dim = ctxs[0]->opt.n_dim;
  m->D = (int)theta_stride(ctxs[0]);  // the sampled coordinates, then the calibration parameters
  m->cal = ctxs[0]->n_cal_nodes > 0;
  m->cal_gen.assign(E, -1);
  m->num_sms = ctxs[0]->num_sms;
  m->status = ctxs[0]->d_status;
  return m;
}

void multi_delete(Multi* m) {
  if (!m) return;
  multi_free_scratch(m);
  delete m;
}

int64_t multi_launches(const Multi* m) { return m ? m->launches : 0; }
// The contexts still share their number of calibration nodes (a context's
// calibration may have been changed since the batch was made).
bool multi_consistent(const Multi* m) {
  if (!m) return false;
  for (int e = 1; e < m->E; ++e)
    if (m->ctxs[e]->n_cal_nodes != m->ctxs[0]->n_cal_nodes) return false;
  return true;
}
int multi_events(const Multi* m) { return m->E; }
int multi_dim(const Multi* m) { return (int)theta_stride(m->ctxs[0]); }  // walk dimension, current
gwl_ctx* multi_ctx(const Multi* m, int e) { return m->ctxs[e]; }
void multi_count(Multi* m, int64_t n) { m->launches += n; }

}  // namespace gwl
