// gwl_calgrad.cu -- derivatives of lnL with respect to the calibration model's
// node values (Section 2.2 of the paper; the model in gwl_bins.cuh).
//
// With C_d,j = (1 + dA_d,j) e^{i dphi_d,j} and dA, dphi natural cubic splines
// through the node values yA_d,k, yphi_d,k (dphi in radians),
//   lnL = sum_d [ Re(K_d sum_j G_d,j C_d,j e^{-2 pi i r_d,j}) - 1/2 |K_d|^2 (H_d + X_d) ],
//   X_d = sum_j dA_d,j (2 + dA_d,j) dH_d,j,
// and with s_k(x) the spline's cardinal function of node k (dA_j = sum_k s_k(x_j) yA_k):
//   d lnL / d yA_d,k   = Re(K_d PA_d,k) - |K_d|^2 PH_d,k,
//   d lnL / d yphi_d,k = -Im(K_d Pphi_d,k),
//   PA_k = sum_j s_k(x_j) tA_j,  tA_j = G_j e^{i dphi_j} e^{-2 pi i r_j},
//   Pphi_k = sum_j s_k(x_j) (1 + dA_j) tA_j,  PH_k = sum_j s_k(x_j) (1 + dA_j) dH_j.
// On spline interval i (nodes i, i+1; local t, h^2/6) the cardinal functions
// are s_k = (1 - t) [k = i] + t [k = i+1] + h^2/6 ((1-t)^3 - (1-t)) Q_ik
// + h^2/6 (t^3 - t) Q_i+1,k (m = Q y the curvatures), so each interval needs
// four moments of each of the five real quantities (tA, Pphi's term: complex;
// PH's: real) per detector -- the bins' four spline weights of the
// calibrated likelihood.  A warp takes a (proposal, window): its lanes stride
// over the window's bins (the phase as in the likelihood: anchored float-float
// in the mixed path, FP64 in the FP64 path), keep the current interval's 20
// moments per detector, and when the interval changes sum them over the warp
// (through shared memory) and fold them through Q into the proposal's 2 nn
// derivatives per detector.  A proposal with one window writes them to grad;
// otherwise each window's go to a slot and the combination kernel adds the
// windows in order.
#include <climits>

#include "gwl_bins.cuh"
#include "gwl_ff.cuh"
#include "gwl_sched.cuh"

namespace gwl {

constexpr int kMom = 20;  // 5 quantities x 4 spline weights

struct CalGradArgs {
  const void* tab;     // mixed: delta rows; FP64: FP64 rows
  int row_elems;
  const float* anchor; // mixed: anchor rows
  float df;
  int64_t M;
  int CH;
  int64_t B;
  int nw_total;
  const PropCommon* pc;
  const void* prop;    // PropMixed or PropF64
  int* ctr;            // [w] proposal counter of window w (this kernel's own)
  const int* hist;     // [w] proposals whose last window is w
  const int* maxcut;   // the batch's largest cut
  int* status;
  const void* cal;     // calibration rows (float or double)
  int cal_row;
  int cal_smem;        // element offset of the window's calibration rows in shared memory
  int warp_smem;       // byte offset of the per-warp scratch in shared memory
  const double* theta;
  int64_t stride;      // doubles per row of theta and grad
  int cal_par;         // first calibration parameter (= n_dim)
  int nn;
  const void* calQ;    // [nn][nn]
  double* grad;        // [B][stride]
  void* cpart;         // [B][nw_total][NDET][2 nn]
};

template <typename Acc, typename Node>
struct CalWarp {        // per-warp scratch (shared memory)
  Node nodes[kMaxDet * kMaxCalNodes];
  Acc scr[32][kMom + 1];  // transposed sums (padded against bank conflicts)
  Acc mom[kMom];
  Acc g[kMaxDet][2 * kMaxCalNodes];  // d lnL / d (yA, yphi) of the (proposal, window)
};

template <bool MIXED>
__device__ __forceinline__ void calgrad_stage(const CalGradArgs& a, void* sm, int j0, int j1, uint64_t* bar) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  const uint32_t bytes = (uint32_t)(j1 - j0) * (uint32_t)a.row_elems * (uint32_t)sizeof(Elem);
  uint32_t abytes = 0;
  int a0 = 0;
  if constexpr (MIXED) {
    a0 = j0 / kAnchor;
    abytes = (uint32_t)((j1 + kAnchor - 1) / kAnchor - a0) * (uint32_t)(kAnchorRowFloats * sizeof(float));
  }
  const uint32_t cbytes = (uint32_t)((j1 - j0 + 1) & ~1) * (uint32_t)a.cal_row * (uint32_t)sizeof(Elem);
  mbar_arrive_expect_tx(bar, bytes + abytes + cbytes);
  bulk_g2s(sm, reinterpret_cast<const Elem*>(a.tab) + (int64_t)j0 * a.row_elems, bytes, bar);
  if constexpr (MIXED)
    bulk_g2s(reinterpret_cast<float*>(sm) + (int64_t)a.CH * a.row_elems, a.anchor + (int64_t)a0 * kAnchorRowFloats,
             abytes, bar);
  bulk_g2s(reinterpret_cast<Elem*>(sm) + a.cal_smem, reinterpret_cast<const Elem*>(a.cal) + (int64_t)j0 * a.cal_row,
           cbytes, bar);
}

// The warp's sums of the current interval's moments (per detector, through
// the scratch) folded into the derivatives of nodes i and i+1 and, through Q,
// of every node; the moments are cleared.
template <int NDET, typename Acc, typename Node>
__device__ __forceinline__ void calgrad_flush(const CalGradArgs& a, CalWarp<Acc, Node>& cw, int i, int lane,
                                              const Acc (&K)[NDET][2], Acc (&M)[NDET][kMom]) {
  const Acc* Q = reinterpret_cast<const Acc*>(a.calQ);
  const int nn = a.nn;
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
#pragma unroll
    for (int q = 0; q < kMom; ++q) cw.scr[lane][q] = M[d][q];
    __syncwarp();
    if (lane < kMom) {
      Acc s = (Acc)0;
      for (int l = 0; l < 32; ++l) s += cw.scr[l][lane];
      cw.mom[lane] = s;
    }
    __syncwarp();
    if (lane < 2 * nn) {
      const int k = lane < nn ? lane : lane - nn;
      // the cardinal function of node k on interval i: weights of the four moments
      const Acc w0 = k == i ? (Acc)1 : (Acc)0, w1 = k == i + 1 ? (Acc)1 : (Acc)0;
      const Acc w2 = Q[i * nn + k], w3 = Q[(i + 1) * nn + k];
      auto P = [&](int qty) {  // sum over the four weights of quantity qty's moments
        const Acc* m = cw.mom + 4 * qty;
        return w0 * m[0] + w1 * m[1] + w2 * m[2] + w3 * m[3];
      };
      Acc out;
      if (lane < nn) {  // amplitude node: Re(K PA) - |K|^2 PH
        out = K[d][0] * P(0) - K[d][1] * P(1) - (K[d][0] * K[d][0] + K[d][1] * K[d][1]) * P(4);
      } else {  // phase node: -Im(K Pphi)
        out = -(K[d][0] * P(3) + K[d][1] * P(2));
      }
      cw.g[d][lane] += out;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kMom; ++q) M[d][q] = (Acc)0;
  }
}

// One bin's terms: quantity values v[d][5] (tA re, im; (1 + dA) tA re, im;
// (1 + dA) dH) and the four spline weights w, from the calibration row.
template <int NDET, typename Acc, typename Node>
__device__ __forceinline__ void calgrad_bin(const Acc* __restrict__ crow, const Node* __restrict__ nodes,
                                            const Acc (&fr0)[NDET], const Acc (&g)[2 * NDET], Acc (&v)[NDET][5],
                                            Acc (&w)[4], int& k) {
  constexpr int NP = (3 + NDET + 1) / 2;
  Acc r[2 * NP];
#pragma unroll
  for (int i = 0; i < 2 * NP; ++i) r[i] = crow[i];
  cal_weights<NDET>(r, w);
  CalBin<NDET, Acc> cb;
  cal_eval<NDET>(crow, nodes, cb);
  if constexpr (sizeof(Acc) == 4) k = __float_as_int(r[2]);
  else k = (int)r[2];
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    const Acc fr = fr0[d] - cb.P[d];
    Acc sn, cs;
    if constexpr (sizeof(Acc) == 4) {
      __sincosf(6.283185307179586f * fr, &sn, &cs);
    } else {
      sincospi(2.0 * fr, &sn, &cs);
    }
    const Acc gr = g[2 * d], gi = g[2 * d + 1];
    const Acc tr = gr * cs + gi * sn, ti = gi * cs - gr * sn;  // G e^{-2 pi i (r - dphi)}
    const Acc a1 = (Acc)1 + cb.A[d];
    v[d][0] = tr;
    v[d][1] = ti;
    v[d][2] = a1 * tr;
    v[d][3] = a1 * ti;
    v[d][4] = a1 * cb.H[d];
  }
}

template <int NDET, bool MIXED>
__global__ void __launch_bounds__(256, 1) k_cal_moments(CalGradArgs a) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  using Acc = Elem;
  using Node = typename std::conditional<MIXED, float4, CalNodeD>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  Elem* sm = reinterpret_cast<Elem*>(smem_raw);
  const int lane = threadIdx.x & 31;
  CalWarp<Acc, Node>& cw = reinterpret_cast<CalWarp<Acc, Node>*>(smem_raw + a.warp_smem)[threadIdx.x >> 5];
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int maxn = *a.maxcut;
  int nw = (maxn + a.CH - 1) / a.CH;
  if (nw > a.nw_total) nw = a.nw_total;
  uint32_t parity = 0;
  int n_w = 0;
  int w = nw < 1 ? 0 : start_window(a.hist, 0, nw, blockIdx.x, gridDim.x, &n_w);
  for (; w < nw; ++w) {
    const int j0 = w * a.CH;
    int64_t j1l = (int64_t)j0 + a.CH;
    if (j1l > a.M) j1l = a.M;
    if (j1l > maxn) j1l = maxn;
    const int j1 = (int)j1l;
    int* ctr = a.ctr + w;
    const bool drained = __syncthreads_or(threadIdx.x == 0 && __ldcg(ctr) >= a.B);
    if (drained) continue;
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      calgrad_stage<MIXED>(a, sm, j0, j1, &bar);
    }
    if (!mbar_wait_bounded(&bar, parity, a.status)) return;
    parity ^= 1u;
    const Elem* crows = sm + a.cal_smem;
    drain_window(ctr, a.B, 1, a.pc, j0, lane, [&](int64_t p, int ncut) {
      const int jend = ncut < j1 ? ncut : j1;
      const PropCommon* c = a.pc + p;
      cal_nodes_fill<NDET, MIXED>(a.theta + p * a.stride + a.cal_par, a.nn, a.calQ, lane, cw.nodes);
      Acc K[NDET][2];
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        K[d][0] = (Acc)c->Kr[d];
        K[d][1] = (Acc)c->Ki[d];
      }
      for (int o = lane; o < NDET * 2 * kMaxCalNodes; o += 32) (&cw.g[0][0])[o] = (Acc)0;
      __syncwarp();
      Acc M[NDET][kMom];
#pragma unroll
      for (int d = 0; d < NDET; ++d)
#pragma unroll
        for (int q = 0; q < kMom; ++q) M[d][q] = (Acc)0;
      int cur = -1;  // the interval whose moments M holds
      // the lane's bins: the anchored phase (mixed) or the FP64 phase
      if constexpr (MIXED) {
        const PropMixed* P = reinterpret_cast<const PropMixed*>(a.prop) + p;
        float ch[kNBasis], cl[kNBasis], th[NDET], tl[NDET], dtl[NDET];
#pragma unroll
        for (int m = 0; m < kNBasis; ++m) {
          ch[m] = P->ch[m];
          cl[m] = P->cl[m];
        }
        const float lane_df = (float)lane * a.df;
#pragma unroll
        for (int d = 0; d < NDET; ++d) {
          th[d] = P->th[d];
          tl[d] = P->tl[d];
          dtl[d] = __fmul_rn(th[d], lane_df);
        }
        const float* sanc = sm + (int64_t)a.CH * a.row_elems;
        constexpr int LO = kNBasis + 2 * NDET;
        const int nblk = (jend - j0 + kAnchor - 1) / kAnchor;
        for (int b0 = 0; b0 < nblk; b0 += 32) {
          float an[NDET];
#pragma unroll
          for (int d = 0; d < NDET; ++d) an[d] = 0.0f;
          bool fast = false;
          if (b0 + lane < nblk) fast = anchor_terms<NDET>(sanc + (int64_t)(b0 + lane) * kAnchorRowFloats, ch, cl, th, tl, an);
          const unsigned fast_mask = __ballot_sync(0xffffffffu, fast);
          const int nb = nblk - b0 < 32 ? nblk - b0 : 32;
          for (int it = 0; it < nb; ++it) {
            float ad[NDET];
#pragma unroll
            for (int d = 0; d < NDET; ++d) ad[d] = __fadd_rn(__shfl_sync(0xffffffffu, an[d], it), dtl[d]);
            const int j = j0 + (b0 + it) * kAnchor + lane;
            const bool in = j < jend;
            float v[NDET][5], wts[4], fr0[NDET], gv[2 * NDET];
            int kk = INT_MAX;
            if (in) {
              const float* row = sm + (int64_t)(j - j0) * a.row_elems;
              float ds;
              if ((fast_mask >> it) & 1u) {
                ds = __fmul_rn(ch[0], row[0]);
#pragma unroll
                for (int m = 1; m < kNBasis; ++m) ds = __fmaf_rn(ch[m], row[m], ds);
                ds = __fsub_rn(ds, nearest_int(ds));
              } else {
                float s, lo;
                {
                  float e;
                  two_prod(ch[0], row[0], s, e);
                  lo = __fmaf_rn(cl[0], row[0], __fmaf_rn(ch[0], row[LO], e));
                }
#pragma unroll
                for (int m = 1; m < kNBasis; ++m) {
                  const float bh = row[m], bl = row[LO + m];
                  float pp, e, t, q;
                  two_prod(ch[m], bh, pp, e);
                  two_sum(s, pp, t, q);
                  s = t;
                  lo = __fmaf_rn(ch[m], bl, __fmaf_rn(cl[m], bh, lo + (q + e)));
                }
                ds = __fadd_rn(__fsub_rn(s, nearest_int(s)), lo);
              }
#pragma unroll
              for (int d = 0; d < NDET; ++d) {
                fr0[d] = __fadd_rn(ds, ad[d]);
                gv[2 * d] = row[kNBasis + 2 * d];
                gv[2 * d + 1] = row[kNBasis + 2 * d + 1];
              }
              calgrad_bin<NDET>(crows + (int64_t)(j - j0) * a.cal_row, cw.nodes, fr0, gv, v, wts, kk);
            }
            // the block's bins may lie in several intervals: take them interval by interval
            bool done = !in;
            while (true) {
              const int kmin = __reduce_min_sync(0xffffffffu, done ? INT_MAX : kk);
              if (kmin == INT_MAX) break;
              if (kmin != cur) {
                if (cur >= 0) calgrad_flush<NDET>(a, cw, cur, lane, K, M);
                cur = kmin;
              }
              if (!done && kk == kmin) {
#pragma unroll
                for (int d = 0; d < NDET; ++d)
#pragma unroll
                  for (int qy = 0; qy < 5; ++qy)
#pragma unroll
                    for (int ww = 0; ww < 4; ++ww) M[d][4 * qy + ww] = fmaf(wts[ww], v[d][qy], M[d][4 * qy + ww]);
                done = true;
              }
            }
          }
        }
      } else {
        const PropF64* P = reinterpret_cast<const PropF64*>(a.prop) + p;
        double cc[kNBasis], tau[NDET];
#pragma unroll
        for (int m = 0; m < kNBasis; ++m) cc[m] = P->c[m];
#pragma unroll
        for (int d = 0; d < NDET; ++d) tau[d] = P->tau[d];
        for (int jb = j0; jb < jend; jb += 32) {
          const int j = jb + lane;
          const bool in = j < jend;
          double v[NDET][5], wts[4], fr0[NDET], gv[2 * NDET];
          int kk = INT_MAX;
          if (in) {
            const double* row = sm + (int64_t)(j - j0) * a.row_elems;
            double r = cc[0] * row[0];
#pragma unroll
            for (int m = 1; m < kNBasis; ++m) r = fma(cc[m], row[m], r);
#pragma unroll
            for (int d = 0; d < NDET; ++d) {
              fr0[d] = fma(tau[d], row[8], r);
              gv[2 * d] = row[9 + 2 * d];
              gv[2 * d + 1] = row[10 + 2 * d];
            }
            calgrad_bin<NDET>(crows + (int64_t)(j - j0) * a.cal_row, cw.nodes, fr0, gv, v, wts, kk);
          }
          bool done = !in;
          while (true) {
            const int kmin = __reduce_min_sync(0xffffffffu, done ? INT_MAX : kk);
            if (kmin == INT_MAX) break;
            if (kmin != cur) {
              if (cur >= 0) calgrad_flush<NDET>(a, cw, cur, lane, K, M);
              cur = kmin;
            }
            if (!done && kk == kmin) {
#pragma unroll
              for (int d = 0; d < NDET; ++d)
#pragma unroll
                for (int qy = 0; qy < 5; ++qy)
#pragma unroll
                  for (int ww = 0; ww < 4; ++ww) M[d][4 * qy + ww] = fma(wts[ww], v[d][qy], M[d][4 * qy + ww]);
              done = true;
            }
          }
        }
      }
      if (cur >= 0) calgrad_flush<NDET>(a, cw, cur, lane, K, M);
      // the (proposal, window)'s derivatives: to grad, or to the window's slot
      const int nwp = (ncut + a.CH - 1) / a.CH;
      const int nq = 2 * a.nn;
      for (int o = lane; o < NDET * nq; o += 32) {
        const int d = o / nq, l = o - d * nq;
        if (nwp == 1) a.grad[p * a.stride + a.cal_par + o] = (double)cw.g[d][l];
        else reinterpret_cast<Acc*>(a.cpart)[(p * a.nw_total + w) * (NDET * nq) + o] = cw.g[d][l];
      }
      __syncwarp();
    });
    n_w -= __ldcg(&a.hist[w]);
  }
}

// ---------------------------------------------------------------- launch
// Dynamic shared memory of k_cal_moments for windows of CH bins: the window's
// rows, anchor rows (mixed) and calibration rows, then eight warps' scratch.
size_t calgrad_smem(const gwl_ctx* c, int CH) {
  const bool mixed = c->opt.precision == GWL_MIXED;
  const size_t el = mixed ? sizeof(float) : sizeof(double);
  int64_t elems = (int64_t)CH * (mixed ? c->row_delta : c->row_doubles);
  if (mixed) elems += (int64_t)((CH + kAnchor - 1) / kAnchor) * kAnchorRowFloats;
  elems += (int64_t)(CH + 1) * (mixed ? cal_row_floats(c->n_det) : cal_row_doubles(c->n_det));
  const size_t off = ((size_t)elems * el + 127) & ~(size_t)127;
  return off + 8 * (mixed ? sizeof(CalWarp<float, float4>) : sizeof(CalWarp<double, CalNodeD>));
}

int64_t calgrad_part_elems(const gwl_ctx* c, int64_t B) {
  int CH = c->grad_window;
  if (CH > c->M) CH = (int)c->M;
  const int64_t nw = (c->M + CH - 1) / CH;
  return B * nw * c->n_det * 2 * c->n_cal_nodes;
}

template <int NDET, bool MIXED>
static cudaError_t run_cal_moments(gwl_ctx* c, int64_t B, int* ctr, const int* hist, void* cpart, double* grad,
                                   const double* theta, cudaStream_t st) {
  using Elem = typename std::conditional<MIXED, float, double>::type;
  using Node = typename std::conditional<MIXED, float4, CalNodeD>::type;
  int CH = c->grad_window;
  if (CH > c->M) CH = (int)c->M;
  CalGradArgs a;
  a.tab = MIXED ? (const void*)c->d_tab_delta : (const void*)c->d_tab_f64;
  a.row_elems = MIXED ? c->row_delta : c->row_doubles;
  a.anchor = c->d_anchor;
  a.df = (float)c->df;
  a.M = c->M;
  a.CH = CH;
  a.B = B;
  a.nw_total = (int)((c->M + CH - 1) / CH);
  a.pc = c->d_pc;
  a.prop = MIXED ? (const void*)c->d_pm : (const void*)c->d_pf;
  a.ctr = ctr;
  a.hist = hist;
  a.maxcut = c->d_work;
  a.status = c->d_status;
  a.cal = MIXED ? (const void*)c->d_cal_f : (const void*)c->d_cal_d;
  a.cal_row = MIXED ? c->row_cal_f : c->row_cal_d;
  int64_t elems = (int64_t)CH * a.row_elems;
  if (MIXED) elems += (int64_t)((CH + kAnchor - 1) / kAnchor) * kAnchorRowFloats;
  a.cal_smem = (int)elems;
  elems += (int64_t)(CH + 1) * a.cal_row;
  size_t off = ((size_t)elems * sizeof(Elem) + 127) & ~(size_t)127;
  a.warp_smem = (int)off;
  const size_t smem = off + 8 * sizeof(CalWarp<Elem, Node>);  // = calgrad_smem(c, CH)
  a.theta = theta;
  a.stride = c->seg.stride;
  a.cal_par = c->opt.n_dim;
  a.nn = c->n_cal_nodes;
  a.calQ = MIXED ? (const void*)c->d_calQ_f : (const void*)c->d_calQ_d;
  a.grad = grad;
  a.cpart = cpart;
  cudaError_t e = raise_smem_limit((const void*)k_cal_moments<NDET, MIXED>, c->device, smem);
  if (e != cudaSuccess) return e;
  const int64_t want = ((B + 7) / 8) * a.nw_total;
  int grid = c->num_sms;
  if (want < grid) grid = (int)(want > 0 ? want : 1);
  ProfScope ps(c, GWL_KERNEL_CALGRAD, st);
  k_cal_moments<NDET, MIXED><<<grid, 256, smem, st>>>(a);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_cal_moments(gwl_ctx* c, int64_t B, int* ctr, const int* hist, void* cpart, double* grad,
                               const double* theta, cudaStream_t st) {
  const bool mixed = c->opt.precision == GWL_MIXED;
  switch (c->n_det) {
    case 1: return mixed ? run_cal_moments<1, true>(c, B, ctr, hist, cpart, grad, theta, st)
                         : run_cal_moments<1, false>(c, B, ctr, hist, cpart, grad, theta, st);
    case 2: return mixed ? run_cal_moments<2, true>(c, B, ctr, hist, cpart, grad, theta, st)
                         : run_cal_moments<2, false>(c, B, ctr, hist, cpart, grad, theta, st);
    case 3: return mixed ? run_cal_moments<3, true>(c, B, ctr, hist, cpart, grad, theta, st)
                         : run_cal_moments<3, false>(c, B, ctr, hist, cpart, grad, theta, st);
    default: return mixed ? run_cal_moments<4, true>(c, B, ctr, hist, cpart, grad, theta, st)
                          : run_cal_moments<4, false>(c, B, ctr, hist, cpart, grad, theta, st);
  }
}

}  // namespace gwl
