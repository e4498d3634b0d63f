// gwl_lanes.cu -- the mixed likelihood bin loop with one proposal per lane.
//
// Same sums as k_window (Eq. 2 regrouped: U_d + i V_d = sum_j G_d,j e^{-2 pi i r_d,j},
// the anchored float-float phase of gwl_bins.cuh), with the work laid out the
// other way round: each lane owns one proposal and the 32 lanes of a warp
// walk the same bins together, so a table row is one broadcast shared-memory
// read for the whole warp, each lane forms its own proposal's anchor terms
// (no lane idles through another proposal's anchor pass), and no warp
// reduction is needed.  The bins are cut into chunks of SEG bins (SEG a
// multiple of the 32-bin anchor block; windows hold whole chunks); a work
// item is (chunk c, group of 32 proposals).  So that the 32 proposals of a
// group end at nearly the same bin, the prologue files every proposal in the
// bucket of its last chunk (bucket_push); the proposals active in chunk c
// are then, in descending bucket order, a prefix of length S_c (S the suffix
// sums of the bucket counts), and item g of chunk c takes positions
// 32 g .. 32 g + 31 of it.  A lane sums its proposal's bins of the chunk in
// FP32 (bin order); a proposal with one chunk is combined at once, otherwise
// each chunk's sums go to a per-(proposal, chunk) slot and the lane that
// completes the last of them adds the slots in chunk order (FP64) and
// combines.  Every proposal's arithmetic is fixed whatever group, warp or CTA
// processes it, so results are deterministic.
//
// Windows, their bulk copies into shared memory (cp.async.bulk on an
// mbarrier with a bounded wait) and the work-weighted start window of each
// CTA are those of k_window.
#include "gwl_bins.cuh"
#include "gwl_sched.cuh"

namespace gwl {

// Largest number of chunks the lane kernel handles (suffix sums in shared memory).
constexpr int kLaneMaxChunks = 2048;
// Largest per-(proposal, chunk) slot array with 64-bin chunks before the
// chunks grow to whole windows.
constexpr int64_t kLaneSlotBytes = 64ll << 20;

struct LaneArgs {
  const float* tab;     // delta rows [M][row_elems]
  const float* anchor;  // anchor rows [ceil(M / 32)][kAnchorRowFloats]
  int row_elems;
  int64_t M;
  int CH;        // bins per window (a multiple of SEG)
  int SEG;       // bins per chunk (a multiple of 32)
  int NCH;       // ceil(M / SEG)
  int nw_total;  // ceil(M / CH)
  int64_t B;
  float df;
  const PropCommon* pc;
  const PropMixed* pm;
  float* slots;       // [B][NCH][2 NDET] per-chunk sums of multi-chunk proposals
  int* work;          // [0] largest cut, [1 + w] item counter of window w
  const int* hist;    // [w] proposals whose last window is w
  int* pdone;         // [B] chunks of proposal p already summed
  const int* bcount;  // [NCH] proposals whose last chunk is K
  const int* blist;   // [NCH][B] those proposals
  double* lnl;        // [B]
  int* status;        // latched error bits
  unsigned long long* ffc;  // diagnostic counter of float-float-delta blocks, or null
};

// The window's rows [j0, j1) and their anchor rows into shared memory (one
// thread; completion on bar): the layout of k_window's mixed path.
__device__ __forceinline__ void lanes_stage(const LaneArgs& a, float* sm, int j0, int j1, uint64_t* bar) {
  const uint32_t bytes = (uint32_t)(j1 - j0) * (uint32_t)a.row_elems * (uint32_t)sizeof(float);
  const int a0 = j0 / kAnchor, a1 = (j1 + kAnchor - 1) / kAnchor;
  const uint32_t abytes = (uint32_t)(a1 - a0) * (uint32_t)(kAnchorRowFloats * sizeof(float));
  mbar_arrive_expect_tx(bar, bytes + abytes);
  bulk_g2s(sm, a.tab + (int64_t)j0 * a.row_elems, bytes, bar);
  bulk_g2s(sm + (int64_t)a.CH * a.row_elems, a.anchor + (int64_t)a0 * kAnchorRowFloats, abytes, bar);
}

// One lane's sums over the bins [jb, jb + 32) of one anchor block, bins at or
// past jb + nb excluded: those read the zero row zr instead (their terms
// vanish), so the loop has no branches.  sr = the block's first delta row
// (broadcast reads), an = the block's anchor terms, tdf = tau_d df; FAST: the
// block's phase deltas run in FP32 (else float-float).  Two bins per
// iteration, in straight-line code, so that their dependent chains interleave.
template <int NDET, bool FAST>
__device__ __forceinline__ void lane_bin(const float* __restrict__ row, const float (&ch)[kNBasis],
                                         const float (&cl)[kNBasis], const float (&an)[NDET],
                                         const float (&tdf)[NDET], float kf, float (&U)[NDET], float (&V)[NDET]) {
  constexpr int RX = 4 * ((kNBasis + 2 * NDET + 3) / 4);       // floats of the FP32-delta bin
  constexpr int RXF = 4 * ((2 * kNBasis + 2 * NDET + 3) / 4);  // floats of the float-float-delta bin
  constexpr int LO = kNBasis + 2 * NDET;
  float v[RXF];
#pragma unroll
  for (int q = 0; q < RX / 4; ++q) *reinterpret_cast<float4*>(&v[4 * q]) = reinterpret_cast<const float4*>(row)[q];
  float ds;
  if constexpr (FAST) {
    ds = __fmul_rn(ch[0], v[0]);
#pragma unroll
    for (int m = 1; m < kNBasis; ++m) ds = __fmaf_rn(ch[m], v[m], ds);
    ds = __fsub_rn(ds, nearest_int(ds));  // exact
  } else {
#pragma unroll
    for (int q = RX / 4; q < RXF / 4; ++q)
      *reinterpret_cast<float4*>(&v[4 * q]) = reinterpret_cast<const float4*>(row)[q];
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
    ds = __fadd_rn(__fsub_rn(s, nearest_int(s)), lo);
  }
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    // |ds + an + tau df k| < 1.5 cycles: the hardware sine and cosine take it unreduced
    const float fr = __fadd_rn(ds, __fmaf_rn(tdf[d], kf, an[d]));
    float sn, cs;
    __sincosf(6.283185307179586f * fr, &sn, &cs);
    const float gr = v[kNBasis + 2 * d], gi = v[kNBasis + 2 * d + 1];
    U[d] = fmaf(gr, cs, fmaf(gi, sn, U[d]));
    V[d] = fmaf(gi, cs, fmaf(-gr, sn, V[d]));
  }
}

template <int NDET>
__device__ __forceinline__ void lane_block(const float* __restrict__ sr, const float* __restrict__ zr, int row_elems,
                                           int nb, const float (&ch)[kNBasis], const float (&cl)[kNBasis],
                                           const float (&an)[NDET], const float (&tdf)[NDET], bool fast,
                                           float (&U)[NDET], float (&V)[NDET]) {
  float kf = 0.0f;
  if (fast) {
#pragma unroll 2
    for (int k = 0; k < kAnchor; k += 2, kf += 2.0f) {
      const float* r0 = k < nb ? sr + k * row_elems : zr;
      const float* r1 = k + 1 < nb ? sr + (k + 1) * row_elems : zr;
      lane_bin<NDET, true>(r0, ch, cl, an, tdf, kf, U, V);
      lane_bin<NDET, true>(r1, ch, cl, an, tdf, kf + 1.0f, U, V);
    }
  } else {
    for (int k = 0; k < kAnchor; k += 2, kf += 2.0f) {
      const float* r0 = k < nb ? sr + k * row_elems : zr;
      const float* r1 = k + 1 < nb ? sr + (k + 1) * row_elems : zr;
      lane_bin<NDET, false>(r0, ch, cl, an, tdf, kf, U, V);
      lane_bin<NDET, false>(r1, ch, cl, an, tdf, kf + 1.0f, U, V);
    }
  }
}

// lnL of proposal p from its FP64 sums (one lane).
template <int NDET>
__device__ __forceinline__ double lane_combine(const PropCommon* __restrict__ c, const double (&U)[NDET],
                                               const double (&V)[NDET]) {
  double acc = 0.0;
#pragma unroll
  for (int d = 0; d < NDET; ++d) acc += c->Kr[d] * U[d] - c->Ki[d] * V[d];
  return acc - 0.5 * c->hh;
}

template <int NDET>
__global__ void __launch_bounds__(256, 2) k_lanes(LaneArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_suf[kLaneMaxChunks + 1];  // S_K = proposals whose last chunk is K or later
  __shared__ int s_off[kAnchor * 2 + 1];      // item offsets of the window's chunks
  float* sm = reinterpret_cast<float*>(smem_raw);
  const float* sanc = sm + (int64_t)a.CH * a.row_elems;
  // a zero row after the anchor rows: bins past a lane's cut read it (their terms vanish)
  float* zrow = sm + (int64_t)a.CH * a.row_elems + (int64_t)((a.CH + kAnchor - 1) / kAnchor) * kAnchorRowFloats;
  for (int i = threadIdx.x; i < a.row_elems; i += blockDim.x) zrow[i] = 0.0f;
  const int lane = threadIdx.x & 31;
  const int cpw = a.CH / a.SEG;  // chunks per window (<= 2 kAnchor: windows <= 2048 bins, chunks >= 32)

  // window 0's rows do not depend on the prologue: their copy starts before the wait
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    lanes_stage(a, sm, 0, a.CH < a.M ? a.CH : (int)a.M, &bar);
  }
  bool w0_pending = true;
  uint32_t parity = 0;
  cudaGridDependencySynchronize();  // the prologue's outputs (cuts, coefficients, buckets) are visible

  const int maxn = a.work[0];
  int nw = (maxn + a.CH - 1) / a.CH;
  if (nw > a.nw_total) nw = a.nw_total;
  // suffix sums of the bucket counts, S_NCH = 0 (a CTA-wide scan from the top bucket down)
  {
    const int per = (a.NCH + 255) / 256;
    const int k1 = a.NCH - threadIdx.x * per;  // this thread sums buckets [k0, k1)
    const int k0 = k1 - per > 0 ? k1 - per : 0;
    int own = 0;
    for (int k = k0; k < k1; ++k) own += __ldcg(&a.bcount[k]);
    // inclusive scan over threads in thread order (thread 0 holds the top buckets)
    int incl = own;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    __shared__ int s_warp[8];
    if (lane == 31) s_warp[threadIdx.x >> 5] = incl;
    __syncthreads();
    int before = incl - own;
    for (int v = 0; v < (int)(threadIdx.x >> 5); ++v) before += s_warp[v];
    int run = before;
    for (int k = k1 - 1; k >= k0; --k) {
      run += __ldcg(&a.bcount[k]);
      s_suf[k] = run;
    }
    if (threadIdx.x == 0) s_suf[a.NCH] = 0;
  }
  __syncthreads();

  int n_w = 0;
  int w = nw < 1 ? 0 : start_window(a.hist, 0, nw, blockIdx.x, gridDim.x, &n_w);
  for (; w < nw; ++w) {
    const int j0 = w * a.CH;
    int64_t j1l = (int64_t)j0 + a.CH;
    if (j1l > a.M) j1l = a.M;
    if (j1l > maxn) j1l = maxn;
    const int j1 = (int)j1l;  // > j0 because w < nw
    const int c_lo = j0 / a.SEG;
    const int c_hi = (j1 + a.SEG - 1) / a.SEG;
    // items of the window: chunk c has ceil(S_c / 32) groups
    if (threadIdx.x == 0) {
      int o = 0;
      for (int c = c_lo; c < c_hi; ++c) {
        s_off[c - c_lo] = o;
        o += (s_suf[c] + 31) >> 5;
      }
      s_off[c_hi - c_lo] = o;
    }
    __syncthreads();
    const int n_items = s_off[c_hi - c_lo];
    int* ctr = a.work + 1 + w;
    const bool drained = __syncthreads_or(threadIdx.x == 0 && __ldcg(ctr) >= n_items);
    if (!drained) {
      if (w0_pending) {
        if (!mbar_wait_bounded(&bar, parity, a.status)) return;
        parity ^= 1u;
        w0_pending = false;
        if (w != 0) __syncthreads();  // every thread has seen the copy land before the barrier is armed again
      }
      if (w != 0) {
        if (threadIdx.x == 0) {
          fence_proxy_async_smem();
          lanes_stage(a, sm, j0, j1, &bar);
        }
        if (!mbar_wait_bounded(&bar, parity, a.status)) return;
        parity ^= 1u;
      }
      while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(ctr, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        int ci = 0;
        while (s_off[ci + 1] <= item) ++ci;
        const int c = c_lo + ci;
        const int pos = 32 * (item - s_off[ci]) + lane;
        const bool active = pos < s_suf[c];
        // this lane's proposal: bucket K with S_{K+1} <= pos < S_K, K >= c
        int64_t p = 0;
        int K = c;
        if (active) {
          int lo = c, hi = a.NCH;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_suf[mid] > pos) lo = mid;
            else hi = mid;
          }
          K = lo;
          p = __ldcg(&a.blist[(int64_t)K * a.B + (pos - s_suf[K + 1])]);
        }
        int ncut = 0;
        float ch[kNBasis], cl[kNBasis], th[NDET], tl[NDET], tdf[NDET];
        if (active) {
          const PropMixed* P = a.pm + p;
#pragma unroll
          for (int q = 0; q < kNBasis / 4; ++q) {
            *reinterpret_cast<float4*>(&ch[4 * q]) = reinterpret_cast<const float4*>(P->ch)[q];
            *reinterpret_cast<float4*>(&cl[4 * q]) = reinterpret_cast<const float4*>(P->cl)[q];
          }
          const float4 t4 = *reinterpret_cast<const float4*>(P->th), l4 = *reinterpret_cast<const float4*>(P->tl);
          const float tt[4] = {t4.x, t4.y, t4.z, t4.w}, ll[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
          for (int d = 0; d < NDET; ++d) {
            th[d] = tt[d];
            tl[d] = ll[d];
          }
          ncut = a.pc[p].ncut;
        } else {
#pragma unroll
          for (int m = 0; m < kNBasis; ++m) ch[m] = cl[m] = 0.0f;
#pragma unroll
          for (int d = 0; d < NDET; ++d) th[d] = tl[d] = 0.0f;
        }
#pragma unroll
        for (int d = 0; d < NDET; ++d) tdf[d] = __fmul_rn(th[d], a.df);
        // bins of this chunk for this lane: [cs0, jend); the group walks to the largest jend
        const int cs0 = c * a.SEG;
        int jend = cs0 + a.SEG;
        if (jend > j1) jend = j1;
        if (jend > ncut) jend = ncut;
        if (!active) jend = cs0;
        const int jg = __reduce_max_sync(0xffffffffu, jend);
        float U[NDET], V[NDET];
#pragma unroll
        for (int d = 0; d < NDET; ++d) U[d] = V[d] = 0.0f;
        for (int jb = cs0; jb < jg; jb += kAnchor) {
          float an[NDET];
          const bool fast = anchor_terms<NDET>(sanc + (int64_t)((jb - j0) / kAnchor) * kAnchorRowFloats, ch, cl, th,
                                               tl, an);
          int nb = jend - jb;
          nb = nb < 0 ? 0 : nb;
          if (a.ffc) {  // one count per block and proposal that takes the float-float delta
            const unsigned n = __popc(__ballot_sync(0xffffffffu, !fast && nb > 0));
            if (lane == 0 && n) atomicAdd(a.ffc, (unsigned long long)n);
          }
          lane_block<NDET>(sm + (int64_t)(jb - j0) * a.row_elems, zrow, a.row_elems, nb, ch, cl, an, tdf, fast, U,
                           V);
        }
        if (!active) continue;
        if (K == 0) {  // the proposal's only chunk
          double Ud[NDET], Vd[NDET];
#pragma unroll
          for (int d = 0; d < NDET; ++d) {
            Ud[d] = (double)U[d];
            Vd[d] = (double)V[d];
          }
          a.lnl[p] = lane_combine<NDET>(a.pc + p, Ud, Vd);
          continue;
        }
        float* slot = a.slots + (p * a.NCH + c) * (2 * NDET);
#pragma unroll
        for (int d = 0; d < NDET; ++d) *reinterpret_cast<float2*>(&slot[2 * d]) = make_float2(U[d], V[d]);
        __threadfence();
        const int done = atomicAdd(&a.pdone[p], 1);
        if (done != K) continue;
        __threadfence();
        // the last chunk: add the chunks' sums in chunk order (FP64) and combine
        double Ud[NDET], Vd[NDET];
#pragma unroll
        for (int d = 0; d < NDET; ++d) Ud[d] = Vd[d] = 0.0;
        const float* q = a.slots + p * a.NCH * (2 * NDET);
        for (int cc = 0; cc <= K; ++cc)
#pragma unroll
          for (int d = 0; d < NDET; ++d) {
            const float2 uv = __ldcg(reinterpret_cast<const float2*>(&q[cc * (2 * NDET) + 2 * d]));
            Ud[d] += (double)uv.x;
            Vd[d] += (double)uv.y;
          }
        a.lnl[p] = lane_combine<NDET>(a.pc + p, Ud, Vd);
      }
    }
    __syncthreads();  // every warp is done with the window's rows before they are replaced
  }
  if (w0_pending) mbar_wait_bounded(&bar, parity, a.status);  // no copy may outlive the CTA
}

// ---------------------------------------------------------------- host side
// Chunk size of the lane kernel for a batch of B on this context, or 0 when
// the warp-per-proposal kernel runs (the FP64 path, the calibration model,
// small batches, segments with too many chunks, or the tuning says so).
int lanes_seg(const gwl_ctx* c, int64_t B) {
  if (c->opt.precision != GWL_MIXED || c->n_cal_nodes) return 0;
  if (c->bin_kernel == GWL_BINS_WARP) return 0;
  if (c->bin_kernel == GWL_BINS_AUTO && B < 2048) return 0;
  const int CH = c->window > c->M ? (int)c->M : c->window;
  if (CH % 32 || CH > 2 * kAnchor * 32) return 0;
  const int seg = c->lane_chunk;
  const int64_t n = (c->M + seg - 1) / seg;
  if (seg >= 32 && CH % seg == 0 && n <= kLaneMaxChunks &&
      B * n * 2 * c->n_det * (int64_t)sizeof(float) <= kLaneSlotBytes)
    return seg;
  const int64_t nch = (c->M + CH - 1) / CH;
  return nch <= kLaneMaxChunks ? CH : 0;
}

int64_t lanes_list_ints(const gwl_ctx* c, int64_t B) {
  const int seg = lanes_seg(c, B);
  return seg ? (c->M + seg - 1) / seg * B : 0;
}

int64_t lanes_slot_floats(const gwl_ctx* c, int64_t B) {
  const int seg = lanes_seg(c, B);
  return seg ? (c->M + seg - 1) / seg * B * 2 * c->n_det : 0;
}

template <int NDET>
static cudaError_t run_lanes(gwl_ctx* c, int64_t B, double* lnl, int* work, int* hist, int* pdone, int* bcount,
                             int seg, cudaStream_t st) {
  const int CH = c->window > c->M ? (int)c->M : c->window;
  LaneArgs a;
  a.tab = c->d_tab_delta;
  a.anchor = c->d_anchor;
  a.row_elems = c->row_delta;
  a.M = c->M;
  a.CH = CH;
  a.SEG = seg;
  a.NCH = (int)((c->M + seg - 1) / seg);
  a.nw_total = (int)((c->M + CH - 1) / CH);
  a.B = B;
  a.df = (float)c->df;
  a.pc = c->d_pc;
  a.pm = c->d_pm;
  a.slots = reinterpret_cast<float*>(c->d_partials);
  a.work = work;
  a.hist = hist;
  a.pdone = pdone;
  a.bcount = bcount;
  a.blist = c->d_blist;
  a.lnl = lnl;
  a.status = c->d_status;
  a.ffc = c->count_ff ? c->d_ffc : nullptr;
  const size_t smem = ((size_t)(CH + 1) * a.row_elems + (size_t)((CH + kAnchor - 1) / kAnchor) * kAnchorRowFloats) *
                      sizeof(float);
  cudaError_t e = raise_smem_limit((const void*)k_lanes<NDET>, c->device, smem);
  if (e != cudaSuccess) return e;
  // every SM busy; fewer CTAs when the batch has few items
  const int64_t items = (B + 31) / 32 * a.NCH;
  int grid = c->num_sms * c->ctas_per_sm;
  if (items < grid) grid = (int)(items > 0 ? items : 1);
  ProfScope ps(c, GWL_KERNEL_BINS, st);
  e = launch_pdl(k_lanes<NDET>, dim3(grid), dim3(256), smem, st, a);
  c->launches++;
  return e;
}

cudaError_t launch_lanes(gwl_ctx* c, int64_t B, double* lnl, int* work, int* hist, int* pdone, int* bcount, int seg,
                         cudaStream_t st) {
  switch (c->n_det) {
    case 1: return run_lanes<1>(c, B, lnl, work, hist, pdone, bcount, seg, st);
    case 2: return run_lanes<2>(c, B, lnl, work, hist, pdone, bcount, seg, st);
    case 3: return run_lanes<3>(c, B, lnl, work, hist, pdone, bcount, seg, st);
    default: return run_lanes<4>(c, B, lnl, work, hist, pdone, bcount, seg, st);
  }
}

}  // namespace gwl
