// gwl_sched.cuh -- work distribution of the windowed bin loops.
//
// The bins of a segment are cut into windows of CH bins; proposal p is active
// in the windows w with w * CH < ncut_p.  Frequency cuts vary by orders of
// magnitude across a batch (f_ISCO ~ 1 / total mass), so the work of window w,
//   W_w = CH * (n_w - h_w / 2)   (n_w active proposals, h_w of them ending in w),
// falls steeply with w.  The prologue builds the histogram h of last windows;
// every CTA of the bin loop then starts in the window that holds its share of
// the total work (CTA b of G at the weighted quantile b / G), drains it, and
// sweeps on through the later windows, skipping those already drained.  Inside
// a window warps claim proposals in chunks sized so that a claim holds about
// one active proposal (B / n_w of them, 1 .. 32), or two when the window holds
// more than two active proposals per warp of the grid (the likelihood's bin
// loop takes pairs in its first claim only).
#pragma once

#include "gwl_device.cuh"

namespace gwl {

// Warp-level: add this warp's proposals to the histogram of last windows
// (one atomic per distinct window).  All 32 lanes must call it; ncut <= 0
// marks a lane without an in-band proposal.
__device__ __forceinline__ void hist_last_window(int ncut, int CH, int* __restrict__ hist) {
  const int L = ncut > 0 ? (ncut - 1) / CH : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, L);
  const int lane = threadIdx.x & 31;
  if (L >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[L], __popc(peers));
}

// Bucket lists of the lane-per-proposal bin loop (gwl_lanes.cu): proposal p
// with ncut > 0 goes to bucket K = (ncut - 1) / seg, the index of its last
// chunk of seg bins, at a slot taken with one atomic per distinct bucket in
// the warp: list[K * B + slot] = p.  The bin loop reads the buckets in
// descending K, so the proposals active in chunk c (those with K >= c) are a
// prefix of that order and neighbours in it have similar cuts.  All 32 lanes
// must call it; ncut <= 0 marks a lane without an in-band proposal.
struct Buckets {
  int* count;  // [ceil(M / seg)] proposals per bucket (cleared before the prologue); null: no buckets
  int* list;   // [ceil(M / seg)][B] proposal indices
  int seg;     // bins per chunk (a multiple of 32)
};

__device__ __forceinline__ void bucket_push(int ncut, int64_t p, const Buckets& bk, int64_t B) {
  const int K = ncut > 0 ? (ncut - 1) / bk.seg : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, K);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (K >= 0 && lane == leader) base = atomicAdd(&bk.count[K], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (K >= 0) bk.list[(int64_t)K * B + base + __popc(peers & ((1u << lane) - 1u))] = (int)p;
}

// CTA-level (256 threads, called by all): the window in [w_lo, nw) in which
// CTA b of G starts, and (*n_start) the proposals active in it.  Returns nw
// when no proposal is active in [w_lo, nw).  In units of CH / 2 bins, the
// cumulative work before relative window r is
//   C_r = sum_{L < r} h_L (2L + 1) + 2 r (N - P_r),   P_r = sum_{L < r} h_L,
// N the proposals ending in [w_lo, nw); CTA b starts in the r with
// C_r <= b C_R / G < C_{r+1}.  Every CTA computes the same prefix sums.
__device__ __forceinline__ int start_window(const int* __restrict__ hist, int w_lo, int nw, int b, int G,
                                            int* n_start) {
  __shared__ long long s_tot[8][2];
  __shared__ int s_res[2];
  const int R = nw - w_lo;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int k = (R + 255) / 256;
  const int r0 = min(t * k, R), r1 = min(r0 + k, R);
  long long cnt = 0, a2 = 0;
  for (int r = r0; r < r1; ++r) {
    const long long h = __ldcg(&hist[w_lo + r]);
    cnt += h;
    a2 += h * (2 * r + 1);
  }
  long long ic = cnt, ia = a2;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const long long yc = __shfl_up_sync(0xffffffffu, ic, off);
    const long long ya = __shfl_up_sync(0xffffffffu, ia, off);
    if (lane >= off) {
      ic += yc;
      ia += ya;
    }
  }
  if (t == 0) {
    s_res[0] = nw;
    s_res[1] = 0;
  }
  if (lane == 31) {
    s_tot[warp][0] = ic;
    s_tot[warp][1] = ia;
  }
  __syncthreads();
  long long P = ic - cnt, A = ia - a2, N = 0, T2 = 0;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    if (v < warp) {
      P += s_tot[v][0];
      A += s_tot[v][1];
    }
    N += s_tot[v][0];
    T2 += s_tot[v][1];
  }
  if (T2 > 0) {
    const long long q = (long long)b * T2 / G;
    for (int r = r0; r < r1; ++r) {
      const long long h = __ldcg(&hist[w_lo + r]);
      const long long C0 = A + 2LL * r * (N - P);
      const long long P1 = P + h, A1 = A + h * (2 * r + 1);
      const long long C1 = A1 + 2LL * (r + 1) * (N - P1);
      if (C0 <= q && q < C1) {  // exactly one thread of the CTA
        s_res[0] = w_lo + r;
        s_res[1] = (int)(N - P);
      }
      P = P1;
      A = A1;
    }
  }
  __syncthreads();
  *n_start = s_res[1];
  return s_res[0];
}

// Proposals per claim in a window with n_active active proposals of B: about
// one active proposal per claim, or (pair) two, half the atomics on the
// window's counter, when the window holds more than two active proposals per
// warp of the grid, so that small batches keep every warp busy.
__device__ __forceinline__ int claim_size(int64_t B, int n_active, bool pair = true) {
  if (n_active <= 0) return 32;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int per = pair && n_active >= 2 * warps ? 2 : 1;
  const int64_t c = per * B / n_active;
  return c < per ? per : (c > 32 ? 32 : (int)c);
}

// Warp-level: drain the proposals of one window from its counter, `chunk` per
// claim; f(p, ncut) runs (on the whole warp) for every proposal with ncut > j0.
// A claim taken earlier on the same counter (pre_chunk > 0: lane 0's pre, the
// value its atomic returned, pre_chunk proposals) is processed first; with
// only_pre the warp stops after it.
template <class F>
__device__ __forceinline__ void drain_window(int* ctr, int64_t B, int chunk, const PropCommon* __restrict__ pc,
                                             int j0, int lane, F&& f, int pre = 0, int pre_chunk = 0,
                                             bool only_pre = false) {
  while (true) {
    int base = 0, n = chunk;
    if (pre_chunk > 0) {
      base = pre;
      n = pre_chunk;
    } else if (lane == 0) {
      base = atomicAdd(ctr, chunk);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= B) break;
    int nc = 0;
    if (lane < n && base + lane < B) nc = pc[base + lane].ncut;
    unsigned act = __ballot_sync(0xffffffffu, nc > j0);
    while (act) {
      const int l = __ffs(act) - 1;
      act &= act - 1;
      f((int64_t)base + l, __shfl_sync(0xffffffffu, nc, l));
    }
    if (only_pre && pre_chunk > 0) break;
    pre_chunk = 0;
  }
}

}  // namespace gwl
