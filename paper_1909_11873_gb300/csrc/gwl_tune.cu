// gwl_tune.cu -- the autotuner of the bin-loop launch shape (gwl_autotune).
//
// The bin loops are tiled by a window of frequency bins staged in shared
// memory and a grid sized in CTAs per SM.
// Which shape is fastest depends on the segment length (bins), the detector
// count (row size) and the batch, so the library times the candidates on the
// caller's own batch and keeps the fastest.  Only public entry points are
// called; every launch goes through gwl_loglike / gwl_grad.
#include <string>
#include <algorithm>
#include <vector>

#include "gwl_internal.h"

namespace gwl {
int set_error(int code, const char* fmt, ...);
}

namespace {

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t init() {
    cudaError_t e = cudaEventCreate(&e0);
    return e == cudaSuccess ? cudaEventCreate(&e1) : e;
  }
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// Best time (ms per call) of two runs of `reps` back-to-back calls after one
// warm-up call; returns a GWL_* code.
template <class F>
int time_calls(Timer& t, cudaStream_t st, F call, double* ms_out) {
  const int reps = 3;
  int rc = call();
  if (rc) return rc;
  double best = 1e30;
  for (int r = 0; r < 2; ++r) {
    cudaError_t e = cudaEventRecord(t.e0, st);
    if (e != cudaSuccess) return gwl::set_error(GWL_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    for (int k = 0; k < reps; ++k)
      if ((rc = call())) return rc;
    if ((e = cudaEventRecord(t.e1, st)) != cudaSuccess || (e = cudaEventSynchronize(t.e1)) != cudaSuccess)
      return gwl::set_error(GWL_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, t.e0, t.e1)) != cudaSuccess)
      return gwl::set_error(GWL_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    if (ms / reps < best) best = ms / reps;
  }
  *ms_out = best;
  return GWL_OK;
}

}  // namespace

extern "C" int gwl_autotune(gwl_ctx* c, const double* theta_dev, int64_t B, int what, gwl_tuning* out,
                            void* stream) {
  if (!c) return gwl::set_error(GWL_ERR_ARG, "null context");
  if (B < 1 || !theta_dev) return gwl::set_error(GWL_ERR_ARG, "autotune needs a non-empty device batch");
  if (what < 1 || what > 3) return gwl::set_error(GWL_ERR_ARG, "bad autotune selector %d", what);
  cudaStream_t st = (cudaStream_t)stream;
  gwl_tuning saved;
  int rc = gwl_get_tuning(c, &saved);
  if (rc) return rc;
  saved.ms_loglike = saved.ms_grad = 0.0;

  // candidate windows for a row size (bytes): multiples of 64 bins that fit in
  // shared memory, at most the segment, partial sums within 2 GB
  auto candidates = [&](size_t row) {
    std::vector<int> ws;
    for (int w = 128; w <= 1536; w += 64) {
      if ((size_t)w * row > gwl::kWindowSmemMax) break;
      if (w >= c->M) {  // windows at least as long as the segment are all the same shape
        ws.push_back(w);
        break;
      }
      const int64_t nw = (c->M + w - 1) / w;
      if (B * nw * gwl::sums_per_det(c) * c->n_det * (int64_t)sizeof(double) > ((int64_t)2 << 30)) continue;
      ws.push_back(w);
    }
    return ws;
  };
  const bool mixed = c->opt.precision == GWL_MIXED;
  if ((what & GWL_TUNE_GRAD) && c->opt.precision == GWL_MIXED_F64PHASE)
    return gwl::set_error(GWL_ERR_ARG, "autotune: gwl_grad is not available in GWL_MIXED_F64PHASE");
  const std::vector<int> windows = candidates(gwl::lnl_row_bytes(c));
  // gradient rows carry the calibration rows too, and the moment pass stages one window of them
  std::vector<int> gwindows =
      candidates(mixed ? sizeof(float) * (c->row_floats + (c->n_cal_nodes ? c->row_cal_f : 0))
                       : sizeof(double) * (c->row_doubles + (c->n_cal_nodes ? c->row_cal_d : 0)));
  if (c->n_cal_nodes)
    gwindows.erase(std::remove_if(gwindows.begin(), gwindows.end(),
                                  [&](int w) { return gwl::calgrad_smem(c, w) > gwl::kCalGradSmemMax; }),
                   gwindows.end());
  if (windows.empty() || gwindows.empty()) return gwl::set_error(GWL_ERR_ARG, "autotune: no window fits");

  double* d_out = nullptr;
  const int64_t n_out = B * (1 + c->seg.stride);
  cudaError_t e = cudaMalloc(&d_out, sizeof(double) * (size_t)n_out);
  if (e != cudaSuccess) return gwl::set_error(GWL_ERR_NOMEM, "autotune: %s", cudaGetErrorString(e));
  Timer t;
  if ((e = t.init()) != cudaSuccess) {
    cudaFree(d_out);
    return gwl::set_error(GWL_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  }

  gwl_tuning best = saved;
  double best_l = 1e30, best_g = 1e30;
  int tried = 0;
  if (what & GWL_TUNE_LOGLIKE) {
    // (layout, lane chunk): the warp layout, then the lane layout with 32- and 64-bin chunks
    const int variants[3][2] = {{GWL_BINS_WARP, 64}, {GWL_BINS_LANE, 32}, {GWL_BINS_LANE, 64}};
    for (const auto& var : variants) {
      if (rc) break;
      for (int ctas = 1; ctas <= 4 && !rc; ++ctas)
        for (int w : windows) {
          gwl_tuning s = saved;
          s.window = w;
          s.ctas_per_sm = ctas;
          s.bin_kernel = var[0];
          s.lane_chunk = var[1];
          if ((rc = gwl_set_tuning(c, &s))) break;
          // the lane layout where it is available, with this chunk (not its whole-window fallback)
          if (var[0] == GWL_BINS_LANE) {
            const int seg = gwl::lanes_seg(c, B);
            if (seg == 0 || (seg != var[1] && var[1] != 64)) continue;
          }
          double ms = 0.0;
          rc = time_calls(t, st, [&] { return gwl_loglike(c, theta_dev, B, d_out, stream); }, &ms);
          if (rc) break;
          ++tried;
          if (ms < best_l) {
            best_l = ms;
            best.window = w;
            best.ctas_per_sm = ctas;
            best.bin_kernel = var[0];
            best.lane_chunk = var[1];
          }
        }
    }
  }
  if (!rc && (what & GWL_TUNE_GRAD)) {
    for (int w : gwindows) {
      gwl_tuning s = saved;
      s.grad_window = w;
      if ((rc = gwl_set_tuning(c, &s))) break;
      double ms = 0.0;
      rc = time_calls(t, st, [&] { return gwl_grad(c, theta_dev, B, d_out, d_out + B, stream); }, &ms);
      if (rc) break;
      ++tried;
      if (ms < best_g) {
        best_g = ms;
        best.grad_window = w;
      }
    }
  }
  if (!rc) rc = gwl_sync(c);  // a bounded wait that ran out during tuning fails the tuning
  cudaFree(d_out);
  if (rc) {
    const std::string msg = gwl_last_error();
    gwl_set_tuning(c, &saved);
    return gwl::set_error(rc, "%s", msg.c_str());
  }
  if ((rc = gwl_set_tuning(c, &best))) return rc;
  if (what & GWL_TUNE_LOGLIKE) c->tuned_ms[0] = best_l;
  if (what & GWL_TUNE_GRAD) c->tuned_ms[1] = best_g;
  c->tuned_n = tried;
  return out ? gwl_get_tuning(c, out) : GWL_OK;
}
