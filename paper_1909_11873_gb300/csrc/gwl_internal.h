// gwl_internal.h -- host-side context and kernel launch wrappers (not part of the ABI).
#pragma once

#include <cstdint>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/gwl.h"
#include "gwl_device.cuh"

struct gwl_ctx {
  int device = 0;
  int num_sms = 0;
  int64_t M = 0;
  int n_det = 0;
  double f0 = 0.0, df = 0.0;
  gwl_options opt{};
  gwl::SegInfo seg{};  // device pointers inside

  // device tables (owned)
  double* d_freqs = nullptr;   // [M]
  double* d_geom = nullptr;    // [n_det][9]
  double* d_H = nullptr;       // [n_det][M]
  float* d_tab_mixed = nullptr;  // [M][mixed_row_floats]
  float* d_tab_delta = nullptr;  // [M][delta_row_floats]: basis deltas from the block anchor, G_d
  float* d_anchor = nullptr;     // [ceil(M / kAnchor)][kAnchorRowFloats]
  int row_delta = 0;
  double* d_tab_f64 = nullptr;   // [M][f64_row_doubles]
  int row_floats = 0, row_doubles = 0;

  // calibration model (gwl_set_calibration); n_cal_nodes == 0: off
  int n_cal_nodes = 0;
  int64_t cal_gen = 0;  // bumped by every gwl_set_calibration that changes the model
  float* d_cal_f = nullptr;      // [M][cal_row_floats]: spline weights, interval, dH_d
  double* d_cal_d = nullptr;     // [M][cal_row_doubles]
  float* d_calQ_f = nullptr;     // [n_nodes][n_nodes]: m = Q y (natural-spline curvatures)
  double* d_calQ_d = nullptr;
  int row_cal_f = 0, row_cal_d = 0;
  double cal_sigma[2] = {0.1, 0.1};  // prior widths of the amplitude and phase corrections (ns_replace, ns_run)

  // device scratch (owned, grown on demand)
  gwl::PropMixed* d_pm = nullptr;
  gwl::PropF64* d_pf = nullptr;
  gwl::PropCommon* d_pc = nullptr;
  int64_t prop_cap = 0;
  double* d_partials = nullptr;  // [B][n_windows][2 n_det]
  int64_t partials_cap = 0;      // in doubles
  double* d_walk = nullptr;      // ns_replace proposals: u' [n][D], theta' [n][D], lnL' [n]
  int64_t walk_cap = 0;          // in doubles
  void* d_wscal = nullptr;       // walk scalars (L*, scale, worst, counter)
  double* d_gmc = nullptr;       // Galilean walk scratch (velocity, reflected points, gradient)
  int64_t gmc_cap = 0;           // in doubles
  int walk_kind = GWL_WALK_RANDOM;
  double gmc_persistence = GWL_GALILEAN_PERSISTENCE;  // velocity kept per Galilean step
  double* d_io = nullptr;        // staging for the host-buffer entry points
  int64_t io_cap = 0;            // in doubles
  void* d_pgrad = nullptr;       // per-proposal tangents of the gradient prologue
  int64_t pgrad_cap = 0;         // in bytes
  void* d_gpartials = nullptr;   // per-window sums of the gradient bin loop
  int64_t gpartials_cap = 0;     // in bytes
  int* d_blist = nullptr;        // lane bin loop: bucket lists of proposals [chunks][B]
  int64_t blist_cap = 0;         // in ints
  int* d_work = nullptr;         // [0] largest cut of the batch, [1 + w] proposal counter of window w
  int64_t work_cap = 0;          // in ints
  int* d_status = nullptr;       // [0] latched status bits
  unsigned long long* d_ffc = nullptr;  // diagnostic: blocks of the mixed bin loop with float-float deltas
  bool count_ff = false;                // count them (gwl_test_ffdelta_blocks)

  // tuning
  // tuning (gwl_set_tuning / gwl_autotune); the windows are set by gwl_create
  int window = 0;       // likelihood bin loop: bins per staged window
  int grad_window = 0;  // gradient bin loop: bins per staged window
  int ctas_per_sm = 3;  // likelihood bin loop grid: CTAs per SM
  int bin_kernel = GWL_BINS_AUTO;  // likelihood bin loop layout
  int lane_chunk = 64;             // lane bin loop: bins per chunk
  double tuned_ms[2] = {0.0, 0.0};  // autotuner: best gwl_loglike / gwl_grad time (ms)
  int tuned_n = 0;                  // autotuner: shapes timed

  int64_t launches = 0;
  int64_t bytes = 0;
  cudaStream_t last_stream = nullptr;

  // optional per-kernel timing with CUDA events recorded on the launch stream
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending[GWL_KERNEL_KINDS];
  std::vector<cudaEvent_t> event_pool;
  double prof_ms[GWL_KERNEL_KINDS] = {0};
  int64_t prof_n[GWL_KERNEL_KINDS] = {0};
};

namespace gwl {
// Largest staged window of a bin loop (bytes of dynamic shared memory), so
// that with the kernels' static shared memory a CTA stays within 227 KB.
constexpr size_t kWindowSmemMax = 192 * 1024;
// Doubles per row of theta: the sampled coordinates, then the calibration parameters.
inline int64_t theta_stride(const gwl_ctx* c) { return c->seg.stride; }
// Bytes of shared memory per bin of the likelihood bin loop's window.
inline size_t lnl_row_bytes(const gwl_ctx* c) {
  const bool mixed = c->opt.precision == GWL_MIXED;
  size_t b = mixed ? sizeof(float) * (size_t)c->row_delta : sizeof(double) * (size_t)c->row_doubles;
  if (c->n_cal_nodes) b += mixed ? sizeof(float) * (size_t)c->row_cal_f : sizeof(double) * (size_t)c->row_cal_d;
  return b;
}
// Per-detector sums a bin loop keeps per (proposal, window): U, V (and the
// calibrated <h|h> correction X).
inline int sums_per_det(const gwl_ctx* c) { return c->n_cal_nodes ? 3 : 2; }

// Raises the dynamic shared-memory limit of `kernel` on `device` (the current
// device) to at least `bytes`.  The limit is a per-device attribute: the
// largest value set so far is remembered per (kernel, device), under a lock,
// so each device gets its own call.
cudaError_t raise_smem_limit(const void* kernel, int device, size_t bytes);

// Records a start event now and a stop event when it goes out of scope, on
// the launch stream, if the context has profiling enabled.
struct ProfScope {
  gwl_ctx* c;
  int kind;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ProfScope(gwl_ctx* c_, int kind_, cudaStream_t st_);
  ~ProfScope();
};
}  // namespace gwl

namespace gwl {

// a1: tables
cudaError_t launch_build_tables(gwl_ctx* c, const double* d_strain, const double* d_psd, cudaStream_t st);
cudaError_t launch_scale_tables(gwl_ctx* c, double sg, cudaStream_t st);
cudaError_t launch_cal_tables(gwl_ctx* c, const double* d_xnode, cudaStream_t st);

// a2-a6: batched log-likelihood
cudaError_t launch_loglike(gwl_ctx* c, const double* theta, int64_t B, double* lnl, cudaStream_t st);
// the same after a kernel that cleared the work counters (work_needed(c, B)
// ints of d_work) and wrote theta: no clearing kernel
cudaError_t launch_loglike_cleared(gwl_ctx* c, const double* theta, int64_t B, double* lnl, cudaStream_t st);
int64_t work_needed(const gwl_ctx* c, int64_t B);
// the lane-per-proposal bin loop (gwl_lanes.cu): chunk size (0: not used), scratch sizes, launch
int lanes_seg(const gwl_ctx* c, int64_t B);
int64_t lanes_list_ints(const gwl_ctx* c, int64_t B);
int64_t lanes_slot_floats(const gwl_ctx* c, int64_t B);
cudaError_t launch_lanes(gwl_ctx* c, int64_t B, double* lnl, int* work, int* hist, int* pdone, int* bcount, int seg,
                         cudaStream_t st);

// Largest dynamic shared memory of the calibrated gradient's second bin loop
// (the rows plus eight warps' scratch) that a window may need.
constexpr size_t kCalGradSmemMax = 220 * 1024;
size_t calgrad_smem(const gwl_ctx* c, int CH);

// a8: log-likelihood and gradient
cudaError_t launch_grad(gwl_ctx* c, const double* theta, int64_t B, double* lnl, double* grad, cudaStream_t st);
int64_t grad_partials_bytes(const gwl_ctx* c, int64_t B);
int64_t prop_grad_bytes(const gwl_ctx* c);

// a7 / a9: random walks and nested sampling
cudaError_t launch_walk(gwl_ctx* c, const double* live_u, const double* live_lnl, int64_t K, const void* scalars,
                        uint64_t seed, int64_t n_chains, int walk_len, const double* chol, double* out_u,
                        double* out_lnl, int32_t* out_nacc, int32_t* out_start, double* pu, double* pth,
                        double* plnl, cudaStream_t st);
size_t walk_scalars_bytes();
size_t gmc_scratch_doubles(int64_t n_chains, int D);
void set_walk_scalars(void* host_buf, double lstar, double scale, int64_t worst, uint64_t counter);
int ns_run_impl(gwl_ctx* c, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                int64_t max_rounds, double scale0, int64_t max_dead, double* dead_lnl, double* dead_logwt,
                double* dead_u, double* res, cudaStream_t st, int use_graph, const double* resume,
                double* checkpoint);
int64_t state_doubles(int64_t K, int64_t D, int64_t max_dead);
int state_check(const double* in, int64_t K, int64_t D);

// many events in one batched evaluation
struct Multi;
Multi* multi_new(gwl_ctx* const* ctxs, int E);
void multi_delete(Multi* m);
cudaError_t multi_prepare(Multi* m, int64_t n_per);
cudaError_t multi_loglike(Multi* m, const double* theta, int64_t n_per, double* lnl, cudaStream_t st);
int64_t multi_launches(const Multi* m);
bool multi_consistent(const Multi* m);
int multi_ns_run(Multi* m, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                 int64_t max_rounds, double scale0, double* res /* [E][11] */, cudaStream_t caller,
                 const double* resume = nullptr, double* checkpoint = nullptr);
int64_t multi_state_doubles(int E, int64_t K, int64_t D);
int multi_state_check(const double* in, int E, int64_t K, int64_t D);
int multi_dim(const Multi* m);

// gwl_loglike_static's fixed array: look its device address up on `dev` (set-up, from gwl_create)
cudaError_t static_scratch_setup(int dev);

// device-path template, for diagnostics and injections
cudaError_t launch_waveform(gwl_ctx* c, const double* theta, int64_t B, double* h, cudaStream_t st);

}  // namespace gwl
