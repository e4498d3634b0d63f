// gwl_api.cu -- the C ABI (include/gwl.h): argument checks, device memory,
// error reporting.  All arithmetic of the likelihood runs in the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gwl_internal.h"

namespace gwl {
int64_t partials_needed(const gwl_ctx* c, int64_t B);
int64_t work_needed(const gwl_ctx* c, int64_t B);
}  // namespace gwl

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? GWL_ERR_NOMEM : GWL_ERR_CUDA, "%s: %s", where,
              cudaGetErrorString(e));
}

template <class T>
cudaError_t dev_alloc(gwl_ctx* c, T** p, int64_t n) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)(n > 0 ? n : 1));
  if (e == cudaSuccess) c->bytes += (int64_t)sizeof(T) * (n > 0 ? n : 1);
  return e;
}

template <class T>
void dev_free(gwl_ctx* c, T*& p, int64_t n) {
  if (p) {
    cudaFree(p);
    c->bytes -= (int64_t)sizeof(T) * (n > 0 ? n : 1);
  }
  p = nullptr;
}

// Grow the per-proposal and partial-sum scratch to hold a batch of B.
int ensure_scratch(gwl_ctx* c, int64_t B) {
  cudaError_t e;

  if (B > c->prop_cap) {
    int64_t cap = B > 2 * c->prop_cap ? B : 2 * c->prop_cap;
    dev_free(c, c->d_pm, c->prop_cap);
    dev_free(c, c->d_pf, c->prop_cap);
    dev_free(c, c->d_pc, c->prop_cap);
    c->prop_cap = 0;
    if ((e = dev_alloc(c, &c->d_pm, cap)) != cudaSuccess) return cuda_fail(e, "scratch");
    if ((e = dev_alloc(c, &c->d_pf, cap)) != cudaSuccess) return cuda_fail(e, "scratch");
    if ((e = dev_alloc(c, &c->d_pc, cap)) != cudaSuccess) return cuda_fail(e, "scratch");
    c->prop_cap = cap;
  }
  const int64_t wneed = gwl::work_needed(c, B);
  if (wneed > c->work_cap) {
    dev_free(c, c->d_work, c->work_cap);
    c->work_cap = 0;
    if ((e = dev_alloc(c, &c->d_work, wneed)) != cudaSuccess) return cuda_fail(e, "scratch");
    c->work_cap = wneed;
  }
  const int64_t lneed = gwl::lanes_list_ints(c, B);
  if (lneed > c->blist_cap) {
    int64_t cap = lneed > 2 * c->blist_cap ? lneed : 2 * c->blist_cap;
    dev_free(c, c->d_blist, c->blist_cap);
    c->blist_cap = 0;
    if ((e = dev_alloc(c, &c->d_blist, cap)) != cudaSuccess) return cuda_fail(e, "scratch");
    c->blist_cap = cap;
  }
  const int64_t need = gwl::partials_needed(c, B);
  if (need > c->partials_cap) {
    int64_t cap = need > 2 * c->partials_cap ? need : 2 * c->partials_cap;
    dev_free(c, c->d_partials, c->partials_cap);
    c->partials_cap = 0;
    if ((e = dev_alloc(c, &c->d_partials, cap)) != cudaSuccess) return cuda_fail(e, "scratch");
    c->partials_cap = cap;
  }
  return GWL_OK;
}

int ensure_bytes(gwl_ctx* c, void** p, int64_t* cap, int64_t need) {
  if (need <= *cap) return GWL_OK;
  const int64_t n = need > 2 * *cap ? need : 2 * *cap;
  if (*p) {
    cudaFree(*p);
    c->bytes -= *cap;
  }
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(p, (size_t)n);
  if (e != cudaSuccess) return cuda_fail(e, "scratch");
  c->bytes += n;
  *cap = n;
  return GWL_OK;
}

int ensure_io(gwl_ctx* c, int64_t n) {
  if (n <= c->io_cap) return GWL_OK;
  dev_free(c, c->d_io, c->io_cap);
  c->io_cap = 0;
  cudaError_t e = dev_alloc(c, &c->d_io, n);
  if (e != cudaSuccess) return cuda_fail(e, "io staging");
  c->io_cap = n;
  return GWL_OK;
}

// m = Q y: the second derivatives at the nodes of the natural cubic spline
// through (x_k, y_k), as a fixed matrix of the node layout.  Interior rows
// k = 1 .. n-2 of  h_{k-1} m_{k-1} + 2 (h_{k-1} + h_k) m_k + h_k m_{k+1}
// = 6 [(y_{k+1} - y_k)/h_k - (y_k - y_{k-1})/h_{k-1}], m_0 = m_{n-1} = 0, are
// solved for all n right-hand sides at once by Gauss-Jordan elimination.
std::vector<double> natural_spline_matrix(int n, const double* x) {
  std::vector<double> Q((size_t)n * n, 0.0);
  const int ni = n - 2;
  if (ni <= 0) return Q;
  std::vector<double> A((size_t)ni * ni, 0.0), R((size_t)ni * n, 0.0);
  for (int i = 0; i < ni; ++i) {
    const int k = i + 1;
    const double hl = x[k] - x[k - 1], hr = x[k + 1] - x[k];
    if (i > 0) A[(size_t)i * ni + i - 1] = hl;
    A[(size_t)i * ni + i] = 2.0 * (hl + hr);
    if (i + 1 < ni) A[(size_t)i * ni + i + 1] = hr;
    R[(size_t)i * n + k - 1] += 6.0 / hl;
    R[(size_t)i * n + k] -= 6.0 / hl + 6.0 / hr;
    R[(size_t)i * n + k + 1] += 6.0 / hr;
  }
  for (int col = 0; col < ni; ++col) {
    int piv = col;
    for (int r = col + 1; r < ni; ++r)
      if (std::fabs(A[(size_t)r * ni + col]) > std::fabs(A[(size_t)piv * ni + col])) piv = r;
    if (piv != col) {
      for (int c2 = 0; c2 < ni; ++c2) std::swap(A[(size_t)col * ni + c2], A[(size_t)piv * ni + c2]);
      for (int c2 = 0; c2 < n; ++c2) std::swap(R[(size_t)col * n + c2], R[(size_t)piv * n + c2]);
    }
    const double inv = 1.0 / A[(size_t)col * ni + col];
    for (int c2 = 0; c2 < ni; ++c2) A[(size_t)col * ni + c2] *= inv;
    for (int c2 = 0; c2 < n; ++c2) R[(size_t)col * n + c2] *= inv;
    for (int r = 0; r < ni; ++r) {
      if (r == col) continue;
      const double f = A[(size_t)r * ni + col];
      if (f == 0.0) continue;
      for (int c2 = 0; c2 < ni; ++c2) A[(size_t)r * ni + c2] -= f * A[(size_t)col * ni + c2];
      for (int c2 = 0; c2 < n; ++c2) R[(size_t)r * n + c2] -= f * R[(size_t)col * n + c2];
    }
  }
  for (int i = 0; i < ni; ++i)
    for (int c2 = 0; c2 < n; ++c2) Q[(size_t)(i + 1) * n + c2] = R[(size_t)i * n + c2];
  return Q;
}

// The compute entry points that do not model calibration refuse a calibrated context.
int no_calibration(const gwl_ctx* c, const char* what) {
  if (c->n_cal_nodes) return fail(GWL_ERR_ARG, "%s is not available with the calibration model", what);
  return GWL_OK;
}
// The FP64-phase mixed mode is a likelihood-only comparison arm.
int likelihood_only(const gwl_ctx* c, const char* what) {
  if (c->opt.precision == GWL_MIXED_F64PHASE)
    return fail(GWL_ERR_ARG, "%s is not available in GWL_MIXED_F64PHASE (likelihood only)", what);
  return GWL_OK;
}
// The Galilean walk needs gwl_grad.
int walk_supported(const gwl_ctx* c, const char* what) {
  if (c->walk_kind == GWL_WALK_GALILEAN && c->opt.precision == GWL_MIXED_F64PHASE)
    return fail(GWL_ERR_ARG, "%s: the Galilean walk is not available in GWL_MIXED_F64PHASE", what);
  return GWL_OK;
}

// The device address of a page-locked host buffer (device-accessible under
// unified addressing), or null for pageable memory.
template <class T>
T* mapped_host(T* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return static_cast<T*>(a.devicePointer);
}

int check_ctx(const gwl_ctx* c) {
  if (!c) return fail(GWL_ERR_ARG, "null context");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
    return fail(GWL_ERR_ARG, "context belongs to device %d but device %d is current", c->device, dev);
  return GWL_OK;
}

}  // namespace

namespace gwl {
int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
}  // namespace gwl

extern "C" {

const char* gwl_last_error(void) { return g_err.c_str(); }

int gwl_create(const double* freqs, int64_t n_bins, const double* strain, const double* psd,
               const gwl_detector* dets, int n_det, const gwl_options* opt, gwl_ctx** out) {
  if (!out) return fail(GWL_ERR_ARG, "out is null");
  *out = nullptr;
  if (!freqs || !strain || !psd || !dets || !opt) return fail(GWL_ERR_ARG, "null input pointer");
  if (n_bins < 2 || n_bins > (int64_t)1 << 30) return fail(GWL_ERR_ARG, "n_bins=%lld out of range", (long long)n_bins);
  if (n_det < 1 || n_det > GWL_MAX_DET) return fail(GWL_ERR_ARG, "n_det=%d out of range [1,%d]", n_det, GWL_MAX_DET);
  if (opt->precision != GWL_FP64 && opt->precision != GWL_MIXED && opt->precision != GWL_MIXED_F64PHASE)
    return fail(GWL_ERR_ARG, "bad precision");
  if (opt->fcut_mode != GWL_FCUT_ISCO && opt->fcut_mode != GWL_FCUT_BAND) return fail(GWL_ERR_ARG, "bad fcut_mode");
  if (opt->n_dim < 1 || opt->n_dim > GWL_N_PARAM) return fail(GWL_ERR_ARG, "n_dim=%d out of range", opt->n_dim);
  bool used[GWL_N_PARAM] = {false};
  for (int i = 0; i < opt->n_dim; ++i) {
    const int k = opt->param_map[i];
    if (k < 0 || k >= GWL_N_PARAM || used[k]) return fail(GWL_ERR_ARG, "bad param_map[%d]=%d", i, k);
    used[k] = true;
    if (opt->prior_kind[i] < 0 || opt->prior_kind[i] > 3) return fail(GWL_ERR_ARG, "bad prior_kind[%d]", i);
  }
  const double f0 = freqs[0];
  const double df = (freqs[n_bins - 1] - freqs[0]) / (double)(n_bins - 1);
  if (!(f0 > 0.0) || !(df > 0.0)) return fail(GWL_ERR_ARG, "frequencies must be positive and ascending");
  for (int64_t j = 0; j < n_bins; ++j) {
    if (std::fabs(freqs[j] - (f0 + (double)j * df)) > 1e-9 * df)
      return fail(GWL_ERR_ARG, "frequencies are not uniformly spaced at bin %lld", (long long)j);
  }
  for (int64_t i = 0; i < (int64_t)n_det * n_bins; ++i)
    if (!(psd[i] > 0.0) || !std::isfinite(psd[i])) return fail(GWL_ERR_ARG, "psd[%lld] not positive", (long long)i);
  for (int64_t i = 0; i < 2 * (int64_t)n_det * n_bins; ++i)
    if (!std::isfinite(strain[i])) return fail(GWL_ERR_ARG, "strain[%lld] not finite", (long long)i);

  gwl_ctx* c = new (std::nothrow) gwl_ctx();
  if (!c) return fail(GWL_ERR_NOMEM, "host allocation failed");
  int rc = GWL_OK;
  double* d_strain = nullptr;
  double* d_psd = nullptr;
  cudaError_t e;
  do {
    if ((e = cudaGetDevice(&c->device)) != cudaSuccess) { rc = cuda_fail(e, "cudaGetDevice"); break; }
    if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) {
      rc = cuda_fail(e, "device attribute");
      break;
    }
    // the fixed array of gwl_loglike_static: its address on this device, looked up afresh
    if ((e = gwl::static_scratch_setup(c->device)) != cudaSuccess) { rc = cuda_fail(e, "static scratch"); break; }
    c->M = n_bins;
    c->n_det = n_det;
    c->f0 = f0;
    c->df = df;
    c->opt = *opt;
    c->row_floats = gwl::mixed_row_floats(n_det);
    c->row_delta = gwl::delta_row_floats(n_det);
    c->row_doubles = gwl::f64_row_doubles(n_det);
    c->window = c->grad_window = opt->precision == GWL_MIXED ? 640 : 384;
    if ((e = dev_alloc(c, &c->d_freqs, n_bins)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = dev_alloc(c, &c->d_geom, 9 * n_det)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = dev_alloc(c, &c->d_H, (int64_t)n_det * n_bins)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = dev_alloc(c, &c->d_tab_mixed, n_bins * c->row_floats)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = dev_alloc(c, &c->d_tab_delta, n_bins * c->row_delta)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = dev_alloc(c, &c->d_anchor, (n_bins + gwl::kAnchor - 1) / gwl::kAnchor * gwl::kAnchorRowFloats)) !=
        cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = dev_alloc(c, &c->d_tab_f64, n_bins * c->row_doubles)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = dev_alloc(c, &c->d_status, 4)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = cudaMalloc(&c->d_wscal, 64)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = cudaMalloc(&d_strain, sizeof(double) * 2 * n_det * n_bins)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    if ((e = cudaMalloc(&d_psd, sizeof(double) * n_det * n_bins)) != cudaSuccess) { rc = cuda_fail(e, "alloc"); break; }
    double geom[9 * GWL_MAX_DET];
    for (int d = 0; d < n_det; ++d)
      for (int k = 0; k < 3; ++k) {
        geom[9 * d + k] = dets[d].vertex[k];
        geom[9 * d + 3 + k] = dets[d].xarm[k];
        geom[9 * d + 6 + k] = dets[d].yarm[k];
      }
    if ((e = cudaMemcpy(c->d_freqs, freqs, sizeof(double) * n_bins, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->d_geom, geom, sizeof(double) * 9 * n_det, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d_strain, strain, sizeof(double) * 2 * n_det * n_bins, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d_psd, psd, sizeof(double) * n_det * n_bins, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(c->d_status, 0, 4 * sizeof(int))) != cudaSuccess) {
      rc = cuda_fail(e, "copy inputs");
      break;
    }
    if ((e = gwl::launch_build_tables(c, d_strain, d_psd, 0)) != cudaSuccess) { rc = cuda_fail(e, "build tables"); break; }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) { rc = cuda_fail(e, "build tables"); break; }
    // normalisation: the largest whole-band <h|h> weight H_d[M-1] -> O(1)
    double hmax = 0.0;
    for (int d = 0; d < n_det; ++d) {
      double hd = 0.0;
      if ((e = cudaMemcpy(&hd, c->d_H + (int64_t)d * n_bins + n_bins - 1, sizeof(double), cudaMemcpyDeviceToHost)) !=
          cudaSuccess)
        break;
      hmax = hd > hmax ? hd : hmax;
    }
    if (e != cudaSuccess) { rc = cuda_fail(e, "normalise tables"); break; }
    const double scale = hmax > 0.0 && std::isfinite(hmax) ? std::ldexp(1.0, (int)std::lround(0.5 * std::log2(hmax))) : 1.0;
    if ((e = gwl::launch_scale_tables(c, 1.0 / scale, 0)) != cudaSuccess) { rc = cuda_fail(e, "normalise tables"); break; }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) { rc = cuda_fail(e, "normalise tables"); break; }
    c->seg.amp_scale = scale;
    gwl::SegInfo& s = c->seg;
    gwl::split_f64(gwl::kAmpConst * gwl::kC / gwl::kMpc * scale, s.amp_c_ff.hi, s.amp_c_ff.lo);
    for (int d = 0; d < GWL_MAX_DET; ++d) {
      for (int k = 0; k < 9; ++k) gwl::split_f64(d < n_det ? geom[9 * d + k] : 0.0, s.geom_ff[d][k].hi, s.geom_ff[d][k].lo);
      for (int k = 0; k < 3; ++k)
        gwl::split_f64(d < n_det ? geom[9 * d + k] / gwl::kC : 0.0, s.vtx_c_ff[d][k].hi, s.vtx_c_ff[d][k].lo);
    }
    s.freqs = c->d_freqs;
    s.H = c->d_H;
    s.geom = c->d_geom;
    s.M = n_bins;
    s.n_det = n_det;
    s.fcut_mode = opt->fcut_mode;
    s.f0 = f0;
    s.df = df;
    s.gmst = opt->gmst;
    s.t_ref = opt->t_ref;
    s.n_dim = opt->n_dim;
    s.stride = opt->n_dim;
    s.inv_df = 1.0 / df;
    for (int k = 0; k < GWL_N_PARAM; ++k) {
      s.fixed[k] = opt->fixed_theta[k];
      s.param_map[k] = k < opt->n_dim ? opt->param_map[k] : 0;
      s.param_pos[k] = -1;
    }
    for (int i = 0; i < opt->n_dim; ++i) s.param_pos[opt->param_map[i]] = i;
  } while (false);
  if (d_strain) cudaFree(d_strain);
  if (d_psd) cudaFree(d_psd);
  if (rc != GWL_OK) {
    gwl_destroy(c);
    return rc;
  }
  *out = c;
  return GWL_OK;
}

int gwl_loglike(gwl_ctx* c, const double* theta_dev, int64_t B, double* lnl_dev, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (B < 0) return fail(GWL_ERR_ARG, "B < 0");
  if (B == 0) return GWL_OK;
  if (!theta_dev || !lnl_dev) return fail(GWL_ERR_ARG, "null device pointer");
  if ((rc = ensure_scratch(c, B))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  cudaError_t e = gwl::launch_loglike(c, theta_dev, B, lnl_dev, st);
  if (e != cudaSuccess) return cuda_fail(e, "gwl_loglike");
  return GWL_OK;
}

int gwl_loglike_host(gwl_ctx* c, const double* theta_host, int64_t B, double* lnl_host, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (B < 0) return fail(GWL_ERR_ARG, "B < 0");
  if (B == 0) return GWL_OK;
  if (!theta_host || !lnl_host) return fail(GWL_ERR_ARG, "null host pointer");
  const int64_t nt = B * gwl::theta_stride(c);
  if ((rc = ensure_io(c, nt + B))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // page-locked buffers are read and written in place by the kernels; pageable ones are staged
  const double* th_dev = mapped_host(theta_host);
  double* l_dev = mapped_host(lnl_host);
  cudaError_t e = cudaSuccess;
  if (!th_dev) {
    th_dev = c->d_io;
    e = cudaMemcpyAsync(c->d_io, theta_host, sizeof(double) * nt, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy theta");
  }
  const bool stage_out = l_dev == nullptr;
  if (stage_out) l_dev = c->d_io + nt;
  if ((rc = gwl_loglike(c, th_dev, B, l_dev, stream))) return rc;
  if (stage_out) {
    e = cudaMemcpyAsync(lnl_host, l_dev, sizeof(double) * B, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy lnL");
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "synchronise");
  return GWL_OK;
}

int gwl_waveform(gwl_ctx* c, const double* theta_dev, int64_t B, double* h_dev, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (B < 0 || B > 65535) return fail(GWL_ERR_ARG, "B=%lld out of range [0, 65535]", (long long)B);
  if (B == 0) return GWL_OK;
  if (!theta_dev || !h_dev) return fail(GWL_ERR_ARG, "null device pointer");
  if ((rc = ensure_scratch(c, B))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  cudaError_t e = gwl::launch_waveform(c, theta_dev, B, h_dev, st);
  if (e != cudaSuccess) return cuda_fail(e, "gwl_waveform");
  return GWL_OK;
}

int gwl_grad(gwl_ctx* c, const double* theta_dev, int64_t B, double* lnl_dev, double* grad_dev, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (B < 0) return fail(GWL_ERR_ARG, "B < 0");
  if (B == 0) return GWL_OK;
  if (!theta_dev || !lnl_dev || !grad_dev) return fail(GWL_ERR_ARG, "null device pointer");
  if ((rc = likelihood_only(c, "gwl_grad"))) return rc;
  if ((rc = ensure_scratch(c, B))) return rc;
  if ((rc = ensure_bytes(c, &c->d_pgrad, &c->pgrad_cap, gwl::prop_grad_bytes(c) * B))) return rc;
  if ((rc = ensure_bytes(c, &c->d_gpartials, &c->gpartials_cap, gwl::grad_partials_bytes(c, B)))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  cudaError_t e = gwl::launch_grad(c, theta_dev, B, lnl_dev, grad_dev, st);
  if (e != cudaSuccess) return cuda_fail(e, "gwl_grad");
  return GWL_OK;
}

int ns_replace(gwl_ctx* c, const double* live_u, const double* live_lnl, int64_t K, int64_t worst, double lnl_star,
               uint64_t seed, uint64_t counter, int64_t n_chains, int walk_len, double scale, const double* chol,
               double* out_u, double* out_lnl, int32_t* out_nacc, int32_t* out_start, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (K < 2) return fail(GWL_ERR_ARG, "K = %lld < 2", (long long)K);
  if (worst < 0 || worst >= K) return fail(GWL_ERR_ARG, "worst = %lld outside [0, K)", (long long)worst);
  if (n_chains < 0 || n_chains > ((int64_t)1 << 31) - 1) return fail(GWL_ERR_ARG, "n_chains out of range");
  if (walk_len < 0) return fail(GWL_ERR_ARG, "walk_len < 0");
  if (!(scale > 0.0) || !std::isfinite(scale)) return fail(GWL_ERR_ARG, "scale must be positive");
  if ((rc = walk_supported(c, "ns_replace"))) return rc;
  if (n_chains == 0) return GWL_OK;
  if (!live_u || !live_lnl || !chol || !out_u || !out_lnl || !out_nacc) return fail(GWL_ERR_ARG, "null device pointer");
  const int D = (int)gwl::theta_stride(c);
  if ((rc = ensure_scratch(c, n_chains))) return rc;
  if ((rc = ensure_bytes(c, (void**)&c->d_walk, &c->walk_cap, (int64_t)sizeof(double) * n_chains * (2 * D + 1))))
    return rc;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  unsigned char hs[64];
  gwl::set_walk_scalars(hs, lnl_star, scale, worst, counter);
  cudaError_t e = cudaMemcpyAsync(c->d_wscal, hs, gwl::walk_scalars_bytes(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "ns_replace");
  if (c->walk_kind == GWL_WALK_GALILEAN) {
    if ((rc = ensure_bytes(c, (void**)&c->d_gmc, &c->gmc_cap, (int64_t)sizeof(double) * gwl::gmc_scratch_doubles(n_chains, D))))
      return rc;
    if ((rc = ensure_bytes(c, &c->d_pgrad, &c->pgrad_cap, gwl::prop_grad_bytes(c) * n_chains))) return rc;
    if ((rc = ensure_bytes(c, &c->d_gpartials, &c->gpartials_cap, gwl::grad_partials_bytes(c, n_chains)))) return rc;
  }
  double* pu = c->d_walk;
  double* pth = pu + n_chains * D;
  double* plnl = pth + n_chains * D;
  e = gwl::launch_walk(c, live_u, live_lnl, K, c->d_wscal, seed, n_chains, walk_len, chol, out_u, out_lnl, out_nacc,
                       out_start, pu, pth, plnl, st);
  if (e != cudaSuccess) return cuda_fail(e, "ns_replace");
  return GWL_OK;
}

int64_t ns_state_doubles(int64_t K, int64_t D, int64_t max_dead) {
  if (K < 2 || D < 1 || max_dead < 0) return -1;
  return gwl::state_doubles(K, D, max_dead);
}

int ns_run(gwl_ctx* c, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz, int64_t max_rounds,
           double scale0, int64_t max_dead, double* dead_lnl, double* dead_logwt, double* dead_u, gwl_ns_result* out,
           void* stream) {
  return ns_run_resumable(c, K, n_chains, walk_len, seed, dlogz, max_rounds, scale0, max_dead, dead_lnl, dead_logwt,
                          dead_u, out, nullptr, nullptr, stream);
}

int ns_run_resumable(gwl_ctx* c, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                     int64_t max_rounds, double scale0, int64_t max_dead, double* dead_lnl, double* dead_logwt,
                     double* dead_u, gwl_ns_result* out, const double* resume, double* checkpoint, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!out) return fail(GWL_ERR_ARG, "out is null");
  if (resume) {
    const int bad = gwl::state_check(resume, K, gwl::theta_stride(c));
    if (bad == 1) return fail(GWL_ERR_ARG, "resume: not a checkpoint of this format");
    if (bad == 2) return fail(GWL_ERR_ARG, "resume: the checkpoint is for another K or walk dimension");
    if (bad) return fail(GWL_ERR_ARG, "resume: inconsistent dead-point count");
  }
  if (K < 2 || n_chains < 1 || walk_len < 1 || max_rounds < 0 || max_dead < 0)
    return fail(GWL_ERR_ARG, "bad sizes (K >= 2, n_chains >= 1, walk_len >= 1 needed)");
  if (!(scale0 > 0.0)) return fail(GWL_ERR_ARG, "scale0 must be positive");
  if (max_dead > 0 && (!dead_lnl || !dead_logwt || !dead_u)) return fail(GWL_ERR_ARG, "null dead-point buffer");
  if (K > 4096 || n_chains > 4096) return fail(GWL_ERR_ARG, "ns_run supports K <= 4096 and n_chains <= 4096");
  if ((rc = walk_supported(c, "ns_run"))) return rc;
  const int64_t nb = n_chains > K ? n_chains : K;
  if ((rc = ensure_scratch(c, nb))) return rc;
  if (c->walk_kind == GWL_WALK_GALILEAN) {
    const int D = (int)gwl::theta_stride(c);
    if ((rc = ensure_bytes(c, (void**)&c->d_gmc, &c->gmc_cap, (int64_t)sizeof(double) * gwl::gmc_scratch_doubles(n_chains, D))))
      return rc;
    if ((rc = ensure_bytes(c, &c->d_pgrad, &c->pgrad_cap, gwl::prop_grad_bytes(c) * nb))) return rc;
    if ((rc = ensure_bytes(c, &c->d_gpartials, &c->gpartials_cap, gwl::grad_partials_bytes(c, nb)))) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  double res[11];
  const int r = gwl::ns_run_impl(c, K, n_chains, walk_len, seed, dlogz, max_rounds, scale0, max_dead, dead_lnl,
                                 dead_logwt, dead_u, res, st, 1, resume, checkpoint);
  if (r != 0) return fail(GWL_ERR_CUDA, "ns_run: %s", cudaGetErrorString(cudaGetLastError()));
  out->lnZ = res[0];
  out->lnZ_err = res[1];
  out->H = res[2];
  out->n_dead = (int64_t)res[3];
  out->n_proposals = (int64_t)res[4];
  out->rounds = (int64_t)res[5];
  out->scale = res[6];
  out->acceptance = res[7];
  out->consumed_per_round = res[8];
  out->dlogz = res[9];
  out->n_dead_returned = (int64_t)res[10];
  return GWL_OK;
}

struct gwl_multi {
  gwl::Multi* m;
  int E;
  int device;
};

int gwl_multi_create(gwl_ctx* const* ctxs, int n_events, gwl_multi** out) {
  if (!out) return fail(GWL_ERR_ARG, "out is null");
  *out = nullptr;
  if (!ctxs || n_events < 1) return fail(GWL_ERR_ARG, "need at least one context");
  for (int e = 0; e < n_events; ++e) {
    const gwl_ctx* c = ctxs[e];
    if (!c) return fail(GWL_ERR_ARG, "context %d is null", e);
    if (c->device != ctxs[0]->device || c->n_det != ctxs[0]->n_det || c->opt.precision != ctxs[0]->opt.precision ||
        c->opt.n_dim != ctxs[0]->opt.n_dim)
      return fail(GWL_ERR_ARG, "context %d differs in device, detectors, precision or dimension", e);
    if (c->n_cal_nodes != ctxs[0]->n_cal_nodes)
      return fail(GWL_ERR_ARG, "context %d differs in its number of calibration nodes", e);
    if (c->opt.precision == GWL_MIXED_F64PHASE) return fail(GWL_ERR_ARG, "context %d is GWL_MIXED_F64PHASE", e);
  }
  int rc = check_ctx(ctxs[0]);
  if (rc) return rc;
  gwl_multi* h = new (std::nothrow) gwl_multi();
  if (!h) return fail(GWL_ERR_NOMEM, "host allocation failed");
  h->m = gwl::multi_new(ctxs, n_events);
  h->E = n_events;
  h->device = ctxs[0]->device;
  *out = h;
  return GWL_OK;
}

int gwl_multi_loglike(gwl_multi* h, const double* theta_dev, int64_t n_per, double* lnl_dev, void* stream) {
  if (!h) return fail(GWL_ERR_ARG, "null multi-event context");
  if (n_per < 0) return fail(GWL_ERR_ARG, "n_per < 0");
  if (n_per == 0) return GWL_OK;
  if (!theta_dev || !lnl_dev) return fail(GWL_ERR_ARG, "null device pointer");
  if (!gwl::multi_consistent(h->m))
    return fail(GWL_ERR_ARG, "the batch's contexts no longer share their number of calibration nodes");
  cudaError_t e = gwl::multi_prepare(h->m, n_per);
  if (e != cudaSuccess) return cuda_fail(e, "gwl_multi_loglike");
  e = gwl::multi_loglike(h->m, theta_dev, n_per, lnl_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gwl_multi_loglike");
  return GWL_OK;
}

int gwl_multi_ns_run(gwl_multi* h, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                     int64_t max_rounds, double scale0, gwl_ns_result* out, void* stream) {
  return gwl_multi_ns_run_resumable(h, K, n_chains, walk_len, seed, dlogz, max_rounds, scale0, out, nullptr, nullptr,
                                    stream);
}

int64_t gwl_multi_ns_state_doubles(const gwl_multi* h, int64_t K) {
  if (!h || K < 2) return -1;
  return gwl::multi_state_doubles(h->E, K, gwl::multi_dim(h->m));
}

int gwl_multi_ns_run_resumable(gwl_multi* h, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                               int64_t max_rounds, double scale0, gwl_ns_result* out, const double* resume,
                               double* checkpoint, void* stream) {
  if (!h || !out) return fail(GWL_ERR_ARG, "null argument");
  if (resume && K >= 2 && gwl::multi_state_check(resume, h->E, K, gwl::multi_dim(h->m)) != 0)
    return fail(GWL_ERR_ARG, "resume buffer does not match this batch, K and walk dimensions");
  if (K < 2 || n_chains < 1 || walk_len < 1 || max_rounds < 0) return fail(GWL_ERR_ARG, "bad sizes");
  if (K > 4096 || n_chains > 4096) return fail(GWL_ERR_ARG, "gwl_multi_ns_run supports K, n_chains <= 4096");
  if (!(scale0 > 0.0)) return fail(GWL_ERR_ARG, "scale0 must be positive");
  if (!gwl::multi_consistent(h->m))
    return fail(GWL_ERR_ARG, "the batch's contexts no longer share their number of calibration nodes");
  std::vector<double> res((size_t)11 * h->E);
  const int r = gwl::multi_ns_run(h->m, K, n_chains, walk_len, seed, dlogz, max_rounds, scale0, res.data(),
                                  (cudaStream_t)stream, resume, checkpoint);
  if (r != 0) return fail(GWL_ERR_CUDA, "gwl_multi_ns_run: %s", cudaGetErrorString(cudaGetLastError()));
  for (int e = 0; e < h->E; ++e) {
    const double* x = res.data() + 11 * e;
    gwl_ns_result& o = out[e];
    o.lnZ = x[0];
    o.lnZ_err = x[1];
    o.H = x[2];
    o.n_dead = (int64_t)x[3];
    o.n_proposals = (int64_t)x[4];
    o.rounds = (int64_t)x[5];
    o.scale = x[6];
    o.acceptance = x[7];
    o.consumed_per_round = x[8];
    o.dlogz = x[9];
    o.n_dead_returned = 0;
  }
  return GWL_OK;
}

int64_t gwl_multi_launch_count(const gwl_multi* h) { return h ? gwl::multi_launches(h->m) : 0; }

void gwl_multi_destroy(gwl_multi* h) {
  if (!h) return;
  gwl::multi_delete(h->m);
  delete h;
}

}  // extern "C"

namespace gwl {
// One thread waits, bounded, on an mbarrier phase that nothing completes: the
// wait runs out and latches the timeout status like a stalled copy would.
__global__ void k_wait_unsignalled(int* __restrict__ status, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_wait_bounded(&bar, 0, status, limit);
  }
}
}  // namespace gwl

extern "C" {

int gwl_test_wait_timeout(gwl_ctx* c, double seconds, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!(seconds > 0.0) || seconds > 2.0) return fail(GWL_ERR_ARG, "seconds=%g out of range (0, 2]", seconds);
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  const long long limit = (long long)(seconds * 2.07e9);  // SM clocks at the maximum clock
  gwl::k_wait_unsignalled<<<1, 32, 0, st>>>(c->d_status, limit);
  c->launches++;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "gwl_test_wait_timeout");
  return GWL_OK;
}

int gwl_test_ffdelta_blocks(gwl_ctx* c, int enable, int64_t* count) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (count) {
    unsigned long long n = 0;
    if (c->d_ffc) {
      cudaError_t e = cudaDeviceSynchronize();
      if (e == cudaSuccess) e = cudaMemcpy(&n, c->d_ffc, sizeof(n), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "gwl_test_ffdelta_blocks");
    }
    *count = (int64_t)n;
  }
  if (enable == 1) {
    cudaError_t e = cudaSuccess;
    if (!c->d_ffc) {
      e = cudaMalloc((void**)&c->d_ffc, sizeof(unsigned long long));
      if (e == cudaSuccess) c->bytes += (int64_t)sizeof(unsigned long long);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemset(c->d_ffc, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "gwl_test_ffdelta_blocks");
    c->count_ff = true;
  } else if (enable == 0) {
    c->count_ff = false;
  } else if (enable != -1) {
    return fail(GWL_ERR_ARG, "gwl_test_ffdelta_blocks: enable=%d not in {-1, 0, 1}", enable);
  }
  return GWL_OK;
}

int gwl_sync(gwl_ctx* c) {
  int rc = check_ctx(c);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "gwl_sync");
  int st = 0;
  e = cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "gwl_sync status");
  if (st) {
    cudaMemset(c->d_status, 0, sizeof(int));
    if (st & gwl::kStatusTimeout) return fail(GWL_ERR_TIMEOUT, "a kernel's bounded wait ran out");
  }
  return GWL_OK;
}

int gwl_set_walk(gwl_ctx* c, int walk_kind) {
  if (!c) return fail(GWL_ERR_ARG, "null context");
  if (walk_kind != GWL_WALK_RANDOM && walk_kind != GWL_WALK_GALILEAN) return fail(GWL_ERR_ARG, "bad walk kind");
  c->walk_kind = walk_kind;
  return GWL_OK;
}

int gwl_set_galilean(gwl_ctx* c, double persistence) {
  if (!c) return fail(GWL_ERR_ARG, "null context");
  if (!(persistence >= 0.0 && persistence <= 1.0)) return fail(GWL_ERR_ARG, "persistence must be in [0, 1]");
  c->gmc_persistence = persistence;
  return GWL_OK;
}

int gwl_set_tuning(gwl_ctx* c, const gwl_tuning* t) {
  if (!c || !t) return fail(GWL_ERR_ARG, "null argument");
  if (t->window < 0 || t->grad_window < 0 || t->ctas_per_sm < 0 || t->ctas_per_sm > 16 || t->bin_kernel < 0 ||
      t->bin_kernel > GWL_BINS_LANE)
    return fail(GWL_ERR_ARG, "bad tuning value");
  if (t->lane_chunk < 0 || t->lane_chunk % 32) return fail(GWL_ERR_ARG, "lane_chunk must be a multiple of 32");
  if (t->window % 32 || t->grad_window % 32)
    return fail(GWL_ERR_ARG, "windows must be multiples of 32 bins (got %d/%d)", t->window, t->grad_window);
  // likelihood rows: the delta table (mixed) or the FP64 table; gradient rows: the mixed or FP64 table
  const bool mixed = c->opt.precision == GWL_MIXED;
  const size_t row = gwl::lnl_row_bytes(c);
  const size_t grow = mixed ? sizeof(float) * c->row_floats : sizeof(double) * c->row_doubles;
  if ((size_t)t->window * row > gwl::kWindowSmemMax || (size_t)t->grad_window * grow > gwl::kWindowSmemMax)
    return fail(GWL_ERR_ARG, "window of %d/%d bins exceeds shared memory", t->window, t->grad_window);
  if (c->n_cal_nodes && t->grad_window &&
      ((size_t)t->grad_window * (grow + (mixed ? sizeof(float) * c->row_cal_f : sizeof(double) * c->row_cal_d)) >
           gwl::kWindowSmemMax ||
       gwl::calgrad_smem(c, t->grad_window) > gwl::kCalGradSmemMax))
    return fail(GWL_ERR_ARG, "gradient window of %d bins exceeds shared memory with the calibration model",
                t->grad_window);
  if (t->window) c->window = t->window;
  if (t->grad_window) c->grad_window = t->grad_window;
  if (t->ctas_per_sm) c->ctas_per_sm = t->ctas_per_sm;
  if (t->bin_kernel) c->bin_kernel = t->bin_kernel;
  if (t->lane_chunk) c->lane_chunk = t->lane_chunk;
  return GWL_OK;
}

int gwl_get_tuning(const gwl_ctx* c, gwl_tuning* out) {
  if (!c || !out) return fail(GWL_ERR_ARG, "null argument");
  out->window = c->window;
  out->ctas_per_sm = c->ctas_per_sm;
  out->grad_window = c->grad_window;
  out->ms_loglike = c->tuned_ms[0];
  out->ms_grad = c->tuned_ms[1];
  out->n_tried = c->tuned_n;
  out->bin_kernel = c->bin_kernel;
  out->lane_chunk = c->lane_chunk;
  return GWL_OK;
}

int gwl_set_calibration(gwl_ctx* c, int n_nodes, const double* node_freqs, double sigma_amp, double sigma_phase) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (n_nodes && (rc = likelihood_only(c, "the calibration model"))) return rc;
  if (n_nodes != 0 && (n_nodes < 2 || n_nodes > GWL_MAX_CAL_NODES))
    return fail(GWL_ERR_ARG, "n_nodes=%d outside {0} and [2, %d]", n_nodes, GWL_MAX_CAL_NODES);
  if (n_nodes && !node_freqs) return fail(GWL_ERR_ARG, "node_freqs is null");
  if (n_nodes && (!(sigma_amp > 0.0) || !(sigma_phase > 0.0) || !std::isfinite(sigma_amp) ||
                  !std::isfinite(sigma_phase)))
    return fail(GWL_ERR_ARG, "calibration prior widths must be positive");
  for (int k = 0; k < n_nodes; ++k) {
    if (!(node_freqs[k] > 0.0) || !std::isfinite(node_freqs[k]))
      return fail(GWL_ERR_ARG, "node_freqs[%d] not positive", k);
    if (k > 0 && !(std::log(node_freqs[k]) > std::log(node_freqs[k - 1])))
      return fail(GWL_ERR_ARG, "node_freqs must increase strictly (at %d)", k);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail(cudaGetLastError(), "gwl_set_calibration");
  dev_free(c, c->d_cal_f, (c->M + 1) * c->row_cal_f);
  dev_free(c, c->d_cal_d, (c->M + 1) * c->row_cal_d);
  dev_free(c, c->d_calQ_f, gwl::kMaxCalNodes * gwl::kMaxCalNodes);
  dev_free(c, c->d_calQ_d, gwl::kMaxCalNodes * gwl::kMaxCalNodes);
  c->n_cal_nodes = 0;
  c->seg.stride = c->opt.n_dim;
  c->cal_gen++;  // multi-event batches holding this context rebuild their descriptors
  if (n_nodes == 0) return GWL_OK;

  std::vector<double> x(n_nodes);
  for (int k = 0; k < n_nodes; ++k) x[k] = std::log(node_freqs[k]);
  const std::vector<double> Q = natural_spline_matrix(n_nodes, x.data());
  std::vector<float> Qf(Q.size());
  for (size_t i = 0; i < Q.size(); ++i) Qf[i] = (float)Q[i];
  c->row_cal_f = gwl::cal_row_floats(c->n_det);
  c->row_cal_d = gwl::cal_row_doubles(c->n_det);
  double* d_x = nullptr;
  cudaError_t e;
  do {
    if ((e = dev_alloc(c, &c->d_cal_f, (c->M + 1) * c->row_cal_f)) != cudaSuccess) break;
    if ((e = dev_alloc(c, &c->d_cal_d, (c->M + 1) * c->row_cal_d)) != cudaSuccess) break;
    if ((e = dev_alloc(c, &c->d_calQ_f, gwl::kMaxCalNodes * gwl::kMaxCalNodes)) != cudaSuccess) break;
    if ((e = dev_alloc(c, &c->d_calQ_d, gwl::kMaxCalNodes * gwl::kMaxCalNodes)) != cudaSuccess) break;
    if ((e = cudaMalloc(&d_x, sizeof(double) * n_nodes)) != cudaSuccess) break;
    if ((e = cudaMemcpy(d_x, x.data(), sizeof(double) * n_nodes, cudaMemcpyHostToDevice)) != cudaSuccess) break;
    if ((e = cudaMemcpy(c->d_calQ_d, Q.data(), sizeof(double) * Q.size(), cudaMemcpyHostToDevice)) != cudaSuccess) break;
    if ((e = cudaMemcpy(c->d_calQ_f, Qf.data(), sizeof(float) * Qf.size(), cudaMemcpyHostToDevice)) != cudaSuccess) break;
    c->n_cal_nodes = n_nodes;
    if ((e = gwl::launch_cal_tables(c, d_x, 0)) != cudaSuccess) break;
    e = cudaDeviceSynchronize();
  } while (false);
  if (d_x) cudaFree(d_x);
  if (e != cudaSuccess) {
    c->n_cal_nodes = 0;
    return cuda_fail(e, "gwl_set_calibration");
  }
  c->seg.stride = c->opt.n_dim + 2 * n_nodes * c->n_det;
  c->cal_sigma[0] = sigma_amp;
  c->cal_sigma[1] = sigma_phase;
  // the likelihood and gradient windows must still fit shared memory with the calibration rows
  const size_t row = gwl::lnl_row_bytes(c);
  while (c->window > 32 && (size_t)c->window * row > gwl::kWindowSmemMax) c->window -= 32;
  const bool mixed = c->opt.precision == GWL_MIXED;
  const size_t grow = (mixed ? sizeof(float) * (c->row_floats + c->row_cal_f) : sizeof(double) * (c->row_doubles + c->row_cal_d));
  while (c->grad_window > 32 && ((size_t)c->grad_window * grow > gwl::kWindowSmemMax ||
                                 gwl::calgrad_smem(c, c->grad_window) > gwl::kCalGradSmemMax))
    c->grad_window -= 32;
  return GWL_OK;
}

int gwl_get_calibration(const gwl_ctx* c, int* n_nodes, int64_t* theta_stride) {
  if (!c) return fail(GWL_ERR_ARG, "null context");
  if (n_nodes) *n_nodes = c->n_cal_nodes;
  if (theta_stride) *theta_stride = c->seg.stride;
  return GWL_OK;
}

int gwl_profile(gwl_ctx* c, int enable) {
  if (!c) return fail(GWL_ERR_ARG, "null context");
  for (int k = 0; k < GWL_KERNEL_KINDS; ++k) {
    for (auto& pr : c->prof_pending[k]) {
      c->event_pool.push_back(pr.first);
      c->event_pool.push_back(pr.second);
    }
    c->prof_pending[k].clear();
    c->prof_ms[k] = 0.0;
    c->prof_n[k] = 0;
  }
  c->profiling = enable != 0;
  return GWL_OK;
}

int gwl_profile_read(gwl_ctx* c, int kind, double* total_ms, int64_t* count) {
  if (!c) return fail(GWL_ERR_ARG, "null context");
  if (kind < 0 || kind >= GWL_KERNEL_KINDS) return fail(GWL_ERR_ARG, "bad kernel kind %d", kind);
  for (auto& pr : c->prof_pending[kind]) {
    cudaError_t e = cudaEventSynchronize(pr.second);
    if (e != cudaSuccess) return cuda_fail(e, "profile");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e != cudaSuccess) return cuda_fail(e, "profile");
    c->prof_ms[kind] += ms;
    c->prof_n[kind] += 1;
    c->event_pool.push_back(pr.first);
    c->event_pool.push_back(pr.second);
  }
  c->prof_pending[kind].clear();
  if (total_ms) *total_ms = c->prof_ms[kind];
  if (count) *count = c->prof_n[kind];
  return GWL_OK;
}

int64_t gwl_device_bytes(const gwl_ctx* c) { return c ? c->bytes : 0; }
int64_t gwl_launch_count(const gwl_ctx* c) { return c ? c->launches : 0; }

void gwl_destroy(gwl_ctx* c) {
  if (!c) return;
  gwl_profile(c, 0);
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  c->event_pool.clear();
  dev_free(c, c->d_freqs, c->M);
  dev_free(c, c->d_geom, 9 * c->n_det);
  dev_free(c, c->d_H, (int64_t)c->n_det * c->M);
  dev_free(c, c->d_tab_mixed, c->M * c->row_floats);
  dev_free(c, c->d_tab_delta, c->M * c->row_delta);
  dev_free(c, c->d_anchor, (c->M + gwl::kAnchor - 1) / gwl::kAnchor * gwl::kAnchorRowFloats);
  dev_free(c, c->d_tab_f64, c->M * c->row_doubles);
  dev_free(c, c->d_cal_f, (c->M + 1) * c->row_cal_f);
  dev_free(c, c->d_cal_d, (c->M + 1) * c->row_cal_d);
  dev_free(c, c->d_calQ_f, gwl::kMaxCalNodes * gwl::kMaxCalNodes);
  dev_free(c, c->d_calQ_d, gwl::kMaxCalNodes * gwl::kMaxCalNodes);
  dev_free(c, c->d_pm, c->prop_cap);
  dev_free(c, c->d_pf, c->prop_cap);
  dev_free(c, c->d_pc, c->prop_cap);
  dev_free(c, c->d_partials, c->partials_cap);
  dev_free(c, c->d_io, c->io_cap);
  dev_free(c, c->d_work, c->work_cap);
  dev_free(c, c->d_blist, c->blist_cap);
  dev_free(c, c->d_status, 4);
  dev_free(c, c->d_ffc, 1);
  if (c->d_pgrad) cudaFree(c->d_pgrad);
  if (c->d_walk) cudaFree(c->d_walk);
  if (c->d_gmc) cudaFree(c->d_gmc);
  if (c->d_wscal) cudaFree(c->d_wscal);
  if (c->d_gpartials) cudaFree(c->d_gpartials);
  delete c;
}

}  // extern "C"

namespace gwl {
cudaError_t raise_smem_limit(const void* kernel, int device, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> set;
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = set[std::make_pair(kernel, device)];
  if (bytes <= have) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

static cudaEvent_t take_event(gwl_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
ProfScope::ProfScope(gwl_ctx* c_, int kind_, cudaStream_t st_) : c(c_), kind(kind_), st(st_) {
  if (!c->profiling) return;
  e0 = take_event(c);
  e1 = take_event(c);
  if (e0) cudaEventRecord(e0, st);
}
ProfScope::~ProfScope() {
  if (!c->profiling || !e0 || !e1) return;
  cudaEventRecord(e1, st);
  c->prof_pending[kind].emplace_back(e0, e1);
}
}  // namespace gwl
