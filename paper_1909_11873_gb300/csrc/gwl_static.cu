// gwl_static.cu -- gwl_loglike_static: the batched log-likelihood with its
// per-call scratch taken from a fixed device array instead of cudaMalloc.
//
// Some callers cannot allocate device memory at the point where they need a
// likelihood batch: a host that hands all free device memory to its own
// caching allocator (a raw cudaMalloc may then fail), or a caller in a loop
// that must not block (cudaMalloc and cudaFree may synchronise the whole
// device).  For them this entry point runs the same kernels as gwl_loglike
// but places the per-proposal coefficients and the per-window partial sums in
// the array below, which the CUDA module reserves on every device that loads
// the library and keeps until the process exits.  The context (tables built
// by gwl_create), theta and lnL stay the caller's.
#include <mutex>

#include "gwl_internal.h"

namespace gwl {
int64_t partials_needed(const gwl_ctx* c, int64_t B);
int64_t work_needed(const gwl_ctx* c, int64_t B);
int set_error(int code, const char* fmt, ...);
}  // namespace gwl

// 16 MiB, shared by every call on the device.
static __device__ __align__(256) unsigned char g_static_scratch[GWL_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// The array's device address on `dev` (current): looked up once and kept.
cudaError_t lookup_scratch(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_addr[dev]) return cudaSuccess;
  const cudaError_t e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_static_scratch);
  if (e != cudaSuccess) g_scratch_addr[dev] = nullptr;
  return e;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of the fixed array that a batch of B needs on this context.
size_t static_bytes_needed(const gwl_ctx* c, int64_t B) {
  size_t n = 0;
  n += align256(sizeof(gwl::PropMixed) * (size_t)B);
  n += align256(sizeof(gwl::PropF64) * (size_t)B);
  n += align256(sizeof(gwl::PropCommon) * (size_t)B);
  n += align256(sizeof(double) * (size_t)gwl::partials_needed(c, B));
  n += align256(sizeof(int) * (size_t)gwl::work_needed(c, B));
  n += align256(sizeof(int) * (size_t)gwl::lanes_list_ints(c, B));
  return n;
}

}  // namespace

namespace gwl {
// Set-up from gwl_create (device `dev` current): look the array's address up
// afresh.  A cudaDeviceReset frees the array with everything else on the
// device, and a context made afterwards must not see the address of the old
// one; contexts made before the reset are invalid anyway.
cudaError_t static_scratch_setup(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return cudaSuccess;  // such devices are refused by the entry point
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_scratch_addr[dev] = nullptr;
  }
  return lookup_scratch(dev);
}
}  // namespace gwl

extern "C" int gwl_loglike_static(gwl_ctx* c, const double* theta_dev, int64_t B, double* lnl_dev, void* stream) {
  if (!c) return gwl::set_error(GWL_ERR_ARG, "null context");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
    return gwl::set_error(GWL_ERR_ARG, "context belongs to device %d but device %d is current", c->device, dev);
  if (B < 0) return gwl::set_error(GWL_ERR_ARG, "B = %lld < 0", (long long)B);
  if (B == 0) return GWL_OK;
  if (!theta_dev || !lnl_dev) return gwl::set_error(GWL_ERR_ARG, "null device pointer");
  const size_t need = static_bytes_needed(c, B);
  if (need > GWL_STATIC_SCRATCH_BYTES)
    return gwl::set_error(GWL_ERR_ARG,
                           "gwl_loglike_static: the batch needs %lld bytes of scratch but the fixed device array "
                           "holds %lld; use a smaller batch or gwl_loglike",
                           (long long)need, (long long)GWL_STATIC_SCRATCH_BYTES);
  if (dev < 0 || dev >= kMaxDevices) return gwl::set_error(GWL_ERR_ARG, "device index %d unsupported", dev);

  // The device address of the fixed array (looked up by gwl_create on this
  // device; looked up here only if that failed).
  void* base = nullptr;
  {
    const cudaError_t e = lookup_scratch(dev);
    if (e != cudaSuccess)
      return gwl::set_error(GWL_ERR_CUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_mu);
    base = g_scratch_addr[dev];
  }

  // Point the context's scratch at the fixed array for this call only.
  unsigned char* p = static_cast<unsigned char*>(base);
  gwl::PropMixed* pm = reinterpret_cast<gwl::PropMixed*>(p);
  p += align256(sizeof(gwl::PropMixed) * (size_t)B);
  gwl::PropF64* pf = reinterpret_cast<gwl::PropF64*>(p);
  p += align256(sizeof(gwl::PropF64) * (size_t)B);
  gwl::PropCommon* pc = reinterpret_cast<gwl::PropCommon*>(p);
  p += align256(sizeof(gwl::PropCommon) * (size_t)B);
  double* partials = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * (size_t)gwl::partials_needed(c, B));
  int* work = reinterpret_cast<int*>(p);
  p += align256(sizeof(int) * (size_t)gwl::work_needed(c, B));
  int* blist = reinterpret_cast<int*>(p);

  gwl::PropMixed* s_pm = c->d_pm;
  gwl::PropF64* s_pf = c->d_pf;
  gwl::PropCommon* s_pc = c->d_pc;
  double* s_part = c->d_partials;
  int* s_work = c->d_work;
  int* s_blist = c->d_blist;
  const bool s_prof = c->profiling;
  c->d_pm = pm;
  c->d_pf = pf;
  c->d_pc = pc;
  c->d_partials = partials;
  c->d_work = work;
  c->d_blist = blist;
  c->profiling = false;  // event pairs are created on demand; keep this call free of any allocation
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  cudaError_t e = gwl::launch_loglike(c, theta_dev, B, lnl_dev, st);
  c->d_pm = s_pm;
  c->d_pf = s_pf;
  c->d_pc = s_pc;
  c->d_partials = s_part;
  c->d_work = s_work;
  c->d_blist = s_blist;
  c->profiling = s_prof;
  if (e != cudaSuccess) return gwl::set_error(GWL_ERR_CUDA, "gwl_loglike_static: %s", cudaGetErrorString(e));
  return GWL_OK;
}
