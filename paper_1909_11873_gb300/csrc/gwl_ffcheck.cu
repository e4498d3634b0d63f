// gwl_ffcheck.cu -- gwl_ff_eval: the float-float elementary functions of the
// mixed prologue, and the FP32 sin(pi x), cos(pi x) of the gradient's bin
// loop, evaluated on given arguments (a diagnostic entry point, so that their
// accuracy can be checked against FP64 references).
#include "gwl_ff.cuh"

namespace gwl {
int set_error(int code, const char* fmt, ...);

__global__ void k_ff_eval(const double* __restrict__ x, int64_t n, int fn, double* __restrict__ out, SinCosTab sct) {
  __shared__ float2 tab[64];
  if (threadIdx.x < 64) tab[threadIdx.x] = sct.v[threadIdx.x];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (fn == GWL_F32_SINPI || fn == GWL_F32_COSPI) {  // sin and cos of pi x = 2 pi (x / 2)
    float sp, cp;
    sincos_cycles_tab(0.5f * (float)x[i], tab, &sp, &cp);
    out[i] = (double)(fn == GWL_F32_SINPI ? sp : cp);
    return;
  }
  const FF a = ff_from(x[i]);
  FF r, s, c;
  switch (fn) {
    case GWL_FF_EXP: r = ff_exp(a); break;
    case GWL_FF_LOG: r = ff_log(a); break;
    case GWL_FF_SIN: ff_sincos(a, &s, &c); r = s; break;
    default: ff_sincos(a, &s, &c); r = c; break;
  }
  out[i] = ff_to_double(r);
}
}  // namespace gwl

extern "C" int gwl_ff_eval(const double* x_dev, int64_t n, int fn, double* out_dev, void* stream) {
  if (n < 0 || (n > 0 && (!x_dev || !out_dev))) return gwl::set_error(GWL_ERR_ARG, "gwl_ff_eval: bad arguments");
  if (fn < GWL_FF_EXP || fn > GWL_F32_COSPI) return gwl::set_error(GWL_ERR_ARG, "gwl_ff_eval: bad function %d", fn);
  if (n == 0) return GWL_OK;
  gwl::k_ff_eval<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x_dev, n, fn, out_dev,
                                                                                gwl::make_sincos_tab());
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gwl::set_error(GWL_ERR_CUDA, "gwl_ff_eval: %s", cudaGetErrorString(e));
  return GWL_OK;
}
