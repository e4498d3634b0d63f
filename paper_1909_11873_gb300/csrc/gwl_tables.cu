// gwl_tables.cu -- per-segment tables, built once by gwl_create.
//
// For every bin j (f = f_j):
//   basis   B_m(f) = f^{-5/3}, f^{-1}, f^{-2/3}, f^{-1/3}, ln f, f^{1/3}, f^{1/3} ln f, f^{2/3}
//   data    G_d,j = 4 df conj(d_d,j) f^{-7/6} / S_d,j * e^{-2 pi i f t_ref}
//   norm    H_d[j] = sum_{i <= j} 4 df f_i^{-7/3} / S_d,i   (inclusive prefix)
// so that, with r_d,j = sum_m c_m B_m(f_j) + tau_d f_j in cycles,
//   <d|h>_d = Re[K_d sum_j G_d,j e^{-2 pi i r_d,j}],   <h|h>_d = |K_d|^2 H_d[ncut - 1]
// (Eq. 2 of the paper, split into a data-dependent and a template-dependent part).
// The mixed likelihood also gets a delta table, dB_m(f_j) = B_m(f_j) - B_m(f_a)
// with a = kAnchor floor(j / kAnchor) (FP64 difference, as a float pair), and
// an anchor table with B_m(f_a) and f_a as float pairs and the largest |dB_m|
// of the block (the last bin's: every B_m is monotonic in f for f > 1 Hz).
#include "gwl_internal.h"

namespace gwl {

__device__ __forceinline__ void basis_values(double f, double (&b)[kNBasis]) {
  const double c1 = cbrt(f);
  const double lf = log(f);
  b[0] = 1.0 / (f * c1 * c1);
  b[1] = 1.0 / f;
  b[2] = 1.0 / (c1 * c1);
  b[3] = 1.0 / c1;
  b[4] = lf;
  b[5] = c1;
  b[6] = c1 * lf;
  b[7] = c1 * c1;
}

__global__ void k_table_rows(const double* __restrict__ freqs, const double* __restrict__ strain,
                             const double* __restrict__ psd, int64_t M, int n_det, double df, double t_ref,
                             float* __restrict__ tab_m, int row_f, double* __restrict__ tab_d, int row_d,
                             float* __restrict__ tab_x, int row_x, float* __restrict__ anc,
                             double* __restrict__ hterm) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const double f = freqs[j];
  double b[kNBasis], ba[kNBasis];
  basis_values(f, b);
  const int64_t ja = j - j % kAnchor;
  basis_values(freqs[ja], ba);
  float* rx = tab_x + j * row_x;
  const int lo_off = kNBasis + 2 * n_det;  // low parts after G
  for (int k = lo_off + kNBasis; k < row_x; ++k) rx[k] = 0.0f;
#pragma unroll
  for (int m = 0; m < kNBasis; ++m) split_f64(b[m] - ba[m], rx[m], rx[lo_off + m]);
  if (j == ja) {
    float* ra = anc + (j / kAnchor) * kAnchorRowFloats;
#pragma unroll
    for (int m = 0; m < kNBasis; ++m) split_f64(b[m], ra[m], ra[kNBasis + m]);
    split_f64(f, ra[16], ra[17]);
    const int64_t jl = (j + kAnchor - 1 < M ? j + kAnchor - 1 : M - 1);
    double bl[kNBasis];
    basis_values(freqs[jl], bl);
#pragma unroll
    for (int m = 0; m < kNBasis; ++m) ra[18 + m] = (float)fabs(bl[m] - b[m]) * 1.0000001f;
    ra[26] = ra[27] = 0.0f;
  }
  float* rm = tab_m + j * row_f;
  double* rd = tab_d + j * row_d;
#pragma unroll
  for (int m = 0; m < kNBasis; ++m) {
    float hi, lo;
    split_f64(b[m], hi, lo);
    rm[m] = hi;
    rm[kNBasis + m] = lo;
    rd[m] = b[m];
  }
  float fh, fl;
  split_f64(f, fh, fl);
  rm[16] = fh;
  rm[17] = fl;
  rd[8] = f;
  // e^{-2 pi i f t_ref}: reduce f t_ref to [0, 1) cycles first
  const double x = f * t_ref;
  const double fr = x - floor(x);
  double sr, cr;
  sincospi(2.0 * fr, &sr, &cr);
  const double f76 = pow(f, -7.0 / 6.0);
  for (int d = 0; d < n_det; ++d) {
    const double S = psd[(int64_t)d * M + j];
    const double w = 4.0 * df * f76 / S;
    const double dr = strain[2 * ((int64_t)d * M + j)];
    const double di = strain[2 * ((int64_t)d * M + j) + 1];
    const double gr = w * (dr * cr - di * sr);
    const double gi = -w * (dr * sr + di * cr);
    rd[9 + 2 * d] = gr;
    rd[10 + 2 * d] = gi;
    rm[18 + 2 * d] = (float)gr;
    rm[19 + 2 * d] = (float)gi;
    rx[kNBasis + 2 * d] = (float)gr;
    rx[kNBasis + 2 * d + 1] = (float)gi;
    hterm[(int64_t)d * M + j] = 4.0 * df * f76 * f76 / S;
  }
  for (int k = 18 + 2 * n_det; k < row_f; ++k) rm[k] = 0.0f;
  for (int k = 9 + 2 * n_det; k < row_d; ++k) rd[k] = 0.0;
}

// In-place inclusive prefix sum of one detector's row, one CTA per detector.
// Each thread sums a contiguous segment serially; segment totals are scanned
// serially by thread 0; the order of additions is fixed (deterministic).
__global__ void k_prefix_scan(double* __restrict__ H, int64_t M) {
  __shared__ double tot[1024];
  double* h = H + (int64_t)blockIdx.x * M;
  const int T = blockDim.x;
  const int64_t seg = (M + T - 1) / T;
  const int64_t a = threadIdx.x * seg;
  const int64_t b = a + seg < M ? a + seg : M;
  double s = 0.0;
  for (int64_t j = a; j < b; ++j) s += h[j];
  tot[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = 0.0;
    for (int t = 0; t < T; ++t) {
      const double v = tot[t];
      tot[t] = run;
      run += v;
    }
  }
  __syncthreads();
  double run = tot[threadIdx.x];
  for (int64_t j = a; j < b; ++j) {
    run += h[j];
    h[j] = run;
  }
}

// Multiply the data weights by 2^-e and the prefix sums by 2^-2e (exact).
__global__ void k_scale_tables(int64_t M, int n_det, double sg, float* __restrict__ tab_m, int row_f,
                               double* __restrict__ tab_d, int row_d, float* __restrict__ tab_x, int row_x,
                               double* __restrict__ H) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  for (int d = 0; d < n_det; ++d) {
    tab_d[j * row_d + 9 + 2 * d] *= sg;
    tab_d[j * row_d + 10 + 2 * d] *= sg;
    tab_m[j * row_f + 18 + 2 * d] = (float)tab_d[j * row_d + 9 + 2 * d];
    tab_m[j * row_f + 19 + 2 * d] = (float)tab_d[j * row_d + 10 + 2 * d];
    tab_x[j * row_x + kNBasis + 2 * d] = tab_m[j * row_f + 18 + 2 * d];
    tab_x[j * row_x + kNBasis + 2 * d + 1] = tab_m[j * row_f + 19 + 2 * d];
    H[(int64_t)d * M + j] *= sg * sg;
  }
}

cudaError_t launch_scale_tables(gwl_ctx* c, double sg, cudaStream_t st) {
  const int T = 256;
  k_scale_tables<<<(unsigned)((c->M + T - 1) / T), T, 0, st>>>(c->M, c->n_det, sg, c->d_tab_mixed, c->row_floats,
                                                                c->d_tab_f64, c->row_doubles, c->d_tab_delta,
                                                                c->row_delta, c->d_H);
  c->launches++;
  return cudaGetLastError();
}

// Calibration rows (layout in gwl_device.cuh): bin j's interval k of the
// nodes xn (ln f_k) -- the first or last interval outside them -- its local
// coordinate t and h^2/6, and the per-detector <h|h> weights dH_d,j of the
// (scaled) prefix sums.
__global__ void k_cal_rows(const double* __restrict__ freqs, const double* __restrict__ H, int64_t M, int n_det,
                           const double* __restrict__ xn, int nn, float* __restrict__ cf, int row_f,
                           double* __restrict__ cd, int row_d) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const double x = log(freqs[j]);
  int k = 0;
  while (k < nn - 2 && x >= xn[k + 1]) ++k;
  const double h = xn[k + 1] - xn[k];
  const double t = (x - xn[k]) / h;
  const double h6 = h * h / 6.0;
  double* rd = cd + j * row_d;
  float* rf = cf + j * row_f;
  rd[0] = t;
  rd[1] = h6;
  rd[2] = (double)k;
  rf[0] = (float)t;
  rf[1] = (float)h6;
  rf[2] = __int_as_float(k);
  for (int d = 0; d < n_det; ++d) {
    const double dh = H[(int64_t)d * M + j] - (j > 0 ? H[(int64_t)d * M + j - 1] : 0.0);
    rd[3 + d] = dh;
    rf[3 + d] = (float)dh;
  }
  for (int i = 3 + n_det; i < row_d; ++i) rd[i] = 0.0;
  for (int i = 3 + n_det; i < row_f; ++i) rf[i] = 0.0f;
}

cudaError_t launch_cal_tables(gwl_ctx* c, const double* d_xnode, cudaStream_t st) {
  const int T = 256;
  // the zero row past the last bin
  cudaError_t e = cudaMemsetAsync(c->d_cal_f + c->M * c->row_cal_f, 0, sizeof(float) * c->row_cal_f, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_cal_d + c->M * c->row_cal_d, 0, sizeof(double) * c->row_cal_d, st);
  if (e != cudaSuccess) return e;
  k_cal_rows<<<(unsigned)((c->M + T - 1) / T), T, 0, st>>>(c->d_freqs, c->d_H, c->M, c->n_det, d_xnode,
                                                            c->n_cal_nodes, c->d_cal_f, c->row_cal_f, c->d_cal_d,
                                                            c->row_cal_d);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_build_tables(gwl_ctx* c, const double* d_strain, const double* d_psd, cudaStream_t st) {
  const int T = 256;
  const int64_t nb = (c->M + T - 1) / T;
  k_table_rows<<<(unsigned)nb, T, 0, st>>>(c->d_freqs, d_strain, d_psd, c->M, c->n_det, c->df, c->opt.t_ref,
                                            c->d_tab_mixed, c->row_floats, c->d_tab_f64, c->row_doubles,
                                            c->d_tab_delta, c->row_delta, c->d_anchor, c->d_H);
  c->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_prefix_scan<<<c->n_det, 1024, 0, st>>>(c->d_H, c->M);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace gwl
