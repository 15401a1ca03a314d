// Grid transfers of the coarse-to-fine scheme (Sec. 3.3, App. C): separable
// periodic Fourier resampling with smoothing in Fourier space.  Along each axis
// the output sample i is the windowed trigonometric interpolant of the input at
// t = i N_in / N_out:
//   out_i = sum_j M[i][j] in_j,
//   M[i][j] = (1/N_in) (w(0) + 2 sum_{k=1..K} w(k) cos(2 pi k (t_i - j) / N_in)),
//   K = floor((min(N_in, N_out) - 1) / 2),
// with w = 1 (plain Fourier interpolation), the Blackman window
// 0.42 + 0.5 cos(pi k/(K+1)) + 0.08 cos(2 pi k/(K+1)) (model up-sampling) or the
// Kaiser window I0(beta sqrt(1 - (k/(K+1))^2)) / I0(beta) (time-series
// low-pass).  The matrices are built on the host in FP64 (closed form above),
// stored in FP32 and applied with FP64 accumulation, axis by axis (x, y, z).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/fwi.h"

namespace {

constexpr int kThreads = 256;

// out[o][i][q] = sum_j MT[j][i] in[o][j][q]; MT stored [n_in][n_out]
__global__ void k_apply_axis(const float* __restrict__ in, float* __restrict__ out,
                             const float* __restrict__ MT, int n_in, int n_out, int64_t inner,
                             int64_t outer) {
  const int64_t total = outer * n_out * inner;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx % inner;
    const int64_t t = idx / inner;
    const int i = (int)(t % n_out);
    const int64_t o = t / n_out;
    const float* src = in + o * n_in * inner + q;
    double acc = 0.0;
    for (int j = 0; j < n_in; ++j) acc += (double)MT[(size_t)j * n_out + i] * (double)__ldg(&src[j * inner]);
    out[idx] = (float)acc;
  }
}

double bessel_i0(double x) {   // power series of I0
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 200; ++k) {
    term *= (x / (2.0 * k)) * (x / (2.0 * k));
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

std::vector<float> build_matrix_t(int n_in, int n_out, int window, double beta) {
  const int K = (std::min(n_in, n_out) - 1) / 2;
  std::vector<double> w(K + 1);
  for (int k = 0; k <= K; ++k) {
    const double r = (double)k / (K + 1);
    if (window == 1) w[k] = 0.42 + 0.5 * std::cos(M_PI * r) + 0.08 * std::cos(2.0 * M_PI * r);
    else if (window == 2) w[k] = bessel_i0(beta * std::sqrt(1.0 - r * r)) / bessel_i0(beta);
    else w[k] = 1.0;
  }
  std::vector<float> mt((size_t)n_in * n_out);
  for (int i = 0; i < n_out; ++i) {
    const double ti = (double)i * n_in / n_out;
    for (int j = 0; j < n_in; ++j) {
      double s = w[0];
      for (int k = 1; k <= K; ++k) s += 2.0 * w[k] * std::cos(2.0 * M_PI * k * (ti - j) / n_in);
      mt[(size_t)j * n_out + i] = (float)(s / n_in);
    }
  }
  return mt;
}

}  // namespace

struct fwi_resampler {
  int n_in[3], n_out[3], window[3];
  double beta;
  bool active[3];
  std::vector<float> mt[3];
  size_t o_mt[3] = {0, 0, 0}, o_a = 0, o_b = 0, bytes = 0;
  char* ws = nullptr;
};

extern "C" {

fwi_status fwi_resampler_create(const int32_t n_in[3], const int32_t n_out[3], const int32_t window[3],
                                double kaiser_beta, double scale, size_t* workspace_bytes, fwi_resampler** out) {
  if (!n_in || !n_out || !window || !workspace_bytes || !out) return FWI_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (n_in[a] < 1 || n_out[a] < 1 || n_in[a] > 8192 || n_out[a] > 8192 || window[a] < 0 || window[a] > 2)
      return FWI_EINVAL;
  if (!(kaiser_beta >= 0.0) || !std::isfinite(scale)) return FWI_EINVAL;
  bool any = false;
  for (int a = 0; a < 3; ++a) any = any || n_in[a] != n_out[a] || window[a] != 0;
  if (!any && scale != 1.0) return FWI_EINVAL;   // a scale rides on the last active axis
  fwi_resampler* R = new (std::nothrow) fwi_resampler;
  if (!R) return FWI_ENOMEM;
  R->beta = kaiser_beta;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t off = 0;
  for (int a = 0; a < 3; ++a) {
    R->n_in[a] = n_in[a];
    R->n_out[a] = n_out[a];
    R->window[a] = window[a];
    R->active[a] = n_in[a] != n_out[a] || window[a] != 0;
    if (R->active[a]) {
      R->mt[a] = build_matrix_t(n_in[a], n_out[a], window[a], kaiser_beta);
      R->o_mt[a] = off;
      off += up(R->mt[a].size() * 4);
    }
  }
  for (int a = 2; a >= 0; --a)
    if (R->active[a]) {
      for (float& v : R->mt[a]) v = (float)(v * scale);
      break;
    }
  // intermediates: after x [nz_in][ny_in][nx_out], after y [nz_in][ny_out][nx_out]
  // (either buffer may hold either intermediate: size both for the larger)
  const size_t sa = (size_t)n_in[2] * n_in[1] * n_out[0], sb = (size_t)n_in[2] * n_out[1] * n_out[0];
  const size_t sm = std::max(sa, sb);
  R->o_a = off;
  off += up(sm * 4);
  R->o_b = off;
  off += up(sm * 4);
  R->bytes = off;
  *workspace_bytes = off;
  *out = R;
  return FWI_OK;
}

fwi_status fwi_resampler_bind_workspace(fwi_resampler* R, void* dev_ptr, size_t bytes) {
  if (!R || !dev_ptr || ((uintptr_t)dev_ptr & 255) || bytes < R->bytes) return FWI_EINVAL;
  R->ws = static_cast<char*>(dev_ptr);
  for (int a = 0; a < 3; ++a)
    if (R->active[a] &&
        cudaMemcpy(R->ws + R->o_mt[a], R->mt[a].data(), R->mt[a].size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return FWI_ECUDA;
  return FWI_OK;
}

fwi_status fwi_resample(fwi_resampler* R, const float* in, float* out, void* stream) {
  if (!R || !R->ws || !in || !out) return FWI_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int* ni = R->n_in;
  const int* no = R->n_out;
  float* A = reinterpret_cast<float*>(R->ws + R->o_a);
  float* B = reinterpret_cast<float*>(R->ws + R->o_b);
  const float* cur = in;
  // the last active axis writes `out`; an array with no active axis is copied
  int last = -1;
  for (int a = 0; a < 3; ++a)
    if (R->active[a]) last = a;
  if (last < 0) {
    const size_t n = (size_t)ni[0] * ni[1] * ni[2] * 4;
    return cudaMemcpyAsync(out, in, n, cudaMemcpyDeviceToDevice, st) == cudaSuccess ? FWI_OK : FWI_ECUDA;
  }
  // shapes along the way: x first, then y, then z
  int64_t dims[3] = {ni[0], ni[1], ni[2]};
  for (int a = 0; a < 3; ++a) {
    if (!R->active[a]) continue;
    int64_t inner = 1, outer = 1;
    for (int b = 0; b < a; ++b) inner *= dims[b];
    for (int b = a + 1; b < 3; ++b) outer *= dims[b];
    float* dst = a == last ? out : (a == 0 ? A : (cur == A ? B : A));
    const int64_t total = outer * no[a] * inner;
    const int blocks = (int)std::min<int64_t>(4 * 148 * 8, (total + kThreads - 1) / kThreads);
    k_apply_axis<<<blocks, kThreads, 0, st>>>(cur, dst, reinterpret_cast<const float*>(R->ws + R->o_mt[a]), ni[a],
                                              no[a], inner, outer);
    dims[a] = no[a];
    cur = dst;
  }
  return cudaGetLastError() == cudaSuccess ? FWI_OK : FWI_ECUDA;
}

fwi_status fwi_resampler_destroy(fwi_resampler* R) {
  delete R;
  return FWI_OK;
}

}  // extern "C"
