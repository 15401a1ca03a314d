// Device side of the stochastic L-BFGS optimiser of Alg. 2: an L-BFGS history
// of m pairs (s, y) of n-vectors (stored in FP32, every dot product accumulated
// in FP64), the two-loop recursion r = H g, and the elementwise steps of the
// iteration (projected step, weighted iterate averaging) and of the
// parameterisations u = c, 1/c, 1/c^2 of Sec. 3.3 with the chain rule for the
// gradient.  The FWI gradient itself comes from fwi_gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/fwi.h"

namespace {

constexpr int kBlocks = 592;      // 4 x 148 SMs
constexpr int kThreads = 256;

template <typename TA, typename TB>
__global__ void k_dot_partial(int64_t n, const TA* __restrict__ a, const TB* __restrict__ b,
                              double* __restrict__ part) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)b[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// sum of the block partials, in the same order in every block (deterministic)
__device__ __forceinline__ double sum_partials(const double* part, int np) {
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    tot = s;
  }
  __syncthreads();
  return tot;
}

// first loop: alpha_i = rho_i s_i'q (from the partials); q -= alpha_i y_i; alpha_i saved
__global__ void k_loop1(int64_t n, const double* __restrict__ part, int np, double rho, double* alpha_i,
                        double* __restrict__ q, const float* __restrict__ y) {
  const double a = rho * sum_partials(part, np);
  if (blockIdx.x == 0 && threadIdx.x == 0) *alpha_i = a;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    q[i] -= a * (double)y[i];
}

// second loop: beta = rho_i y_i'r (from the partials); r += (alpha_i - beta) s_i
__global__ void k_loop2(int64_t n, const double* __restrict__ part, int np, double rho,
                        const double* __restrict__ alpha_i, double* __restrict__ r, const float* __restrict__ s) {
  const double c = *alpha_i - rho * sum_partials(part, np);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] += c * (double)s[i];
}

// out = a x; also called in place (x == out): no __restrict__ on either pointer
__global__ void k_scale_copy(int64_t n, double a, const double* x, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * x[i];
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)x[i];
}

__global__ void k_step_project(int64_t n, double* __restrict__ u, const double* __restrict__ z, double nu,
                               double lo, double hi) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = fmin(fmax(u[i] + nu * z[i], lo), hi);
}

__global__ void k_accumulate_w(int64_t n, double* __restrict__ acc, const double* __restrict__ u, double w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc[i] += w * u[i];
}

// u -> c: kind 0 u = c, 1 u = 1/c (slowness), 2 u = 1/c^2 (squared slowness)
__global__ void k_param_to_speed(int64_t n, int kind, const double* __restrict__ u, float* __restrict__ c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = u[i];
    c[i] = (float)(kind == 0 ? v : (kind == 1 ? 1.0 / v : 1.0 / sqrt(v)));
  }
}

// dD/du = dD/dc dc/du: kind 1 dc/du = -c^2, kind 2 dc/du = -c^3 / 2
__global__ void k_grad_to_param(int64_t n, int kind, const float* __restrict__ c, const double* __restrict__ gc,
                                double* __restrict__ gu) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double cc = c[i];
    gu[i] = kind == 0 ? gc[i] : (kind == 1 ? -cc * cc * gc[i] : -0.5 * cc * cc * cc * gc[i]);
  }
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>(kBlocks, std::max<int64_t>(1, (n + kThreads - 1) / kThreads)); }

}  // namespace

struct fwi_lbfgs {
  int64_t n;
  int m;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  float* S = nullptr;       // [m][n]
  float* Y = nullptr;       // [m][n]
  double* part = nullptr;   // [kBlocks]
  double* alpha = nullptr;  // [m]
  std::vector<int> order;   // ring slots, oldest first
  std::vector<double> rho;  // per slot
  double gamma = 1.0;       // s'y / y'y of the newest pair
};

extern "C" {

fwi_status fwi_lbfgs_create(int64_t n, int32_t m, size_t* workspace_bytes, fwi_lbfgs** out) {
  if (!workspace_bytes || !out || n <= 0 || m <= 0 || m > 1024) return FWI_EINVAL;
  fwi_lbfgs* L = new (std::nothrow) fwi_lbfgs;
  if (!L) return FWI_ENOMEM;
  L->n = n;
  L->m = m;
  L->rho.assign(m, 0.0);
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  L->ws_bytes = up((size_t)m * n * 4) * 2 + up(kBlocks * 8) + up((size_t)m * 8);
  *workspace_bytes = L->ws_bytes;
  *out = L;
  return FWI_OK;
}

fwi_status fwi_lbfgs_bind_workspace(fwi_lbfgs* L, void* dev_ptr, size_t bytes) {
  if (!L || !dev_ptr || ((uintptr_t)dev_ptr & 255) || bytes < L->ws_bytes) return FWI_EINVAL;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  char* p = static_cast<char*>(dev_ptr);
  L->ws = p;
  L->S = reinterpret_cast<float*>(p);
  p += up((size_t)L->m * L->n * 4);
  L->Y = reinterpret_cast<float*>(p);
  p += up((size_t)L->m * L->n * 4);
  L->part = reinterpret_cast<double*>(p);
  p += up(kBlocks * 8);
  L->alpha = reinterpret_cast<double*>(p);
  L->order.clear();
  L->gamma = 1.0;
  return FWI_OK;
}

fwi_status fwi_lbfgs_push(fwi_lbfgs* L, const double* s, const double* y, void* stream, int32_t* stored) {
  if (!L || !L->ws || !s || !y) return FWI_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = blocks_for(L->n);
  double dots[2];
  k_dot_partial<double, double><<<nb, kThreads, 0, st>>>(L->n, s, y, L->part);
  std::vector<double> hp(nb);
  if (cudaMemcpyAsync(hp.data(), L->part, nb * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return FWI_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FWI_ECUDA;
  dots[0] = 0.0;
  for (double v : hp) dots[0] += v;
  k_dot_partial<double, double><<<nb, kThreads, 0, st>>>(L->n, y, y, L->part);
  if (cudaMemcpyAsync(hp.data(), L->part, nb * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return FWI_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FWI_ECUDA;
  dots[1] = 0.0;
  for (double v : hp) dots[1] += v;
  const bool keep = dots[0] > 0.0;   // positive curvature only (keeps H positive definite)
  if (stored) *stored = keep ? 1 : 0;
  if (!keep) return FWI_OK;
  int slot;
  if ((int)L->order.size() < L->m) {
    slot = (int)L->order.size();
  } else {
    slot = L->order.front();
    L->order.erase(L->order.begin());
  }
  L->order.push_back(slot);
  L->rho[slot] = 1.0 / dots[0];
  L->gamma = dots[0] / dots[1];
  k_to_f32<<<nb, kThreads, 0, st>>>(L->n, s, L->S + (size_t)slot * L->n);
  k_to_f32<<<nb, kThreads, 0, st>>>(L->n, y, L->Y + (size_t)slot * L->n);
  return cudaGetLastError() == cudaSuccess ? FWI_OK : FWI_ECUDA;
}

fwi_status fwi_lbfgs_apply(fwi_lbfgs* L, const double* g, double h0, double* out, void* stream) {
  if (!L || !L->ws || !g || !out) return FWI_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = blocks_for(L->n);
  const int64_t n = L->n;
  k_scale_copy<<<nb, kThreads, 0, st>>>(n, 1.0, g, out);          // q = g
  for (int k = (int)L->order.size() - 1; k >= 0; --k) {
    const int sl = L->order[k];
    k_dot_partial<float, double><<<nb, kThreads, 0, st>>>(n, L->S + (size_t)sl * n, out, L->part);
    k_loop1<<<nb, kThreads, 0, st>>>(n, L->part, nb, L->rho[sl], L->alpha + sl, out, L->Y + (size_t)sl * n);
  }
  const double scale = h0 > 0.0 ? h0 : (L->order.empty() ? 1.0 : L->gamma);
  k_scale_copy<<<nb, kThreads, 0, st>>>(n, scale, out, out);     // r = H_0 q
  for (int k = 0; k < (int)L->order.size(); ++k) {
    const int sl = L->order[k];
    k_dot_partial<float, double><<<nb, kThreads, 0, st>>>(n, L->Y + (size_t)sl * n, out, L->part);
    k_loop2<<<nb, kThreads, 0, st>>>(n, L->part, nb, L->rho[sl], L->alpha + sl, out, L->S + (size_t)sl * n);
  }
  return cudaGetLastError() == cudaSuccess ? FWI_OK : FWI_ECUDA;
}

int32_t fwi_lbfgs_size(const fwi_lbfgs* L) { return L ? (int32_t)L->order.size() : 0; }

fwi_status fwi_lbfgs_destroy(fwi_lbfgs* L) {
  delete L;
  return FWI_OK;
}

fwi_status fwi_vec_step_project(int64_t n, double* u, const double* z, double nu, double u_min, double u_max,
                                void* stream) {
  if (n <= 0 || !u || !z || !(u_min <= u_max)) return FWI_EINVAL;
  k_step_project<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(n, u, z, nu, u_min, u_max);
  return cudaGetLastError() == cudaSuccess ? FWI_OK : FWI_ECUDA;
}

fwi_status fwi_vec_accumulate(int64_t n, double* acc, const double* u, double w, void* stream) {
  if (n <= 0 || !acc || !u) return FWI_EINVAL;
  k_accumulate_w<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(n, acc, u, w);
  return cudaGetLastError() == cudaSuccess ? FWI_OK : FWI_ECUDA;
}

fwi_status fwi_param_to_speed(int64_t n, int32_t kind, const double* u, float* c, void* stream) {
  if (n <= 0 || !u || !c || kind < 0 || kind > 2) return FWI_EINVAL;
  k_param_to_speed<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(n, kind, u, c);
  return cudaGetLastError() == cudaSuccess ? FWI_OK : FWI_ECUDA;
}

fwi_status fwi_grad_to_param(int64_t n, int32_t kind, const float* c, const double* gc, double* gu,
                             void* stream) {
  if (n <= 0 || !c || !gc || !gu || kind < 0 || kind > 2) return FWI_EINVAL;
  k_grad_to_param<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(n, kind, c, gc, gu);
  return cudaGetLastError() == cudaSuccess ? FWI_OK : FWI_ECUDA;
}

}  // extern "C"
