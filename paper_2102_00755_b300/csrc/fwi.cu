// C ABI of the B300 time-domain FWI hot path: plan, workspace, forward and
// gradient calls (Alg. 1, App. B).  See include/fwi.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/fwi.h"
#include "kernels.cuh"
#include "launch.cuh"
#include "plane2.cuh"
#include "split2.cuh"

using namespace fwi;

namespace {

constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------ small kernels
__global__ void k_prepare_c(const float* __restrict__ c, float* __restrict__ c2, int64_t n,
                            float c_ref, int* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = c[i];
    if (!(v > 0.f && v <= c_ref)) *bad = 1;
    c2[i] = v * v;
  }
}

// per-call coefficients at the sparse voxels (FP64 arithmetic, FP32 result)
__global__ void k_prepare_coefs(const float* __restrict__ c, double dt, double dx,
                                const int* us_vox, int n_us, float* us_coef,
                                const int* ur_vox, int n_ur, float* ur_coef,
                                const int* gam_idx, int n_gamma, float* coefG,
                                const int* lay_idx, int n_layer, float* inv3c2) {
  const int tot = n_us + n_ur + n_gamma + n_layer;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
    if (i < n_us) {
      us_coef[i] = (float)(2.0 * dt / (3.0 * dx * (double)c[us_vox[i]]));
    } else if (i < n_us + n_ur) {
      const int u = i - n_us;
      ur_coef[u] = (float)(2.0 * dt / (3.0 * dx * (double)c[ur_vox[u]]));
    } else if (i < n_us + n_ur + n_gamma) {
      const int j = i - n_us - n_ur;
      const double cv = c[gam_idx[j]];
      coefG[j] = (float)(2.0 / (dt * cv * cv * cv));
    } else {
      const int j = i - n_us - n_ur - n_gamma;
      const double cv = c[lay_idx[j]];
      inv3c2[j] = (float)(1.0 / (3.0 * cv * cv));
    }
  }
}

// amp[k][n][u] = coef_u * (sum_{i at u} w[k][i]) * s(t_n): the encoded source (Sec. 3.2)
// delay (optional, [K][n_src] whole time steps, Eq. 13): emitter i of super-shot k
// emits s(t_n - delay dt), zero outside the wavelet's samples
// coef: [models][n_us], shot k uses model k when per_model, else model 0
__global__ void k_source_amp(const float* __restrict__ w, int n_src, const float* __restrict__ coef0,
                             const int* mptr, const int* mem, int n_us, const float* __restrict__ wav,
                             int nt, const int* __restrict__ delay, float* __restrict__ amp, int per_model) {
  const int n = blockIdx.x;
  const int k = blockIdx.y;
  const float s = wav[n];
  const float* coef = coef0 + (per_model ? (size_t)k * n_us : 0);
  for (int u = threadIdx.x; u < n_us; u += blockDim.x) {
    float ws = 0.f;
    for (int e = mptr[u]; e < mptr[u + 1]; ++e) {
      const size_t ki = (size_t)k * n_src + mem[e];
      if (delay) {
        const int m = n - delay[ki];
        if (m >= 0 && m < nt) ws += w[ki] * wav[m];
      } else {
        ws += w[ki];
      }
    }
    amp[((size_t)k * nt + n) * n_us + u] = coef[u] * (delay ? ws : ws * s);
  }
}

// f_hat[k][n][r] = sum_i w[k][i] f_i[n][r] (Sec. 3.2), FP64 accumulation
__global__ void k_encode(const float* __restrict__ raw, const float* __restrict__ w, int n_src,
                         int K, int64_t per_src, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per_src;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc[kMaxSims];
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int i = 0; i < n_src; ++i) {
      const double v = raw[(size_t)i * per_src + e];
      for (int k = 0; k < K; ++k) acc[k] += (double)w[(size_t)k * n_src + i] * v;
    }
    for (int k = 0; k < K; ++k) out[(size_t)k * per_src + e] = (float)acc[k];
  }
}

// f_hat[k][n][r] = sum_i w[k][i] f_i[n - d[k][i]][r] (Eq. 13, whole-step delays), zero
// where n - d falls outside the nt_obs recorded samples; FP64 accumulation
__global__ void k_encode_delayed(const float* __restrict__ raw, const float* __restrict__ w,
                                 const int* __restrict__ delay, int n_src, int K, int nt_obs, int nt,
                                 int n_rec, float* __restrict__ out) {
  const int64_t tot = (int64_t)nt * n_rec;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(e / n_rec), r = (int)(e - (int64_t)n * n_rec);
    double acc[kMaxSims];
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int i = 0; i < n_src; ++i) {
      for (int k = 0; k < K; ++k) {
        const int m = n - delay[(size_t)k * n_src + i];
        if (m >= 0 && m < nt_obs)
          acc[k] += (double)w[(size_t)k * n_src + i] * (double)raw[((size_t)i * nt_obs + m) * n_rec + r];
      }
    }
    for (int k = 0; k < K; ++k) out[(size_t)k * tot + e] = (float)acc[k];
  }
}

// q^n = f^(Nt-n) - f_obs^(Nt-n); Q^n = sum_{m<=n} q^m (FP64 running sum, FP32 store);
// block partials of D = 0.5 sum q^2 (Alg. 1)
__global__ void k_misfit(const float* __restrict__ f, const float* __restrict__ fo, int nt, int n_rec,
                         float* __restrict__ qf, double* __restrict__ dpart) {
  const int k = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (r < n_rec) {
    const float* fk = f + (size_t)k * nt * n_rec;
    const float* ok = fo + (size_t)k * nt * n_rec;
    float* qk = qf + (size_t)k * nt * n_rec;
    double acc = 0.0;
    for (int n = 0; n < nt; ++n) {
      const size_t src = (size_t)(nt - 1 - n) * n_rec + r;
      const double q = (double)fk[src] - (double)ok[src];
      acc += q;
      d += 0.5 * q * q;
      qk[(size_t)n * n_rec + r] = (float)acc;
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = d;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) dpart[(size_t)k * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_misfit_final(const double* dpart, int nblk, int K, double* misfit) {
  const int k = threadIdx.x;
  if (k < K) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += dpart[(size_t)k * nblk + b];
    misfit[k] = s;
  }
}

// grad_k(Gamma) += 2/(dt c0^3) (p+ - 2 p0 + p-) p_adj  (Alg. 1; second difference, product
// and accumulator in FP64).  The two-step mass kernels do the same inside the next
// iteration's adjoint launch; this kernel serves the other kernel families and the
// last iteration.
__global__ void k_accumulate(const float* __restrict__ ring, const float* __restrict__ pa,
                             const float* __restrict__ coefG0, int n_gamma, int sa, int sb, int sc,
                             double* __restrict__ acc, const int* bad, int k0, int per_model) {
  if (*bad) return;
  const int k = k0 + blockIdx.y;
  const float* coefG = coefG0 + (per_model ? (size_t)k * n_gamma : 0);
  const float* rk = ring + (size_t)k * kRing * n_gamma;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_gamma; j += gridDim.x * blockDim.x) {
    const double d2 = (double)rk[(size_t)sa * n_gamma + j] - 2.0 * (double)rk[(size_t)sb * n_gamma + j] +
                      (double)rk[(size_t)sc * n_gamma + j];
    acc[(size_t)k * n_gamma + j] += (double)coefG[j] * d2 * (double)pa[(size_t)k * n_gamma + j];
  }
}

// grad = scale * mean_k acc_k on Gamma; with each_shot, grad[k] = scale * acc_k (one
// gradient per super-shot, [K][nvox])
__global__ void k_grad_final(const double* __restrict__ acc, const int* __restrict__ gam_idx,
                             int n_gamma, int K, double scale, double* __restrict__ grad, int each_shot,
                             int64_t nvox) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_gamma; j += gridDim.x * blockDim.x) {
    if (each_shot) {
      for (int k = 0; k < K; ++k) grad[(size_t)k * nvox + gam_idx[j]] = scale * acc[(size_t)k * n_gamma + j];
    } else {
      double s = 0.0;
      for (int k = 0; k < K; ++k) s += acc[(size_t)k * n_gamma + j];
      grad[gam_idx[j]] = scale * s / K;
    }
  }
}

// c0 of the TR box (Sec. 3.1): cb[x + nxb (y + nyb z)] = c[(x0 + x) + nx ((y0 + y) + ny (z0 + z))]
__global__ void k_crop(const float* __restrict__ c, int nx, int ny, int x0, int y0, int z0, int nxb, int nyb,
                       int nzb, float* __restrict__ cb) {
  const int64_t n = (int64_t)nxb * nyb * nzb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nxb);
    const int64_t r = i / nxb;
    const int y = (int)(r % nyb), z = (int)(r / nyb);
    cb[i] = c[((int64_t)(z + z0) * ny + (y + y0)) * nx + (x + x0)];
  }
}

// ------------------------------------------------------------ host helpers
// Radix schedule of one axis: order 0 = 8, 4, 2, 3, 5; 1 = 4, 2, 3, 5 (no 8);
// 2 = the order-0 passes reversed (largest radix last).
bool factor235(int n, AxisPlan* A, int order = 0) {
  int m = n, ns = 0;
  int r[kMaxStages + 8];
  if (order != 1)
    while (m % 8 == 0) { r[ns++] = 8; m /= 8; }
  while (m % 4 == 0) { r[ns++] = 4; m /= 4; }
  while (m % 2 == 0) { r[ns++] = 2; m /= 2; }
  while (m % 3 == 0) { r[ns++] = 3; m /= 3; }
  while (m % 5 == 0) { r[ns++] = 5; m /= 5; }
  if (m != 1 || ns > kMaxStages) return false;
  for (int s = 0; s < ns; ++s) A->radix[s] = order == 2 ? r[ns - 1 - s] : r[s];
  A->n = n;
  A->nstages = ns;
  return true;
}

double wavenumber(int j, int n, double dx) {
  const int m = (j < (n + 1) / 2) ? j : j - n;
  return 2.0 * kPi * m / (n * dx);
}

// PML multiplier (reading of App. B): sigma = alpha c_ref/dx (d/P)^4, Lambda = exp(-sigma dt/2)
double pml_value(int i, int n, int P, double alpha, double c_ref, double dx, double dt, bool stag) {
  if (P <= 0 || alpha == 0.0) return 1.0;
  const double x = i + (stag ? 0.5 : 0.0);
  double d = 0.0;
  if (x < P) d = P - x;
  else if (x > n - 1 - P) d = x - (n - 1 - P);
  const double sigma = alpha * (c_ref / dx) * std::pow(d / P, 4.0);
  return std::exp(-sigma * dt / 2.0);
}

// Sparse voxel lists grouped by pair line: key = z * npair + y / 2.  `pf` is the
// float offset of the voxel in the plane buffer seen as pair lines of 2 hx complex
// values: 4 hx (y/2) + 2x + (y & 1).
struct Csr {
  std::vector<int> ptr;   // [nz*npair + 1]
  std::vector<int> vox;   // linear voxel of each entry
  std::vector<int> pf;    // offset inside the pair line
  std::vector<int> mptr;  // members per entry (unique lists)
  std::vector<int> mem;   // member ids
};

struct KeyGeom {
  int nx, ny, nz, npair, hx;
  int key(int v) const {
    const int plane = nx * ny;
    const int z = v / plane, r = v - z * plane, y = r / nx;
    return z * npair + y / 2;
  }
  int pf(int v) const {
    const int r = v % (nx * ny), y = r / nx, x = r - y * nx;
    return 4 * hx * (y / 2) + 2 * x + (y & 1);
  }
};

void finish_ptr(std::vector<int>& ptr) {
  for (size_t k = 1; k < ptr.size(); ++k) ptr[k] += ptr[k - 1];
}

// unique voxels in increasing order, with the ids that map to each
Csr build_unique(const int32_t* idx, int n, const KeyGeom& g) {
  std::map<int, std::vector<int>> by;
  for (int i = 0; i < n; ++i) by[idx[i]].push_back(i);
  Csr c;
  c.ptr.assign((size_t)g.nz * g.npair + 1, 0);
  c.mptr.push_back(0);
  for (auto& kv : by) {
    c.ptr[g.key(kv.first) + 1]++;
    c.vox.push_back(kv.first);
    c.pf.push_back(g.pf(kv.first));
    for (int m : kv.second) c.mem.push_back(m);
    c.mptr.push_back((int)c.mem.size());
  }
  finish_ptr(c.ptr);
  return c;
}

// all entries of an (index, id) list sorted by index
Csr build_sorted(const std::vector<std::pair<int, int>>& e, const KeyGeom& g) {
  Csr c;
  c.ptr.assign((size_t)g.nz * g.npair + 1, 0);
  for (auto& v : e) {
    c.ptr[g.key(v.first) + 1]++;
    c.vox.push_back(v.first);
    c.pf.push_back(g.pf(v.first));
    c.mem.push_back(v.second);
  }
  finish_ptr(c.ptr);
  return c;
}

struct Layout {
  size_t total = 0;
  size_t add(size_t bytes) {
    const size_t o = total;
    total += (bytes + 255) & ~size_t(255);
    return o;
  }
};

}  // namespace

// ------------------------------------------------------------ the plan
struct fwi_plan {
  fwi_problem prob;     // scalars (pointers cleared)
  int K;                // max shots
  int hx, npair, mspec, plane;
  int64_t nvox;
  AxisPlan ax, ay, az;
  size_t smem_plane, smem_mass, smem_zmom, smem_zmass;
  int epl;   // values staged per lane in the runtime warp FFT passes (8 or 16)
  int fxy;   // specialised plane side (0: runtime schedules)
  int p2;    // plane side of the two-step register-transform plane kernels (0: not used)
  size_t smem_p2;
  int z2;    // nz of the two-step register-transform z pass (0: not used)
  size_t smem_z2[2];
  int s2;    // plane side of the two-step split-plane kernels (0: not used)
  size_t smem_y2, smem_x2;
  int fz;    // specialised z length (0: runtime schedules)
  int tz;    // z-pass tile width (columns)
  int split; // XY work split into column and row-pair passes (large planes)
  size_t smem_ypass3, smem_ypass1, smem_xmom, smem_xmass;
  fwi_schedule sched;
  // host tables
  std::vector<float2> tw, ap[3], am[3];
  std::vector<float> kx2, ky2, kz2, lam[3], lams[3], wavelet;
  Csr us, ur, rr, lay, gam;
  int n_us, n_ur;
  // workspace offsets
  Layout L;
  size_t o_tw, o_kx2, o_ky2, o_kz2, o_ap[3], o_am[3], o_lam[3], o_lams[3];
  size_t o_us_ptr, o_us_pf, o_us_vox, o_us_mptr, o_us_mem;
  size_t o_ur_ptr, o_ur_pf, o_ur_vox, o_ur_mptr, o_ur_mem;
  size_t o_rr_ptr, o_rr_pf, o_rr_col, o_lay_ptr, o_lay_vox, o_lay_pf, o_gam_ptr, o_gam_vox, o_gam_pf;
  size_t o_wav;
  size_t o_bad, o_c2, o_us_coef, o_ur_coef, o_coefG, o_inv3c2, o_amp, o_traces, o_obs, o_qf,
      o_ghist, o_ring, o_pa, o_acc, o_dpart;
  size_t o_sims, sim_bytes, sim_field, sim_spec;
  int nblk_misfit;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  // bumped by every workspace binding and schedule change: a batch graph captured
  // before the change holds stale pointers or launch shapes and must be re-captured
  uint64_t generation = 0;
  // TR re-simulation on a box enclosing Gamma (Sec. 3.1): a plan of the box's grid that
  // runs only TR simulations, with its workspace and the cropped sound speed inside
  // this plan's workspace.  tr_only marks such a box plan.
  fwi_plan* tr = nullptr;
  bool tr_only = false;
  int models = 1;       // sound-speed models: K when each super-shot has its own, else 1
  int tr_origin[3] = {0, 0, 0};
  size_t o_trc = 0, o_trws = 0;
  cudaStream_t last = nullptr;
  bool used = false;
  // extra streams of the stream-group form, with the fork event and one join event each
  static constexpr int kMaxGroups = 4;
  cudaStream_t side[kMaxGroups - 1] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kMaxGroups - 1] = {};
  // profiling hook
  int prof_mask = 0;
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;   // pairs
  std::vector<int> prof_kind;         // kernel of each pair
  int prof_used = 0;
  int64_t prof_sims[4] = {0, 0, 0, 0};
};

namespace {

template <typename T>
T* at(fwi_plan* p, size_t off) { return reinterpret_cast<T*>(p->ws + off); }

void sim_ptrs(fwi_plan* p, int s, SimPtrs* out, int role, int shot) {
  char* base = p->ws + p->o_sims + (size_t)s * p->sim_bytes;
  for (int c = 0; c < 3; ++c) {
    out->v[c] = reinterpret_cast<float*>(base + c * p->sim_field);
    out->rho[c] = reinterpret_cast<float*>(base + (3 + c) * p->sim_field);
    out->spec[c] = reinterpret_cast<float2*>(base + 6 * p->sim_field + c * p->sim_spec);
  }
  out->role = role;
  out->shot = shot;
  out->model = p->models > 1 ? shot : 0;
}

void base_params(fwi_plan* p, StepParams* P) {
  std::memset(P, 0, sizeof(*P));
  const fwi_problem& q = p->prob;
  P->nx = q.nx; P->ny = q.ny; P->nz = q.nz;
  P->hx = p->hx; P->npair = p->npair;
  P->nvox = p->nvox; P->plane = p->plane; P->mspec = p->mspec; P->nt = q.nt;
  P->n_rec = q.n_rec; P->n_layer = q.n_layer; P->n_gamma = q.n_gamma;
  P->n_us = p->n_us; P->n_ur = p->n_ur;
  P->ax = p->ax; P->ay = p->ay; P->az = p->az;
  P->tw = at<float2>(p, p->o_tw);
  P->kx2 = at<float>(p, p->o_kx2); P->ky2 = at<float>(p, p->o_ky2); P->kz2 = at<float>(p, p->o_kz2);
  for (int c = 0; c < 3; ++c) {
    P->ap[c] = at<float2>(p, p->o_ap[c]);
    P->am[c] = at<float2>(p, p->o_am[c]);
    P->lam[c] = at<float>(p, p->o_lam[c]);
    P->lams[c] = at<float>(p, p->o_lams[c]);
  }
  P->half_cdt = (float)(q.c_ref * q.dt / 2.0);
  {
    // largest argument c_ref dt |k| / 2 of the sinc in kappa (Eq. 18): |k_xi| <= pi / dx
    const double amax = q.c_ref * q.dt / 2.0 * std::sqrt(3.0) * M_PI / q.dx;
    P->kappa_series = amax <= 3.1 ? 1 : 0;
  }
  P->inv_n = (float)(1.0 / (double)p->nvox);
  P->dt_over_rho0 = (float)(q.dt / q.rho0);
  P->dt_rho0 = (float)(q.dt * q.rho0);
  P->c2 = at<float>(p, p->o_c2);
  P->bad = at<int>(p, p->o_bad);
  P->us_ptr = at<int>(p, p->o_us_ptr); P->us_vox = at<int>(p, p->o_us_vox);
  P->us_pf = at<int>(p, p->o_us_pf);
  P->amp_src = at<float>(p, p->o_amp);
  P->ur_ptr = at<int>(p, p->o_ur_ptr); P->ur_vox = at<int>(p, p->o_ur_vox);
  P->ur_pf = at<int>(p, p->o_ur_pf);
  P->ur_mptr = at<int>(p, p->o_ur_mptr); P->ur_mem = at<int>(p, p->o_ur_mem);
  P->ur_coef = at<float>(p, p->o_ur_coef);
  P->qf = at<float>(p, p->o_qf);
  P->rr_ptr = at<int>(p, p->o_rr_ptr); P->rr_pf = at<int>(p, p->o_rr_pf);
  P->rr_col = at<int>(p, p->o_rr_col);
  P->traces = at<float>(p, p->o_traces);
  P->lay_ptr = at<int>(p, p->o_lay_ptr); P->lay_vox = at<int>(p, p->o_lay_vox);
  P->lay_pf = at<int>(p, p->o_lay_pf);
  P->ghist = at<float>(p, p->o_ghist);
  P->inv3c2 = at<float>(p, p->o_inv3c2);
  P->gam_ptr = at<int>(p, p->o_gam_ptr); P->gam_pf = at<int>(p, p->o_gam_pf);
  P->pa = at<float>(p, p->o_pa);
  P->ring = at<float>(p, p->o_ring);
  P->acc = at<double>(p, p->o_acc);
  P->coefG = at<float>(p, p->o_coefG);
}

thread_local char g_last_cuda_error[256] = "";

fwi_status cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s (%s)", what, cudaGetErrorName(e),
                cudaGetErrorString(e));
  return FWI_ECUDA;
}

#define CK(x)                                       \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

// after a kernel launch: report a launch failure with the launch site's name
#define LAUNCHED(label)                                        \
  do {                                                         \
    cudaError_t e_ = cudaGetLastError();                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, "launch " label); \
  } while (0)

// Kernel instantiations: specialised transforms for square planes of side FXY in
// {32, 64, 96, 128, 160} and z lengths FZ in {32, 48, 64, 80, 96, 128}; any other
// 2-3-5-smooth size (up to 512) takes the runtime radix schedule (F = 0) with 8
// (axes <= 256) or 16 values staged per lane.
#define PLANE_DISPATCH(p, CALL)                                         \
  switch ((p)->fxy) {                                                   \
    case 32: { constexpr int E = 8, F = 32; CALL; } break;              \
    case 64: { constexpr int E = 8, F = 64; CALL; } break;              \
    case 96: { constexpr int E = 8, F = 96; CALL; } break;              \
    case 128: { constexpr int E = 8, F = 128; CALL; } break;            \
    case 160: { constexpr int E = 8, F = 160; CALL; } break;            \
    default:                                                            \
      if ((p)->epl == 8) { constexpr int E = 8, F = 0; CALL; }          \
      else { constexpr int E = 16, F = 0; CALL; }                       \
  }
// Two-step register-transform plane kernels: square planes of these sides.
#define P2_DISPATCH(p, CALL)                                            \
  switch ((p)->p2) {                                                    \
    case 32: { constexpr int N = 32; CALL; } break;                     \
    case 64: { constexpr int N = 64; CALL; } break;                     \
    case 96: { constexpr int N = 96; CALL; } break;                     \
    case 128: { constexpr int N = 128; CALL; } break;                   \
    case 135: { constexpr int N = 135; CALL; } break;                   \
    case 160: { constexpr int N = 160; CALL; } break;                   \
    default: break;                                                     \
  }
#define Z2_DISPATCH_T(p, TZ, CALL)                                      \
  switch ((p)->z2) {                                                    \
    case 32: { constexpr int NZ = 32; CALL; } break;                    \
    case 48: { constexpr int NZ = 48; CALL; } break;                    \
    case 64: { constexpr int NZ = 64; CALL; } break;                    \
    case 80: { constexpr int NZ = 80; CALL; } break;                    \
    case 96: { constexpr int NZ = 96; CALL; } break;                    \
    case 128: { constexpr int NZ = 128; CALL; } break;                  \
    case 135: { constexpr int NZ = 135; CALL; } break;                  \
    case 256: { constexpr int NZ = 256; CALL; } break;                  \
    default: break;                                                     \
  }
#define S2_DISPATCH(p, CALL)                                            \
  switch ((p)->s2) {                                                    \
    case 243: { constexpr int N = 243; CALL; } break;                   \
    case 256: { constexpr int N = 256; CALL; } break;                   \
    case 480: { constexpr int N = 480; CALL; } break;                   \
    default: break;                                                     \
  }
#define Z2_DISPATCH(p, CALL)                                            \
  if ((p)->tz == 32) { constexpr int TZ = 32; Z2_DISPATCH_T(p, TZ, CALL) } \
  else { constexpr int TZ = 16; Z2_DISPATCH_T(p, TZ, CALL) }
#define Z_DISPATCH_T(p, TZ, CALL)                                       \
  switch ((p)->fz) {                                                    \
    case 32: { constexpr int E = 8, FZ = 32; CALL; } break;             \
    case 48: { constexpr int E = 8, FZ = 48; CALL; } break;             \
    case 64: { constexpr int E = 8, FZ = 64; CALL; } break;             \
    case 80: { constexpr int E = 8, FZ = 80; CALL; } break;             \
    case 96: { constexpr int E = 8, FZ = 96; CALL; } break;             \
    case 128: { constexpr int E = 8, FZ = 128; CALL; } break;           \
    default:                                                            \
      if ((p)->epl == 8) { constexpr int E = 8, FZ = 0; CALL; }         \
      else { constexpr int E = 16, FZ = 0; CALL; }                      \
  }
#define Z_DISPATCH(p, CALL)                                             \
  if ((p)->tz == 32) { constexpr int TZ = 32; Z_DISPATCH_T(p, TZ, CALL) } \
  else { constexpr int TZ = 16; Z_DISPATCH_T(p, TZ, CALL) }

// The dynamic shared-memory cap is a per-kernel (not per-plan) attribute shared by
// every plan that launches the same instantiation, so it is set to the device's
// opt-in maximum, never to one plan's size; each launch still requests only what
// its plan needs, which is what sets occupancy.
int smem_optin_max() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v > 0 ? v : 48 * 1024;
}

void set_attrs(fwi_plan* p) {
  const int cap = smem_optin_max();
  if (p->epl == 8) attrs_split<8>(cap);
  else attrs_split<16>(cap);
  PLANE_DISPATCH(p, (attrs_plane<E, F>(cap)));
  P2_DISPATCH(p, (attrs_plane2<N>(cap)));
  Z2_DISPATCH_T(p, 0, (attrs_zpass2<NZ>(cap)));
  S2_DISPATCH(p, (attrs_split2<N>(cap)));
  Z_DISPATCH_T(p, 0, (attrs_zpass<E, FZ>(cap)));
  // Touch every small kernel too, so that modules are loaded before any stream
  // capture of a call (a first launch inside a capture may not load them).
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_prepare_c);
  cudaFuncGetAttributes(&a, k_prepare_coefs);
  cudaFuncGetAttributes(&a, k_source_amp);
  cudaFuncGetAttributes(&a, k_encode);
  cudaFuncGetAttributes(&a, k_misfit);
  cudaFuncGetAttributes(&a, k_misfit_final);
  cudaFuncGetAttributes(&a, k_accumulate);
  cudaFuncGetAttributes(&a, k_grad_final);
  cudaFuncGetAttributes(&a, k_crop);
}

void prof_begin(fwi_plan* p, int kernel, cudaStream_t st, int nsims, int* slot) {
  *slot = -1;
  if (!p->prof_on || !((p->prof_mask >> kernel) & 1)) return;
  // an event recorded into a stream capture becomes a graph dependency, not a
  // timestamp: launches issued while the stream is being captured are not timed
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
  if (2 * (p->prof_used + 1) > (int)p->prof_ev.size()) return;
  *slot = p->prof_used++;
  p->prof_kind[*slot] = kernel;
  p->prof_sims[kernel] += nsims;
  cudaEventRecord(p->prof_ev[2 * *slot], st);
}
void prof_end(fwi_plan* p, cudaStream_t st, int slot) {
  if (slot >= 0) cudaEventRecord(p->prof_ev[2 * slot + 1], st);
}

// One time step for a batch of simulations (four launches).
template <int EL>
fwi_status launch_step_split(fwi_plan* p, const StepParams& P, cudaStream_t st) {
  const dim3 gz((p->mspec + p->tz - 1) / p->tz, P.nsims);
  const dim3 gy((p->hx + kTY - 1) / kTY, p->prob.nz, P.nsims);
  const int g1 = std::max(1, 16 * EL / p->hx), g2 = std::max(1, 8 * EL / p->hx);
  const int warps = kTpbPlane / 32;
  const dim3 gx1((p->npair + warps * g1 - 1) / (warps * g1), p->prob.nz, P.nsims);
  const dim3 gx2((p->npair + warps * g2 - 1) / (warps * g2), p->prob.nz, P.nsims);
  const int ty2 = ty2_for(p->s2 > 0 ? p->s2 : 1);
  const dim3 gy2((p->hx + ty2 - 1) / ty2, p->prob.nz, P.nsims);
  const int npc2 = npc2_for(p->s2);
  const dim3 gx2b((p->npair + npc2 - 1) / npc2, p->prob.nz, P.nsims);
  int slot;
  prof_begin(p, FWI_K_ZPASS_MOMENTUM, st, P.nsims, &slot);
  if (p->z2) {
    Z2_DISPATCH(p, (launch_zpass2<NZ>(0, TZ, gz, p->smem_z2[0], st, P)));
    LAUNCHED("k_zpass2<momentum>");
  } else {
    Z_DISPATCH(p, (launch_zpass<E, FZ>(0, TZ, gz, p->smem_zmom, st, P)));
    LAUNCHED("k_zpass<momentum>");
  }
  prof_end(p, st, slot);
  prof_begin(p, FWI_K_PLANE_MOMENTUM, st, P.nsims, &slot);
  if (p->s2) {
    S2_DISPATCH(p, (launch_split2<N>(Y_INV_MOM, gy2, p->smem_y2, st, P)));
    LAUNCHED("k_ypass2<inverse, momentum>");
    S2_DISPATCH(p, (launch_split2<N>(4, gx2b, p->smem_x2, st, P)));
    LAUNCHED("k_xpass2_mom");
    S2_DISPATCH(p, (launch_split2<N>(Y_FWD3, gy2, p->smem_y2, st, P)));
    LAUNCHED("k_ypass2<forward x3>");
  } else {
    launch_split<EL>(Y_INV_MOM, gy, p->smem_ypass3, st, P);
    LAUNCHED("k_ypass<inverse, momentum>");
    launch_split<EL>(4, gx1, p->smem_xmom, st, P);
    LAUNCHED("k_xpass_mom");
    launch_split<EL>(Y_FWD3, gy, p->smem_ypass3, st, P);
    LAUNCHED("k_ypass<forward x3>");
  }
  prof_end(p, st, slot);
  prof_begin(p, FWI_K_ZPASS_MASS, st, P.nsims, &slot);
  if (p->z2) {
    Z2_DISPATCH(p, (launch_zpass2<NZ>(1, TZ, gz, p->smem_z2[1], st, P)));
    LAUNCHED("k_zpass2<mass>");
  } else {
    Z_DISPATCH(p, (launch_zpass<E, FZ>(1, TZ, gz, p->smem_zmass, st, P)));
    LAUNCHED("k_zpass<mass>");
  }
  prof_end(p, st, slot);
  prof_begin(p, FWI_K_PLANE_MASS, st, P.nsims, &slot);
  if (p->s2) {
    S2_DISPATCH(p, (launch_split2<N>(Y_INV_MASS, gy2, p->smem_y2, st, P)));
    LAUNCHED("k_ypass2<inverse, mass>");
    S2_DISPATCH(p, (launch_split2<N>(5, gx2b, p->smem_x2, st, P)));
    LAUNCHED("k_xpass2_mass");
    S2_DISPATCH(p, (launch_split2<N>(Y_FWD1, gy2, p->smem_y2, st, P)));
    LAUNCHED("k_ypass2<forward x1>");
  } else {
    launch_split<EL>(Y_INV_MASS, gy, p->smem_ypass3, st, P);
    LAUNCHED("k_ypass<inverse, mass>");
    launch_split<EL>(5, gx2, p->smem_xmass, st, P);
    LAUNCHED("k_xpass_mass");
    launch_split<EL>(Y_FWD1, gy, p->smem_ypass1, st, P);
    LAUNCHED("k_ypass<forward x1>");
  }
  prof_end(p, st, slot);
  return FWI_OK;
}

fwi_status launch_step_batch(fwi_plan* p, const StepParams& P, cudaStream_t st) {
  if (p->split) return p->epl == 8 ? launch_step_split<8>(p, P, st) : launch_step_split<16>(p, P, st);
  const dim3 gz((p->mspec + p->tz - 1) / p->tz, P.nsims);
  const dim3 gp(p->prob.nz, P.nsims);
  int slot;
  prof_begin(p, FWI_K_ZPASS_MOMENTUM, st, P.nsims, &slot);
  if (p->z2) {
    Z2_DISPATCH(p, (launch_zpass2<NZ>(0, TZ, gz, p->smem_z2[0], st, P)));
    LAUNCHED("k_zpass2<momentum>");
  } else {
    Z_DISPATCH(p, (launch_zpass<E, FZ>(0, TZ, gz, p->smem_zmom, st, P)));
    LAUNCHED("k_zpass<momentum>");
  }
  prof_end(p, st, slot);
  prof_begin(p, FWI_K_PLANE_MOMENTUM, st, P.nsims, &slot);
  if (p->p2) {
    P2_DISPATCH(p, (launch_plane2<N>(0, gp, p->smem_p2, st, P)));
    LAUNCHED("k_plane2_mom");
  } else {
    PLANE_DISPATCH(p, (launch_plane<E, F>(0, gp, p->smem_plane, st, P)));
    LAUNCHED("k_plane_mom");
  }
  prof_end(p, st, slot);
  prof_begin(p, FWI_K_ZPASS_MASS, st, P.nsims, &slot);
  if (p->z2) {
    Z2_DISPATCH(p, (launch_zpass2<NZ>(1, TZ, gz, p->smem_z2[1], st, P)));
    LAUNCHED("k_zpass2<mass>");
  } else {
    Z_DISPATCH(p, (launch_zpass<E, FZ>(1, TZ, gz, p->smem_zmass, st, P)));
    LAUNCHED("k_zpass<mass>");
  }
  prof_end(p, st, slot);
  prof_begin(p, FWI_K_PLANE_MASS, st, P.nsims, &slot);
  if (p->p2) {
    P2_DISPATCH(p, (launch_plane2<N>(1, gp, p->smem_p2, st, P)));
    LAUNCHED("k_plane2_mass");
  } else {
    PLANE_DISPATCH(p, (launch_plane<E, F>(1, gp, p->smem_mass, st, P)));
    LAUNCHED("k_plane_mass");
  }
  prof_end(p, st, slot);
  return FWI_OK;
}

// One time step: all simulations in one launch sequence, or (plain form) one
// launch sequence per simulation.
fwi_status launch_step(fwi_plan* p, const StepParams& P, cudaStream_t st) {
  const int spl = p->prob.sims_per_launch;
  if (spl <= 0 || spl >= P.nsims) return launch_step_batch(p, P, st);
  for (int s0 = 0; s0 < P.nsims; s0 += spl) {
    StepParams Q = P;
    Q.nsims = std::min(spl, P.nsims - s0);
    for (int i = 0; i < Q.nsims; ++i) {
      Q.sims[i] = P.sims[s0 + i];
      Q.tidx[i] = P.tidx[s0 + i];
      Q.slot[i] = P.slot[s0 + i];
    }
    const fwi_status s = launch_step_batch(p, Q, st);
    if (s != FWI_OK) return s;
  }
  return FWI_OK;
}

// Launch shapes and shared-memory sizes of the plan's current schedule.
fwi_status apply_schedule(fwi_plan* p) {
  const fwi_problem& q = p->prob;
  const fwi_schedule& sc = p->sched;
  p->epl = std::max(q.nx, std::max(q.ny, q.nz)) <= 256 ? 8 : 16;
  auto in = [](int v, std::initializer_list<int> l) {
    for (int x : l)
      if (x == v) return true;
    return false;
  };
  p->split = sc.split_plane;
  p->fxy = (!p->split && sc.specialized && q.nx == q.ny && in(q.nx, {32, 64, 96, 128, 160})) ? q.nx : 0;
  p->fz = (sc.specialized && in(q.nz, {32, 48, 64, 80, 96, 128})) ? q.nz : 0;
  p->tz = sc.z_tile;
  p->p2 = 0;
  p->smem_p2 = 0;
  p->z2 = 0;
  p->smem_z2[0] = p->smem_z2[1] = 0;
  p->s2 = 0;
  p->smem_y2 = p->smem_x2 = 0;
  if (sc.specialized == 2) {   // two-step kernels where built (planes, z pass or both)
    if (!p->split && q.nx == q.ny && in(q.nx, {32, 64, 96, 128, 135, 160})) {
      p->p2 = q.nx;
      P2_DISPATCH(p, (p->smem_p2 = Plane2<N, N>::SMEM));
      if (p->smem_p2 > 227 * 1024) p->p2 = 0;
    }
    if (in(q.nz, {32, 48, 64, 80, 96, 128, 135, 256})) {
      p->z2 = q.nz;
      Z2_DISPATCH(p, (p->smem_z2[0] = Z2<NZ, TZ>::smem(0), p->smem_z2[1] = Z2<NZ, TZ>::smem(1)));
      if (p->smem_z2[0] > 227 * 1024) p->z2 = 0;
    }
    if (p->split && q.nx == q.ny && in(q.nx, {243, 256, 480})) {
      p->s2 = q.nx;
      S2_DISPATCH(p, (p->smem_y2 = Y2<N, ty2_for(N)>::SMEM, p->smem_x2 = X2<N, npc2_for(N)>::SMEM));
      if (p->smem_y2 > 227 * 1024 || p->smem_x2 > 227 * 1024) p->s2 = 0;
    }
    if (!p->p2 && !p->z2 && !p->s2) return FWI_ENOTSUP;
  }
  const int tw_x = p->ax.tw_off, tw_y = p->ay.tw_off, tw_z = p->az.tw_off;
  if (!factor235(q.nx, &p->ax, sc.radix_order) || !factor235(q.ny, &p->ay, sc.radix_order) ||
      !factor235(q.nz, &p->az, sc.radix_order))
    return FWI_ENOTSUP;
  p->ax.tw_off = tw_x;
  p->ay.tw_off = tw_y;
  p->az.tw_off = tw_z;
  const int ntw = ((q.nx + q.ny + 31) & ~31);
  // pair lines per warp group: momentum (x work budget 256) and mass (128)
  auto group = [&](int budget) {
    int g = 1;
    if (p->fxy > 0) {
      while (2 * g <= budget / p->fxy) g *= 2;
    } else {
      g = std::max(1, budget * p->epl / (16 * p->hx));
    }
    return g;
  };
  const size_t base = ((size_t)ntw + (size_t)p->npair * 2 * p->hx) * sizeof(float2);
  const size_t warps = kTpbPlane / 32;
  p->smem_plane = base + warps * 1 * 2 * group(256) * q.nx * 4;   // one staged array
  p->smem_mass = base + warps * 4 * 2 * group(128) * q.nx * 4;    // four staged arrays
  const size_t ztw = (size_t)((q.nz + 31) & ~31);
  p->smem_zmom = (ztw + (size_t)(2 * p->tz + 4) * q.nz) * sizeof(float2);
  p->smem_zmass = (ztw + (size_t)(3 * p->tz + 4) * q.nz) * sizeof(float2);
  // split planes: column passes over y and warp-owned row pairs for the x work
  {
    const size_t ytw = (size_t)((q.ny + 31) & ~31);
    p->smem_ypass3 = (ytw + (size_t)(3 * kTY + 4) * q.ny) * sizeof(float2);
    p->smem_ypass1 = (ytw + (size_t)(1 * kTY + 4) * q.ny) * sizeof(float2);
    const int g1 = std::max(1, 16 * p->epl / p->hx), g2 = std::max(1, 8 * p->epl / p->hx);
    const size_t xtw = (size_t)((q.nx + 31) & ~31);
    p->smem_xmom = (xtw + warps * (size_t)g1 * 2 * p->hx) * sizeof(float2) + warps * 2 * g1 * q.nx * 4;
    p->smem_xmass = (xtw + warps * (size_t)g2 * 2 * p->hx) * sizeof(float2) + warps * 4 * 2 * g2 * q.nx * 4;
  }
  if (std::max(q.nx, std::max(q.ny, q.nz)) > 512 || p->smem_zmass > 227 * 1024) return FWI_ENOTSUP;
  if (p->split ? (p->smem_ypass3 > 227 * 1024 || p->smem_xmass > 227 * 1024) : p->smem_mass > 227 * 1024)
    return FWI_ENOTSUP;
  return FWI_OK;
}

fwi_status zero_sim(fwi_plan* p, int s, cudaStream_t st) {
  CK(cudaMemsetAsync(p->ws + p->o_sims + (size_t)s * p->sim_bytes, 0, p->sim_bytes, st));
  return FWI_OK;
}

// common per-call preparation: c^2, range flag, sparse coefficients
// c: [models][nvox], one model per super-shot when the plan has per-shot models
fwi_status prepare(fwi_plan* p, const float* c, cudaStream_t st) {
  const fwi_problem& q = p->prob;
  CK(cudaMemsetAsync(p->ws + p->o_bad, 0, sizeof(int), st));
  if (p->tr && p->tr->ws) CK(cudaMemsetAsync(p->tr->ws + p->tr->o_bad, 0, sizeof(int), st));
  for (int m = 0; m < p->models; ++m) {
    const float* cm = c + (size_t)m * p->nvox;
    k_prepare_c<<<592, 256, 0, st>>>(cm, at<float>(p, p->o_c2) + (size_t)m * p->nvox, p->nvox, (float)q.c_ref,
                                     at<int>(p, p->o_bad));
    LAUNCHED("k_prepare_c");
    k_prepare_coefs<<<148, 256, 0, st>>>(
        cm, q.dt, q.dx, at<int>(p, p->o_us_vox), p->n_us, at<float>(p, p->o_us_coef) + (size_t)m * p->n_us,
        at<int>(p, p->o_ur_vox), p->n_ur, at<float>(p, p->o_ur_coef) + (size_t)m * p->n_ur, at<int>(p, p->o_gam_vox),
        q.n_gamma, at<float>(p, p->o_coefG) + (size_t)m * q.n_gamma, at<int>(p, p->o_lay_vox), q.n_layer,
        at<float>(p, p->o_inv3c2) + (size_t)m * q.n_layer);
    LAUNCHED("k_prepare_coefs");
  }
  return FWI_OK;
}

// The two-step mass kernels (whole planes or split planes) carry the deferred Gamma
// accumulation; the other kernel families leave it to k_accumulate.
bool fused_accumulation(const fwi_plan* p) { return p->p2 != 0 || p->s2 != 0; }

// Stream groups: shots [g*KG, min(K, (g+1)*KG)) of group g advance on stream g (0 = the
// caller's stream), forked from and joined to it.
int group_count(const fwi_plan* p, int K) { return std::max(1, std::min(p->sched.stream_groups, K)); }
cudaStream_t group_stream(const fwi_plan* p, int g, cudaStream_t st) { return g == 0 ? st : p->side[g - 1]; }
fwi_status fork_groups(fwi_plan* p, int G, cudaStream_t st) {
  if (G < 2) return FWI_OK;
  CK(cudaEventRecord(p->ev_fork, st));
  for (int g = 1; g < G; ++g) CK(cudaStreamWaitEvent(p->side[g - 1], p->ev_fork, 0));
  return FWI_OK;
}
fwi_status join_groups(fwi_plan* p, int G, cudaStream_t st) {
  for (int g = 1; g < G; ++g) {
    CK(cudaEventRecord(p->ev_join[g - 1], p->side[g - 1]));
    CK(cudaStreamWaitEvent(st, p->ev_join[g - 1], 0));
  }
  return FWI_OK;
}

// TR initial value (Alg. 1): p(layer) <- g^Nt, ring slot 0 <- p(Gamma), forward XY
// transform of p, for the K TR simulations of T on plan p's grid
fwi_status launch_tr_init(fwi_plan* p, const StepParams& T, int K, cudaStream_t st) {
  const fwi_problem& q = p->prob;
  if (p->split) {
    const int warps = kTpbPlane / 32;
    const dim3 gy((p->hx + kTY - 1) / kTY, q.nz, K);
    if (p->epl == 8) {
      const int g = std::max(1, 16 * 8 / p->hx);
      launch_split<8>(6, dim3((p->npair + warps * g - 1) / (warps * g), q.nz, K), p->smem_xmom, st, T);
      LAUNCHED("k_xpass_tr_init");
      launch_split<8>(Y_FWD1, gy, p->smem_ypass1, st, T);
    } else {
      const int g = std::max(1, 16 * 16 / p->hx);
      launch_split<16>(6, dim3((p->npair + warps * g - 1) / (warps * g), q.nz, K), p->smem_xmom, st, T);
      LAUNCHED("k_xpass_tr_init");
      launch_split<16>(Y_FWD1, gy, p->smem_ypass1, st, T);
    }
    LAUNCHED("k_ypass<forward x1>");
  } else {
    PLANE_DISPATCH(p, (launch_plane<E, F>(2, dim3(q.nz, K), p->smem_plane, st, T)));
    LAUNCHED("k_tr_init");
  }
  return FWI_OK;
}

fwi_status run_forward(fwi_plan* p, const float* w, const int* delay, int K, bool record_layer,
                       float* traces, cudaStream_t st) {
  const fwi_problem& q = p->prob;
  k_source_amp<<<dim3(q.nt, K), 128, 0, st>>>(w, q.n_src, at<float>(p, p->o_us_coef),
                                              at<int>(p, p->o_us_mptr), at<int>(p, p->o_us_mem), p->n_us,
                                              at<float>(p, p->o_wav), q.nt, delay, at<float>(p, p->o_amp),
                                              p->models > 1 ? 1 : 0);
  LAUNCHED("k_source_amp");
  StepParams P;
  base_params(p, &P);
  P.record_layer = record_layer ? 1 : 0;
  P.traces = traces;
  P.nsims = K;
  for (int k = 0; k < K; ++k) {
    sim_ptrs(p, k, &P.sims[k], ROLE_FORWARD, k);
    fwi_status s = zero_sim(p, k, st);
    if (s != FWI_OK) return s;
  }
  const int G = group_count(p, K), KG = (K + G - 1) / G;
  StepParams Q[fwi_plan::kMaxGroups];
  for (int g = 0; g < G; ++g) {
    Q[g] = P;
    Q[g].nsims = std::max(0, std::min(K, (g + 1) * KG) - g * KG);
    for (int k = 0; k < Q[g].nsims; ++k) Q[g].sims[k] = P.sims[g * KG + k];
  }
  fwi_status s = fork_groups(p, G, st);
  if (s != FWI_OK) return s;
  for (int n = 0; n < q.nt; ++n) {
    for (int g = 0; g < G; ++g) {
      if (Q[g].nsims == 0) continue;
      for (int k = 0; k < Q[g].nsims; ++k) Q[g].tidx[k] = n;
      if ((s = launch_step(p, Q[g], group_stream(p, g, st))) != FWI_OK) return s;
    }
  }
  return join_groups(p, G, st);
}

fwi_status check_call(fwi_plan* p, int K) {
  // A non-sticky error left by another library would otherwise be reported as
  // ours by the launch checks below; faults that poison the context persist.
  (void)cudaGetLastError();
  if (!p || !p->ws) return FWI_EINVAL;
  if (K < 1 || K > p->K) return FWI_EINVAL;
  return FWI_OK;
}


// Workspace layout of a plan.  A plan that only runs TR simulations for another plan
// (tr_only: the TR box of Sec. 3.1) keeps no traces, data, boundary history or
// accumulators, and K simulation states instead of 2K; a plan with a TR box keeps K
// (its adjoint simulations) and the box plan's workspace and cropped sound speed.
void plan_layout(fwi_plan* p) {
  const fwi_problem& q = p->prob;
  const int64_t nvox = p->nvox;
  p->L = Layout();
  Layout& L = p->L;
  const int K = p->K, nt = q.nt;
  const size_t per_call = p->tr_only ? 0 : 1;   // buffers a TR-only plan does not need
  p->o_tw = L.add(p->tw.size() * sizeof(float2));
  p->o_kx2 = L.add(p->kx2.size() * 4); p->o_ky2 = L.add(p->ky2.size() * 4); p->o_kz2 = L.add(p->kz2.size() * 4);
  for (int a = 0; a < 3; ++a) {
    p->o_ap[a] = L.add(p->ap[a].size() * sizeof(float2));
    p->o_am[a] = L.add(p->am[a].size() * sizeof(float2));
    p->o_lam[a] = L.add(p->lam[a].size() * 4);
    p->o_lams[a] = L.add(p->lams[a].size() * 4);
  }
  const size_t nkey = (size_t)q.nz * p->npair + 1;
  p->o_us_ptr = L.add(nkey * 4); p->o_us_pf = L.add(p->n_us * 4); p->o_us_vox = L.add(p->n_us * 4);
  p->o_us_mptr = L.add((p->n_us + 1) * 4); p->o_us_mem = L.add(q.n_src * 4);
  p->o_ur_ptr = L.add(nkey * 4); p->o_ur_pf = L.add(p->n_ur * 4); p->o_ur_vox = L.add(p->n_ur * 4);
  p->o_ur_mptr = L.add((p->n_ur + 1) * 4); p->o_ur_mem = L.add(q.n_rec * 4);
  p->o_rr_ptr = L.add(nkey * 4); p->o_rr_pf = L.add(q.n_rec * 4); p->o_rr_col = L.add(q.n_rec * 4);
  p->o_lay_ptr = L.add(nkey * 4); p->o_lay_vox = L.add((size_t)q.n_layer * 4 + 4);
  p->o_lay_pf = L.add((size_t)q.n_layer * 4 + 4);
  p->o_gam_ptr = L.add(nkey * 4); p->o_gam_vox = L.add((size_t)q.n_gamma * 4);
  p->o_gam_pf = L.add((size_t)q.n_gamma * 4);
  p->o_wav = L.add((size_t)nt * 4);
  p->o_bad = L.add(4);
  const size_t M = p->models;
  p->o_c2 = L.add(M * nvox * 4);
  p->o_us_coef = L.add(M * p->n_us * 4); p->o_ur_coef = L.add(M * p->n_ur * 4);
  p->o_coefG = L.add(M * q.n_gamma * 4); p->o_inv3c2 = L.add(M * q.n_layer * 4 + 4);
  p->o_amp = L.add(per_call * K * nt * p->n_us * 4);
  p->o_traces = L.add(per_call * K * nt * q.n_rec * 4);
  p->o_obs = L.add(per_call * K * nt * q.n_rec * 4);
  p->o_qf = L.add(per_call * K * nt * q.n_rec * 4);
  p->o_ghist = L.add(per_call * K * nt * q.n_layer * 4 + 4);
  p->o_ring = L.add(per_call * K * kRing * q.n_gamma * 4);
  p->o_pa = L.add(per_call * K * q.n_gamma * 4);
  p->o_acc = L.add(per_call * K * q.n_gamma * 8);
  p->nblk_misfit = (q.n_rec + 255) / 256;
  p->o_dpart = L.add(per_call * K * p->nblk_misfit * 8);
  p->sim_field = ((size_t)nvox * 4 + 255) & ~size_t(255);
  p->sim_spec = ((size_t)p->mspec * q.nz * sizeof(float2) + 255) & ~size_t(255);
  p->sim_bytes = 6 * p->sim_field + 3 * p->sim_spec;
  p->o_sims = L.add((size_t)((p->tr_only || p->tr) ? 1 : 2) * K * p->sim_bytes);
  if (p->tr) {
    p->o_trc = L.add(M * p->tr->nvox * 4);
    p->o_trws = L.add(p->tr->L.total);
  }
}

}  // namespace

extern "C" {

const char* fwi_last_cuda_error(void) { return g_last_cuda_error; }

const char* fwi_status_string(fwi_status s) {
  switch (s) {
    case FWI_OK: return "ok";
    case FWI_EINVAL: return "invalid argument";
    case FWI_ENOMEM: return "out of memory / workspace too small";
    case FWI_EUNSTABLE: return "sound speed outside (0, c_ref]: unstable";
    case FWI_ETIMEOUT: return "device wait timed out";
    case FWI_ECUDA: return "CUDA error";
    case FWI_ECANCELLED: return "cancelled";
    case FWI_ENOTSUP: return "grid not supported";
  }
  return "unknown status";
}

}  // extern "C"

namespace {
// fwi_plan_create; tr_only = a plan that runs only the TR simulations of another plan
fwi_status fwi_plan_create_impl(const fwi_problem* prob, bool tr_only, size_t* workspace_bytes, fwi_plan** out) {
  if (!prob || !workspace_bytes || !out) return FWI_EINVAL;
  const fwi_problem& q = *prob;
  if (q.nx < 2 || q.ny < 2 || q.nz < 2 || q.nt < 3 || q.n_src < 1 || q.n_rec < 1 ||
      q.n_gamma < 1 || q.n_layer < 0 || q.max_shots < 1 || q.max_shots > kMaxSims / 2)
    return FWI_EINVAL;
  if (!(q.dx > 0) || !(q.dt > 0) || !(q.c_ref > 0) || !(q.rho0 > 0) || q.pml_alpha < 0 || q.c_rec < 0)
    return FWI_EINVAL;
  if (!q.src_idx || !q.rec_idx || !q.gamma_idx || (q.n_layer > 0 && !q.layer_idx) || !q.wavelet)
    return FWI_EINVAL;
  if (q.pairing != FWI_PAIRING_LITERAL && q.pairing != FWI_PAIRING_EXACT) return FWI_EINVAL;
  if (q.sims_per_launch < 0 || (q.per_shot_models != 0 && q.per_shot_models != 1)) return FWI_EINVAL;
  for (int a = 0; a < 3; ++a) {
    const int n = a == 0 ? q.nx : (a == 1 ? q.ny : q.nz);
    if (q.pml[a] < 0 || 2 * q.pml[a] > n) return FWI_EINVAL;
  }
  const int64_t nvox = (int64_t)q.nx * q.ny * q.nz;
  if (nvox >= (int64_t)1 << 31) return FWI_ENOTSUP;
  auto in_range = [&](const int32_t* v, int n) {
    for (int i = 0; i < n; ++i)
      if (v[i] < 0 || v[i] >= nvox) return false;
    return true;
  };
  if (!in_range(q.src_idx, q.n_src) || !in_range(q.rec_idx, q.n_rec) ||
      !in_range(q.gamma_idx, q.n_gamma) || !in_range(q.layer_idx, q.n_layer))
    return FWI_EINVAL;
  for (int i = 1; i < q.n_gamma; ++i)
    if (q.gamma_idx[i] <= q.gamma_idx[i - 1]) return FWI_EINVAL;
  for (int i = 1; i < q.n_layer; ++i)
    if (q.layer_idx[i] <= q.layer_idx[i - 1]) return FWI_EINVAL;
  for (int i = 0; i < q.n_layer; ++i)
    if (!std::binary_search(q.gamma_idx, q.gamma_idx + q.n_gamma, q.layer_idx[i])) return FWI_EINVAL;

  fwi_plan* p = new (std::nothrow) fwi_plan();
  if (!p) return FWI_ENOMEM;
  p->prob = q;
  p->tr_only = tr_only;
  p->models = q.per_shot_models ? q.max_shots : 1;
  p->prob.src_idx = p->prob.rec_idx = p->prob.layer_idx = p->prob.gamma_idx = nullptr;
  p->prob.wavelet = nullptr;
  p->K = q.max_shots;
  p->nvox = nvox;
  p->hx = q.nx / 2 + 1;
  p->npair = (q.ny + 1) / 2;
  p->plane = q.nx * q.ny;
  p->mspec = p->hx * q.ny;
  if (!factor235(q.nx, &p->ax) || !factor235(q.ny, &p->ay) || !factor235(q.nz, &p->az)) {
    delete p;
    return FWI_ENOTSUP;
  }
  // twiddles W[k] = exp(-2 pi i k / N), per axis, FP64 -> FP32
  AxisPlan* axes[3] = {&p->ax, &p->ay, &p->az};
  for (int a = 0; a < 3; ++a) {
    axes[a]->tw_off = (int)p->tw.size();
    const int n = axes[a]->n;
    for (int k = 0; k < n; ++k) {
      const double ang = -2.0 * kPi * (double)k / (double)n;
      p->tw.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
    }
  }
  // wavenumbers and the staggered x/y/z factors i k exp(+-i k dx/2) (Eq. 19)
  const int lens[3] = {p->hx, q.ny, q.nz};
  const int ns[3] = {q.nx, q.ny, q.nz};
  std::vector<float>* k2[3] = {&p->kx2, &p->ky2, &p->kz2};
  for (int a = 0; a < 3; ++a) {
    for (int j = 0; j < lens[a]; ++j) {
      const double k = wavenumber(j, ns[a], q.dx);
      k2[a]->push_back((float)(k * k));
      const double h = k * q.dx / 2.0;
      // i k (cos h +- i sin h) = (-+ k sin h) + i k cos h
      p->ap[a].push_back(make_float2((float)(-k * std::sin(h)), (float)(k * std::cos(h))));
      p->am[a].push_back(make_float2((float)(k * std::sin(h)), (float)(k * std::cos(h))));
    }
    for (int i = 0; i < ns[a]; ++i) {
      p->lam[a].push_back((float)pml_value(i, ns[a], q.pml[a], q.pml_alpha, q.c_ref, q.dx, q.dt, false));
      p->lams[a].push_back((float)pml_value(i, ns[a], q.pml[a], q.pml_alpha, q.c_ref, q.dx, q.dt, true));
    }
  }
  p->wavelet.assign(prob->wavelet, prob->wavelet + q.nt);
  const KeyGeom kg{q.nx, q.ny, q.nz, p->npair, p->hx};
  p->us = build_unique(prob->src_idx, q.n_src, kg);
  p->ur = build_unique(prob->rec_idx, q.n_rec, kg);
  p->n_us = (int)p->us.vox.size();
  p->n_ur = (int)p->ur.vox.size();
  {
    std::vector<std::pair<int, int>> e;
    for (int r = 0; r < q.n_rec; ++r) e.push_back({prob->rec_idx[r], r});
    std::stable_sort(e.begin(), e.end());
    p->rr = build_sorted(e, kg);                 // receivers to record, with their column
    e.clear();
    for (int j = 0; j < q.n_layer; ++j) e.push_back({prob->layer_idx[j], j});
    p->lay = build_sorted(e, kg);
    e.clear();
    for (int j = 0; j < q.n_gamma; ++j) e.push_back({prob->gamma_idx[j], j});
    p->gam = build_sorted(e, kg);
  }

  // launch shapes: every axis must fit one warp group (n <= 512)
  // default schedule: two-step kernels where built (whole planes, else split planes),
  // else the compile-time or runtime transforms (whole planes, else split planes)
  bool placed = false;
  for (const fwi_schedule sc : {fwi_schedule{2, 0, 32, 0, 4}, fwi_schedule{2, 0, 32, 1, 4},
                                fwi_schedule{1, 0, 32, 0, 4}, fwi_schedule{1, 0, 32, 1, 4}}) {
    p->sched = sc;
    if (apply_schedule(p) == FWI_OK) {
      placed = true;
      break;
    }
  }
  if (!placed) {
    delete p;
    return FWI_ENOTSUP;
  }
  plan_layout(p);
  *workspace_bytes = p->L.total;
  *out = p;
  return FWI_OK;
}
}  // namespace

extern "C" {

fwi_status fwi_plan_create(const fwi_problem* prob, size_t* workspace_bytes, fwi_plan** out) {
  return fwi_plan_create_impl(prob, false, workspace_bytes, out);
}

fwi_status fwi_plan_bind_workspace(fwi_plan* p, void* dev_ptr, size_t bytes) {
  if (!p || !dev_ptr || ((uintptr_t)dev_ptr & 255)) return FWI_EINVAL;
  if (bytes < p->L.total) return FWI_ENOMEM;
  p->ws = static_cast<char*>(dev_ptr);
  p->ws_bytes = bytes;
  p->generation++;
  auto up = [&](size_t off, const void* src, size_t n) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    return cudaMemcpy(p->ws + off, src, n, cudaMemcpyHostToDevice);
  };
  CK(up(p->o_tw, p->tw.data(), p->tw.size() * sizeof(float2)));
  CK(up(p->o_kx2, p->kx2.data(), p->kx2.size() * 4));
  CK(up(p->o_ky2, p->ky2.data(), p->ky2.size() * 4));
  CK(up(p->o_kz2, p->kz2.data(), p->kz2.size() * 4));
  for (int a = 0; a < 3; ++a) {
    CK(up(p->o_ap[a], p->ap[a].data(), p->ap[a].size() * sizeof(float2)));
    CK(up(p->o_am[a], p->am[a].data(), p->am[a].size() * sizeof(float2)));
    CK(up(p->o_lam[a], p->lam[a].data(), p->lam[a].size() * 4));
    CK(up(p->o_lams[a], p->lams[a].data(), p->lams[a].size() * 4));
  }
  auto upc = [&](const Csr& c, size_t o_ptr, size_t o_vox, size_t o_pf) -> cudaError_t {
    cudaError_t e;
    if ((e = up(o_ptr, c.ptr.data(), c.ptr.size() * 4)) != cudaSuccess) return e;
    if ((e = up(o_vox, c.vox.data(), c.vox.size() * 4)) != cudaSuccess) return e;
    return up(o_pf, c.pf.data(), c.pf.size() * 4);
  };
  CK(upc(p->us, p->o_us_ptr, p->o_us_vox, p->o_us_pf));
  CK(up(p->o_us_mptr, p->us.mptr.data(), p->us.mptr.size() * 4));
  CK(up(p->o_us_mem, p->us.mem.data(), p->us.mem.size() * 4));
  CK(upc(p->ur, p->o_ur_ptr, p->o_ur_vox, p->o_ur_pf));
  CK(up(p->o_ur_mptr, p->ur.mptr.data(), p->ur.mptr.size() * 4));
  CK(up(p->o_ur_mem, p->ur.mem.data(), p->ur.mem.size() * 4));
  CK(up(p->o_rr_ptr, p->rr.ptr.data(), p->rr.ptr.size() * 4));
  CK(up(p->o_rr_pf, p->rr.pf.data(), p->rr.pf.size() * 4));
  CK(up(p->o_rr_col, p->rr.mem.data(), p->rr.mem.size() * 4));
  CK(upc(p->lay, p->o_lay_ptr, p->o_lay_vox, p->o_lay_pf));
  CK(upc(p->gam, p->o_gam_ptr, p->o_gam_vox, p->o_gam_pf));
  CK(up(p->o_wav, p->wavelet.data(), p->wavelet.size() * 4));
  for (int g = 0; g < fwi_plan::kMaxGroups - 1; ++g) {
    if (!p->side[g]) CK(cudaStreamCreateWithFlags(&p->side[g], cudaStreamNonBlocking));
    if (!p->ev_join[g]) CK(cudaEventCreateWithFlags(&p->ev_join[g], cudaEventDisableTiming));
  }
  if (!p->ev_fork) CK(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  set_attrs(p);
  CK(cudaGetLastError());
  if (p->tr) {
    const fwi_status st = fwi_plan_bind_workspace(p->tr, p->ws + p->o_trws, p->tr->L.total);
    if (st != FWI_OK) return st;
  }
  return FWI_OK;
}

namespace {
fwi_status forward_impl(fwi_plan* p, const float* c, const float* weights, const int* delay, int32_t K,
                        float* traces, void* stream) {
  fwi_status s = check_call(p, K);
  if (s != FWI_OK) return s;
  if (!c || !weights || !traces) return FWI_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  p->last = st;
  p->used = true;
  if ((s = prepare(p, c, st)) != FWI_OK) return s;
  return run_forward(p, weights, delay, K, false, traces, st);
}
fwi_status gradient_impl(fwi_plan* p, const float* c, const float* weights, const int* delay, int32_t K,
                         const float* observed, int32_t observed_encoded, int32_t observed_nt, double* misfit,
                         double* grad, float* traces, void* stream);
}  // namespace

fwi_status fwi_forward(fwi_plan* p, const float* c, const float* weights, int32_t K, float* traces,
                       void* stream) {
  return forward_impl(p, c, weights, nullptr, K, traces, stream);
}
fwi_status fwi_forward_delayed(fwi_plan* p, const float* c, const float* weights, const int32_t* delay,
                               int32_t K, float* traces, void* stream) {
  if (!delay) return FWI_EINVAL;
  return forward_impl(p, c, weights, delay, K, traces, stream);
}
fwi_status fwi_gradient(fwi_plan* p, const float* c, const float* weights, int32_t K,
                        const float* observed, int32_t observed_encoded, double* misfit, double* grad,
                        float* traces, void* stream) {
  return gradient_impl(p, c, weights, nullptr, K, observed, observed_encoded, p ? p->prob.nt : 0, misfit,
                       grad, traces, stream);
}
fwi_status fwi_gradient_delayed(fwi_plan* p, const float* c, const float* weights, const int32_t* delay,
                                int32_t K, const float* observed, int32_t observed_encoded,
                                int32_t observed_nt, double* misfit, double* grad, float* traces,
                                void* stream) {
  if (!delay || !p) return FWI_EINVAL;
  if (!observed_encoded && (observed_nt < 1 || observed_nt > p->prob.nt)) return FWI_EINVAL;
  return gradient_impl(p, c, weights, delay, K, observed, observed_encoded, observed_nt, misfit, grad, traces,
                       stream);
}

namespace {

fwi_status gradient_impl(fwi_plan* p, const float* c, const float* weights, const int* delay, int32_t K,
                         const float* observed, int32_t observed_encoded, int32_t observed_nt, double* misfit,
                         double* grad, float* traces, void* stream) {
  fwi_status s = check_call(p, K);
  if (s != FWI_OK) return s;
  if (!c || !weights || !observed || !misfit || !grad) return FWI_EINVAL;
  const fwi_problem& q = p->prob;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  p->last = st;
  p->used = true;
  const int nt = q.nt, Nt = nt - 1;
  if ((s = prepare(p, c, st)) != FWI_OK) return s;
  // observed data, encoded
  const float* obs = observed;
  if (!observed_encoded) {
    if (delay) {
      k_encode_delayed<<<592, 256, 0, st>>>(observed, weights, delay, q.n_src, K, observed_nt, nt, q.n_rec,
                                            at<float>(p, p->o_obs));
      LAUNCHED("k_encode_delayed");
    } else {
      const int64_t per = (int64_t)nt * q.n_rec;
      k_encode<<<592, 256, 0, st>>>(observed, weights, q.n_src, K, per, at<float>(p, p->o_obs));
      LAUNCHED("k_encode");
    }
    obs = at<float>(p, p->o_obs);
  }
  // forward, recording traces and the boundary-layer history
  if ((s = run_forward(p, weights, delay, K, true, at<float>(p, p->o_traces), st)) != FWI_OK) return s;
  // residual, misfit, cumulative sum
  k_misfit<<<dim3(p->nblk_misfit, K), 256, 0, st>>>(at<float>(p, p->o_traces), obs, nt, q.n_rec,
                                                    at<float>(p, p->o_qf), at<double>(p, p->o_dpart));
  LAUNCHED("k_misfit");
  k_misfit_final<<<1, 32, 0, st>>>(at<double>(p, p->o_dpart), p->nblk_misfit, K, misfit);
  LAUNCHED("k_misfit_final");
  CK(cudaMemsetAsync(p->ws + p->o_acc, 0, (size_t)K * q.n_gamma * 8, st));
  // Adjoint simulations 0..K-1 on this plan's grid; TR simulations on the grid of tp:
  // this plan (simulations K..2K-1) or its TR box (Sec. 3.1; the box plan's simulations
  // 0..K-1, c0 cropped from the full model, the boundary history and the ring shared).
  fwi_plan* tp = p->tr ? p->tr : p;
  if (p->tr) {
    const fwi_problem& b = tp->prob;
    for (int m = 0; m < p->models; ++m) {
      k_crop<<<592, 256, 0, st>>>(c + (size_t)m * p->nvox, q.nx, q.ny, p->tr_origin[0], p->tr_origin[1],
                                  p->tr_origin[2], b.nx, b.ny, b.nz, at<float>(p, p->o_trc) + (size_t)m * tp->nvox);
      LAUNCHED("k_crop");
    }
    if ((s = prepare(tp, at<float>(p, p->o_trc), st)) != FWI_OK) return s;
  }
  StepParams P, T;
  base_params(p, &P);
  base_params(tp, &T);
  T.ghist = P.ghist;
  T.ring = P.ring;
  const int tr0 = p->tr ? 0 : K;
  for (int k = 0; k < K; ++k) {
    sim_ptrs(p, k, &P.sims[k], ROLE_ADJOINT, k);
    sim_ptrs(tp, tr0 + k, &T.sims[k], ROLE_TR, k);
    if ((s = zero_sim(p, k, st)) != FWI_OK) return s;
    if ((s = zero_sim(tp, tr0 + k, st)) != FWI_OK) return s;
  }
  // TR initial value and the lead TR step (m = 1)
  T.nsims = K;
  for (int k = 0; k < K; ++k) {
    T.tidx[k] = 1;
    T.slot[k] = 1;
  }
  if ((s = launch_tr_init(tp, T, K, st)) != FWI_OK) return s;
  if ((s = launch_step(tp, T, st)) != FWI_OK) return s;
  // interleaved adjoint and TR iterations
  const bool exact = q.pairing == FWI_PAIRING_EXACT;
  const int nit = exact ? Nt + 1 : Nt - 1;
  const int nblk = (q.n_gamma + 255) / 256;
  // The two-step mass kernels add iteration it's gradient term inside iteration it + 1's
  // adjoint launch (before they overwrite pa); the last iteration's, and every
  // iteration's for the other kernel families, runs as k_accumulate.
  const bool fused = fused_accumulation(p);
  auto accumulate = [&](int it, int k0, int nk, cudaStream_t gs) -> fwi_status {
    k_accumulate<<<dim3(nblk, nk), 256, 0, gs>>>(at<float>(p, p->o_ring), at<float>(p, p->o_pa),
                                                 at<float>(p, p->o_coefG), q.n_gamma, it % kRing,
                                                 (it + 1) % kRing, (it + 2) % kRing, at<double>(p, p->o_acc),
                                                 at<int>(p, p->o_bad), k0, p->models > 1 ? 1 : 0);
    LAUNCHED("k_accumulate");
    return FWI_OK;
  };
  // shots [k0, k0 + nk) advance on stream gs: their adjoint simulations (k) and TR
  // simulations (K + k) in one launch sequence, then their Gamma accumulation
  auto iterate = [&](int it, int k0, int nk, cudaStream_t gs) -> fwi_status {
    const int qi = exact ? it : it + 1;    // row of Q injected by this adjoint step
    const int m = it + 2;                  // TR state produced in this iteration
    const int slot = m % kRing;
    StepParams S = P;
    S.nsims = nk;
    for (int k = 0; k < nk; ++k) {
      S.sims[k] = P.sims[k0 + k];
      S.tidx[k] = qi;
    }
    if (fused && it > 0) {
      S.acc_prev = 1;
      S.acc_slot[0] = (it - 1) % kRing;
      S.acc_slot[1] = it % kRing;
      S.acc_slot[2] = (it + 1) % kRing;
    }
    StepParams R = T;                      // TR simulations of these shots
    R.nsims = nk;
    for (int k = 0; k < nk; ++k) {
      R.sims[k] = T.sims[k0 + k];
      R.tidx[k] = m;
      R.slot[k] = slot;
    }
    if (m <= Nt && !p->tr) {               // adjoint and TR simulations share each launch
      S.nsims = 2 * nk;
      for (int k = 0; k < nk; ++k) {
        S.sims[nk + k] = R.sims[k];
        S.tidx[nk + k] = m;
        S.slot[nk + k] = slot;
      }
    } else if (m > Nt) {
      for (int k = k0; k < k0 + nk; ++k)
        CK(cudaMemsetAsync(at<float>(p, p->o_ring) + ((size_t)k * kRing + slot) * q.n_gamma, 0,
                           (size_t)q.n_gamma * 4, gs));
    }
    fwi_status r = launch_step(p, S, gs);
    if (r != FWI_OK) return r;
    if (m <= Nt && p->tr && (r = launch_step(tp, R, gs)) != FWI_OK) return r;
    return fused ? FWI_OK : accumulate(it, k0, nk, gs);
  };
  const int G = group_count(p, K), KG = (K + G - 1) / G;
  if ((s = fork_groups(p, G, st)) != FWI_OK) return s;
  for (int it = 0; it < nit; ++it) {
    for (int g = 0; g < G; ++g) {
      const int k0 = g * KG, nk = std::min(K, k0 + KG) - k0;
      if (nk > 0 && (s = iterate(it, k0, nk, group_stream(p, g, st))) != FWI_OK) return s;
    }
  }
  if (fused) {
    for (int g = 0; g < G; ++g) {
      const int k0 = g * KG, nk = std::min(K, k0 + KG) - k0;
      if (nk > 0 && (s = accumulate(nit - 1, k0, nk, group_stream(p, g, st))) != FWI_OK) return s;
    }
  }
  if ((s = join_groups(p, G, st)) != FWI_OK) return s;
  // mean over shots, scaled to dD/dc if requested
  const double scale = q.c_rec > 0 ? q.dx * q.c_rec / 2.0 : 1.0;
  const int each = p->models > 1 ? 1 : 0;            // one gradient per super-shot
  CK(cudaMemsetAsync(grad, 0, (size_t)(each ? K : 1) * p->nvox * 8, st));
  k_grad_final<<<(q.n_gamma + 255) / 256, 256, 0, st>>>(at<double>(p, p->o_acc), at<int>(p, p->o_gam_vox),
                                                        q.n_gamma, K, scale, grad, each, p->nvox);
  LAUNCHED("k_grad_final");
  if (traces)
    CK(cudaMemcpyAsync(traces, p->ws + p->o_traces, (size_t)K * nt * q.n_rec * 4,
                       cudaMemcpyDeviceToDevice, st));
  CK(cudaGetLastError());
  return FWI_OK;
}
}  // namespace

fwi_status fwi_plan_status(fwi_plan* p) {
  if (!p || !p->ws) return FWI_EINVAL;
  if (!p->used) return FWI_OK;
  CK(cudaStreamSynchronize(p->last));
  int bad = 0;
  CK(cudaMemcpy(&bad, p->ws + p->o_bad, sizeof(int), cudaMemcpyDeviceToHost));
  if (!bad && p->tr)                         // the TR box plan keeps its own flag
    CK(cudaMemcpy(&bad, p->tr->ws + p->tr->o_bad, sizeof(int), cudaMemcpyDeviceToHost));
  return bad ? FWI_EUNSTABLE : FWI_OK;
}

int64_t fwi_plan_voxel_steps(const fwi_plan* p, int32_t K, int32_t gradient) {
  if (!p) return -1;
  const int64_t nt = p->prob.nt, Nt = nt - 1;
  int64_t steps = nt;
  int64_t tr = 0;
  if (gradient) {
    const bool exact = p->prob.pairing == FWI_PAIRING_EXACT;
    tr = Nt;                                       // TR: lead step + loop steps with m <= Nt
    steps += exact ? Nt + 1 : Nt - 1;              // adjoint
  }
  return (steps * p->nvox + tr * (p->tr ? p->tr->nvox : p->nvox)) * K;
}

int64_t fwi_plan_launches(const fwi_plan* p, int32_t K, int32_t gradient) {
  if (!p || K < 1) return -1;
  const int64_t nt = p->prob.nt, Nt = nt - 1;
  const int spl = p->prob.sims_per_launch;
  // kernel launches of one time step over nsims simulations on plan q's grid
  auto step = [&](const fwi_plan* q, int nsims) -> int64_t {
    const int64_t seqs = (spl <= 0 || spl >= nsims) ? 1 : (nsims + spl - 1) / spl;
    return (q->split ? 8 : 4) * seqs;
  };
  const fwi_plan* tp = p->tr ? p->tr : p;
  const int G = group_count(p, K), KG = (K + G - 1) / G;
  int64_t n = 2 * p->models + 1;                        // prepare x2 per model, source amplitudes
  for (int g = 0; g < G; ++g) {                         // forward steps (groups with shots)
    const int ng = std::min(K, (g + 1) * KG) - g * KG;
    if (ng > 0) n += nt * step(p, ng);
  }
  if (gradient) {
    const bool exact = p->prob.pairing == FWI_PAIRING_EXACT;
    const int64_t nit = exact ? Nt + 1 : Nt - 1;
    if (p->tr) n += 3 * p->models;                      // crop and prepare of the box, per model
    n += 2 + (tp->split ? 2 : 1) + step(tp, K);         // misfit x2, TR init, lead TR step
    const int64_t full = std::min<int64_t>(nit, Nt - 1);  // iterations with a TR step
    const int64_t acc = fused_accumulation(p) ? 0 : 1;  // k_accumulate per iteration
    for (int g = 0; g < G; ++g) {
      const int ng = std::min(K, (g + 1) * KG) - g * KG;
      if (ng <= 0) continue;
      const int64_t with_tr = p->tr ? step(p, ng) + step(tp, ng) : step(p, 2 * ng);
      n += full * (with_tr + acc) + (nit - full) * (step(p, ng) + acc);
      if (!acc) n += 1;                                 // last iteration's accumulation
    }
    n += 1;                                             // gradient scatter
  }
  return n;
}

fwi_status fwi_plan_profile(fwi_plan* p, int32_t kernel_mask, int32_t enable, int32_t capacity) {
  if (!p || kernel_mask < 0 || kernel_mask > 15 || capacity < 0) return FWI_EINVAL;
  if (!enable) {
    p->prof_on = false;
    return FWI_OK;
  }
  if ((int)p->prof_ev.size() < 2 * capacity) {
    for (int i = (int)p->prof_ev.size(); i < 2 * capacity; ++i) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      p->prof_ev.push_back(e);
    }
    p->prof_kind.resize(capacity);
  }
  p->prof_mask = kernel_mask;
  p->prof_used = 0;
  for (int k = 0; k < 4; ++k) p->prof_sims[k] = 0;
  p->prof_on = true;
  return FWI_OK;
}

fwi_status fwi_plan_profile_read(fwi_plan* p, double* ms, int64_t* launches, int64_t* sims) {
  if (!p || !ms || !launches || !sims) return FWI_EINVAL;
  for (int k = 0; k < 4; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
    sims[k] = p->prof_sims[k];
    p->prof_sims[k] = 0;
  }
  if (p->prof_used > 0) CK(cudaEventSynchronize(p->prof_ev[2 * p->prof_used - 1]));
  for (int i = 0; i < p->prof_used; ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, p->prof_ev[2 * i], p->prof_ev[2 * i + 1]));
    ms[p->prof_kind[i]] += t;
    launches[p->prof_kind[i]] += 1;
  }
  p->prof_used = 0;
  return FWI_OK;
}

// ---- allocation-free adjoint source ------------------------------------------------
// Scratch for the block partial sums of the misfit: a file-scope device array, so
// callers that cannot allocate device memory can still run this stage.
static __device__ __align__(256) double g_noalloc_partials[FWI_NOALLOC_MAX_PARTIALS];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256];   // device address of the array, per device ordinal

fwi_status fwi_adjoint_source_noalloc(const float* traces, const float* observed, int32_t K,
                                      int32_t nt, int32_t n_rec, float* qcum, double* misfit,
                                      void* stream) {
  if (!traces || !observed || !qcum || !misfit || K < 1 || K > 32 || nt < 1 || n_rec < 1)
    return FWI_EINVAL;
  const int nblk = (n_rec + 255) / 256;
  if ((int64_t)K * nblk > FWI_NOALLOC_MAX_PARTIALS) return FWI_EINVAL;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return FWI_EINVAL;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // host code may not use the array's name as a device address: look it up
      void* ptr = nullptr;
      CK(cudaGetSymbolAddress(&ptr, g_noalloc_partials));
      g_noalloc_ptr[dev] = ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_misfit<<<dim3(nblk, K), 256, 0, st>>>(traces, observed, nt, n_rec, qcum, static_cast<double*>(scratch));
  k_misfit_final<<<1, 32, 0, st>>>(static_cast<const double*>(scratch), nblk, K, misfit);
  CK(cudaGetLastError());
  return FWI_OK;
}

// ---- batched form: one captured graph over several plans --------------------------------
struct fwi_batch {
  std::vector<fwi_plan*> plans;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t origin = nullptr;  // capture stream (the caller's may be the legacy default)
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> key;     // arguments the graph was captured with
  int64_t nodes = 0;
  std::vector<int> chain;         // chain of each plan; empty: one chain per plan
};

fwi_status fwi_batch_create(int32_t n, fwi_plan* const* plans, fwi_batch** out) {
  if (n < 1 || !plans || !out) return FWI_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !plans[i]->ws) return FWI_EINVAL;
    // a plan listed twice would run on two chains at once over one workspace
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return FWI_EINVAL;
  }
  fwi_batch* b = new (std::nothrow) fwi_batch();
  if (!b) return FWI_ENOMEM;
  b->plans.assign(plans, plans + n);
  b->side.resize(n);
  b->join.resize(n);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    fwi_batch_destroy(b);
    return FWI_ECUDA;
  }
  *out = b;
  return FWI_OK;
}

fwi_status fwi_batch_gradient(fwi_batch* b, const float* const* c, const float* const* w, const int32_t* K,
                              const float* const* observed, const int32_t* observed_encoded,
                              double* const* misfit, double* const* grad, void* stream) {
  if (!b || !c || !w || !K || !observed || !observed_encoded || !misfit || !grad) return FWI_EINVAL;
  const int n = (int)b->plans.size();
  std::vector<uintptr_t> key;
  for (int i = 0; i < n; ++i) {
    fwi_status s = check_call(b->plans[i], K[i]);
    if (s != FWI_OK) return s;
    key.insert(key.end(), {(uintptr_t)c[i], (uintptr_t)w[i], (uintptr_t)K[i], (uintptr_t)observed[i],
                           (uintptr_t)observed_encoded[i], (uintptr_t)misfit[i], (uintptr_t)grad[i],
                           (uintptr_t)b->plans[i]->generation});
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!b->exec || key != b->key) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    // capture on the batch's own stream: nothing runs during capture
    cudaStream_t cs = b->origin;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    fwi_status s = FWI_OK;
    if (cudaEventRecord(b->fork, cs) != cudaSuccess) s = FWI_ECUDA;
    // chain h runs its plans one after another, in batch order, on side stream h
    for (int h = 0; h < n && s == FWI_OK; ++h) {
      bool any = false;
      for (int i = 0; i < n && s == FWI_OK; ++i) {
        if ((b->chain.empty() ? i : b->chain[i]) != h) continue;
        if (!any && cudaStreamWaitEvent(b->side[h], b->fork, 0) != cudaSuccess) { s = FWI_ECUDA; break; }
        any = true;
        s = fwi_gradient(b->plans[i], c[i], w[i], K[i], observed[i], observed_encoded[i], misfit[i], grad[i],
                         nullptr, b->side[h]);
      }
      if (!any || s != FWI_OK) continue;
      if (cudaEventRecord(b->join[h], b->side[h]) != cudaSuccess) s = FWI_ECUDA;
      if (s == FWI_OK && cudaStreamWaitEvent(cs, b->join[h], 0) != cudaSuccess) s = FWI_ECUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (s != FWI_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return s != FWI_OK ? s : FWI_ECUDA;
    }
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    b->nodes = (int64_t)nn;
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      b->exec = nullptr;
      return FWI_ECUDA;
    }
    b->key = key;
  }
  for (int i = 0; i < n; ++i) {
    b->plans[i]->last = st;
    b->plans[i]->used = true;
  }
  CK(cudaGraphLaunch(b->exec, st));
  return FWI_OK;
}

int64_t fwi_batch_nodes(const fwi_batch* b) { return b ? b->nodes : -1; }

fwi_status fwi_batch_set_chains(fwi_batch* b, const int32_t* chain) {
  if (!b) return FWI_EINVAL;
  const int n = (int)b->plans.size();
  std::vector<int> ch;
  if (chain) {
    for (int i = 0; i < n; ++i)
      if (chain[i] < 0 || chain[i] >= n) return FWI_EINVAL;
    ch.assign(chain, chain + n);
  }
  if (ch != b->chain && b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->key.clear();
  }
  b->chain = ch;
  return FWI_OK;
}

fwi_status fwi_batch_destroy(fwi_batch* b) {
  if (!b) return FWI_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s : b->side)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
  return FWI_OK;
}

fwi_status fwi_plan_set_schedule(fwi_plan* p, const fwi_schedule* sc) {
  if (!p || !sc) return FWI_EINVAL;
  if (sc->specialized < 0 || sc->specialized > 2 || sc->radix_order < 0 || sc->radix_order > 2 ||
      (sc->z_tile != 16 && sc->z_tile != 32) || (sc->split_plane != 0 && sc->split_plane != 1) ||
      (sc->stream_groups != 1 && sc->stream_groups != 2 && sc->stream_groups != 4))
    return FWI_EINVAL;
  const fwi_schedule old = p->sched;
  p->sched = *sc;
  if (apply_schedule(p) != FWI_OK) {
    p->sched = old;
    apply_schedule(p);
    return FWI_ENOTSUP;
  }
  p->generation++;
  if (p->ws) set_attrs(p);
  return FWI_OK;
}

fwi_status fwi_plan_get_schedule(const fwi_plan* p, fwi_schedule* sc) {
  if (!p || !sc) return FWI_EINVAL;
  *sc = p->sched;
  return FWI_OK;
}

fwi_status fwi_plan_set_tr_box(fwi_plan* p, const int32_t origin[3], const int32_t size[3], const int32_t pml[3],
                               size_t* workspace_bytes) {
  if (!p || !origin || !size || !pml || !workspace_bytes || p->ws || p->tr_only) return FWI_EINVAL;
  const fwi_problem& q = p->prob;
  const int n[3] = {q.nx, q.ny, q.nz};
  for (int a = 0; a < 3; ++a)
    if (origin[a] < 0 || size[a] < 2 || origin[a] + size[a] > n[a] || pml[a] < 0 || 2 * pml[a] > size[a])
      return FWI_EINVAL;
  // Gamma and the boundary layer in box coordinates (cropping keeps their order); every
  // Gamma voxel must lie inside the box and outside the box's PML
  auto to_box = [&](int v, int32_t* out) {
    const int x = v % q.nx, y = (v / q.nx) % q.ny, z = v / (q.nx * q.ny);
    const int c[3] = {x - origin[0], y - origin[1], z - origin[2]};
    for (int a = 0; a < 3; ++a)
      if (c[a] < pml[a] || c[a] > size[a] - 1 - pml[a]) return false;
    *out = c[0] + size[0] * (c[1] + size[1] * c[2]);
    return true;
  };
  std::vector<int32_t> gam(q.n_gamma), lay(q.n_layer);
  for (int j = 0; j < q.n_gamma; ++j)
    if (!to_box(p->gam.vox[j], &gam[j])) return FWI_EINVAL;
  for (int j = 0; j < q.n_layer; ++j)
    if (!to_box(p->lay.vox[j], &lay[j])) return FWI_EINVAL;
  fwi_problem b = q;
  b.nx = size[0]; b.ny = size[1]; b.nz = size[2];
  for (int a = 0; a < 3; ++a) b.pml[a] = pml[a];
  // the box plan runs no forward or adjoint simulation: one placeholder transducer each
  const int32_t none = 0;
  b.n_src = b.n_rec = 1;
  b.src_idx = b.rec_idx = &none;
  b.gamma_idx = gam.data();
  b.layer_idx = lay.data();
  b.wavelet = p->wavelet.data();
  size_t sub_bytes = 0;
  fwi_plan* sub = nullptr;
  const fwi_status st = fwi_plan_create_impl(&b, true, &sub_bytes, &sub);
  if (st != FWI_OK) return st;
  if (p->tr) fwi_plan_destroy(p->tr);
  p->tr = sub;
  for (int a = 0; a < 3; ++a) p->tr_origin[a] = origin[a];
  plan_layout(p);
  *workspace_bytes = p->L.total;
  return FWI_OK;
}

fwi_status fwi_plan_destroy(fwi_plan* p) {
  if (p) {
    if (p->tr) fwi_plan_destroy(p->tr);
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    for (int g = 0; g < fwi_plan::kMaxGroups - 1; ++g) {
      if (p->side[g]) cudaStreamDestroy(p->side[g]);
      if (p->ev_join[g]) cudaEventDestroy(p->ev_join[g]);
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  }
  delete p;
  return FWI_OK;
}

}  // extern "C"
