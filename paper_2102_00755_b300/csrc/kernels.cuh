// Device kernels of one time step of the split-density k-space scheme (Alg. 1)
// and of the gradient bookkeeping around it.
//
// Per step and simulation the scheme needs 4 forward and 6 inverse 3D real
// transforms (App. B).  They are organised in four launches over batches of
// simulations that advance in lockstep:
//
//   zpass<MOM>    P_xy -> Q = IFFT_z(kappa/N FFT_z P_xy), R = IFFT_z(kappa a+_z/N FFT_z P_xy)
//   plane_mom     per z-plane: d+_xi p = IFFT_xy(a+_x Q | a+_y Q | R); v_xi update (PML);
//                 forward XY transform of the new v_xi -> V_xi,xy
//   zpass<MASS>   V_xi,xy -> IFFT_z(kappa/N FFT_z .) (x, y) and with a-_z (z)
//   plane_mass    per z-plane: d-_xi v_xi = IFFT_xy(a-_x . | a-_y . | .); rho_xi update
//                 (PML); p = c0^2 sum rho_xi; source / adjoint injection or TR
//                 Dirichlet layer; record receivers, boundary layer, Gamma;
//                 forward XY transform of p -> P_xy for the next step
//
// The x and y factors i k_xi exp(+-i k_xi dx/2) of Eq. 19 are constant along a
// z column, so they are applied in the plane kernels and the z pass only needs
// kappa (and the z factor).  Spectra are half spectra in x (hx = nx/2 + 1),
// stored as [z][ky][kx] complex FP32.  Real XY transforms pack two rows
// (y = 2p, 2p + 1) into one complex line of length nx.
#pragma once
#include <cstdint>

#include "fft_smem.cuh"

namespace fwi {

constexpr int kMaxSims = 16;
constexpr int kTpbPlane = 512;
constexpr int kTpbZ = 256;
constexpr int kZTile = 16;

enum Role : int { ROLE_FORWARD = 0, ROLE_ADJOINT = 1, ROLE_TR = 2 };

struct SimPtrs {
  float* v[3];
  float* rho[3];
  float2* spec[3];
  int role;
  int shot;
};

// Everything a step launch needs; passed by value as a __grid_constant__.
struct StepParams {
  // geometry
  int nx, ny, nz, hx, npair, nxp, hxp;
  int64_t nvox;        // nx*ny*nz
  int plane;           // nx*ny
  int mspec;           // hx*ny (spectrum plane)
  int nt;              // time samples (Nt + 1)
  int n_rec, n_layer, n_gamma, n_us, n_ur;
  AxisPlan ax, ay, az;
  const float2* tw;
  // spectral factors (FP32, built in FP64 on the host)
  const float* kx2;    // [hx]
  const float* ky2;    // [ny]
  const float* kz2;    // [nz]
  const float2* ap[3]; // a+_xi: i k exp(+i k dx/2), [hx], [ny], [nz]
  const float2* am[3]; // a-_xi
  float half_cdt;      // c_ref dt / 2
  float inv_n;         // 1 / (nx ny nz)
  // PML (1D)
  const float* lam[3];
  const float* lams[3];
  float dt_over_rho0;
  float dt_rho0;
  // model
  const float* c2;     // [nvox] c0^2
  const int* bad;      // device flag: sound speed out of range -> skip work
  // sparse, per z-plane CSR
  const int* us_ptr; const int* us_off;                 // unique emitter voxels
  const float* amp_src;                                 // [K][nt][n_us]
  const int* ur_ptr; const int* ur_off;                 // unique receiver voxels
  const int* ur_mptr; const int* ur_mem;                // members (receiver columns)
  const float* ur_coef;                                 // 2 dt / (3 dx c0)
  const float* qf;                                      // [K][nt][n_rec] cumulative residual
  const int* rr_ptr; const int* rr_off; const int* rr_col;  // receivers to record
  float* traces;                                        // [K][nt][n_rec]
  const int* lay_ptr; const int* lay_idx;               // boundary layer (sorted)
  float* ghist;                                         // [K][nt][n_layer] recorded p
  const float* inv3c2;                                  // [n_layer] 1/(3 c0^2)
  const int* gam_ptr; const int* gam_idx;               // Gamma (sorted)
  float* pa;                                            // [K][n_gamma] adjoint p on Gamma
  float* ring;                                          // [K][3][n_gamma] TR p on Gamma
  int record_layer;                                     // forward: record the layer
  // batch
  int nsims;
  SimPtrs sims[kMaxSims];
  int tidx[kMaxSims];   // forward: n; adjoint: row of Q injected; TR: m (uses g[Nt-m])
  int slot[kMaxSims];   // TR: ring slot written
};

// Plane geometry handed by value to the non-inlined helpers.
struct PlaneGeom {
  int nx, ny, hx, npair, nxp, hxp;
};
__device__ __forceinline__ PlaneGeom plane_geom(const StepParams& P) {
  PlaneGeom g;
  g.nx = P.nx; g.ny = P.ny; g.hx = P.hx; g.npair = P.npair; g.nxp = P.nxp; g.hxp = P.hxp;
  return g;
}

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float pair_get(const float2* Z, int nxp, int x, int y) {
  const float2 z = Z[(y >> 1) * nxp + x];
  return (y & 1) ? z.y : z.x;
}
__device__ __forceinline__ void pair_set(float2* Z, int nxp, int x, int y, float val) {
  float2* z = &Z[(y >> 1) * nxp + x];
  if (y & 1) z->y = val; else z->x = val;
}

// Y[ky][kx] (row stride hxp) -> Z[p][x] (row stride nxp): Hermitian extension in x
// of the two half spectra of rows 2p, 2p+1 and the pair packing Z = A + iB.
// In place, in batches of pairs taken in increasing order: pair p's output
// [p nxp, (p+1) nxp) never reaches the rows 2p', 2p'+1 (p' > p) still to be read
// because nxp <= 2 hxp.
template <int EPT>
__device__ __forceinline__ void c2r_pack(float2* sm, const PlaneGeom P) {
  const int nx = P.nx, hx = P.hx, ny = P.ny;
  const int T = blockDim.x;
  const int ppb = max(1, (EPT * T) / nx);   // pairs per batch
  for (int p0 = 0; p0 < P.npair; p0 += ppb) {
    const int total = min(ppb, P.npair - p0) * nx;
    float2 zv[EPT];
#pragma unroll
    for (int b = 0; b < EPT; ++b) {
      const int idx = threadIdx.x + b * T;
      if (idx < total) {
        const int p = p0 + idx / nx;
        const int k = idx % nx;
        const bool mir = k >= hx;
        const int kk = mir ? nx - k : k;
        float2 A = sm[(2 * p) * P.hxp + kk];
        float2 B = (2 * p + 1 < ny) ? sm[(2 * p + 1) * P.hxp + kk] : make_float2(0.f, 0.f);
        if (kk == 0 || 2 * kk == nx) { A.y = 0.f; B.y = 0.f; }
        if (mir) { A.y = -A.y; B.y = -B.y; }
        zv[b] = make_float2(A.x - B.y, A.y + B.x);
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < EPT; ++b) {
      const int idx = threadIdx.x + b * T;
      if (idx < total) sm[(p0 + idx / nx) * P.nxp + idx % nx] = zv[b];
    }
    __syncthreads();
  }
}

// Z[p][k] (after the forward x transform of rows 2p + i 2p+1) -> Y[y][kx]:
// A = (Z_k + conj Z_(N-k)) / 2, B = (Z_k - conj Z_(N-k)) / (2i).  In place, in
// batches of pairs taken in decreasing order (the mirror of c2r_pack).
template <int EPT>
__device__ __forceinline__ void r2c_unpack(float2* sm, const PlaneGeom P) {
  const int nx = P.nx, hx = P.hx, ny = P.ny;
  const int T = blockDim.x;
  constexpr int MI = (EPT + 1) / 2;
  const int ppb = max(1, (MI * T) / hx);
  for (int p1 = P.npair; p1 > 0; p1 -= ppb) {
    const int p0 = max(0, p1 - ppb);
    const int total = (p1 - p0) * hx;
    float2 av[MI], bv[MI];
#pragma unroll
    for (int b = 0; b < MI; ++b) {
      const int idx = threadIdx.x + b * T;
      if (idx < total) {
        const int p = p0 + idx / hx;
        const int k = idx % hx;
        const float2 zk = sm[p * P.nxp + k];
        const float2 zm = sm[p * P.nxp + (k == 0 ? 0 : nx - k)];
        av[b] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        bv[b] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MI; ++b) {
      const int idx = threadIdx.x + b * T;
      if (idx < total) {
        const int p = p0 + idx / hx;
        const int k = idx % hx;
        sm[(2 * p) * P.hxp + k] = av[b];
        if (2 * p + 1 < ny) sm[(2 * p + 1) * P.hxp + k] = bv[b];
      }
    }
    __syncthreads();
  }
}

// Forward XY transform of the real plane held as pairs in Z -> global spectrum plane.
template <int EPT>
__device__ void xy_forward_store(float2* sm, const StepParams& P, float2* __restrict__ dst) {
  fft_lines<false, EPT>(sm, P.npair, P.nxp, 1, P.ax, P.tw);
  r2c_unpack<EPT>(sm, plane_geom(P));
  fft_lines<false, EPT>(sm, P.hx, 1, P.hxp, P.ay, P.tw);
  const int total = P.mspec;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int ky = idx / P.hx;
    const int kx = idx - ky * P.hx;
    dst[idx] = sm[ky * P.hxp + kx];
  }
  __syncthreads();
}

// Global spectrum plane times the x (comp 0) or y (comp 1) factor, or as is
// (comp 2) -> inverse XY transform -> real plane as pairs in Z.
template <int EPT>
__device__ void xy_inverse_load(float2* sm, const StepParams& P, const float2* __restrict__ src,
                                const float2* __restrict__ fac, int comp) {
  const int total = P.mspec;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int ky = idx / P.hx;
    const int kx = idx - ky * P.hx;
    float2 v = src[idx];
    if (comp == 0) v = cmul(v, __ldg(&fac[kx]));
    else if (comp == 1) v = cmul(v, __ldg(&fac[ky]));
    sm[ky * P.hxp + kx] = v;
  }
  __syncthreads();
  fft_lines<true, EPT>(sm, P.hx, 1, P.hxp, P.ay, P.tw);
  c2r_pack<EPT>(sm, plane_geom(P));
  fft_lines<true, EPT>(sm, P.npair, P.nxp, 1, P.ax, P.tw);
}

__device__ __forceinline__ size_t plane_smem_elems(const StepParams& P) {
  const int a = P.npair * P.nxp, b = P.ny * P.hxp;
  return (size_t)(a > b ? a : b);
}

// ------------------------------------------------------------------ z pass
// MODE 0 (momentum): in spec[0] -> spec[0] = Q, spec[1] = R.
// MODE 1 (mass): spec[2] (x), spec[0] (y), spec[1] (z) in place.
template <int MODE, int EPT>
__global__ void __launch_bounds__(kTpbZ) k_zpass(const __grid_constant__ StepParams P) {
  if (*P.bad) return;
  extern __shared__ float2 zsm[];
  const SimPtrs& S = P.sims[blockIdx.y];
  constexpr int NSL = MODE == 0 ? 2 : 3;   // slots held in shared memory
  constexpr int RS = NSL * kZTile;         // row stride (complex)
  const int m0 = blockIdx.x * kZTile;
  const int M = P.mspec;
  const int nz = P.nz;
  const size_t zstride = (size_t)M;
  // load
  const int nin = MODE == 0 ? 1 : 3;
  for (int idx = threadIdx.x; idx < nin * nz * kZTile; idx += blockDim.x) {
    const int ml = idx % kZTile;
    const int t = idx / kZTile;
    const int z = t % nz;
    const int s = t / nz;
    const float2* src = MODE == 0 ? S.spec[0] : (s == 0 ? S.spec[2] : (s == 1 ? S.spec[0] : S.spec[1]));
    const int m = m0 + ml;
    zsm[z * RS + s * kZTile + ml] = (m < M) ? src[(size_t)z * zstride + m] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_lines<false, EPT>(zsm, nin * kZTile, 1, RS, P.az, P.tw);
  // multiply by kappa / N (and the z factor)
  for (int idx = threadIdx.x; idx < nz * kZTile; idx += blockDim.x) {
    const int ml = idx % kZTile;
    const int z = idx / kZTile;
    const int m = m0 + ml;
    if (m >= M) continue;
    const int ky = m / P.hx;
    const int kx = m - ky * P.hx;
    const float kk = __ldg(&P.kx2[kx]) + __ldg(&P.ky2[ky]) + __ldg(&P.kz2[z]);
    const float a = P.half_cdt * sqrtf(kk);
    const float kap = (a > 0.f ? sinf(a) / a : 1.f) * P.inv_n;
    if (MODE == 0) {
      const float2 v = zsm[z * RS + ml];
      zsm[z * RS + ml] = cscale(v, kap);
      zsm[z * RS + kZTile + ml] = cmul(cscale(v, kap), __ldg(&P.ap[2][z]));
    } else {
      zsm[z * RS + ml] = cscale(zsm[z * RS + ml], kap);
      zsm[z * RS + kZTile + ml] = cscale(zsm[z * RS + kZTile + ml], kap);
      zsm[z * RS + 2 * kZTile + ml] = cmul(cscale(zsm[z * RS + 2 * kZTile + ml], kap), __ldg(&P.am[2][z]));
    }
  }
  __syncthreads();
  fft_lines<true, EPT>(zsm, NSL * kZTile, 1, RS, P.az, P.tw);
  for (int idx = threadIdx.x; idx < NSL * nz * kZTile; idx += blockDim.x) {
    const int ml = idx % kZTile;
    const int t = idx / kZTile;
    const int z = t % nz;
    const int s = t / nz;
    const int m = m0 + ml;
    if (m >= M) continue;
    float2* dst = MODE == 0 ? (s == 0 ? S.spec[0] : S.spec[1])
                            : (s == 0 ? S.spec[2] : (s == 1 ? S.spec[0] : S.spec[1]));
    dst[(size_t)z * zstride + m] = zsm[z * RS + s * kZTile + ml];
  }
}

// ------------------------------------------------------------------ momentum plane
template <int EPT>
__global__ void __launch_bounds__(kTpbPlane, 1) k_plane_mom(const __grid_constant__ StepParams P) {
  if (*P.bad) return;
  extern __shared__ float2 sm[];
  const int z = blockIdx.x;
  const SimPtrs& S = P.sims[blockIdx.y];
  const size_t soff = (size_t)z * P.mspec;
  const size_t voff = (size_t)z * P.plane;
  const int nx = P.nx, ny = P.ny;
  // component order z, x, y: R -> V_z (same buffer), Q -> V_x (spec[2]), Q -> V_y (spec[0])
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = cc == 0 ? 2 : cc - 1;
    const float2* src = (comp == 2 ? S.spec[1] : S.spec[0]) + soff;
    float2* dst = (comp == 2 ? S.spec[1] : (comp == 0 ? S.spec[2] : S.spec[0])) + soff;
    xy_inverse_load<EPT>(sm, P, src, P.ap[comp], comp);
    // v_xi <- Lambda^s (Lambda^s v_xi - dt/rho0 d+_xi p)
    float* v = S.v[comp] + voff;
    const float* lam = P.lams[comp];
    const float lz = __ldg(&lam[comp == 2 ? z : 0]);
    const int total = P.npair * nx;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int p = idx / nx;
      const int x = idx - p * nx;
      const float2 d = sm[p * P.nxp + x];
      const int y0 = 2 * p, y1 = 2 * p + 1;
      float l0, l1;
      if (comp == 0) { l0 = l1 = __ldg(&lam[x]); }
      else if (comp == 1) { l0 = __ldg(&lam[y0]); l1 = (y1 < ny) ? __ldg(&lam[y1]) : 1.f; }
      else { l0 = l1 = lz; }
      const float v0 = l0 * (l0 * v[y0 * nx + x] - P.dt_over_rho0 * d.x);
      float v1 = 0.f;
      v[y0 * nx + x] = v0;
      if (y1 < ny) {
        v1 = l1 * (l1 * v[y1 * nx + x] - P.dt_over_rho0 * d.y);
        v[y1 * nx + x] = v1;
      }
      sm[p * P.nxp + x] = make_float2(v0, v1);
    }
    __syncthreads();
    xy_forward_store<EPT>(sm, P, dst);
  }
}

// ------------------------------------------------------------------ mass plane
template <int EPT>
__global__ void __launch_bounds__(kTpbPlane, 1) k_plane_mass(const __grid_constant__ StepParams P) {
  if (*P.bad) return;
  extern __shared__ float2 sm[];
  float* ssum = reinterpret_cast<float*>(sm + plane_smem_elems(P));   // [ny][nx] sum rho
  const int z = blockIdx.x;
  const SimPtrs& S = P.sims[blockIdx.y];
  const int role = S.role;
  const int shot = S.shot;
  const int tix = P.tidx[blockIdx.y];
  const size_t soff = (size_t)z * P.mspec;
  const size_t voff = (size_t)z * P.plane;
  const int nx = P.nx, ny = P.ny;
  const int total = P.npair * nx;
  // component order x (spec[2]), z (spec[1]), y (spec[0])
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = cc == 0 ? 0 : (cc == 1 ? 2 : 1);
    const float2* src = (comp == 0 ? S.spec[2] : (comp == 2 ? S.spec[1] : S.spec[0])) + soff;
    xy_inverse_load<EPT>(sm, P, src, P.am[comp], comp);
    // rho_xi <- Lambda (Lambda rho_xi - dt rho0 d-_xi v_xi)
    float* rho = S.rho[comp] + voff;
    const float* lam = P.lam[comp];
    const float lz = __ldg(&lam[comp == 2 ? z : 0]);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int p = idx / nx;
      const int x = idx - p * nx;
      const float2 d = sm[p * P.nxp + x];
      const int y0 = 2 * p, y1 = 2 * p + 1;
      float l0, l1;
      if (comp == 0) { l0 = l1 = __ldg(&lam[x]); }
      else if (comp == 1) { l0 = __ldg(&lam[y0]); l1 = (y1 < ny) ? __ldg(&lam[y1]) : 1.f; }
      else { l0 = l1 = lz; }
      const float r0 = l0 * (l0 * rho[y0 * nx + x] - P.dt_rho0 * d.x);
      rho[y0 * nx + x] = r0;
      ssum[y0 * nx + x] = (cc == 0) ? r0 : ssum[y0 * nx + x] + r0;
      if (y1 < ny) {
        const float r1 = l1 * (l1 * rho[y1 * nx + x] - P.dt_rho0 * d.y);
        rho[y1 * nx + x] = r1;
        ssum[y1 * nx + x] = (cc == 0) ? r1 : ssum[y1 * nx + x] + r1;
      }
    }
    __syncthreads();
  }
  // sparse updates of rho_xi on this plane: injection or the TR Dirichlet layer
  const float* c2 = P.c2 + voff;
  if (role == ROLE_FORWARD) {
    const float* amp = P.amp_src + ((size_t)shot * P.nt + tix) * P.n_us;
    for (int u = P.us_ptr[z] + threadIdx.x; u < P.us_ptr[z + 1]; u += blockDim.x) {
      const int off = P.us_off[u];
      const float a = amp[u];
      for (int c = 0; c < 3; ++c) S.rho[c][voff + off] += a;
      ssum[off] += 3.f * a;
    }
  } else if (role == ROLE_ADJOINT) {
    const float* q = P.qf + ((size_t)shot * P.nt + tix) * P.n_rec;
    for (int u = P.ur_ptr[z] + threadIdx.x; u < P.ur_ptr[z + 1]; u += blockDim.x) {
      float s = 0.f;
      for (int e = P.ur_mptr[u]; e < P.ur_mptr[u + 1]; ++e) s += q[P.ur_mem[e]];
      const float a = P.ur_coef[u] * s;
      const int off = P.ur_off[u];
      for (int c = 0; c < 3; ++c) S.rho[c][voff + off] += a;
      ssum[off] += 3.f * a;
    }
  } else {  // TR: rho_xi(layer) <- g^(Nt - m) / (3 c0^2)
    const float* g = P.ghist + ((size_t)shot * P.nt + (P.nt - 1 - tix)) * P.n_layer;
    for (int j = P.lay_ptr[z] + threadIdx.x; j < P.lay_ptr[z + 1]; j += blockDim.x) {
      const int off = (int)(P.lay_idx[j] - voff);
      const float val = g[j] * P.inv3c2[j];
      for (int c = 0; c < 3; ++c) S.rho[c][voff + off] = val;
      ssum[off] = 3.f * val;
    }
  }
  __syncthreads();
  // p = c0^2 (rho_x + rho_y + rho_z), as pairs in Z
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int p = idx / nx;
    const int x = idx - p * nx;
    const int y0 = 2 * p, y1 = 2 * p + 1;
    const float p0 = c2[y0 * nx + x] * ssum[y0 * nx + x];
    const float p1 = (y1 < ny) ? c2[y1 * nx + x] * ssum[y1 * nx + x] : 0.f;
    sm[p * P.nxp + x] = make_float2(p0, p1);
  }
  __syncthreads();
  // recording
  if (role == ROLE_FORWARD) {
    float* f = P.traces + ((size_t)shot * P.nt + tix) * P.n_rec;
    for (int e = P.rr_ptr[z] + threadIdx.x; e < P.rr_ptr[z + 1]; e += blockDim.x) {
      const int off = P.rr_off[e];
      f[P.rr_col[e]] = pair_get(sm, P.nxp, off % nx, off / nx);
    }
    if (P.record_layer) {
      float* g = P.ghist + ((size_t)shot * P.nt + tix) * P.n_layer;
      for (int j = P.lay_ptr[z] + threadIdx.x; j < P.lay_ptr[z + 1]; j += blockDim.x) {
        const int off = (int)(P.lay_idx[j] - voff);
        g[j] = pair_get(sm, P.nxp, off % nx, off / nx);
      }
    }
  } else {
    float* out = role == ROLE_ADJOINT ? P.pa + (size_t)shot * P.n_gamma
                                      : P.ring + ((size_t)shot * 3 + P.slot[blockIdx.y]) * P.n_gamma;
    for (int j = P.gam_ptr[z] + threadIdx.x; j < P.gam_ptr[z + 1]; j += blockDim.x) {
      const int off = (int)(P.gam_idx[j] - voff);
      out[j] = pair_get(sm, P.nxp, off % nx, off / nx);
    }
  }
  __syncthreads();
  xy_forward_store<EPT>(sm, P, S.spec[0] + soff);
}

// TR initial value: p(layer) <- g^Nt, zero elsewhere; ring slot 0 <- p(Gamma);
// P_xy <- forward XY transform of that p.  State fields are zeroed by the host.
template <int EPT>
__global__ void __launch_bounds__(kTpbPlane, 1) k_tr_init(const __grid_constant__ StepParams P) {
  if (*P.bad) return;
  extern __shared__ float2 sm[];
  const int z = blockIdx.x;
  const SimPtrs& S = P.sims[blockIdx.y];
  const int shot = S.shot;
  const size_t voff = (size_t)z * P.plane;
  const int nx = P.nx;
  const int total = P.npair * P.nxp;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) sm[idx] = make_float2(0.f, 0.f);
  __syncthreads();
  const float* g = P.ghist + ((size_t)shot * P.nt + (P.nt - 1)) * P.n_layer;
  for (int j = P.lay_ptr[z] + threadIdx.x; j < P.lay_ptr[z + 1]; j += blockDim.x) {
    const int off = (int)(P.lay_idx[j] - voff);
    pair_set(sm, P.nxp, off % nx, off / nx, g[j]);
  }
  __syncthreads();
  float* out = P.ring + ((size_t)shot * 3 + 0) * P.n_gamma;
  for (int j = P.gam_ptr[z] + threadIdx.x; j < P.gam_ptr[z + 1]; j += blockDim.x) {
    const int off = (int)(P.gam_idx[j] - voff);
    out[j] = pair_get(sm, P.nxp, off % nx, off / nx);
  }
  __syncthreads();
  xy_forward_store<EPT>(sm, P, S.spec[0] + (size_t)z * P.mspec);
}

}  // namespace fwi
