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
// stored as [z][ky][kx] complex FP32.
//
// Shared-memory plane layout.  The plane buffer holds npair = ceil(ny/2) regions
// of 2*hx complex values.  Seen as a spectrum it is Y[ky][kx] with row stride hx
// (rows 2p and 2p+1 fill region p); seen as real data it is Z[p][x], the complex
// line of length nx packing rows 2p (real part) and 2p+1 (imaginary part) of a
// real plane, stored at the start of region p.  Because both views of a pair of
// rows occupy the same region, the C2R/R2C repacking, the x transforms, the field
// updates and all per-voxel sparse work of a pair of rows are done by the one
// warp that owns it, with __syncwarp only; block barriers separate the y
// transforms (columns) from the x work (rows).
#pragma once
#include <cstdint>

#include "fft_smem.cuh"

namespace fwi {

constexpr int kMaxSims = 16;
constexpr int kTpbPlane = 256;
constexpr int kTpbZ = 256;

enum Role : int { ROLE_FORWARD = 0, ROLE_ADJOINT = 1, ROLE_TR = 2 };

// Slots of the ring that holds the TR pressure on Gamma, P(m) in slot m % kRing.  The
// accumulation of an iteration reads P(it), P(it+1), P(it+2) while the same launch's TR
// simulations of the next iteration write P(it+3): four slots keep them apart.
constexpr int kRing = 4;

struct SimPtrs {
  float* v[3];
  float* rho[3];
  float2* spec[3];
  int role;
  int shot;
  int model;           // sound-speed model of this simulation (0 unless each shot has its own)
};

// Everything a step launch needs; passed by value as a __grid_constant__.
// Sparse lists are CSR over the key z * npair + p (the pair of rows 2p, 2p+1 of
// plane z); each entry carries the voxel index and pf = 4 hx (y/2) + 2x + (y & 1),
// the float offset of voxel (x, y) in the plane buffer viewed as pair lines.
struct StepParams {
  // geometry
  int nx, ny, nz, hx, npair;
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
  int kappa_series;    // 1: c_ref dt |k| / 2 <= 3.1 everywhere, kappa from the sinc series in s = a^2
  float inv_n;         // 1 / (nx ny nz)
  // PML (1D)
  const float* lam[3];
  const float* lams[3];
  float dt_over_rho0;
  float dt_rho0;
  // model
  const float* c2;     // [nvox] c0^2
  const int* bad;      // device flag: sound speed out of range -> skip work
  // sparse lists, CSR per pair line
  const int* us_ptr; const int* us_vox; const int* us_pf;  // unique emitter voxels
  const float* amp_src;                                    // [K][nt][n_us]
  const int* ur_ptr; const int* ur_vox; const int* ur_pf;  // unique receiver voxels
  const int* ur_mptr; const int* ur_mem;                   // members (receiver columns)
  const float* ur_coef;                                    // 2 dt / (3 dx c0)
  const float* qf;                                         // [K][nt][n_rec] cumulative residual
  const int* rr_ptr; const int* rr_pf; const int* rr_col;  // receivers to record
  float* traces;                                           // [K][nt][n_rec]
  const int* lay_ptr; const int* lay_vox; const int* lay_pf;  // boundary layer (sorted)
  float* ghist;                                            // [K][nt][n_layer] recorded p
  const float* inv3c2;                                     // [n_layer] 1/(3 c0^2)
  const int* gam_ptr; const int* gam_pf;                   // Gamma (sorted)
  float* pa;                                               // [K][n_gamma] adjoint p on Gamma
  float* ring;                                             // [K][kRing][n_gamma] TR p on Gamma
  int record_layer;                                        // forward: record the layer
  // Gradient accumulation of the previous iteration, done by the adjoint-role mass
  // kernel before it overwrites pa (two-step kernels only): acc[k][j] += coefG[j]
  // (P(s0) - 2 P(s1) + P(s2))[j] pa_old[k][j] in FP64, ring slots acc_slot[0..2].
  double* acc;                                             // [K][n_gamma]
  const float* coefG;                                      // [n_gamma] 2 / (dt c0^3)
  int acc_prev;                                            // 1: accumulate before writing pa
  int acc_slot[3];
  // batch
  int nsims;
  SimPtrs sims[kMaxSims];
  int tidx[kMaxSims];   // forward: n; adjoint: row of Q injected; TR: m (uses g[Nt-m])
  int slot[kMaxSims];   // TR: ring slot written
};

// Per-model arrays ([models][n], contiguous; one model unless each super-shot has its own):
// c0^2 on the grid and the sound-speed dependent coefficients at the sparse voxels.
__device__ __forceinline__ const float* c2_of(const StepParams& P, const SimPtrs& Q) {
  return P.c2 + (size_t)Q.model * P.nvox;
}
__device__ __forceinline__ const float* ur_coef_of(const StepParams& P, const SimPtrs& Q) {
  return P.ur_coef + (size_t)Q.model * P.n_ur;
}
__device__ __forceinline__ const float* inv3c2_of(const StepParams& P, const SimPtrs& Q) {
  return P.inv3c2 + (size_t)Q.model * P.n_layer;
}
__device__ __forceinline__ const float* coefG_of(const StepParams& P, const SimPtrs& Q) {
  return P.coefG + (size_t)Q.model * P.n_gamma;
}

// ------------------------------------------------------------------ helpers
// Asynchronous global -> shared copies (cp.async): a thread issues all its copies
// of a phase, then waits once, so the DRAM latency is paid once per phase.
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Shared memory of a plane kernel: twiddles of x and y, then the plane buffer,
// then per-warp staging for the state rows of the pair lines being worked on.
__device__ __forceinline__ float2* stage_twiddles(float2* sm, const StepParams& P) {
  const int n = P.ax.n + P.ay.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = P.tw[P.ax.tw_off + i];
  return sm + ((n + 31) & ~31);
}

// Pair lines p0 .. p0+nl-1 as C2R input: Y rows 2p, 2p+1 -> Z[p] (Hermitian
// extension in x, Z = A + iB, DC and Nyquist bins made real).  One warp.
template <int PI>
__device__ __forceinline__ void warp_c2r_pack(float2* reg, int nl, int nx, int hx, int ny, int p0,
                                              int lane) {
  const int tot = nl * nx;
  const float rnx = 1.0f / (float)nx;
  float2 zv[PI];
#pragma unroll
  for (int i = 0; i < PI; ++i) {
    const int b = lane + 32 * i;
    if (b < tot) {
      const int l = fdivi(b, rnx);
      const int k = b - l * nx;
      const bool mir = k >= hx;
      const int kk = mir ? nx - k : k;
      const float2* R0 = reg + l * 2 * hx;
      float2 A = R0[kk];
      float2 B = (2 * (p0 + l) + 1 < ny) ? R0[hx + kk] : make_float2(0.f, 0.f);
      if (kk == 0 || 2 * kk == nx) { A.y = 0.f; B.y = 0.f; }
      if (mir) { A.y = -A.y; B.y = -B.y; }
      zv[i] = make_float2(A.x - B.y, A.y + B.x);
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < PI; ++i) {
    const int b = lane + 32 * i;
    if (b < tot) {
      const int l = fdivi(b, rnx);
      reg[l * 2 * hx + (b - l * nx)] = zv[i];
    }
  }
  __syncwarp();
}

// Z[p] after the forward x transform -> Y rows 2p, 2p+1:
// A = (Z_k + conj Z_(N-k)) / 2, B = (Z_k - conj Z_(N-k)) / (2i).  One warp.
template <int MI>
__device__ __forceinline__ void warp_r2c_unpack(float2* reg, int nl, int nx, int hx, int ny, int p0,
                                                int lane) {
  const int tot = nl * hx;
  const float rhx = 1.0f / (float)hx;
  float2 av[MI], bv[MI];
#pragma unroll
  for (int i = 0; i < MI; ++i) {
    const int b = lane + 32 * i;
    if (b < tot) {
      const int l = fdivi(b, rhx);
      const int k = b - l * hx;
      const float2* Z = reg + l * 2 * hx;
      const float2 zk = Z[k];
      const float2 zm = Z[k == 0 ? 0 : nx - k];
      av[i] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      bv[i] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < MI; ++i) {
    const int b = lane + 32 * i;
    if (b < tot) {
      const int l = fdivi(b, rhx);
      const int k = b - l * hx;
      float2* R0 = reg + l * 2 * hx;
      R0[k] = av[i];
      if (2 * (p0 + l) + 1 < ny) R0[hx + k] = bv[i];
    }
  }
  __syncwarp();
}

// Prefetch rows 2 p0 .. 2 (p0 + nl) - 1 (clipped to ny) of a plane array into the
// warp's staging area (row-major, nx floats per row).  Asynchronous: wait with
// cp_async_wait_all() and __syncwarp() before reading.
__device__ __forceinline__ void warp_prefetch_rows(float* stage, const float* __restrict__ plane, int p0,
                                                   int nl, int nx, int ny, int lane) {
  const int y0 = 2 * p0;
  const int rows = min(2 * nl, ny - y0);
  const int tot = rows * nx;
  const float* src = plane + (size_t)y0 * nx;
  for (int i = lane; i < tot; i += 32) cp_async4(&stage[i], &src[i]);
}

// Compile-time configuration of the plane kernels.  FX, FY > 0: specialised
// transforms for nx = FX, ny = FY; 0: runtime radix schedules with EPL values
// staged per lane.  GX pair lines (x work) and GY columns (y transforms) per warp
// group; PI / UI: per-lane staging of the C2R packing / R2C unpacking.  XW = 256
// is the x work budget per group (pair lines * nx); the mass kernel halves it to
// keep its four staged state arrays small.
__host__ __device__ constexpr int pow2_floor(int v) { return v <= 1 ? 1 : 2 * pow2_floor(v / 2); }

template <int EPL, int FX, int FY, int XW = 256>
struct PlaneCfg {
  static constexpr int GXc = FX > 0 ? pow2_floor(XW / FX) : 0;
  static constexpr int GYc = FY > 0 ? pow2_floor(256 / FY) : 0;
  static constexpr int PI = FX > 0 ? (GXc * FX + 31) / 32 : EPL;
  // runtime path: a lone line of nx = 32 EPL has hx = 16 EPL + 1 bins
  static constexpr int UI = FX > 0 ? (GXc * (FX / 2 + 1) + 31) / 32 : EPL / 2 + 1;
  __device__ static int gx(const StepParams& P) {
    if (FX > 0) return GXc;
    const int g = XW * EPL / (16 * P.hx);   // group * 2 hx <= XW EPL / 8 <= 32 EPL
    return g < 1 ? 1 : g;
  }
  __device__ static int gy(const StepParams& P) { return FY > 0 ? GYc : lines_per_group<EPL>(P.ny); }
  template <bool INV>
  __device__ static void fft_x(float2* reg, int nl, const StepParams& P, const float2* twx, int lane) {
    if constexpr (FX > 0) ct_fft_n<FX, INV, GXc, false>(reg, nl, 2 * P.hx, 1, P.ax, twx, lane);
    else warp_fft<INV, EPL>(reg, nl, 2 * P.hx, 1, P.ax, twx, lane);
  }
  template <bool INV>
  __device__ static void fft_y(float2* col, int nl, const StepParams& P, const float2* twy, int lane) {
    if constexpr (FY > 0) ct_fft_n<FY, INV, GYc, true>(col, nl, 1, P.hx, P.ay, twy, lane);
    else warp_fft<INV, EPL>(col, nl, 1, P.hx, P.ay, twy, lane);
  }
};

// Block: global spectrum plane -> Y (asynchronous copies), times the x (comp 0)
// or y (comp 1) factor or as is (comp 2); barrier; inverse y transforms (warp
// groups of columns); barrier.
template <class C>
__device__ __forceinline__ void load_and_inverse_y(float2* sm, const float2* twy, const StepParams& P,
                                                   const float2* __restrict__ src,
                                                   const float2* __restrict__ fac, int comp) {
  const int total = P.mspec;
  const float rhx = 1.0f / (float)P.hx;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) cp_async8(&sm[idx], &src[idx]);
  cp_async_wait_all();
  if (comp < 2) {
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int ky = fdivi(idx, rhx);
      const int kx = idx - ky * P.hx;
      sm[idx] = cmul(sm[idx], __ldg(&fac[comp == 0 ? kx : ky]));
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = C::gy(P);
  for (int c0 = warp * G; c0 < P.hx; c0 += nw * G)
    C::template fft_y<true>(sm + c0, min(G, P.hx - c0), P, twy, lane);
  __syncthreads();
}

// Block: forward y transforms (warp groups of columns); barrier; Y -> global; barrier.
template <class C>
__device__ __forceinline__ void forward_y_and_store(float2* sm, const float2* twy, const StepParams& P,
                                                    float2* __restrict__ dst) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = C::gy(P);
  for (int c0 = warp * G; c0 < P.hx; c0 += nw * G)
    C::template fft_y<false>(sm + c0, min(G, P.hx - c0), P, twy, lane);
  __syncthreads();
  for (int idx = threadIdx.x; idx < P.mspec; idx += blockDim.x) dst[idx] = sm[idx];
  __syncthreads();
}

// ------------------------------------------------------------------ z pass
// MODE 0 (momentum): in spec[0] -> spec[0] = Q, spec[1] = R.
// MODE 1 (mass): spec[2] (x), spec[0] (y), spec[1] (z) in place.
// A CTA holds TZ adjacent (ky, kx) columns of every slot for all z; the row
// stride RS = slots * TZ + 4 keeps the lanes of a warp (adjacent columns, then
// z) on distinct banks.  FZ > 0: specialised z transforms (nz = FZ).
template <int EPL, int FZ, int TZc>
struct ZCfg {
  static constexpr int TZ = TZc;
  static constexpr int GZc = FZ > 0 ? pow2_floor(256 / FZ < 32 ? 256 / FZ : 32) : 0;
  __device__ static int gz(int nz) { return FZ > 0 ? GZc : min(lines_per_group<EPL>(nz), TZ); }
  template <bool INV>
  __device__ static void fft_z(float2* col, int nl, int rs, const StepParams& P, const float2* twz,
                               int lane) {
    if constexpr (FZ > 0) ct_fft_n<FZ, INV, GZc, true>(col, nl, 1, rs, P.az, twz, lane);
    else warp_fft<INV, EPL>(col, nl, 1, rs, P.az, twz, lane);
  }
};

template <int MODE, int EPL, int FZ, int TZc>
__global__ void __launch_bounds__(kTpbZ, 2) k_zpass(const __grid_constant__ StepParams P) {
  if (*P.bad) return;
  using C = ZCfg<EPL, FZ, TZc>;
  constexpr int TZ = C::TZ;
  extern __shared__ float2 zsm_raw[];
  const SimPtrs& S = P.sims[blockIdx.y];
  constexpr int NSL = MODE == 0 ? 2 : 3;   // slots held in shared memory
  constexpr int RS = NSL * TZ + 4;         // row stride (complex)
  const int nz = FZ > 0 ? FZ : P.nz;
  float2* twz = zsm_raw;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) twz[i] = P.tw[P.az.tw_off + i];
  float2* zsm = zsm_raw + ((nz + 31) & ~31);
  const int m0 = blockIdx.x * TZ;
  const int M = P.mspec;
  const size_t zstride = (size_t)M;
  const int nin = MODE == 0 ? 1 : 3;
  for (int idx = threadIdx.x; idx < nin * nz * TZ; idx += blockDim.x) {
    const int ml = idx % TZ;
    const int t = idx / TZ;
    const int s = t / nz;
    const int z = t - s * nz;
    const float2* src = MODE == 0 ? S.spec[0] : (s == 0 ? S.spec[2] : (s == 1 ? S.spec[0] : S.spec[1]));
    const int m = m0 + ml;
    if (m < M) cp_async8(&zsm[z * RS + s * TZ + ml], &src[(size_t)z * zstride + m]);
    else zsm[z * RS + s * TZ + ml] = make_float2(0.f, 0.f);
  }
  cp_async_wait_all();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = C::gz(nz);
  // warp w takes groups of G columns of one slot: forward z, kappa (and z factor), inverse z
  const int gps = (TZ + G - 1) / G;   // groups per slot
  for (int g = warp; g < nin * gps; g += nw) {
    const int s = g / gps;
    const int c0 = (g - s * gps) * G;
    const int nl = min(G, TZ - c0);
    float2* col = zsm + s * TZ + c0;
    C::template fft_z<false>(col, nl, RS, P, twz, lane);
    for (int e = lane; e < nl * nz; e += 32) {
      const int z = e / nl;
      const int l = e - z * nl;
      const int m = m0 + c0 + l;
      if (m >= M) continue;
      const int ky = m / P.hx;
      const int kx = m - ky * P.hx;
      const float kk = __ldg(&P.kx2[kx]) + __ldg(&P.ky2[ky]) + __ldg(&P.kz2[z]);
      const float a = P.half_cdt * sqrtf(kk);
      const float kap = (a > 0.f ? sinf(a) / a : 1.f) * P.inv_n;
      float2* q = &col[z * RS + l];
      const float2 v = cscale(*q, kap);
      if (MODE == 0) {
        *q = v;
        col[z * RS + TZ + l] = cmul(v, __ldg(&P.ap[2][z]));
      } else {
        *q = (s == 2) ? cmul(v, __ldg(&P.am[2][z])) : v;
      }
    }
    __syncwarp();
    C::template fft_z<true>(col, nl, RS, P, twz, lane);
    if (MODE == 0) C::template fft_z<true>(col + TZ, nl, RS, P, twz, lane);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NSL * nz * TZ; idx += blockDim.x) {
    const int ml = idx % TZ;
    const int t = idx / TZ;
    const int s = t / nz;
    const int z = t - s * nz;
    const int m = m0 + ml;
    if (m >= M) continue;
    float2* dst = MODE == 0 ? (s == 0 ? S.spec[0] : S.spec[1])
                            : (s == 0 ? S.spec[2] : (s == 1 ? S.spec[0] : S.spec[1]));
    dst[(size_t)z * zstride + m] = zsm[z * RS + s * TZ + ml];
  }
}

// ------------------------------------------------------------------ momentum plane
template <int EPL, int FX, int FY>
__global__ void __launch_bounds__(kTpbPlane, 2) k_plane_mom(const __grid_constant__ StepParams P) {
  using C = PlaneCfg<EPL, FX, FY>;
  if (*P.bad) return;
  extern __shared__ float2 sm_raw[];
  const float2* twx = sm_raw;
  const float2* twy = sm_raw + P.ax.n;
  float2* sm = stage_twiddles(sm_raw, P);
  const int stage_n = 2 * C::gx(P) * P.nx;          // floats per warp and array
  float* stage = reinterpret_cast<float*>(sm + P.npair * 2 * P.hx) + (threadIdx.x >> 5) * stage_n;
  const int z = blockIdx.x;
  const SimPtrs& S = P.sims[blockIdx.y];
  const size_t soff = (size_t)z * P.mspec;
  const size_t voff = (size_t)z * P.plane;
  const int nx = P.nx, ny = P.ny, hx = P.hx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = C::gx(P);
  // component order z, x, y: R -> V_z (same buffer), Q -> V_x (spec[2]), Q -> V_y (spec[0])
#pragma unroll 1
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = cc == 0 ? 2 : cc - 1;
    const float2* src = (comp == 2 ? S.spec[1] : S.spec[0]) + soff;
    float2* dst = (comp == 2 ? S.spec[1] : (comp == 0 ? S.spec[2] : S.spec[0])) + soff;
    load_and_inverse_y<C>(sm, twy, P, src, P.ap[comp], comp);
    float* v = S.v[comp] + voff;
    const float* lam = P.lams[comp];
    const float lz = __ldg(&lam[comp == 2 ? z : 0]);
    for (int p0 = warp * G; p0 < P.npair; p0 += nw * G) {
      const int nl = min(G, P.npair - p0);
      float2* reg = sm + p0 * 2 * hx;
      warp_prefetch_rows(stage, v, p0, nl, nx, ny, lane);       // overlaps the x transform
      warp_c2r_pack<C::PI>(reg, nl, nx, hx, ny, p0, lane);
      C::template fft_x<true>(reg, nl, P, twx, lane);
      cp_async_wait_all();
      __syncwarp();
      // v_xi <- Lambda^s (Lambda^s v_xi - dt/rho0 d+_xi p), then back into Z for the forward x FFT
      for (int l = 0; l < nl; ++l) {
        const int y0 = 2 * (p0 + l), y1 = y0 + 1;
        float2* Z = reg + l * 2 * hx;
        const float* s0 = stage + (2 * l) * nx;
        for (int x = lane; x < nx; x += 32) {
          const float2 d = Z[x];
          float l0, l1;
          if (comp == 0) { l0 = l1 = __ldg(&lam[x]); }
          else if (comp == 1) { l0 = __ldg(&lam[y0]); l1 = (y1 < ny) ? __ldg(&lam[y1]) : 1.f; }
          else { l0 = l1 = lz; }
          const float v0 = l0 * (l0 * s0[x] - P.dt_over_rho0 * d.x);
          v[y0 * nx + x] = v0;
          float v1 = 0.f;
          if (y1 < ny) {
            v1 = l1 * (l1 * s0[nx + x] - P.dt_over_rho0 * d.y);
            v[y1 * nx + x] = v1;
          }
          Z[x] = make_float2(v0, v1);
        }
      }
      __syncwarp();
      C::template fft_x<false>(reg, nl, P, twx, lane);
      warp_r2c_unpack<C::UI>(reg, nl, nx, hx, ny, p0, lane);
    }
    __syncthreads();
    forward_y_and_store<C>(sm, twy, P, dst);
  }
}

// ------------------------------------------------------------------ mass plane
template <int EPL, int FX, int FY>
__global__ void __launch_bounds__(kTpbPlane, 2) k_plane_mass(const __grid_constant__ StepParams P) {
  using C = PlaneCfg<EPL, FX, FY, 128>;
  if (*P.bad) return;
  extern __shared__ float2 sm_raw[];
  const float2* twx = sm_raw;
  const float2* twy = sm_raw + P.ax.n;
  float2* sm = stage_twiddles(sm_raw, P);
  const int stage_n = 2 * C::gx(P) * P.nx;          // floats per warp and array
  float* stage = reinterpret_cast<float*>(sm + P.npair * 2 * P.hx) + (threadIdx.x >> 5) * 4 * stage_n;
  const int z = blockIdx.x;
  const SimPtrs& S = P.sims[blockIdx.y];
  const int role = S.role;
  const int shot = S.shot;
  const int tix = P.tidx[blockIdx.y];
  const size_t soff = (size_t)z * P.mspec;
  const size_t voff = (size_t)z * P.plane;
  const int nx = P.nx, ny = P.ny, hx = P.hx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = C::gx(P);
  const float* c2 = c2_of(P, S) + voff;
  const float* rx = S.rho[0] + voff;
  const float* rz = S.rho[2] + voff;
  // component order x (spec[2]), z (spec[1]), y (spec[0]); the last one assembles p
#pragma unroll 1
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = cc == 0 ? 0 : (cc == 1 ? 2 : 1);
    const float2* src = (comp == 0 ? S.spec[2] : (comp == 2 ? S.spec[1] : S.spec[0])) + soff;
    load_and_inverse_y<C>(sm, twy, P, src, P.am[comp], comp);
    float* rho = S.rho[comp] + voff;
    const float* lam = P.lam[comp];
    const float lz = __ldg(&lam[comp == 2 ? z : 0]);
    for (int p0 = warp * G; p0 < P.npair; p0 += nw * G) {
      const int nl = min(G, P.npair - p0);
      float2* reg = sm + p0 * 2 * hx;
      // prefetch rho_xi (and, for the last component, rho_x, rho_z, c0^2) rows
      warp_prefetch_rows(stage, rho, p0, nl, nx, ny, lane);
      if (cc == 2) {
        warp_prefetch_rows(stage + stage_n, rx, p0, nl, nx, ny, lane);
        warp_prefetch_rows(stage + 2 * stage_n, rz, p0, nl, nx, ny, lane);
        warp_prefetch_rows(stage + 3 * stage_n, c2, p0, nl, nx, ny, lane);
      }
      warp_c2r_pack<C::PI>(reg, nl, nx, hx, ny, p0, lane);
      C::template fft_x<true>(reg, nl, P, twx, lane);
      cp_async_wait_all();
      __syncwarp();
      // rho_xi <- Lambda (Lambda rho_xi - dt rho0 d-_xi v_xi); last component: p = c0^2 sum rho
      for (int l = 0; l < nl; ++l) {
        const int y0 = 2 * (p0 + l), y1 = y0 + 1;
        float2* Z = reg + l * 2 * hx;
        const int o0 = (2 * l) * nx, o1 = o0 + nx;
        for (int x = lane; x < nx; x += 32) {
          const float2 d = Z[x];
          float l0, l1;
          if (comp == 0) { l0 = l1 = __ldg(&lam[x]); }
          else if (comp == 1) { l0 = __ldg(&lam[y0]); l1 = (y1 < ny) ? __ldg(&lam[y1]) : 1.f; }
          else { l0 = l1 = lz; }
          const int i0 = y0 * nx + x, i1 = y1 * nx + x;
          const float r0 = l0 * (l0 * stage[o0 + x] - P.dt_rho0 * d.x);
          rho[i0] = r0;
          float r1 = 0.f;
          if (y1 < ny) {
            r1 = l1 * (l1 * stage[o1 + x] - P.dt_rho0 * d.y);
            rho[i1] = r1;
          }
          if (cc == 2) {
            const float* sx = stage + stage_n;
            const float* sz = stage + 2 * stage_n;
            const float* sc = stage + 3 * stage_n;
            const float p0v = sc[o0 + x] * (sx[o0 + x] + r0 + sz[o0 + x]);
            const float p1v = (y1 < ny) ? sc[o1 + x] * (sx[o1 + x] + r1 + sz[o1 + x]) : 0.f;
            Z[x] = make_float2(p0v, p1v);
          }
        }
      }
      if (cc < 2) continue;
      __syncwarp();
      // sparse updates of rho_xi and p on these pair lines, then recording
      const int key0 = z * P.npair + p0;
      float* zf = reinterpret_cast<float*>(sm);
      if (role == ROLE_FORWARD) {
        const float* amp = P.amp_src + ((size_t)shot * P.nt + tix) * P.n_us;
        for (int u = P.us_ptr[key0] + lane; u < P.us_ptr[key0 + nl]; u += 32) {
          const int vx = P.us_vox[u];
          const float a = amp[u];
          S.rho[0][vx] += a;
          S.rho[1][vx] += a;
          S.rho[2][vx] += a;
          zf[P.us_pf[u]] += c2_of(P, S)[vx] * (3.f * a);
        }
      } else if (role == ROLE_ADJOINT) {
        const float* q = P.qf + ((size_t)shot * P.nt + tix) * P.n_rec;
        for (int u = P.ur_ptr[key0] + lane; u < P.ur_ptr[key0 + nl]; u += 32) {
          float s = 0.f;
          for (int e = P.ur_mptr[u]; e < P.ur_mptr[u + 1]; ++e) s += q[P.ur_mem[e]];
          const float a = ur_coef_of(P, S)[u] * s;
          const int vx = P.ur_vox[u];
          S.rho[0][vx] += a;
          S.rho[1][vx] += a;
          S.rho[2][vx] += a;
          zf[P.ur_pf[u]] += c2_of(P, S)[vx] * (3.f * a);
        }
      } else {  // TR: rho_xi(layer) <- g^(Nt - m) / (3 c0^2)
        const float* g = P.ghist + ((size_t)shot * P.nt + (P.nt - 1 - tix)) * P.n_layer;
        for (int j = P.lay_ptr[key0] + lane; j < P.lay_ptr[key0 + nl]; j += 32) {
          const int vx = P.lay_vox[j];
          const float val = g[j] * inv3c2_of(P, S)[j];
          S.rho[0][vx] = val;
          S.rho[1][vx] = val;
          S.rho[2][vx] = val;
          zf[P.lay_pf[j]] = c2_of(P, S)[vx] * (3.f * val);
        }
      }
      __syncwarp();
      if (role == ROLE_FORWARD) {
        float* f = P.traces + ((size_t)shot * P.nt + tix) * P.n_rec;
        for (int e = P.rr_ptr[key0] + lane; e < P.rr_ptr[key0 + nl]; e += 32) f[P.rr_col[e]] = zf[P.rr_pf[e]];
        if (P.record_layer) {
          float* g = P.ghist + ((size_t)shot * P.nt + tix) * P.n_layer;
          for (int j = P.lay_ptr[key0] + lane; j < P.lay_ptr[key0 + nl]; j += 32) g[j] = zf[P.lay_pf[j]];
        }
      } else {
        float* out = role == ROLE_ADJOINT ? P.pa + (size_t)shot * P.n_gamma
                                          : P.ring + ((size_t)shot * kRing + P.slot[blockIdx.y]) * P.n_gamma;
        for (int j = P.gam_ptr[key0] + lane; j < P.gam_ptr[key0 + nl]; j += 32) out[j] = zf[P.gam_pf[j]];
      }
      __syncwarp();
      C::template fft_x<false>(reg, nl, P, twx, lane);
      warp_r2c_unpack<C::UI>(reg, nl, nx, hx, ny, p0, lane);
    }
    __syncthreads();
  }
  forward_y_and_store<C>(sm, twy, P, S.spec[0] + soff);
}

// TR initial value: p(layer) <- g^Nt, zero elsewhere; ring slot 0 <- p(Gamma);
// P_xy <- forward XY transform of that p.  State fields are zeroed by the host.
template <int EPL, int FX, int FY>
__global__ void __launch_bounds__(kTpbPlane, 2) k_tr_init(const __grid_constant__ StepParams P) {
  using C = PlaneCfg<EPL, FX, FY>;
  if (*P.bad) return;
  extern __shared__ float2 sm_raw[];
  const float2* twx = sm_raw;
  const float2* twy = sm_raw + P.ax.n;
  float2* sm = stage_twiddles(sm_raw, P);
  const int z = blockIdx.x;
  const SimPtrs& S = P.sims[blockIdx.y];
  const int shot = S.shot;
  const int hx = P.hx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = C::gx(P);
  const float* g = P.ghist + ((size_t)shot * P.nt + (P.nt - 1)) * P.n_layer;
  float* out = P.ring + ((size_t)shot * kRing + 0) * P.n_gamma;
  __syncthreads();
  for (int p0 = warp * G; p0 < P.npair; p0 += nw * G) {
    const int nl = min(G, P.npair - p0);
    float2* reg = sm + p0 * 2 * hx;
    for (int i = lane; i < nl * 2 * hx; i += 32) reg[i] = make_float2(0.f, 0.f);
    __syncwarp();
    const int key0 = z * P.npair + p0;
    float* zf = reinterpret_cast<float*>(sm);
    for (int j = P.lay_ptr[key0] + lane; j < P.lay_ptr[key0 + nl]; j += 32) zf[P.lay_pf[j]] = g[j];
    __syncwarp();
    for (int j = P.gam_ptr[key0] + lane; j < P.gam_ptr[key0 + nl]; j += 32) out[j] = zf[P.gam_pf[j]];
    __syncwarp();
    C::template fft_x<false>(reg, nl, P, twx, lane);
    warp_r2c_unpack<C::UI>(reg, nl, P.nx, hx, P.ny, p0, lane);
  }
  __syncthreads();
  forward_y_and_store<C>(sm, twy, P, S.spec[0] + (size_t)z * P.mspec);
}

}  // namespace fwi

namespace fwi {

// ======================================================================= split planes
// Planes too large for one CTA's shared memory run each XY half-step as
//   k_ypass (columns: y transforms of TY adjacent kx columns of one z-plane) and
//   k_xpass (warps own pair lines of one z-plane: C2R, x transforms, field update,
//            sparse work, R2C; rows are read from and written back to global memory).
// Per step: zpass<MOM>, ypass<INV_MOM>, xpass<MOM>, ypass<FWD3>, zpass<MASS>,
// ypass<INV_MASS>, xpass<MASS>, ypass<FWD1>.

enum YKind : int { Y_INV_MOM = 0, Y_INV_MASS = 1, Y_FWD3 = 2, Y_FWD1 = 3 };
constexpr int kTY = 16;

// Y_INV_MOM:  spec[0] = Q, spec[1] = R  ->  spec[2] = IFFT_y(Q) (x factor applied later),
//             spec[0] = IFFT_y(a+_y Q), spec[1] = IFFT_y(R)
// Y_INV_MASS: spec[2], spec[0] (times a-_y), spec[1]: inverse y, in place
// Y_FWD3:     spec[2], spec[0], spec[1]: forward y, in place
// Y_FWD1:     spec[0]: forward y, in place
template <int KIND, int EPL>
__global__ void __launch_bounds__(kTpbZ, 2) k_ypass(const __grid_constant__ StepParams P) {
  if (*P.bad) return;
  extern __shared__ float2 ysm_raw[];
  const SimPtrs& S = P.sims[blockIdx.z];
  constexpr int NSL = KIND == Y_FWD1 ? 1 : 3;
  constexpr int RS = NSL * kTY + 4;
  constexpr bool INV = KIND == Y_INV_MOM || KIND == Y_INV_MASS;
  const int ny = P.ny, hx = P.hx;
  float2* twy = ysm_raw;
  for (int i = threadIdx.x; i < ny; i += blockDim.x) twy[i] = P.tw[P.ay.tw_off + i];
  float2* sm = ysm_raw + ((ny + 31) & ~31);
  const int k0 = blockIdx.x * kTY;
  const size_t zoff = (size_t)blockIdx.y * P.mspec;
  auto src_of = [&](int s) -> float2* {
    if (KIND == Y_INV_MOM) return s == 2 ? S.spec[1] : S.spec[0];
    if (KIND == Y_FWD1) return S.spec[0];
    return s == 0 ? S.spec[2] : (s == 1 ? S.spec[0] : S.spec[1]);
  };
  auto dst_of = [&](int s) -> float2* {
    if (KIND == Y_INV_MOM) return s == 0 ? S.spec[2] : (s == 1 ? S.spec[0] : S.spec[1]);
    return src_of(s);
  };
  for (int idx = threadIdx.x; idx < NSL * ny * kTY; idx += blockDim.x) {
    const int ml = idx % kTY;
    const int t = idx / kTY;
    const int s = t / ny;
    const int y = t - s * ny;
    const int kx = k0 + ml;
    if (kx < hx) cp_async8(&sm[y * RS + s * kTY + ml], &src_of(s)[zoff + (size_t)y * hx + kx]);
    else sm[y * RS + s * kTY + ml] = make_float2(0.f, 0.f);
  }
  cp_async_wait_all();
  __syncthreads();
  if (KIND == Y_INV_MOM || KIND == Y_INV_MASS) {   // y factor on the y component's slot
    for (int idx = threadIdx.x; idx < ny * kTY; idx += blockDim.x) {
      const int ml = idx % kTY;
      const int y = idx / kTY;
      const float2 f = KIND == Y_INV_MOM ? __ldg(&P.ap[1][y]) : __ldg(&P.am[1][y]);
      sm[y * RS + 1 * kTY + ml] = cmul(sm[y * RS + 1 * kTY + ml], f);
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = min(lines_per_group<EPL>(ny), kTY);
  const int gps = (kTY + G - 1) / G;
  for (int g = warp; g < NSL * gps; g += nw) {
    const int s = g / gps;
    const int c0 = (g - s * gps) * G;
    warp_fft<INV, EPL>(sm + s * kTY + c0, min(G, kTY - c0), 1, RS, P.ay, twy, lane);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NSL * ny * kTY; idx += blockDim.x) {
    const int ml = idx % kTY;
    const int t = idx / kTY;
    const int s = t / ny;
    const int y = t - s * ny;
    const int kx = k0 + ml;
    if (kx < hx) dst_of(s)[zoff + (size_t)y * hx + kx] = sm[y * RS + s * kTY + ml];
  }
}

// Rows 2p, 2p+1 of a y-transformed spectrum plane -> the warp's pair-line region
// (asynchronous; the missing row of an odd ny is zero).
__device__ __forceinline__ void warp_load_pairs(float2* reg, const float2* __restrict__ plane, int p0,
                                                int nl, int hx, int ny, int lane) {
  const int rows = min(2 * nl, ny - 2 * p0);
  const int tot = rows * hx;
  const float2* src = plane + (size_t)(2 * p0) * hx;
  for (int i = lane; i < tot; i += 32) cp_async8(&reg[i], &src[i]);
  for (int i = tot + lane; i < 2 * nl * hx; i += 32) reg[i] = make_float2(0.f, 0.f);
}
__device__ __forceinline__ void warp_store_pairs(const float2* reg, float2* __restrict__ plane, int p0,
                                                 int nl, int hx, int ny, int lane) {
  const int rows = min(2 * nl, ny - 2 * p0);
  float2* dst = plane + (size_t)(2 * p0) * hx;
  for (int i = lane; i < rows * hx; i += 32) dst[i] = reg[i];
}

// x work of the momentum half-step on split planes (see k_plane_mom).
template <int EPL>
__global__ void __launch_bounds__(kTpbPlane, 2) k_xpass_mom(const __grid_constant__ StepParams P) {
  if (*P.bad) return;
  using C = PlaneCfg<EPL, 0, 0>;
  extern __shared__ float2 xsm_raw[];
  const float2* twx = xsm_raw;
  const int nx = P.nx, ny = P.ny, hx = P.hx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) xsm_raw[i] = P.tw[P.ax.tw_off + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = C::gx(P);
  float2* reg = xsm_raw + ((nx + 31) & ~31) + warp * G * 2 * hx;
  float* stage = reinterpret_cast<float*>(xsm_raw + ((nx + 31) & ~31) + nw * G * 2 * hx) + warp * 2 * G * nx;
  const int z = blockIdx.y;
  const SimPtrs& S = P.sims[blockIdx.z];
  const size_t soff = (size_t)z * P.mspec;
  const size_t voff = (size_t)z * P.plane;
  const int p0 = (blockIdx.x * nw + warp) * G;
  if (p0 >= P.npair) return;
  const int nl = min(G, P.npair - p0);
  // component z (spec[1]), x (spec[2] = IFFT_y(Q), times a+_x here), y (spec[0])
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = cc == 0 ? 2 : cc - 1;
    float2* buf = (comp == 2 ? S.spec[1] : (comp == 0 ? S.spec[2] : S.spec[0])) + soff;
    float* v = S.v[comp] + voff;
    warp_load_pairs(reg, buf, p0, nl, hx, ny, lane);
    warp_prefetch_rows(stage, v, p0, nl, nx, ny, lane);
    cp_async_wait_all();
    __syncwarp();
    if (comp == 0) {
      for (int i = lane; i < nl * 2 * hx; i += 32) reg[i] = cmul(reg[i], __ldg(&P.ap[0][i % hx]));
      __syncwarp();
    }
    warp_c2r_pack<C::PI>(reg, nl, nx, hx, ny, p0, lane);
    C::template fft_x<true>(reg, nl, P, twx, lane);
    const float* lam = P.lams[comp];
    const float lz = __ldg(&lam[comp == 2 ? z : 0]);
    for (int l = 0; l < nl; ++l) {
      const int y0 = 2 * (p0 + l), y1 = y0 + 1;
      float2* Z = reg + l * 2 * hx;
      const float* s0 = stage + (2 * l) * nx;
      for (int x = lane; x < nx; x += 32) {
        const float2 d = Z[x];
        float l0, l1;
        if (comp == 0) { l0 = l1 = __ldg(&lam[x]); }
        else if (comp == 1) { l0 = __ldg(&lam[y0]); l1 = (y1 < ny) ? __ldg(&lam[y1]) : 1.f; }
        else { l0 = l1 = lz; }
        const float v0 = l0 * (l0 * s0[x] - P.dt_over_rho0 * d.x);
        v[y0 * nx + x] = v0;
        float v1 = 0.f;
        if (y1 < ny) {
          v1 = l1 * (l1 * s0[nx + x] - P.dt_over_rho0 * d.y);
          v[y1 * nx + x] = v1;
        }
        Z[x] = make_float2(v0, v1);
      }
    }
    __syncwarp();
    C::template fft_x<false>(reg, nl, P, twx, lane);
    warp_r2c_unpack<C::UI>(reg, nl, nx, hx, ny, p0, lane);
    warp_store_pairs(reg, buf, p0, nl, hx, ny, lane);
    __syncwarp();
  }
}

// x work of the mass half-step on split planes (see k_plane_mass); writes the
// x-transformed p rows into spec[0] (the y transform follows in k_ypass<Y_FWD1>).
template <int EPL>
__global__ void __launch_bounds__(kTpbPlane, 2) k_xpass_mass(const __grid_constant__ StepParams P) {
  if (*P.bad) return;
  using C = PlaneCfg<EPL, 0, 0, 128>;
  extern __shared__ float2 xsm_raw[];
  const float2* twx = xsm_raw;
  const int nx = P.nx, ny = P.ny, hx = P.hx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) xsm_raw[i] = P.tw[P.ax.tw_off + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = C::gx(P);
  const int stage_n = 2 * G * nx;
  float2* reg = xsm_raw + ((nx + 31) & ~31) + warp * G * 2 * hx;
  float* stage = reinterpret_cast<float*>(xsm_raw + ((nx + 31) & ~31) + nw * G * 2 * hx) + warp * 4 * stage_n;
  const int z = blockIdx.y;
  const SimPtrs& S = P.sims[blockIdx.z];
  const int role = S.role, shot = S.shot, tix = P.tidx[blockIdx.z];
  const size_t soff = (size_t)z * P.mspec;
  const size_t voff = (size_t)z * P.plane;
  const int p0 = (blockIdx.x * nw + warp) * G;
  if (p0 >= P.npair) return;
  const int nl = min(G, P.npair - p0);
  const float* c2 = c2_of(P, S) + voff;
  const float* rx = S.rho[0] + voff;
  const float* rz = S.rho[2] + voff;
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = cc == 0 ? 0 : (cc == 1 ? 2 : 1);
    float2* buf = (comp == 0 ? S.spec[2] : (comp == 2 ? S.spec[1] : S.spec[0])) + soff;
    float* rho = S.rho[comp] + voff;
    warp_load_pairs(reg, buf, p0, nl, hx, ny, lane);
    warp_prefetch_rows(stage, rho, p0, nl, nx, ny, lane);
    if (cc == 2) {
      warp_prefetch_rows(stage + stage_n, rx, p0, nl, nx, ny, lane);
      warp_prefetch_rows(stage + 2 * stage_n, rz, p0, nl, nx, ny, lane);
      warp_prefetch_rows(stage + 3 * stage_n, c2, p0, nl, nx, ny, lane);
    }
    cp_async_wait_all();
    __syncwarp();
    if (comp == 0) {
      for (int i = lane; i < nl * 2 * hx; i += 32) reg[i] = cmul(reg[i], __ldg(&P.am[0][i % hx]));
      __syncwarp();
    }
    warp_c2r_pack<C::PI>(reg, nl, nx, hx, ny, p0, lane);
    C::template fft_x<true>(reg, nl, P, twx, lane);
    const float* lam = P.lam[comp];
    const float lz = __ldg(&lam[comp == 2 ? z : 0]);
    for (int l = 0; l < nl; ++l) {
      const int y0 = 2 * (p0 + l), y1 = y0 + 1;
      float2* Z = reg + l * 2 * hx;
      const int o0 = (2 * l) * nx, o1 = o0 + nx;
      for (int x = lane; x < nx; x += 32) {
        const float2 d = Z[x];
        float l0, l1;
        if (comp == 0) { l0 = l1 = __ldg(&lam[x]); }
        else if (comp == 1) { l0 = __ldg(&lam[y0]); l1 = (y1 < ny) ? __ldg(&lam[y1]) : 1.f; }
        else { l0 = l1 = lz; }
        const int i0 = y0 * nx + x, i1 = y1 * nx + x;
        const float r0 = l0 * (l0 * stage[o0 + x] - P.dt_rho0 * d.x);
        rho[i0] = r0;
        float r1 = 0.f;
        if (y1 < ny) {
          r1 = l1 * (l1 * stage[o1 + x] - P.dt_rho0 * d.y);
          rho[i1] = r1;
        }
        if (cc == 2) {
          const float* sx = stage + stage_n;
          const float* sz = stage + 2 * stage_n;
          const float* sc = stage + 3 * stage_n;
          const float p0v = sc[o0 + x] * (sx[o0 + x] + r0 + sz[o0 + x]);
          const float p1v = (y1 < ny) ? sc[o1 + x] * (sx[o1 + x] + r1 + sz[o1 + x]) : 0.f;
          Z[x] = make_float2(p0v, p1v);
        }
      }
    }
    __syncwarp();
    if (cc < 2) continue;
    // sparse updates of rho_xi and p on these pair lines, then recording (offsets
    // pf are relative to the plane buffer; this warp's region starts at pair p0)
    const int key0 = z * P.npair + p0;
    float* zf = reinterpret_cast<float*>(reg) - 4 * hx * p0;
    if (role == ROLE_FORWARD) {
      const float* amp = P.amp_src + ((size_t)shot * P.nt + tix) * P.n_us;
      for (int u = P.us_ptr[key0] + lane; u < P.us_ptr[key0 + nl]; u += 32) {
        const int vx = P.us_vox[u];
        const float a = amp[u];
        S.rho[0][vx] += a;
        S.rho[1][vx] += a;
        S.rho[2][vx] += a;
        zf[P.us_pf[u]] += c2_of(P, S)[vx] * (3.f * a);
      }
    } else if (role == ROLE_ADJOINT) {
      const float* q = P.qf + ((size_t)shot * P.nt + tix) * P.n_rec;
      for (int u = P.ur_ptr[key0] + lane; u < P.ur_ptr[key0 + nl]; u += 32) {
        float s = 0.f;
        for (int e = P.ur_mptr[u]; e < P.ur_mptr[u + 1]; ++e) s += q[P.ur_mem[e]];
        const float a = ur_coef_of(P, S)[u] * s;
        const int vx = P.ur_vox[u];
        S.rho[0][vx] += a;
        S.rho[1][vx] += a;
        S.rho[2][vx] += a;
        zf[P.ur_pf[u]] += c2_of(P, S)[vx] * (3.f * a);
      }
    } else {
      const float* g = P.ghist + ((size_t)shot * P.nt + (P.nt - 1 - tix)) * P.n_layer;
      for (int j = P.lay_ptr[key0] + lane; j < P.lay_ptr[key0 + nl]; j += 32) {
        const int vx = P.lay_vox[j];
        const float val = g[j] * inv3c2_of(P, S)[j];
        S.rho[0][vx] = val;
        S.rho[1][vx] = val;
        S.rho[2][vx] = val;
        zf[P.lay_pf[j]] = c2_of(P, S)[vx] * (3.f * val);
      }
    }
    __syncwarp();
    if (role == ROLE_FORWARD) {
      float* f = P.traces + ((size_t)shot * P.nt + tix) * P.n_rec;
      for (int e = P.rr_ptr[key0] + lane; e < P.rr_ptr[key0 + nl]; e += 32) f[P.rr_col[e]] = zf[P.rr_pf[e]];
      if (P.record_layer) {
        float* g = P.ghist + ((size_t)shot * P.nt + tix) * P.n_layer;
        for (int j = P.lay_ptr[key0] + lane; j < P.lay_ptr[key0 + nl]; j += 32) g[j] = zf[P.lay_pf[j]];
      }
    } else {
      float* out = role == ROLE_ADJOINT ? P.pa + (size_t)shot * P.n_gamma
                                        : P.ring + ((size_t)shot * kRing + P.slot[blockIdx.z]) * P.n_gamma;
      for (int j = P.gam_ptr[key0] + lane; j < P.gam_ptr[key0 + nl]; j += 32) out[j] = zf[P.gam_pf[j]];
    }
    __syncwarp();
    C::template fft_x<false>(reg, nl, P, twx, lane);
    warp_r2c_unpack<C::UI>(reg, nl, nx, hx, ny, p0, lane);
    warp_store_pairs(reg, S.spec[0] + soff, p0, nl, hx, ny, lane);
  }
}

// TR initial value on split planes: x work only (k_ypass<Y_FWD1> follows).
template <int EPL>
__global__ void __launch_bounds__(kTpbPlane, 2) k_xpass_tr_init(const __grid_constant__ StepParams P) {
  if (*P.bad) return;
  using C = PlaneCfg<EPL, 0, 0>;
  extern __shared__ float2 xsm_raw[];
  const float2* twx = xsm_raw;
  const int nx = P.nx, ny = P.ny, hx = P.hx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) xsm_raw[i] = P.tw[P.ax.tw_off + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = C::gx(P);
  float2* reg = xsm_raw + ((nx + 31) & ~31) + warp * G * 2 * hx;
  const int z = blockIdx.y;
  const SimPtrs& S = P.sims[blockIdx.z];
  const int shot = S.shot;
  const int p0 = (blockIdx.x * nw + warp) * G;
  if (p0 >= P.npair) return;
  const int nl = min(G, P.npair - p0);
  for (int i = lane; i < nl * 2 * hx; i += 32) reg[i] = make_float2(0.f, 0.f);
  __syncwarp();
  const int key0 = z * P.npair + p0;
  float* zf = reinterpret_cast<float*>(reg) - 4 * hx * p0;
  const float* g = P.ghist + ((size_t)shot * P.nt + (P.nt - 1)) * P.n_layer;
  for (int j = P.lay_ptr[key0] + lane; j < P.lay_ptr[key0 + nl]; j += 32) zf[P.lay_pf[j]] = g[j];
  __syncwarp();
  float* out = P.ring + ((size_t)shot * kRing + 0) * P.n_gamma;
  for (int j = P.gam_ptr[key0] + lane; j < P.gam_ptr[key0 + nl]; j += 32) out[j] = zf[P.gam_pf[j]];
  __syncwarp();
  C::template fft_x<false>(reg, nl, P, twx, lane);
  warp_r2c_unpack<C::UI>(reg, nl, nx, hx, ny, p0, lane);
  warp_store_pairs(reg, S.spec[0] + (size_t)z * P.mspec, p0, nl, hx, ny, lane);
}

}  // namespace fwi
