// Split-plane XY work with two-step register transforms, for planes too large
// for one CTA's shared memory (the 243^2 and 480^2 serving grids).  Each XY
// half-step of Alg. 1 (App. B, Eqs. 18-19 in x and y) runs as
//   k_ypass2   y transforms of TY adjacent kx columns of one z-plane, straight from
//              and to global memory: step A reads, step B writes (one barrier);
//   k_xpass2_* NPC row pairs of one z-plane: rows into shared memory, C2R packing
//              and x-inverse step A, x-inverse step B with the field update and the
//              forward x step A, forward step B, R2C unpacking to global rows.
// The order per step matches the split path of kernels.cuh: zpass<MOM>,
// ypass<INV_MOM>, xpass<MOM>, ypass<FWD3>, zpass<MASS>, ypass<INV_MASS>,
// xpass<MASS>, ypass<FWD1>.
#pragma once
#include "plane2.cuh"

namespace fwi {

// kx columns per CTA of the split y passes: 16 unless the step-B lines are long (8);
// 243 takes three step-A tasks per thread and 16 columns (see Y2::RA)
__host__ __device__ constexpr int ty2_for(int n) { return n == 243 || n / split_n1(n) <= 16 ? 16 : 8; }
#ifndef P2_NPC243
#define P2_NPC243 14
#endif
// row pairs per CTA of the split x passes: 243 = 9 x 27 gives 9 update tasks per pair,
// so 14 pairs (126 tasks on 128 threads) keep the update phase's threads busy and leave
// shared memory for the staged old rows (21 pairs without staging: 20 % slower)
constexpr int npc2_for(int n) { return n == 243 ? P2_NPC243 : 8; }

template <int NY, int TY>
struct Y2 {
  static constexpr int N1 = split_n1(NY), N2 = NY / N1;
  // Step A has TY N2 tasks (DFT_N1), step B TY N1 (DFT_N2, the heavy ones).  When N2 is
  // a multiple N2 = RA N1 with RA > 1 (243 = 9 x 27: RA = 3), a thread takes RA step-A
  // tasks of its column so that step B fills all TY N1 threads; otherwise one step-A
  // task per thread and step B on the first TY N1.
  static constexpr int RA = (N2 % N1 == 0 && N2 / N1 > 1 && N2 > 24) ? N2 / N1 : 1;
  static constexpr int NT = TY * N2 / RA;
  static_assert(N1 <= N2, "step B runs on the first TY * N1 threads");
  // Row r of the step-A buffer starts at r TY + (r / N2) PAD.  With TY = 8, a step-B
  // half-warp reads two blocks of N2 rows; PAD = 8 puts them on opposite bank halves
  // when N2 TY = 0 (mod 16).
  static constexpr int PAD = (TY < 16 && (N2 * TY) % 16 == 0) ? 8 : 0;
  __host__ __device__ static constexpr int row(int r) { return r * TY + (r / N2) * PAD; }
  // Long step-B lines (N2 > 16) leave no registers to prefetch the next slot's step-A
  // inputs: GST stages them in shared memory with cp.async during the current step B.
  static constexpr bool GST = RA == 1 && N2 > 16;
  static constexpr int BSZ = NY * TY + N1 * PAD;          // step-A output buffer
  static constexpr size_t SMEM = (size_t)(NY + BSZ + (GST ? NY * TY : 0)) * 8;
  // two CTAs per SM where the register budget allows it without spilling the step-B lines
  static constexpr int MINB = (N2 <= 24 && NY > 256) || RA > 1 ? 2 : 1;
};

template <int KIND, int NY, int TY>
__global__ void __launch_bounds__(Y2<NY, TY>::NT, Y2<NY, TY>::MINB) k_ypass2(const __grid_constant__ StepParams P) {
  using C = Y2<NY, TY>;
  constexpr int N1 = C::N1, N2 = C::N2;
  constexpr bool INV = KIND == Y_INV_MOM || KIND == Y_INV_MASS;
  constexpr int NSL = KIND == Y_FWD1 ? 1 : 3;
  if (*P.bad) return;
  extern __shared__ __align__(16) float2 ys2[];
  float2* tw = ys2;
  float2* b = ys2 + NY;
  for (int i = threadIdx.x; i < NY; i += C::NT) tw[i] = P.tw[P.ay.tw_off + i];
  const SimPtrs& S = P.sims[blockIdx.z];
  const int HX = P.hx;
  const size_t zoff = (size_t)blockIdx.y * P.mspec;
  const int k0 = blockIdx.x * TY;
  auto src_of = [&](int s) -> const float2* {
    if (KIND == Y_INV_MOM) return s == 2 ? S.spec[1] : S.spec[0];
    if (KIND == Y_FWD1) return S.spec[0];
    return s == 0 ? S.spec[2] : (s == 1 ? S.spec[0] : S.spec[1]);
  };
  auto dst_of = [&](int s) -> float2* {
    if (KIND == Y_INV_MOM) return s == 0 ? S.spec[2] : (s == 1 ? S.spec[0] : S.spec[1]);
    return const_cast<float2*>(src_of(s));
  };
  // the y factor multiplies slot 1 of the inverse passes (a+_y: momentum, a-_y: mass)
  const float2* fac = KIND == Y_INV_MOM ? P.ap[1] : P.am[1];
  if constexpr (C::RA > 1) {
    // RA step-A tasks per thread (column mlA, j2 = j2A + r N2 / RA), all loads first
    constexpr int RA = C::RA;
    const int ml = threadIdx.x % TY, j2a = threadIdx.x / TY;
    const int kx = k0 + ml;
#pragma unroll 1
    for (int s = 0; s < NSL; ++s) {
      const float2* src = src_of(s) + zoff;
      float2 a[RA][N1];
      sfor<0, RA>([&](auto R) {
        constexpr int r = decltype(R)::value;
        sfor<0, N1>([&](auto J1) {
          constexpr int j1 = decltype(J1)::value;
          const int ky = j2a + (N2 / RA) * r + N2 * j1;
          float2 v = kx < HX ? src[(size_t)ky * HX + kx] : make_float2(0.f, 0.f);
          if (INV && s == 1) v = cmul(v, __ldg(&fac[ky]));
          a[r][j1] = v;
        });
      });
      __syncthreads();   // twiddles staged; the previous slot's buffer consumed
      sfor<0, RA>([&](auto R) {
        constexpr int r = decltype(R)::value;
        const int j2 = j2a + (N2 / RA) * r;
        RDft<N1, INV>::run(a[r]);
        float2 w[N1];
        tw_row<N1>(tw, j2, w);
        sfor<0, N1>([&](auto K1) {
          constexpr int k1 = decltype(K1)::value;
          float2 v = a[r][k1];
          if (k1 > 0) v = INV ? cmulc(v, w[k1]) : cmul(v, w[k1]);
          b[C::row(j2 + N2 * k1) + ml] = v;
        });
      });
      __syncthreads();
      const int k1B = threadIdx.x / TY;
      float2 x[N2];
      sfor<0, N2>([&](auto J2) { x[decltype(J2)::value] = b[C::row(N2 * k1B + decltype(J2)::value) + ml]; });
      RDft<N2, INV>::run(x);
      if (kx < HX) {
        float2* dst = dst_of(s) + zoff;
        sfor<0, N2>([&](auto K2) {
          constexpr int k2 = decltype(K2)::value;
          dst[(size_t)(k1B + N1 * k2) * HX + kx] = x[k2];
        });
      }
    }
    return;
  }
  const int mlA = threadIdx.x % TY, j2A = threadIdx.x / TY;
  const int kxA = k0 + mlA;
  float2* g = b + C::BSZ;   // staged inputs [ky][TY] (C::GST)
  auto stage = [&](int s) {
    const float2* src = src_of(s) + zoff;
    for (int i = threadIdx.x; i < NY * TY; i += C::NT) {
      const int ky = i / TY, ml = i - ky * TY;
      if (k0 + ml < HX) cp_async8(&g[i], &src[(size_t)ky * HX + k0 + ml]);
      else g[i] = make_float2(0.f, 0.f);
    }
    cp_async_commit();
  };
  float2 a[N1];
  auto load_a = [&](int s) {
    const float2* src = src_of(s) + zoff;
    sfor<0, N1>([&](auto J1) {
      constexpr int j1 = decltype(J1)::value;
      const int ky = j2A + N2 * j1;
      float2 v;
      if constexpr (C::GST) v = g[ky * TY + mlA];
      else v = kxA < HX ? src[(size_t)ky * HX + kxA] : make_float2(0.f, 0.f);
      if (INV && s == 1) v = cmul(v, __ldg(&fac[ky]));
      a[j1] = v;
    });
  };
  if constexpr (C::GST) stage(0);
  else load_a(0);
  const bool hasB = threadIdx.x < TY * N1;
  const int mlB = threadIdx.x % TY, k1B = threadIdx.x / TY;
  const int kxB = k0 + mlB;
#pragma unroll 1
  for (int s = 0; s < NSL; ++s) {
    if constexpr (C::GST) cp_async_wait_all();
    __syncthreads();   // twiddles staged; the previous slot's buffer consumed
    if (C::GST) load_a(s);                          // from the staged inputs
    else if (N2 > 16 && s > 0) load_a(s);
    RDft<N1, INV>::run(a);
    float2 w[N1];
    tw_row<N1>(tw, j2A, w);
    sfor<0, N1>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      float2 v = a[k1];
      if (k1 > 0) v = INV ? cmulc(v, w[k1]) : cmul(v, w[k1]);
      b[C::row(j2A + N2 * k1) + mlA] = v;
    });
    __syncthreads();
    if constexpr (C::GST) {
      if (s + 1 < NSL) stage(s + 1);              // in flight during step B
    } else if (N2 <= 16 && s + 1 < NSL) {
      load_a(s + 1);                              // in flight during step B (short lines)
    }
    if (hasB) {
      float2 x[N2];
      sfor<0, N2>([&](auto J2) { x[decltype(J2)::value] = b[C::row(N2 * k1B + decltype(J2)::value) + mlB]; });
      RDft<N2, INV>::run(x);
      if (kxB < HX) {
        float2* dst = dst_of(s) + zoff;
        sfor<0, N2>([&](auto K2) {
          constexpr int k2 = decltype(K2)::value;
          dst[(size_t)(k1B + N1 * k2) * HX + kxB] = x[k2];
        });
      }
    }
  }
}

// ---------------------------------------------------------------------------
// x passes over NPC row pairs of one z-plane
template <int NX, int NPC>
struct X2 {
  static constexpr int NXc = NX, NPCc = NPC;
  static constexpr int HX = NX / 2 + 1;
  static constexpr int AX1 = split_n1(NX), AX2 = NX / AX1;
  // Padded row lengths of the step-A outputs (PA: x-inverse, PB: x-forward) and the pair
  // stride, per size for the fewest shared-memory wavefronts over all phases (a bank
  // model of every access).  PST = 2 (mod 16) makes the x-inverse reads and writes
  // conflict-free: a half-warp there holds eight pairs at two adjacent columns, and the
  // pair offsets 2p, p < 8, plus 0 or 1 cover the 16 banks once.
  static constexpr bool T243 = NX == 243 && (NPC == 21 || NPC == 14);
  static constexpr int PA = T243 ? 33 : AX2 + 1;
  static constexpr int PB = T243 ? 11 : AX1 + 1;
  static constexpr int PST_MIN = cmax3(2 * HX, AX1 * PA, AX2 * PB);
  static constexpr int PST = NX == 480 && NPC == 8 ? 514 : NX == 256 && NPC == 8 ? 274 : T243 ? 297 : (PST_MIN | 1);
  static_assert(PST >= PST_MIN, "pair regions must not overlap");
  static constexpr int T3 = NPC * AX2, T4 = NPC * AX1, TU = NPC * HX;
  // one round of the update phase (T4 tasks: step B, field update, forward step A); the
  // lighter x-inverse step A (T3 tasks) takes one round too unless that would leave more
  // than half the threads idle in the update
  static constexpr int NT = ((T3 <= 2 * T4 ? (T3 > T4 ? T3 : T4) : T4) + 31) / 32 * 32;
  static constexpr int TWP = (2 * NX + 1) & ~1;
  // Old field values of the update: staged rows of the pass's 2 NPC rows in shared memory
  // (STG, where two CTAs per SM still fit), else read from global memory.  Staged rows
  // are RS floats apart with 2 RS = 20 (mod 32): a warp's update tasks (20 columns per
  // row pair) then read 32 distinct banks.
  static constexpr bool STG = (NX == 480 && NPC == 8) || (NX == 243 && NPC == 14);
  static constexpr int RS = NX == 480 && STG ? 490 : NX == 243 && STG ? 244 : NX;
  static constexpr size_t SMEM = (size_t)(TWP + 2 * NPC * PST) * 8 + (STG ? (size_t)2 * NPC * RS * 4 : 0);
  static constexpr bool REMAP = false;
  __host__ __device__ static constexpr int row_off(int y) { return y * RS; }
};

// rows 0 .. nyl-1 of a field (row length NX, this pass's first row at src) -> staged rows
template <class G>
__device__ __forceinline__ void x2_stage_old(float* R, const float* __restrict__ src, int nyl) {
  // 8-byte pieces where every row starts 8-byte aligned (even NX and RS), else 4-byte ones
  constexpr int W = (G::NXc % 2 == 0 && G::RS % 2 == 0) ? 2 : 1;
  constexpr int H = G::NXc / W;
  for (int i = threadIdx.x; i < 2 * G::NPCc * H; i += G::NT) {
    const int y = i / H, c = i - y * H;
    if (y < nyl) {
      if constexpr (W == 2) cp_async8(R + G::row_off(y) + 2 * c, src + y * G::NXc + 2 * c);
      else cp_async4(R + G::row_off(y) + c, src + y * G::NXc + c);
    }
  }
  cp_async_commit();
}

template <class G>
__device__ __forceinline__ void x2_stage_twiddles(float2* tw, const StepParams& P) {
  for (int i = threadIdx.x; i < 2 * G::NXc; i += G::NT) {
    int e = i;
    if (i >= G::NXc) {
      const int t = i - G::NXc, k1p = t / G::AX1, j2p = t - k1p * G::AX1;
      e = j2p * k1p;
    }
    tw[i] = P.tw[P.ax.tw_off + e];
  }
}

// rows 2 p0 .. 2 p0 + 2 NPC - 1 (y < ny) of a spectrum plane -> pair regions of X
template <class G>
__device__ __forceinline__ void x2_load_rows(float2* X, const float2* __restrict__ src, int p0, int ny) {
  for (int i = threadIdx.x; i < 2 * G::NPCc * G::HX; i += G::NT) {
    const int r = i / G::HX, kx = i - r * G::HX;
    const int y = 2 * p0 + r;
    if (y < ny) cp_async8(&X[(r >> 1) * G::PST + (r & 1) * G::HX + kx], &src[(size_t)y * G::HX + kx]);
  }
  cp_async_commit();
}

// C2R packing (x factor applied to the half spectrum first) and x-inverse step A -> S
template <class G>
__device__ __forceinline__ void x2_xinv_a(const float2* X, float2* S, const float2* twx,
                                          const float2* __restrict__ fac, int nyl) {
  for (int t = threadIdx.x; t < G::T3; t += G::NT) {
    const int j2 = t / G::NPCc, p = t - j2 * G::NPCc;
    if (2 * p >= nyl) continue;
    const float2* ra = X + p * G::PST;
    const float2* rb = ra + G::HX;
    const bool hasb = 2 * p + 1 < nyl;
    float2 z[G::AX1];
    sfor<0, G::AX1>([&](auto J1) {
      constexpr int j1 = decltype(J1)::value;
      const int k = j2 + G::AX2 * j1;
      const bool mir = k >= G::HX;
      const int kk = mir ? G::NXc - k : k;
      float2 a = ra[kk], b = hasb ? rb[kk] : make_float2(0.f, 0.f);
      if (fac) {
        const float2 f = __ldg(&fac[kk]);
        a = cmul(a, f);
        b = cmul(b, f);
      }
      if (kk == 0 || 2 * kk == G::NXc) { a.y = 0.f; b.y = 0.f; }
      if (mir) { a.y = -a.y; b.y = -b.y; }
      z[j1] = make_float2(a.x - b.y, a.y + b.x);
    });
    RDft<G::AX1, true>::run(z);
    sfor<1, G::AX1>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      z[k1] = cmulc(z[k1], twx[j2 * k1]);
    });
    float2* o = S + p * G::PST + j2;
    sfor<0, G::AX1>([&](auto K1) { o[decltype(K1)::value * G::PA] = z[decltype(K1)::value]; });
  }
}

// R2C unpacking of the pairs' Z (in) -> rows 2 p0 .. of a global spectrum plane
template <class G>
__device__ __forceinline__ void x2_unpack_store(const float2* in, float2* __restrict__ dst, int p0, int ny) {
  for (int t = threadIdx.x; t < G::TU; t += G::NT) {
    const int p = t / G::HX, kx = t - p * G::HX;
    const int y0 = 2 * (p0 + p);
    if (y0 >= ny) continue;
    const float2* zp = in + p * G::PST;
    const float2 zk = zp[kx], zm = zp[kx == 0 ? 0 : G::NXc - kx];
    dst[(size_t)y0 * G::HX + kx] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    if (y0 + 1 < ny) dst[(size_t)(y0 + 1) * G::HX + kx] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
  }
}

// x work of the momentum half-step on split planes: components z (spec[1]), x (spec[2],
// times a+_x), y (spec[0]); each: C2R, d+ p, v update with PML, R2C, back to its buffer
template <int NX, int NPC>
__global__ void __launch_bounds__(X2<NX, NPC>::NT, 2) k_xpass2_mom(const __grid_constant__ StepParams P) {
  using G = X2<NX, NPC>;
  if (*P.bad) return;
  extern __shared__ __align__(16) float2 xs2[];
  const float2* twx = xs2;
  const float2* twxT = xs2 + NX;
  float2* S = xs2 + G::TWP;
  float2* X = S + NPC * G::PST;
  float* R = reinterpret_cast<float*>(X + NPC * G::PST);   // staged old rows (G::STG)
  const int z = blockIdx.y;
  const SimPtrs& Q = P.sims[blockIdx.z];
  const int ny = P.ny, p0 = blockIdx.x * NPC;
  const int nyl = min(2 * NPC, ny - 2 * p0);
  const size_t soff = (size_t)z * P.mspec, voff = (size_t)z * P.plane + (size_t)(2 * p0) * NX;
  auto buf_of = [&](int comp) { return (comp == 2 ? Q.spec[1] : (comp == 0 ? Q.spec[2] : Q.spec[0])) + soff; };
  x2_load_rows<G>(X, buf_of(2), p0, ny);
  x2_stage_twiddles<G>(xs2, P);
  const float lz = __ldg(&P.lams[2][z]);
#pragma unroll 1
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = cc == 0 ? 2 : cc - 1;
    float2* buf = buf_of(comp);
    float* v = Q.v[comp] + voff;
    cp_async_wait_all();
    __syncthreads();
    if constexpr (G::STG) x2_stage_old<G>(R, v, nyl);
    x2_xinv_a<G>(X, S, twx, comp == 0 ? P.ap[0] : nullptr, nyl);
    if constexpr (G::STG) cp_async_wait_all();
    __syncthreads();
    p2_mom_update<G, !G::STG>(S, X, twxT, v, G::STG ? R : v, comp == 1 ? P.lams[1] + 2 * p0 : P.lams[comp], comp,
                              lz, P.dt_over_rho0, nyl);
    __syncthreads();
    p2_xfwd_b<G>(X, S);
    __syncthreads();
    if (cc < 2) x2_load_rows<G>(X, buf_of(cc == 0 ? 0 : 1), p0, ny);   // overlaps the stores
    x2_unpack_store<G>(S, buf, p0, ny);
  }
}

// x work of the mass half-step on split planes: components x (spec[2], times a-_x),
// z (spec[1]), y (spec[0]); rho updates, p = c0^2 sum rho, sparse injection /
// Dirichlet / recording on these pairs, R2C of p -> rows of spec[0]
template <int NX, int NPC>
__global__ void __launch_bounds__(X2<NX, NPC>::NT, 2) k_xpass2_mass(const __grid_constant__ StepParams P) {
  using G = X2<NX, NPC>;
  if (*P.bad) return;
  extern __shared__ __align__(16) float2 xs2[];
  const float2* twx = xs2;
  const float2* twxT = xs2 + NX;
  float2* S = xs2 + G::TWP;
  float2* X = S + NPC * G::PST;
  float* R = reinterpret_cast<float*>(X + NPC * G::PST);   // staged old rows (G::STG)
  const int z = blockIdx.y;
  const SimPtrs& Q = P.sims[blockIdx.z];
  const int role = Q.role, shot = Q.shot, tix = P.tidx[blockIdx.z];
  const int ny = P.ny, p0 = blockIdx.x * NPC;
  const int nyl = min(2 * NPC, ny - 2 * p0);
  const int npl = (nyl + 1) / 2;
  const size_t soff = (size_t)z * P.mspec, voff = (size_t)z * P.plane + (size_t)(2 * p0) * NX;
  const float lz = __ldg(&P.lam[2][z]);
  x2_load_rows<G>(X, Q.spec[2] + soff, p0, ny);
  x2_stage_twiddles<G>(xs2, P);
#pragma unroll 1
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = cc == 0 ? 0 : (cc == 1 ? 2 : 1);
    float* rg = Q.rho[comp] + voff;
    cp_async_wait_all();
    __syncthreads();
    if constexpr (G::STG) x2_stage_old<G>(R, rg, nyl);
    x2_xinv_a<G>(X, S, twx, comp == 0 ? P.am[0] : nullptr, nyl);
    if constexpr (G::STG) cp_async_wait_all();
    __syncthreads();
    const float* lam = comp == 1 ? P.lam[1] + 2 * p0 : P.lam[comp];
    const float* rin = G::STG ? R : rg;
    if (cc < 2) {
      x2_load_rows<G>(X, (cc == 0 ? Q.spec[1] : Q.spec[0]) + soff, p0, ny);   // overlaps the update
      p2_mass_update<G, false, !G::STG>(S, nullptr, rg, rin, lam, comp, lz, P.dt_rho0, nyl);
    } else {
      p2_mass_update<G, true, !G::STG>(S, X, rg, rin, lam, comp, lz, P.dt_rho0, nyl);
    }
  }
  __syncthreads();
  p2_assemble_p<G>(X, Q.rho[0] + voff, Q.rho[2] + voff, c2_of(P, Q) + voff, nyl);
  __syncthreads();
  // sparse updates of rho_xi and p on these pairs, then recording.  List offsets pf
  // address pair regions of 2 hx complex of the whole plane; here pair p0 + q sits at
  // region q of stride PST.
  const int key0 = z * P.npair + p0, key1 = key0 + npl;
  float* zf = reinterpret_cast<float*>(X);
  auto loc = [&](int pf) {
    const int q = pf / (4 * G::HX);
    return pf + q * (2 * G::PST - 4 * G::HX) - p0 * 2 * G::PST;
  };
  if (role == ROLE_FORWARD) {
    const float* amp = P.amp_src + ((size_t)shot * P.nt + tix) * P.n_us;
    for (int u = P.us_ptr[key0] + threadIdx.x; u < P.us_ptr[key1]; u += G::NT) {
      const int vx = P.us_vox[u];
      const float a = amp[u];
      Q.rho[0][vx] += a;
      Q.rho[1][vx] += a;
      Q.rho[2][vx] += a;
      zf[loc(P.us_pf[u])] += c2_of(P, Q)[vx] * (3.f * a);
    }
  } else if (role == ROLE_ADJOINT) {
    const float* q = P.qf + ((size_t)shot * P.nt + tix) * P.n_rec;
    for (int u = P.ur_ptr[key0] + threadIdx.x; u < P.ur_ptr[key1]; u += G::NT) {
      float s = 0.f;
      for (int e = P.ur_mptr[u]; e < P.ur_mptr[u + 1]; ++e) s += q[P.ur_mem[e]];
      const float a = ur_coef_of(P, Q)[u] * s;
      const int vx = P.ur_vox[u];
      Q.rho[0][vx] += a;
      Q.rho[1][vx] += a;
      Q.rho[2][vx] += a;
      zf[loc(P.ur_pf[u])] += c2_of(P, Q)[vx] * (3.f * a);
    }
  } else {  // TR: rho_xi(layer) <- g^(Nt - m) / (3 c0^2)
    const float* g = P.ghist + ((size_t)shot * P.nt + (P.nt - 1 - tix)) * P.n_layer;
    for (int j = P.lay_ptr[key0] + threadIdx.x; j < P.lay_ptr[key1]; j += G::NT) {
      const int vx = P.lay_vox[j];
      const float val = g[j] * inv3c2_of(P, Q)[j];
      Q.rho[0][vx] = val;
      Q.rho[1][vx] = val;
      Q.rho[2][vx] = val;
      zf[loc(P.lay_pf[j])] = c2_of(P, Q)[vx] * (3.f * val);
    }
  }
  __syncthreads();
  if (role == ROLE_FORWARD) {
    float* f = P.traces + ((size_t)shot * P.nt + tix) * P.n_rec;
    for (int e = P.rr_ptr[key0] + threadIdx.x; e < P.rr_ptr[key1]; e += G::NT) f[P.rr_col[e]] = zf[loc(P.rr_pf[e])];
    if (P.record_layer) {
      float* g = P.ghist + ((size_t)shot * P.nt + tix) * P.n_layer;
      for (int j = P.lay_ptr[key0] + threadIdx.x; j < P.lay_ptr[key1]; j += G::NT) g[j] = zf[loc(P.lay_pf[j])];
    }
  } else {
    p2_record_gamma(P, Q, zf, role, shot, P.slot[blockIdx.z], P.gam_ptr[key0], P.gam_ptr[key1], G::NT, loc);
  }
  // the recording above only reads X; the forward x step A below reads X and writes S
  // forward x step A of p (pairs in X) -> S, then step B, R2C unpacking -> rows of spec[0]
  for (int t = threadIdx.x; t < G::T4; t += G::NT) {
    const int p = t / G::AX1, k1 = t - p * G::AX1;
    if (2 * p >= nyl) continue;
    const float2* r = X + p * G::PST + k1;
    float2 zz[G::AX2];
    sfor<0, G::AX2>([&](auto K2) { zz[decltype(K2)::value] = r[G::AX1 * decltype(K2)::value]; });
    p2_xfwd_a<G>(zz, p, k1, S, twxT);
  }
  __syncthreads();
  p2_xfwd_b<G>(S, X);
  __syncthreads();
  x2_unpack_store<G>(X, Q.spec[0] + soff, p0, ny);
}

}  // namespace fwi
