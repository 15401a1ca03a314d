// Fused plane kernels with register-resident two-step line transforms for
// compile-time plane sizes (the momentum and mass halves of one step of Alg. 1,
// with the k-space derivatives of App. B, Eqs. 18-19, in the xy directions).
//
// A CTA owns one z-plane of one simulation.  Per field component the work is
// seven phases separated by block barriers, over two shared buffers S and X:
//
//   1 y-inverse, step A   global spectrum (x or y factor applied) -> DFT_BY1 of the
//                         stride-BY2 rows of each column, twiddle          -> S
//   2 y-inverse, step B   DFT_BY2 of each column block                    -> X (rows)
//   3 x-inverse, step A   C2R packing of rows 2p, 2p+1 into Z = A + iB (Hermitian
//                         extension), DFT_AX1 of the stride-AX2 subsequences -> S
//   4 x-inverse, step B   DFT_AX2 gives the derivative at x = k1 + AX1 k2 of both
//                         rows in registers; PML update of the field (global, read
//                         and written in place); forward x step A on the new values
//                         (their subsequence is exactly the stride-AX1 one)   -> X
//   5 x-forward, step B   DFT_AX1                                          -> S (Z)
//   6 y-forward, step A   R2C unpacking of rows from Z, DFT_BY1, twiddle   -> X
//   7 y-forward, step B   DFT_BY2 -> global spectrum
//
// Lines are mapped to threads so that every access is conflict-free or
// coalesced: for the y transforms consecutive threads take consecutive kx; for
// the x transforms of phase 3 consecutive threads take consecutive row pairs
// (the pair stride PST is odd); phases 4 and 5 read rows padded to an odd
// length.  A step-A output of a line of length N = N1 N2 is the sequence
// Y[j2][k1] = exp(-+2 pi i j2 k1 / N) DFT_N1(x[j2 + N2 j1])[k1], step B gives
// X[k1 + N1 k2] = DFT_N2(Y[.][k1])[k2].  Twiddle tables are staged in shared
// memory from the host's FP64-built W_N[k] = exp(-2 pi i k / N).
#pragma once
#include "kernels.cuh"
#include "rfft.cuh"

namespace fwi {

#ifndef P2_TW_POW
#define P2_TW_POW 1
#endif
#ifndef P2_REMAP
#define P2_REMAP 1
#endif
#ifndef P2_NT160
#define P2_NT160 512
#endif
#ifndef P2_NT135
#define P2_NT135 352
#endif
#ifndef P2_NT96
#define P2_NT96 512
#endif
#ifndef P2_NT64
#define P2_NT64 288
#endif
#ifndef P2_NT128
#define P2_NT128 640
#endif

__host__ __device__ constexpr int cmax3(int a, int b, int c) { return a > b ? (a > c ? a : c) : (b > c ? b : c); }

template <int NX, int NY>
struct Plane2 {
  static constexpr int NXc = NX, NYc = NY;
  static constexpr int HX = NX / 2 + 1;
  static constexpr int NP = (NY + 1) / 2;
  static constexpr int AX1 = split_n1(NX), AX2 = NX / AX1;
  static constexpr int BY1 = split_n1(NY), BY2 = NY / BY1;
  static constexpr int PA = AX2 + 1;     // padded row of the x-inverse step-A output
  static constexpr int PB = AX1 + 1;     // padded row of the x-forward step-A output
  static constexpr int PST = cmax3(2 * HX, AX1 * PA, AX2 * PB) | 1;   // pair stride (odd)
  // task counts of the phases
  static constexpr int T1 = HX * BY2, T2 = HX * BY1, T3 = NP * AX2, T4 = NP * AX1;
  // Threads per CTA (one CTA per SM: the plane buffers take most of shared memory).
  // Chosen per size by measurement, among counts whose registers fit 64K per SM; for
  // 128 the phases' 1040, 520, 1024 and 512 tasks take 2, 1, 2 and 1 rounds of 640
  // threads (544 fills the rounds better but hides less latency: 0.7 % slower); for 160,
  // whose planes cannot be staged, 512 threads hide more of the global loads than 416
  // (+4.8 % on a 160 x 160 x 80 gradient) and 640 less (+0.6 %); for 96, 512 rather than
  // 416 (+2.1 % on a 96 x 96 x 48 gradient); 135 and 64 gain nothing from 448 / 384.
  static constexpr int NT = NX == 128 ? P2_NT128 : NX == 135 ? P2_NT135 : NX == 160 ? P2_NT160 : NX == 96 ? P2_NT96
                          : NX == 64 ? P2_NT64 : 128;
  static constexpr int TW = NX + NX + NY;                 // twx, twxT, twy
  // Phase-4 task order.  Tasks (p, k1) of one half-warp read and write 64-bit words at
  // p PST + k1 + const in S and X; with AX1 = 8 and PST = PA = 1 (mod 16) the row pairs
  // p and p + 1 would share seven of their eight banks.  REMAP pairs p with p + 8
  // instead (PST 8 = 8 mod 16: disjoint banks); the warp's four row pairs are then
  // p, p + 8, p + 1, p + 9.
  static constexpr bool REMAP = P2_REMAP && AX1 == 8 && AX2 % 16 == 0 && PST % 16 == 1 && NP % 16 == 0;
  // staging buffer (complex units) for the next global input: a spectrum plane, or a
  // real field plane with padded rows.  Row y starts at row_off(y) floats (a multiple of
  // 4: 16-byte copies).  The phase-4 reads of one warp take 8 floats from each of the
  // rows 2p of its four row pairs: rows NX + 4 long make p = 0..3 (the order without
  // REMAP) hit the bank windows 0, 8, 16, 24; with REMAP, rows NX + 8 long plus 8 floats
  // on every other block of 16 rows do the same for p, p + 8, p + 1, p + 9.
  static constexpr int RS = REMAP ? NX + 8 : NX + 4;
  __host__ __device__ static constexpr int row_off(int y) { return y * RS + (REMAP ? 8 * ((y >> 4) & 1) : 0); }
  static constexpr int GS = (HX * NY > (row_off(NY - 1) + NX + 1) / 2) ? HX * NY : (row_off(NY - 1) + NX + 1) / 2;
  static constexpr int TWP = (TW + 1) & ~1;              // keeps the buffers 16-byte aligned
  static constexpr size_t SMEM_NOSTAGE = (size_t)(TWP + 2 * NP * PST) * 8;
  static constexpr bool STAGE = SMEM_NOSTAGE + (size_t)GS * 8 <= 227 * 1024 && (HX * NY) % 2 == 0;
  static constexpr size_t SMEM = SMEM_NOSTAGE + (STAGE ? (size_t)GS * 8 : 0);
};

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// asynchronous copy of a spectrum plane (HX * NY complex, contiguous) into G
template <class G>
__device__ __forceinline__ void p2_fetch_spec(float2* Gb, const float2* __restrict__ src) {
  static_assert((G::HX * G::NYc) % 2 == 0, "spectrum planes are copied in 16-byte pieces");
  static_assert((G::TWP + G::NP * G::PST) % 2 == 0, "buffers must start on 16-byte boundaries");
  constexpr int n16 = G::HX * G::NYc / 2;
  for (int i = threadIdx.x; i < n16; i += G::NT) cp_async16(Gb + 2 * i, src + 2 * i);
  cp_async_commit();
}
// asynchronous copy of a real field plane (NY rows of NX floats) into G, rows padded
template <class G>
__device__ __forceinline__ void p2_fetch_rows(float2* Gb, const float* __restrict__ src) {
  static_assert(G::NXc % 4 == 0, "rows are copied in 16-byte pieces");
  constexpr int per_row = G::NXc / 4;
  float* d = reinterpret_cast<float*>(Gb);
  for (int i = threadIdx.x; i < G::NYc * per_row; i += G::NT) {
    const int y = i / per_row, c = i - y * per_row;
    cp_async16(d + G::row_off(y) + 4 * c, src + y * G::NXc + 4 * c);
  }
  cp_async_commit();
}

#ifndef P2_STAGE_STATE
#define P2_STAGE_STATE 1
#endif

__host__ __device__ constexpr int hibit(int k) { return k <= 1 ? k : 2 * hibit(k / 2); }

// w[k] = tab[base * k * step]... for k < M: the step-A twiddles of one task.  With
// P2_TW_POW the powers of two are read from the table and the others formed as
// products (fewer shared-memory loads, a few ulp of extra rounding).
template <int M>
__device__ __forceinline__ void tw_row(const float2* tab, int stride, float2 (&w)[M]) {
  w[0] = make_float2(1.f, 0.f);
  sfor<1, M>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr int h = hibit(k);
    if constexpr (P2_TW_POW && h != k) w[k] = cmul(w[h], w[k - h]);
    else w[k] = tab[k * stride];
  });
}

template <class G>
__device__ __forceinline__ float2* p2_row(float2* buf, int ky) {
  return buf + (ky >> 1) * G::PST + (ky & 1) * G::HX;
}

// phase-4 task t -> row pair p and column k1 (see Plane2::REMAP)
template <class G>
__device__ __forceinline__ void p2_task4(int t, int& p, int& k1) {
  const int q = t / G::AX1;
  k1 = t - q * G::AX1;
  if constexpr (G::REMAP) p = (q & ~15) | ((q & 1) << 3) | ((q >> 1) & 7);
  else p = q;
}

// twiddles: twx[e] = W_NX^e, twxT[k1' AX1 + j2'] = W_NX^(j2' k1'), twy[e] = W_NY^e
template <class G>
__device__ __forceinline__ void p2_stage_twiddles(float2* tw, const StepParams& P) {
  for (int i = threadIdx.x; i < G::TW; i += blockDim.x) {
    float2 w;
    if (i < 2 * G::AX1 * G::AX2) {
      int e = i;
      if (i >= G::AX1 * G::AX2) {
        const int t = i - G::AX1 * G::AX2;
        const int k1p = t / G::AX1, j2p = t - k1p * G::AX1;
        e = j2p * k1p;
      }
      w = P.tw[P.ax.tw_off + e];
    } else {
      w = P.tw[P.ay.tw_off + (i - 2 * G::AX1 * G::AX2)];
    }
    tw[i] = w;
  }
}

// phase 1: global spectrum plane (factor: 0 none, 1 per kx, 2 per ky) -> S
template <class G>
__device__ __forceinline__ void p2_yinv_a(float2* S, const float2* src, int fk,
                                          const float2* __restrict__ fac, const float2* twy) {
  for (int t = threadIdx.x; t < G::T1; t += G::NT) {
    const int j2 = t / G::HX, kx = t - j2 * G::HX;
    float2 a[G::BY1];
    sfor<0, G::BY1>([&](auto J1) {
      constexpr int j1 = decltype(J1)::value;
      a[j1] = src[(j2 + G::BY2 * j1) * G::HX + kx];   // staged plane (shared) or global
    });
    if (fk == 1) {
      const float2 f = __ldg(&fac[kx]);
      sfor<0, G::BY1>([&](auto J1) { a[decltype(J1)::value] = cmul(a[decltype(J1)::value], f); });
    } else if (fk == 2) {
      sfor<0, G::BY1>([&](auto J1) {
        constexpr int j1 = decltype(J1)::value;
        a[j1] = cmul(a[j1], __ldg(&fac[j2 + G::BY2 * j1]));
      });
    }
    RDft<G::BY1, true>::run(a);
    float2 w[G::BY1];
    tw_row<G::BY1>(twy, j2, w);
    sfor<1, G::BY1>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      a[k1] = cmulc(a[k1], w[k1]);
    });
    sfor<0, G::BY1>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      p2_row<G>(S, j2 + G::BY2 * k1)[kx] = a[k1];
    });
  }
}

// phase 2 (INV) and 7 (!INV, to global): column step B
template <class G, bool INV>
__device__ __forceinline__ void p2_y_b(const float2* in, float2* out_smem, float2* __restrict__ out_glob) {
  for (int t = threadIdx.x; t < G::T2; t += G::NT) {
    const int k1 = t / G::HX, kx = t - k1 * G::HX;
    float2 a[G::BY2];
    sfor<0, G::BY2>([&](auto J2) {
      constexpr int j2 = decltype(J2)::value;
      a[j2] = p2_row<G>(const_cast<float2*>(in), G::BY2 * k1 + j2)[kx];
    });
    RDft<G::BY2, INV>::run(a);
    if (INV) {
      sfor<0, G::BY2>([&](auto K2) {
        constexpr int k2 = decltype(K2)::value;
        p2_row<G>(out_smem, k1 + G::BY1 * k2)[kx] = a[k2];
      });
    } else {
      sfor<0, G::BY2>([&](auto K2) {
        constexpr int k2 = decltype(K2)::value;
        out_glob[(k1 + G::BY1 * k2) * G::HX + kx] = a[k2];
      });
    }
  }
}

// phase 3: rows (pair-line layout in X) -> C2R packing -> x step A -> S
template <class G>
__device__ __forceinline__ void p2_xinv_a(const float2* X, float2* S, const float2* twx) {
  for (int t = threadIdx.x; t < G::T3; t += G::NT) {
    const int j2 = t / G::NP, p = t - j2 * G::NP;
    const float2* ra = X + p * G::PST;
    const float2* rb = ra + G::HX;
    const bool hasb = 2 * p + 1 < G::NYc;
    float2 z[G::AX1];
    sfor<0, G::AX1>([&](auto J1) {
      constexpr int j1 = decltype(J1)::value;
      const int k = j2 + G::AX2 * j1;
      float2 a, b = make_float2(0.f, 0.f);
      if (k < G::HX) {
        a = ra[k];
        if (hasb) b = rb[k];
        if (k == 0 || 2 * k == G::NXc) { a.y = 0.f; b.y = 0.f; }
      } else {
        const int kk = G::NXc - k;
        a = ra[kk];
        if (hasb) b = rb[kk];
        a.y = -a.y;
        b.y = -b.y;
      }
      z[j1] = make_float2(a.x - b.y, a.y + b.x);
    });
    RDft<G::AX1, true>::run(z);
    float2 w[G::AX1];
    tw_row<G::AX1>(twx, j2, w);
    sfor<1, G::AX1>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      z[k1] = cmulc(z[k1], w[k1]);
    });
    float2* o = S + p * G::PST + j2;
    sfor<0, G::AX1>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      o[k1 * G::PA] = z[k1];
    });
  }
}

// forward x step A of the values z[k2] at x = k1 + AX1 k2 of pair p -> out
template <class G>
__device__ __forceinline__ void p2_xfwd_a(float2* z, int p, int k1, float2* out, const float2* twxT) {
  RDft<G::AX2, false>::run(z);
  float2* o = out + p * G::PST + k1;
  float2 w[G::AX2];
  tw_row<G::AX2>(twxT + k1, G::AX1, w);
  sfor<0, G::AX2>([&](auto K1P) {
    constexpr int k1p = decltype(K1P)::value;
    o[k1p * G::PB] = k1p == 0 ? z[k1p] : cmul(z[k1p], w[k1p]);
  });
}

// phase 5: x step B (forward) -> Z[k] of each pair in `out`
template <class G>
__device__ __forceinline__ void p2_xfwd_b(const float2* in, float2* out) {
  for (int t = threadIdx.x; t < G::T3; t += G::NT) {
    const int p = t / G::AX2, k1p = t - p * G::AX2;
    const float2* r = in + p * G::PST + k1p * G::PB;
    float2 u[G::AX1];
    sfor<0, G::AX1>([&](auto J) { u[decltype(J)::value] = r[decltype(J)::value]; });
    RDft<G::AX1, false>::run(u);
    float2* o = out + p * G::PST + k1p;
    sfor<0, G::AX1>([&](auto K2) {
      constexpr int k2 = decltype(K2)::value;
      o[G::AX2 * k2] = u[k2];
    });
  }
}

// phase 6: R2C unpacking of rows from Z (in) -> y step A (forward) -> out
template <class G>
__device__ __forceinline__ void p2_yfwd_a(const float2* in, float2* out, const float2* twy) {
  for (int t = threadIdx.x; t < G::T1; t += G::NT) {
    const int j2 = t / G::HX, kx = t - j2 * G::HX;
    const int km = kx == 0 ? 0 : G::NXc - kx;
    float2 a[G::BY1];
    sfor<0, G::BY1>([&](auto J1) {
      constexpr int j1 = decltype(J1)::value;
      const int ky = j2 + G::BY2 * j1;
      const float2* zp = in + (ky >> 1) * G::PST;
      const float2 zk = zp[kx], zm = zp[km];
      a[j1] = (ky & 1) ? make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x))
                       : make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    });
    RDft<G::BY1, false>::run(a);
    float2 w[G::BY1];
    tw_row<G::BY1>(twy, j2, w);
    sfor<1, G::BY1>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      a[k1] = cmul(a[k1], w[k1]);
    });
    sfor<0, G::BY1>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      p2_row<G>(out, j2 + G::BY2 * k1)[kx] = a[k1];
    });
  }
}

// Old field values come from the staged rows in shared memory, or (GIN) from global memory,
// where each element is read once by the thread that later overwrites it and by no other
// thread: a read-only (non-coherent) load is then safe, and it lets the loads of all k2 be
// issued before the stores instead of one round trip after another.
template <bool GIN>
__device__ __forceinline__ float old_value(const float* p) {
  if constexpr (GIN) return __ldg(p);
  else return *p;
}

// phase 4, momentum: derivative of both rows in registers, v_comp update in place
// (Lambda^s (Lambda^s v - dt/rho0 d+ p)), then forward x step A of the new v -> out
template <class G, bool GIN>
__device__ __forceinline__ void p2_mom_update(const float2* S, float2* out, const float2* twxT,
                                              float* __restrict__ v, const float* vin,
                                              const float* __restrict__ lam, int comp, float lz, float dtr,
                                              int nyl) {
  for (int t = threadIdx.x; t < G::T4; t += G::NT) {
    int p, k1;
    p2_task4<G>(t, p, k1);
    const int y0 = 2 * p, y1 = y0 + 1;
    if (y0 >= nyl) continue;
    const bool has1 = y1 < nyl;
    float* v0p = v + y0 * G::NXc + k1;
    float* v1p = v0p + G::NXc;
    // old values: global rows, or staged rows (y0 even: rows y0 and y0 + 1 share a block of 16)
    const float* i0 = vin + (GIN ? y0 * G::NXc : G::row_off(y0)) + k1;
    const float* i1 = i0 + (GIN ? G::NXc : G::RS);
    // the old field is loaded ahead of the transform unless that would hold too many
    // registers (long step-B lines)
    constexpr bool PRE = G::AX2 <= 16;
    float s0[PRE ? G::AX2 : 1], s1[PRE ? G::AX2 : 1];
    if constexpr (PRE) {
      sfor<0, G::AX2>([&](auto K2) {
        constexpr int k2 = decltype(K2)::value;
        s0[k2] = old_value<GIN>(&i0[G::AX1 * k2]);
        s1[k2] = has1 ? old_value<GIN>(&i1[G::AX1 * k2]) : 0.f;
      });
    }
    float2 z[G::AX2];
    const float2* r = S + p * G::PST + k1 * G::PA;
    sfor<0, G::AX2>([&](auto J) { z[decltype(J)::value] = r[decltype(J)::value]; });
    RDft<G::AX2, true>::run(z);
    float l0 = lz, l1 = lz;
    if (comp == 1) {
      l0 = __ldg(&lam[y0]);
      l1 = has1 ? __ldg(&lam[y1]) : 1.f;
    }
    sfor<0, G::AX2>([&](auto K2) {
      constexpr int k2 = decltype(K2)::value;
      float a0 = l0, a1 = l1;
      if (comp == 0) a0 = a1 = __ldg(&lam[k1 + G::AX1 * k2]);
      float o0v, o1v;
      if constexpr (PRE) { o0v = s0[k2]; o1v = s1[k2]; }
      else { o0v = old_value<GIN>(&i0[G::AX1 * k2]); o1v = has1 ? old_value<GIN>(&i1[G::AX1 * k2]) : 0.f; }
      const float n0 = a0 * (a0 * o0v - dtr * z[k2].x);
      v0p[G::AX1 * k2] = n0;
      float n1 = 0.f;
      if (has1) {
        n1 = a1 * (a1 * o1v - dtr * z[k2].y);
        v1p[G::AX1 * k2] = n1;
      }
      z[k2] = make_float2(n0, n1);
    });
    p2_xfwd_a<G>(z, p, k1, out, twxT);
  }
}

// phase 4, mass: rho_comp <- Lambda (Lambda rho - dt rho0 d- v); for the last
// component the new rho_y is also written as pairs to pout, where p2_assemble_p turns
// it into p = c0^2 (rho_x + rho_y + rho_z).
template <class G, bool LAST, bool GIN>
__device__ __forceinline__ void p2_mass_update(const float2* S, float2* pout, float* __restrict__ rho,
                                               const float* rin, const float* __restrict__ lam,
                                               int comp, float lz, float dtr0, int nyl) {
  for (int t = threadIdx.x; t < G::T4; t += G::NT) {
    int p, k1;
    p2_task4<G>(t, p, k1);
    const int y0 = 2 * p, y1 = y0 + 1;
    if (y0 >= nyl) continue;
    const bool has1 = y1 < nyl;
    const int o0 = y0 * G::NXc + k1, o1 = o0 + G::NXc;
    const float* i0 = rin + (GIN ? y0 * G::NXc : G::row_off(y0)) + k1;
    const float* i1 = i0 + (GIN ? G::NXc : G::RS);
    constexpr bool PRE = G::AX2 <= 16;   // as in the momentum update
    float s0[PRE ? G::AX2 : 1], s1[PRE ? G::AX2 : 1];
    if constexpr (PRE) {
      sfor<0, G::AX2>([&](auto K2) {
        constexpr int k2 = decltype(K2)::value;
        s0[k2] = old_value<GIN>(&i0[G::AX1 * k2]);
        s1[k2] = has1 ? old_value<GIN>(&i1[G::AX1 * k2]) : 0.f;
      });
    }
    float2 z[G::AX2];
    const float2* r = S + p * G::PST + k1 * G::PA;
    sfor<0, G::AX2>([&](auto J) { z[decltype(J)::value] = r[decltype(J)::value]; });
    RDft<G::AX2, true>::run(z);
    float l0 = lz, l1 = lz;
    if (comp == 1) {
      l0 = __ldg(&lam[y0]);
      l1 = has1 ? __ldg(&lam[y1]) : 1.f;
    }
    float2* po = pout + p * G::PST + k1;
    sfor<0, G::AX2>([&](auto K2) {
      constexpr int k2 = decltype(K2)::value;
      constexpr int xo = G::AX1 * k2;
      float a0 = l0, a1 = l1;
      if (comp == 0) a0 = a1 = __ldg(&lam[k1 + xo]);
      float o0v, o1v;
      if constexpr (PRE) { o0v = s0[k2]; o1v = s1[k2]; }
      else { o0v = old_value<GIN>(&i0[xo]); o1v = has1 ? old_value<GIN>(&i1[xo]) : 0.f; }
      const float r0 = a0 * (a0 * o0v - dtr0 * z[k2].x);
      rho[o0 + xo] = r0;
      float r1 = 0.f;
      if (has1) {
        r1 = a1 * (a1 * o1v - dtr0 * z[k2].y);
        rho[o1 + xo] = r1;
      }
      if (LAST) po[xo] = make_float2(r0, r1);
    });
  }
}

// p = c0^2 (rho_x + rho_y + rho_z) on the rows held as pairs in X (Alg. 1, pressure-density
// relation): the new rho_y of pair q is at X[q PST + x] (rows 2q, 2q + 1), rho_x, rho_z and
// c0^2 come from global rows (row length NX, first row at the pointers).  Consecutive
// threads take consecutive x, 16 bytes per load where rows allow it, so the three arrays
// are read in full 128-byte lines with a quarter of the load instructions of a per-voxel
// gather.  rho_x and rho_z were written earlier in this launch by the same CTA, with a
// block barrier in between: they are read with ordinary (coherent) loads.  The sum is
// formed as (rho_x + rho_y) + rho_z.
template <class G>
__device__ __forceinline__ void p2_assemble_p(float2* X, const float* rx, const float* rz,
                                              const float* __restrict__ c2, int nyl) {
  constexpr int NXc = G::NXc;
  constexpr int V = NXc % 4 == 0 ? 4 : 1;
  constexpr int QV = NXc / V;
  const int npl = (nyl + 1) / 2;
  for (int t = threadIdx.x; t < npl * QV; t += G::NT) {
    const int q = t / QV, x = V * (t - q * QV);
    const int y0 = 2 * q;
    const bool has1 = y0 + 1 < nyl;
    const int o0 = y0 * NXc + x, o1 = o0 + NXc;
    float2* xp = X + q * G::PST + x;
    if constexpr (V == 4) {
      const float4 a0 = *reinterpret_cast<const float4*>(rx + o0);
      const float4 b0 = *reinterpret_cast<const float4*>(rz + o0);
      const float4 c0 = __ldg(reinterpret_cast<const float4*>(c2 + o0));
      float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = a1, c1 = a1;
      if (has1) {
        a1 = *reinterpret_cast<const float4*>(rx + o1);
        b1 = *reinterpret_cast<const float4*>(rz + o1);
        c1 = __ldg(reinterpret_cast<const float4*>(c2 + o1));
      }
      const float av0[4] = {a0.x, a0.y, a0.z, a0.w}, bv0[4] = {b0.x, b0.y, b0.z, b0.w};
      const float cv0[4] = {c0.x, c0.y, c0.z, c0.w}, av1[4] = {a1.x, a1.y, a1.z, a1.w};
      const float bv1[4] = {b1.x, b1.y, b1.z, b1.w}, cv1[4] = {c1.x, c1.y, c1.z, c1.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 r = xp[j];
        xp[j] = make_float2(cv0[j] * (av0[j] + r.x + bv0[j]), has1 ? cv1[j] * (av1[j] + r.y + bv1[j]) : 0.f);
      }
    } else {
      const float2 r = xp[0];
      const float p0v = __ldg(&c2[o0]) * (rx[o0] + r.x + rz[o0]);
      const float p1v = has1 ? __ldg(&c2[o1]) * (rx[o1] + r.y + rz[o1]) : 0.f;
      xp[0] = make_float2(p0v, p1v);
    }
  }
}

// float offset pf of the pair-line plane buffer (regions of 2 hx complex) -> the
// same voxel in a buffer of pair stride PST
template <class G>
__device__ __forceinline__ int p2_pf(int pf) {
  const int q = pf / (4 * G::HX);
  return pf + q * (2 * G::PST - 4 * G::HX);
}

// Record the pressure on Gamma for the entries [j0, j1) of this CTA's Gamma list: the
// adjoint role writes pa (first adding the previous iteration's term of the gradient,
// acc += 2/(dt c0^3) (P(s0) - 2 P(s1) + P(s2)) pa_old, in FP64, when P.acc_prev is set:
// Alg. 1's accumulation, deferred by one launch because P(s2) is written by the TR
// simulations of the launch that produced pa_old), the TR role writes its ring slot.
// `at(pf)` maps a list offset to the shared plane buffer.
template <class AT>
__device__ __forceinline__ void p2_record_gamma(const StepParams& P, const SimPtrs& Q, const float* zf, int role,
                                                int shot, int slot, int j0, int j1, int stride, AT at) {
  if (role == ROLE_ADJOINT) {
    float* pa = P.pa + (size_t)shot * P.n_gamma;
    if (P.acc_prev) {
      const size_t n = P.n_gamma;
      const float* rk = P.ring + (size_t)shot * kRing * n;
      const float* r0 = rk + P.acc_slot[0] * n;
      const float* r1 = rk + P.acc_slot[1] * n;
      const float* r2 = rk + P.acc_slot[2] * n;
      double* acc = P.acc + (size_t)shot * n;
      const float* cg = coefG_of(P, Q);
      for (int j = j0 + (int)threadIdx.x; j < j1; j += stride) {
        const double d2 = (double)r0[j] - 2.0 * (double)r1[j] + (double)r2[j];
        acc[j] += (double)cg[j] * d2 * (double)pa[j];
        pa[j] = zf[at(P.gam_pf[j])];
      }
    } else {
      for (int j = j0 + (int)threadIdx.x; j < j1; j += stride) pa[j] = zf[at(P.gam_pf[j])];
    }
  } else {
    float* out = P.ring + ((size_t)shot * kRing + slot) * P.n_gamma;
    for (int j = j0 + (int)threadIdx.x; j < j1; j += stride) out[j] = zf[at(P.gam_pf[j])];
  }
}

template <int NX, int NY>
__global__ void __launch_bounds__(Plane2<NX, NY>::NT, 1) k_plane2_mom(const __grid_constant__ StepParams P) {
  using G = Plane2<NX, NY>;
  if (*P.bad) return;
  extern __shared__ __align__(16) float2 sm2[];
  const float2* twx = sm2;
  const float2* twxT = sm2 + NX;
  const float2* twy = sm2 + 2 * NX;
  float2* S = sm2 + G::TWP;
  float2* X = S + G::NP * G::PST;
  float2* Gb = X + G::NP * G::PST;      // staging buffer (when G::STAGE)
  const int z = blockIdx.x;
  const SimPtrs& Q = P.sims[blockIdx.y];
  const size_t soff = (size_t)z * (G::HX * NY);
  const size_t voff = (size_t)z * (NX * NY);
  // component order z, x, y: R -> V_z (spec[1]), Q -> V_x (spec[2]), Q -> V_y (spec[0])
  auto src_of = [&](int comp) { return (comp == 2 ? Q.spec[1] : Q.spec[0]) + soff; };
  auto comp_of = [](int cc) { return cc == 0 ? 2 : cc - 1; };
  auto phase1 = [&](int comp) {
    p2_yinv_a<G>(S, G::STAGE ? Gb : src_of(comp), comp == 2 ? 0 : (comp == 0 ? 1 : 2), P.ap[comp], twy);
  };
  if constexpr (G::STAGE) p2_fetch_spec<G>(Gb, src_of(2));
  p2_stage_twiddles<G>(sm2, P);
  const float lz = __ldg(&P.lams[2][z]);
  if constexpr (G::STAGE) cp_async_wait_all();
  __syncthreads();
  phase1(comp_of(0));
#pragma unroll 1
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = comp_of(cc);
    float2* dst = (comp == 2 ? Q.spec[1] : (comp == 0 ? Q.spec[2] : Q.spec[0])) + soff;
    float* vg = Q.v[comp] + voff;
    constexpr bool SS = G::STAGE && P2_STAGE_STATE;
    __syncthreads();
    if constexpr (SS) p2_fetch_rows<G>(Gb, vg);      // overlaps phases 2 and 3
    p2_y_b<G, true>(S, X, nullptr);
    __syncthreads();
    p2_xinv_a<G>(X, S, twx);
    if constexpr (SS) cp_async_wait_all();
    __syncthreads();
    p2_mom_update<G, !SS>(S, X, twxT, vg, SS ? reinterpret_cast<const float*>(Gb) : vg, P.lams[comp], comp, lz,
                          P.dt_over_rho0, NY);
    __syncthreads();
    if constexpr (G::STAGE) {                        // next spectrum overlaps phases 5-7
      if (cc < 2) p2_fetch_spec<G>(Gb, src_of(comp_of(cc + 1)));
    }
    p2_xfwd_b<G>(X, S);
    __syncthreads();
    p2_yfwd_a<G>(S, X, twy);
    if constexpr (G::STAGE) cp_async_wait_all();
    __syncthreads();
    p2_y_b<G, false>(X, nullptr, dst);
    // phase 1 of the next component shares this interval: it writes S (last read by
    // phase 6) from the staged spectrum, phase 7 reads X
    if (cc < 2) phase1(comp_of(cc + 1));
  }
}

template <int NX, int NY>
__global__ void __launch_bounds__(Plane2<NX, NY>::NT, 1) k_plane2_mass(const __grid_constant__ StepParams P) {
  using G = Plane2<NX, NY>;
  if (*P.bad) return;
  extern __shared__ __align__(16) float2 sm2[];
  const float2* twx = sm2;
  const float2* twxT = sm2 + NX;
  const float2* twy = sm2 + 2 * NX;
  float2* S = sm2 + G::TWP;
  float2* X = S + G::NP * G::PST;
  float2* Gb = X + G::NP * G::PST;      // staging buffer (when G::STAGE)
  const int z = blockIdx.x;
  const SimPtrs& Q = P.sims[blockIdx.y];
  const int role = Q.role, shot = Q.shot, tix = P.tidx[blockIdx.y];
  const size_t soff = (size_t)z * (G::HX * NY);
  const size_t voff = (size_t)z * (NX * NY);
  const float lz = __ldg(&P.lam[2][z]);
  // component order x (spec[2]), z (spec[1]), y (spec[0]); the last one assembles p.
  // Spectra of the second and third components are staged in X, which is free from
  // the end of phase 3 to the next phase 2; rho rows in the staging buffer.
  if constexpr (G::STAGE) p2_fetch_spec<G>(Gb, Q.spec[2] + soff);
  p2_stage_twiddles<G>(sm2, P);
  constexpr bool SS = G::STAGE && P2_STAGE_STATE;
#pragma unroll 1
  for (int cc = 0; cc < 3; ++cc) {
    const int comp = cc == 0 ? 0 : (cc == 1 ? 2 : 1);
    float* rg = Q.rho[comp] + voff;
    const float2* src = cc == 0 ? (G::STAGE ? Gb : Q.spec[2] + soff) : X;
    cp_async_wait_all();
    __syncthreads();
    p2_yinv_a<G>(S, src, comp == 2 ? 0 : (comp == 0 ? 1 : 2), P.am[comp], twy);
    __syncthreads();
    if constexpr (SS) p2_fetch_rows<G>(Gb, rg);      // overlaps phases 2 and 3
    p2_y_b<G, true>(S, X, nullptr);
    __syncthreads();
    p2_xinv_a<G>(X, S, twx);
    if constexpr (SS) cp_async_wait_all();
    __syncthreads();
    const float* rin = SS ? reinterpret_cast<const float*>(Gb) : rg;
    if (cc < 2) {
      p2_fetch_spec<G>(X, (cc == 0 ? Q.spec[1] : Q.spec[0]) + soff);   // overlaps phase 4
      p2_mass_update<G, false, !SS>(S, nullptr, rg, rin, P.lam[comp], comp, lz, P.dt_rho0, NY);
    } else {
      p2_mass_update<G, true, !SS>(S, X, rg, rin, P.lam[1], 1, lz, P.dt_rho0, NY);
    }
  }
  __syncthreads();
  p2_assemble_p<G>(X, Q.rho[0] + voff, Q.rho[2] + voff, c2_of(P, Q) + voff, NY);
  __syncthreads();
  // sparse updates of rho_xi and p on this plane, then recording
  const int key0 = z * G::NP, key1 = key0 + G::NP;
  float* zf = reinterpret_cast<float*>(X);
  if (role == ROLE_FORWARD) {
    const float* amp = P.amp_src + ((size_t)shot * P.nt + tix) * P.n_us;
    for (int u = P.us_ptr[key0] + threadIdx.x; u < P.us_ptr[key1]; u += G::NT) {
      const int vx = P.us_vox[u];
      const float a = amp[u];
      Q.rho[0][vx] += a;
      Q.rho[1][vx] += a;
      Q.rho[2][vx] += a;
      zf[p2_pf<G>(P.us_pf[u])] += c2_of(P, Q)[vx] * (3.f * a);
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
      zf[p2_pf<G>(P.ur_pf[u])] += c2_of(P, Q)[vx] * (3.f * a);
    }
  } else {  // TR: rho_xi(layer) <- g^(Nt - m) / (3 c0^2)
    const float* g = P.ghist + ((size_t)shot * P.nt + (P.nt - 1 - tix)) * P.n_layer;
    for (int j = P.lay_ptr[key0] + threadIdx.x; j < P.lay_ptr[key1]; j += G::NT) {
      const int vx = P.lay_vox[j];
      const float val = g[j] * inv3c2_of(P, Q)[j];
      Q.rho[0][vx] = val;
      Q.rho[1][vx] = val;
      Q.rho[2][vx] = val;
      zf[p2_pf<G>(P.lay_pf[j])] = c2_of(P, Q)[vx] * (3.f * val);
    }
  }
  __syncthreads();
  if (role == ROLE_FORWARD) {
    float* f = P.traces + ((size_t)shot * P.nt + tix) * P.n_rec;
    for (int e = P.rr_ptr[key0] + threadIdx.x; e < P.rr_ptr[key1]; e += G::NT) f[P.rr_col[e]] = zf[p2_pf<G>(P.rr_pf[e])];
    if (P.record_layer) {
      float* g = P.ghist + ((size_t)shot * P.nt + tix) * P.n_layer;
      for (int j = P.lay_ptr[key0] + threadIdx.x; j < P.lay_ptr[key1]; j += G::NT) g[j] = zf[p2_pf<G>(P.lay_pf[j])];
    }
  } else {
    p2_record_gamma(P, Q, zf, role, shot, P.slot[blockIdx.y], P.gam_ptr[key0], P.gam_ptr[key1], G::NT,
                    [](int pf) { return p2_pf<G>(pf); });
  }
  // the recording above only reads X, the forward x step A below reads X and writes S: they share
  // one barrier interval
  // forward x step A of p (pairs in X) -> S, then step B, R2C unpacking and y
  for (int t = threadIdx.x; t < G::T4; t += G::NT) {
    int p, k1;
    p2_task4<G>(t, p, k1);
    const float2* r = X + p * G::PST + k1;
    float2 zz[G::AX2];
    sfor<0, G::AX2>([&](auto K2) { zz[decltype(K2)::value] = r[G::AX1 * decltype(K2)::value]; });
    p2_xfwd_a<G>(zz, p, k1, S, twxT);
  }
  __syncthreads();
  p2_xfwd_b<G>(S, X);
  __syncthreads();
  p2_yfwd_a<G>(X, S, twy);
  __syncthreads();
  p2_y_b<G, false>(S, nullptr, Q.spec[0] + soff);
}

}  // namespace fwi

namespace fwi {

// ---------------------------------------------------------------------------
// z pass with two-step register transforms (compile-time nz).  A CTA holds TZ
// adjacent (ky, kx) spectrum columns; consecutive threads take consecutive
// columns, so global rows are read and written as TZ * 8 contiguous bytes and
// shared rows [z][TZ] are conflict-free.  Per column and output:
//   forward step A (from global) -> smem -> forward step B gives X[kz] at
//   kz = k1 + N1 k2 in registers -> times kappa / N (and the z factor) ->
//   inverse step A on that stride-N1 subsequence -> smem -> inverse step B
//   -> global.
// MODE 0 (momentum): spec[0] -> Q (spec[0]) and R = Q a+_z (spec[1]).
// MODE 1 (mass): spec[2] (x), spec[0] (y), spec[1] (z, times a-_z), in place.
// kappa(k) / N = sinc(c_ref dt |k| / 2) / N (Eq. 18).  For arguments a <= 3.1 the sinc is
// the Taylor series of sin(a)/a, sum (-1)^n a^(2n) / (2n+1)!, truncated after a^18 (error
// below 2e-10 there) and evaluated by Horner's rule in s = a^2 = (c_ref dt / 2)^2 |k|^2:
// no square root, sine or division.  Otherwise sinf(a) / a.
__device__ __forceinline__ float kappa_over_n(float kk, const StepParams& P) {
  if (P.kappa_series) {
    const float s = P.half_cdt * P.half_cdt * kk;
    float r = -1.0f / 121645100408832000.0f;                 // -1/19!
    r = fmaf(r, s, 1.0f / 355687428096000.0f);               //  1/17!
    r = fmaf(r, s, -1.0f / 1307674368000.0f);                // -1/15!
    r = fmaf(r, s, 1.0f / 6227020800.0f);                    //  1/13!
    r = fmaf(r, s, -1.0f / 39916800.0f);                     // -1/11!
    r = fmaf(r, s, 1.0f / 362880.0f);                        //  1/9!
    r = fmaf(r, s, -1.0f / 5040.0f);                         // -1/7!
    r = fmaf(r, s, 1.0f / 120.0f);                           //  1/5!
    r = fmaf(r, s, -1.0f / 6.0f);                            // -1/3!
    r = fmaf(r, s, 1.0f);
    return r * P.inv_n;
  }
  const float a = P.half_cdt * sqrtf(kk);
  return (a > 0.f ? sinf(a) / a : 1.f) * P.inv_n;
}

template <int NZ, int TZ>
struct Z2 {
  static constexpr int N1 = split_n1(NZ), N2 = NZ / N1;
  static constexpr int NT = TZ * N2;                 // forward step A: one task per thread
  static_assert(N1 <= N2, "step B runs one task per thread on the first TZ * N1 threads");
  static constexpr int TW = NZ + NZ;                 // W_NZ^e and the transposed table
  static constexpr size_t smem(int mode) { return (size_t)(TW + (mode == 0 ? 3 : 2) * NZ * TZ) * 8; }
};

template <int MODE, int NZ, int TZ>
__global__ void __launch_bounds__(Z2<NZ, TZ>::NT) k_zpass2(const __grid_constant__ StepParams P) {
  using C = Z2<NZ, TZ>;
  constexpr int N1 = C::N1, N2 = C::N2;
  if (*P.bad) return;
  extern __shared__ float2 zs2[];
  float2* tw = zs2;                     // tw[e] = W^e, e < NZ
  float2* twT = zs2 + NZ;               // twT[k1' N1 + k1] = W^(k1 k1'), k1' < N2, k1 < N1
  float2* b0 = zs2 + C::TW;
  float2* b1 = b0 + NZ * TZ;
  float2* b2 = b1 + NZ * TZ;
  for (int i = threadIdx.x; i < C::TW; i += C::NT) {
    int e = i;
    if (i >= NZ) {
      const int t = i - NZ, k1p = t / N1, k1 = t - k1p * N1;
      e = k1 * k1p;
    }
    tw[i] = P.tw[P.az.tw_off + e];
  }
  const SimPtrs& Q = P.sims[blockIdx.y];
  const int M = P.mspec;
  const int m0 = blockIdx.x * TZ;
  const float rhx = 1.0f / (float)P.hx;
  const int nslot = MODE == 0 ? 1 : 3;
  auto src_of = [&](int s) {
    return MODE == 0 ? Q.spec[0] : (s == 0 ? Q.spec[2] : (s == 1 ? Q.spec[0] : Q.spec[1]));
  };
  // forward step A inputs of this thread (column m0 + ml, rows j2 + N2 j1); the next
  // slot's are loaded before the current slot's step B (software pipelining)
  const int mlA = threadIdx.x % TZ, j2A = threadIdx.x / TZ;
  float2 a[N1];
  auto load_a = [&](int s) {
    const float2* src = src_of(s);
    const int m = m0 + mlA;
    sfor<0, N1>([&](auto J1) {
      constexpr int j1 = decltype(J1)::value;
      a[j1] = m < M ? __ldg(&src[(size_t)(j2A + N2 * j1) * M + m]) : make_float2(0.f, 0.f);
    });
  };
  load_a(0);
  // kappa / N of this thread's step-B column and kz = k1 + N1 k2, shared by all slots
  const bool hasB = threadIdx.x < TZ * N1;
  const int mlB = threadIdx.x % TZ, k1B = threadIdx.x / TZ;
  float kap[N2];
  {
    const int m = m0 + mlB;
    const int mm = m < M ? m : M - 1;
    const int ky = fdivi(mm, rhx);
    const int kx = mm - ky * P.hx;
    const float kxy = __ldg(&P.kx2[kx]) + __ldg(&P.ky2[ky]);
    sfor<0, N2>([&](auto K2) {
      constexpr int k2 = decltype(K2)::value;
      kap[k2] = hasB ? kappa_over_n(kxy + __ldg(&P.kz2[k1B + N1 * k2]), P) : 0.f;
    });
  }
#pragma unroll 1
  for (int s = 0; s < nslot; ++s) {
    __syncthreads();   // twiddles staged; previous slot's buffers consumed
    // forward step A: DFT_N1 of x[j2 + N2 j1], twiddle -> b0
    {
      const int ml = mlA, j2 = j2A;
      RDft<N1, false>::run(a);
      float2 w[N1];
      tw_row<N1>(tw, j2, w);
      sfor<0, N1>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        b0[(j2 + N2 * k1) * TZ + ml] = k1 == 0 ? a[k1] : cmul(a[k1], w[k1]);
      });
    }
    __syncthreads();
    if (MODE == 1 && s + 1 < nslot) load_a(s + 1);
    // forward step B, kappa, inverse step A (per output) -> b1 (, b2)
    if (hasB) {
      const int ml = mlB, k1 = k1B;
      float2 x[N2];
      sfor<0, N2>([&](auto J2) { x[decltype(J2)::value] = b0[(N2 * k1 + decltype(J2)::value) * TZ + ml]; });
      RDft<N2, false>::run(x);
      float2 r[N2];
      sfor<0, N2>([&](auto K2) {
        constexpr int k2 = decltype(K2)::value;
        const int kz = k1 + N1 * k2;
        const float2 v = cscale(x[k2], kap[k2]);
        if constexpr (MODE == 0) {
          x[k2] = v;
          r[k2] = cmul(v, __ldg(&P.ap[2][kz]));
        } else {
          x[k2] = (s == 2) ? cmul(v, __ldg(&P.am[2][kz])) : v;
        }
      });
      // inverse: the held values are the stride-N1 subsequence kz = k1 + N1 k2
      float2 w[N2];
      tw_row<N2>(twT + k1, N1, w);
      RDft<N2, true>::run(x);
      sfor<0, N2>([&](auto K1P) {
        constexpr int k1p = decltype(K1P)::value;
        b1[(k1p * N1 + k1) * TZ + ml] = k1p == 0 ? x[k1p] : cmulc(x[k1p], w[k1p]);
      });
      if constexpr (MODE == 0) {
        RDft<N2, true>::run(r);
        sfor<0, N2>([&](auto K1P) {
          constexpr int k1p = decltype(K1P)::value;
          b2[(k1p * N1 + k1) * TZ + ml] = k1p == 0 ? r[k1p] : cmulc(r[k1p], w[k1p]);
        });
      }
    }
    __syncthreads();
    // inverse step B: DFT_N1 over k1 for each k1', output z = k1' + N2 k2' -> global
    for (int t = threadIdx.x; t < TZ * N2; t += C::NT) {
      const int ml = t % TZ, k1p = t / TZ;
      const int m = m0 + ml;
      for (int o = 0; o < (MODE == 0 ? 2 : 1); ++o) {
        const float2* bb = o == 0 ? b1 : b2;
        float2* dst = MODE == 0 ? (o == 0 ? Q.spec[0] : Q.spec[1])
                                : (s == 0 ? Q.spec[2] : (s == 1 ? Q.spec[0] : Q.spec[1]));
        float2 u[N1];
        sfor<0, N1>([&](auto K1) { u[decltype(K1)::value] = bb[(k1p * N1 + decltype(K1)::value) * TZ + ml]; });
        RDft<N1, true>::run(u);
        if (m < M) {
          sfor<0, N1>([&](auto K2P) {
            constexpr int k2p = decltype(K2P)::value;
            dst[(size_t)(k1p + N2 * k2p) * M + m] = u[k2p];
          });
        }
      }
    }
  }
}

}  // namespace fwi
