// Register-resident DFTs of compile-time length, the building block of the
// two-step line transforms used by the fused plane kernels.
//
// RDft<M, INV>::run(v) transforms M complex values held in registers (natural
// order in and out, sign -1 forward / +1 inverse, unscaled).  Lengths 2, 3, 4,
// 5 and 8 use the butterflies of fft_smem.cuh; a composite M = r * m is split
// Cooley-Tukey style: DFT_m over the stride-r subsequences x[j2 + r j1], the
// twiddles exp(-+2 pi i j2 k1 / M), then DFT_r over j2, giving X[k1 + m k2].
// Every index is a compile-time constant, so the arrays stay in registers and
// the twiddles are immediate operands; they are computed at compile time in
// double precision from the Taylor series of sin and cos after reduction of the
// angle to [0, pi/4] by the octant symmetries, and rounded once to FP32.
#pragma once
#include "fft_smem.cuh"

namespace fwi {

template <int I>
struct IC {
  static constexpr int value = I;
};

// compile-time loop: f(IC<B>()), f(IC<B+1>()), ..., f(IC<E-1>())
template <int B, int E, class F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(IC<B>());
    sfor<B + 1, E>(f);
  }
}

struct CF {
  float x, y;
};

__host__ __device__ constexpr double ct_sin_series(double a) {
  double term = a, sum = a;
  for (int n = 1; n < 14; ++n) {
    term *= -a * a / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double ct_cos_series(double a) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 14; ++n) {
    term *= -a * a / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}

// exp(sign * 2 pi i e / m) for 0 <= e < m
__host__ __device__ constexpr CF ct_unit(int e, int m, int sign) {
  double t = (double)e / (double)m;
  bool neg_s = false, neg_c = false, swap = false;
  if (t > 0.5) { t = 1.0 - t; neg_s = true; }     // cos(2pi - a) = cos a, sin(2pi - a) = -sin a
  if (t > 0.25) { t = 0.5 - t; neg_c = true; }    // cos(pi - a) = -cos a, sin(pi - a) = sin a
  if (t > 0.125) { t = 0.25 - t; swap = true; }   // cos(pi/2 - a) = sin a
  const double a = 2.0 * 3.14159265358979323846264338327950288 * t;
  double c = ct_cos_series(a), s = ct_sin_series(a);
  if (swap) { const double u = c; c = s; s = u; }
  if (neg_c) c = -c;
  if (neg_s) s = -s;
  return CF{(float)c, (float)(sign * s)};
}

// v * exp(-+2 pi i E / M) with a compile-time exponent
template <int E, int M, bool INV>
__host__ __device__ __forceinline__ float2 twc(float2 v) {
  constexpr int e = E % M;
  if constexpr (e == 0) {
    return v;
  } else if constexpr (2 * e == M) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (4 * e == M) {
    return mul_mi<INV>(v);
  } else if constexpr (4 * e == 3 * M) {
    return mul_mi<!INV>(v);
  } else {
    constexpr CF w = ct_unit(e, M, INV ? 1 : -1);
    return make_float2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
  }
}

// a * conj(w)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 w) {
  return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}

template <int M>
struct RFac {
  static constexpr int r = (M % 4 == 0) ? 4 : (M % 3 == 0) ? 3 : (M % 5 == 0) ? 5 : 2;
};

template <int M, bool INV>
struct RDft {
  __host__ __device__ __forceinline__ static void run(float2* v) {
    if constexpr (M == 1) {
    } else if constexpr (M == 2 || M == 3 || M == 4 || M == 5 || M == 8) {
      Dft<M, INV>::run(v);
    } else {
      constexpr int r = RFac<M>::r, m = M / r;
      float2 t[M];
      sfor<0, r>([&](auto J2) {
        constexpr int j2 = decltype(J2)::value;
        float2 s[m];
        sfor<0, m>([&](auto J1) { s[decltype(J1)::value] = v[j2 + r * decltype(J1)::value]; });
        RDft<m, INV>::run(s);
        sfor<0, m>([&](auto K1) {
          constexpr int k1 = decltype(K1)::value;
          t[j2 * m + k1] = twc<j2 * k1, M, INV>(s[k1]);
        });
      });
      sfor<0, m>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        float2 u[r];
        sfor<0, r>([&](auto J2) { u[decltype(J2)::value] = t[decltype(J2)::value * m + k1]; });
        RDft<r, INV>::run(u);
        sfor<0, r>([&](auto K2) { v[k1 + m * decltype(K2)::value] = u[decltype(K2)::value]; });
      });
    }
  }
};

// Two-step split of a line length N = N1 * N2 (N1 <= N2, as balanced as possible):
// step A is DFT_N1 over the stride-N2 subsequences, step B DFT_N2.
__host__ __device__ constexpr int split_n1(int n) {
  int best = 1;
  for (int d = 1; d * d <= n; ++d)
    if (n % d == 0) best = d;
  return best;
}

}  // namespace fwi
