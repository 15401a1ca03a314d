// Shared-memory mixed-radix (2, 3, 4, 5, 8) complex FFT on groups of lines.
//
// The k-space derivative of App. B (Eqs. 18-19) needs 3D discrete Fourier
// transforms of real fields on grids whose sides are products of 2, 3 and 5
// (the PML is sized so that they are, App. B).  A warp transforms a group of
// lines held in shared memory with a Stockham autosort sequence of radix-R
// passes: pass (R, Ns) reads butterfly j's inputs at j + r*N/R, applies the
// twiddles exp(-+2 pi i r (j mod Ns) / (Ns R)), does an R-point DFT in
// registers and writes output r to (j/Ns)*Ns*R + (j mod Ns) + r*Ns.  Lines are
// owned by one warp for the whole transform, so passes synchronise with
// __syncwarp only.  Twiddles come from a per-axis FP32 table
// W[k] = exp(-2 pi i k / N) built in FP64 on the host and staged in shared memory.
#pragma once
#include <cuda_runtime.h>

namespace fwi {

constexpr int kMaxStages = 12;

struct AxisPlan {
  int n;                    // transform length
  int nstages;              // number of radix passes
  int radix[kMaxStages];    // radix of each pass (2, 3, 4, 5 or 8)
  int tw_off;               // offset of this axis' W table in the twiddle array
};

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__host__ __device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// R-point DFT in registers, sign -1 (forward) or +1 (inverse), no scaling.
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  __host__ __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct Dft<4, INV> {
  __host__ __device__ __forceinline__ static void run(float2* v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV>
struct Dft<3, INV> {
  __host__ __device__ __forceinline__ static void run(float2* v) {
    const float s1 = 0.86602540378443864676f;  // sin(2 pi / 3)
    float2 t = cadd(v[1], v[2]);
    float2 u = csub(v[1], v[2]);
    float2 b = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    float2 su = mul_mi<INV>(cscale(u, s1));  // -+ i s1 u
    v[0] = cadd(v[0], t);
    v[1] = cadd(b, su);
    v[2] = csub(b, su);
  }
};

template <bool INV>
struct Dft<5, INV> {
  __host__ __device__ __forceinline__ static void run(float2* v) {
    const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
    const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
    const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
    const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
    float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    float2 a0 = v[0];
    float2 b1 = make_float2(a0.x + c1 * t1.x + c2 * t2.x, a0.y + c1 * t1.y + c2 * t2.y);
    float2 b2 = make_float2(a0.x + c2 * t1.x + c1 * t2.x, a0.y + c2 * t1.y + c1 * t2.y);
    float2 e1 = mul_mi<INV>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
    float2 e2 = mul_mi<INV>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
    v[0] = cadd(a0, cadd(t1, t2));
    v[1] = cadd(b1, e1);
    v[4] = csub(b1, e1);
    v[2] = cadd(b2, e2);
    v[3] = csub(b2, e2);
  }
};

template <bool INV>
struct Dft<8, INV> {
  // split into even/odd outputs: u_r = a_r + a_(r+4), w_r = (a_r - a_(r+4)) W8^r,
  // y_(2k) = DFT4(u)_k, y_(2k+1) = DFT4(w)_k
  __host__ __device__ __forceinline__ static void run(float2* v) {
    const float h = 0.70710678118654752440f;
    float2 u[4], w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      u[r] = cadd(v[r], v[r + 4]);
      w[r] = csub(v[r], v[r + 4]);
    }
    // W8 = exp(-+ i pi/4)
    w[1] = INV ? make_float2(h * (w[1].x - w[1].y), h * (w[1].x + w[1].y))
               : make_float2(h * (w[1].x + w[1].y), h * (w[1].y - w[1].x));
    w[2] = mul_mi<INV>(w[2]);
    w[3] = INV ? make_float2(-h * (w[3].x + w[3].y), h * (w[3].x - w[3].y))
               : make_float2(h * (w[3].y - w[3].x), -h * (w[3].x + w[3].y));
    Dft<4, INV>::run(u);
    Dft<4, INV>::run(w);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = u[k];
      v[2 * k + 1] = w[k];
    }
  }
};

// a / d for 0 <= a < 2^22 and d >= 1, given r = 1.0f / d: (a + 1/2) / d is at least
// 1/(2d) away from an integer and the FP32 product errs by less than that.
__device__ __forceinline__ int fdivi(int a, float r) { return __float2int_rz(((float)a + 0.5f) * r); }

// One Stockham radix-R pass, run by a single warp over `nbf` butterflies that
// belong to nbf / nb lines (nb = N / R butterflies per line).  Element e of line
// l lives at buf[l*ls + e*es]; `tw` is the axis' W table in shared memory.  The
// warp loads all its butterflies before __syncwarp and stores after it, so the
// pass runs in place.  Each lane stages at most about EPL values: requires
// nbf <= 32 * ceil(EPL / R).  Kept out of line so that the register budgets of
// the different radices are not summed where a kernel dispatches on R.
template <int R, bool INV, int EPL>
__device__ __noinline__ void warp_pass(float2* buf, int nbf, int nb, int ls, int es, int Ns,
                                          int twstep, const float2* tw, int lane) {
  constexpr int MB = (EPL + R - 1) / R;
  const float rnb = 1.0f / (float)nb;
  const float rns = 1.0f / (float)Ns;
  float2 v[MB][R];
  int ob[MB];
#pragma unroll
  for (int i = 0; i < MB; ++i) {
    const int b = lane + 32 * i;
    ob[i] = -1;
    if (b < nbf) {
      const int line = fdivi(b, rnb);
      const int j = b - line * nb;
      const int jq = fdivi(j, rns);
      const int jm = j - jq * Ns;
      const float2* L = buf + line * ls;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = L[(j + r * nb) * es];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[r * jm * twstep];
          if (INV) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      Dft<R, INV>::run(v[i]);
      ob[i] = line * ls + (jq * Ns * R + jm) * es;
    }
  }
  __syncwarp();
  const int os = Ns * es;
#pragma unroll
  for (int i = 0; i < MB; ++i) {
    if (ob[i] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[ob[i] + r * os] = v[i][r];
    }
  }
  __syncwarp();
}

// Transform `nl` lines of length A.n by one warp (unnormalised).  Requires
// nl * A.n <= 32 * EPL.
template <bool INV, int EPL>
__device__ __forceinline__ void warp_fft(float2* buf, int nl, int ls, int es, const AxisPlan& A,
                                         const float2* tw, int lane) {
  const int N = A.n;
  int Ns = 1;
#pragma unroll 1
  for (int s = 0; s < A.nstages; ++s) {
    const int R = A.radix[s];
    const int nb = N / R;
    const int tws = N / (Ns * R);
    switch (R) {
      case 2: warp_pass<2, INV, EPL>(buf, nl * nb, nb, ls, es, Ns, tws, tw, lane); break;
      case 3: warp_pass<3, INV, EPL>(buf, nl * nb, nb, ls, es, Ns, tws, tw, lane); break;
      case 4: warp_pass<4, INV, EPL>(buf, nl * nb, nb, ls, es, Ns, tws, tw, lane); break;
      case 5: warp_pass<5, INV, EPL>(buf, nl * nb, nb, ls, es, Ns, tws, tw, lane); break;
      default: warp_pass<8, INV, EPL>(buf, nl * nb, nb, ls, es, Ns, tws, tw, lane); break;
    }
    Ns *= R;
  }
}

// Lines per warp group for an axis of length n (nl * n <= 32 * EPL).
template <int EPL>
__host__ __device__ __forceinline__ int lines_per_group(int n) { return n >= 32 * EPL ? 1 : 32 * EPL / n; }


// ---------------------------------------------------------------------------
// Compile-time specialised line transforms for the common lengths: the radix
// schedule, divisors, group sizes and loop bounds are constants, everything is
// inlined.  LF = true maps consecutive lanes to consecutive lines (used when the
// lines are adjacent columns, so lanes touch adjacent words).

template <int M>
struct FirstRadix {
  static constexpr int value = (M % 8 == 0) ? 8 : (M % 4 == 0) ? 4 : (M % 2 == 0) ? 2 : (M % 3 == 0) ? 3 : 5;
};

template <int N, int R, int NS, bool INV, int G, bool LF>
__device__ __forceinline__ void ct_pass(float2* buf, int ls, int es, const float2* tw, int lane) {
  constexpr int NB = N / R;
  constexpr int TOT = G * NB;
  constexpr int MB = (TOT + 31) / 32;
  constexpr int TWS = N / (NS * R);
  float2 v[MB][R];
  int ob[MB];
#pragma unroll
  for (int i = 0; i < MB; ++i) {
    const int b = lane + 32 * i;
    ob[i] = -1;
    if (TOT % 32 == 0 || b < TOT) {
      const int line = LF ? b % G : b / NB;
      const int j = LF ? b / G : b % NB;
      const int jm = j % NS;
      const int jq = j / NS;
      const float2* L = buf + line * ls;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = L[(j + r * NB) * es];
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[r * jm * TWS];
          if (INV) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      Dft<R, INV>::run(v[i]);
      ob[i] = line * ls + (jq * NS * R + jm) * es;
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < MB; ++i) {
    if (ob[i] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[ob[i] + r * NS * es] = v[i][r];
    }
  }
  __syncwarp();
}

template <int N, int M, int NS, bool INV, int G, bool LF>
__device__ __forceinline__ void ct_fft_rec(float2* buf, int ls, int es, const float2* tw, int lane) {
  if constexpr (M > 1) {
    constexpr int R = FirstRadix<M>::value;
    static_assert(M % R == 0, "length must be a product of 2, 3 and 5");
    ct_pass<N, R, NS, INV, G, LF>(buf, ls, es, tw, lane);
    ct_fft_rec<N, M / R, NS * R, INV, G, LF>(buf, ls, es, tw, lane);
  }
}

// G lines of length N by one warp (all G lines present).
template <int N, bool INV, int G, bool LF>
__device__ __forceinline__ void ct_fft(float2* buf, int ls, int es, const float2* tw, int lane) {
  ct_fft_rec<N, N, 1, INV, G, LF>(buf, ls, es, tw, lane);
}

// nl <= G lines: a full group in one go, a partial group line by line (same
// arithmetic, still specialised).
template <int N, bool INV, int G, bool LF>
__device__ __forceinline__ void ct_fft_n(float2* buf, int nl, int ls, int es, const AxisPlan& A,
                                         const float2* tw, int lane) {
  (void)A;
  if (nl == G) {
    ct_fft<N, INV, G, LF>(buf, ls, es, tw, lane);
  } else {
    for (int l = 0; l < nl; ++l) ct_fft<N, INV, 1, LF>(buf + l * ls, ls, es, tw, lane);
  }
}

}  // namespace fwi
