// Shared-memory mixed-radix (2, 3, 4, 5, 8) complex FFT on batches of lines.
//
// The k-space derivative of App. B (Eqs. 18-19) needs 3D discrete Fourier
// transforms of real fields on grids whose sides are products of 2, 3 and 5
// (the PML is sized so that they are, App. B).  These routines transform many
// lines held in one CTA's shared memory with a Stockham autosort sequence of
// radix-R passes: pass (R, Ns) reads butterfly j's inputs at j + r*N/R, applies
// the twiddles exp(-+2 pi i r (j mod Ns) / (Ns R)), does an R-point DFT in
// registers and writes output r to (j/Ns)*Ns*R + (j mod Ns) + r*Ns.  Every
// thread loads all its butterflies before a barrier and stores them after it,
// so each pass runs in place.  Twiddles come from a per-axis FP32 table
// W[k] = exp(-2 pi i k / N) built in FP64 on the host.
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

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// R-point DFT in registers, sign -1 (forward) or +1 (inverse), no scaling.
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct Dft<4, INV> {
  __device__ __forceinline__ static void run(float2* v) {
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
  __device__ __forceinline__ static void run(float2* v) {
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
  __device__ __forceinline__ static void run(float2* v) {
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
  __device__ __forceinline__ static void run(float2* v) {
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

// One Stockham pass over `nlines` lines of length N; element e of line l lives
// at buf[l*ls + e*es].  Requires nlines * N <= EPT * blockDim.x.
template <int R, bool INV, int EPT>
__device__ __forceinline__ void fft_pass(float2* buf, int nlines, int ls, int es, int N, int Ns,
                                         const float2* __restrict__ tw) {
  constexpr int MB = (EPT + R - 1) / R;
  const int nb = N / R;
  const int total = nlines * nb;
  const int T = blockDim.x;
  const int twstep = N / (Ns * R);
  float2 v[MB][R];
  int obase[MB];
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int idx = threadIdx.x + b * T;
    obase[b] = -1;
    if (idx < total) {
      const int line = idx / nb;
      const int j = idx - line * nb;
      const int jm = j % Ns;
      const float2* L = buf + line * ls;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = L[(j + r * nb) * es];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = __ldg(&tw[r * jm * twstep]);
          if (INV) w.y = -w.y;
          v[b][r] = cmul(v[b][r], w);
        }
      }
      Dft<R, INV>::run(v[b]);
      obase[b] = line * ls + ((j / Ns) * Ns * R + jm) * es;
    }
  }
  __syncthreads();
  const int ostride = Ns * es;
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    if (obase[b] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[obase[b] + r * ostride] = v[b][r];
    }
  }
  __syncthreads();
}

// Full transform of `nlines` lines (unnormalised).  Lines are processed in
// balanced batches of at most EPT * blockDim.x elements so that each thread
// stages at most EPT values per pass (requires N <= EPT * blockDim.x).
// Callers synchronise before; the routine ends with a barrier.  The axis plan
// is taken by value: it is never read through a pointer into kernel parameters.
template <bool INV, int EPT>
__device__ __forceinline__ void fft_lines(float2* buf, int nlines, int ls, int es, const AxisPlan A,
                                       const float2* __restrict__ twall) {
  const float2* tw = twall + A.tw_off;
  const int N = A.n;
  const int cap = EPT * (int)blockDim.x;
  int lpb = cap / N;
  const int nbat = (nlines + lpb - 1) / lpb;
  lpb = (nlines + nbat - 1) / nbat;
  for (int l0 = 0; l0 < nlines; l0 += lpb) {
    const int nl = min(lpb, nlines - l0);
    float2* bb = buf + l0 * ls;
    int Ns = 1;
    for (int s = 0; s < A.nstages; ++s) {
      const int R = A.radix[s];
      switch (R) {
        case 2: fft_pass<2, INV, EPT>(bb, nl, ls, es, N, Ns, tw); break;
        case 3: fft_pass<3, INV, EPT>(bb, nl, ls, es, N, Ns, tw); break;
        case 4: fft_pass<4, INV, EPT>(bb, nl, ls, es, N, Ns, tw); break;
        case 5: fft_pass<5, INV, EPT>(bb, nl, ls, es, N, Ns, tw); break;
        default: fft_pass<8, INV, EPT>(bb, nl, ls, es, N, Ns, tw); break;
      }
      Ns *= R;
    }
  }
}

}  // namespace fwi
