// fft_core.cuh - shared-memory mixed-radix FFT building blocks for sm_103a.
//
// A CTA holds a batch of pencils in shared memory and transforms them with a
// Stockham auto-sort sequence of radix-R stages (R in {2,3,4,8,12,16}); each
// stage keeps its R points in registers (small DFT below), applies the
// inter-stage twiddles from a per-length table staged in shared memory, and
// writes the other buffer of a ping-pong pair, so the result comes out in
// natural order without a bit-reversal pass.  Shared-memory layout of a batch:
//   element e of pencil p lives at (p / PT) * CS + e * ES + (p % PT)
// (PT pencils per "component" side by side, odd ES so that threads walking
// consecutive pencils hit distinct banks).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df64.cuh"

namespace scfft {

// ---------------------------------------------------------------- complex
template <typename T> struct cplx_of;
template <> struct cplx_of<float> { typedef float2 type; };
template <> struct cplx_of<double> { typedef double2 type; };
template <> struct cplx_of<dfloat> { typedef dfloat2 type; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
// FP32 complex sums as packed two-lane instructions of sm_100 and later (one instruction for
// the real and imaginary parts; each lane rounds as the scalar add does, and b * -1 + a
// rounds exactly as a - b).  A product that feeds such a sum is rounded on its own instead
// of being fused into it, so results can differ from the scalar forms in the last bit.
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 scl(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 scl(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {  // a * conj(b)
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V conj_(V a) { return mk(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> __device__ __forceinline__ V mul_mi(V a) {
  return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

// cos(k pi / 24) for k = 0..12 (exact values of the 48th roots of unity).
__host__ __device__ constexpr double cos24_tab(int k) {
  return k == 0 ? 1.0 : k == 1 ? 0.9914448613738104111445575 : k == 2 ? 0.9659258262890682867497432
       : k == 3 ? 0.9238795325112867561281832 : k == 4 ? 0.8660254037844386467637232
       : k == 5 ? 0.7933533402912351645797770 : k == 6 ? 0.7071067811865475244008444
       : k == 7 ? 0.6087614290087206394160975 : k == 8 ? 0.5 : k == 9 ? 0.3826834323650897717284600
       : k == 10 ? 0.2588190451025207623488988 : k == 11 ? 0.1305261922200515915484062 : 0.0;
}
// cos(m pi / 24) for any integer m
__host__ __device__ constexpr double cos24(int m) {
  return (m % 48 + 48) % 48 <= 12 ? cos24_tab((m % 48 + 48) % 48)
       : (m % 48 + 48) % 48 <= 24 ? -cos24_tab(24 - (m % 48 + 48) % 48)
       : (m % 48 + 48) % 48 <= 36 ? -cos24_tab((m % 48 + 48) % 48 - 24)
       : cos24_tab(48 - (m % 48 + 48) % 48);
}
__host__ __device__ constexpr double sin24(int m) { return cos24(m - 12); }

// a * W_R^m with W_R = exp(-2 pi i / R) (forward) or its conjugate (inverse); R divides 48.
template <typename V, int R, bool INV> struct TwiddleConst {
  static __device__ __forceinline__ V apply(V a, int m) {
    // angle 2 pi m / R = (2 m * 24 / R) * pi / 24; m is a compile-time constant at every
    // call site, so the branches below fold and multiples of pi/2 cost no multiply
    // (IEEE forbids the compiler from dropping x*0 or x*1 on its own)
    const int q = ((2 * m * 24 / R) % 48 + 48) % 48;
    typedef decltype(a.x) T;
    if (q == 0) return a;
    if (q == 24) return mk(-a.x, -a.y);
    if (q == 12) return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);  // * (+i) / (-i)
    if (q == 36) return INV ? mk(a.y, -a.x) : mk(-a.y, a.x);
    const T c = (T)cos24(q), s = (T)sin24(q);
    if (q % 12 == 6) {  // odd multiples of pi/4: |c| = |s|
      const T h = (T)0.7071067811865475244008444;
      const T sc = c > 0 ? (T)1 : (T)-1, ss = s > 0 ? (T)1 : (T)-1;
      // forward: a * (c - i s); inverse: a * (c + i s)
      return INV ? mk(h * (sc * a.x - ss * a.y), h * (ss * a.x + sc * a.y))
                 : mk(h * (sc * a.x + ss * a.y), h * (sc * a.y - ss * a.x));
    }
    return INV ? mk(a.x * c - a.y * s, a.x * s + a.y * c) : mk(a.x * c + a.y * s, a.y * c - a.x * s);
  }
};
// double-float: the constants are the nearest double-floats of the FP64 values (folded at
// compile time); the sign flips of the odd multiples of pi/4 are negations, not products
template <int R, bool INV> struct TwiddleConst<dfloat2, R, INV> {
  static __device__ __forceinline__ dfloat2 apply(dfloat2 a, int m) {
    const int q = ((2 * m * 24 / R) % 48 + 48) % 48;
    if (q == 0) return a;
    if (q == 24) return mk(-a.x, -a.y);
    if (q == 12) return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);
    if (q == 36) return INV ? mk(a.y, -a.x) : mk(-a.y, a.x);
    if (q % 12 == 6) {
      const dfloat h(0.7071067811865475244008444);
      const dfloat ax = cos24(q) > 0 ? a.x : -a.x, ay = cos24(q) > 0 ? a.y : -a.y;  // sign(c) a
      const dfloat bx = sin24(q) > 0 ? a.x : -a.x, by = sin24(q) > 0 ? a.y : -a.y;  // sign(s) a
      return INV ? mk(h * (ax - by), h * (bx + ay)) : mk(h * (ax + by), h * (ay - bx));
    }
    const dfloat c(cos24(q)), s(sin24(q));
    return INV ? mk(a.x * c - a.y * s, a.x * s + a.y * c) : mk(a.x * c + a.y * s, a.y * c - a.x * s);
  }
};
template <typename V, int R, bool INV> __device__ __forceinline__ V twiddle_const(V a, int m) {
  return TwiddleConst<V, R, INV>::apply(a, m);
}

// ---------------------------------------------------------------- small DFTs
template <int R, bool INV, typename V> struct DFT;

template <bool INV, typename V> struct DFT<2, INV, V> {
  static __device__ __forceinline__ void run(V* v) {
    V a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <bool INV, typename V> struct DFT<3, INV, V> {
  static __device__ __forceinline__ void run(V* v) {
    typedef decltype(v[0].x) T;
    const T h = (T)0.5, r = (T)0.8660254037844386467637232;  // sqrt(3)/2
    V s = v[1] + v[2], d = v[1] - v[2];
    V m = v[0] - scl(s, h);
    V x0 = v[0] + s;
    // w = exp(-+ 2 pi i/3): X1 = m -+ i r d, X2 = m +- i r d
    V rd = mul_mi<INV>(scl(d, r));
    v[0] = x0;
    v[1] = m + rd;
    v[2] = m - rd;
  }
};

template <bool INV, typename V> struct DFT<4, INV, V> {
  static __device__ __forceinline__ void run(V* v) {
    V a0 = v[0] + v[2], a1 = v[0] - v[2];
    V b0 = v[1] + v[3], b1 = mul_mi<INV>(v[1] - v[3]);
    v[0] = a0 + b0;
    v[2] = a0 - b0;
    v[1] = a1 + b1;
    v[3] = a1 - b1;
  }
};

// FP32: the sums as packed instructions; the products by -+i stay scalar (a packed form would
// need the real and imaginary parts swapped first)
template <bool INV> struct DFT<4, INV, float2> {
  static __device__ __forceinline__ void run(float2* v) {
    const float2 a0 = v[0] + v[2], a1 = v[0] - v[2];
    const float2 b0 = v[1] + v[3], b1 = v[1] - v[3];
    v[0] = a0 + b0;
    v[2] = a0 - b0;
    // a1 + (-+i) b1 and a1 - (-+i) b1
    v[1] = INV ? make_float2(a1.x - b1.y, a1.y + b1.x) : make_float2(a1.x + b1.y, a1.y - b1.x);
    v[3] = INV ? make_float2(a1.x + b1.y, a1.y - b1.x) : make_float2(a1.x - b1.y, a1.y + b1.x);
  }
};

// R = P * Q by one Cooley-Tukey split in registers:
// n = P n2 + n1, k = k1 + Q k2:  X[k1 + Q k2] = sum_n1 W_P^{n1 k2} W_R^{n1 k1} (sum_n2 x[P n2 + n1] W_Q^{n2 k1})
template <int P, int Q, bool INV, typename V>
__device__ __forceinline__ void dft_split(V* v) {
  constexpr int R = P * Q;
  V y[R];
#pragma unroll
  for (int n1 = 0; n1 < P; ++n1) {
    V t[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) t[n2] = v[P * n2 + n1];
    DFT<Q, INV, V>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) y[n1 * Q + k1] = (n1 * k1 == 0) ? t[k1] : twiddle_const<V, R, INV>(t[k1], n1 * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) {
    V t[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) t[n1] = y[n1 * Q + k1];
    DFT<P, INV, V>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) v[k1 + Q * k2] = t[k2];
  }
}

template <bool INV, typename V> struct DFT<8, INV, V> {
  static __device__ __forceinline__ void run(V* v) { dft_split<2, 4, INV, V>(v); }
};
template <bool INV, typename V> struct DFT<12, INV, V> {
  static __device__ __forceinline__ void run(V* v) { dft_split<3, 4, INV, V>(v); }
};
template <bool INV, typename V> struct DFT<16, INV, V> {
  static __device__ __forceinline__ void run(V* v) { dft_split<4, 4, INV, V>(v); }
};

// ---------------------------------------------------------------- half-zero inputs
// DFTh<R>: the same transform when v[R/2 .. R-1] are zero (zero-padded data), without the
// additions of those zeros.  R = P * 4 splits as in dft_split, and with n = P n2 + n1 the
// zero inputs are exactly n2 >= 2 of every first-stage 4-point transform.
template <int R, bool INV, typename V> struct DFTh;

template <bool INV, typename V> struct DFTh<2, INV, V> {
  static __device__ __forceinline__ void run(V* v) { v[1] = v[0]; }
};

template <bool INV, typename V> struct DFTh<4, INV, V> {
  static __device__ __forceinline__ void run(V* v) {
    const V a = v[0], b = v[1], ib = mul_mi<INV>(v[1]);
    v[0] = a + b;
    v[2] = a - b;
    v[1] = a + ib;
    v[3] = a - ib;
  }
};

template <bool INV> struct DFTh<4, INV, float2> {
  static __device__ __forceinline__ void run(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = a + b;
    v[2] = a - b;
    v[1] = INV ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, a.y - b.x);
    v[3] = INV ? make_float2(a.x + b.y, a.y - b.x) : make_float2(a.x - b.y, a.y + b.x);
  }
};

template <int P, bool INV, typename V>
__device__ __forceinline__ void dft_split_h(V* v) {
  constexpr int Q = 4, R = P * Q;
  V y[R];
#pragma unroll
  for (int n1 = 0; n1 < P; ++n1) {
    V t[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q / 2; ++n2) t[n2] = v[P * n2 + n1];
    DFTh<Q, INV, V>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) y[n1 * Q + k1] = (n1 * k1 == 0) ? t[k1] : twiddle_const<V, R, INV>(t[k1], n1 * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) {
    V t[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) t[n1] = y[n1 * Q + k1];
    DFT<P, INV, V>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) v[k1 + Q * k2] = t[k2];
  }
}

template <bool INV, typename V> struct DFTh<8, INV, V> {
  static __device__ __forceinline__ void run(V* v) { dft_split_h<2, INV, V>(v); }
};
template <bool INV, typename V> struct DFTh<12, INV, V> {
  static __device__ __forceinline__ void run(V* v) { dft_split_h<3, INV, V>(v); }
};
template <bool INV, typename V> struct DFTh<16, INV, V> {
  static __device__ __forceinline__ void run(V* v) { dft_split_h<4, INV, V>(v); }
};

// DFT of v, whose upper half is known to be zero when HALF is set
template <int R, bool INV, bool HALF, typename V> __device__ __forceinline__ void dft_maybe_half(V* v) {
  if constexpr (HALF) DFTh<R, INV, V>::run(v);
  else DFT<R, INV, V>::run(v);
}

// ---------------------------------------------------------------- plans
struct FftPlan {
  int L;       // transform length
  int ns;      // number of stages
  int r[4];    // radix of each stage (product = L)
};

// Batch geometry in shared memory (see the header comment).
struct Batch {
  int P;   // pencils
  int PT;  // pencils per component block
  int ES;  // element stride (in complex elements)
  int CS;  // component block stride
};

__device__ __forceinline__ int pbase(const Batch& b, int p) { return (p / b.PT) * b.CS + (p % b.PT); }

// One Stockham stage: for j in [0, L/R), k = j mod Ns,
//   v_q = src[j + q L/R] * W_{Ns R}^{q k};  v = DFT_R(v);  dst[(j/Ns) Ns R + k + q Ns] = v_q
template <int R, bool INV, typename V>
__device__ __forceinline__ void stockham_stage(const V* __restrict__ src, V* __restrict__ dst, const V* __restrict__ tw,
                                               int L, int Ns, const Batch& b) {
  const int LR = L / R;
  const int tasks = b.P * LR;
  const int twstep = L / (Ns * R);  // W_{Ns R}^{qk} = W_L^{q k twstep}
  for (int t = threadIdx.x; t < tasks; t += blockDim.x) {
    const int p = t % b.P;
    const int j = t / b.P;
    const int k = j % Ns;
    const int base = pbase(b, p);
    V v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = src[base + (j + q * LR) * b.ES];
    if (Ns > 1) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const V w = tw[q * k * twstep];
        v[q] = INV ? cmulc(v[q], w) : cmul(v[q], w);
      }
    }
    DFT<R, INV, V>::run(v);
    const int d0 = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[base + (d0 + q * Ns) * b.ES] = v[q];
  }
}

// Full transform of every pencil of the batch.  Data starts in buf[0]; returns
// the index (0/1) of the buffer holding the result.  Ends with __syncthreads().
template <bool INV, typename V>
__device__ int fft_batch(V* buf0, V* buf1, const V* tw, const FftPlan& pl, const Batch& b) {
  V* src = buf0;
  V* dst = buf1;
  int Ns = 1;
  int which = 0;
  for (int s = 0; s < pl.ns; ++s) {
    const int R = pl.r[s];
    switch (R) {
      case 2: stockham_stage<2, INV>(src, dst, tw, pl.L, Ns, b); break;
      case 3: stockham_stage<3, INV>(src, dst, tw, pl.L, Ns, b); break;
      case 4: stockham_stage<4, INV>(src, dst, tw, pl.L, Ns, b); break;
      case 8: stockham_stage<8, INV>(src, dst, tw, pl.L, Ns, b); break;
      case 12: stockham_stage<12, INV>(src, dst, tw, pl.L, Ns, b); break;
      default: stockham_stage<16, INV>(src, dst, tw, pl.L, Ns, b); break;
    }
    __syncthreads();
    V* t = src;
    src = dst;
    dst = t;
    which ^= 1;
    Ns *= R;
  }
  return which;
}

}  // namespace scfft
