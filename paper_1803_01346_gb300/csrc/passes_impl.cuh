// passes_impl.cuh - the shared-memory FFT pass kernels and their launchers, as templates over
// the element type (float, double, dfloat); passes.cu instantiates them for float and double,
// passes_df64.cu for dfloat (two translation units, compiled in parallel).
//
// Every 3D transform is split into three batched 1D passes along x, y and z on
// the layouts [comp][z][y][x] (real) and [comp][z][y][kx] (half spectrum,
// row stride sx).  Pointwise work is fused into the passes:
//   x passes  : C2R of a half-spectrum row, the node-wise step (power law of
//               Eq. 1 / Omega_out Ohm law, dh^0 assembly, mask + zero pad, the
//               Eq. 5 update and its residual), then R2C of the result.
//   z passes  : forward z FFT, the spectral curl multiply i S(k) k x F, or the
//               kernel-spectrum cross product K^ x F of Eq. 7, inverse z FFT.
//   y passes  : plain y FFTs, pruned to the nonzero input / needed output rows
//               on the zero-padded grid.
// Two real rows of one component travel as the real and imaginary parts of one
// complex pencil in the x passes (two real transforms for one complex one).
#pragma once
#include <math.h>
#include <stdio.h>

#include "scfft_internal.cuh"

namespace scfft {

template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ dfloat2 vzero<dfloat2>() { return mk(dfloat(0.f, 0.f), dfloat(0.f, 0.f)); }

// Euclidean norm of the change of one node's iterate (the Eq. 5 residual's summand): in FP64
// for the FP32 and FP64 passes, from the high parts of the double-float difference for the
// double-float passes (a stop test needs no more)
__device__ __forceinline__ double dnorm3(float v0, float o0, float v1, float o1, float v2, float o2) {
  const double d0 = (double)v0 - (double)o0, d1 = (double)v1 - (double)o1, d2 = (double)v2 - (double)o2;
  return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}
__device__ __forceinline__ double dnorm3(double v0, double o0, double v1, double o1, double v2, double o2) {
  const double d0 = v0 - o0, d1 = v1 - o1, d2 = v2 - o2;
  return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}
__device__ __forceinline__ double dnorm3(dfloat v0, dfloat o0, dfloat v1, dfloat o1, dfloat v2, dfloat o2) {
  const float d0 = (v0 - o0).hi, d1 = (v1 - o1).hi, d2 = (v2 - o2).hi;
  return (double)sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
}

// Power law of Eq. 1: returns rho(|j|) for |j| = jn.  FP32 evaluates
// |j/jc|^(n-1) as 2^((n-1) log2(|j|/jc)) so that large n cannot overflow an
// intermediate power; FP64 uses pow directly.
__device__ __forceinline__ float rho_power(float jn, float jcv, float n, float e0) {
  if (jn == 0.f) return (n == 1.f) ? e0 / jcv : 0.f;
  return (e0 / jcv) * exp2f((n - 1.f) * log2f(jn / jcv));
}
__device__ __forceinline__ double rho_power(double jn, double jcv, double n, double e0) {
  if (jn == 0.0) return (n == 1.0) ? e0 / jcv : 0.0;
  return (e0 / jcv) * pow(jn / jcv, n - 1.0);
}

// ---------------------------------------------------------------- x passes
template <typename T>
struct XArgs {
  typedef typename cplx_of<T>::type V;
  Geo g;
  int QP;            // row pairs per component per CTA
  int Lin, Lout;     // C2R length (0 = real input), R2C length (0 = real output)
  int Lmax;
  FftPlan pin, pout;
  const V* spec_in;
  int in_rows, in_sx;
  V* spec_out;
  int out_rows, out_sx;
  const V* tw_in;
  const V* tw_out;
  const double* src_f64;
  const T* src_t;     // real input rows in the pass's own type (instead of src_f64), or nullptr
  double* dst_f64;
  const double* warm;
  const uint8_t* mask;
  const T* jc;
  const T* hold;
  T* hnew;
  PointParams pp;
  Ctrl* ctrl;
  double* partials;
  int check_done;
  int out_buf;
  // mask/pad pass of an Eq. 5 iteration: only the rows of Omega's box (y in [by0, by1), z in
  // [bz0, bz1)); the source vanishes outside, and nothing downstream reads the rows left out
  int use_box, by0, by1, bz0, bz1;
};

// flat (z, y) row index of the pass's q-th row: every row of the grid, or the box's rows
template <typename T> __device__ __forceinline__ int flat_row(const XArgs<T>& a, int q) {
  if (!a.use_box) return q;
  const int nyb = a.by1 - a.by0, zb = q / nyb;
  return (a.bz0 + zb) * a.g.ny + a.by0 + (q - zb * nyb);
}

template <typename T>
__device__ __forceinline__ T* half_of(typename cplx_of<T>::type* p, int h) {
  return reinterpret_cast<T*>(p) + h;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) xpass_kernel(const XArgs<T> a) {
  typedef typename cplx_of<T>::type V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.check_done && a.ctrl->done) return;

  const int tid = threadIdx.x, nth = blockDim.x;
  const int QP = a.QP, ES = QP + 1, CS = a.Lmax * ES;
  const int R = 2 * QP;
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int nrows = a.use_box ? (a.bz1 - a.bz0) * (a.by1 - a.by0) : ny * nz;
  const long long N = a.g.N;
  const int q0 = blockIdx.x * R;
  V* bufA = reinterpret_cast<V*>(smem_raw);
  V* bufB = bufA + 3 * CS;
  V* twi = bufB + 3 * CS;
  V* two = twi + 256;
  const Batch b{3 * QP, QP, ES, CS};

  for (int i = tid; i < a.Lin; i += nth) twi[i] = a.tw_in[i];
  for (int i = tid; i < a.Lout; i += nth) two[i] = a.tw_out[i];

  constexpr bool kC2R = (MODE != X_FWD_F64 && MODE != X_PAD_F64 && MODE != X_ADJ_PAD && MODE != X_ADJ_IN);
  constexpr bool kR2C = (MODE != X_TO_F64 && MODE != X_CROP_F64 && MODE != X_ADJ_COMBINE);

  V* data;
  V* other;
  if (kC2R) {
    const int L = a.Lin, H = L / 2 + 1;
    // phase 1: half spectra of the 2QP rows of each component -> bufB[c][k][r]
    for (int idx = tid; idx < 3 * R * H; idx += nth) {
      const int k = idx % H, r = (idx / H) % R, c = idx / (H * R);
      const int q = q0 + r;
      V v = vzero<V>();
      if (q < nrows) {
        const int fq = flat_row(a, q), z = fq / ny, y = fq - z * ny;
        v = a.spec_in[((size_t)(c * nz + z) * a.in_rows + y) * a.in_sx + k];
      }
      if (k == 0 || k == L / 2) v.y = 0;  // C2R reads only the real part of DC and Nyquist
      bufB[(c * H + k) * R + r] = v;
    }
    __syncthreads();
    // phase 2: Z[k] = A[k] + i B[k], Z[L-k] = conj(A[k]) + i conj(B[k])
    for (int idx = tid; idx < 3 * QP * H; idx += nth) {
      const int k = idx % H, pr = (idx / H) % QP, c = idx / (H * QP);
      const V A = bufB[(c * H + k) * R + 2 * pr], B = bufB[(c * H + k) * R + 2 * pr + 1];
      const int base = c * CS + pr;
      bufA[base + k * ES] = mk(A.x - B.y, A.y + B.x);
      if (k > 0 && k < L / 2) bufA[base + (L - k) * ES] = mk(A.x + B.y, B.x - A.y);
    }
    __syncthreads();
    const int w = fft_batch<true>(bufA, bufB, twi, a.pin, b);
    data = w ? bufB : bufA;
    other = w ? bufA : bufB;
  } else {
    for (int idx = tid; idx < 3 * R * nx; idx += nth) {
      const int n = idx % nx, r = (idx / nx) % R, c = idx / (nx * R);
      const int q = q0 + r;
      T v = 0;
      if (q < nrows) {
        const size_t node = (size_t)flat_row(a, q) * nx + n;
        v = a.src_t ? a.src_t[(size_t)c * N + node] : (T)a.src_f64[(size_t)c * N + node];
        if (MODE == X_ADJ_PAD && a.mask[node]) v = 0;   // (1 - chi)
        if (MODE == X_ADJ_IN && !a.mask[node]) v = 0;   // chi
      }
      *half_of<T>(&bufA[c * CS + (r >> 1) + n * ES], r & 1) = v;
    }
    data = bufA;
    other = bufB;
  }

  // ---- node-wise step on the real rows held in `data`
  double part = 0.0;
  if (kC2R) {
    typedef typename acc_of<T>::type A;
    const PointParams& pp = a.pp;
    const T he0 = (T)pp.hedot[0], he1 = (T)pp.hedot[1], he2 = (T)pp.hedot[2];
    for (int idx = tid; idx < R * nx; idx += nth) {
      const int n = idx % nx, r = idx / nx;
      const int q = q0 + r;
      if (q >= nrows) continue;
      const size_t node = (size_t)flat_row(a, q) * nx + n;
      T* p0 = half_of<T>(&data[0 * CS + (r >> 1) + n * ES], r & 1);
      T* p1 = half_of<T>(&data[1 * CS + (r >> 1) + n * ES], r & 1);
      T* p2 = half_of<T>(&data[2 * CS + (r >> 1) + n * ES], r & 1);
      T v0 = *p0, v1 = *p1, v2 = *p2;
      if (MODE == X_POWERLAW) {
        A w0 = to_acc(v0), w1 = to_acc(v1), w2 = to_acc(v2);
        A rho;
        if (a.mask[node]) {
          A jcv = a.jc ? to_acc(a.jc[node]) : (A)pp.jc;
          if (pp.law) {
            // e(j, h): jc(h) = jc / (1 + |h| / h0) (Kim), e = rho(|A j|) A^2 j
            if (pp.kim_h0 > 0) {
              const A h0 = (A)a.src_f64[node], h1 = (A)a.src_f64[N + node], h2 = (A)a.src_f64[2 * N + node];
              jcv = jcv / ((A)1 + sqrt(h0 * h0 + h1 * h1 + h2 * h2) / (A)pp.kim_h0);
            }
            const A ax = (A)pp.aniso[0], ay = (A)pp.aniso[1], az = (A)pp.aniso[2];
            const A u0 = ax * w0, u1 = ay * w1, u2 = az * w2;
            rho = rho_power(sqrt(u0 * u0 + u1 * u1 + u2 * u2), jcv, (A)pp.n, (A)pp.e0);
            w0 *= rho * ax * ax; w1 *= rho * ay * ay; w2 *= rho * az * az;
          } else {
            const A jn = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
            rho = rho_power(jn, jcv, (A)pp.n, (A)pp.e0);
            w0 *= rho; w1 *= rho; w2 *= rho;
          }
        } else {
          rho = (A)pp.rho_out;
          w0 *= rho; w1 *= rho; w2 *= rho;
        }
        v0 = from_acc<T>(w0); v1 = from_acc<T>(w1); v2 = from_acc<T>(w2);
      } else if (MODE == X_ASSEMBLE) {
        if (a.mask[node]) {
          const T s = -(T)pp.inv_mu0;
          v0 *= s; v1 *= s; v2 *= s;
        } else {
          v0 = (T)a.warm[node]; v1 = (T)a.warm[N + node]; v2 = (T)a.warm[2 * N + node];
        }
        a.hnew[node] = v0; a.hnew[N + node] = v1; a.hnew[2 * N + node] = v2;
      } else if (MODE == X_MASKPAD) {
        if (!a.mask[node]) { v0 = 0; v1 = 0; v2 = 0; }
      } else if (MODE == X_UPDATE) {
        const T o0 = a.hold[node], o1 = a.hold[N + node], o2 = a.hold[2 * N + node];
        if (a.mask[node]) {
          v0 = o0; v1 = o1; v2 = o2;
        } else {
          v0 = he0 + v0; v1 = he1 + v1; v2 = he2 + v2;
          part += dnorm3(v0, o0, v1, o1, v2, o2);
        }
        a.hnew[node] = v0; a.hnew[N + node] = v1; a.hnew[2 * N + node] = v2;
      } else if (MODE == X_TO_F64 || MODE == X_CROP_F64) {
        a.dst_f64[node] = (double)v0; a.dst_f64[N + node] = (double)v1; a.dst_f64[2 * N + node] = (double)v2;
      } else if (MODE == X_ADJ_CROP) {
        if (!a.mask[node]) { v0 = 0; v1 = 0; v2 = 0; }
      } else if (MODE == X_ADJ_COMBINE) {
        const bool in = a.mask[node];
        a.dst_f64[node] = (double)v0 + (in ? a.src_f64[node] : 0.0);
        a.dst_f64[N + node] = (double)v1 + (in ? a.src_f64[N + node] : 0.0);
        a.dst_f64[2 * N + node] = (double)v2 + (in ? a.src_f64[2 * N + node] : 0.0);
      } else if (MODE == X_ADJ_POWERLAW) {
        // lam_e = -(curl lam_u)/mu0; lam_j = J_e^T lam_e; J_e = rho (I + (n-1) jhat jhat^T) in Omega
        const A s = -(A)pp.inv_mu0;
        const A l0 = s * to_acc(v0), l1 = s * to_acc(v1), l2 = s * to_acc(v2);
        A w0, w1, w2;
        if (a.mask[node]) {
          const A j0 = (A)a.src_f64[node], j1 = (A)a.src_f64[N + node], j2 = (A)a.src_f64[2 * N + node];
          const A jcv = a.jc ? to_acc(a.jc[node]) : (A)pp.jc;
          const A jn = sqrt(j0 * j0 + j1 * j1 + j2 * j2);
          const A rho = rho_power(jn, jcv, (A)pp.n, (A)pp.e0);
          const A jl = j0 * l0 + j1 * l1 + j2 * l2;
          const A f = jn > 0 ? ((A)pp.n - 1) * jl / (jn * jn) : (A)0;
          w0 = rho * (l0 + f * j0); w1 = rho * (l1 + f * j1); w2 = rho * (l2 + f * j2);
          if (a.dst_f64) a.dst_f64[node] = (double)(-(A)pp.n * rho / jcv * jl);
        } else {
          const A r = (A)pp.rho_out;
          w0 = r * l0; w1 = r * l1; w2 = r * l2;
          if (a.dst_f64) a.dst_f64[node] = 0.0;
        }
        v0 = from_acc<T>(w0); v1 = from_acc<T>(w1); v2 = from_acc<T>(w2);
      }
      if (kR2C) { *p0 = v0; *p1 = v1; *p2 = v2; }
    }
  }
  // zero padding of the R2C input beyond nx (padded transforms) or of rows past the grid
  if (kR2C) {
    const int L = a.Lout;
    for (int idx = tid; idx < 3 * QP * L; idx += nth) {
      const int n = idx % L, pr = (idx / L) % QP, c = idx / (L * QP);
      const int q = q0 + 2 * pr;
      if (n >= nx || q >= nrows) data[c * CS + pr + n * ES] = vzero<V>();
      else if (q + 1 >= nrows) half_of<T>(&data[c * CS + pr + n * ES], 1)[0] = 0;
    }
  }
  __syncthreads();

  if (kR2C) {
    const int w = fft_batch<false>(data, other, two, a.pout, b);
    const V* res = w ? other : data;
    const int L = a.Lout, H = L / 2 + 1;
    const T half = (T)0.5;
    for (int idx = tid; idx < 3 * R * H; idx += nth) {
      const int k = idx % H, r = (idx / H) % R, c = idx / (H * R);
      const int q = q0 + r;
      if (q >= nrows) continue;
      const int base = c * CS + (r >> 1);
      const V Zk = res[base + k * ES];
      const V Zm = res[base + ((L - k) % L) * ES];
      V o;
      if ((r & 1) == 0) o = mk((Zk.x + Zm.x) * half, (Zk.y - Zm.y) * half);
      else o = mk((Zk.y + Zm.y) * half, (Zm.x - Zk.x) * half);
      const int fq = flat_row(a, q), z = fq / ny, y = fq - z * ny;
      a.spec_out[((size_t)(c * nz + z) * a.out_rows + y) * a.out_sx + k] = o;
    }
  }

  if (MODE == X_UPDATE) {
    // deterministic two-level reduction of the Eq. 5 residual
    __shared__ double red[kThreads / 32];
    __shared__ int am_last;
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int i = 0; i < nth / 32; ++i) s += red[i];
      a.partials[blockIdx.x] = s;
      __threadfence();
      const unsigned prev = atomicAdd(&a.ctrl->counter, 1u);
      am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) {
      __threadfence();
      double s = 0.0;
      for (int i = tid; i < (int)gridDim.x; i += nth) s += __ldcg(&a.partials[i]);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      __syncthreads();
      if ((tid & 31) == 0) red[tid >> 5] = s;
      __syncthreads();
      if (tid == 0) {
        double tot = 0.0;
        for (int i = 0; i < nth / 32; ++i) tot += red[i];
        const double r = tot * a.pp.inv_nout;
        Ctrl* c = a.ctrl;
        c->residual = r;
        c->iters = a.pp.iter + 1;
        c->cur = a.out_buf;
        const bool finite = isfinite(r);
        if (!finite) c->status = 6;  // SCFFT_ENONFINITE
        c->done = (!finite || r < a.pp.tol) ? 1 : 0;
        c->counter = 0;
      }
    }
  }
  if (MODE == X_ASSEMBLE && blockIdx.x == 0 && tid == 0) {
    a.ctrl->done = 0;
    a.ctrl->iters = 0;
    a.ctrl->cur = 0;
    a.ctrl->counter = 0;
    a.ctrl->residual = 0.0;
  }
}

// ---------------------------------------------------------------- y passes
template <typename T>
struct YArgs {
  typedef typename cplx_of<T>::type V;
  V* base;
  int rows, sx, HX, nzs, TC;
  int Lin, Lout;
  FftPlan pl;
  const V* tw;
  const Ctrl* ctrl;
  int check_done;
  int zoff, ylo, yhi;  // planes z = zoff + blockIdx.y; input rows outside [ylo, yhi) read as zero
};

template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads) ypass_kernel(const YArgs<T> a) {
  typedef typename cplx_of<T>::type V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.check_done && a.ctrl->done) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int TC = a.TC, ES = TC + 1, L = a.pl.L;
  V* bufA = reinterpret_cast<V*>(smem_raw);
  V* bufB = bufA + L * ES;
  V* tw = bufB + L * ES;
  const int c = blockIdx.z, z = a.zoff + blockIdx.y, kx0 = blockIdx.x * TC;
  for (int i = tid; i < L; i += nth) tw[i] = a.tw[i];
  V* col = a.base + ((size_t)(c * a.nzs + z) * a.rows) * a.sx + kx0;
  for (int idx = tid; idx < L * TC; idx += nth) {
    const int ci = idx % TC, l = idx / TC;
    V v = vzero<V>();
    if (l < a.Lin && l >= a.ylo && l < a.yhi && kx0 + ci < a.HX) v = col[(size_t)l * a.sx + ci];
    bufA[l * ES + ci] = v;
  }
  __syncthreads();
  const Batch b{TC, TC, ES, 0};
  const int w = fft_batch<INV>(bufA, bufB, tw, a.pl, b);
  const V* res = w ? bufB : bufA;
  for (int idx = tid; idx < a.Lout * TC; idx += nth) {
    const int ci = idx % TC, l = idx / TC;
    if (kx0 + ci < a.HX) col[(size_t)l * a.sx + ci] = res[l * ES + ci];
  }
}

// ---------------------------------------------------------------- z passes
template <typename T>
struct ZArgs {
  typedef typename cplx_of<T>::type V;
  V* base;
  int rows, sx, HX, nzs, TC;
  FftPlan pl;
  const V* tw;
  // curl
  const T* kt0; const T* kt1; const T* kt2;
  const T* st0; const T* st1; const T* st2;
  T scale;
  // kernel
  const T* kap;
  int nx, ny, nz;
  const Ctrl* ctrl;
  int check_done;
  int zlo, zhi;  // the padded pass's input planes outside [zlo, zhi) read as zero
};

template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads) zpass_kernel(const ZArgs<T> a) {
  typedef typename cplx_of<T>::type V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.check_done && a.ctrl->done) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int TC = a.TC, ES = TC + 1, L = a.pl.L, CS = L * ES;
  V* bufA = reinterpret_cast<V*>(smem_raw);
  V* bufB = bufA + 3 * CS;
  V* tw = bufB + 3 * CS;
  const int y = blockIdx.y, kx0 = blockIdx.x * TC;
  for (int i = tid; i < L; i += nth) tw[i] = a.tw[i];
  const size_t cstride = (size_t)a.nzs * a.rows * a.sx;  // one component
  const size_t zstride = (size_t)a.rows * a.sx;
  V* col = a.base + (size_t)y * a.sx + kx0;
  for (int idx = tid; idx < 3 * L * TC; idx += nth) {
    const int ci = idx % TC, l = (idx / TC) % L, c = idx / (TC * L);
    V v = vzero<V>();
    if (l < a.nzs && l >= a.zlo && l < a.zhi && kx0 + ci < a.HX) v = col[c * cstride + l * zstride + ci];
    bufA[c * CS + l * ES + ci] = v;
  }
  __syncthreads();
  const Batch b{3 * TC, TC, ES, CS};
  int w = fft_batch<false>(bufA, bufB, tw, a.pl, b);
  V* res = w ? bufB : bufA;
  V* oth = w ? bufA : bufB;
  for (int idx = tid; idx < L * TC; idx += nth) {
    const int ci = idx % TC, l = idx / TC;
    const int kx = kx0 + ci;
    if (kx >= a.HX) continue;
    const int o = l * ES + ci;
    const V F0 = res[o], F1 = res[CS + o], F2 = res[2 * CS + o];
    T ax, ay, az, s;
    if (KIND == 0) {
      ax = a.kt0[kx]; ay = a.kt1[y]; az = a.kt2[l];
      s = a.st0[kx] * a.st1[y] * a.st2[l] * a.scale;
    } else {
      const int fy = (y <= a.ny) ? y : 2 * a.ny - y;
      const int fz = (l <= a.nz) ? l : 2 * a.nz - l;
      const T sy = (y <= a.ny) ? (T)1 : (T)-1;
      const T sz = (l <= a.nz) ? (T)1 : (T)-1;
      const size_t oct = (size_t)(a.nz + 1) * (a.ny + 1) * (a.nx + 1);
      const size_t off = ((size_t)fz * (a.ny + 1) + fy) * (a.nx + 1) + kx;
      ax = a.kap[off]; ay = sy * a.kap[oct + off]; az = sz * a.kap[2 * oct + off];
      s = (T)1;
    }
    // G = i s (a x F)
    const V cx = mk(ay * F2.x - az * F1.x, ay * F2.y - az * F1.y);
    const V cy = mk(az * F0.x - ax * F2.x, az * F0.y - ax * F2.y);
    const V cz = mk(ax * F1.x - ay * F0.x, ax * F1.y - ay * F0.y);
    res[o] = mk(-s * cx.y, s * cx.x);
    res[CS + o] = mk(-s * cy.y, s * cy.x);
    res[2 * CS + o] = mk(-s * cz.y, s * cz.x);
  }
  __syncthreads();
  w = fft_batch<true>(res, oth, tw, a.pl, b);
  const V* fin = w ? oth : res;
  for (int idx = tid; idx < 3 * a.nzs * TC; idx += nth) {
    const int ci = idx % TC, l = (idx / TC) % a.nzs, c = idx / (TC * a.nzs);
    if (kx0 + ci < a.HX) col[c * cstride + l * zstride + ci] = fin[c * CS + l * ES + ci];
  }
}

// ---------------------------------------------------------------- launchers
template <typename T> static int x_pairs(int Lmax) {
  // keep each ping-pong buffer around 24 KB so that several CTAs share an SM
  const int bytes_per_pair = 2 * 3 * Lmax * (int)sizeof(typename cplx_of<T>::type);
  int qp = (48 * 1024) / bytes_per_pair - 1;
  int p2 = 1;  // power of two, so that the element stride QP + 1 is odd
  while (p2 * 2 <= qp && p2 < 8) p2 *= 2;
  return p2;
}

template <typename T>
static cudaError_t launch_x_impl(const Launch<T>& L, XMode mode, const PointParams& pp, const double* src_f64,
                                 const T* src_t, double* dst_f64, const double* warm, int in_buf, int out_buf,
                                 bool check_done) {
  typedef typename cplx_of<T>::type V;
  if (mode == X_POWERLAW_H) mode = X_POWERLAW;
  if (mode == X_UPDATE_FD) mode = X_UPDATE;  // its R2C output is not read by the stencil curl
  XArgs<T> a{};
  const Geo& g = L.g;
  a.g = g;
  const bool pin = (mode == X_UPDATE || mode == X_CROP_F64 || mode == X_ADJ_CROP);
  const bool pout = (mode == X_MASKPAD || mode == X_PAD_F64 || mode == X_ADJ_PAD);
  const bool c2r = !(mode == X_FWD_F64 || mode == X_PAD_F64 || mode == X_ADJ_PAD || mode == X_ADJ_IN);
  const bool r2c = !(mode == X_TO_F64 || mode == X_CROP_F64 || mode == X_ADJ_COMBINE);
  a.Lin = c2r ? (pin ? 2 * g.nx : g.nx) : 0;
  a.Lout = r2c ? (pout ? 2 * g.nx : g.nx) : 0;
  a.Lmax = a.Lin > a.Lout ? a.Lin : a.Lout;
  if (a.Lmax < g.nx) a.Lmax = g.nx;
  a.QP = x_pairs<T>(a.Lmax);
  if (a.Lin) a.pin = make_plan(a.Lin);
  if (a.Lout) a.pout = make_plan(a.Lout);
  a.spec_in = pin ? L.w->Pd : L.w->U;
  a.in_rows = pin ? 2 * g.ny : g.ny;
  a.in_sx = pin ? g.sxp : g.sxu;
  a.spec_out = pout ? L.w->Pd : L.w->U;
  a.out_rows = pout ? 2 * g.ny : g.ny;
  a.out_sx = pout ? g.sxp : g.sxu;
  a.tw_in = a.Lin ? (pin ? L.w->twp[0] : L.w->twu[0]) : nullptr;
  a.tw_out = a.Lout ? (pout ? L.w->twp[0] : L.w->twu[0]) : nullptr;
  a.src_f64 = src_f64;
  a.src_t = src_t;
  a.dst_f64 = dst_f64;
  a.warm = warm;
  a.mask = L.mask;
  a.jc = L.w->jc;
  a.hold = L.w->Hd[in_buf];
  a.hnew = L.w->Hd[out_buf];
  a.pp = pp;
  a.ctrl = L.ctrl;
  a.partials = L.partials;
  a.check_done = check_done ? 1 : 0;
  a.out_buf = out_buf;
  a.use_box = (L.use_box && mode == X_MASKPAD) ? 1 : 0;
  a.by0 = L.by0;
  a.by1 = L.by1;
  a.bz0 = L.bz0;
  a.bz1 = L.bz1;
  const int rows = a.use_box ? (L.bz1 - L.bz0) * (L.by1 - L.by0) : g.ny * g.nz;
  const int R = 2 * a.QP;
  const int grid = (rows + R - 1) / R;
  const size_t smem = (size_t)(2 * 3 * a.Lmax * (a.QP + 1) + 512) * sizeof(V);
  switch (mode) {
#define XCASE(M)                                                                                         \
  case M:                                                                                                \
    allow_smem<xpass_kernel<T, M>>();                                                                  \
    xpass_kernel<T, M><<<grid, kThreads, smem, L.st>>>(a);                                               \
    return checked_launch("xpass_kernel", dim3(grid), kThreads, smem);
    XCASE(X_FWD_F64) XCASE(X_POWERLAW) XCASE(X_ASSEMBLE) XCASE(X_MASKPAD) XCASE(X_UPDATE) XCASE(X_TO_F64)
    XCASE(X_PAD_F64) XCASE(X_CROP_F64) XCASE(X_ADJ_PAD) XCASE(X_ADJ_CROP) XCASE(X_ADJ_COMBINE) XCASE(X_ADJ_IN)
    XCASE(X_ADJ_POWERLAW)
#undef XCASE
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_x(const Launch<T>& L, XMode mode, const PointParams& pp, const double* src_f64, double* dst_f64,
                     const double* warm, int in_buf, int out_buf, bool check_done) {
  // the FP32 forward passes use the register-resident kernels; the transposed
  // (reverse-mode) passes use the shared-memory kernel in every precision
  if constexpr (sizeof(T) == 4)
    if (mode < X_ADJ_PAD || mode == X_POWERLAW_H || mode == X_UPDATE_FD)
      return launch_x_reg(L, mode, pp, src_f64, dst_f64, warm, in_buf, out_buf, check_done);
  return launch_x_impl<T>(L, mode, pp, src_f64, nullptr, dst_f64, warm, in_buf, out_buf, check_done);
}

template <typename T>
cudaError_t launch_x_pad_rows(const Launch<T>& L, const PointParams& pp, const T* rows, bool check_done) {
  return launch_x_impl<T>(L, X_PAD_F64, pp, nullptr, rows, nullptr, nullptr, 0, 0, check_done);
}

template <typename T> static int col_tile() { return sizeof(T) == 4 ? 16 : 8; }

template <typename T>
cudaError_t launch_y(const Launch<T>& L, bool padded, bool inverse, bool check_done) {
  typedef typename cplx_of<T>::type V;
  if constexpr (sizeof(T) == 4) return launch_y_reg(L, padded, inverse, check_done);
  const Geo& g = L.g;
  YArgs<T> a{};
  a.base = padded ? L.w->Pd : L.w->U;
  a.rows = padded ? 2 * g.ny : g.ny;
  a.sx = padded ? g.sxp : g.sxu;
  a.HX = padded ? g.nx + 1 : g.nx / 2 + 1;
  a.nzs = g.nz;
  a.TC = col_tile<T>();
  const int Ly = padded ? 2 * g.ny : g.ny;
  a.pl = make_plan(Ly);
  a.Lin = (padded && !inverse) ? g.ny : Ly;
  a.Lout = (padded && inverse) ? g.ny : Ly;
  a.tw = padded ? L.w->twp[1] : L.w->twu[1];
  a.ctrl = L.ctrl;
  a.check_done = check_done ? 1 : 0;
  // the padded forward pass of an Eq. 5 iteration: only the planes and rows of Omega's box
  const bool box = L.use_box && padded && !inverse;
  a.zoff = box ? L.bz0 : 0;
  a.ylo = box ? L.by0 : 0;
  a.yhi = box ? L.by1 : Ly;
  dim3 grid((a.HX + a.TC - 1) / a.TC, box ? L.bz1 - L.bz0 : g.nz, 3);
  const size_t smem = (size_t)(2 * Ly * (a.TC + 1) + 256) * sizeof(V);
  if (inverse) {
    allow_smem<ypass_kernel<T, true>>();
    ypass_kernel<T, true><<<grid, kThreads, smem, L.st>>>(a);
    return checked_launch("ypass_kernel inv", grid, kThreads, smem);
  } else {
    allow_smem<ypass_kernel<T, false>>();
    ypass_kernel<T, false><<<grid, kThreads, smem, L.st>>>(a);
    return checked_launch("ypass_kernel fwd", grid, kThreads, smem);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_z(const Launch<T>& L, bool padded, bool check_done, double scale) {
  typedef typename cplx_of<T>::type V;
  if constexpr (sizeof(T) == 4) return launch_z_reg(L, padded, check_done, scale);
  const Geo& g = L.g;
  ZArgs<T> a{};
  a.base = padded ? L.w->Pd : L.w->U;
  a.rows = padded ? 2 * g.ny : g.ny;
  a.sx = padded ? g.sxp : g.sxu;
  a.HX = padded ? g.nx + 1 : g.nx / 2 + 1;
  a.nzs = g.nz;
  a.TC = col_tile<T>();
  const int Lz = padded ? 2 * g.nz : g.nz;
  // keep the 3-component ping-pong pair within ~80 KB, so that two CTAs share an SM (the
  // 256-point padded transform then takes two columns per CTA)
  while (a.TC > 2 && (size_t)(2 * 3 * Lz * (a.TC + 1)) * sizeof(V) > 80 * 1024) a.TC /= 2;
  a.pl = make_plan(Lz);
  a.tw = padded ? L.w->twp[2] : L.w->twu[2];
  a.kt0 = L.w->kt[0]; a.kt1 = L.w->kt[1]; a.kt2 = L.w->kt[2];
  a.st0 = L.w->st[0]; a.st1 = L.w->st[1]; a.st2 = L.w->st[2];
  a.scale = (T)scale;
  a.kap = L.w->kap;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
  a.ctrl = L.ctrl;
  a.check_done = check_done ? 1 : 0;
  a.zlo = (padded && L.use_box) ? L.bz0 : 0;  // the source box of an Eq. 5 iteration
  a.zhi = (padded && L.use_box) ? L.bz1 : Lz;
  dim3 grid((a.HX + a.TC - 1) / a.TC, a.rows, 1);
  const size_t smem = (size_t)(2 * 3 * Lz * (a.TC + 1) + 256) * sizeof(V);
  if (padded) {
    allow_smem<zpass_kernel<T, 1>>();
    zpass_kernel<T, 1><<<grid, kThreads, smem, L.st>>>(a);
    return checked_launch("zpass_kernel 1", grid, kThreads, smem);
  } else {
    allow_smem<zpass_kernel<T, 0>>();
    zpass_kernel<T, 0><<<grid, kThreads, smem, L.st>>>(a);
    return checked_launch("zpass_kernel 0", grid, kThreads, smem);
  }
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_z_curl(const Launch<T>& L, bool check_done, double scale) {
  return launch_z<T>(L, false, check_done, scale);
}
template <typename T> cudaError_t launch_z_kernel(const Launch<T>& L, bool check_done) {
  return launch_z<T>(L, true, check_done, 1.0);
}

#define INST_PASSES(T)                                                                                           \
  template cudaError_t launch_x<T>(const Launch<T>&, XMode, const PointParams&, const double*, double*,        \
                                   const double*, int, int, bool);                                             \
  template cudaError_t launch_x_pad_rows<T>(const Launch<T>&, const PointParams&, const T*, bool);             \
  template cudaError_t launch_y<T>(const Launch<T>&, bool, bool, bool);                                        \
  template cudaError_t launch_z_curl<T>(const Launch<T>&, bool, double);                                       \
  template cudaError_t launch_z_kernel<T>(const Launch<T>&, bool);

}  // namespace scfft
