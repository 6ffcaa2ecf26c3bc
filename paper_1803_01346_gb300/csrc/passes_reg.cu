// passes_reg.cu - register-resident y and z passes for the FP32 path.
//
// A length L = R1 * R2 transform of a tile of TC consecutive kx columns is
// done in two register stages with one shared-memory transpose between them
// (the "four-step" split):
//   X[k2 + R2 k1] = sum_n1 W_R1^{n1 k1} W_L^{n1 k2} ( sum_n2 x[n1 + R1 n2] W_R2^{n2 k2} )
// Thread (c, n1) loads its R2 points straight from global memory, runs the
// R2-point DFT, applies W_L^{n1 k2} and writes one transpose; thread (c, k2)
// reads R1 points back and runs the R1-point DFT, leaving X[k2 + R2 k1] in
// registers.  On the zero-padded grid the forward input has only the first
// L/2 rows (n2 < R2/2, skipped at load) and the inverse output keeps only the
// first L/2 rows (k1 < R1/2 or m2 < R2/2, skipped at store).
//
// The z passes keep the three field components of a column in registers so
// the spectral curl (i S(k) k x F) or the kernel-spectrum product (K^ x F,
// Eq. 7) is applied between the forward and inverse transforms without
// another trip through memory.  The inverse after the product uses the mirror
// split y[m1 + R1 m2] = sum_k2 W_R2^{-m2 k2} W_L^{-m1 k2} (sum_k1 X[k2 + R2 k1] W_R1^{-m1 k1}),
// which starts from exactly the registers the forward split ends with.
#include "scfft_internal.cuh"

namespace scfft {

namespace {

constexpr int kPad8 = 8;  // row padding (complex elements) that spreads half-warps over all banks

template <int R1, int R2> struct RegGeom {
  static constexpr int L = R1 * R2;
};

template <typename V> __device__ __forceinline__ V tw_mul(V a, V w, bool inv) { return inv ? cmulc(a, w) : cmul(a, w); }

template <typename V> __device__ __forceinline__ V zero_v();
template <> __device__ __forceinline__ float2 zero_v<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_v<double2>() { return make_double2(0.0, 0.0); }

}  // namespace

// ---------------------------------------------------------------- y pass
// grid (ceil(HX/TC), nzs, 3), block TC*R1 threads.
template <typename T, int R1, int R2, int TC, bool INV, bool PIN, bool POUT>
__global__ void __launch_bounds__(TC * R1) ypass_reg_kernel(typename cplx_of<T>::type* __restrict__ base, int rows,
                                                            int sx, int HX, int nzs,
                                                            const typename cplx_of<T>::type* __restrict__ twg,
                                                            const Ctrl* ctrl, int check_done) {
  typedef typename cplx_of<T>::type V;
  constexpr int L = R1 * R2;
  constexpr int S2 = R1 * TC + kPad8;  // transpose row stride
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (check_done && ctrl->done) return;
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* sm = tw + L;
  const int t = threadIdx.x;
  for (int i = t; i < L; i += TC * R1) tw[i] = twg[i];
  const int c = t % TC, n1 = t / TC;
  const int cz = blockIdx.z, z = blockIdx.y, kx = blockIdx.x * TC + c;
  const bool colok = kx < HX;
  V* col = base + ((size_t)(cz * nzs + z) * rows) * sx + kx;
  V v[R2];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    if (PIN && n2 >= R2 / 2) {
      v[n2] = zero_v<V>();
    } else {
      v[n2] = colok ? col[(size_t)(n1 + R1 * n2) * sx] : zero_v<V>();
    }
  }
  __syncthreads();  // twiddles staged
  DFT<R2, INV, V>::run(v);
#pragma unroll
  for (int k2 = 1; k2 < R2; ++k2) v[k2] = tw_mul(v[k2], tw[n1 * k2], INV);
#pragma unroll
  for (int k2 = 0; k2 < R2; ++k2) sm[k2 * S2 + n1 * TC + c] = v[k2];
  __syncthreads();
  if (n1 < R2) {
    const int k2 = n1;
    V w[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) w[m] = sm[k2 * S2 + m * TC + c];
    DFT<R1, INV, V>::run(w);
    if (colok) {
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        if (POUT && k1 >= R1 / 2) continue;
        col[(size_t)(k2 + R2 * k1) * sx] = w[k1];
      }
    }
  }
}

// ---------------------------------------------------------------- z pass (3 components)
// KIND 0: spectral curl on the unpadded grid (L = nz, no pruning).
// KIND 1: kernel-spectrum product on the padded grid (L = 2nz, pruned in/out).
// grid (ceil(HX/TC), rows), block TC*R1 threads.
template <typename T, int R1, int R2, int TC, int KIND>
__global__ void __launch_bounds__(TC * R1) zpass_reg_kernel(typename cplx_of<T>::type* __restrict__ base, int rows,
                                                            int sx, int HX, int nzs,
                                                            const typename cplx_of<T>::type* __restrict__ twg,
                                                            const T* __restrict__ kt0, const T* __restrict__ kt1,
                                                            const T* __restrict__ kt2, const T* __restrict__ st0,
                                                            const T* __restrict__ st1, const T* __restrict__ st2,
                                                            T scale, const T* __restrict__ kap, int nx, int ny,
                                                            int nz, const Ctrl* ctrl, int check_done) {
  typedef typename cplx_of<T>::type V;
  constexpr int L = R1 * R2;
  constexpr bool PR = (KIND == 1);         // pruned input and output
  constexpr int S2 = R1 * TC + kPad8;      // forward transpose: [k2][n1][c]
  constexpr int S1 = R2 * TC + kPad8;      // inverse transpose: [m1][k2][c]
  constexpr int CSF = R2 * S2, CSI = R1 * S1;
  constexpr int CS = CSF > CSI ? CSF : CSI;  // one component's transpose buffer
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (check_done && ctrl->done) return;
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* sm = tw + L;
  const int t = threadIdx.x;
  for (int i = t; i < L; i += TC * R1) tw[i] = twg[i];
  const int c = t % TC, n1 = t / TC;
  const int y = blockIdx.y, kx = blockIdx.x * TC + c;
  const bool colok = kx < HX;
  const size_t zstride = (size_t)rows * sx;
  const size_t cstride = (size_t)nzs * zstride;
  V* col = base + (size_t)y * sx + kx;

  // ---- forward, stage A: R2-point DFTs along n2 for the three components
  V v[3][R2];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      if (PR && n2 >= R2 / 2) v[q][n2] = zero_v<V>();
      else v[q][n2] = colok ? col[q * cstride + (size_t)(n1 + R1 * n2) * zstride] : zero_v<V>();
    }
  __syncthreads();  // twiddles staged
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    DFT<R2, false, V>::run(v[q]);
#pragma unroll
    for (int k2 = 1; k2 < R2; ++k2) v[q][k2] = cmul(v[q][k2], tw[n1 * k2]);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) sm[q * CS + k2 * S2 + n1 * TC + c] = v[q][k2];
  }
  __syncthreads();
  const bool actB = n1 < R2;
  const int k2 = n1;
  V w[3][R1];
  if (actB) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
      for (int m = 0; m < R1; ++m) w[q][m] = sm[q * CS + k2 * S2 + m * TC + c];
      DFT<R1, false, V>::run(w[q]);
    }
    // ---- product at kz = k2 + R2 k1
    const int kxc = colok ? kx : 0;
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const int kz = k2 + R2 * k1;
      T ax, ay, az, s;
      if (KIND == 0) {
        ax = kt0[kxc]; ay = kt1[y]; az = kt2[kz];
        s = st0[kxc] * st1[y] * st2[kz] * scale;
      } else {
        const int fy = (y <= ny) ? y : 2 * ny - y;
        const int fz = (kz <= nz) ? kz : 2 * nz - kz;
        const size_t oct = (size_t)(nz + 1) * (ny + 1) * (nx + 1);
        const size_t off = ((size_t)fz * (ny + 1) + fy) * (nx + 1) + kxc;
        ax = kap[off];
        ay = (y <= ny) ? kap[oct + off] : -kap[oct + off];
        az = (kz <= nz) ? kap[2 * oct + off] : -kap[2 * oct + off];
        s = (T)1;
      }
      const V F0 = w[0][k1], F1 = w[1][k1], F2 = w[2][k1];
      // G = i s (a x F)
      const V cx = mk(ay * F2.x - az * F1.x, ay * F2.y - az * F1.y);
      const V cy = mk(az * F0.x - ax * F2.x, az * F0.y - ax * F2.y);
      const V cz = mk(ax * F1.x - ay * F0.x, ax * F1.y - ay * F0.y);
      w[0][k1] = mk(-s * cx.y, s * cx.x);
      w[1][k1] = mk(-s * cy.y, s * cy.x);
      w[2][k1] = mk(-s * cz.y, s * cz.x);
    }
  }
  __syncthreads();  // forward transpose buffer is free again
  // ---- inverse, stage A': R1-point inverse DFTs along k1, twiddle, transpose
  if (actB) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      DFT<R1, true, V>::run(w[q]);
#pragma unroll
      for (int m1 = 0; m1 < R1; ++m1) {
        const V a = (m1 == 0) ? w[q][m1] : cmulc(w[q][m1], tw[m1 * k2]);
        sm[q * CS + m1 * S1 + k2 * TC + c] = a;
      }
    }
  }
  __syncthreads();
  // ---- inverse, stage B': R2-point inverse DFTs along k2, output rows m1 + R1 m2
  const int m1 = n1;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
#pragma unroll
    for (int j = 0; j < R2; ++j) v[q][j] = sm[q * CS + m1 * S1 + j * TC + c];
    DFT<R2, true, V>::run(v[q]);
    if (colok) {
#pragma unroll
      for (int m2 = 0; m2 < R2; ++m2) {
        if (PR && m2 >= R2 / 2) continue;
        col[q * cstride + (size_t)(m1 + R1 * m2) * zstride] = v[q][m2];
      }
    }
  }
}

// ---------------------------------------------------------------- launchers
namespace {

template <int R1, int R2, int TC, bool INV, bool PIN, bool POUT>
cudaError_t go_y(const Launch<float>& L, float2* base, int rows, int sx, int HX, const float2* tw, bool chk) {
  constexpr int Lt = R1 * R2;
  const size_t smem = sizeof(float2) * (Lt + R2 * (R1 * TC + kPad8));
  auto k = ypass_reg_kernel<float, R1, R2, TC, INV, PIN, POUT>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((HX + TC - 1) / TC, L.g.nz, 3);
  k<<<grid, TC * R1, smem, L.st>>>(base, rows, sx, HX, L.g.nz, tw, L.ctrl, chk ? 1 : 0);
  return cudaGetLastError();
}

template <int R1, int R2, int TC, int KIND>
cudaError_t go_z(const Launch<float>& L, float2* base, int rows, int sx, int HX, const float2* tw, double scale,
                 bool chk) {
  constexpr int Lt = R1 * R2;
  constexpr int CSF = R2 * (R1 * TC + kPad8), CSI = R1 * (R2 * TC + kPad8);
  constexpr int CS = CSF > CSI ? CSF : CSI;
  const size_t smem = sizeof(float2) * (Lt + 3 * CS);
  auto k = zpass_reg_kernel<float, R1, R2, TC, KIND>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((HX + TC - 1) / TC, rows, 1);
  const Work<float>& w = *L.w;
  k<<<grid, TC * R1, smem, L.st>>>(base, rows, sx, HX, L.g.nz, tw, w.kt[0], w.kt[1], w.kt[2], w.st[0], w.st[1],
                                   w.st[2], (float)scale, w.kap, L.g.nx, L.g.ny, L.g.nz, L.ctrl, chk ? 1 : 0);
  return cudaGetLastError();
}

// Dispatch a length to its (R1, R2) split with R1 >= R2.
template <template <int, int> class F, typename... A> cudaError_t by_length(int Lt, A&&... a) {
  switch (Lt) {
    case 16: return F<4, 4>::run(a...);
    case 32: return F<8, 4>::run(a...);
    case 48: return F<12, 4>::run(a...);
    case 64: return F<8, 8>::run(a...);
    case 96: return F<12, 8>::run(a...);
    case 128: return F<16, 8>::run(a...);
    case 192: return F<16, 12>::run(a...);
    case 256: return F<16, 16>::run(a...);
  }
  return cudaErrorInvalidValue;
}

template <int R1, int R2> struct YFwdU {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    return go_y<R1, R2, 16, false, false, false>(L, L.w->U, g.ny, g.sxu, g.nx / 2 + 1, L.w->twu[1], chk);
  }
};
template <int R1, int R2> struct YInvU {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    return go_y<R1, R2, 16, true, false, false>(L, L.w->U, g.ny, g.sxu, g.nx / 2 + 1, L.w->twu[1], chk);
  }
};
template <int R1, int R2> struct YFwdP {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    return go_y<R1, R2, 16, false, true, false>(L, L.w->Pd, 2 * g.ny, g.sxp, g.nx + 1, L.w->twp[1], chk);
  }
};
template <int R1, int R2> struct YInvP {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    return go_y<R1, R2, 16, true, false, true>(L, L.w->Pd, 2 * g.ny, g.sxp, g.nx + 1, L.w->twp[1], chk);
  }
};
template <int R1, int R2> struct ZCurl {
  static cudaError_t run(const Launch<float>& L, bool chk, double scale) {
    const Geo& g = L.g;
    return go_z<R1, R2, 8, 0>(L, L.w->U, g.ny, g.sxu, g.nx / 2 + 1, L.w->twu[2], scale, chk);
  }
};
template <int R1, int R2> struct ZKern {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    return go_z<R1, R2, 8, 1>(L, L.w->Pd, 2 * g.ny, g.sxp, g.nx + 1, L.w->twp[2], 1.0, chk);
  }
};

}  // namespace

cudaError_t launch_y_reg(const Launch<float>& L, bool padded, bool inverse, bool check_done) {
  const int Ly = padded ? 2 * L.g.ny : L.g.ny;
  if (!padded) return inverse ? by_length<YInvU>(Ly, L, check_done) : by_length<YFwdU>(Ly, L, check_done);
  return inverse ? by_length<YInvP>(Ly, L, check_done) : by_length<YFwdP>(Ly, L, check_done);
}

cudaError_t launch_z_reg(const Launch<float>& L, bool padded, bool check_done, double scale) {
  if (!padded) return by_length<ZCurl>(L.g.nz, L, check_done, scale);
  return by_length<ZKern>(2 * L.g.nz, L, check_done);
}

}  // namespace scfft
