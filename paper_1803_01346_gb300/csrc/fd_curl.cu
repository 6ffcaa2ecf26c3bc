// fd_curl.cu - the local-stencil curl option: the three curls of the right-hand side
// (j = curl h of Eq. 4, dh_in = -curl e / mu0 of Eq. 3, and the curl of dh^i inside Eq. 5)
// by second-order central differences on the periodic grid,
//   (d_a f)(i) = (f(i + e_a) - f(i - e_a)) / (2 d_a),
// instead of the smoothed spectral derivatives.  Each curl is a stencil over the 3*N node
// values (one thread per node, x fastest, neighbours from L1/L2), so the unpadded grid's FFT
// passes drop out: the pre-stage is two stencil kernels and an Eq. 5 iteration becomes
// [masked curl] -> padded R2C -> y -> z (K^ x F) -> y -> C2R + update.
#include "scfft_internal.cuh"

namespace scfft {

namespace {

template <typename T> __device__ __forceinline__ T rho_fd(T jn, T jcv, T n, T e0);
template <> __device__ __forceinline__ float rho_fd(float jn, float jcv, float n, float e0) {
  if (jn == 0.f) return (n == 1.f) ? e0 / jcv : 0.f;
  return (e0 / jcv) * exp2f((n - 1.f) * log2f(jn / jcv));
}
template <> __device__ __forceinline__ double rho_fd(double jn, double jcv, double n, double e0) {
  if (jn == 0.0) return (n == 1.0) ? e0 / jcv : 0.0;
  return (e0 / jcv) * pow(jn / jcv, n - 1.0);
}

// Reads component q of a field at node (x, y, z): from an FP64 array or an FP32 array.
struct Src {
  const double* f64;
  const float* f32;
  __device__ __forceinline__ double at(long long i) const { return f64 ? f64[i] : (double)f32[i]; }
};

// curl by central differences at node (x, y, z) of the field in src (3 components of N)
template <typename T, typename F>
__device__ __forceinline__ void curl_at(const F& f, int x, int y, int z, const Geo& g, T inv2d0, T inv2d1, T inv2d2,
                                        T c[3]) {
  const long long N = g.N;
  const int xp = x + 1 == g.nx ? 0 : x + 1, xm = x == 0 ? g.nx - 1 : x - 1;
  const int yp = y + 1 == g.ny ? 0 : y + 1, ym = y == 0 ? g.ny - 1 : y - 1;
  const int zp = z + 1 == g.nz ? 0 : z + 1, zm = z == 0 ? g.nz - 1 : z - 1;
  const long long row = ((long long)z * g.ny + y) * g.nx;
  const long long iyp = ((long long)z * g.ny + yp) * g.nx + x, iym = ((long long)z * g.ny + ym) * g.nx + x;
  const long long izp = ((long long)zp * g.ny + y) * g.nx + x, izm = ((long long)zm * g.ny + y) * g.nx + x;
  const long long ixp = row + xp, ixm = row + xm;
  // c_x = d_y f_z - d_z f_y; c_y = d_z f_x - d_x f_z; c_z = d_x f_y - d_y f_x (each difference
  // taken in the source's precision, then rounded to T)
  c[0] = (T)(f(2 * N + iyp) - f(2 * N + iym)) * inv2d1 - (T)(f(N + izp) - f(N + izm)) * inv2d2;
  c[1] = (T)(f(izp) - f(izm)) * inv2d2 - (T)(f(2 * N + ixp) - f(2 * N + ixm)) * inv2d0;
  c[2] = (T)(f(N + ixp) - f(N + ixm)) * inv2d0 - (T)(f(iyp) - f(iym)) * inv2d1;
}

// e = rho(j) j in Omega (Eq. 1, or the e(j, h) law of PointParams::law), rho_out j outside,
// with j = curl h; e -> out (T, 3N)
template <typename T>
__global__ void fd_efield_kernel(Src h, const uint8_t* __restrict__ mask, const T* __restrict__ jcmap, Geo g, T inv2d0,
                                 T inv2d1, T inv2d2, PointParams pp, T* __restrict__ out) {
  const long long N = g.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long r = i / g.nx;
    const int y = (int)(r % g.ny), z = (int)(r / g.ny);
    typedef typename acc_of<T>::type A;  // the law's arithmetic (FP64 for double-float)
    T jt[3];
    curl_at<T>([&](long long k) { return h.at(k); }, x, y, z, g, inv2d0, inv2d1, inv2d2, jt);
    const A j[3] = {to_acc(jt[0]), to_acc(jt[1]), to_acc(jt[2])};
    A f[3];
    if (mask[i]) {
      A jcv = jcmap ? to_acc(jcmap[i]) : (A)pp.jc;
      A a[3] = {(A)1, (A)1, (A)1};
      if (pp.law) {
        if (pp.kim_h0 > 0) {
          const A h0 = (A)h.at(i), h1 = (A)h.at(N + i), h2 = (A)h.at(2 * N + i);
          jcv = jcv / ((A)1 + sqrt(h0 * h0 + h1 * h1 + h2 * h2) / (A)pp.kim_h0);
        }
        for (int q = 0; q < 3; ++q) a[q] = (A)pp.aniso[q];
      }
      const A u0 = a[0] * j[0], u1 = a[1] * j[1], u2 = a[2] * j[2];
      const A rho = rho_fd<A>(sqrt(u0 * u0 + u1 * u1 + u2 * u2), jcv, (A)pp.n, (A)pp.e0);
      for (int q = 0; q < 3; ++q) f[q] = rho * a[q] * a[q];
    } else {
      f[0] = f[1] = f[2] = (A)pp.rho_out;
    }
    out[i] = from_acc<T>(f[0] * j[0]);
    out[N + i] = from_acc<T>(f[1] * j[1]);
    out[2 * N + i] = from_acc<T>(f[2] * j[2]);
  }
}

// dh^0 = -curl e / mu0 on Omega, the warm start on Omega_out -> hd0; then the state of the
// Eq. 5 loop is reset and the rhs parameters copied to the device, as the spectral path's
// assembly pass does
template <typename T>
__global__ void fd_assemble_kernel(const T* __restrict__ e, Src warm, const uint8_t* __restrict__ mask, Geo g,
                                   T inv2d0, T inv2d1, T inv2d2, PointParams pp, T* __restrict__ hd0, PointParams* ppd,
                                   const PointParams* pps, Ctrl* ctrl) {
  const long long N = g.N;
  const T s = -(T)pp.inv_mu0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    if (mask[i]) {
      const int x = (int)(i % g.nx);
      const long long r = i / g.nx;
      const int y = (int)(r % g.ny), z = (int)(r / g.ny);
      T c[3];
      curl_at<T>([&](long long k) { return e[k]; }, x, y, z, g, inv2d0, inv2d1, inv2d2, c);
      hd0[i] = s * c[0];
      hd0[N + i] = s * c[1];
      hd0[2 * N + i] = s * c[2];
    } else {
      hd0[i] = (T)warm.at(i);
      hd0[N + i] = (T)warm.at(N + i);
      hd0[2 * N + i] = (T)warm.at(2 * N + i);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *ppd = pps ? *pps : pp;
    ctrl->trips = 0;
    ctrl->done = 0;
    ctrl->iters = 0;
    ctrl->cur = 0;
    ctrl->counter = 0;
    ctrl->residual = 0.0;
  }
}

// j_in = chi curl dh^i (the source of Eq. 5), dh^i the iterate the device's iteration count
// selects; returns at entry once the Eq. 5 stop was reached (check_done)
template <typename T>
__global__ void fd_curl_mask_kernel(const uint8_t* __restrict__ mask, Geo g, T inv2d0, T inv2d1, T inv2d2,
                                    T* __restrict__ out, const Ctrl* ctrl, int check_done, const T* h0, const T* h1) {
  if (check_done && ctrl->done) return;
  const T* src = (*reinterpret_cast<volatile const int*>(&ctrl->iters) & 1) ? h1 : h0;
  const long long N = g.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    if (mask[i]) {
      const int x = (int)(i % g.nx);
      const long long r = i / g.nx;
      const int y = (int)(r % g.ny), z = (int)(r / g.ny);
      T c[3];
      curl_at<T>([&](long long k) { return src[k]; }, x, y, z, g, inv2d0, inv2d1, inv2d2, c);
      out[i] = c[0];
      out[N + i] = c[1];
      out[2 * N + i] = c[2];
    } else {
      out[i] = (T)0;
      out[N + i] = (T)0;
      out[2 * N + i] = (T)0;
    }
  }
}

int fd_blocks(long long n) {
  const long long b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

template <typename T>
cudaError_t launch_fd_efield(const Launch<T>& L, const PointParams& pp, const double* h64, const float* h32,
                             const double* d, T* out) {
  Src s{h64, h32};
  fd_efield_kernel<T><<<fd_blocks(L.g.N), 256, 0, L.st>>>(s, L.mask, L.w->jc, L.g, (T)(0.5 / d[0]), (T)(0.5 / d[1]),
                                                          (T)(0.5 / d[2]), pp, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fd_assemble(const Launch<T>& L, const PointParams& pp, const T* e, const double* warm64,
                               const float* warm32, const double* d) {
  Src w{warm64, warm32};
  fd_assemble_kernel<T><<<fd_blocks(L.g.N), 256, 0, L.st>>>(e, w, L.mask, L.g, (T)(0.5 / d[0]), (T)(0.5 / d[1]),
                                                            (T)(0.5 / d[2]), pp, L.w->Hd[0], L.ppd, L.pps,
                                                            L.ctrl);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fd_curl_mask(const Launch<T>& L, T* out, const double* d, bool check_done) {
  fd_curl_mask_kernel<T><<<fd_blocks(L.g.N), 256, 0, L.st>>>(L.mask, L.g, (T)(0.5 / d[0]), (T)(0.5 / d[1]),
                                                             (T)(0.5 / d[2]), out, L.ctrl, check_done ? 1 : 0,
                                                             L.w->Hd[0], L.w->Hd[1]);
  return cudaGetLastError();
}

#define INST_FD(T)                                                                                                 \
  template cudaError_t launch_fd_efield<T>(const Launch<T>&, const PointParams&, const double*, const float*,     \
                                           const double*, T*);                                                    \
  template cudaError_t launch_fd_assemble<T>(const Launch<T>&, const PointParams&, const T*, const double*,       \
                                             const float*, const double*);                                        \
  template cudaError_t launch_fd_curl_mask<T>(const Launch<T>&, T*, const double*, bool);
INST_FD(float)
INST_FD(double)
INST_FD(dfloat)
#undef INST_FD

}  // namespace scfft
