// passes.cu - the FFT pass kernels of the right-hand side (§2, Eqs. 1-7): launch diagnostics,
// plans, the small kernels and the kernel spectrum here; the shared-memory pass templates in
// passes_impl.cuh, instantiated here for float and double (passes_df64.cu: dfloat).
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
#include "passes_impl.cuh"

namespace scfft {

// ---------------------------------------------------------------- launch diagnostics
static char g_launch_fail[256] = "";

cudaError_t checked_launch(const char* what, dim3 grid, int block, size_t smem) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    snprintf(g_launch_fail, sizeof(g_launch_fail), "%s grid (%u,%u,%u) block %d smem %zu: %s", what, grid.x, grid.y,
             grid.z, block, smem, cudaGetErrorString(e));
  return e;
}

const char* last_launch_failure() { return g_launch_fail; }

// ---------------------------------------------------------------- plans
bool length_supported(int L) {
  switch (L) {
    case 16: case 32: case 48: case 64: case 96: case 128: case 192: case 256: return true;
    default: return false;
  }
}

FftPlan make_plan(int L) {
  FftPlan p{};
  p.L = L;
  auto set = [&](int a, int b) { p.ns = b ? 2 : 1; p.r[0] = a; p.r[1] = b; };
  switch (L) {
    case 16: set(16, 0); break;
    case 32: set(8, 4); break;
    case 48: set(16, 3); break;
    case 64: set(8, 8); break;
    case 96: set(8, 12); break;
    case 128: set(16, 8); break;
    case 192: set(16, 12); break;
    case 256: set(16, 16); break;
    default: p.ns = 0; break;
  }
  return p;
}

// ---------------------------------------------------------------- small kernels
template <typename T>
__global__ void finalize_kernel(const T* __restrict__ h0, const T* __restrict__ h1, const Ctrl* ctrl,
                                double* __restrict__ hdot, double* __restrict__ warm, long long n3) {
  const T* src = ctrl->cur ? h1 : h0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
    const double v = (double)src[i];
    hdot[i] = v;
    if (warm) warm[i] = v;
  }
}

template <typename T>
__global__ void convert_kernel(const double* __restrict__ src, T* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

// Kernel spectrum: sample dV grad G_sigma on the octant of offsets
// m_a in [0, n_a) (the m_a = -n_a planes are zero by construction).
__global__ void sample_kernel(double* __restrict__ K, long long cstride, int nx, int ny, int nz, double dx,
                              double dy, double dz, double sigma) {
  const long long N = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int mx = (int)(i % nx), my = (int)((i / nx) % ny), mz = (int)(i / ((long long)nx * ny));
    const double rx = mx * dx, ry = my * dy, rz = mz * dz;
    const double r2 = rx * rx + ry * ry + rz * rz;
    double gx = 0, gy = 0, gz = 0;
    if (r2 > 0) {
      const double r = sqrt(r2);
      const double u = r / (1.4142135623730950488 * sigma);
      // d/dr [erf(u)/(4 pi r)] = [(2/sqrt(pi)) u exp(-u^2) - erf(u)] / (4 pi r^2)
      const double g = (1.1283791670955125739 * u * exp(-u * u) - erf(u)) / (12.566370614359172954 * r2);
      const double dV = dx * dy * dz;
      gx = dV * g * rx / r; gy = dV * g * ry / r; gz = dV * g * rz / r;
    }
    K[i] = gx; K[cstride + i] = gy; K[2 * cstride + i] = gz;
  }
}

// Separable transform of one axis of an array (d2 slowest, d0 fastest):
//   odd : out[k] = -2 sum_{m=1}^{n-1} sin(pi k m / n) in[m]
//   even: out[k] = in[0] + 2 sum_{m=1}^{n-1} cos(pi k m / n) in[m]
// for k in [0, n]; the transformed axis grows from n to n+1 entries.
__global__ void axis_transform(const double* __restrict__ in, double* __restrict__ out, int d0, int d1, int d2,
                               int axis, int odd) {
  const int n = axis == 0 ? d0 : axis == 1 ? d1 : d2;
  const int o0 = d0 + (axis == 0), o1 = d1 + (axis == 1), o2 = d2 + (axis == 2);
  const long long tot = (long long)o0 * o1 * o2;
  const long long istr = axis == 0 ? 1 : axis == 1 ? d0 : (long long)d0 * d1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int i0 = (int)(i % o0), i1 = (int)((i / o0) % o1), i2 = (int)(i / ((long long)o0 * o1));
    const int k = axis == 0 ? i0 : axis == 1 ? i1 : i2;
    const long long b0 = axis == 0 ? 0 : i0, b1 = axis == 1 ? 0 : i1, b2 = axis == 2 ? 0 : i2;
    const double* src = in + (b2 * d1 + b1) * d0 + b0;
    double acc = odd ? 0.0 : src[0];
    for (int m = 1; m < n; ++m) {
      double sv, cv;
      sincospi((double)((long long)k * m % (2 * n)) / n, &sv, &cv);
      acc += (odd ? -2.0 * sv : 2.0 * cv) * src[m * istr];
    }
    out[i] = acc;
  }
}

__global__ void scale_convert_kernel(const double* __restrict__ src, double s, float* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)(src[i] * s);
}
// [3][oct] -> [oct] x float4 {a = 0, 1, 2, 0}: one 16-byte load per point in the z pass's product
__global__ void interleave_kernel(const float* __restrict__ src, float4* __restrict__ dst, long long oct) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < oct; i += (long long)gridDim.x * blockDim.x)
    dst[i] = make_float4(src[i], src[oct + i], src[2 * oct + i], 0.f);
}
__global__ void scale_convert_kernel(const double* __restrict__ src, double s, double* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i] * s;
}
__global__ void scale_convert_kernel(const double* __restrict__ src, double s, dfloat* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = dfloat(src[i] * s);
}

// ---------------------------------------------------------------- launchers
static int grid_for(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename T> cudaError_t launch_finalize(const Launch<T>& L, double* hdot, double* warm) {
  const long long n3 = 3 * L.g.N;
  finalize_kernel<T><<<grid_for(n3), kThreads, 0, L.st>>>(L.w->Hd[0], L.w->Hd[1], L.ctrl, hdot, warm, n3);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_convert(const double* src, T* dst, long long n, cudaStream_t st) {
  convert_kernel<T><<<grid_for(n), kThreads, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// scratch: 2 * 3 * (nx+1)(ny+1)(nz+1) doubles
template <typename T>
cudaError_t launch_kernel_spectrum(const Launch<T>& L, double Lx, double Ly, double Lz, double sigma, double* scratch) {
  const Geo& g = L.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const double dx = 2 * Lx / nx, dy = 2 * Ly / ny, dz = 2 * Lz / nz;
  const long long N = g.N;
  const long long oct = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  double* A = scratch;
  double* B = scratch + 3 * oct;
  // component c of the sampled octant sits at A + c*oct with dims (nx, ny, nz); each
  // axis transform grows one dimension by one: A -x-> B -y-> A -z-> B.
  sample_kernel<<<grid_for(N), kThreads, 0, L.st>>>(A, oct, nx, ny, nz, dx, dy, dz, sigma);
  for (int c = 0; c < 3; ++c) {
    double* a0 = A + c * oct;
    double* b0 = B + c * oct;
    axis_transform<<<grid_for((long long)(nx + 1) * ny * nz), kThreads, 0, L.st>>>(a0, b0, nx, ny, nz, 0, c == 0);
    axis_transform<<<grid_for((long long)(nx + 1) * (ny + 1) * nz), kThreads, 0, L.st>>>(b0, a0, nx + 1, ny, nz, 1,
                                                                                       c == 1);
    axis_transform<<<grid_for(oct), kThreads, 0, L.st>>>(a0, b0, nx + 1, ny + 1, nz, 2, c == 2);
  }
  scale_convert_kernel<<<grid_for(3 * oct), kThreads, 0, L.st>>>(B, 1.0 / (8.0 * (double)N), L.w->kap, 3 * oct);
  if constexpr (sizeof(T) == 4) interleave_kernel<<<grid_for(oct), kThreads, 0, L.st>>>(L.w->kap, L.w->kap4, oct);
  return cudaGetLastError();
}

#define INST(T)                                                                                                  \
  template cudaError_t launch_finalize<T>(const Launch<T>&, double*, double*);                                 \
  template cudaError_t launch_convert<T>(const double*, T*, long long, cudaStream_t);                          \
  template cudaError_t launch_kernel_spectrum<T>(const Launch<T>&, double, double, double, double, double*);
INST(float)
INST(double)
INST(dfloat)
#undef INST
INST_PASSES(float)
INST_PASSES(double)

}  // namespace scfft
