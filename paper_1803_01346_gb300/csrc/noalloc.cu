// noalloc.cu - an allocation-free variant of the smoothed spectral curl.
//
// Some callers cannot allocate device memory at the point where they need the
// curl: code that runs inside a region where cudaMalloc is forbidden or
// unsafe (while another library holds the stream in a capture, inside a
// real-time loop whose memory budget was fixed up front, or from a host
// framework that owns every device allocation itself).  scfft_curl_noalloc
// serves them: it needs no context and allocates nothing, device or host.  Its
// scratch (the half spectrum and the per-grid tables) lives in one file-scope
// __device__ array of kNoAllocBytes, which every GPU that loads this library
// keeps until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Each call rewrites all of it that it reads (tables first, then
// the forward x pass fills every spectrum entry the later passes read), so
// nothing has to start at zero.  Two calls whose work overlaps on the GPU
// (different streams, or different host threads on one device) race on the
// array and corrupt each other's results: serialize them.
#include <math.h>

#include <mutex>

#include "scfft.h"
#include "scfft_internal.cuh"

using namespace scfft;

namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;  // 8 MiB: grids up to 64^3 nodes
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch for each device.  In host code the
// symbol name is only a host-side stand-in, never a device address.  The
// address is looked up again on every call made outside a stream capture (the
// module, and the array with it, may have been reloaded at another address
// after a device reset); a call inside a capture uses the cached address.
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

#define NCK(x)                                  \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      note_cuda_error(e_, "noalloc.cu", __LINE__); \
      return SCFFT_ECUDA;                       \
    }                                           \
  } while (0)

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Per-grid tables, written on the device: twiddles W_L^m for L = nx, ny, nz;
// derivative wavenumbers pi m / L_a (0 on the Nyquist entry) and smoothing
// factors exp(-sigma^2 k^2 / 2) for the x half spectrum and the full y, z axes.
__global__ void noalloc_tables(double2* tw, double* kt, double* st, int nx, int ny, int nz, double Lx, double Ly,
                               double Lz, double sigma) {
  const int n[3] = {nx, ny, nz};
  const double L[3] = {Lx, Ly, Lz};
  int toff = 0, koff = 0;
  for (int a = 0; a < 3; ++a) {
    for (int m = threadIdx.x; m < n[a]; m += blockDim.x) {
      double s, c;
      sincospi(2.0 * m / n[a], &s, &c);
      tw[toff + m] = make_double2(c, -s);
    }
    const int len = a == 0 ? n[0] / 2 + 1 : n[a];
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const int m = (a == 0) ? i : (i < n[a] / 2 ? i : i - n[a]);
      const double k = M_PI * m / L[a];
      kt[koff + i] = (i == n[a] / 2) ? 0.0 : k;
      st[koff + i] = exp(-0.5 * sigma * sigma * k * k);
    }
    toff += n[a];
    koff += len;
  }
}

bool grid_ok(int n) { return n == 16 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128; }

}  // namespace

extern "C" scfft_status scfft_curl_noalloc(const scfft_grid* grid, double sigma_scale, const double* f, double* out,
                                           void* stream) {
  if (!grid || !f || !out || f == out || !(sigma_scale >= 0) || !isfinite(sigma_scale)) return SCFFT_EINVAL;
  if (!grid_ok(grid->nx) || !grid_ok(grid->ny) || !grid_ok(grid->nz)) return SCFFT_EINVAL;
  if (!(grid->Lx > 0) || !(grid->Ly > 0) || !(grid->Lz > 0)) return SCFFT_EINVAL;
  Geo g{};
  g.nx = grid->nx; g.ny = grid->ny; g.nz = grid->nz;
  g.sxu = (grid->nx / 2 + 1 + 7) / 8 * 8;
  g.sxp = (grid->nx + 1 + 7) / 8 * 8;
  g.N = (long long)g.nx * g.ny * g.nz;
  // carve the scratch: twiddles | wavenumbers | smoothing | half spectrum
  const size_t ntw = (size_t)g.nx + g.ny + g.nz;
  const size_t nk = (size_t)g.nx / 2 + 1 + g.ny + g.nz;
  const size_t off_kt = align256(ntw * sizeof(double2));
  const size_t off_st = off_kt + align256(nk * sizeof(double));
  const size_t off_u = off_st + align256(nk * sizeof(double));
  const size_t need = off_u + sizeof(double2) * 3 * (size_t)g.nz * g.ny * g.sxu;
  if (need > kNoAllocBytes) return SCFFT_ESIZE;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the scratch address belongs to the device of the stream, which must be the current device
  // (kernels are launched on the current device)
  int dev = 0, sdev = 0;
  NCK(cudaGetDevice(&dev));
  NCK(cudaStreamGetDevice(s, &sdev));
  if (sdev != dev || dev < 0 || dev >= kMaxDevices) return SCFFT_EINVAL;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  NCK(cudaStreamIsCapturing(s, &cap));
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
      if (cap != cudaStreamCaptureStatusNone) return SCFFT_ESTATE;  // first call on this device inside a capture
      void* p = nullptr;
      NCK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      if (!p) return SCFFT_ECUDA;
      g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_scratch_addr[dev];
  }

  Work<double> w;
  double2* tw = reinterpret_cast<double2*>(base);
  double* kt = reinterpret_cast<double*>(base + off_kt);
  double* st = reinterpret_cast<double*>(base + off_st);
  w.U = reinterpret_cast<double2*>(base + off_u);
  w.twu[0] = tw; w.twu[1] = tw + g.nx; w.twu[2] = tw + g.nx + g.ny;
  w.kt[0] = kt; w.kt[1] = kt + g.nx / 2 + 1; w.kt[2] = kt + g.nx / 2 + 1 + g.ny;
  w.st[0] = st; w.st[1] = st + g.nx / 2 + 1; w.st[2] = st + g.nx / 2 + 1 + g.ny;
  const double dx = 2 * grid->Lx / g.nx, dy = 2 * grid->Ly / g.ny, dz = 2 * grid->Lz / g.nz;
  const double sigma = sigma_scale * 0.5 * sqrt(dx * dx + dy * dy + dz * dz);

  Launch<double> L;
  L.g = g;
  L.w = &w;
  L.ctrl = nullptr;      // the curl passes never consult the control block
  L.mask = nullptr;
  L.partials = nullptr;
  L.st = s;
  PointParams pp{};
  noalloc_tables<<<1, 256, 0, s>>>(tw, kt, st, g.nx, g.ny, g.nz, grid->Lx, grid->Ly, grid->Lz, sigma);
  NCK(cudaGetLastError());
  NCK(launch_x<double>(L, X_FWD_F64, pp, f, nullptr, nullptr, 0, 0, false));
  NCK(launch_y<double>(L, false, false, false));
  NCK(launch_z_curl<double>(L, false, 1.0 / (double)g.N));
  NCK(launch_y<double>(L, false, true, false));
  NCK(launch_x<double>(L, X_TO_F64, pp, nullptr, out, nullptr, 0, 0, false));
  return SCFFT_OK;
}
