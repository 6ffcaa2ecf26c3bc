// scfft_internal.cuh - device workspaces, control block and pass launchers
// shared by the translation units of the library.
#pragma once
#include <cuda.h>  // CUtensorMap (types only; the encoder is fetched through the runtime)
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_core.cuh"

namespace scfft {

constexpr int kThreads = 256;  // every FFT pass kernel runs 256-thread CTAs

// Allow a kernel the largest dynamic shared memory a CTA may use, once per
// kernel (thread-safe static initialisation).  Raising the cap once, instead of
// setting it to each launch's size, keeps launches from concurrent host threads
// (batched instances of different sizes) from racing on the attribute.
template <auto Kern> inline void allow_smem() {
  static const cudaError_t once = [] {
    cudaFuncAttributes fa{};
    int dev = 0, optin = 0;
    cudaError_t e = cudaFuncGetAttributes(&fa, Kern);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the cap covers dynamic shared memory only: leave room for the kernel's static arrays
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
  }();
  (void)once;
}

// Device-side control block of one context (one rhs at a time per context).
struct Ctrl {
  int done;           // Eq. 5 stop reached: loop kernels of later iterations return at entry
  int iters;          // iterations executed in the current rhs
  int cur;            // which iterate buffer (0/1) holds the latest dh/dt
  int status;         // latched device status (scfft_status value)
  unsigned counter;   // arrival counter of the last-CTA reduction
  unsigned trips;     // trips of the graph-captured Eq. 5 loop in the current rhs (its hard bound)
  double residual;    // last Eq. 5 residual
  double err;         // last integrator error norm
  unsigned counter2;  // arrival counter of the error-norm reduction
  unsigned pad2_;
  unsigned long long iter_total;  // Eq. 5 iterations executed since the context was created
};

// Grid geometry and strides.
struct Geo {
  int nx, ny, nz;
  int sxu;        // row stride (complex) of the unpadded half spectrum, >= nx/2+1
  int sxp;        // row stride of the padded half spectrum, >= nx+1
  long long N;    // nx*ny*nz
};

// TMA descriptors of the FP32 padded y passes: the padded half spectrum Pd as read by the
// forward pass (its first ny rows) and by the inverse pass (all 2ny rows).
struct YMaps {
  CUtensorMap m[2];
};

// Launch schedule of the FP32 register passes (chosen by scfft_autotune): how the spectral
// columns are tiled over CTAs and how the padded y passes load, never the arithmetic of a
// column, so every schedule gives the same bits.
struct Sched {
  int zk_tc = 8;   // padded z pass (Biot-Savart kernel product): columns per CTA, 4 or 8
  int zc_tc = 8;   // smoothed-curl z pass: columns per CTA, 8 or 16
  int yu_tc = 8;   // unpadded y passes: columns per CTA, 8 or 16
  int yp_tma = 1;  // padded y passes: TMA-fed persistent kernel (1) or plain loads, 16 columns (0)
  int zk_tm = 0;   // padded z pass, 16 x 16 split: own-slot spectra in tensor memory (1) or shared memory (0)
  int box_fused = 0;  // Eq. 5 iteration: the three passes on Omega's box fused into one launch (1) or not (0)
  int xu3 = 0;        // Eq. 5 update pass: three components side by side in three warp groups (1) or one after another (0)
};

// Device workspaces of one FFT precision T.
template <typename T>
struct Work {
  typedef typename cplx_of<T>::type V;
  V* U = nullptr;        // [3][nz][ny][sxu]  unpadded half spectrum
  V* Pd = nullptr;       // [3][nz][2ny][sxp] padded half spectrum, z pruned to nz planes
  T* Hd[2] = {nullptr, nullptr};  // [3][N] iterates dh^i of Eq. 5
  T* jc = nullptr;       // [N] jc map or nullptr (uniform)
  T* kap = nullptr;      // [3][nz+1][ny+1][nx+1] imaginary part of the kernel spectrum / (8N)
  float4* kap4 = nullptr; // FP32 only: the same octant interleaved, [nz+1][ny+1][nx+1] x {a=0,1,2, 0}
  T* kt[3] = {nullptr, nullptr, nullptr};  // derivative wavenumbers (0 on Nyquist): nx/2+1, ny, nz
  T* st[3] = {nullptr, nullptr, nullptr};  // Gaussian smoothing factor per axis: nx/2+1, ny, nz
  V* twu[3] = {nullptr, nullptr, nullptr}; // twiddles W_L^m, L = nx, ny, nz
  V* twp[3] = {nullptr, nullptr, nullptr}; // twiddles, L = 2nx, 2ny, 2nz
  YMaps* ym = nullptr;   // FP32 only: TMA descriptors of the y passes (nullptr: plain-load y passes)
  T* Jd = nullptr;       // [3][N] masked stencil curl of the iterate (local-stencil curl option only)
  Sched sched;           // FP32 only: launch schedule of the register passes
};

enum XMode : int {
  X_FWD_F64 = 0,  // real f64 rows -> R2C(nx) -> U
  X_POWERLAW = 1, // U -> C2R(nx) -> e(j) (Eq. 1 / rho_out) -> R2C(nx) -> U
  X_ASSEMBLE = 2, // U -> C2R(nx) -> dh^0 = -c/mu0 on Omega, warm on Omega_out -> Hd[0]; R2C(nx) -> U
  X_MASKPAD = 3,  // U -> C2R(nx) -> chi_Omega * (.) , zero pad -> R2C(2nx) -> Pd
  X_UPDATE = 4,   // Pd -> C2R(2nx), crop -> Eq. 5 update + residual -> Hd[next]; R2C(nx) -> U
  X_TO_F64 = 5,   // U -> C2R(nx) -> real f64 rows
  X_PAD_F64 = 6,  // real f64 rows -> zero pad -> R2C(2nx) -> Pd
  X_CROP_F64 = 7, // Pd -> C2R(2nx), crop -> real f64 rows
  // transposed steps of the fixed-iteration rhs (reverse mode):
  X_ADJ_PAD = 8,      // real f64 rows x (1 - chi) -> zero pad -> R2C(2nx) -> Pd
  X_ADJ_CROP = 9,     // Pd -> C2R(2nx), crop -> x chi -> R2C(nx) -> U
  X_ADJ_COMBINE = 10, // U -> C2R(nx) -> dst = chi * src + (.)   (f64 rows)
  X_ADJ_IN = 11,      // real f64 rows x chi -> R2C(nx) -> U
  X_ADJ_POWERLAW = 12, // U -> C2R(nx) -> lam_e = -(.)/mu0 -> power-law Jacobian^T (forward j in src) -> R2C(nx) -> U;
                       //   dst (N values, optional) = d e/d jc . lam_e
  X_POWERLAW_H = 13,   // as X_POWERLAW with the e(j, h) law of PointParams::law (the state h read from src)
  X_UPDATE_FD = 14     // as X_UPDATE without the R2C of the new iterate (the stencil curl reads it as is)
};

// Scalars of the material law and the Eq. 5 update.
struct PointParams {
  double n;           // power-law exponent
  double e0;          // e0
  double jc;          // uniform jc (used when the map is absent)
  double rho_out;     // Omega_out resistivity
  double inv_mu0;     // 1/mu0
  double hedot[3];    // dh_e/dt at the rhs time
  double tol;         // Eq. 5 stop threshold delta_it * max(|dh_e/dt|, 1)
  double inv_nout;    // 1 / |Omega_out|
  int iter;           // iteration index i (X_UPDATE)
  int max_iter;
  // e(j, h) law in Omega (scfft_set_ej_law): law = 0 is Eq. 1; law = 1 uses
  // jc(h) = jc / (1 + |h| / kim_h0) (kim_h0 > 0) and e = rho(|A j|) A^2 j, A = diag(aniso)
  int law;
  double kim_h0;
  double aniso[3];
};

template <typename T>
struct Launch {
  Geo g;
  Work<T>* w;          // host copy of the workspace pointers
  Ctrl* ctrl;          // device
  const uint8_t* mask; // device [N]
  double* partials;    // device, one double per CTA of the x passes
  PointParams* ppd = nullptr;  // device copy of the current rhs's PointParams (read by the Eq. 5 update pass)
  const PointParams* pps = nullptr;  // device source of that copy (the assembly pass reads it instead of its
                                     // argument when set: rhs parameters computed on the device)
  int* fault = nullptr;        // host: armed one-shot fault injection (scfft_inject_fault), or nullptr
  cudaStream_t st;
  // Support of the source chi_Omega curl dh^i of the Eq. 5 convolution: Omega's bounding box of
  // node rows y in [by0, by1) (even bounds) and planes z in [bz0, bz1).  With use_box set, the
  // FP32 passes that transform that source forward (mask and pad in x, the padded y pass, the
  // padded z pass's input) skip everything outside the box, where it is zero.
  int by0 = 0, by1 = 0, bz0 = 0, bz1 = 0;
  bool use_box = false;
};

// Pass launchers (defined in passes.cu, instantiated for float, double and dfloat).
template <typename T> cudaError_t launch_x(const Launch<T>& L, XMode mode, const PointParams& pp,
                                           const double* src_f64, double* dst_f64, const double* warm,
                                           int in_buf, int out_buf, bool check_done);
// X_PAD_F64 with its real input rows in the pass's own type (FP64 and double-float passes)
template <typename T> cudaError_t launch_x_pad_rows(const Launch<T>& L, const PointParams& pp, const T* rows,
                                                    bool check_done);
template <typename T> cudaError_t launch_y(const Launch<T>& L, bool padded, bool inverse, bool check_done);
template <typename T> cudaError_t launch_z_curl(const Launch<T>& L, bool check_done, double scale);
template <typename T> cudaError_t launch_z_kernel(const Launch<T>& L, bool check_done);
template <typename T> cudaError_t launch_finalize(const Launch<T>& L, double* hdot, double* warm);
template <typename T> cudaError_t launch_kernel_spectrum(const Launch<T>& L, double Lx, double Ly, double Lz,
                                                         double sigma, double* scratch);
template <typename T> cudaError_t launch_convert(const double* src, T* dst, long long n, cudaStream_t st);

// Register-resident FP32 y and z passes (passes_reg.cu); the FP32 path uses these.
cudaError_t launch_y_reg(const Launch<float>& L, bool padded, bool inverse, bool check_done);
// TMA-fed y passes (ypass_tma.cu): descriptors built once per workspace; the launcher returns
// cudaErrorNotSupported when there are none or the length has no instantiation.
bool make_ymaps(Work<float>& w, const Geo& g);
cudaError_t launch_y_tma(const Launch<float>& L, bool padded, bool inverse, bool check_done);
cudaError_t launch_z_reg(const Launch<float>& L, bool padded, bool check_done, double scale);
// The curl's inverse y pass, the mask/pad x pass and the padded forward y pass of an Eq. 5
// iteration (all on Omega's box) as one launch (boxpass.cu); box_fused_ok: the launch applies
// (the box set, nx == ny, a supported length); cudaErrorNotSupported where it does not apply or
// the box's rows do not fit shared memory (the three passes run instead).
bool box_fused_ok(const Launch<float>& L);
cudaError_t launch_box_fused(const Launch<float>& L, bool check_done);

cudaError_t launch_x_reg(const Launch<float>& L, XMode mode, const PointParams& pp, const double* src_f64,
                         double* dst_f64, const double* warm, int in_buf, int out_buf, bool check_done);
// The same with FP32 source rows / FP32 warm start (used by the FP32 integrator's stages).
cudaError_t launch_x_reg_io(const Launch<float>& L, XMode mode, const PointParams& pp, const double* src_f64,
                            const float* src_f32, double* dst_f64, const double* warm, const float* warm_f32,
                            int in_buf, int out_buf, bool check_done);

// Local-stencil curl option (fd_curl.cu): d = cell sizes (dx, dy, dz).
template <typename T> cudaError_t launch_fd_efield(const Launch<T>& L, const PointParams& pp, const double* h64,
                                                   const float* h32, const double* d, T* out);
template <typename T> cudaError_t launch_fd_assemble(const Launch<T>& L, const PointParams& pp, const T* e,
                                                     const double* warm64, const float* warm32, const double* d);
template <typename T> cudaError_t launch_fd_curl_mask(const Launch<T>& L, T* out, const double* d, bool check_done);

// Launch diagnostics: the last failed launch (kernel, grid, block, shared memory).
cudaError_t checked_launch(const char* what, dim3 grid, int block, size_t smem);
const char* last_launch_failure();
// Record the CUDA error behind an SCFFT_ECUDA for scfft_last_cuda_error() (defined in capi.cu).
void note_cuda_error(cudaError_t e, const char* file, int line);

FftPlan make_plan(int L);
bool length_supported(int L);

}  // namespace scfft
