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
// The z passes take the three field components of a column tile through the
// forward transform one after another, apply the spectral curl (i S(k) k x F)
// or the kernel-spectrum product (K^ x F, Eq. 7) on the natural-order spectra
// in shared memory, and transform back, all in one trip through memory.  The
// inverse uses the mirror split
//   y[m1 + R1 m2] = sum_k2 W_R2^{-m2 k2} W_L^{-m1 k2} (sum_k1 X[k2 + R2 k1] W_R1^{-m1 k1}).
#include "scfft_internal.cuh"

namespace scfft {

namespace {

constexpr int kPad8 = 8;  // row padding (complex elements) that spreads half-warps over all banks
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
// 16-byte asynchronous global -> shared copy (L2 only), and the wait for all of this thread's copies
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Tensor memory (TMEM) as per-thread storage.  A warp reaches only the 32 lanes of its quarter
// (warp % 4) of the 128 lanes, one lane per thread, with the 32x32b access shape, so a value
// a thread stores is read back only by that thread.  Allocation is by columns, one warp per
// CTA; every CTA that allocates frees its columns before it exits.
__device__ __forceinline__ void tm_alloc(unsigned* slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"((unsigned)__cvta_generic_to_shared(slot)), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
#define SCFFT_U(v) "r"(__float_as_uint(v))
// store 4 complex (8 columns) of two slots; returns once the stores are complete
__device__ __forceinline__ void tm_st4x2(unsigned ta, const float2* a, unsigned tb, const float2* b) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%10, %11, %12, %13, %14, %15, %16, %17};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(ta), "r"(tb),
      SCFFT_U(a[0].x), SCFFT_U(a[0].y), SCFFT_U(a[1].x), SCFFT_U(a[1].y), SCFFT_U(a[2].x), SCFFT_U(a[2].y),
      SCFFT_U(a[3].x), SCFFT_U(a[3].y), SCFFT_U(b[0].x), SCFFT_U(b[0].y), SCFFT_U(b[1].x), SCFFT_U(b[1].y),
      SCFFT_U(b[2].x), SCFFT_U(b[2].y), SCFFT_U(b[3].x), SCFFT_U(b[3].y)
      : "memory");
}
// store 16 complex (32 columns); returns once the stores are complete
__device__ __forceinline__ void tm_st16(unsigned ta, const float2* a) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(ta),
      SCFFT_U(a[0].x), SCFFT_U(a[0].y), SCFFT_U(a[1].x), SCFFT_U(a[1].y), SCFFT_U(a[2].x), SCFFT_U(a[2].y),
      SCFFT_U(a[3].x), SCFFT_U(a[3].y), SCFFT_U(a[4].x), SCFFT_U(a[4].y), SCFFT_U(a[5].x), SCFFT_U(a[5].y),
      SCFFT_U(a[6].x), SCFFT_U(a[6].y), SCFFT_U(a[7].x), SCFFT_U(a[7].y), SCFFT_U(a[8].x), SCFFT_U(a[8].y),
      SCFFT_U(a[9].x), SCFFT_U(a[9].y), SCFFT_U(a[10].x), SCFFT_U(a[10].y), SCFFT_U(a[11].x), SCFFT_U(a[11].y),
      SCFFT_U(a[12].x), SCFFT_U(a[12].y), SCFFT_U(a[13].x), SCFFT_U(a[13].y), SCFFT_U(a[14].x), SCFFT_U(a[14].y),
      SCFFT_U(a[15].x), SCFFT_U(a[15].y)
      : "memory");
}
#undef SCFFT_U
// load 4 complex of two slots; the values are complete when the call returns
__device__ __forceinline__ void tm_ld4x2(unsigned ta, float2* a, unsigned tb, float2* b) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
    b[i] = make_float2(__uint_as_float(r[8 + 2 * i]), __uint_as_float(r[8 + 2 * i + 1]));
  }
}
// load 16 complex (32 columns); the values are complete when the call returns
__device__ __forceinline__ void tm_ld16(unsigned ta, float2* a) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
}

template <typename V> __device__ __forceinline__ V tw_mul(V a, V w, bool inv) { return inv ? cmulc(a, w) : cmul(a, w); }

template <typename V> __device__ __forceinline__ V zero_v();
template <> __device__ __forceinline__ float2 zero_v<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_v<double2>() { return make_double2(0.0, 0.0); }

}  // namespace

// ---------------------------------------------------------------- y pass
// grid (ceil(HX/TC), planes, 3), block TC*R1 threads; the planes are z = zoff + blockIdx.y.  Rows
// outside [ylo, yhi): the forward pass reads them as zero (a source that vanishes outside
// Omega's box), the inverse pass does not write them (nothing downstream reads them).
template <typename T, int R1, int R2, int TC, bool INV, bool PIN, bool POUT>
__global__ void __launch_bounds__(TC * R1) ypass_reg_kernel(typename cplx_of<T>::type* __restrict__ base, int rows,
                                                            int sx, int HX, int nzs,
                                                            const typename cplx_of<T>::type* __restrict__ twg,
                                                            const Ctrl* ctrl, int check_done, int ahead, int zoff,
                                                            int ylo, int yhi) {
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
  const int cz = blockIdx.z, z = zoff + blockIdx.y, kx = blockIdx.x * TC + c;
  const bool colok = kx < HX;
  V* col = base + ((size_t)(cz * nzs + z) * rows) * sx + kx;
  if (ahead > 0) {  // prefetch into L2 the input columns of the CTA one wave of resident CTAs later
    const int gx = gridDim.x, gy = gridDim.y;
    const int nb = blockIdx.x + gx * (blockIdx.y + gy * blockIdx.z) + ahead;
    if (nb < gx * gy * (int)gridDim.z) {
      const int bx = nb % gx, zz = zoff + (nb / gx) % gy, cc = nb / (gx * gy);
      const V* ncol = base + ((size_t)(cc * nzs + zz) * rows) * sx + bx * TC;
      constexpr int NR = PIN ? L / 2 : L;
      const int last = (bx * TC + TC <= HX ? TC : HX - bx * TC) - 1;
      for (int i = t; i < 2 * NR; i += TC * R1) prefetch_l2(ncol + (size_t)(i >> 1) * sx + ((i & 1) ? last : 0));
    }
  }
  V v[R2];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    if (PIN && n2 >= R2 / 2) {
      v[n2] = zero_v<V>();
    } else {
      const int row = n1 + R1 * n2;
      v[n2] = (colok && (INV || (row >= ylo && row < yhi))) ? col[(size_t)row * sx] : zero_v<V>();
    }
  }
  __syncthreads();  // twiddles staged
  dft_maybe_half<R2, INV, PIN>(v);
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
        if (INV && (k2 + R2 * k1 < ylo || k2 + R2 * k1 >= yhi)) continue;
        col[(size_t)(k2 + R2 * k1) * sx] = w[k1];
      }
    }
  }
}

template <int R1, int R2, int TC, int KIND>
__global__ void zpass_reg2_kernel(float2* __restrict__ base, int rows, int sx, int HX, int nzs,
                                  const float2* __restrict__ twg, const float* __restrict__ kt0,
                                  const float* __restrict__ kt1, const float* __restrict__ kt2,
                                  const float* __restrict__ st0, const float* __restrict__ st1,
                                  const float* __restrict__ st2, float scale, const float4* __restrict__ kap4, int nx,
                                  int ny, int nz, const Ctrl* ctrl, int check_done, int zlo, int zhi);

template <int TC>
__global__ void zpass_tm2_kernel(float2* __restrict__ base, int rows, int sx, int HX, int nzs,
                                 const float2* __restrict__ twg, const float4* __restrict__ kap4, int nx, int ny,
                                 int nz, const Ctrl* ctrl, int check_done, int zlo, int zhi);

// ---------------------------------------------------------------- launchers
namespace {

// PF: prefetch the next wave's input columns into L2 (measured faster on the padded passes,
// slower on the unpadded ones, which also run narrower CTAs)
template <int R1, int R2, int TC, bool INV, bool PIN, bool POUT, bool PF>
cudaError_t go_y(const Launch<float>& L, float2* base, int rows, int sx, int HX, const float2* tw, bool chk) {
  constexpr int Lt = R1 * R2;
  const size_t smem = sizeof(float2) * (Lt + R2 * (R1 * TC + kPad8));
  auto k = ypass_reg_kernel<float, R1, R2, TC, INV, PIN, POUT>;
  allow_smem<ypass_reg_kernel<float, R1, R2, TC, INV, PIN, POUT>>();
  // the padded forward pass and the curl's unpadded inverse pass of an Eq. 5 iteration: only
  // the planes and rows of Omega's box
  const bool box = L.use_box && (PIN || (INV && !POUT));
  dim3 grid((HX + TC - 1) / TC, box ? L.bz1 - L.bz0 : L.g.nz, 3);
  static const int resident = [&] {  // CTAs resident at once: the prefetch distance
    if (!PF) return 0;
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, TC * R1, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm > 0 && sms > 0 ? per_sm * sms : 0;
  }();
  k<<<grid, TC * R1, smem, L.st>>>(base, rows, sx, HX, L.g.nz, tw, L.ctrl, chk ? 1 : 0, resident, box ? L.bz0 : 0,
                                   box ? L.by0 : 0, box ? L.by1 : rows);
  return cudaGetLastError();
}

template <int R1, int R2, int TC, int KIND>
cudaError_t go_z(const Launch<float>& L, float2* base, int rows, int sx, int HX, const float2* tw, double scale,
                 bool chk) {
  constexpr int Lt = R1 * R2;
  constexpr int CS = (R1 == R2 && KIND >= 1) ? cmax(R2 * (R1 * TC + kPad8), R1 * (R2 * TC + kPad8))
                               : cmax(cmax(R2 * (R1 * TC + kPad8), R1 * (R2 * TC + kPad8)), Lt * TC);
  // (the own-slot form stages K^ in component 2's buffer once the forward transforms are done)
  const size_t smem = sizeof(float2) * (Lt + 3 * CS);
  static_assert((Lt + 2 * CS) % 2 == 0, "16-byte alignment of the staged kernel spectrum");
  auto k = zpass_reg2_kernel<R1, R2, TC, KIND>;
  allow_smem<zpass_reg2_kernel<R1, R2, TC, KIND>>();
  constexpr bool PACK = (R1 == R2 && KIND >= 1);  // as in the kernel's column map
  if (KIND >= 1 && Lt != 2 * L.g.nz) return cudaErrorInvalidValue;  // the padded pass folds kz about Lt/2
  const int nfull = HX / TC, rem = HX - nfull * TC;
  const dim3 grid = PACK ? dim3(nfull * rows + (rows * rem + TC - 1) / TC, 1, 1) : dim3((HX + TC - 1) / TC, rows, 1);
  const Work<float>& w = *L.w;
  // box: the padded pass's input planes, or the curl pass's output planes (both Omega's box)
  const bool box = L.use_box;
  k<<<grid, TC * R1, smem, L.st>>>(base, rows, sx, HX, L.g.nz, tw, w.kt[0], w.kt[1], w.kt[2], w.st[0], w.st[1],
                                   w.st[2], (float)scale, w.kap4, L.g.nx, L.g.ny, L.g.nz, L.ctrl, chk ? 1 : 0,
                                   box ? L.bz0 : 0, box ? L.bz1 : Lt);
  return cudaGetLastError();
}

// The two-buffer tensor-memory form of the padded z pass (256-point z transforms only).
template <int TC> cudaError_t go_z_tm2(const Launch<float>& L, bool chk) {
  constexpr int Lt = 256, CS = 16 * (16 * TC + kPad8);
  const size_t smem = sizeof(float2) * (Lt + 2 * CS);
  auto k = zpass_tm2_kernel<TC>;
  allow_smem<zpass_tm2_kernel<TC>>();
  const Geo& g = L.g;
  if (2 * g.nz != Lt) return cudaErrorInvalidValue;
  const int rows = 2 * g.ny, HX = g.nx + 1;
  const int nfull = HX / TC, rem = HX - nfull * TC;
  const dim3 grid(nfull * rows + (rows * rem + TC - 1) / TC, 1, 1);
  const bool box = L.use_box;
  k<<<grid, TC * 16, smem, L.st>>>(L.w->Pd, rows, g.sxp, HX, g.nz, L.w->twp[2], L.w->kap4, g.nx, g.ny, g.nz, L.ctrl,
                                   chk ? 1 : 0, box ? L.bz0 : 0, box ? L.bz1 : Lt);
  return checked_launch("zpass_tm2_kernel", grid, TC * 16, smem);
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

// (the column tiles TC of the unpadded y passes and of both z passes follow the context's
// schedule, Sched; the tile changes which CTA holds a column, not the column's arithmetic)
template <int R1, int R2> struct YFwdU {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    if (L.w->sched.yu_tc == 16)
      return go_y<R1, R2, 16, false, false, false, false>(L, L.w->U, g.ny, g.sxu, g.nx / 2 + 1, L.w->twu[1], chk);
    return go_y<R1, R2, 8, false, false, false, false>(L, L.w->U, g.ny, g.sxu, g.nx / 2 + 1, L.w->twu[1], chk);
  }
};
template <int R1, int R2> struct YInvU {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    if (L.w->sched.yu_tc == 16)
      return go_y<R1, R2, 16, true, false, false, false>(L, L.w->U, g.ny, g.sxu, g.nx / 2 + 1, L.w->twu[1], chk);
    return go_y<R1, R2, 8, true, false, false, false>(L, L.w->U, g.ny, g.sxu, g.nx / 2 + 1, L.w->twu[1], chk);
  }
};
template <int R1, int R2> struct YFwdP {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    return go_y<R1, R2, 16, false, true, false, true>(L, L.w->Pd, 2 * g.ny, g.sxp, g.nx + 1, L.w->twp[1], chk);
  }
};
template <int R1, int R2> struct YInvP {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    return go_y<R1, R2, 16, true, false, true, true>(L, L.w->Pd, 2 * g.ny, g.sxp, g.nx + 1, L.w->twp[1], chk);
  }
};
template <int R1, int R2> struct ZCurl {
  static cudaError_t run(const Launch<float>& L, bool chk, double scale) {
    const Geo& g = L.g;
    if (L.w->sched.zc_tc == 16)
      return go_z<R1, R2, 16, 0>(L, L.w->U, g.ny, g.sxu, g.nx / 2 + 1, L.w->twu[2], scale, chk);
    return go_z<R1, R2, 8, 0>(L, L.w->U, g.ny, g.sxu, g.nx / 2 + 1, L.w->twu[2], scale, chk);
  }
};
template <int R1, int R2> struct ZKern {
  static cudaError_t run(const Launch<float>& L, bool chk) {
    const Geo& g = L.g;
    // the tensor-memory form of the own-slot product exists for the 16 x 16 split (L = 256)
    if constexpr (R1 == 16 && R2 == 16) {
      if (L.w->sched.zk_tm == 2) return L.w->sched.zk_tc == 4 ? go_z_tm2<4>(L, chk) : go_z_tm2<8>(L, chk);
      if (L.w->sched.zk_tm) {
        if (L.w->sched.zk_tc == 4)
          return go_z<R1, R2, 4, 2>(L, L.w->Pd, 2 * g.ny, g.sxp, g.nx + 1, L.w->twp[2], 1.0, chk);
        return go_z<R1, R2, 8, 2>(L, L.w->Pd, 2 * g.ny, g.sxp, g.nx + 1, L.w->twp[2], 1.0, chk);
      }
    }
    if (L.w->sched.zk_tc == 4)
      return go_z<R1, R2, 4, 1>(L, L.w->Pd, 2 * g.ny, g.sxp, g.nx + 1, L.w->twp[2], 1.0, chk);
    return go_z<R1, R2, 8, 1>(L, L.w->Pd, 2 * g.ny, g.sxp, g.nx + 1, L.w->twp[2], 1.0, chk);
  }
};

}  // namespace

cudaError_t launch_y_reg(const Launch<float>& L, bool padded, bool inverse, bool check_done) {
  if (L.w->ym && L.w->sched.yp_tma) {
    const cudaError_t e = launch_y_tma(L, padded, inverse, check_done);
    if (e != cudaErrorNotSupported) return e;
  }
  const int Ly = padded ? 2 * L.g.ny : L.g.ny;
  if (!padded) return inverse ? by_length<YInvU>(Ly, L, check_done) : by_length<YFwdU>(Ly, L, check_done);
  return inverse ? by_length<YInvP>(Ly, L, check_done) : by_length<YFwdP>(Ly, L, check_done);
}

cudaError_t launch_z_reg(const Launch<float>& L, bool padded, bool check_done, double scale) {
  if (!padded) return by_length<ZCurl>(L.g.nz, L, check_done, scale);
  return by_length<ZKern>(2 * L.g.nz, L, check_done);
}

}  // namespace scfft

// ============================================================================
// x passes (FP32): C2R of a half-spectrum row pair, the node-wise step, R2C.
//
// Two real rows a, b of one component travel as z = a + i b.  The C2R of
// length Li = R1i R2i leaves thread (p, k2) with z at x = k2 + R2i k1; with
// the R2C split R1o = R2i those are exactly the inputs n1' + R1o n2' (n1' = k2,
// n2' = k1) of the forward transform of length Lo = R1o R2o, so the node-wise
// step and the R2C start from the C2R's registers.  A last pass through
// shared memory pairs Z[k] with Z[Lo-k] to separate the two rows' spectra.
// ============================================================================
namespace scfft {

struct XRArgs {
  Geo g;
  const float2* spec_in;
  int in_rows, in_sx;
  float2* spec_out;
  int out_rows, out_sx;
  const float2* tw_in;
  const float2* tw_out;
  const double* src_f64;
  const float* src_f32;   // FP32 source rows instead of src_f64 (integrator stages)
  double* dst_f64;
  const double* warm;
  const float* warm_f32;  // FP32 warm start instead of warm
  const uint8_t* mask;
  const float* jc;
  const float* hold;
  float* hnew;
  float* hbuf[2];         // both iterate buffers: the update pass picks by the device iteration count
  PointParams pp;
  PointParams* ppd;       // device copy of pp (written by the assemble pass, read by the update pass)
  const PointParams* pps; // device source of that copy, or nullptr (pp is copied)
  Ctrl* ctrl;
  double* partials;
  int check_done;
  int out_buf;
  // mask/pad pass of an Eq. 5 iteration: only the row pairs of Omega's box (y in [by0, by1),
  // z in [bz0, bz1)); the rows outside hold zeros of the source and are not read downstream
  int use_box, by0, by1, bz0, bz1;
  // mask/pad pass: each work item is one component of a tile (the components are independent
  // in this mode), three times the parallelism of a tile of all three
  int comp_split;
};

namespace {

// (z, y) of the first row of row pair gp, over every pair of the grid or over the box's
__device__ __forceinline__ void pair_rows(const XRArgs& a, int gp, int& z, int& y) {
  if (a.use_box) {
    const int hp = (a.by1 - a.by0) >> 1, zb = gp / hp;
    z = a.bz0 + zb;
    y = a.by0 + 2 * (gp - zb * hp);
  } else {
    const int q = 2 * gp;
    z = q / a.g.ny;
    y = q - z * a.g.ny;
  }
}
__host__ __device__ __forceinline__ int pair_count(const XRArgs& a) {
  return a.use_box ? (a.bz1 - a.bz0) * ((a.by1 - a.by0) >> 1) : a.g.ny * a.g.nz / 2;
}


template <int MODE, int R1i, int R2i, int R2o> struct XS {
  static constexpr bool C2R = !(MODE == X_FWD_F64 || MODE == X_PAD_F64);
  static constexpr bool R2C = !(MODE == X_TO_F64 || MODE == X_CROP_F64 || MODE == X_UPDATE_FD);
  static constexpr bool PADIN = (MODE == X_UPDATE || MODE == X_UPDATE_FD || MODE == X_CROP_F64);  // C2R length 2nx, keep x < nx
  static constexpr bool PADOUT = (MODE == X_MASKPAD || MODE == X_PAD_F64);  // R2C length 2nx, input x < nx
  static constexpr int R1o = R2i;
  static constexpr int Li = R1i * R2i;
  static constexpr int Lo = R1o * R2o;
  // threads per row pair: a power of two, so that a pair's threads are lanes of one warp
  static constexpr int TP0 = cmax(cmax(R1i, R2i), R2o);
  static constexpr int TP = TP0 <= 4 ? 4 : TP0 <= 8 ? 8 : 16;
  static constexpr int KX = PADIN ? R1i / 2 : R1i;  // k1 slots that hold x < nx after the C2R
};

__device__ __forceinline__ float rho_of(float jx, float jy, float jz, bool in, float jcv, const PointParams& pp) {
  if (!in) return (float)pp.rho_out;
  const float jn = sqrtf(jx * jx + jy * jy + jz * jz);
  const float n = (float)pp.n, e0 = (float)pp.e0;
  if (jn == 0.f) return n == 1.f ? e0 / jcv : 0.f;
  return (e0 / jcv) * exp2f((n - 1.f) * log2f(jn / jcv));
}

// the e(j, h) law (PointParams::law): jc(h) = jc / (1 + |h| / h0), e = rho(|A j|) A^2 j; returns
// the factors f_a with e_a = f_a j_a
__device__ __forceinline__ void law_factors(float jx, float jy, float jz, bool in, float jcv, float hx, float hy,
                                            float hz, const PointParams& pp, float f[3]) {
  if (!in) {
    f[0] = f[1] = f[2] = (float)pp.rho_out;
    return;
  }
  if (pp.kim_h0 > 0) jcv = jcv / (1.f + sqrtf(hx * hx + hy * hy + hz * hz) / (float)pp.kim_h0);
  const float ax = (float)pp.aniso[0], ay = (float)pp.aniso[1], az = (float)pp.aniso[2];
  const float r = rho_of(ax * jx, ay * jy, az * jz, true, jcv, pp);
  f[0] = r * ax * ax;
  f[1] = r * ay * ay;
  f[2] = r * az * az;
}

}  // namespace

template <int MODE, int R1i, int R2i, int R2o, int P>
__global__ void xpass_reg2_kernel(const XRArgs a);
template <int R1i, int R2i, int R2o, int P>
__global__ void xupdate3_kernel(const XRArgs a);

namespace {

constexpr int kPairs = 8;  // row pairs per CTA (x 3 components)

template <int MODE, int R1i, int R2i, int R2o>
cudaError_t go_x(const XRArgs& a, cudaStream_t st) {
  typedef XS<MODE, R1i, R2i, R2o> S;
  constexpr int XL = S::C2R ? (S::PADIN ? S::Li / 2 : S::Li) : (S::PADOUT ? S::Lo / 2 : S::Lo);
  constexpr int TT = cmax(cmax(S::C2R ? R2i * (R1i + 1) : 1, S::R2C ? R2o * (S::R1o + 1) : 1), S::R2C ? S::Lo : 1);
  const size_t smem =
      sizeof(float2) * ((S::Li > 0 ? S::Li : 1) + (S::Lo > 0 ? S::Lo : 1) + 3 * kPairs * XL + kPairs * TT);
  auto k = xpass_reg2_kernel<MODE, R1i, R2i, R2o, kPairs>;
  allow_smem<xpass_reg2_kernel<MODE, R1i, R2i, R2o, kPairs>>();
  const int npairs = pair_count(a);
  const int ntiles = (npairs + kPairs - 1) / kPairs * ((MODE == X_MASKPAD && a.comp_split) ? 3 : 1);
  // one wave of resident CTAs (the kernel loops over tiles)
  static const int resident = [&] {
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kPairs * S::TP, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm > 0 && sms > 0 ? per_sm * sms : 1024;
  }();
  const int grid = ntiles < resident ? ntiles : resident;
  k<<<grid, kPairs * S::TP, smem, st>>>(a);
  return checked_launch("xpass_reg2_kernel", dim3(grid), kPairs * S::TP, smem);
}

constexpr int kPairs3 = 8;  // row pairs per tile of the three-group update pass (x 3 components; 4 measured slower)

template <int R1i, int R2i, int R2o>
cudaError_t go_xu3(const XRArgs& a, cudaStream_t st) {
  typedef XS<X_UPDATE, R1i, R2i, R2o> S;
  constexpr int XL = S::Li / 2;
  constexpr int TT = cmax(cmax(R2i * (R1i + 1), R2o * (S::R1o + 1)), S::Lo);
  constexpr int NT = 3 * kPairs3 * S::TP;
  const size_t smem = sizeof(float2) * (S::Li + S::Lo + 3 * kPairs3 * XL + 3 * kPairs3 * TT);
  auto k = xupdate3_kernel<R1i, R2i, R2o, kPairs3>;
  allow_smem<xupdate3_kernel<R1i, R2i, R2o, kPairs3>>();
  const int ntiles = (pair_count(a) + kPairs3 - 1) / kPairs3;
  static const int resident = [&] {
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm > 0 && sms > 0 ? per_sm * sms : 1024;
  }();
  const int grid = ntiles < resident ? ntiles : resident;
  k<<<grid, NT, smem, st>>>(a);
  return checked_launch("xupdate3_kernel", dim3(grid), NT, smem);
}

// Splits per unpadded length n: C2R(n) = (a, b), C2R(2n) = (c, d); the R2C
// splits follow from R1o = R2i (see the section comment).
template <int MODE> cudaError_t go_x_n(int n, const XRArgs& a, cudaStream_t st, bool split3 = false) {
#define XN(NN, A_, B_, C_, D_)                                                                   \
  case NN:                                                                                       \
    if constexpr (MODE == X_UPDATE) if (split3) return go_xu3<C_, D_, C_ / 2>(a, st);            \
    if constexpr (MODE == X_FWD_F64) return go_x<MODE, 1, B_, A_>(a, st);                        \
    else if constexpr (MODE == X_PAD_F64) return go_x<MODE, 1, B_, 2 * A_>(a, st);               \
    else if constexpr (MODE == X_POWERLAW || MODE == X_POWERLAW_H || MODE == X_ASSEMBLE) return go_x<MODE, A_, B_, A_>(a, st); \
    else if constexpr (MODE == X_MASKPAD) return go_x<MODE, A_, B_, 2 * A_>(a, st);              \
    else if constexpr (MODE == X_TO_F64) return go_x<MODE, A_, B_, 1>(a, st);                    \
    else if constexpr (MODE == X_UPDATE) return go_x<MODE, C_, D_, C_ / 2>(a, st);               \
    else if constexpr (MODE == X_UPDATE_FD) return go_x<MODE, C_, D_, 1>(a, st);                 \
    else return go_x<MODE, C_, D_, 1>(a, st);
  switch (n) {
    XN(16, 4, 4, 8, 4)
    XN(32, 4, 8, 8, 8)
    XN(48, 4, 12, 8, 12)
    XN(64, 4, 16, 8, 16)
    XN(96, 8, 12, 16, 12)
    XN(128, 8, 16, 16, 16)
  }
#undef XN
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_x_reg(const Launch<float>& L, XMode mode, const PointParams& pp, const double* src_f64,
                         double* dst_f64, const double* warm, int in_buf, int out_buf, bool check_done) {
  return launch_x_reg_io(L, mode, pp, src_f64, nullptr, dst_f64, warm, nullptr, in_buf, out_buf, check_done);
}

cudaError_t launch_x_reg_io(const Launch<float>& L, XMode mode, const PointParams& pp, const double* src_f64,
                            const float* src_f32, double* dst_f64, const double* warm, const float* warm_f32,
                            int in_buf, int out_buf, bool check_done) {
  const Geo& g = L.g;
  XRArgs a{};
  a.g = g;
  const bool pin = (mode == X_UPDATE || mode == X_UPDATE_FD || mode == X_CROP_F64);
  const bool pout = (mode == X_MASKPAD || mode == X_PAD_F64);
  a.spec_in = pin ? L.w->Pd : L.w->U;
  a.in_rows = pin ? 2 * g.ny : g.ny;
  a.in_sx = pin ? g.sxp : g.sxu;
  a.spec_out = pout ? L.w->Pd : L.w->U;
  a.out_rows = pout ? 2 * g.ny : g.ny;
  a.out_sx = pout ? g.sxp : g.sxu;
  a.tw_in = pin ? L.w->twp[0] : L.w->twu[0];
  a.tw_out = pout ? L.w->twp[0] : L.w->twu[0];
  a.src_f64 = src_f64;
  a.src_f32 = src_f32;
  a.dst_f64 = dst_f64;
  a.warm = warm;
  a.warm_f32 = warm_f32;
  a.mask = L.mask;
  a.jc = L.w->jc;
  a.hold = L.w->Hd[in_buf];
  a.hnew = L.w->Hd[out_buf];
  a.hbuf[0] = L.w->Hd[0];
  a.hbuf[1] = L.w->Hd[1];
  a.pp = pp;
  a.ppd = L.ppd;
  a.pps = L.pps;
  a.ctrl = L.ctrl;
  a.partials = L.partials;
  a.check_done = check_done ? 1 : 0;
  a.out_buf = out_buf;
  a.use_box = (L.use_box && mode == X_MASKPAD) ? 1 : 0;
  a.comp_split = a.use_box;  // the mask/pad pass of an Eq. 5 iteration: one wave of small work
  a.by0 = L.by0;
  a.by1 = L.by1;
  a.bz0 = L.bz0;
  a.bz1 = L.bz1;
  switch (mode) {
    case X_FWD_F64: return go_x_n<X_FWD_F64>(g.nx, a, L.st);
    case X_POWERLAW: return go_x_n<X_POWERLAW>(g.nx, a, L.st);
    case X_POWERLAW_H: return go_x_n<X_POWERLAW_H>(g.nx, a, L.st);
    case X_ASSEMBLE: return go_x_n<X_ASSEMBLE>(g.nx, a, L.st);
    case X_MASKPAD: return go_x_n<X_MASKPAD>(g.nx, a, L.st);
    case X_UPDATE: return go_x_n<X_UPDATE>(g.nx, a, L.st, L.w->sched.xu3 != 0);
    case X_UPDATE_FD: return go_x_n<X_UPDATE_FD>(g.nx, a, L.st);
    case X_TO_F64: return go_x_n<X_TO_F64>(g.nx, a, L.st);
    case X_PAD_F64: return go_x_n<X_PAD_F64>(g.nx, a, L.st);
    case X_CROP_F64: return go_x_n<X_CROP_F64>(g.nx, a, L.st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace scfft

// ============================================================================
// Lower-register variants: the three components go through the FFT stages one
// after another (16 complex values per thread at a time), and the
// cross-component steps (curl / kernel-spectrum product in z, the node-wise
// step in x) read all three from shared memory.  This doubles the resident
// warps per SM of the 3-component register versions above.
// ============================================================================
namespace scfft {

template <int R1, int R2, int TC, int KIND>
__global__ void __launch_bounds__(TC * R1, (R1 == R2 && KIND >= 1) ? 4 : 1) zpass_reg2_kernel(float2* __restrict__ base, int rows, int sx, int HX,
                                                             int nzs, const float2* __restrict__ twg,
                                                             const float* __restrict__ kt0,
                                                             const float* __restrict__ kt1,
                                                             const float* __restrict__ kt2,
                                                             const float* __restrict__ st0,
                                                             const float* __restrict__ st1,
                                                             const float* __restrict__ st2, float scale,
                                                             const float4* __restrict__ kap4, int nx, int ny, int nz,
                                                             const Ctrl* ctrl, int check_done, int zlo, int zhi) {
  constexpr int L = R1 * R2;
  constexpr bool PR = (KIND >= 1);
  // KIND 2: the own-slot spectra of components 0 and 1 live in tensor memory instead of
  // shared memory (the same arithmetic in the same order, so the same bits as KIND 1)
  constexpr bool TM = (KIND == 2);
  constexpr int S2 = R1 * TC + kPad8;  // forward transpose [k2][n1][c]
  constexpr int S1 = R2 * TC + kPad8;  // inverse transpose [m1][k2][c]
  constexpr bool OWN = (R1 == R2 && KIND >= 1);  // own-slot product (square split, Biot-Savart kernel)
  static_assert(!TM || (OWN && R1 == 16), "tensor-memory spectra: the own-slot form of the 16 x 16 split");
  constexpr int CS = OWN ? cmax(R2 * S2, R1 * S1) : cmax(cmax(R2 * S2, R1 * S1), L * TC);
  constexpr int NT = TC * R1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (check_done && ctrl->done) return;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* F = tw + L;
  const int t = threadIdx.x;
  for (int i = t; i < L; i += NT) tw[i] = twg[i];
  const int c = t % TC, n1 = t / TC;
  // Column map.  The curl's pass: grid (ceil(HX / TC), rows), TC consecutive kx of row y per
  // CTA.  The padded pass: a 1-D grid whose regular CTAs take TC consecutive kx of one row;
  // the kx left over when HX is not a multiple of TC (the Nyquist column kx = HX - 1 of the
  // half spectrum) are packed TC (row, kx) pairs to a CTA and run first, so no CTA runs
  // mostly empty columns (packing measured slower in the curl's pass).
  constexpr bool PACK = OWN;
  int y, kx;
  bool colok;
  if constexpr (PACK) {
    const int nfull = HX / TC, rem = HX - nfull * TC;
    const int ntail = (rows * rem + TC - 1) / TC;
    const int b = blockIdx.x;
    if (b >= ntail) {
      y = (b - ntail) / nfull;
      kx = (b - ntail - y * nfull) * TC + c;
      colok = true;
    } else {
      const int e = b * TC + c;
      colok = e < rows * rem;
      y = colok ? e / rem : 0;
      kx = colok ? nfull * TC + (e - y * rem) : 0;
    }
  } else {
    y = blockIdx.y;
    kx = blockIdx.x * TC + c;
    colok = kx < HX;
  }
  const size_t zstride = (size_t)rows * sx;
  const size_t cstride = (size_t)nzs * zstride;
  float2* col = base + (size_t)y * sx + kx;
  // (an L2 prefetch of the input columns of the CTA one wave later paid at three CTAs per SM;
  // at four it measured 2% slower and is gone)
  // KIND 2: 64 tensor-memory columns per CTA, 16 complex of component 0 at columns 0-31 and of
  // component 1 at 32-63 in each thread's lane (at most eight CTAs of this kernel fit an SM by
  // registers, so the 512 columns of an SM always suffice)
  __shared__ unsigned tm_slot;
  if constexpr (TM) {
    if (t < 32) tm_alloc(&tm_slot, 64u);
    tm_fence_before();
  }
  __syncthreads();  // twiddles staged (and the tensor-memory address published)
  unsigned tmq = 0;  // this thread's lane of the allocation
  if constexpr (TM) {
    tm_fence_after();
    tmq = tm_slot + ((unsigned)(32 * ((t >> 5) & 3)) << 16);
  }
  // This thread's twiddles W_L^{n1 j}: stage A uses j = k2 with its own n1, and
  // stage A' (run by the thread whose k2 equals this n1) uses j = m1, so one set
  // of registers serves both directions for all three components.
  constexpr int TJ = cmax(R1, R2);
  float2 twr[TJ];
#pragma unroll
  for (int jj = 0; jj < TJ; ++jj) twr[jj] = tw[(n1 * jj) % L];

  // all three components' inputs are loaded up front (one memory latency, not three)
  constexpr int NL = PR ? R2 / 2 : R2;
  float2 pre[3][NL];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int n2 = 0; n2 < NL; ++n2)
      // (input planes outside [zlo, zhi) are zero: the source vanishes outside Omega's box)
      pre[q][n2] = (colok && (!PR || (n1 + R1 * n2 >= zlo && n1 + R1 * n2 < zhi)))
                       ? col[q * cstride + (size_t)(n1 + R1 * n2) * zstride]
                       : make_float2(0.f, 0.f);
  if constexpr (OWN) {
    // Forward, one component at a time.  In stage B the thread (c, k2 = n1 < R2) reads the
    // slots Fq[k2 S2 + m TC + c] that no other thread reads, so it writes its spectrum
    // X_q[k2 + R2 k1] back into those same slots without a barrier ("own slots"); the
    // last component's spectrum stays in registers.
    float2 w2[R1];
    // This column's kernel spectrum K^(kx, fy, fz), fz = 0..nz (the fold of kz, which halves the
    // reads), is copied with 16-byte cp.async into Ks[fz][c]: in component 2's buffer once every
    // thread has read it (shared-memory spectra), or (tensor-memory spectra) in component 0's
    // buffer, free once component 0's spectrum has gone to tensor memory, so that the copy runs
    // during component 1's and 2's transforms.
    float4* Ks = reinterpret_cast<float4*>(F + (TM ? 0 : 2) * CS);
    static_assert(CS * sizeof(float2) >= (L / 2 + 1) * TC * sizeof(float4), "K^ fits a component's buffer");
    auto copy_kernel_spectrum = [&] {
      const int fy = (y <= ny) ? y : 2 * ny - y;
      const size_t plane = (size_t)(ny + 1) * (nx + 1);
      const float4* src = kap4 + (size_t)fy * (nx + 1) + (colok ? kx : 0);
      for (int fz = n1; fz <= L / 2; fz += R1) cp_async16(Ks + fz * TC + c, src + fz * plane);
    };
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float2* Fq = F + q * CS;
      float2 v[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) v[n2] = n2 < NL ? pre[q][n2] : make_float2(0.f, 0.f);
      dft_maybe_half<R2, false, PR>(v);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) Fq[k2 * S2 + n1 * TC + c] = k2 == 0 ? v[0] : cmul(v[k2], twr[k2]);
      __syncthreads();
      // (past this barrier every thread has moved component 0's spectrum to tensor memory)
      if (TM && q == 1) copy_kernel_spectrum();
      if (n1 < R2) {
        float2 w[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) w[m] = Fq[n1 * S2 + m * TC + c];
        DFT<R1, false, float2>::run(w);
        if (TM && q < 2) {
          tm_st16(tmq + 32u * q, w);
        } else {
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) {
            if (q < 2)
              Fq[n1 * S2 + k1 * TC + c] = w[k1];
            else
              w2[k1] = w[k1];
          }
        }
      }
    }
    // Keeping K^ out of a buffer of its own (as when it was copied during the forward transforms)
    // leaves 53 KB per CTA, so four CTAs fit per SM (128 registers): measured 5% faster.
    if constexpr (!TM) {
      __syncthreads();  // component 2's buffer read by all
      copy_kernel_spectrum();
    }
    cp_async_wait_all();
    __syncthreads();  // Ks complete and visible
    // ---- product at kz = k2 + R2 k1 on the thread's own points; components 0, 1 from
    // their own slots, component 2 in registers.  K^ is odd in ky (component y) and in kz
    // (component z) about the fold.
    if (n1 < R2) {
      const int k2 = n1;
      const float syg = (y <= ny) ? 1.f : -1.f;
      float2* F0 = F + k2 * S2 + c;
      float2* F1 = F0 + CS;
      if constexpr (TM) {
        // four points of components 0 and 1 per tensor-memory load and store
#pragma unroll
        for (int b = 0; b < R1 / 4; ++b) {
          float2 g0[4], g1[4];
          tm_ld4x2(tmq + 8u * b, g0, tmq + 32u + 8u * b, g1);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k1 = 4 * b + i;
            const int kz = k2 + R2 * k1;
            const int fz = (kz <= L / 2) ? kz : L - kz;
            const float4 K = Ks[fz * TC + c];
            const float ax = K.x, ay = syg * K.y, az = (kz <= L / 2) ? K.z : -K.z;
            const float2 G0 = g0[i], G1 = g1[i], G2 = w2[k1];
            const float2 cx = make_float2(ay * G2.x - az * G1.x, ay * G2.y - az * G1.y);
            const float2 cy = make_float2(az * G0.x - ax * G2.x, az * G0.y - ax * G2.y);
            const float2 cz = make_float2(ax * G1.x - ay * G0.x, ax * G1.y - ay * G0.y);
            g0[i] = make_float2(-cx.y, cx.x);
            g1[i] = make_float2(-cy.y, cy.x);
            w2[k1] = make_float2(-cz.y, cz.x);
          }
          tm_st4x2(tmq + 8u * b, g0, tmq + 32u + 8u * b, g1);
        }
      } else {
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
          const int kz = k2 + R2 * k1;
          const int fz = (kz <= L / 2) ? kz : L - kz;  // L = 2 nz: a constant, so most folds resolve at compile time
          const float4 K = Ks[fz * TC + c];
          const float ax = K.x, ay = syg * K.y, az = (kz <= L / 2) ? K.z : -K.z;
          const float2 G0 = F0[k1 * TC], G1 = F1[k1 * TC], G2 = w2[k1];
          const float2 cx = make_float2(ay * G2.x - az * G1.x, ay * G2.y - az * G1.y);
          const float2 cy = make_float2(az * G0.x - ax * G2.x, az * G0.y - ax * G2.y);
          const float2 cz = make_float2(ax * G1.x - ay * G0.x, ax * G1.y - ay * G0.y);
          F0[k1 * TC] = make_float2(-cx.y, cx.x);
          F1[k1 * TC] = make_float2(-cy.y, cy.x);
          w2[k1] = make_float2(-cz.y, cz.x);
        }
      }
    }
    // ---- inverse: y[m1 + R1 m2] = sum_k2 W_R2^{-m2 k2} W_L^{-m1 k2} (sum_k1 X[k2 + R2 k1] W_R1^{-m1 k1}).
    // Stage A' of component q writes transposed into buffer q once every thread has read
    // that buffer's own slots: component 2 (in registers) right after the first barrier,
    // component 0 after the next, component 1 after the one after.
    __syncthreads();
    float2 wr[R1];
#pragma unroll
    for (int q = 2; q < 5; ++q) {
      const int qb = q % 3;
      if (n1 < R2) {
        const int k2 = n1;
        float2* Fb = F + qb * CS;
        if (q == 2) {
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) wr[k1] = w2[k1];
        }
        DFT<R1, true, float2>::run(wr);
#pragma unroll
        for (int m1 = 0; m1 < R1; ++m1) Fb[m1 * S1 + k2 * TC + c] = m1 == 0 ? wr[0] : cmulc(wr[m1], twr[m1]);
        if (q < 4) {  // the next component's own slots, read before the barrier that frees its buffer
          if constexpr (TM) {
            tm_ld16(tmq + 32u * (q - 2), wr);
          } else {
            const float2* Fn = F + (q - 2) * CS + k2 * S2 + c;
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) wr[k1] = Fn[k1 * TC];
          }
        }
      }
      if (TM && q == 3) tm_fence_before();  // the last tensor-memory access of every thread
      __syncthreads();
    }
    if constexpr (TM) {
      if (t < 32) {
        tm_fence_after();
        tm_dealloc(tm_slot, 64u);
      }
    }
    // the last stage is left rolled over the components: a third of the unrolled code, and
    // fewer registers (154, from 168), measured 2% faster
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {
      const float2* Fq = F + q * CS;
      float2 v[R2];
#pragma unroll
      for (int j = 0; j < R2; ++j) v[j] = Fq[n1 * S1 + j * TC + c];
      DFT<R2, true, float2>::run(v);
      if (colok) {
#pragma unroll
        for (int m2 = 0; m2 < R2; ++m2) {
          if (PR && m2 >= R2 / 2) continue;
          // (the curl's pass of an Eq. 5 iteration writes only the planes of Omega's box: the
          // masked curl downstream reads nothing else)
          if (!PR && (n1 + R1 * m2 < zlo || n1 + R1 * m2 >= zhi)) continue;
          col[q * cstride + (size_t)(n1 + R1 * m2) * zstride] = v[m2];
        }
      }
    }
  } else {
    // R1 > R2 leaves threads idle in stage B, and the curl's spectra plus its separable
    // factors do not fit the register budget of the own-slot form: the product runs on
    // all threads over natural-order spectra [kz][c]
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float2* Fq = F + q * CS;
      float2 v[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) v[n2] = n2 < NL ? pre[q][n2] : make_float2(0.f, 0.f);
      dft_maybe_half<R2, false, PR>(v);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) Fq[k2 * S2 + n1 * TC + c] = k2 == 0 ? v[0] : cmul(v[k2], twr[k2]);
      __syncthreads();
      float2 w[R1];
      if (n1 < R2) {
#pragma unroll
        for (int m = 0; m < R1; ++m) w[m] = Fq[n1 * S2 + m * TC + c];
        DFT<R1, false, float2>::run(w);
      }
      __syncthreads();
      if (n1 < R2) {
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) Fq[(n1 + R2 * k1) * TC + c] = w[k1];
      }
    }
    __syncthreads();
    // ---- product on the natural-order spectra [kz][c]; a fixed trip count, unrolled so
    // the kernel-spectrum loads of several points are in flight together
    static_assert((L * TC) % NT == 0, "product loop trip count");
    static_assert(NT % TC == 0, "a thread keeps its column in the product loop");
    const int yc = y, kxx = colok ? kx : 0;  // idx % TC == c on every trip
#pragma unroll 8
    for (int j = 0; j < L * TC / NT; ++j) {
      const int idx = t + j * NT;
      const int kz = idx / TC;
      float ax, ay, az, s;
      if (KIND == 0) {
        ax = kt0[kxx]; ay = kt1[yc]; az = kt2[kz];
        s = st0[kxx] * st1[yc] * st2[kz] * scale;
      } else {
        const int y = yc;
        const int fy = (y <= ny) ? y : 2 * ny - y;
        const int fz = (kz <= nz) ? kz : 2 * nz - kz;
        const float4 K = kap4[((size_t)fz * (ny + 1) + fy) * (nx + 1) + kxx];
        ax = K.x;
        ay = (y <= ny) ? K.y : -K.y;
        az = (kz <= nz) ? K.z : -K.z;
        s = 1.f;
      }
      const float2 F0 = F[idx], F1 = F[CS + idx], F2 = F[2 * CS + idx];
      const float2 cx = make_float2(ay * F2.x - az * F1.x, ay * F2.y - az * F1.y);
      const float2 cy = make_float2(az * F0.x - ax * F2.x, az * F0.y - ax * F2.y);
      const float2 cz = make_float2(ax * F1.x - ay * F0.x, ax * F1.y - ay * F0.y);
      F[idx] = make_float2(-s * cx.y, s * cx.x);
      F[CS + idx] = make_float2(-s * cy.y, s * cy.x);
      F[2 * CS + idx] = make_float2(-s * cz.y, s * cz.x);
    }
    __syncthreads();
    // ---- inverse: y[m1 + R1 m2] = sum_k2 W_R2^{-m2 k2} W_L^{-m1 k2} (sum_k1 X[k2 + R2 k1] W_R1^{-m1 k1})
    for (int q = 0; q < 3; ++q) {
      float2* Fq = F + q * CS;
      float2 w[R1];
      if (n1 < R2) {
        const int k2 = n1;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) w[k1] = Fq[(k2 + R2 * k1) * TC + c];
        DFT<R1, true, float2>::run(w);
      }
      __syncthreads();
      if (n1 < R2) {
        const int k2 = n1;
#pragma unroll
        for (int m1 = 0; m1 < R1; ++m1) Fq[m1 * S1 + k2 * TC + c] = m1 == 0 ? w[0] : cmulc(w[m1], twr[m1]);
      }
      __syncthreads();
      float2 v[R2];
#pragma unroll
      for (int j = 0; j < R2; ++j) v[j] = Fq[n1 * S1 + j * TC + c];
      DFT<R2, true, float2>::run(v);
      if (colok) {
#pragma unroll
        for (int m2 = 0; m2 < R2; ++m2) {
          if (PR && m2 >= R2 / 2) continue;
          // (the curl's pass of an Eq. 5 iteration writes only the planes of Omega's box: the
          // masked curl downstream reads nothing else)
          if (!PR && (n1 + R1 * m2 < zlo || n1 + R1 * m2 >= zhi)) continue;
          col[q * cstride + (size_t)(n1 + R1 * m2) * zstride] = v[m2];
        }
      }
    }
  }
}

// Padded z pass with the Biot-Savart kernel product, 256-point z transforms (16 x 16 split), in
// a leaner form: the spectra of components 0 and 1 wait for the product in tensor memory (as in
// KIND 2), so the transposes need only two shared-memory buffers (A, B) instead of three, and a
// component's input is loaded while the previous component is transformed instead of all three
// up front.  37 KB of shared memory and at most 80 registers per thread: six CTAs per SM (24
// warps) instead of four.  The arithmetic of every point is that of zpass_reg2_kernel in the same
// order, so the results are the same bits.
//   forward:  component 0 through A, 1 through B, 2 through B (after one more barrier); K^ is
//             copied into A while components 1 and 2 are transformed
//   inverse:  component 2 through B, 0 through A, 1 through B
template <int TC>
__global__ void __launch_bounds__(TC * 16, 6)
    zpass_tm2_kernel(float2* __restrict__ base, int rows, int sx, int HX, int nzs, const float2* __restrict__ twg,
                     const float4* __restrict__ kap4, int nx, int ny, int nz, const Ctrl* ctrl, int check_done,
                     int zlo, int zhi) {
  constexpr int R = 16, L = R * R, NL = R / 2;
  constexpr int S2 = R * TC + kPad8;  // transpose row stride (both directions: R1 = R2)
  constexpr int CS = R * S2;          // one buffer
  constexpr int NT = TC * R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (check_done && ctrl->done) return;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* FA = tw + L;
  float2* FB = FA + CS;
  float4* Ks = reinterpret_cast<float4*>(FA);
  static_assert(CS * sizeof(float2) >= (L / 2 + 1) * TC * sizeof(float4), "K^ fits buffer A");
  static_assert(L % 2 == 0, "16-byte alignment of buffer A");
  const int t = threadIdx.x;
  for (int i = t; i < L; i += NT) tw[i] = twg[(i % R) * (i / R)];  // [j][n1]: W_L^{n1 j}
  const int c = t % TC, n1 = t / TC;
  // column map: TC consecutive kx of one row per CTA; the Nyquist columns kx = HX - 1 packed TC
  // (row, kx) pairs to a CTA, and those CTAs first (as in zpass_reg2_kernel)
  int y, kx;
  bool colok;
  {
    const int nfull = HX / TC, rem = HX - nfull * TC;
    const int ntail = (rows * rem + TC - 1) / TC;
    const int b = blockIdx.x;
    if (b >= ntail) {
      y = (b - ntail) / nfull;
      kx = (b - ntail - y * nfull) * TC + c;
      colok = true;
    } else {
      const int e = b * TC + c;
      colok = e < rows * rem;
      y = colok ? e / rem : 0;
      kx = colok ? nfull * TC + (e - y * rem) : 0;
    }
  }
  const size_t zstride = (size_t)rows * sx;
  const size_t cstride = (size_t)nzs * zstride;
  float2* col = base + (size_t)y * sx + kx;
  // 64 tensor-memory columns: component 0's 16 complex at columns 0-31, component 1's at 32-63
  __shared__ unsigned tm_slot;
  if (t < 32) tm_alloc(&tm_slot, 64u);
  tm_fence_before();
  __syncthreads();  // twiddles staged, tensor-memory address published
  tm_fence_after();
  const unsigned tmq = tm_slot + ((unsigned)(32 * ((t >> 5) & 3)) << 16);
  const float2* twn = tw + n1;  // W_L^{n1 j} at twn[j * R] (table laid out [j][n1])

  // input of one component: planes n1 + R n2 < L / 2, zero outside [zlo, zhi)
  bool zin[NL];
#pragma unroll
  for (int n2 = 0; n2 < NL; ++n2) zin[n2] = colok && n1 + R * n2 >= zlo && n1 + R * n2 < zhi;
  float2 nxt[NL];
#pragma unroll
  for (int n2 = 0; n2 < NL; ++n2)
    nxt[n2] = zin[n2] ? col[(size_t)(n1 + R * n2) * zstride] : make_float2(0.f, 0.f);
  float2 w2[R];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float2 v[R];
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) v[n2] = n2 < NL ? nxt[n2] : make_float2(0.f, 0.f);
    if (q < 2) {  // the next component's input, in flight during this component's transform
#pragma unroll
      for (int n2 = 0; n2 < NL; ++n2)
        nxt[n2] = zin[n2] ? col[(q + 1) * cstride + (size_t)(n1 + R * n2) * zstride] : make_float2(0.f, 0.f);
    }
    dft_maybe_half<R, false, true>(v);
    float2* Fq = q == 0 ? FA : FB;
    if (q == 2) __syncthreads();  // every thread has read component 1's transpose out of B
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) Fq[k2 * S2 + n1 * TC + c] = k2 == 0 ? v[0] : cmul(v[k2], twn[k2 * R]);
    __syncthreads();
    if (q == 1) {
      // component 0's transpose has been read out of A by every thread: copy this column's
      // kernel spectrum K^(kx, fy, fz), fz = 0..L/2 (kz folded), into A with 16-byte cp.async
      const int fy = (y <= ny) ? y : 2 * ny - y;
      const size_t plane = (size_t)(ny + 1) * (nx + 1);
      const float4* src = kap4 + (size_t)fy * (nx + 1) + (colok ? kx : 0);
      for (int fz = n1; fz <= L / 2; fz += R) cp_async16(Ks + fz * TC + c, src + fz * plane);
    }
    float2 w[R];
#pragma unroll
    for (int m = 0; m < R; ++m) w[m] = Fq[n1 * S2 + m * TC + c];
    DFT<R, false, float2>::run(w);
    if (q < 2) {
      tm_st16(tmq + 32u * (unsigned)q, w);
    } else {
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) w2[k1] = w[k1];
    }
  }
  cp_async_wait_all();
  __syncthreads();  // K^ complete and visible
  // ---- product at kz = k2 + R k1 (k2 = n1) on the thread's own points: components 0 and 1 from
  // tensor memory, component 2 in registers; K^ is odd in ky (component y) and in kz (component z)
  // about the fold
  {
    const int k2 = n1;
    const float syg = (y <= ny) ? 1.f : -1.f;
#pragma unroll
    for (int b = 0; b < R / 4; ++b) {
      float2 g0[4], g1[4];
      tm_ld4x2(tmq + 8u * b, g0, tmq + 32u + 8u * b, g1);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k1 = 4 * b + i;
        const int kz = k2 + R * k1;
        const int fz = (kz <= L / 2) ? kz : L - kz;
        const float4 K = Ks[fz * TC + c];
        const float ax = K.x, ay = syg * K.y, az = (kz <= L / 2) ? K.z : -K.z;
        const float2 G0 = g0[i], G1 = g1[i], G2 = w2[k1];
        const float2 cx = make_float2(ay * G2.x - az * G1.x, ay * G2.y - az * G1.y);
        const float2 cy = make_float2(az * G0.x - ax * G2.x, az * G0.y - ax * G2.y);
        const float2 cz = make_float2(ax * G1.x - ay * G0.x, ax * G1.y - ay * G0.y);
        g0[i] = make_float2(-cx.y, cx.x);
        g1[i] = make_float2(-cy.y, cy.x);
        w2[k1] = make_float2(-cz.y, cz.x);
      }
      tm_st4x2(tmq + 8u * b, g0, tmq + 32u + 8u * b, g1);
    }
  }
  // ---- inverse: y[m1 + R m2] = sum_k2 W_R^{-m2 k2} W_L^{-m1 k2} (sum_k1 X[k2 + R k1] W_R^{-m1 k1}),
  // the outputs m2 < R/2 (planes below L/2) only
  // components in the order 2 (through B), 0 (through A), 1 (through B); stage A' of one
  // component and stage B' of the previous one share a barrier interval.  Stage A' of component
  // 2 (from registers) comes first; the rest is a loop left rolled (less code: instruction-cache
  // misses stalled the unrolled form), the same arithmetic.
  {
    DFT<R, true, float2>::run(w2);
#pragma unroll
    for (int m1 = 0; m1 < R; ++m1) FB[m1 * S2 + n1 * TC + c] = m1 == 0 ? w2[0] : cmulc(w2[m1], twn[m1 * R]);
  }
  __syncthreads();  // (also: every thread is past the product, so A is free)
#pragma unroll 1
  for (int s = 1; s < 4; ++s) {
    {  // stage B' of the component of step s - 1
      const int q = s == 1 ? 2 : (s == 2 ? 0 : 1);
      const float2* Fb = s == 2 ? FA : FB;
      float2 v[R];
#pragma unroll
      for (int j = 0; j < R; ++j) v[j] = Fb[n1 * S2 + j * TC + c];
      DFT<R, true, float2>::run(v);
      if (colok) {
#pragma unroll
        for (int m2 = 0; m2 < R / 2; ++m2) col[q * cstride + (size_t)(n1 + R * m2) * zstride] = v[m2];
      }
    }
    if (s < 3) {  // stage A' of component 0 (through A), then 1 (through B)
      float2* Fb = s == 1 ? FA : FB;
      float2 wr[R];
      tm_ld16(tmq + 32u * (unsigned)(s - 1), wr);
      DFT<R, true, float2>::run(wr);
#pragma unroll
      for (int m1 = 0; m1 < R; ++m1) Fb[m1 * S2 + n1 * TC + c] = m1 == 0 ? wr[0] : cmulc(wr[m1], twn[m1 * R]);
      if (s == 2) tm_fence_before();  // the last tensor-memory access of every thread
      __syncthreads();  // s = 1: B has been read by all
      if (s == 2 && t < 32) {
        tm_fence_after();
        tm_dealloc(tm_slot, 64u);
      }
    }
  }
}

// End of an Eq. 5 update pass: the CTA's residual sum (part, per thread) to partials[block];
// the last CTA adds the partials in block order (deterministic), sets the residual, the
// iteration count and the stop flag, and resets the arrival counter.
__device__ __forceinline__ void residual_finish(const XRArgs& a, double part, int it, int NT) {
  const int tid = threadIdx.x;
  __shared__ double red[32];
  __shared__ int am_last;
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) red[tid >> 5] = part;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < (NT + 31) / 32; ++i) s += red[i];
    a.partials[blockIdx.x] = s;
    __threadfence();
    const unsigned prev = atomicAdd(&a.ctrl->counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    double s = 0.0;
    for (int i = tid; i < (int)gridDim.x; i += NT) s += __ldcg(&a.partials[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < (NT + 31) / 32; ++i) tot += red[i];
      const double rres = tot * a.ppd->inv_nout;
      Ctrl* c = a.ctrl;
      c->residual = rres;
      c->iters = it + 1;
      c->iter_total += 1;
      c->cur = (it + 1) & 1;
      const bool finite = isfinite(rres);
      if (!finite) c->status = 6;  // SCFFT_ENONFINITE
      c->done = (!finite || rres < a.ppd->tol) ? 1 : 0;
      c->counter = 0;
    }
  }
}

// x pass, one component at a time; the node-wise step reads the three
// components' real rows from shared memory RS[q][p][x] (complex = rows a, b).
// At most 128 registers (four CTAs per SM): the batched node-wise loads would otherwise
// take the Eq. 5 update pass to 152 registers and three CTAs, which measured slower.
template <int MODE, int R1i, int R2i, int R2o, int P>
__global__ void __launch_bounds__(P * XS<MODE, R1i, R2i, R2o>::TP, 4)
    xpass_reg2_kernel(const XRArgs a) {
  typedef XS<MODE, R1i, R2i, R2o> S;
  constexpr int TP = S::TP, R1o = S::R1o, Li = S::Li, Lo = S::Lo;
  constexpr bool UPD = (MODE == X_UPDATE || MODE == X_UPDATE_FD);  // the Eq. 5 update
  constexpr int NT = P * TP;
  constexpr int XL = S::C2R ? (S::PADIN ? Li / 2 : Li) : (S::PADOUT ? Lo / 2 : Lo);  // nx
  constexpr int TT = cmax(cmax(S::C2R ? R2i * (R1i + 1) : 1, S::R2C ? R2o * (R1o + 1) : 1), S::R2C ? Lo : 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.check_done && a.ctrl->done) return;
  // The update pass takes the iteration index from the device (Ctrl::iters, advanced by its
  // own last CTA) and dh_e/dt, the stop threshold and 1/|Omega_out| from the device copy of
  // the rhs parameters, so the same launch serves every iteration of a captured loop.
  const float* h_old = a.hold;
  float* h_new = a.hnew;
  int it = 0;
  float hef[3] = {0.f, 0.f, 0.f};
  if (UPD) {
    it = *reinterpret_cast<volatile const int*>(&a.ctrl->iters);
    h_old = a.hbuf[it & 1];
    h_new = a.hbuf[(it + 1) & 1];
#pragma unroll
    for (int q = 0; q < 3; ++q) hef[q] = (float)a.ppd->hedot[q];
  }
  float2* twi = reinterpret_cast<float2*>(smem_raw);
  float2* two = twi + (Li > 0 ? Li : 1);
  float2* RS = two + (Lo > 0 ? Lo : 1);  // [3][P][XL]
  float2* T = RS + 3 * P * XL;           // [P][TT]
  const int tid = threadIdx.x;
  const int p = tid / TP, r = tid % TP;
  // twiddle tables laid out [k2][n1] (entry k2 R + n1 holds W^{n1 k2}), so that the lanes n1 of
  // a pair read consecutive words in the first stage instead of a stride of k2 (bank conflicts)
  if (S::C2R)
    for (int i = tid; i < Li; i += NT) twi[i] = a.tw_in[(i % R1i) * (i / R1i)];
  if (S::R2C)
    for (int i = tid; i < Lo; i += NT) two[i] = a.tw_out[(i % R1o) * (i / R1o)];
  const int ny = a.g.ny, nz = a.g.nz;
  const long long N = a.g.N;
  const int npairs = pair_count(a);
  constexpr bool CSPL = (MODE == X_MASKPAD);  // the components are independent in this mode
  const bool split = CSPL && a.comp_split;
  const int ntiles = (npairs + P - 1) / P;
  const int nwork = split ? 3 * ntiles : ntiles;
  float partf = 0.f;
  static_assert(XL % TP == 0 && 32 % TP == 0, "a row pair's nodes split evenly over its lanes, inside one warp");
  __syncthreads();  // twiddle tables
  // persistent CTAs: each walks tiles of P row pairs with a stride of the grid.  Inside a tile
  // every shared-memory exchange stays within one row pair, whose TP lanes lie in one warp, so
  // the tile needs warp barriers only and the warps of a CTA run independently of each other.
  // Lane r of pair p owns the nodes x = r + TP j of both rows in the node-wise step.
  for (int wk = blockIdx.x; wk < nwork; wk += gridDim.x) {
    // a work item: tile wk of all three components, or (split) component wk % 3 of tile wk / 3
    const int tile = split ? wk / 3 : wk;
    const int q0 = split ? wk - 3 * tile : 0, q1 = split ? q0 + 1 : 3;
    // prefetch the next tile's first-phase rows into L2 while this tile runs
    if (!split && tile + (int)gridDim.x < ntiles) {
      const int nrow0 = 2 * (tile + (int)gridDim.x) * P;
      if constexpr (S::C2R) {
        const int lines = ((Li / 2 + 1) * 8 + 127) / 128;
        for (int i = tid; i < 2 * P * lines; i += NT) {
          const int ln = i % lines, rr = i / lines;
          const int qrow = nrow0 + rr;
          if (qrow < 2 * npairs) {
            int zz, yy;
            pair_rows(a, qrow >> 1, zz, yy);
            yy += qrow & 1;
            prefetch_l2(a.spec_in + ((size_t)zz * a.in_rows + yy) * a.in_sx + ln * 16);
          }
        }
      } else {
        const int rl8 = (XL * 8 + 127) / 128;
        for (int i = tid; i < 3 * 2 * P * rl8; i += NT) {
          const int ln = i % rl8, rr = (i / rl8) % (2 * P), q = i / (rl8 * 2 * P);
          if (nrow0 + rr < 2 * npairs) {
            if (a.src_f32)
              prefetch_l2(a.src_f32 + q * N + (size_t)(nrow0 + rr) * XL + ln * 32);
            else
              prefetch_l2(a.src_f64 + q * N + (size_t)(nrow0 + rr) * XL + ln * 16);
          }
        }
      }
    }
    const int gp = tile * P + p;
    const bool pok = gp < npairs;
    int z, ya;
    pair_rows(a, pok ? gp : 0, z, ya);
    const int qa = z * ny + ya;  // flat index of the pair's first row
    float2* Tp = T + p * TT;

    // L2 prefetch of everything this CTA reads after its first phase (components 1
    // and 2 of the input rows, and the node-wise step's rows), so that those later
    // phases see L2 rather than DRAM latency; it costs no registers.
    if (!split) {
      const int row0 = 2 * tile * P;  // first (z, y) row of this CTA
      const int nrow = 2 * P;
      if constexpr (S::C2R) {
        const int lines = ((Li / 2 + 1) * 8 + 127) / 128;  // 128-byte lines per half-spectrum row
        for (int i = tid; i < 2 * nrow * lines; i += NT) {
          const int ln = i % lines, rr = (i / lines) % nrow, q = 1 + i / (lines * nrow);
          const int qrow = row0 + rr;
          if (qrow < 2 * npairs) {
            int zz, yy;
            pair_rows(a, qrow >> 1, zz, yy);
            yy += qrow & 1;
            prefetch_l2(a.spec_in + ((size_t)(q * nz + zz) * a.in_rows + yy) * a.in_sx + ln * 16);
          }
        }
      }
      const size_t nb0 = (size_t)row0 * XL;
      const int rl = (XL * 4 + 127) / 128;  // lines per FP32 node row
      if (UPD)
        for (int i = tid; i < 3 * nrow * rl; i += NT) {
          const int ln = i % rl, rr = (i / rl) % nrow, q = i / (rl * nrow);
          if (row0 + rr < 2 * npairs) prefetch_l2(h_old + q * N + nb0 + (size_t)rr * XL + ln * 32);
        }
      if (MODE == X_ASSEMBLE && a.warm)
        for (int i = tid; i < 3 * nrow * 2 * rl; i += NT) {
          const int ln = i % (2 * rl), rr = (i / (2 * rl)) % nrow, q = i / (2 * rl * nrow);
          if (row0 + rr < 2 * npairs) prefetch_l2(a.warm + q * N + nb0 + (size_t)rr * XL + ln * 16);
        }
      if (UPD || MODE == X_ASSEMBLE || MODE == X_MASKPAD || MODE == X_POWERLAW || MODE == X_POWERLAW_H)
        for (int i = tid * 128; i < nrow * XL; i += NT * 128)
          if (row0 + i / XL < 2 * npairs) {
            int zz, yy;
            const int qrow = row0 + i / XL;
            pair_rows(a, qrow >> 1, zz, yy);
            yy += qrow & 1;
            prefetch_l2(a.mask + ((size_t)zz * ny + yy) * XL + i % XL);
          }
    }

    if constexpr (S::C2R) {
      for (int q = q0; q < q1; ++q) {
        const int n1 = r;
        if (n1 < R1i) {
          const float2* ra = a.spec_in + ((size_t)(q * nz + z) * a.in_rows + ya) * a.in_sx;
          const float2* rb = ra + a.in_sx;
          float2 v[R2i];
  #pragma unroll
          for (int n2 = 0; n2 < R2i; ++n2) {
            const int k = n1 + R1i * n2;
            const bool lo = k <= Li / 2;
            const int kk = lo ? k : Li - k;
            float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
            if (pok) { A = ra[kk]; B = rb[kk]; }
            if (kk == 0 || kk == Li / 2) { A.y = 0.f; B.y = 0.f; }
            v[n2] = lo ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, B.x - A.y);
          }
          DFT<R2i, true, float2>::run(v);
  #pragma unroll
          for (int k2 = 0; k2 < R2i; ++k2) Tp[k2 * (R1i + 1) + n1] = k2 == 0 ? v[0] : cmulc(v[k2], twi[k2 * R1i + n1]);
        }
        __syncwarp();
        const int k2 = r;
        if (k2 < R2i) {
          float2 w[R1i];
  #pragma unroll
          for (int m = 0; m < R1i; ++m) w[m] = Tp[k2 * (R1i + 1) + m];
          DFT<R1i, true, float2>::run(w);
  #pragma unroll
          for (int k1 = 0; k1 < S::KX; ++k1) RS[(q * P + p) * XL + k2 + R2i * k1] = w[k1];
        }
        __syncwarp();
      }
    } else {
      // real rows of this lane's pair into RS, in unrolled batches of RB loads per thread (the
      // loads of a batch are in flight together; a plain loop would wait for each before its
      // shared store)
      constexpr int JT = 3 * (XL / TP), RB = 8;
#pragma unroll 1
      for (int j0 = 0; j0 < JT; j0 += RB) {
        float2 zb[RB];
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
          const int j = j0 + jj, q = j / (XL / TP), x = r + TP * (j - q * (XL / TP));
          zb[jj] = make_float2(0.f, 0.f);
          if (j < JT && pok) {
            const size_t na = (size_t)qa * XL + x;
            zb[jj] = a.src_f32 ? make_float2(a.src_f32[q * N + na], a.src_f32[q * N + na + XL])
                               : make_float2((float)a.src_f64[q * N + na], (float)a.src_f64[q * N + na + XL]);
          }
        }
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
          const int j = j0 + jj, q = j / (XL / TP), x = r + TP * (j - q * (XL / TP));
          if (j < JT) RS[(q * P + p) * XL + x] = zb[jj];
        }
      }
      __syncwarp();
    }

    // ---- node-wise step.  All of a thread's node-wise global reads are issued first, in
    // one unrolled batch (one memory latency per tile, not one per node pair), and the
    // arithmetic and stores follow.
    if constexpr (S::C2R) {
      const PointParams& pp = a.pp;
      constexpr int J = XL / TP;  // node pairs per thread: x = r + TP j of the lane's own row pair
      constexpr bool MASKED = MODE == X_POWERLAW || MODE == X_POWERLAW_H || MODE == X_ASSEMBLE || MODE == X_MASKPAD ||
                              UPD;
      constexpr int NO = UPD || MODE == X_ASSEMBLE ? 3 : (MODE == X_POWERLAW ? 1 : (MODE == X_POWERLAW_H ? 4 : 0));
      bool mk[J][2];
      float ov[J][NO > 0 ? NO : 1][2];  // hold (update), warm start (assemble), jc (power law)
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int x = r + TP * j;
        const bool ok = pok;
        const size_t na = (size_t)qa * XL + x, nb = na + XL;
        mk[j][0] = mk[j][1] = false;
#pragma unroll
        for (int q = 0; q < (NO > 0 ? NO : 1); ++q) ov[j][q][0] = ov[j][q][1] = 0.f;
        if (ok) {
          if (MASKED) {
            mk[j][0] = a.mask[na];
            mk[j][1] = a.mask[nb];
          }
          if (UPD) {
#pragma unroll
            for (int q = 0; q < NO; ++q) {
              ov[j][q][0] = h_old[q * N + na];
              ov[j][q][1] = h_old[q * N + nb];
            }
          } else if (MODE == X_ASSEMBLE) {
#pragma unroll
            for (int q = 0; q < NO; ++q) {
              ov[j][q][0] = a.warm_f32 ? a.warm_f32[q * N + na] : (float)a.warm[q * N + na];
              ov[j][q][1] = a.warm_f32 ? a.warm_f32[q * N + nb] : (float)a.warm[q * N + nb];
            }
          } else if (MODE == X_POWERLAW) {
            ov[j][0][0] = a.jc ? a.jc[na] : (float)pp.jc;
            ov[j][0][1] = a.jc ? a.jc[nb] : (float)pp.jc;
          } else if (MODE == X_POWERLAW_H) {
            ov[j][0][0] = a.jc ? a.jc[na] : (float)pp.jc;
            ov[j][0][1] = a.jc ? a.jc[nb] : (float)pp.jc;
            if (pp.kim_h0 > 0) {
#pragma unroll
              for (int q = 0; q < 3; ++q) {
                ov[j][1 + q][0] = a.src_f32 ? a.src_f32[q * N + na] : (float)a.src_f64[q * N + na];
                ov[j][1 + q][1] = a.src_f32 ? a.src_f32[q * N + nb] : (float)a.src_f64[q * N + nb];
              }
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int x = r + TP * j, pp2 = p;
        if (!pok) continue;
        const size_t na = (size_t)qa * XL + x, nb = na + XL;
        const bool ia = mk[j][0], ib = mk[j][1];
        float2 u[3];
  #pragma unroll
        for (int q = 0; q < 3; ++q) u[q] = RS[(q * P + pp2) * XL + x];
        if (MODE == X_POWERLAW) {
          const float ra = rho_of(u[0].x, u[1].x, u[2].x, ia, ov[j][0][0], pp);
          const float rb = rho_of(u[0].y, u[1].y, u[2].y, ib, ov[j][0][1], pp);
  #pragma unroll
          for (int q = 0; q < 3; ++q) u[q] = make_float2(u[q].x * ra, u[q].y * rb);
        } else if (MODE == X_POWERLAW_H) {
          float fa[3], fb[3];
          law_factors(u[0].x, u[1].x, u[2].x, ia, ov[j][0][0], ov[j][NO > 1 ? 1 : 0][0], ov[j][NO > 2 ? 2 : 0][0],
                      ov[j][NO > 3 ? 3 : 0][0], pp, fa);
          law_factors(u[0].y, u[1].y, u[2].y, ib, ov[j][0][1], ov[j][NO > 1 ? 1 : 0][1], ov[j][NO > 2 ? 2 : 0][1],
                      ov[j][NO > 3 ? 3 : 0][1], pp, fb);
  #pragma unroll
          for (int q = 0; q < 3; ++q) u[q] = make_float2(u[q].x * fa[q], u[q].y * fb[q]);
        } else if (MODE == X_ASSEMBLE) {
          const float s = -(float)pp.inv_mu0;
  #pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float va = ia ? s * u[q].x : ov[j][q][0];
            const float vb = ib ? s * u[q].y : ov[j][q][1];
            h_new[q * N + na] = va;
            h_new[q * N + nb] = vb;
            u[q] = make_float2(va, vb);
          }
        } else if (MODE == X_MASKPAD) {
          // (a split work item holds one component; the other slots are not read downstream)
  #pragma unroll
          for (int q = 0; q < 3; ++q) u[q] = make_float2(ia ? u[q].x : 0.f, ib ? u[q].y : 0.f);
        } else if (UPD) {
          // per-node |dh^{i+1} - dh^i| in FP32 (the FP32 path's own precision); the
          // per-thread sum stays FP32, the CTA and grid sums are FP64
          float da = 0.f, db = 0.f;
  #pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float oa = ov[j][q][0], ob = ov[j][q][1];
            const float he = hef[q];
            const float va = ia ? oa : he + u[q].x;
            const float vb = ib ? ob : he + u[q].y;
            h_new[q * N + na] = va;
            h_new[q * N + nb] = vb;
            const float dda = va - oa, ddb = vb - ob;
            da += dda * dda;
            db += ddb * ddb;
            u[q] = make_float2(va, vb);
          }
          if (!ia) partf += sqrtf(da);
          if (!ib) partf += sqrtf(db);
        } else {  // X_TO_F64, X_CROP_F64
  #pragma unroll
          for (int q = 0; q < 3; ++q) {
            a.dst_f64[q * N + na] = (double)u[q].x;
            a.dst_f64[q * N + nb] = (double)u[q].y;
          }
        }
        if (S::R2C) {
  #pragma unroll
          for (int q = 0; q < 3; ++q) RS[(q * P + pp2) * XL + x] = u[q];
        }
      }
      __syncwarp();
    }

    if constexpr (S::R2C) {
      for (int q = q0; q < q1; ++q) {
        const int n1 = r;
        if (n1 < R1o) {
          float2 u[R2o];
  #pragma unroll
          for (int n2 = 0; n2 < R2o; ++n2) {
            const int x = n1 + R1o * n2;
            u[n2] = (x < XL) ? RS[(q * P + p) * XL + x] : make_float2(0.f, 0.f);
          }
          dft_maybe_half<R2o, false, S::PADOUT>(u);
  #pragma unroll
          for (int k2 = 0; k2 < R2o; ++k2) Tp[k2 * (R1o + 1) + n1] = k2 == 0 ? u[0] : cmul(u[k2], two[k2 * R1o + n1]);
        }
        __syncwarp();
        const int k2 = r;
        float2 Zr[R1o];
        if (k2 < R2o) {
  #pragma unroll
          for (int m = 0; m < R1o; ++m) Zr[m] = Tp[k2 * (R1o + 1) + m];
          DFT<R1o, false, float2>::run(Zr);
        }
        // separate the two rows: A = (Z[k] + conj Z[Lo-k])/2, B = (Z[k] - conj Z[Lo-k])/(2i).
        // Thread k2 holds Z[k2 + R2o k1]; the mirror Lo - k lives in thread R2o - k2 at
        // register R1o - 1 - k1 (k2 > 0) or in this thread at (R1o - k1) mod R1o (k2 = 0),
        // so a warp shuffle inside the pair's lanes replaces a trip through shared memory.
        const int lane = tid & 31;
        const int src = lane - k2 + (k2 == 0 ? 0 : R2o - k2);
        float2* ra = a.spec_out + ((size_t)(q * nz + z) * a.out_rows + ya) * a.out_sx;
        float2* rb = ra + a.out_sx;
#pragma unroll
        for (int k1 = 0; k1 <= R1o / 2; ++k1) {
          const float2 sh = make_float2(__shfl_sync(0xffffffffu, Zr[R1o - 1 - k1].x, src),
                                        __shfl_sync(0xffffffffu, Zr[R1o - 1 - k1].y, src));
          const float2 Zk = Zr[k1];
          const float2 Zm = k2 == 0 ? Zr[(R1o - k1) % R1o] : sh;
          const int k = k2 + R2o * k1;
          if (k2 < R2o && pok && k <= Lo / 2) {
            ra[k] = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
            rb[k] = make_float2(0.5f * (Zk.y + Zm.y), 0.5f * (Zm.x - Zk.x));
          }
        }
        __syncwarp();  // the next component's stage A' overwrites Tp
      }
    }
    __syncwarp();  // the pair's shared buffers are reused by the next tile
  }

  if (UPD) residual_finish(a, (double)partf, it, NT);
  if (MODE == X_ASSEMBLE && blockIdx.x == 0 && tid == 0) {
    *a.ppd = a.pps ? *a.pps : a.pp;
    a.ctrl->trips = 0;
    a.ctrl->done = 0;
    a.ctrl->iters = 0;
    a.ctrl->cur = 0;
    a.ctrl->counter = 0;
    a.ctrl->residual = 0.0;
  }
}


// Eq. 5 update pass with the three components side by side: a CTA of three warp groups, group
// g running component g's C2R (length 2nx, crop) and R2C (length nx) for a tile of P row pairs,
// so that the three components' input rows are in flight at once (the one-component-at-a-time
// pass waits for them one after another); the node-wise step between the transforms, which
// needs all three components of a node, runs on all groups over shared memory (group g takes
// the nodes x = r + TP j, j = g mod 3, of its lane r).  Every element's arithmetic is that of
// xpass_reg2_kernel<X_UPDATE> in the same order, so the iterate and the transforms are the same
// bits; the residual's per-thread FP32 sums cover other nodes, so its last bits may differ.
template <int R1i, int R2i, int R2o, int P>
__global__ void __launch_bounds__(3 * P * XS<X_UPDATE, R1i, R2i, R2o>::TP, 16 / P) xupdate3_kernel(const XRArgs a) {
  typedef XS<X_UPDATE, R1i, R2i, R2o> S;
  constexpr int TP = S::TP, R1o = S::R1o, Li = S::Li, Lo = S::Lo;
  constexpr int NG = P * TP;    // threads of a group
  constexpr int NT = 3 * NG;
  constexpr int XL = Li / 2;    // nx
  constexpr int TT = cmax(cmax(R2i * (R1i + 1), R2o * (R1o + 1)), Lo);
  constexpr int J = XL / TP;    // node pairs of a lane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.check_done && a.ctrl->done) return;
  const int it = *reinterpret_cast<volatile const int*>(&a.ctrl->iters);
  const float* h_old = a.hbuf[it & 1];
  float* h_new = a.hbuf[(it + 1) & 1];
  float hef[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) hef[q] = (float)a.ppd->hedot[q];
  float2* twi = reinterpret_cast<float2*>(smem_raw);
  float2* two = twi + Li;
  float2* RS = two + Lo;         // [3][P][XL]
  float2* T = RS + 3 * P * XL;   // [3][P][TT]
  const int tid = threadIdx.x;
  const int g = tid / NG, lt = tid - g * NG;
  const int p = lt / TP, r = lt % TP;
  for (int i = tid; i < Li; i += NT) twi[i] = a.tw_in[(i % R1i) * (i / R1i)];
  for (int i = tid; i < Lo; i += NT) two[i] = a.tw_out[(i % R1o) * (i / R1o)];
  const int ny = a.g.ny, nz = a.g.nz;
  const long long N = a.g.N;
  const int npairs = pair_count(a);
  const int ntiles = (npairs + P - 1) / P;
  float partf = 0.f;
  static_assert(XL % TP == 0 && 32 % TP == 0 && NG % 32 == 0, "a pair's lanes in one warp, groups of whole warps");
  __syncthreads();  // twiddle tables
  float2* Tp = T + (g * P + p) * TT;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // L2 prefetch of the next tile's input rows (all three components) and of this tile's
    // node-wise rows (previous iterate, mask), which are read after the transforms
    {
      const int lines = ((Li / 2 + 1) * 8 + 127) / 128;
      if (tile + (int)gridDim.x < ntiles) {
        const int nrow0 = 2 * (tile + (int)gridDim.x) * P;
        for (int i = tid; i < 3 * 2 * P * lines; i += NT) {
          const int ln = i % lines, rr = (i / lines) % (2 * P), q = i / (lines * 2 * P);
          const int qrow = nrow0 + rr;
          if (qrow < 2 * npairs) {
            int zz, yy;
            pair_rows(a, qrow >> 1, zz, yy);
            yy += qrow & 1;
            prefetch_l2(a.spec_in + ((size_t)(q * nz + zz) * a.in_rows + yy) * a.in_sx + ln * 16);
          }
        }
      }
      const int row0 = 2 * tile * P, nrow = 2 * P;
      const size_t nb0 = (size_t)row0 * XL;
      const int rl = (XL * 4 + 127) / 128;
      for (int i = tid; i < 3 * nrow * rl; i += NT) {
        const int ln = i % rl, rr = (i / rl) % nrow, q = i / (rl * nrow);
        if (row0 + rr < 2 * npairs) prefetch_l2(h_old + q * N + nb0 + (size_t)rr * XL + ln * 32);
      }
      for (int i = tid * 128; i < nrow * XL; i += NT * 128)
        if (row0 + i / XL < 2 * npairs) {
          int zz, yy;
          const int qrow = row0 + i / XL;
          pair_rows(a, qrow >> 1, zz, yy);
          yy += qrow & 1;
          prefetch_l2(a.mask + ((size_t)zz * ny + yy) * XL + i % XL);
        }
    }
    const int gp = tile * P + p;
    const bool pok = gp < npairs;
    int z, ya;
    pair_rows(a, pok ? gp : 0, z, ya);
    const int qa = z * ny + ya;
    // ---- C2R (length 2nx) of component g, the first nx outputs kept
    {
      const int q = g;
      const int n1 = r;
      if (n1 < R1i) {
        const float2* ra = a.spec_in + ((size_t)(q * nz + z) * a.in_rows + ya) * a.in_sx;
        const float2* rb = ra + a.in_sx;
        float2 v[R2i];
#pragma unroll
        for (int n2 = 0; n2 < R2i; ++n2) {
          const int k = n1 + R1i * n2;
          const bool lo = k <= Li / 2;
          const int kk = lo ? k : Li - k;
          float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
          if (pok) { A = ra[kk]; B = rb[kk]; }
          if (kk == 0 || kk == Li / 2) { A.y = 0.f; B.y = 0.f; }
          v[n2] = lo ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, B.x - A.y);
        }
        DFT<R2i, true, float2>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < R2i; ++k2) Tp[k2 * (R1i + 1) + n1] = k2 == 0 ? v[0] : cmulc(v[k2], twi[k2 * R1i + n1]);
      }
      __syncwarp();
      const int k2 = r;
      if (k2 < R2i) {
        float2 w[R1i];
#pragma unroll
        for (int m = 0; m < R1i; ++m) w[m] = Tp[k2 * (R1i + 1) + m];
        DFT<R1i, true, float2>::run(w);
#pragma unroll
        for (int k1 = 0; k1 < S::KX; ++k1) RS[(q * P + p) * XL + k2 + R2i * k1] = w[k1];
      }
    }
    __syncthreads();  // the three components' rows of the tile in RS
    // ---- node-wise step (Eq. 5 update and residual) on the nodes x = r + TP j, j = g mod 3
    {
      constexpr int JG = (J + 2) / 3;  // node pairs of a thread, at most
      bool mk[JG][2];
      float ov[JG][3][2];
#pragma unroll
      for (int jj = 0; jj < JG; ++jj) {
        const int j = g + 3 * jj;
        const int x = r + TP * j;
        const size_t na = (size_t)qa * XL + x, nb = na + XL;
        mk[jj][0] = mk[jj][1] = false;
#pragma unroll
        for (int q = 0; q < 3; ++q) ov[jj][q][0] = ov[jj][q][1] = 0.f;
        if (pok && j < J) {
          mk[jj][0] = a.mask[na];
          mk[jj][1] = a.mask[nb];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            ov[jj][q][0] = h_old[q * N + na];
            ov[jj][q][1] = h_old[q * N + nb];
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < JG; ++jj) {
        const int j = g + 3 * jj;
        if (!pok || j >= J) continue;
        const int x = r + TP * j;
        const size_t na = (size_t)qa * XL + x, nb = na + XL;
        const bool ia = mk[jj][0], ib = mk[jj][1];
        float2 u[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) u[q] = RS[(q * P + p) * XL + x];
        float da = 0.f, db = 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float oa = ov[jj][q][0], ob = ov[jj][q][1];
          const float he = hef[q];
          const float va = ia ? oa : he + u[q].x;
          const float vb = ib ? ob : he + u[q].y;
          h_new[q * N + na] = va;
          h_new[q * N + nb] = vb;
          const float dda = va - oa, ddb = vb - ob;
          da += dda * dda;
          db += ddb * ddb;
          u[q] = make_float2(va, vb);
        }
        if (!ia) partf += sqrtf(da);
        if (!ib) partf += sqrtf(db);
#pragma unroll
        for (int q = 0; q < 3; ++q) RS[(q * P + p) * XL + x] = u[q];
      }
    }
    __syncthreads();  // the updated rows of every component in RS
    // ---- R2C (length nx) of component g
    {
      const int q = g;
      const int n1 = r;
      if (n1 < R1o) {
        float2 u[R2o];
#pragma unroll
        for (int n2 = 0; n2 < R2o; ++n2) {
          const int x = n1 + R1o * n2;
          u[n2] = (x < XL) ? RS[(q * P + p) * XL + x] : make_float2(0.f, 0.f);
        }
        dft_maybe_half<R2o, false, S::PADOUT>(u);
#pragma unroll
        for (int k2 = 0; k2 < R2o; ++k2) Tp[k2 * (R1o + 1) + n1] = k2 == 0 ? u[0] : cmul(u[k2], two[k2 * R1o + n1]);
      }
      __syncwarp();
      const int k2 = r;
      float2 Zr[R1o];
      if (k2 < R2o) {
#pragma unroll
        for (int m = 0; m < R1o; ++m) Zr[m] = Tp[k2 * (R1o + 1) + m];
        DFT<R1o, false, float2>::run(Zr);
      }
      const int lane = tid & 31;
      const int src = lane - k2 + (k2 == 0 ? 0 : R2o - k2);
      float2* ra = a.spec_out + ((size_t)(q * nz + z) * a.out_rows + ya) * a.out_sx;
      float2* rb = ra + a.out_sx;
#pragma unroll
      for (int k1 = 0; k1 <= R1o / 2; ++k1) {
        const float2 sh = make_float2(__shfl_sync(0xffffffffu, Zr[R1o - 1 - k1].x, src),
                                      __shfl_sync(0xffffffffu, Zr[R1o - 1 - k1].y, src));
        const float2 Zk = Zr[k1];
        const float2 Zm = k2 == 0 ? Zr[(R1o - k1) % R1o] : sh;
        const int k = k2 + R2o * k1;
        if (k2 < R2o && pok && k <= Lo / 2) {
          ra[k] = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
          rb[k] = make_float2(0.5f * (Zk.y + Zm.y), 0.5f * (Zm.x - Zk.x));
        }
      }
      __syncwarp();  // the group's next C2R overwrites its transpose scratch
    }
  }
  residual_finish(a, (double)partf, it, NT);
}

}  // namespace scfft
