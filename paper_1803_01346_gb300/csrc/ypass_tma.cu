// ypass_tma.cu - the FP32 padded y passes fed by the Tensor Memory Accelerator.
//
// A y pass transforms every (component, z) plane of a half spectrum along y, one tile of
// TC consecutive kx columns at a time (the four-step split of passes_reg.cu:
//   X[k2 + R2 k1] = sum_n1 W_R1^{n1 k1} W_L^{n1 k2} ( sum_n2 x[n1 + R1 n2] W_R2^{n2 k2} ) ).
// Here the CTAs are persistent and a tile's input reaches shared memory as one
// cp.async.bulk.tensor copy (a box of TC columns x the rows the transform reads), issued two
// tiles ahead into a pair of stage buffers and completed on an mbarrier, so each SM always has
// loads in flight while it transforms and stores the current tile.  A stage buffer whose input
// is in registers also holds the tile's transpose, so no third buffer is needed.  Columns past
// the half spectrum's last kx lie outside the tensor map and arrive as zeros.  Every wait on an
// mbarrier is bounded; a wait that gives up latches SCFFT_ETIMEOUT in the device control
// block, drains the other stage's copy (bounded again) and ends the CTA.
#include "scfft.h"
#include "scfft_internal.cuh"

namespace scfft {

namespace {

constexpr int kPadT = 8;  // transpose row padding (complex elements), as in passes_reg.cu

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_addr(m)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for the phase of the given parity, giving up after about a second of SM clock.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(m, parity))
    if (clock64() - t0 > 2000000000LL) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* m) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(m))
      : "memory");
}

template <int R1, int R2, int TC, bool PIN> struct YT {
  static constexpr int L = R1 * R2;
  static constexpr int NRB = PIN ? L / 2 : L;     // rows in the box (the forward padded pass reads L/2)
  static constexpr int SB = NRB * TC;             // complex elements a box brings
  static constexpr int S2 = R1 * TC + kPadT;      // transpose row stride
  // a stage buffer also holds the tile's transpose once its input is in registers
  static constexpr int SBX = ((SB > R2 * S2 ? SB : R2 * S2) + 15) / 16 * 16;
  static constexpr size_t smem = 128 + sizeof(float2) * (2 * SBX + L);
};

// grid: persistent (at most one wave); block TC*R1 threads; tiles t = chunk + nch * p over the
// 3 nzp planes p = (component, z = zoff + p mod nzp); input rows outside [ylo, yhi) read as zero
// (the forward pass of an Eq. 5 iteration runs on Omega's box only: its source vanishes outside).
template <int R1, int R2, int TC, bool INV, bool PIN, bool POUT>
__global__ void __launch_bounds__(TC * R1) ypass_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                            float2* __restrict__ base, int rows, int sx, int HX,
                                                            int nzs, const float2* __restrict__ twg, Ctrl* ctrl,
                                                            int check_done, int inject, int zoff, int nzp, int ylo,
                                                            int yhi) {
  typedef YT<R1, R2, TC, PIN> S;
  constexpr int L = S::L, SB = S::SB, SBX = S::SBX, S2 = S::S2, NT = TC * R1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (check_done && ctrl->done) return;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);         // [2]
  float2* stage = reinterpret_cast<float2*>(smem_raw + 128);      // [2][SBX], 128-byte aligned
  float2* tw = stage + 2 * SBX;                                   // [L]
  const int t = threadIdx.x, c = t % TC, n1 = t / TC;
  const int nch = (HX + TC - 1) / TC, ntiles = nch * 3 * nzp;
  // plane of the tile's columns in the [component][z] planes of the spectrum
  auto plane_of = [&](int tile) { const int p = tile / nch, q = p / nzp; return q * nzs + zoff + (p - q * nzp); };
  const unsigned bytes = (unsigned)(SB * sizeof(float2));
  if (t == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_fence_init();
  }
  for (int i = t; i < L; i += NT) tw[i] = twg[i];
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int tile = blockIdx.x + s * gridDim.x;
      if (tile < ntiles) {
        // (inject: a test of the timeout path; stage 0 then waits for 16 bytes that never come)
        mbar_expect_tx(&mbar[s], bytes + (s == 0 && inject ? 16u : 0u));
        tma_load_3d(stage + s * SBX, &tmap, (tile % nch) * TC, 0, plane_of(tile), &mbar[s]);
      }
    }
  }
  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int s = it & 1;
    const bool timed_out = !mbar_wait_bounded(&mbar[s], (it >> 1) & 1);
    float2* st = stage + s * SBX;
    float2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2)
      v[n2] = ((PIN && n2 >= R2 / 2) || n1 + R1 * n2 < ylo || n1 + R1 * n2 >= yhi) ? make_float2(0.f, 0.f)
                                                                                  : st[(n1 + R1 * n2) * TC + c];
    if (__syncthreads_or(timed_out)) {  // every thread has read stage s (or the wait gave up)
      if (t == 0) {
        ctrl->status = SCFFT_ETIMEOUT;
        const int other = tile + (int)gridDim.x;  // the copy still in flight into the other stage
        if (other < ntiles) (void)mbar_wait_bounded(&mbar[s ^ 1], ((it + 1) >> 1) & 1);
      }
      return;
    }
    const int chunk = tile % nch, plane = plane_of(tile);
    const int kx = chunk * TC + c;
    const bool colok = kx < HX;
    float2* col = base + (size_t)plane * rows * sx + kx;
    dft_maybe_half<R2, INV, PIN>(v);
#pragma unroll
    for (int k2 = 1; k2 < R2; ++k2) v[k2] = INV ? cmulc(v[k2], tw[n1 * k2]) : cmul(v[k2], tw[n1 * k2]);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) st[k2 * S2 + n1 * TC + c] = v[k2];  // transpose in the consumed stage
    __syncthreads();
    if (n1 < R2) {
      const int k2 = n1;
      float2 w[R1];
#pragma unroll
      for (int m = 0; m < R1; ++m) w[m] = st[k2 * S2 + m * TC + c];
      DFT<R1, INV, float2>::run(w);
      if (colok) {
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
          if (POUT && k1 >= R1 / 2) continue;
          col[(size_t)(k2 + R2 * k1) * sx] = w[k1];
        }
      }
    }
    __syncthreads();  // stage s is free: refill it two tiles ahead
    if (t == 0) {
      const int nt = tile + 2 * (int)gridDim.x;
      if (nt < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&mbar[s], bytes);
        tma_load_3d(stage + s * SBX, &tmap, (nt % nch) * TC, 0, plane_of(nt), &mbar[s]);
      }
    }
  }
}

template <int R1, int R2, bool INV, bool PIN, bool POUT>
cudaError_t go_y_tma(const Launch<float>& L, const CUtensorMap& map, float2* base, int rows, int sx, int HX,
                     const float2* tw, bool chk) {
  constexpr int TC = 16;
  typedef YT<R1, R2, TC, PIN> S;
  auto k = ypass_tma_kernel<R1, R2, TC, INV, PIN, POUT>;
  allow_smem<ypass_tma_kernel<R1, R2, TC, INV, PIN, POUT>>();
  const bool box = L.use_box && PIN;  // the forward pass of an Eq. 5 iteration: Omega's box only
  const int nzp = box ? L.bz1 - L.bz0 : L.g.nz;
  const int ntiles = ((HX + TC - 1) / TC) * 3 * nzp;
  static const int resident = [&] {  // one wave of resident CTAs (the kernel loops over tiles)
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, TC * R1, S::smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm > 0 && sms > 0 ? per_sm * sms : 152;
  }();
  const int grid = ntiles < resident ? ntiles : resident;
  const int inject = (L.fault && *L.fault == SCFFT_FAULT_TMA_WAIT) ? 1 : 0;
  if (inject) *L.fault = 0;  // one shot
  k<<<grid, TC * R1, S::smem, L.st>>>(map, base, rows, sx, HX, L.g.nz, tw, L.ctrl, chk ? 1 : 0, inject,
                                      box ? L.bz0 : 0, nzp, box ? L.by0 : 0, box ? L.by1 : rows);
  return cudaGetLastError();
}

template <int R1, int R2>
cudaError_t ytma(const Launch<float>& L, bool inverse, bool chk) {
  const Work<float>& w = *L.w;
  const Geo& g = L.g;
  if (inverse)
    return go_y_tma<R1, R2, true, false, true>(L, w.ym->m[1], w.Pd, 2 * g.ny, g.sxp, g.nx + 1, w.twp[1], chk);
  return go_y_tma<R1, R2, false, true, false>(L, w.ym->m[0], w.Pd, 2 * g.ny, g.sxp, g.nx + 1, w.twp[1], chk);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// One 3-D map over a half spectrum [planes][rows][sx] of 8-byte complex values: dim 0 holds
// the HX valid columns (the rest of each row reads as zeros), box = 16 columns x box_rows rows.
bool encode_map(CUtensorMap* m, float2* base, int HX, int rows, int sx, int planes, int box_rows) {
  const EncodeTiledFn fn = encode_fn();
  if (!fn || box_rows > 256) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)HX, (cuuint64_t)rows, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)sx * 8, (cuuint64_t)rows * sx * 8};
  const cuuint32_t box[3] = {16, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool make_ymaps(Work<float>& w, const Geo& g) {
  YMaps* ym = new YMaps;
  const bool ok = encode_map(&ym->m[0], w.Pd, g.nx + 1, 2 * g.ny, g.sxp, 3 * g.nz, g.ny) &&
                  encode_map(&ym->m[1], w.Pd, g.nx + 1, 2 * g.ny, g.sxp, 3 * g.nz, 2 * g.ny);
  if (!ok) {
    delete ym;
    return false;
  }
  w.ym = ym;
  return true;
}

// The padded passes only: on the unpadded half spectrum (HX = nx/2 + 1 columns, a 16-column
// tile leaves 15 of the last tile's columns empty) the plain 8-column kernel measured faster.
cudaError_t launch_y_tma(const Launch<float>& L, bool padded, bool inverse, bool check_done) {
  if (!L.w->ym || !padded) return cudaErrorNotSupported;
  switch (2 * L.g.ny) {
    case 32: return ytma<8, 4>(L, inverse, check_done);
    case 64: return ytma<8, 8>(L, inverse, check_done);
    case 96: return ytma<12, 8>(L, inverse, check_done);
    case 128: return ytma<16, 8>(L, inverse, check_done);
    case 192: return ytma<16, 12>(L, inverse, check_done);
    case 256: return ytma<16, 16>(L, inverse, check_done);
  }
  return cudaErrorNotSupported;
}

}  // namespace scfft
