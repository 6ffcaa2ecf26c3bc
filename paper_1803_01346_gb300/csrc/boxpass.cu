// boxpass.cu - the three FP32 passes of an Eq. 5 iteration that see only Omega's box, fused.
//
// Between the smoothed curl's z pass and the padded z pass, an Eq. 5 iteration runs, on the
// planes z and rows y of Omega's bounding box only (the source chi_Omega curl dh^i vanishes
// elsewhere):
//   1. the inverse y transform of the curl's half spectrum (length ny, output rows of the box),
//   2. the x pass: C2R (length nx) of each row pair, the mask chi_Omega, zero padding and the
//      R2C of length 2nx,
//   3. the forward y transform of the padded half spectrum (length 2ny; input rows of the box,
//      zero elsewhere), all 2ny output rows.
// Every step acts on one (component, plane) alone, so one CTA runs all three for one
// (component, plane) with the intermediates in shared memory: the curl's half spectrum is read
// once from global memory and the padded spectrum written once, instead of three launches that
// each make a round trip through L2.  The box holds few planes (40 of 128 for the lens), so the
// separate passes are short single waves whose latency chains dominate them.
//
// The arithmetic of each step is that of the separate passes (passes_reg.cu: ypass_reg_kernel
// and the mask/pad mode of xpass_reg2_kernel), in the same order, so the results are the same
// bits; only where the intermediates live and which thread runs which column differ.
#include "scfft_internal.cuh"

namespace scfft {

namespace {

// 544 threads: the steps use 528 (33 x 16).  Seventeen warps put five on one of the SM's four
// schedulers, whose quarter of the register file (16384) then caps a thread at 96 registers.
constexpr int kBoxWarps = 17;
constexpr int kBoxThreads = 32 * kBoxWarps;
constexpr int kBoxUse = 528;                  // threads that take columns in the y steps
constexpr int kPadB = 8;                      // transpose row padding (complex elements)

__host__ __device__ constexpr int bmax(int a, int b) { return a > b ? a : b; }
// splits R1 x R2 (R1 >= R2) of the y lengths, as the separate passes choose them
__host__ __device__ constexpr int split_r1(int L) {
  return L == 16 ? 4 : L == 32 ? 8 : L == 48 ? 12 : L == 64 ? 8 : L == 96 ? 12 : L == 128 ? 16 : L == 192 ? 16 : 16;
}
// C2R length n = A x B of the x pass (R1i = A, R2i = B; the R2C of length 2n: R1o = B, R2o = 2A)
__host__ __device__ constexpr int xa_of(int n) { return n == 96 || n == 128 ? 8 : 4; }

template <int N> struct BoxShape {
  // step 1: inverse y, length N
  static constexpr int R1y = split_r1(N), R2y = N / R1y, TC1 = kBoxUse / R1y, S2y = R1y * TC1 + kPadB;
  // step 2: x pass
  static constexpr int R1i = xa_of(N), R2i = N / R1i, R1o = R2i, R2o = 2 * R1i;
  static constexpr int Li = N, Lo = 2 * N;
  static constexpr int TP0 = bmax(bmax(R1i, R2i), R2o);
  static constexpr int TP = TP0 <= 4 ? 4 : TP0 <= 8 ? 8 : 16;  // lanes per row pair
  static constexpr int TT = bmax(bmax(R2i * (R1i + 1), R2o * (R1o + 1)), Lo);  // per-pair scratch
  static constexpr int XL = N;
  // step 3: forward y, length 2N
  static constexpr int R1p = split_r1(2 * N), R2p = 2 * N / R1p, TC3 = kBoxUse / R1p, S2p = R1p * TC3 + kPadB;
  static constexpr int HXu = N / 2 + 1, HXp = N + 1;
  static constexpr int NTW = N + Li + Lo + 2 * N;  // twiddle tables staged in shared memory
  static_assert(TC1 * R1y == kBoxUse && TC3 * R1p == kBoxUse, "the y steps tile the 528 threads");
  static_assert(32 % TP == 0 && XL % TP == 0, "a row pair's lanes lie in one warp");
};

struct BoxArgs {
  const float2* U;        // [3][nz][ny][sxu] curl half spectrum (box planes valid)
  float2* Pd;             // [3][nz][2ny][sxp] padded half spectrum (box planes written)
  const uint8_t* mask;    // [nz][ny][nx]
  const float2* tw_y;     // W_ny^m
  const float2* tw_x;     // W_nx^m
  const float2* tw_xp;    // W_2nx^m
  const float2* tw_yp;    // W_2ny^m
  const Ctrl* ctrl;
  int check_done;
  int nz, sxu, sxp;
  int by0, by1, bz0, bz1;
  int pr;                 // row pairs per round of step 2
  int offA, offS, offB;   // shared-memory regions (complex elements)
};

template <int N>
__global__ void __launch_bounds__(kBoxThreads, 1) boxpass_kernel(const BoxArgs a) {
  typedef BoxShape<N> S;
  constexpr int R1y = S::R1y, R2y = S::R2y, TC1 = S::TC1, S2y = S::S2y;
  constexpr int R1i = S::R1i, R2i = S::R2i, R1o = S::R1o, R2o = S::R2o, Li = S::Li, Lo = S::Lo;
  constexpr int TP = S::TP, TT = S::TT, XL = S::XL;
  constexpr int R1p = S::R1p, R2p = S::R2p, TC3 = S::TC3, S2p = S::S2p;
  constexpr int HXu = S::HXu, HXp = S::HXp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.check_done && a.ctrl->done) return;
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* ty = sm;              // [N]       W_N^m
  float2* twi = ty + N;         // [Li]      C2R twiddles laid out [k2][n1]
  float2* two = twi + Li;       // [Lo]      R2C twiddles laid out [k2][n1]
  float2* tp = two + Lo;        // [2N]      W_2N^m
  float2* A = sm + a.offA;      // [nbr][HXu]  box rows of the inverse y transform
  float2* Sc = sm + a.offS;     // scratch of steps 1 and 2
  float2* B = sm + a.offB;      // [nbr][HXp]  box rows of the padded R2C
  float2* Sc3 = A;              // scratch of step 3 (A and Sc, contiguous, free by then)
  const int t = threadIdx.x;
  const int nbz = a.bz1 - a.bz0, nbr = a.by1 - a.by0;
  const int q = blockIdx.x / nbz, z = a.bz0 + (blockIdx.x - q * nbz);
  for (int i = t; i < N; i += kBoxThreads) ty[i] = a.tw_y[i];
  for (int i = t; i < Li; i += kBoxThreads) twi[i] = a.tw_x[(i % R1i) * (i / R1i)];
  for (int i = t; i < Lo; i += kBoxThreads) two[i] = a.tw_xp[(i % R1o) * (i / R1o)];
  for (int i = t; i < 2 * N; i += kBoxThreads) tp[i] = a.tw_yp[i];
  __syncthreads();

  // ---- step 1: inverse y transform (length N) of the curl's half spectrum, box rows kept
  {
    const int c = t % TC1, n1 = t / TC1;  // threads t >= 528: n1 >= R1y, idle
    const float2* plane = a.U + ((size_t)(q * a.nz + z) * N) * a.sxu;
    for (int base = 0; base < HXu; base += TC1) {
      const int kx = base + c;
      const bool colok = kx < HXu && n1 < R1y;
      if (n1 < R1y) {
        float2 v[R2y];
#pragma unroll
        for (int n2 = 0; n2 < R2y; ++n2) v[n2] = colok ? plane[(size_t)(n1 + R1y * n2) * a.sxu + kx] : make_float2(0.f, 0.f);
        DFT<R2y, true, float2>::run(v);
#pragma unroll
        for (int k2 = 1; k2 < R2y; ++k2) v[k2] = cmulc(v[k2], ty[n1 * k2]);
#pragma unroll
        for (int k2 = 0; k2 < R2y; ++k2) Sc[k2 * S2y + n1 * TC1 + c] = v[k2];
      }
      __syncthreads();
      if (n1 < R2y) {
        const int k2 = n1;
        float2 w[R1y];
#pragma unroll
        for (int m = 0; m < R1y; ++m) w[m] = Sc[k2 * S2y + m * TC1 + c];
        DFT<R1y, true, float2>::run(w);
        if (kx < HXu) {
#pragma unroll
          for (int k1 = 0; k1 < R1y; ++k1) {
            const int row = k2 + R2y * k1;
            if (row >= a.by0 && row < a.by1) A[(row - a.by0) * HXu + kx] = w[k1];
          }
        }
      }
      __syncthreads();
    }
  }

  // ---- step 2: x pass of the box's row pairs: C2R (length N), mask, zero pad, R2C (length 2N)
  {
    const int p = t / TP, r = t % TP;
    const int npairs = nbr >> 1;
    float2* Tp = Sc + p * TT;
    for (int base = 0; base < npairs; base += a.pr) {
      const int gp = base + p;
      const bool pok = p < a.pr && gp < npairs;
      const int la = 2 * (pok ? gp : 0);  // the pair's first row within the box
      const int ya = a.by0 + la;
      // C2R: two real rows a, b as one complex row
      if (p < a.pr) {
        const int n1 = r;
        if (n1 < R1i) {
          const float2* ra = A + la * HXu;
          const float2* rb = ra + HXu;
          float2 v[R2i];
#pragma unroll
          for (int n2 = 0; n2 < R2i; ++n2) {
            const int k = n1 + R1i * n2;
            const bool lo = k <= Li / 2;
            const int kk = lo ? k : Li - k;
            float2 Av = make_float2(0.f, 0.f), Bv = make_float2(0.f, 0.f);
            if (pok) { Av = ra[kk]; Bv = rb[kk]; }
            if (kk == 0 || kk == Li / 2) { Av.y = 0.f; Bv.y = 0.f; }
            v[n2] = lo ? make_float2(Av.x - Bv.y, Av.y + Bv.x) : make_float2(Av.x + Bv.y, Bv.x - Av.y);
          }
          DFT<R2i, true, float2>::run(v);
#pragma unroll
          for (int k2 = 0; k2 < R2i; ++k2) Tp[k2 * (R1i + 1) + n1] = k2 == 0 ? v[0] : cmulc(v[k2], twi[k2 * R1i + n1]);
        }
      }
      __syncwarp();
      float2 w[R1i];
      if (p < a.pr && r < R2i) {
        const int k2 = r;
#pragma unroll
        for (int m = 0; m < R1i; ++m) w[m] = Tp[k2 * (R1i + 1) + m];
        DFT<R1i, true, float2>::run(w);
      }
      __syncwarp();  // the pair's real rows (x < N) go where its transpose was
      float2* RS = Tp;
      if (p < a.pr && r < R2i) {
#pragma unroll
        for (int k1 = 0; k1 < R1i; ++k1) RS[r + R2i * k1] = w[k1];
      }
      __syncwarp();
      // the mask; lane r owns the nodes x = r + TP j of both rows
      if (pok) {
        const uint8_t* ma = a.mask + ((size_t)z * N + ya) * N;
        const uint8_t* mb = ma + N;
#pragma unroll
        for (int j = 0; j < XL / TP; ++j) {
          const int x = r + TP * j;
          const float2 u = RS[x];
          RS[x] = make_float2(ma[x] ? u.x : 0.f, mb[x] ? u.y : 0.f);
        }
      }
      __syncwarp();
      // R2C of the zero-padded pair (input x < N)
      float2 u[R2o];
      if (p < a.pr && r < R1o) {
        const int n1 = r;
#pragma unroll
        for (int n2 = 0; n2 < R2o; ++n2) {
          const int x = n1 + R1o * n2;
          u[n2] = (x < XL) ? RS[x] : make_float2(0.f, 0.f);
        }
      }
      __syncwarp();
      if (p < a.pr && r < R1o) {
        const int n1 = r;
        dft_maybe_half<R2o, false, true>(u);
#pragma unroll
        for (int k2 = 0; k2 < R2o; ++k2) Tp[k2 * (R1o + 1) + n1] = k2 == 0 ? u[0] : cmul(u[k2], two[k2 * R1o + n1]);
      }
      __syncwarp();
      const int k2 = r;
      float2 Zr[R1o];
      if (p < a.pr && k2 < R2o) {
#pragma unroll
        for (int m = 0; m < R1o; ++m) Zr[m] = Tp[k2 * (R1o + 1) + m];
        DFT<R1o, false, float2>::run(Zr);
      }
      // separate the two rows: A = (Z[k] + conj Z[Lo-k])/2, B = (Z[k] - conj Z[Lo-k])/(2i); the
      // mirror Lo - k lives in lane R2o - k2 at register R1o - 1 - k1 (k2 > 0) or in this lane
      // at (R1o - k1) mod R1o (k2 = 0).  Every lane of the warp takes part in the shuffles.
      const int lane = t & 31;
      const int src = lane - k2 + (k2 == 0 ? 0 : R2o - k2);
      float2* oa = B + la * HXp;
      float2* ob = oa + HXp;
#pragma unroll
      for (int k1 = 0; k1 <= R1o / 2; ++k1) {
        const float2 sh = make_float2(__shfl_sync(0xffffffffu, Zr[R1o - 1 - k1].x, src),
                                      __shfl_sync(0xffffffffu, Zr[R1o - 1 - k1].y, src));
        const float2 Zk = Zr[k1];
        const float2 Zm = k2 == 0 ? Zr[(R1o - k1) % R1o] : sh;
        const int k = k2 + R2o * k1;
        if (k2 < R2o && pok && k <= Lo / 2) {
          oa[k] = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
          ob[k] = make_float2(0.5f * (Zk.y + Zm.y), 0.5f * (Zm.x - Zk.x));
        }
      }
      __syncwarp();  // the next round reuses the pair's scratch
    }
  }
  __syncthreads();

  // ---- step 3: forward y transform (length 2N) of the padded half spectrum: input rows of the
  // box (zero elsewhere, and zero padding from row N on), all 2N output rows to global memory
  {
    const int c = t % TC3, n1 = t / TC3;
    float2* plane = a.Pd + ((size_t)(q * a.nz + z) * (2 * N)) * a.sxp;
    for (int base = 0; base < HXp; base += TC3) {
      const int kx = base + c;
      const bool colok = kx < HXp;
      if (n1 < R1p) {
        float2 v[R2p];
#pragma unroll
        for (int n2 = 0; n2 < R2p; ++n2) {
          if (n2 >= R2p / 2) {
            v[n2] = make_float2(0.f, 0.f);
          } else {
            const int row = n1 + R1p * n2;
            v[n2] = (colok && row >= a.by0 && row < a.by1) ? B[(row - a.by0) * HXp + kx] : make_float2(0.f, 0.f);
          }
        }
        dft_maybe_half<R2p, false, true>(v);
#pragma unroll
        for (int k2 = 1; k2 < R2p; ++k2) v[k2] = cmul(v[k2], tp[n1 * k2]);
#pragma unroll
        for (int k2 = 0; k2 < R2p; ++k2) Sc3[k2 * S2p + n1 * TC3 + c] = v[k2];
      }
      __syncthreads();
      if (n1 < R2p) {
        const int k2 = n1;
        float2 w[R1p];
#pragma unroll
        for (int m = 0; m < R1p; ++m) w[m] = Sc3[k2 * S2p + m * TC3 + c];
        DFT<R1p, false, float2>::run(w);
        if (colok) {
#pragma unroll
          for (int k1 = 0; k1 < R1p; ++k1) plane[(size_t)(k2 + R2p * k1) * a.sxp + kx] = w[k1];
        }
      }
      __syncthreads();
    }
  }
}

// Shared-memory layout of one launch (complex elements): twiddles | A (box rows x HXu) |
// scratch | B (box rows x HXp); false when the box's rows do not fit.
struct BoxPlan {
  int pr, offA, offS, offB;
  size_t smem;
};

template <int N> bool box_plan(const Launch<float>& L, BoxPlan& P) {
  typedef BoxShape<N> S;
  const Geo& g = L.g;
  const int nbr = L.by1 - L.by0, nbz = L.bz1 - L.bz0;
  if (nbr <= 0 || nbz <= 0 || (nbr & 1) || (L.by0 & 1) || L.by1 > g.ny || L.bz1 > g.nz) return false;
  const int npairs = nbr / 2;
  static const int optin = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
                                                   cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return v;
  }();
  const int nA = nbr * S::HXu, nB = nbr * S::HXp;
  const int s1 = S::R2y * S::S2y, s3 = S::R2p * S::S2p;
  // row pairs per round of step 2: as few rounds as the CTA's pair slots allow, spread evenly
  const int slots = kBoxThreads / S::TP;
  const int rounds = (npairs + slots - 1) / slots;
  P.pr = (npairs + rounds - 1) / rounds;
  const int nS = bmax(bmax(s1, P.pr * S::TT), s3 - nA);
  P.offA = (S::NTW + 1) / 2 * 2;
  P.offS = P.offA + (nA + 1) / 2 * 2;
  P.offB = P.offS + (nS + 1) / 2 * 2;
  P.smem = sizeof(float2) * (size_t)(P.offB + nB);
  return P.smem <= (size_t)optin;
}

template <int N> cudaError_t go_box(const Launch<float>& L, bool chk) {
  BoxPlan P;
  if (!box_plan<N>(L, P)) return cudaErrorNotSupported;
  const Geo& g = L.g;
  auto k = boxpass_kernel<N>;
  allow_smem<boxpass_kernel<N>>();
  BoxArgs a{};
  a.U = L.w->U;
  a.Pd = L.w->Pd;
  a.mask = L.mask;
  a.tw_y = L.w->twu[1];
  a.tw_x = L.w->twu[0];
  a.tw_xp = L.w->twp[0];
  a.tw_yp = L.w->twp[1];
  a.ctrl = L.ctrl;
  a.check_done = chk ? 1 : 0;
  a.nz = g.nz;
  a.sxu = g.sxu;
  a.sxp = g.sxp;
  a.by0 = L.by0;
  a.by1 = L.by1;
  a.bz0 = L.bz0;
  a.bz1 = L.bz1;
  a.pr = P.pr;
  a.offA = P.offA;
  a.offS = P.offS;
  a.offB = P.offB;
  const dim3 grid(3 * (L.bz1 - L.bz0));  // one CTA per (component, plane of the box)
  k<<<grid, kBoxThreads, P.smem, L.st>>>(a);
  return checked_launch("boxpass_kernel", grid, kBoxThreads, P.smem);
}

}  // namespace

bool box_fused_ok(const Launch<float>& L) {
  const Geo& g = L.g;
  if (!L.use_box || g.nx != g.ny) return false;
  BoxPlan P;
  switch (g.nx) {
    case 16: return box_plan<16>(L, P);
    case 32: return box_plan<32>(L, P);
    case 48: return box_plan<48>(L, P);
    case 64: return box_plan<64>(L, P);
    case 96: return box_plan<96>(L, P);
    case 128: return box_plan<128>(L, P);
  }
  return false;
}

cudaError_t launch_box_fused(const Launch<float>& L, bool check_done) {
  if (!L.use_box || L.g.nx != L.g.ny) return cudaErrorNotSupported;
  switch (L.g.nx) {
    case 16: return go_box<16>(L, check_done);
    case 32: return go_box<32>(L, check_done);
    case 48: return go_box<48>(L, check_done);
    case 64: return go_box<64>(L, check_done);
    case 96: return go_box<96>(L, check_done);
    case 128: return go_box<128>(L, check_done);
  }
  return cudaErrorNotSupported;
}

}  // namespace scfft
