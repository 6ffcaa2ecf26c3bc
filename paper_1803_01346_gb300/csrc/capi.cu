// capi.cu - the C ABI of include/scfft.h: context, geometry, kernel-spectrum
// precompute, the right-hand side driver (§2, Eqs. 1-5), the BS23 time
// integrator (the method of lines with "ode23", §2) and per-pass profiling.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "scfft.h"
#include "scfft_internal.cuh"

using namespace scfft;

namespace {
constexpr int kProfPool = 1 << 14;  // event pairs buffered before a flush
}
struct AdjRec;   // a recorded trajectory of the reverse mode (defined with it below)
struct StepDev;  // device state of scfft_advance (defined with it below)
struct PathDev;  // the applied-field path on the device
namespace {
void free_rec(scfft_ctx* c);
}

struct scfft_ctx {
  Geo g{};
  double L[3]{};
  scfft_material mat{};
  scfft_options opt{};
  cudaStream_t st = nullptr;
  Work<float> wf;
  Work<double> wd;
  Work<dfloat> wq;  // double-float FFT passes (SCFFT_PREC_DF64)
  int box[4] = {0, 0, 0, 0};  // bounding box of Omega's nodes: y in [box0, box1) (even), z in [box2, box3)
  Ctrl* ctrl = nullptr;        // device
  PointParams* ppd = nullptr;  // device copy of the current rhs's PointParams
  double* partials = nullptr;  // device
  // FP32 Eq. 5 loop as one CUDA graph: a WHILE conditional node around one iteration
  cudaGraph_t loop_graph = nullptr;
  cudaGraphExec_t loop_exec = nullptr;
  bool loop_failed = false;
  int fault = 0;  // armed fault injection (scfft_inject_fault)
  // FP32 path: Ctrl::iter_total already folded into stats, and whether graph-run rhs calls
  // of the integrator have not been folded in yet (their statistics are read once per step)
  unsigned long long iters_seen = 0;
  bool graph_pending = false;
  uint8_t* mask = nullptr;     // device
  long long nout = 0;
  // curls of the rhs: SCFFT_CURL_SPECTRAL (§2) or SCFFT_CURL_FD (scfft_set_curl)
  int curl_kind = SCFFT_CURL_SPECTRAL;
  double dcell[3]{};  // cell sizes dx, dy, dz
  // e(j, h) law in Omega (scfft_set_ej_law); law = 0 is Eq. 1
  int law = 0;
  double kim_h0 = 0.0;
  double aniso[3] = {1.0, 1.0, 1.0};
  bool have_geom = false, have_kernel = false, have_path = false;
  // field path
  std::vector<double> kt, khe;
  double sin_amp = 0, sin_period = 1, sin_t0 = 0, sin_t1 = 0, sin_dir[3] = {0, 0, 1};
  // host mirror of Ctrl and synchronisation
  Ctrl* hctrl = nullptr;  // pinned, 3 slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // integrator (FP64): ynew, k1..k4, ytmp, internal warm start
  double* ib = nullptr;
  double* k[4] = {nullptr, nullptr, nullptr, nullptr};
  bool fsal_valid = false;
  double fsal_t = 0;
  const double* fsal_h = nullptr;
  const double* fsal_g = nullptr;
  unsigned long long* errbits = nullptr;  // device
  unsigned long long* herr = nullptr;     // pinned
  // FP32-path integrator: stage derivatives, stage state, increment (FP32),
  // candidate state and Kahan compensation of the accepted sums (FP64)
  float* ib32 = nullptr;
  float* k32[4] = {nullptr, nullptr, nullptr, nullptr};
  float* ytmp32 = nullptr;
  float* g32 = nullptr;
  float* d32 = nullptr;
  double* ynew64 = nullptr;
  double* comp64 = nullptr;
  const float* last32 = nullptr;  // output of the most recent rhs (the next warm start)
  // reverse mode: forward j, two cotangent buffers (FP64) and per-block sums of mu_a
  double* adj = nullptr;
  double* adj_part = nullptr;
  double* hadj_part = nullptr;  // pinned
  int adj_part_cap = 0;
  AdjRec* rec = nullptr;  // recorded trajectory of scfft_adjoint_record
  // device-resident stepping (scfft_advance): step state, path, per-stage rhs parameters and
  // the step graph (rebuilt when the buffers it was built on or any setting change)
  StepDev* sdev = nullptr;     // device
  StepDev* hsdev = nullptr;    // pinned host mirror
  PathDev* pathd = nullptr;    // device
  PointParams* ppsd = nullptr; // device, 3 stages
  cudaGraph_t step_graph = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  const double* step_h = nullptr;
  const double* step_warm = nullptr;
  float* step_k[4] = {nullptr, nullptr, nullptr, nullptr};
  unsigned long long step_epoch = 0;
  unsigned long long epoch = 1;  // bumped by every setting the step graph bakes in
  bool path_dirty = true;
  scfft_stats stats{};
  // profiling
  bool prof_on = false;
  std::vector<cudaEvent_t> pev;
  std::vector<int> pkind;
  int pused = 0;
  double pms[SCFFT_NKINDS]{};
  long long pcnt[SCFFT_NKINDS]{};
};

namespace {
// The most recent CUDA error behind an SCFFT_ECUDA (process wide, for diagnostics).
std::mutex g_err_mutex;
char g_err_text[512] = "";
}  // namespace

void scfft::note_cuda_error(cudaError_t e, const char* file, int line) {
  std::lock_guard<std::mutex> lock(g_err_mutex);
  snprintf(g_err_text, sizeof(g_err_text), "%s (%s) at %s:%d; last failed launch: %s", cudaGetErrorName(e),
           cudaGetErrorString(e), file, line, last_launch_failure());
}

namespace {

#define CK(x)                                     \
  do {                                            \
    cudaError_t e_ = (x);                         \
    if (e_ != cudaSuccess) {                      \
      note_cuda_error(e_, "capi.cu", __LINE__);   \
      return SCFFT_ECUDA;                         \
    }                                             \
  } while (0)

#define CS_(x)                            \
  do {                                    \
    scfft_status s_ = (x);                \
    if (s_ != SCFFT_OK) return s_;        \
  } while (0)

int round_up(int a, int m) { return (a + m - 1) / m * m; }

bool grid_ok(int n) { return n == 16 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128; }

template <typename T> Work<T>& work(scfft_ctx* c);
template <> Work<float>& work<float>(scfft_ctx* c) { return c->wf; }
template <> Work<double>& work<double>(scfft_ctx* c) { return c->wd; }
template <> Work<dfloat>& work<dfloat>(scfft_ctx* c) { return c->wq; }

// Calls f with a value of the context's FFT element type: float (SCFFT_PREC_F32), double
// (SCFFT_PREC_F64) or dfloat (SCFFT_PREC_DF64).
template <typename F> auto by_prec(const scfft_ctx* c, F&& f) {
  if (c->opt.precision == SCFFT_PREC_F32) return f(float{});
  if (c->opt.precision == SCFFT_PREC_DF64) return f(dfloat{});
  return f(double{});
}

template <typename T> Launch<T> launch_of(scfft_ctx* c) {
  Launch<T> L;
  L.g = c->g;
  L.w = &work<T>(c);
  L.ctrl = c->ctrl;
  L.mask = c->mask;
  L.partials = c->partials;
  L.ppd = c->ppd;
  L.fault = &c->fault;
  L.st = c->st;
  L.by0 = c->box[0];
  L.by1 = c->box[1];
  L.bz0 = c->box[2];
  L.bz1 = c->box[3];
  return L;
}

// The same launch description with the source box on (the forward passes of an Eq. 5 iteration).
template <typename T> Launch<T> boxed(const Launch<T>& L) {
  Launch<T> B = L;
  B.use_box = B.by1 > B.by0 && B.bz1 > B.bz0;
  return B;
}

// The schedule asks for the fused box passes and they apply to this launch (FP32, nx == ny).
bool box_fused_on(const Launch<float>& L) { return L.w->sched.box_fused && box_fused_ok(L); }

// ---------------------------------------------------------------- profiling
cudaError_t prof_flush(scfft_ctx* c) {
  if (c->pused == 0) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < c->pused; ++i) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, c->pev[2 * i], c->pev[2 * i + 1]) == cudaSuccess) {
      c->pms[c->pkind[i]] += ms;
      c->pcnt[c->pkind[i]] += 1;
    }
  }
  c->pused = 0;
  return cudaSuccess;
}

// Run one kernel launcher, counting it and (when profiling) bracketing it with events.
template <typename F> cudaError_t run(scfft_ctx* c, int kind, F&& f) {
  int slot = -1;
  if (c->prof_on) {
    if (c->pused == kProfPool) {
      cudaError_t e = prof_flush(c);
      if (e != cudaSuccess) return e;
    }
    slot = c->pused++;
    c->pkind[slot] = kind;
    cudaEventRecord(c->pev[2 * slot], c->st);
  }
  cudaError_t e = f();
  if (slot >= 0) cudaEventRecord(c->pev[2 * slot + 1], c->st);
  c->stats.launches += 1;
  return e;
}

// ---------------------------------------------------------------- field path
// dh_e/dt at t (right derivative, or left at a kink when left != 0)
void hedot_at(const scfft_ctx* c, double t, int left, double out[3]) {
  out[0] = out[1] = out[2] = 0;
  const int K = (int)c->kt.size();
  for (int s = 0; s + 1 < K; ++s) {
    const double lo = c->kt[s], hi = c->kt[s + 1];
    const bool in = left ? (lo < t && t <= hi) : (lo <= t && t < hi);
    if (in) {
      for (int a = 0; a < 3; ++a) out[a] = (c->khe[3 * (s + 1) + a] - c->khe[3 * s + a]) / (hi - lo);
      break;
    }
  }
  if (c->sin_amp != 0) {
    const bool in = left ? (c->sin_t0 < t && t <= c->sin_t1) : (c->sin_t0 <= t && t < c->sin_t1);
    if (in) {
      const double w = 2 * M_PI / c->sin_period;
      const double v = c->sin_amp * w * cos(w * (t - c->sin_t0));
      for (int a = 0; a < 3; ++a) out[a] += v * c->sin_dir[a];
    }
  }
}

std::vector<double> kinks_of(const scfft_ctx* c) {
  std::vector<double> k(c->kt.begin(), c->kt.end());
  if (c->sin_amp != 0) {
    k.push_back(c->sin_t0);
    k.push_back(c->sin_t1);
  }
  std::sort(k.begin(), k.end());
  return k;
}

// ---------------------------------------------------------------- workspaces
template <typename T> scfft_status alloc_work(scfft_ctx* c) {
  typedef typename cplx_of<T>::type V;
  Work<T>& w = work<T>(c);
  const Geo& g = c->g;
  const long long N = g.N;
  CK(cudaMalloc(&w.U, sizeof(V) * 3 * (size_t)g.nz * g.ny * g.sxu));
  CK(cudaMalloc(&w.Pd, sizeof(V) * 3 * (size_t)g.nz * 2 * g.ny * g.sxp));
  CK(cudaMalloc(&w.Hd[0], sizeof(T) * 3 * N));
  CK(cudaMalloc(&w.Hd[1], sizeof(T) * 3 * N));
  CK(cudaMalloc(&w.kap, sizeof(T) * 3 * (size_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1)));
  if constexpr (sizeof(T) == 4) CK(cudaMalloc(&w.kap4, sizeof(float4) * (size_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1)));
  const int n[3] = {g.nx, g.ny, g.nz};
  const double sig = c->opt.sigma_scale * 0.5 *
                     sqrt(pow(2 * c->L[0] / g.nx, 2) + pow(2 * c->L[1] / g.ny, 2) + pow(2 * c->L[2] / g.nz, 2));
  for (int a = 0; a < 3; ++a) {
    // derivative wavenumbers k = pi m / L_a (period 2 L_a), 0 on the Nyquist entry; smoothing exp(-sigma^2 k^2/2)
    const int len = a == 0 ? n[0] / 2 + 1 : n[a];
    std::vector<T> kt(len), st(len);
    for (int i = 0; i < len; ++i) {
      const int m = (a == 0) ? i : (i < n[a] / 2 ? i : i - n[a]);
      const double k = M_PI * m / c->L[a];
      kt[i] = (i == n[a] / 2) ? (T)0 : (T)k;
      st[i] = (T)exp(-0.5 * sig * sig * k * k);
    }
    CK(cudaMalloc(&w.kt[a], sizeof(T) * len));
    CK(cudaMalloc(&w.st[a], sizeof(T) * len));
    CK(cudaMemcpy(w.kt[a], kt.data(), sizeof(T) * len, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(w.st[a], st.data(), sizeof(T) * len, cudaMemcpyHostToDevice));
    for (int pad = 0; pad < 2; ++pad) {
      const int Lt = pad ? 2 * n[a] : n[a];
      std::vector<V> tw(Lt);
      for (int m = 0; m < Lt; ++m) {
        const long double ang = 2.0L * 3.14159265358979323846264338327950288L * m / Lt;
        V v;
        v.x = (T)cosl(ang);
        v.y = (T)(-sinl(ang));
        tw[m] = v;
      }
      V** dst = pad ? &w.twp[a] : &w.twu[a];
      CK(cudaMalloc(dst, sizeof(V) * Lt));
      CK(cudaMemcpy(*dst, tw.data(), sizeof(V) * Lt, cudaMemcpyHostToDevice));
    }
  }
  // FP32: descriptors for the TMA-fed y passes (without them the y passes load directly)
  if constexpr (sizeof(T) == 4) {
    if (!make_ymaps(w, g)) w.ym = nullptr;
  }
  return SCFFT_OK;
}

template <typename T> void free_work(Work<T>& w) {
  cudaFree(w.U); cudaFree(w.Pd); cudaFree(w.Hd[0]); cudaFree(w.Hd[1]); cudaFree(w.jc); cudaFree(w.kap); cudaFree(w.kap4);
  delete w.ym;
  cudaFree(w.Jd);
  for (int a = 0; a < 3; ++a) { cudaFree(w.kt[a]); cudaFree(w.st[a]); cudaFree(w.twu[a]); cudaFree(w.twp[a]); }
  w = Work<T>();
}

PointParams base_params(const scfft_ctx* c) {
  PointParams pp{};
  pp.n = c->mat.n;
  pp.e0 = c->mat.e0;
  pp.jc = c->mat.jc;
  pp.rho_out = c->mat.rho_out;
  pp.inv_mu0 = 1.0 / c->mat.mu0;
  pp.inv_nout = c->nout > 0 ? 1.0 / (double)c->nout : 0.0;
  pp.max_iter = c->opt.max_iter;
  pp.law = c->law;
  pp.kim_h0 = c->kim_h0;
  for (int a = 0; a < 3; ++a) pp.aniso[a] = c->aniso[a];
  return pp;
}

// ---------------------------------------------------------------- rhs
// Spectral curl of the half spectrum held in U: y fwd, z (fwd, curl, inv), y inv.
template <typename T> cudaError_t curl_in_U(scfft_ctx* c, const Launch<T>& L, bool check_done) {
  cudaError_t e;
  if ((e = run(c, SCFFT_K_Y_FWD_U, [&] { return launch_y<T>(L, false, false, check_done); })) != cudaSuccess) return e;
  if ((e = run(c, SCFFT_K_Z_CURL, [&] { return launch_z_curl<T>(L, check_done, 1.0 / (double)L.g.N); })) !=
      cudaSuccess)
    return e;
  return run(c, SCFFT_K_Y_INV_U, [&] { return launch_y<T>(L, false, true, check_done); });
}

// One iteration of Eq. 5 (the i-th): U holds R2C_x of dh^i on entry and of dh^{i+1} on exit.
// The masked stencil curl of the iterate and the zero-padded R2C of it (local-stencil curl option).
template <typename T> cudaError_t fd_maskpad(scfft_ctx* c, const Launch<T>& L, const PointParams& pp, bool chk) {
  cudaError_t e;
  if ((e = run(c, SCFFT_K_Z_CURL, [&] { return launch_fd_curl_mask<T>(L, L.w->Jd, c->dcell, chk); })) != cudaSuccess)
    return e;
  return run(c, SCFFT_K_X_MASKPAD, [&] {
    if constexpr (sizeof(T) == 4)
      return launch_x_reg_io(L, X_PAD_F64, pp, nullptr, L.w->Jd, nullptr, nullptr, nullptr, 0, 0, chk);
    else
      return launch_x_pad_rows<T>(L, pp, L.w->Jd, chk);
  });
}

template <typename T> cudaError_t iteration(scfft_ctx* c, const Launch<T>& L, PointParams pp, int i, bool chk) {
  cudaError_t e;
  const bool fd = c->curl_kind == SCFFT_CURL_FD;
  const Launch<T> LB = boxed(L);  // the source chi curl dh^i vanishes outside Omega's box
  bool fused = false;              // FP32: the three passes on Omega's box as one launch
  if (fd) {
    if ((e = fd_maskpad<T>(c, L, pp, chk)) != cudaSuccess) return e;
  } else {
    // the curl of dh^i: forward over the whole grid; its z output and the inverse y pass only
    // where the mask keeps it (Omega's box)
    if ((e = run(c, SCFFT_K_Y_FWD_U, [&] { return launch_y<T>(L, false, false, chk); })) != cudaSuccess) return e;
    if ((e = run(c, SCFFT_K_Z_CURL, [&] { return launch_z_curl<T>(LB, chk, 1.0 / (double)L.g.N); })) !=
        cudaSuccess)
      return e;
    if constexpr (std::is_same<T, float>::value) {
      fused = box_fused_on(LB);
      // the curl's inverse y pass, the mask/pad x pass and the padded forward y pass, fused
      if (fused && (e = run(c, SCFFT_K_BOX, [&] { return launch_box_fused(LB, chk); })) != cudaSuccess) return e;
    }
    if (!fused) {
      if ((e = run(c, SCFFT_K_Y_INV_U, [&] { return launch_y<T>(LB, false, true, chk); })) != cudaSuccess) return e;
      if ((e = run(c, SCFFT_K_X_MASKPAD,
                   [&] { return launch_x<T>(LB, X_MASKPAD, pp, nullptr, nullptr, nullptr, 0, 0, chk); })) !=
          cudaSuccess)
        return e;
    }
  }
  if (!fused && (e = run(c, SCFFT_K_Y_FWD_P, [&] { return launch_y<T>(LB, true, false, chk); })) != cudaSuccess)
    return e;
  if ((e = run(c, SCFFT_K_Z_KERNEL, [&] { return launch_z_kernel<T>(LB, chk); })) != cudaSuccess) return e;
  if ((e = run(c, SCFFT_K_Y_INV_P, [&] { return launch_y<T>(L, true, true, chk); })) != cudaSuccess) return e;
  pp.iter = i;
  return run(c, SCFFT_K_X_UPDATE, [&] {
    return launch_x<T>(L, fd ? X_UPDATE_FD : X_UPDATE, pp, nullptr, nullptr, nullptr, i & 1, (i + 1) & 1, chk);
  });
}

// ---------------------------------------------------------------- Eq. 5 loop as a CUDA graph
// The FP32 path runs the whole Eq. 5 iteration loop of one rhs as one graph launch: a WHILE
// conditional node whose body is one iteration (the eight passes) followed by a one-thread
// kernel that sets the loop condition from the device flags (stop reached, status,
// iteration cap).  No iteration is queued past convergence and the host takes no part
// in the loop.  The update pass reads its iteration index and the rhs parameters from
// device memory, so the captured launches stay valid for every rhs of the context.
__global__ void loop_cond_kernel(cudaGraphConditionalHandle h, Ctrl* ctrl, int max_iter) {
  // the trip count bounds the loop by itself, whatever the update pass did
  const unsigned trips = ++ctrl->trips;
  const unsigned go =
      (ctrl->done == 0 && ctrl->status == 0 && ctrl->iters < max_iter && trips < (unsigned)max_iter) ? 1u : 0u;
  cudaGraphSetConditional(h, go);
}

constexpr int kLoopLaunches = 9;    // kernels per iteration of the graph body
constexpr int kLoopLaunchesBox = 7; // the same with the fused box passes
constexpr int kLoopLaunchesFd = 7;  // the same with the local-stencil curl

cudaError_t loop_body(const Launch<float>& L, const PointParams& pp, cudaGraphConditionalHandle h, int max_iter,
                      bool fd, const double* dcell) {
  cudaError_t e;
  bool fused = false;
  if (fd) {
    if ((e = launch_fd_curl_mask<float>(L, L.w->Jd, dcell, false)) != cudaSuccess) return e;
    if ((e = launch_x_reg_io(L, X_PAD_F64, pp, nullptr, L.w->Jd, nullptr, nullptr, nullptr, 0, 0, false)) !=
        cudaSuccess)
      return e;
  } else {
    if ((e = launch_y<float>(L, false, false, false)) != cudaSuccess) return e;
    if ((e = launch_z_curl<float>(boxed(L), false, 1.0 / (double)L.g.N)) != cudaSuccess) return e;
    fused = box_fused_on(boxed(L));
    if (fused) {
      if ((e = launch_box_fused(boxed(L), false)) != cudaSuccess) return e;
    } else {
      if ((e = launch_y<float>(boxed(L), false, true, false)) != cudaSuccess) return e;
      if ((e = launch_x<float>(boxed(L), X_MASKPAD, pp, nullptr, nullptr, nullptr, 0, 0, false)) != cudaSuccess)
        return e;
    }
  }
  if (!fused && (e = launch_y<float>(boxed(L), true, false, false)) != cudaSuccess) return e;
  if ((e = launch_z_kernel<float>(boxed(L), false)) != cudaSuccess) return e;
  if ((e = launch_y<float>(L, true, true, false)) != cudaSuccess) return e;
  if ((e = launch_x<float>(L, fd ? X_UPDATE_FD : X_UPDATE, pp, nullptr, nullptr, nullptr, 0, 1, false)) != cudaSuccess)
    return e;
  loop_cond_kernel<<<1, 1, 0, L.st>>>(h, L.ctrl, max_iter);
  return cudaGetLastError();
}

// Build the loop graph once per context; false (and the host-driven loop) if the driver
// refuses any step.
bool loop_graph_ready(scfft_ctx* c) {
  if (c->loop_exec) return true;
  if (c->loop_failed) return false;
  c->loop_failed = true;  // until the build succeeds
  // capture on a private stream: the context's stream may be the legacy default stream,
  // which cannot be captured; the graph itself is launched on the context's stream
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  Launch<float> L = launch_of<float>(c);
  L.st = cs;
  L.fault = nullptr;  // a fault is never captured into the loop graph
  const PointParams pp = base_params(c);
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaGraphConditionalHandle h{};
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams np{};
  cudaGraphNode_t node{};
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (ok) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
      const bool launched =
          loop_body(L, pp, h, c->opt.max_iter, c->curl_kind == SCFFT_CURL_FD, c->dcell) == cudaSuccess;
      cudaGraph_t captured = nullptr;
      ok = cudaStreamEndCapture(cs, &captured) == cudaSuccess && launched;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  cudaStreamDestroy(cs);
  if (!ok) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // clear the (non-sticky) error of the refused step; the host-driven loop takes over
    return false;
  }
  c->loop_graph = g;
  c->loop_exec = ex;
  c->loop_failed = false;
  return true;
}

// Inputs and outputs of one rhs: FP64 arrays (public entry points, the FP64
// integrator) or FP32 arrays (stages of the FP32 integrator).
struct RhsIO {
  const double* h64 = nullptr;
  const float* h32 = nullptr;
  const double* warm64 = nullptr;
  const float* warm32 = nullptr;
  double* out64 = nullptr;       // dh/dt
  double* warm_out64 = nullptr;  // dh/dt again, as the next warm start
  float* out32 = nullptr;
};

__global__ void finalize_f32_kernel(const float* __restrict__ h0, const float* __restrict__ h1, const Ctrl* ctrl,
                                    float* __restrict__ out, long long n3) {
  const float* src = ctrl->cur ? h1 : h0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    out[i] = src[i];
}

template <typename T>
cudaError_t x_io(const Launch<T>& L, XMode mode, const PointParams& pp, const RhsIO& io) {
  if constexpr (sizeof(T) == 4)
    return launch_x_reg_io(L, mode, pp, io.h64, io.h32, nullptr, io.warm64, io.warm32, 0, 0, false);
  else
    return launch_x<T>(L, mode, pp, io.h64, nullptr, io.warm64, 0, 0, false);
}

// FP32 path: fold the device's iteration counter into the host statistics (graph-run
// iterations also count their kLoopLaunches kernels here).
void absorb_ctrl(scfft_ctx* c, const Ctrl& hc, bool graph_iters) {
  const unsigned long long d = hc.iter_total - c->iters_seen;
  c->iters_seen = hc.iter_total;
  c->stats.iterations += (long long)d;
  if (graph_iters)
    c->stats.launches += (long long)(c->curl_kind == SCFFT_CURL_FD     ? kLoopLaunchesFd
                                     : box_fused_on(boxed(launch_of<float>(c))) ? kLoopLaunchesBox
                                                                                : kLoopLaunches) *
                         (long long)d;
  c->stats.last_iters = hc.iters;
  c->stats.last_residual = hc.residual;
  c->graph_pending = false;
}

// Read the device control block (synchronising the stream) and fold in the statistics of
// graph-run rhs calls that have not been read yet; returns the latched device status.
scfft_status flush_pending(scfft_ctx* c) {
  if (!c->graph_pending) return SCFFT_OK;
  CK(cudaMemcpyAsync(c->hctrl + 2, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  const Ctrl hc = c->hctrl[2];
  absorb_ctrl(c, hc, true);
  return (scfft_status)hc.status;
}

// defer (the FP32 integrator's stages): when the loop runs as a graph and the caller wants
// no iteration count, return without reading the device state back; the step reads it once.
template <typename T>
scfft_status rhs_impl(scfft_ctx* c, double t, int left, const RhsIO& io, int* iters_out, bool defer = false) {
  if constexpr (sizeof(T) == 4) {
    if (c->graph_pending && !(defer && !iters_out && !c->prof_on)) CS_(flush_pending(c));
  }
  Launch<T> L = launch_of<T>(c);
  PointParams pp = base_params(c);
  hedot_at(c, t, left, pp.hedot);
  const double hn = sqrt(pp.hedot[0] * pp.hedot[0] + pp.hedot[1] * pp.hedot[1] + pp.hedot[2] * pp.hedot[2]);
  pp.tol = c->opt.delta_it * (hn > 1.0 ? hn : 1.0);
  // pre-stage: j = curl h; e = rho(j) j; dh^0 = -curl e / mu0 on Omega, warm on Omega_out
  if (c->curl_kind == SCFFT_CURL_FD) {
    // two stencil passes: e (into the second iterate buffer, free here), then dh^0
    T* ebuf = L.w->Hd[1];
    CK(run(c, SCFFT_K_X_POWERLAW, [&] {
      if constexpr (sizeof(T) == 4) return launch_fd_efield<T>(L, pp, io.h64, io.h32, c->dcell, ebuf);
      else return launch_fd_efield<T>(L, pp, io.h64, nullptr, c->dcell, ebuf);
    }));
    CK(run(c, SCFFT_K_X_ASSEMBLE, [&] {
      if constexpr (sizeof(T) == 4) return launch_fd_assemble<T>(L, pp, ebuf, io.warm64, io.warm32, c->dcell);
      else return launch_fd_assemble<T>(L, pp, ebuf, io.warm64, nullptr, c->dcell);
    }));
  } else {
    CK(run(c, SCFFT_K_X_FWD, [&] { return x_io<T>(L, X_FWD_F64, pp, io); }));
    CK(curl_in_U<T>(c, L, false));
    if (c->law) {  // the e(j, h) law reads the state h at each node
      CK(run(c, SCFFT_K_X_POWERLAW, [&] { return x_io<T>(L, X_POWERLAW_H, pp, io); }));
    } else {
      CK(run(c, SCFFT_K_X_POWERLAW,
             [&] { return launch_x<T>(L, X_POWERLAW, pp, nullptr, nullptr, nullptr, 0, 0, false); }));
    }
    CK(curl_in_U<T>(c, L, false));
    CK(run(c, SCFFT_K_X_ASSEMBLE, [&] { return x_io<T>(L, X_ASSEMBLE, pp, io); }));
  }
  const int maxit = c->opt.max_iter;
  const bool early = c->opt.delta_it > 0 && c->nout > 0;
  int launched = 0;
  bool graphed = false;
  if constexpr (sizeof(T) == 4) {
    if (c->nout > 0 && maxit > 0 && !c->prof_on && loop_graph_ready(c)) {
      CK(cudaGraphLaunch(c->loop_exec, c->st));
      graphed = true;
    }
  }
  if (c->nout > 0 && !graphed) {
    // With an early stop the host keeps one iteration queued ahead: before
    // queueing iteration i it waits for the flag copied after iteration i-2.
    // An iteration queued after convergence returns at entry (device flag), so
    // at most one iteration of launches is wasted.  (While profiling, the host
    // waits for iteration i-1 instead, so that every profiled launch does real
    // work.)
    const int ahead = c->prof_on ? 1 : 2;
    for (int i = 0; i < maxit; ++i) {
      if (early && i >= ahead) {
        CK(cudaEventSynchronize(c->ev[(i - ahead) & 1]));
        if (c->hctrl[(i - ahead) & 1].done) break;
      }
      CK(iteration<T>(c, L, pp, i, early));
      ++launched;
      if (early) {
        CK(cudaMemcpyAsync(&c->hctrl[i & 1], c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->st));
        CK(cudaEventRecord(c->ev[i & 1], c->st));
      }
    }
  }
  if (io.out32) {
    if constexpr (sizeof(T) == 4) {
      const long long n3 = 3 * c->g.N;
      const Work<float>& w = c->wf;
      CK(run(c, SCFFT_K_FINALIZE, [&] {
        finalize_f32_kernel<<<(int)std::min<long long>((n3 + 255) / 256, 152 * 8), 256, 0, c->st>>>(
            w.Hd[0], w.Hd[1], c->ctrl, io.out32, n3);
        return cudaGetLastError();
      }));
    } else {
      return SCFFT_EINVAL;
    }
  } else {
    CK(run(c, SCFFT_K_FINALIZE, [&] { return launch_finalize<T>(L, io.out64, io.warm_out64); }));
  }
  c->stats.rhs_calls += 1;
  if (graphed && defer && !iters_out) {
    c->graph_pending = true;
    return SCFFT_OK;
  }
  if (iters_out || early || graphed) {
    CK(cudaMemcpyAsync(c->hctrl + 2, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const Ctrl hc = c->hctrl[2];
    if constexpr (sizeof(T) == 4) {
      absorb_ctrl(c, hc, graphed);
    } else {
      c->stats.iterations += hc.iters;
      c->stats.last_iters = hc.iters;
      c->stats.last_residual = hc.residual;
    }
    if (iters_out) *iters_out = hc.iters;
    if (hc.status != 0) return (scfft_status)hc.status;
    if (iters_out && c->nout > 0 && maxit > 0 && !(hc.residual < pp.tol) && c->opt.delta_it > 0)
      return SCFFT_ENOCONV;
  } else {
    c->stats.iterations += launched;
    c->stats.last_iters = launched;
    if constexpr (sizeof(T) == 4) c->iters_seen += (unsigned long long)launched;  // no early stop: all ran
  }
  return SCFFT_OK;
}

scfft_status rhs_any(scfft_ctx* c, double t, int left, const double* h, double* warm, double* hdot, int* it) {
  RhsIO io;
  io.h64 = h;
  io.warm64 = warm;
  io.out64 = hdot;
  io.warm_out64 = warm;
  return by_prec(c, [&](auto z) { return rhs_impl<decltype(z)>(c, t, left, io, it); });
}

template <typename T> scfft_status curl_impl(scfft_ctx* c, const double* f, double* out) {
  Launch<T> L = launch_of<T>(c);
  PointParams pp = base_params(c);
  CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_FWD_F64, pp, f, nullptr, nullptr, 0, 0, false); }));
  CK(curl_in_U<T>(c, L, false));
  CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_TO_F64, pp, nullptr, out, nullptr, 0, 0, false); }));
  return SCFFT_OK;
}

template <typename T> scfft_status phi_impl(scfft_ctx* c, const double* j, double* out) {
  Launch<T> L = launch_of<T>(c);
  PointParams pp = base_params(c);
  CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_PAD_F64, pp, j, nullptr, nullptr, 0, 0, false); }));
  CK(run(c, SCFFT_K_Y_FWD_P, [&] { return launch_y<T>(L, true, false, false); }));
  CK(run(c, SCFFT_K_Z_KERNEL, [&] { return launch_z_kernel<T>(L, false); }));
  CK(run(c, SCFFT_K_Y_INV_P, [&] { return launch_y<T>(L, true, true, false); }));
  CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_CROP_F64, pp, nullptr, out, nullptr, 0, 0, false); }));
  return SCFFT_OK;
}

// ---------------------------------------------------------------- BS23 (FP64 state)
__global__ void combine_kernel(double* __restrict__ out, const double* __restrict__ y, double h, double c1,
                               const double* __restrict__ k1, double c2, const double* __restrict__ k2, double c3,
                               const double* __restrict__ k3, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = c1 * k1[i];
    if (k2) s += c2 * k2[i];
    if (k3) s += c3 * k3[i];
    out[i] = y[i] + h * s;
  }
}

// err_i = h (e1 k1 + e2 k2 + e3 k3 + e4 k4); norm = max_i |err_i| / max(rtol|y|, rtol|ynew|, atol)
// (a max is order independent, so the atomic combine is deterministic)
__global__ void errnorm_kernel(const double* __restrict__ y, const double* __restrict__ yn, double h, double e1,
                               const double* __restrict__ k1, double e2, const double* __restrict__ k2, double e3,
                               const double* __restrict__ k3, double e4, const double* __restrict__ k4, double rtol,
                               double atol, long long n, unsigned long long* out) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double e = h * (e1 * k1[i] + e2 * k2[i] + e3 * k3[i] + e4 * k4[i]);
    const double w = fmax(fmax(rtol * fabs(y[i]), rtol * fabs(yn[i])), atol);
    const double r = fabs(e) / w;
    m = (r > m || r != r) ? r : m;  // NaN propagates
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double q = __shfl_xor_sync(0xffffffffu, m, o);
    m = (q > m || q != q) ? q : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void fill3_kernel(double* __restrict__ g, double a, double b, double c, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    g[i] = a; g[N + i] = b; g[2 * N + i] = c;
  }
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(b, 1), 152 * 8);
}

scfft_status ensure_rk(scfft_ctx* c) {
  if (c->ib) return SCFFT_OK;
  const long long n3 = 3 * c->g.N;
  if (cudaMalloc(&c->ib, sizeof(double) * 7 * n3) != cudaSuccess) return SCFFT_ENOMEM;
  for (int i = 0; i < 4; ++i) c->k[i] = c->ib + (1 + i) * n3;
  return SCFFT_OK;
}

// One accepted BS23 step from *t (rejected trials are retried with a smaller
// step).  The step never passes tstop nor a kink of the path and ends exactly
// on them when clipped.  dt_fixed > 0: take exactly that step (clipped the
// same way) with no error control.  FSAL: the first stage is reused from the
// previous accepted step of the same (h, g) unless that step ended on a kink.
scfft_status bs23_step(scfft_ctx* c, double* t_io, double* dt_io, double tstop, double* h, double* g,
                       double dt_fixed, int* rej_out) {
  CS_(ensure_rk(c));
  const long long n3 = 3 * c->g.N;
  double* ynew = c->ib;
  double* ytmp = c->ib + 5 * n3;
  double** k = c->k;
  const double t = *t_io;
  double dt = dt_fixed > 0 ? dt_fixed : *dt_io;
  const std::vector<double> kinks = kinks_of(c);
  double nxt = tstop;
  for (double v : kinks)
    if (v > t && v < nxt) nxt = v;
  if (!(c->fsal_valid && c->fsal_t == t && c->fsal_h == h && c->fsal_g == g)) {
    CS_(rhs_any(c, t, 0, h, g, k[0], nullptr));
  }
  // Bogacki-Shampine 3(2): c = (0, 1/2, 3/4, 1); a21 = 1/2; a31 = 0, a32 = 3/4;
  // b = (2/9, 1/3, 4/9, 0); bhat = (7/24, 1/4, 1/3, 1/8); e = b - bhat
  const double a21 = 0.5, a32 = 0.75, b1 = 2.0 / 9.0, b2 = 1.0 / 3.0, b3 = 4.0 / 9.0;
  const double e1 = 2.0 / 9.0 - 7.0 / 24.0, e2 = 1.0 / 3.0 - 0.25, e3 = 4.0 / 9.0 - 1.0 / 3.0, e4 = -0.125;
  const int blocks = blocks_for(n3);
  int rej = 0;
  for (;;) {
    const double hs = std::min(dt, nxt - t);
    const bool hits = (hs == nxt - t);
    const bool end_left = hits && std::binary_search(kinks.begin(), kinks.end(), nxt);
    if (!(hs > 1e-14 * std::max(1.0, fabs(t)))) {
      c->fsal_valid = false;
      return SCFFT_ESTEP;
    }
    CK(run(c, SCFFT_K_RK, [&] {
      combine_kernel<<<blocks, 256, 0, c->st>>>(ytmp, h, hs, a21, k[0], 0, nullptr, 0, nullptr, n3);
      return cudaGetLastError();
    }));
    CS_(rhs_any(c, t + 0.5 * hs, 0, ytmp, g, k[1], nullptr));
    CK(run(c, SCFFT_K_RK, [&] {
      combine_kernel<<<blocks, 256, 0, c->st>>>(ytmp, h, hs, 0.0, k[0], a32, k[1], 0, nullptr, n3);
      return cudaGetLastError();
    }));
    CS_(rhs_any(c, t + 0.75 * hs, 0, ytmp, g, k[2], nullptr));
    CK(run(c, SCFFT_K_RK, [&] {
      combine_kernel<<<blocks, 256, 0, c->st>>>(ynew, h, hs, b1, k[0], b2, k[1], b3, k[2], n3);
      return cudaGetLastError();
    }));
    CS_(rhs_any(c, hits ? nxt : t + hs, end_left ? 1 : 0, ynew, g, k[3], nullptr));
    double en = 0.0;
    if (!(dt_fixed > 0)) {
      CK(cudaMemsetAsync(c->errbits, 0, sizeof(unsigned long long), c->st));
      CK(run(c, SCFFT_K_RK, [&] {
        errnorm_kernel<<<blocks, 256, 0, c->st>>>(h, ynew, hs, e1, k[0], e2, k[1], e3, k[2], e4, k[3], c->opt.rtol,
                                                 c->opt.atol, n3, c->errbits);
        return cudaGetLastError();
      }));
      CK(cudaMemcpyAsync(c->herr, c->errbits, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      const unsigned long long bits = *c->herr;
      memcpy(&en, &bits, sizeof(double));
      if (!(en == en)) {
        c->fsal_valid = false;
        return SCFFT_ENONFINITE;
      }
    }
    if (en <= 1.0) {
      const double tn = hits ? nxt : t + hs;
      CK(cudaMemcpyAsync(h, ynew, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->st));
      c->stats.accepted += 1;
      if (end_left) {
        c->fsal_valid = false;  // the next first stage takes the right derivative at the kink
      } else {
        std::swap(k[0], k[3]);
        c->fsal_valid = true;
        c->fsal_t = tn;
        c->fsal_h = h;
        c->fsal_g = g;
      }
      *t_io = tn;
      if (dt_fixed > 0) {
        *dt_io = dt_fixed;
      } else {
        const double fac = en == 0.0 ? 5.0 : std::min(5.0, std::max(0.2, 0.9 * pow(en, -1.0 / 3.0)));
        *dt_io = hs * fac;
      }
      if (rej_out) *rej_out = rej;
      c->stats.t = tn;
      c->stats.dt = *dt_io;
      return SCFFT_OK;
    }
    ++rej;
    c->stats.rejected += 1;
    dt = hs * std::max(0.2, 0.9 * pow(en, -1.0 / 3.0));
  }
}

// ---------------------------------------------------------------- BS23, FP32 FFT path
// Stage derivatives and stage states are FP32 (the precision the FP32 rhs
// produces and consumes); the accepted state stays FP64 and its sums are
// compensated (Kahan), so no per-element FP64 arithmetic beyond one add and the
// compensation update runs per step.
__global__ void combine32_kernel(float* __restrict__ out, const double* __restrict__ y, float h, float c1,
                                 const float* __restrict__ k1, float c2, const float* __restrict__ k2, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = c1 * k1[i];
    if (k2) s += c2 * k2[i];
    out[i] = (float)y[i] + h * s;
  }
}

// ynew = y + d with d = h (b1 k1 + b2 k2 + b3 k3) (d kept for the compensated accept)
__global__ void candidate32_kernel(double* __restrict__ ynew, float* __restrict__ d, const double* __restrict__ y,
                                   float h, float b1, const float* __restrict__ k1, float b2,
                                   const float* __restrict__ k2, float b3, const float* __restrict__ k3, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float di = h * (b1 * k1[i] + b2 * k2[i] + b3 * k3[i]);
    d[i] = di;
    ynew[i] = y[i] + (double)di;
  }
}

// |v| as a float from the high word of the double alone (exponent re-biased, the top 20
// mantissa bits kept, so relative error below 2^-20; 0 below the float range, inf above):
// integer work instead of an FP64-to-FP32 conversion, for the error norm's weights only.
__device__ __forceinline__ float abs_f32_of(double v) {
  const int hi = __double2hiint(v);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  if (e <= 0) return 0.f;
  if (e >= 255) return __int_as_float(0x7f800000);
  return __int_as_float((e << 23) | ((hi & 0xfffff) << 3));
}

// max_i |h sum_j e_j k_j| / max(rtol |y|, rtol |ynew|, atol), FP32; nonnegative
// float bit patterns order like the floats, so an integer max combines them
__global__ void errnorm32_kernel(const double* __restrict__ y, const double* __restrict__ yn, float h, float e1,
                                 const float* __restrict__ k1, float e2, const float* __restrict__ k2, float e3,
                                 const float* __restrict__ k3, float e4, const float* __restrict__ k4, float rtol,
                                 float atol, long long n, unsigned* out) {
  float m = 0.f;
  auto one = [&](double yv, double ynv, float a1, float a2, float a3, float a4) {
    const float e = h * (e1 * a1 + e2 * a2 + e3 * a3 + e4 * a4);
    const float w = fmaxf(rtol * fmaxf(abs_f32_of(yv), abs_f32_of(ynv)), atol);
    const float r = fabsf(e) / w;
    m = (r > m || r != r) ? r : m;
  };
  const long long stride = (long long)gridDim.x * blockDim.x, t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // (two elements per thread and trip with 16- and 8-byte loads where every array allows it)
  const bool vec = (((uintptr_t)y | (uintptr_t)yn) & 15) == 0 &&
                   (((uintptr_t)k1 | (uintptr_t)k2 | (uintptr_t)k3 | (uintptr_t)k4) & 7) == 0;
  long long i0 = 0;
  if (vec) {
    for (long long i = t0; i < n / 2; i += stride) {
      const double2 yv = reinterpret_cast<const double2*>(y)[i], nv = reinterpret_cast<const double2*>(yn)[i];
      const float2 a = reinterpret_cast<const float2*>(k1)[i], b = reinterpret_cast<const float2*>(k2)[i];
      const float2 cc = reinterpret_cast<const float2*>(k3)[i], dd = reinterpret_cast<const float2*>(k4)[i];
      one(yv.x, nv.x, a.x, b.x, cc.x, dd.x);
      one(yv.y, nv.y, a.y, b.y, cc.y, dd.y);
    }
    i0 = n / 2 * 2;
  }
  for (long long i = i0 + t0; i < n; i += stride) one(y[i], yn[i], k1[i], k2[i], k3[i], k4[i]);
  for (int o = 16; o > 0; o >>= 1) {
    const float q = __shfl_xor_sync(0xffffffffu, m, o);
    m = (q > m || q != q) ? q : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// accept: y <- y + d with Kahan compensation c; and the caller's FP64 warm start <- the
// latest rhs result (FP32)
__device__ __forceinline__ void accept_one(double& y, double& c, float d, float last, double& warm) {
  const double u = (double)d - c;
  const double t = y + u;
  c = (t - y) - u;
  y = t;
  warm = (double)last;
}
// (two elements per thread and trip with 16- and 8-byte loads where every array allows it)
__global__ void accept32_kernel(double* __restrict__ y, double* __restrict__ c, const float* __restrict__ d,
                                const float* __restrict__ last, double* __restrict__ warm, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x, t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool vec = (((uintptr_t)y | (uintptr_t)c | (uintptr_t)warm) & 15) == 0 && (((uintptr_t)d | (uintptr_t)last) & 7) == 0;
  long long i0 = 0;
  if (vec) {
    double2* y2 = reinterpret_cast<double2*>(y);
    double2* c2 = reinterpret_cast<double2*>(c);
    double2* w2 = reinterpret_cast<double2*>(warm);
    const float2* d2 = reinterpret_cast<const float2*>(d);
    const float2* l2 = reinterpret_cast<const float2*>(last);
    for (long long i = t0; i < n / 2; i += stride) {
      double2 yv = y2[i], cv = c2[i], wv;
      const float2 dv = d2[i], lv = l2[i];
      accept_one(yv.x, cv.x, dv.x, lv.x, wv.x);
      accept_one(yv.y, cv.y, dv.y, lv.y, wv.y);
      y2[i] = yv;
      c2[i] = cv;
      w2[i] = wv;
    }
    i0 = n / 2 * 2;
  }
  for (long long i = i0 + t0; i < n; i += stride) accept_one(y[i], c[i], d[i], last[i], warm[i]);
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

scfft_status ensure_rk32(scfft_ctx* c) {
  if (c->ib32) return SCFFT_OK;
  const long long n3 = 3 * c->g.N;
  if (cudaMalloc(&c->ib32, sizeof(float) * 7 * n3) != cudaSuccess) return SCFFT_ENOMEM;
  if (cudaMalloc(&c->ynew64, sizeof(double) * 2 * n3) != cudaSuccess) return SCFFT_ENOMEM;
  for (int i = 0; i < 4; ++i) c->k32[i] = c->ib32 + i * n3;
  c->ytmp32 = c->ib32 + 4 * n3;
  c->g32 = c->ib32 + 5 * n3;
  c->d32 = c->ib32 + 6 * n3;
  c->comp64 = c->ynew64 + n3;
  return SCFFT_OK;
}

scfft_status rhs32(scfft_ctx* c, double t, int left, const double* h64, const float* h32, const float* warm32,
                   float* out) {
  RhsIO io;
  io.h64 = h64;
  io.h32 = h32;
  io.warm32 = warm32;
  io.out32 = out;
  scfft_status s = rhs_impl<float>(c, t, left, io, nullptr, true);
  c->last32 = out;
  return s;
}

// One accepted BS23 step of the FP32 path (same control as bs23_step).
scfft_status bs23_step_f32(scfft_ctx* c, double* t_io, double* dt_io, double tstop, double* h, double* warm,
                           double dt_fixed, int* rej_out) {
  CS_(ensure_rk32(c));
  const long long n3 = 3 * c->g.N;
  float** k = c->k32;
  const double t = *t_io;
  double dt = dt_fixed > 0 ? dt_fixed : *dt_io;
  const std::vector<double> kinks = kinks_of(c);
  double nxt = tstop;
  for (double v : kinks)
    if (v > t && v < nxt) nxt = v;
  const int blocks = blocks_for(n3);
  if (!(c->fsal_valid && c->fsal_t == t && c->fsal_h == h && c->fsal_g == warm)) {
    // new trajectory (or the caller changed h / warm): warm start from the caller,
    // fresh first stage, compensation reset
    CK(run(c, SCFFT_K_RK, [&] {
      f64_to_f32_kernel<<<blocks, 256, 0, c->st>>>(warm, c->g32, n3);
      return cudaGetLastError();
    }));
    CK(cudaMemsetAsync(c->comp64, 0, sizeof(double) * n3, c->st));
    CS_(rhs32(c, t, 0, h, nullptr, c->g32, k[0]));
  }
  const float a21 = 0.5f, a32 = 0.75f, b1 = 2.0f / 9.0f, b2 = 1.0f / 3.0f, b3 = 4.0f / 9.0f;
  const float e1 = (float)(2.0 / 9.0 - 7.0 / 24.0), e2 = (float)(1.0 / 3.0 - 0.25),
              e3 = (float)(4.0 / 9.0 - 1.0 / 3.0), e4 = -0.125f;
  int rej = 0;
  for (;;) {
    const double hs = std::min(dt, nxt - t);
    const bool hits = (hs == nxt - t);
    const bool end_left = hits && std::binary_search(kinks.begin(), kinks.end(), nxt);
    if (!(hs > 1e-14 * std::max(1.0, fabs(t)))) {
      c->fsal_valid = false;
      return SCFFT_ESTEP;
    }
    const float hf = (float)hs;
    CK(run(c, SCFFT_K_RK, [&] {
      combine32_kernel<<<blocks, 256, 0, c->st>>>(c->ytmp32, h, hf, a21, k[0], 0.f, nullptr, n3);
      return cudaGetLastError();
    }));
    CS_(rhs32(c, t + 0.5 * hs, 0, nullptr, c->ytmp32, c->last32, k[1]));
    CK(run(c, SCFFT_K_RK, [&] {
      combine32_kernel<<<blocks, 256, 0, c->st>>>(c->ytmp32, h, hf, 0.f, k[0], a32, k[1], n3);
      return cudaGetLastError();
    }));
    CS_(rhs32(c, t + 0.75 * hs, 0, nullptr, c->ytmp32, c->last32, k[2]));
    CK(run(c, SCFFT_K_RK, [&] {
      candidate32_kernel<<<blocks, 256, 0, c->st>>>(c->ynew64, c->d32, h, hf, b1, k[0], b2, k[1], b3, k[2], n3);
      return cudaGetLastError();
    }));
    CS_(rhs32(c, hits ? nxt : t + hs, end_left ? 1 : 0, c->ynew64, nullptr, c->last32, k[3]));
    double en = 0.0;
    if (!(dt_fixed > 0)) {
      CK(cudaMemsetAsync(c->errbits, 0, sizeof(unsigned long long), c->st));
      CK(run(c, SCFFT_K_RK, [&] {
        errnorm32_kernel<<<blocks, 256, 0, c->st>>>(h, c->ynew64, hf, e1, k[0], e2, k[1], e3, k[2], e4, k[3],
                                                   (float)c->opt.rtol, (float)c->opt.atol, n3,
                                                   reinterpret_cast<unsigned*>(c->errbits));
        return cudaGetLastError();
      }));
      CK(cudaMemcpyAsync(c->herr, c->errbits, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
      if (c->graph_pending) {
        const scfft_status ds = flush_pending(c);  // synchronises the stream
        if (ds != SCFFT_OK) {
          c->fsal_valid = false;
          return ds;
        }
      }
      CK(cudaStreamSynchronize(c->st));
      unsigned bits;
      memcpy(&bits, c->herr, sizeof(unsigned));
      float ef;
      memcpy(&ef, &bits, sizeof(float));
      en = (double)ef;
      if (!(en == en)) {
        c->fsal_valid = false;
        return SCFFT_ENONFINITE;
      }
    }
    if (c->graph_pending) {  // fixed step: no error norm was read, read the device state here
      const scfft_status ds = flush_pending(c);
      if (ds != SCFFT_OK) {
        c->fsal_valid = false;
        return ds;
      }
    }
    if (en <= 1.0) {
      const double tn = hits ? nxt : t + hs;
      // the accepted state, and the caller's warm start (FP64) following the most recent rhs result
      CK(run(c, SCFFT_K_RK, [&] {
        accept32_kernel<<<blocks, 256, 0, c->st>>>(h, c->comp64, c->d32, c->last32, warm, n3);
        return cudaGetLastError();
      }));
      c->stats.accepted += 1;
      if (end_left) {
        c->fsal_valid = false;
      } else {
        std::swap(k[0], k[3]);
        c->fsal_valid = true;
        c->fsal_t = tn;
        c->fsal_h = h;
        c->fsal_g = warm;
      }
      *t_io = tn;
      if (dt_fixed > 0) {
        *dt_io = dt_fixed;
      } else {
        const double fac = en == 0.0 ? 5.0 : std::min(5.0, std::max(0.2, 0.9 * pow(en, -1.0 / 3.0)));
        *dt_io = hs * fac;
      }
      if (rej_out) *rej_out = rej;
      c->stats.t = tn;
      c->stats.dt = *dt_io;
      return SCFFT_OK;
    }
    ++rej;
    c->stats.rejected += 1;
    dt = hs * std::max(0.2, 0.9 * pow(en, -1.0 / 3.0));
  }
}

// ---------------------------------------------------------------- device-resident stepping
// scfft_advance runs up to K accepted BS23 steps of the FP32 path as one CUDA graph launch:
// a WHILE conditional node over trials whose body computes, on the device, the trial step and
// the rhs parameters of its three stages (dh_e/dt of the path and the Eq. 5 stop threshold at
// each stage time), the stage states, the three stage rhs (each with its Eq. 5 loop as a
// nested WHILE node), the candidate, the error norm, and the step controller (accept or
// reject, the next step size), then applies an accepted step.  The host reads the step state
// back once, after the launch.
}  // namespace

struct PathDev {
  int nk;
  int pad_;
  double kt[64];
  double khe[3 * 64];
  double sin_amp, sin_period, sin_t0, sin_t1;
  double sin_dir[3];
};

struct StepDev {
  double t, dt, tlim, hs;      // time, proposed step, stop of this launch, trial step
  double delta_it;             // Eq. 5 tolerance
  double rtol, atol;
  int hits, end_left;          // the trial ends on tlim; tlim is a kink (left derivative there)
  int tlim_kink;
  int accepted;                // the last trial was accepted
  int steps, target;           // accepted steps so far, wanted
  int trials, max_trials;
  int status;                  // scfft_status of a device-side failure
  unsigned errbits;            // error norm (float bits; integer max of nonnegative floats)
};

namespace {

// dh_e/dt at t on the device (the host's hedot_at, term by term)
__device__ void hedot_dev(const PathDev* p, double t, int left, double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  for (int s = 0; s + 1 < p->nk; ++s) {
    const double lo = p->kt[s], hi = p->kt[s + 1];
    const bool in = left ? (lo < t && t <= hi) : (lo <= t && t < hi);
    if (in) {
      for (int a = 0; a < 3; ++a) out[a] = (p->khe[3 * (s + 1) + a] - p->khe[3 * s + a]) / (hi - lo);
      break;
    }
  }
  if (p->sin_amp != 0) {
    const bool in = left ? (p->sin_t0 < t && t <= p->sin_t1) : (p->sin_t0 <= t && t < p->sin_t1);
    if (in) {
      const double w = 2 * M_PI / p->sin_period;
      const double v = p->sin_amp * w * cos(w * (t - p->sin_t0));
      for (int a = 0; a < 3; ++a) out[a] += v * p->sin_dir[a];
    }
  }
}

__global__ void step_begin_kernel(StepDev* sd, const PathDev* path, PointParams base, PointParams* pps) {
  const double t = sd->t;
  double hs = fmin(sd->dt, sd->tlim - t);
  const int hits = hs == sd->tlim - t;
  if (!(hs > 1e-14 * fmax(1.0, fabs(t)))) {
    sd->status = SCFFT_ESTEP;
    hs = 0.0;
  }
  sd->hs = hs;
  sd->hits = hits;
  sd->end_left = hits && sd->tlim_kink;
  sd->errbits = 0u;
  sd->trials += 1;
  const double ts[3] = {t + 0.5 * hs, t + 0.75 * hs, hits ? sd->tlim : t + hs};
  const int left[3] = {0, 0, sd->end_left};
  for (int s = 0; s < 3; ++s) {
    PointParams pp = base;
    hedot_dev(path, ts[s], left[s], pp.hedot);
    const double hn = sqrt(pp.hedot[0] * pp.hedot[0] + pp.hedot[1] * pp.hedot[1] + pp.hedot[2] * pp.hedot[2]);
    pp.tol = sd->delta_it * (hn > 1.0 ? hn : 1.0);
    pps[s] = pp;
  }
}

__global__ void combine32d_kernel(float* __restrict__ out, const double* __restrict__ y, const StepDev* sd, float c1,
                                  const float* __restrict__ k1, float c2, const float* __restrict__ k2, long long n) {
  const float h = (float)sd->hs;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = c1 * k1[i];
    if (k2) s += c2 * k2[i];
    out[i] = (float)y[i] + h * s;
  }
}

__global__ void candidate32d_kernel(double* __restrict__ ynew, float* __restrict__ d, const double* __restrict__ y,
                                    const StepDev* sd, float b1, const float* __restrict__ k1, float b2,
                                    const float* __restrict__ k2, float b3, const float* __restrict__ k3, long long n) {
  const float h = (float)sd->hs;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float di = h * (b1 * k1[i] + b2 * k2[i] + b3 * k3[i]);
    d[i] = di;
    ynew[i] = y[i] + (double)di;
  }
}

__global__ void errnorm32d_kernel(const double* __restrict__ y, const double* __restrict__ yn, StepDev* sd, float e1,
                                  const float* __restrict__ k1, float e2, const float* __restrict__ k2, float e3,
                                  const float* __restrict__ k3, float e4, const float* __restrict__ k4, float rtol,
                                  float atol, long long n) {
  const float h = (float)sd->hs;
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float e = h * (e1 * k1[i] + e2 * k2[i] + e3 * k3[i] + e4 * k4[i]);
    const float w = fmaxf(rtol * fmaxf(abs_f32_of(y[i]), abs_f32_of(yn[i])), atol);
    const float r = fabsf(e) / w;
    m = (r > m || r != r) ? r : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float q = __shfl_xor_sync(0xffffffffu, m, o);
    m = (q > m || q != q) ? q : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(&sd->errbits, __float_as_uint(m));
}

// accept or reject the trial, propose the next step (the host controller's rule), and set
// the trial loop's condition
__global__ void step_end_kernel(StepDev* sd, const Ctrl* ctrl, cudaGraphConditionalHandle h) {
  const double en = (double)__uint_as_float(sd->errbits);
  if (sd->status == 0 && ctrl->status != 0) sd->status = ctrl->status;
  if (sd->status == 0 && !(en == en)) sd->status = SCFFT_ENONFINITE;
  sd->accepted = 0;
  if (sd->status == 0) {
    const double hs = sd->hs;
    if (en <= 1.0) {
      sd->accepted = 1;
      sd->t = sd->hits ? sd->tlim : sd->t + hs;
      const double fac = en == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(en, -1.0 / 3.0)));
      sd->dt = hs * fac;
      sd->steps += 1;
    } else {
      sd->dt = hs * fmax(0.2, 0.9 * pow(en, -1.0 / 3.0));
    }
  }
  const bool go = sd->status == 0 && sd->steps < sd->target && !(sd->accepted && sd->hits) &&
                  sd->trials < sd->max_trials;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// an accepted trial: y <- y + d (Kahan), the caller's warm start <- the last rhs result, and the
// first stage of the next step <- the last stage (FSAL)
__global__ void accept32d_kernel(double* __restrict__ y, double* __restrict__ c, const float* __restrict__ d,
                                 const float* __restrict__ last, double* __restrict__ warm, float* __restrict__ k0,
                                 const StepDev* sd, long long n) {
  if (!sd->accepted) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double yi = y[i];
    const double u = (double)d[i] - c[i];
    const double t = yi + u;
    c[i] = (t - yi) - u;
    y[i] = t;
    const float l = last[i];
    warm[i] = (double)l;
    k0[i] = l;
  }
}

__global__ void set_cond_kernel(cudaGraphConditionalHandle h) { cudaGraphSetConditional(h, 1u); }

// Add a WHILE node running the Eq. 5 loop body at the current point of the capture on cs;
// its body is captured on cs2.  The handle is set to 1 by a kernel just before the node (a
// default value applies only at the start of each top-level launch).
bool capture_eq5_loop(scfft_ctx* c, cudaStream_t cs, cudaStream_t cs2, const PointParams& pp) {
  cudaGraphConditionalHandle hh{};
  cudaStreamCaptureStatus stc;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(cs, &stc, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess ||
      stc != cudaStreamCaptureStatusActive)
    return false;
  if (cudaGraphConditionalHandleCreate(&hh, g, 0, 0) != cudaSuccess) return false;
  set_cond_kernel<<<1, 1, 0, cs>>>(hh);
  if (cudaGetLastError() != cudaSuccess) return false;
  if (cudaStreamGetCaptureInfo(cs, &stc, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess) return false;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hh;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node{};
  if (cudaGraphAddNode(&node, g, deps, nullptr, nd, &np) != cudaSuccess) return false;
  if (cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return false;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return false;
  Launch<float> L2 = launch_of<float>(c);
  L2.st = cs2;
  L2.fault = nullptr;
  const bool ok = loop_body(L2, pp, hh, c->opt.max_iter, c->curl_kind == SCFFT_CURL_FD, c->dcell) == cudaSuccess;
  cudaGraph_t captured = nullptr;
  return cudaStreamEndCapture(cs2, &captured) == cudaSuccess && ok;
}

// One stage rhs of the FP32 path captured on cs: the pre-stage passes with the stage's
// parameters read from the device (pps), the Eq. 5 loop, and the result into out.
bool capture_stage(scfft_ctx* c, cudaStream_t cs, cudaStream_t cs2, const PointParams* pps, const double* h64,
                   const float* h32, const float* warm32, float* out) {
  Launch<float> L = launch_of<float>(c);
  L.st = cs;
  L.fault = nullptr;
  L.pps = pps;
  const PointParams pp = base_params(c);
  if (c->curl_kind == SCFFT_CURL_FD) {
    if (launch_fd_efield<float>(L, pp, h64, h32, c->dcell, L.w->Hd[1]) != cudaSuccess) return false;
    if (launch_fd_assemble<float>(L, pp, L.w->Hd[1], nullptr, warm32, c->dcell) != cudaSuccess) return false;
  } else {
    if (launch_x_reg_io(L, X_FWD_F64, pp, h64, h32, nullptr, nullptr, nullptr, 0, 0, false) != cudaSuccess) return false;
    if (launch_y<float>(L, false, false, false) != cudaSuccess) return false;
    if (launch_z_curl<float>(L, false, 1.0 / (double)L.g.N) != cudaSuccess) return false;
    if (launch_y<float>(L, false, true, false) != cudaSuccess) return false;
    const cudaError_t e = c->law ? launch_x_reg_io(L, X_POWERLAW_H, pp, h64, h32, nullptr, nullptr, nullptr, 0, 0, false)
                                 : launch_x<float>(L, X_POWERLAW, pp, nullptr, nullptr, nullptr, 0, 0, false);
    if (e != cudaSuccess) return false;
    if (launch_y<float>(L, false, false, false) != cudaSuccess) return false;
    if (launch_z_curl<float>(L, false, 1.0 / (double)L.g.N) != cudaSuccess) return false;
    if (launch_y<float>(L, false, true, false) != cudaSuccess) return false;
    if (launch_x_reg_io(L, X_ASSEMBLE, pp, nullptr, nullptr, nullptr, nullptr, warm32, 0, 0, false) != cudaSuccess)
      return false;
  }
  if (c->nout > 0 && c->opt.max_iter > 0 && !capture_eq5_loop(c, cs, cs2, pp)) return false;
  const long long n3 = 3 * c->g.N;
  finalize_f32_kernel<<<(int)std::min<long long>((n3 + 255) / 256, 152 * 8), 256, 0, cs>>>(c->wf.Hd[0], c->wf.Hd[1],
                                                                                          c->ctrl, out, n3);
  return cudaGetLastError() == cudaSuccess;
}

// Add the trial loop of context c for the state buffers h, warm (FP32 path) to graph g as a
// WHILE node with no dependencies; false if the driver refuses any part.
bool add_step_loop(scfft_ctx* c, cudaGraph_t g, double* h, double* warm) {
  cudaStream_t cs = nullptr, cs2 = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking) != cudaSuccess) {
    if (cs) cudaStreamDestroy(cs);
    cudaGetLastError();
    return false;
  }
  const long long n3 = 3 * c->g.N;
  const int blocks = blocks_for(n3);
  float** k = c->k32;
  const float a21 = 0.5f, a32 = 0.75f, b1 = 2.0f / 9.0f, b2 = 1.0f / 3.0f, b3 = 4.0f / 9.0f;
  const float e1 = (float)(2.0 / 9.0 - 7.0 / 24.0), e2 = (float)(1.0 / 3.0 - 0.25),
              e3 = (float)(4.0 / 9.0 - 1.0 / 3.0), e4 = -0.125f;
  cudaGraphConditionalHandle hw{};
  bool ok = cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams np{};
  cudaGraphNode_t node{};
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hw;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (ok) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
      bool good = true;
      step_begin_kernel<<<1, 1, 0, cs>>>(c->sdev, c->pathd, base_params(c), c->ppsd);
      good = good && cudaGetLastError() == cudaSuccess;
      // stage 2: the warm start is the most recent rhs result, kept in k[3]
      combine32d_kernel<<<blocks, 256, 0, cs>>>(c->ytmp32, h, c->sdev, a21, k[0], 0.f, nullptr, n3);
      good = good && cudaGetLastError() == cudaSuccess &&
             capture_stage(c, cs, cs2, c->ppsd + 0, nullptr, c->ytmp32, k[3], k[1]);
      combine32d_kernel<<<blocks, 256, 0, cs>>>(c->ytmp32, h, c->sdev, 0.f, k[0], a32, k[1], n3);
      good = good && cudaGetLastError() == cudaSuccess &&
             capture_stage(c, cs, cs2, c->ppsd + 1, nullptr, c->ytmp32, k[1], k[2]);
      candidate32d_kernel<<<blocks, 256, 0, cs>>>(c->ynew64, c->d32, h, c->sdev, b1, k[0], b2, k[1], b3, k[2], n3);
      good = good && cudaGetLastError() == cudaSuccess &&
             capture_stage(c, cs, cs2, c->ppsd + 2, c->ynew64, nullptr, k[2], k[3]);
      errnorm32d_kernel<<<blocks, 256, 0, cs>>>(h, c->ynew64, c->sdev, e1, k[0], e2, k[1], e3, k[2], e4, k[3],
                                                 (float)c->opt.rtol, (float)c->opt.atol, n3);
      step_end_kernel<<<1, 1, 0, cs>>>(c->sdev, c->ctrl, hw);
      accept32d_kernel<<<blocks, 256, 0, cs>>>(h, c->comp64, c->d32, k[3], warm, k[0], c->sdev, n3);
      good = good && cudaGetLastError() == cudaSuccess;
      cudaGraph_t captured = nullptr;
      ok = cudaStreamEndCapture(cs, &captured) == cudaSuccess && good;
    }
  }
  cudaStreamDestroy(cs);
  cudaStreamDestroy(cs2);
  if (!ok) cudaGetLastError();
  return ok;
}

// the step graph of one context for the buffers h, warm
bool build_step_graph(scfft_ctx* c, double* h, double* warm) {
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->step_graph) cudaGraphDestroy(c->step_graph);
  c->step_exec = nullptr;
  c->step_graph = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess && add_step_loop(c, g, h, warm);
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (!ok) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  c->step_graph = g;
  c->step_exec = ex;
  c->step_h = h;
  c->step_warm = warm;
  for (int i = 0; i < 4; ++i) c->step_k[i] = c->k32[i];
  c->step_epoch = c->epoch;
  return true;
}

// kernels launched per trial of the step graph outside the Eq. 5 loops
int step_graph_launches(const scfft_ctx* c) {
  const int pre = c->curl_kind == SCFFT_CURL_FD ? 2 : 9;
  return 3 * (pre + 2) + 2 + 1 + 1 + 1 + 1;  // stages (+ cond set, finalize), combines, candidate, norm, end, accept
}

// Everything before the graph launch of scfft_advance on the context's stream: step state,
// path, the first stage (computed unless FSAL), the buffer roles the graph was built on.
// need_graph: the context's own step graph must be (re)built for h, warm.
scfft_status advance_prologue(scfft_ctx* c, double t, double dt, double tstop, int nsteps, double* h, double* warm,
                              bool* need_graph) {
  CS_(ensure_rk32(c));
  const long long n3 = 3 * c->g.N;
  const int blocks = blocks_for(n3);
  if (!c->sdev) {
    if (cudaMalloc(&c->sdev, sizeof(StepDev)) != cudaSuccess || cudaMalloc(&c->pathd, sizeof(PathDev)) != cudaSuccess ||
        cudaMalloc(&c->ppsd, 3 * sizeof(PointParams)) != cudaSuccess ||
        cudaHostAlloc(&c->hsdev, sizeof(StepDev), 0) != cudaSuccess) {
      cudaGetLastError();
      return SCFFT_ENOMEM;
    }
  }
  if (c->path_dirty) {
    PathDev p{};
    p.nk = (int)c->kt.size();
    for (int i = 0; i < p.nk; ++i) p.kt[i] = c->kt[i];
    for (int i = 0; i < 3 * p.nk; ++i) p.khe[i] = c->khe[i];
    p.sin_amp = c->sin_amp;
    p.sin_period = c->sin_period;
    p.sin_t0 = c->sin_t0;
    p.sin_t1 = c->sin_t1;
    for (int a = 0; a < 3; ++a) p.sin_dir[a] = c->sin_dir[a];
    CK(cudaMemcpy(c->pathd, &p, sizeof(p), cudaMemcpyHostToDevice));
    c->path_dirty = false;
  }
  if (c->graph_pending) CS_(flush_pending(c));
  const std::vector<double> kinks = kinks_of(c);
  double tlim = tstop;
  for (double v : kinks)
    if (v > t && v < tlim) tlim = v;
  const bool tlim_kink = tlim < tstop || std::binary_search(kinks.begin(), kinks.end(), tlim);
  // the first stage: reused (FSAL) or computed here, as scfft_step does
  if (!(c->fsal_valid && c->fsal_t == t && c->fsal_h == h && c->fsal_g == warm)) {
    CK(run(c, SCFFT_K_RK, [&] {
      f64_to_f32_kernel<<<blocks, 256, 0, c->st>>>(warm, c->g32, n3);
      return cudaGetLastError();
    }));
    CK(cudaMemsetAsync(c->comp64, 0, sizeof(double) * n3, c->st));
    CS_(rhs32(c, t, 0, h, nullptr, c->g32, c->k32[0]));
    if (c->graph_pending) CS_(flush_pending(c));
  }
  // the graph keeps its own buffer roles: first stage in step_k[0], most recent rhs result in step_k[3]
  if (c->step_k[0] && c->k32[0] != c->step_k[0]) {
    CK(cudaMemcpyAsync(c->step_k[0], c->k32[0], sizeof(float) * n3, cudaMemcpyDeviceToDevice, c->st));
    if (c->last32 == c->k32[0]) c->last32 = c->step_k[0];
    for (int i = 0; i < 4; ++i) c->k32[i] = c->step_k[i];
  }
  if (c->last32 != c->k32[3]) {
    CK(cudaMemcpyAsync(c->k32[3], c->last32, sizeof(float) * n3, cudaMemcpyDeviceToDevice, c->st));
    c->last32 = c->k32[3];
  }
  *need_graph = !c->step_exec || c->step_h != h || c->step_warm != warm || c->step_epoch != c->epoch;
  StepDev sd{};
  sd.t = t;
  sd.dt = dt;
  sd.tlim = tlim;
  sd.tlim_kink = tlim_kink ? 1 : 0;
  sd.delta_it = c->opt.delta_it;
  sd.rtol = c->opt.rtol;
  sd.atol = c->opt.atol;
  sd.target = nsteps;
  sd.max_trials = 100 * nsteps + 100;
  *c->hsdev = sd;
  CK(cudaMemcpyAsync(c->sdev, c->hsdev, sizeof(StepDev), cudaMemcpyHostToDevice, c->st));
  return SCFFT_OK;
}

// the read-back of the step state, queued on stream st after the graph
cudaError_t advance_readback(scfft_ctx* c, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(c->hsdev, c->sdev, sizeof(StepDev), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->hctrl + 2, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  return e;
}

// after the read-back has completed: statistics, time, step size, FSAL
scfft_status advance_epilogue(scfft_ctx* c, double* t_io, double* dt_io, double* h, double* warm, int* done) {
  const StepDev r = *c->hsdev;
  absorb_ctrl(c, c->hctrl[2], true);
  c->stats.rhs_calls += 3LL * r.trials;
  c->stats.launches += (long long)step_graph_launches(c) * r.trials;
  c->stats.accepted += r.steps;
  c->stats.rejected += r.trials - r.steps;
  c->last32 = c->k32[3];
  *done = r.steps;
  if (r.status != 0) {
    c->fsal_valid = false;
    return (scfft_status)r.status;
  }
  *t_io = r.t;
  *dt_io = r.dt;
  c->stats.t = r.t;
  c->stats.dt = r.dt;
  const bool kink_end = r.accepted && r.hits && r.end_left;
  c->fsal_valid = r.steps > 0 ? !kink_end : c->fsal_valid;
  if (c->fsal_valid) {
    c->fsal_t = r.t;
    c->fsal_h = h;
    c->fsal_g = warm;
  }
  return SCFFT_OK;
}

scfft_status advance_f32(scfft_ctx* c, double* t_io, double* dt_io, double tstop, int nsteps, double* h,
                         double* warm, int* done) {
  bool need_graph = false;
  CS_(advance_prologue(c, *t_io, *dt_io, tstop, nsteps, h, warm, &need_graph));
  if (need_graph && !build_step_graph(c, h, warm)) return SCFFT_ECUDA;
  CK(cudaGraphLaunch(c->step_exec, c->st));
  CK(advance_readback(c, c->st));
  CK(cudaStreamSynchronize(c->st));
  return advance_epilogue(c, t_io, dt_io, h, warm, done);
}

// One graph over a batch of FP32 contexts: every instance's trial loop as a WHILE node of its
// own, side by side with no dependencies, so one launch advances all instances concurrently.
struct BatchGraph {
  std::vector<scfft_ctx*> ctx;
  std::vector<const double*> h, warm;
  std::vector<unsigned long long> epoch;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> ready;
};
std::mutex g_batch_mutex;
BatchGraph* g_batch = nullptr;  // the last batch graph (rebuilt when the batch changes)

void free_batch_graph(BatchGraph* b) {
  if (!b) return;
  if (b->ex) cudaGraphExecDestroy(b->ex);
  if (b->g) cudaGraphDestroy(b->g);
  if (b->done) cudaEventDestroy(b->done);
  for (cudaEvent_t e : b->ready) cudaEventDestroy(e);
  delete b;
}

// ---------------------------------------------------------------- reverse mode of one rhs
constexpr int kSumBlocks = 152 * 2;

// per-block sums of (1 - chi) lam over the nodes, per component (deterministic: the host adds the blocks in order)
__global__ void chib_sum_kernel(const double* __restrict__ lam, const uint8_t* __restrict__ mask, long long N,
                                double* __restrict__ part) {
  double s[3] = {0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    if (!mask[i]) { s[0] += lam[i]; s[1] += lam[N + i]; s[2] += lam[2 * N + i]; }
  __shared__ double red[3][8];
  for (int q = 0; q < 3; ++q) {
    double v = s[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[threadIdx.x][w];
    part[blockIdx.x * 3 + threadIdx.x] = v;
  }
}

// mu_g = (1 - chi) lam
__global__ void chib_mask_kernel(const double* __restrict__ lam, const uint8_t* __restrict__ mask, long long N,
                                 double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const bool in = mask[i];
    out[i] = in ? 0.0 : lam[i];
    out[N + i] = in ? 0.0 : lam[N + i];
    out[2 * N + i] = in ? 0.0 : lam[2 * N + i];
  }
}

template <typename T>
scfft_status vjp_impl(scfft_ctx* c, const double* h, const double* lam, double* mu_h, double* mu_g, double* mu_jc,
                      double* mu_a) {
  const long long N = c->g.N, n3 = 3 * N;
  const int K = c->opt.max_iter;
  if (!c->adj) CK(cudaMalloc(&c->adj, sizeof(double) * 3 * n3));
  if (c->adj_part_cap < K + 1) {
    cudaFree(c->adj_part);
    if (c->hadj_part) cudaFreeHost(c->hadj_part);
    c->adj_part = nullptr;
    c->hadj_part = nullptr;
    c->adj_part_cap = 0;
    CK(cudaMalloc(&c->adj_part, sizeof(double) * 3 * kSumBlocks * (K + 1)));
    CK(cudaHostAlloc(&c->hadj_part, sizeof(double) * 3 * kSumBlocks * (K + 1), 0));
    c->adj_part_cap = K + 1;
  }
  double* jf = c->adj;
  double* lb[2] = {c->adj + n3, c->adj + 2 * n3};
  Launch<T> L = launch_of<T>(c);
  PointParams pp = base_params(c);
  // forward j = C h (the power law's Jacobian needs it)
  CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_FWD_F64, pp, h, nullptr, nullptr, 0, 0, false); }));
  CK(curl_in_U<T>(c, L, false));
  CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_TO_F64, pp, nullptr, jf, nullptr, 0, 0, false); }));
  // transposed iterations: lam_i = chi lam_{i+1} + C chi Phi (1 - chi) lam_{i+1}
  const double* cur = lam;
  for (int i = 0; i < K; ++i) {
    double* nxt = lb[i & 1];
    CK(run(c, SCFFT_K_OTHER, [&] {
      chib_sum_kernel<<<kSumBlocks, 256, 0, c->st>>>(cur, c->mask, N, c->adj_part + (size_t)i * 3 * kSumBlocks);
      return cudaGetLastError();
    }));
    CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_ADJ_PAD, pp, cur, nullptr, nullptr, 0, 0, false); }));
    CK(run(c, SCFFT_K_Y_FWD_P, [&] { return launch_y<T>(L, true, false, false); }));
    CK(run(c, SCFFT_K_Z_KERNEL, [&] { return launch_z_kernel<T>(L, false); }));
    CK(run(c, SCFFT_K_Y_INV_P, [&] { return launch_y<T>(L, true, true, false); }));
    CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_ADJ_CROP, pp, nullptr, nullptr, nullptr, 0, 0, false); }));
    CK(curl_in_U<T>(c, L, false));
    CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_ADJ_COMBINE, pp, cur, nxt, nullptr, 0, 0, false); }));
    cur = nxt;
  }
  // dh^0 = chi u + (1 - chi) g:  mu_g = (1 - chi) lam_0,  lam_u = chi lam_0
  if (mu_g)
    CK(run(c, SCFFT_K_OTHER, [&] {
      chib_mask_kernel<<<blocks_for(N), 256, 0, c->st>>>(cur, c->mask, N, mu_g);
      return cudaGetLastError();
    }));
  // u = -C e / mu0; e = E(j); j = C h
  CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_ADJ_IN, pp, cur, nullptr, nullptr, 0, 0, false); }));
  CK(curl_in_U<T>(c, L, false));
  CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_ADJ_POWERLAW, pp, jf, mu_jc, nullptr, 0, 0, false); }));
  CK(curl_in_U<T>(c, L, false));
  CK(run(c, SCFFT_K_OTHER, [&] { return launch_x<T>(L, X_TO_F64, pp, nullptr, mu_h, nullptr, 0, 0, false); }));
  if (mu_a) {
    CK(cudaMemcpyAsync(c->hadj_part, c->adj_part, sizeof(double) * 3 * kSumBlocks * K, cudaMemcpyDeviceToHost, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  if (mu_a) {
    mu_a[0] = mu_a[1] = mu_a[2] = 0.0;
    for (int i = 0; i < K; ++i)
      for (int b = 0; b < kSumBlocks; ++b)
        for (int q = 0; q < 3; ++q) mu_a[q] += c->hadj_part[((size_t)i * kSumBlocks + b) * 3 + q];
  }
  return SCFFT_OK;
}

scfft_status step_any(scfft_ctx* c, double* t, double* dt, double tstop, double* h, double* warm, double dt_fixed,
                      int* rej) {
  return c->opt.precision == SCFFT_PREC_F32 ? bs23_step_f32(c, t, dt, tstop, h, warm, dt_fixed, rej)
                                            : bs23_step(c, t, dt, tstop, h, warm, dt_fixed, rej);
}

}  // namespace

extern "C" {

const char* scfft_status_string(scfft_status s) {
  switch (s) {
    case SCFFT_OK: return "ok";
    case SCFFT_EINVAL: return "invalid argument";
    case SCFFT_ENOMEM: return "out of memory";
    case SCFFT_ECUDA: return "CUDA runtime error";
    case SCFFT_ENOCONV: return "Eq. 5 iteration hit max_iter";
    case SCFFT_ESTEP: return "step size underflow";
    case SCFFT_ENONFINITE: return "non-finite value in a residual or error norm";
    case SCFFT_ETIMEOUT: return "bounded device wait timed out";
    case SCFFT_ESTATE: return "call out of order";
    case SCFFT_ESIZE: return "problem larger than the fixed preallocated maximum";
  }
  return "unknown status";
}

const char* scfft_kind_name(int kind) {
  static const char* names[SCFFT_NKINDS] = {
      "x_fwd_state", "x_powerlaw", "x_assemble", "x_maskpad", "x_update", "y_fwd_unpadded", "y_inv_unpadded",
      "z_curl",      "y_fwd_padded", "y_inv_padded", "z_kernel", "finalize", "rk_stage", "io_pass",
      "box_fused"};
  return (kind >= 0 && kind < SCFFT_NKINDS) ? names[kind] : "unknown";
}

scfft_status scfft_create(const scfft_grid* grid, const scfft_material* mat, const scfft_options* opt, void* stream,
                          scfft_ctx** out) {
  if (!grid || !mat || !opt || !out) return SCFFT_EINVAL;
  *out = nullptr;
  if (!grid_ok(grid->nx) || !grid_ok(grid->ny) || !grid_ok(grid->nz)) return SCFFT_EINVAL;
  if (!(grid->Lx > 0) || !(grid->Ly > 0) || !(grid->Lz > 0)) return SCFFT_EINVAL;
  if (!(mat->n >= 1) || !(mat->e0 > 0) || !(mat->jc > 0) || !(mat->rho_out >= 0) || !(mat->mu0 > 0))
    return SCFFT_EINVAL;
  if (opt->max_iter < 0 || !(opt->delta_it >= 0) || !(opt->sigma_scale >= 0) || !isfinite(opt->sigma_scale))
    return SCFFT_EINVAL;
  if (!(opt->rtol > 0) || !(opt->atol > 0)) return SCFFT_EINVAL;
  if (opt->precision != SCFFT_PREC_F64 && opt->precision != SCFFT_PREC_F32 && opt->precision != SCFFT_PREC_DF64)
    return SCFFT_EINVAL;
  scfft_ctx* c = new (std::nothrow) scfft_ctx();
  if (!c) return SCFFT_ENOMEM;
  c->g.nx = grid->nx; c->g.ny = grid->ny; c->g.nz = grid->nz;
  c->g.sxu = round_up(grid->nx / 2 + 1, 8);
  c->g.sxp = round_up(grid->nx + 1, 8);
  c->g.N = (long long)grid->nx * grid->ny * grid->nz;
  c->L[0] = grid->Lx; c->L[1] = grid->Ly; c->L[2] = grid->Lz;
  c->dcell[0] = 2 * grid->Lx / grid->nx; c->dcell[1] = 2 * grid->Ly / grid->ny; c->dcell[2] = 2 * grid->Lz / grid->nz;
  c->mat = *mat;
  c->opt = *opt;
  c->st = (cudaStream_t)stream;
  // default schedule: the two-buffer tensor-memory z pass where it exists (a 256-point padded z
  // transform), measured the fastest of the three forms
  if (2 * c->g.nz == 256) c->wf.sched.zk_tm = 2;
  scfft_status s = SCFFT_OK;
  if (cudaMalloc(&c->ctrl, sizeof(Ctrl)) != cudaSuccess || cudaMalloc(&c->ppd, sizeof(PointParams)) != cudaSuccess ||
      cudaMalloc(&c->partials, sizeof(double) * (c->g.ny * c->g.nz / 2 + 8)) != cudaSuccess ||
      cudaMalloc(&c->mask, c->g.N) != cudaSuccess || cudaHostAlloc(&c->hctrl, 3 * sizeof(Ctrl), 0) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(&c->errbits, sizeof(unsigned long long)) != cudaSuccess ||
      cudaHostAlloc(&c->herr, sizeof(unsigned long long), 0) != cudaSuccess) {
    s = SCFFT_ENOMEM;
  }
  if (s == SCFFT_OK) s = by_prec(c, [&](auto z) { return alloc_work<decltype(z)>(c); });
  if (s == SCFFT_OK && cudaMemset(c->ctrl, 0, sizeof(Ctrl)) != cudaSuccess) s = SCFFT_ECUDA;
  if (s != SCFFT_OK) {
    scfft_destroy(c);
    return s == SCFFT_ECUDA ? SCFFT_ENOMEM : s;
  }
  memset(c->hctrl, 0, 3 * sizeof(Ctrl));
  *out = c;
  return SCFFT_OK;
}

void scfft_destroy(scfft_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  free_rec(c);
  {  // a batch graph built on this context is dropped with it
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    if (g_batch && std::find(g_batch->ctx.begin(), g_batch->ctx.end(), c) != g_batch->ctx.end()) {
      free_batch_graph(g_batch);
      g_batch = nullptr;
    }
  }
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->step_graph) cudaGraphDestroy(c->step_graph);
  cudaFree(c->sdev); cudaFree(c->pathd); cudaFree(c->ppsd);
  if (c->hsdev) cudaFreeHost(c->hsdev);
  free_work(c->wf);
  free_work(c->wd);
  free_work(c->wq);
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  if (c->loop_graph) cudaGraphDestroy(c->loop_graph);
  cudaFree(c->ctrl); cudaFree(c->ppd); cudaFree(c->partials); cudaFree(c->mask); cudaFree(c->ib); cudaFree(c->errbits);
  cudaFree(c->ib32); cudaFree(c->ynew64); cudaFree(c->adj); cudaFree(c->adj_part);
  if (c->hadj_part) cudaFreeHost(c->hadj_part);
  if (c->hctrl) cudaFreeHost(c->hctrl);
  if (c->herr) cudaFreeHost(c->herr);
  for (int i = 0; i < 2; ++i) if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  for (cudaEvent_t e : c->pev) cudaEventDestroy(e);
  delete c;
}

scfft_status scfft_set_geometry(scfft_ctx* c, const uint8_t* mask) {
  if (!c || !mask) return SCFFT_EINVAL;
  const Geo& g = c->g;
  long long nin = 0;
  int y0 = g.ny, y1 = 0, z0 = g.nz, z1 = 0;
  for (int z = 0; z < g.nz; ++z)
    for (int y = 0; y < g.ny; ++y)
      for (int x = 0; x < g.nx; ++x) {
        if (!mask[((long long)z * g.ny + y) * g.nx + x]) continue;
        ++nin;
        if (x < 2 || y < 2 || z < 2 || x >= g.nx - 2 || y >= g.ny - 2 || z >= g.nz - 2) return SCFFT_EINVAL;
        y0 = std::min(y0, y);
        y1 = std::max(y1, y + 1);
        z0 = std::min(z0, z);
        z1 = std::max(z1, z + 1);
      }
  if (nin == 0) return SCFFT_EINVAL;
  // the row pairs of the x passes start at even y: round the box out to even bounds
  c->box[0] = y0 & ~1;
  c->box[1] = std::min(g.ny, (y1 + 1) & ~1);
  c->box[2] = z0;
  c->box[3] = z1;
  // the captured Eq. 5 loop holds the launches of the old box
  CK(cudaStreamSynchronize(c->st));
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  if (c->loop_graph) cudaGraphDestroy(c->loop_graph);
  c->loop_exec = nullptr;
  c->loop_graph = nullptr;
  c->loop_failed = false;
  std::vector<uint8_t> m(mask, mask + g.N);
  for (auto& v : m) v = v ? 1 : 0;
  CK(cudaMemcpy(c->mask, m.data(), g.N, cudaMemcpyHostToDevice));
  c->nout = g.N - nin;
  c->have_geom = true;
  c->fsal_valid = false;
  c->epoch++;
  return SCFFT_OK;
}

scfft_status scfft_set_jc_map(scfft_ctx* c, const double* jc) {
  if (!c) return SCFFT_EINVAL;
  const long long N = c->g.N;
  c->fsal_valid = false;
  c->epoch++;
  return by_prec(c, [&](auto z) -> scfft_status {
    typedef decltype(z) T;
    Work<T>& w = work<T>(c);
    cudaFree(w.jc);
    w.jc = nullptr;
    if (jc) {
      CK(cudaMalloc(&w.jc, sizeof(T) * N));
      CK(launch_convert<T>(jc, w.jc, N, c->st));
    }
    return SCFFT_OK;
  });
}

}  // extern "C"

// ---------------------------------------------------------------- schedule autotuner
namespace {

// Schedules chosen per device and grid, shared by every context of that grid (a batch of
// instances tunes once per grid size).
std::mutex g_tune_mutex;
std::map<std::vector<int>, Sched> g_tune_cache;

// Drop the captured graphs of a context: they hold the launches of the old schedule.
void drop_loop_graph(scfft_ctx* c) {
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  if (c->loop_graph) cudaGraphDestroy(c->loop_graph);
  c->loop_exec = nullptr;
  c->loop_graph = nullptr;
  c->loop_failed = false;
  c->epoch++;  // the step graph and the batch graph are rebuilt on their next launch
}

void to_public(const Sched& s, scfft_schedule* o) {
  o->z_kernel_tile = s.zk_tc;
  o->z_curl_tile = s.zc_tc;
  o->y_unpadded_tile = s.yu_tc;
  o->y_padded_tma = s.yp_tma;
  o->z_kernel_tmem = s.zk_tm;
  o->box_fused = s.box_fused;
  o->x_update_split = s.xu3;
}

bool sched_ok(const scfft_schedule* s) {
  return (s->z_kernel_tile == 4 || s->z_kernel_tile == 8) && (s->z_curl_tile == 8 || s->z_curl_tile == 16) &&
         (s->y_unpadded_tile == 8 || s->y_unpadded_tile == 16) && (s->y_padded_tma == 0 || s->y_padded_tma == 1) &&
         (s->z_kernel_tmem >= 0 && s->z_kernel_tmem <= 2) && (s->box_fused == 0 || s->box_fused == 1) &&
         (s->x_update_split == 0 || s->x_update_split == 1);
}

// the tensor-memory form of the padded z pass exists for its 16 x 16 split (a 256-point z transform)
bool tmem_z_ok(const scfft_ctx* c) { return 2 * c->g.nz == 256; }

// Mean device time (us) of one call of f (a few pass launches) on the context's stream: three
// untimed calls, then ten between CUDA events.
template <typename F> scfft_status time_us(scfft_ctx* c, F&& f, double* us) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SCFFT_ECUDA;
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
  for (int i = 0; i < 10 && e == cudaSuccess; ++i) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    note_cuda_error(e, __FILE__, __LINE__);
    return SCFFT_ECUDA;
  }
  *us = 1e3 * ms / 10.0;
  return SCFFT_OK;
}

// Time each candidate of each knob of the FP32 passes on the context's own workspace (the
// passes transform its scratch spectra in place; their contents are not used afterwards) and
// keep the fastest (the second candidate only when it is faster by more than 3%, so that timing
// noise does not flip a choice); knobs act on different passes, so they are tuned one at a time.
scfft_status autotune_f32(scfft_ctx* c, double us[15]) {
  Launch<float> L = launch_of<float>(c);
  L.fault = nullptr;
  Sched& s = c->wf.sched;
  const double inv_n = 1.0 / (double)c->g.N;
  // candidates cand[0..n): the fastest, where it beats cand[0] (the default) by more than 3%
  auto pick_n = [&](int* knob, const int* cand, int n, double* t, auto launch) -> scfft_status {
    for (int k = 0; k < n; ++k) {
      *knob = cand[k];
      CS_(time_us(c, launch, &t[k]));
    }
    int best = 0;
    for (int k = 1; k < n; ++k)
      if (t[k] < 0.97 * t[0] && t[k] < t[best]) best = k;
    *knob = cand[best];
    return SCFFT_OK;
  };
  auto pick = [&](int* knob, const int cand[2], double* t, auto launch) -> scfft_status {
    return pick_n(knob, cand, 2, t, launch);
  };
  const int zk[2] = {8, 4}, zc[2] = {8, 16}, yu[2] = {8, 16}, yp[2] = {1, 0}, zm[3] = {2, 1, 0};
  // the padded z pass as the Eq. 5 iteration runs it: input planes of Omega's box only
  const Launch<float> LZ = boxed(L);
  s.zk_tm = tmem_z_ok(c) ? 2 : 0;
  CS_(pick(&s.zk_tc, zk, us + 0, [&] { return launch_z_kernel<float>(LZ, false); }));
  if (tmem_z_ok(c)) CS_(pick_n(&s.zk_tm, zm, 3, us + 8, [&] { return launch_z_kernel<float>(LZ, false); }));
  CS_(pick(&s.zc_tc, zc, us + 2, [&] { return launch_z_curl<float>(L, false, inv_n); }));
  CS_(pick(&s.yu_tc, yu, us + 4, [&] {
    const cudaError_t e = launch_y<float>(L, false, false, false);
    return e != cudaSuccess ? e : launch_y<float>(L, false, true, false);
  }));
  if (c->wf.ym) {
    CS_(pick(&s.yp_tma, yp, us + 6, [&] {
      const cudaError_t e = launch_y<float>(L, true, false, false);
      return e != cudaSuccess ? e : launch_y<float>(L, true, true, false);
    }));
  } else {
    s.yp_tma = 0;
  }
  // the Eq. 5 update pass, components one after another or side by side; the pass advances the
  // device's iteration state, which is put back afterwards (its iterate and spectrum outputs
  // are scratch)
  {
    Ctrl saved;
    CK(cudaMemcpyAsync(&saved, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const int xs[2] = {0, 1};
    PointParams pu = base_params(c);
    const scfft_status ts = pick(&s.xu3, xs, us + 13, [&] {
      return launch_x<float>(L, X_UPDATE, pu, nullptr, nullptr, nullptr, 0, 1, false);
    });
    CK(cudaMemcpyAsync(c->ctrl, &saved, sizeof(Ctrl), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    CS_(ts);
  }
  // the three passes on Omega's box against the fused pass (after the y passes' own choice)
  const Launch<float> LB = boxed(L);
  s.box_fused = 0;
  if (box_fused_ok(LB) && c->curl_kind == SCFFT_CURL_SPECTRAL) {
    const int bf[2] = {0, 1};
    PointParams pp = base_params(c);
    CS_(pick(&s.box_fused, bf, us + 11, [&] {
      if (s.box_fused) return launch_box_fused(LB, false);
      cudaError_t e = launch_y<float>(LB, false, true, false);
      if (e == cudaSuccess) e = launch_x<float>(LB, X_MASKPAD, pp, nullptr, nullptr, nullptr, 0, 0, false);
      return e != cudaSuccess ? e : launch_y<float>(LB, true, false, false);
    }));
  }
  return SCFFT_OK;
}

}  // namespace

extern "C" {

scfft_status scfft_autotune(scfft_ctx* c, int retune, scfft_schedule* out) {
  if (!c) return SCFFT_EINVAL;
  if (out) memset(out, 0, sizeof(*out));
  if (c->opt.precision != SCFFT_PREC_F32) {  // the shared-memory passes have no schedule to choose
    if (out) to_public(Sched(), out);
    return SCFFT_OK;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const std::vector<int> key = {dev, c->g.nx, c->g.ny, c->g.nz};
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  CK(cudaStreamSynchronize(c->st));
  auto it = g_tune_cache.find(key);
  if (it != g_tune_cache.end() && !retune) {
    c->wf.sched = it->second;
  } else {
    double us[15] = {0};
    CS_(autotune_f32(c, us));
    g_tune_cache[key] = c->wf.sched;
    if (out)
      for (int i = 0; i < 15; ++i) out->us[i] = us[i];
  }
  drop_loop_graph(c);
  if (out) to_public(c->wf.sched, out);
  return SCFFT_OK;
}

scfft_status scfft_get_schedule(scfft_ctx* c, scfft_schedule* out) {
  if (!c || !out) return SCFFT_EINVAL;
  memset(out, 0, sizeof(*out));
  to_public(c->opt.precision == SCFFT_PREC_F32 ? c->wf.sched : Sched(), out);
  return SCFFT_OK;
}

scfft_status scfft_set_schedule(scfft_ctx* c, const scfft_schedule* s) {
  if (!c || !s || !sched_ok(s)) return SCFFT_EINVAL;
  if (c->opt.precision != SCFFT_PREC_F32) return SCFFT_EINVAL;
  if (s->y_padded_tma && !c->wf.ym) return SCFFT_EINVAL;
  if (s->z_kernel_tmem && !tmem_z_ok(c)) return SCFFT_EINVAL;
  CK(cudaStreamSynchronize(c->st));
  c->wf.sched.zk_tm = s->z_kernel_tmem;
  c->wf.sched.zk_tc = s->z_kernel_tile;
  c->wf.sched.zc_tc = s->z_curl_tile;
  c->wf.sched.yu_tc = s->y_unpadded_tile;
  c->wf.sched.yp_tma = s->y_padded_tma;
  c->wf.sched.box_fused = s->box_fused;
  c->wf.sched.xu3 = s->x_update_split;
  drop_loop_graph(c);
  return SCFFT_OK;
}

scfft_status scfft_set_curl(scfft_ctx* c, int kind) {
  if (!c || (kind != SCFFT_CURL_SPECTRAL && kind != SCFFT_CURL_FD)) return SCFFT_EINVAL;
  if (kind == c->curl_kind) return SCFFT_OK;
  if (kind == SCFFT_CURL_FD) {
    const size_t bytes = by_prec(c, [](auto z) { return sizeof(z); }) * 3 * (size_t)c->g.N;
    void** jd = by_prec(c, [&](auto z) { return (void**)&work<decltype(z)>(c).Jd; });
    if (!*jd && cudaMalloc(jd, bytes) != cudaSuccess) {
      cudaGetLastError();
      *jd = nullptr;
      return SCFFT_ENOMEM;
    }
  }
  CK(cudaStreamSynchronize(c->st));
  // the Eq. 5 loop graph holds the launches of one curl kind: rebuilt on the next rhs
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  if (c->loop_graph) cudaGraphDestroy(c->loop_graph);
  c->loop_exec = nullptr;
  c->loop_graph = nullptr;
  c->loop_failed = false;
  c->curl_kind = kind;
  c->fsal_valid = false;
  c->epoch++;
  return SCFFT_OK;
}

scfft_status scfft_set_ej_law(scfft_ctx* c, const scfft_ej_law* law) {
  if (!c || !law) return SCFFT_EINVAL;
  if (!(law->kim_h0 >= 0) || !isfinite(law->kim_h0)) return SCFFT_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!(law->aniso[a] > 0) || !isfinite(law->aniso[a])) return SCFFT_EINVAL;
  c->kim_h0 = law->kim_h0;
  for (int a = 0; a < 3; ++a) c->aniso[a] = law->aniso[a];
  c->law = (law->kim_h0 > 0 || law->aniso[0] != 1.0 || law->aniso[1] != 1.0 || law->aniso[2] != 1.0) ? 1 : 0;
  c->fsal_valid = false;
  c->epoch++;
  return SCFFT_OK;
}

scfft_status scfft_set_field_path(scfft_ctx* c, const scfft_field_path* p) {
  if (!c || !p || p->nknots < 1 || p->nknots > 64 || !p->t || !p->he) return SCFFT_EINVAL;
  for (int k = 0; k + 1 < p->nknots; ++k)
    if (!(p->t[k + 1] > p->t[k])) return SCFFT_EINVAL;
  if (p->sin_amp != 0 && (!(p->sin_period > 0) || !(p->sin_t1 >= p->sin_t0))) return SCFFT_EINVAL;
  c->kt.assign(p->t, p->t + p->nknots);
  c->khe.assign(p->he, p->he + 3 * p->nknots);
  c->sin_amp = p->sin_amp;
  c->sin_period = p->sin_period;
  c->sin_t0 = p->sin_t0;
  c->sin_t1 = p->sin_t1;
  for (int a = 0; a < 3; ++a) c->sin_dir[a] = p->sin_dir[a];
  c->have_path = true;
  c->fsal_valid = false;
  c->path_dirty = true;
  c->epoch++;
  return SCFFT_OK;
}

scfft_status scfft_precompute_kernel(scfft_ctx* c) {
  if (!c) return SCFFT_EINVAL;
  const Geo& g = c->g;
  const long long oct = (long long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
  double* scratch = nullptr;
  if (cudaMalloc(&scratch, sizeof(double) * 6 * oct) != cudaSuccess) return SCFFT_ENOMEM;
  const double dx = 2 * c->L[0] / g.nx, dy = 2 * c->L[1] / g.ny, dz = 2 * c->L[2] / g.nz;
  const double sig = c->opt.sigma_scale * 0.5 * sqrt(dx * dx + dy * dy + dz * dz);
  cudaError_t e = by_prec(c, [&](auto z) {
    typedef decltype(z) T;
    return launch_kernel_spectrum<T>(launch_of<T>(c), c->L[0], c->L[1], c->L[2], sig, scratch);
  });
  cudaError_t e2 = cudaStreamSynchronize(c->st);
  cudaFree(scratch);
  if (e != cudaSuccess || e2 != cudaSuccess) return SCFFT_ECUDA;
  c->have_kernel = true;
  c->fsal_valid = false;
  c->epoch++;
  return SCFFT_OK;
}

scfft_status scfft_rhs(scfft_ctx* c, double t, int left, const double* h, double* warm, double* hdot, int* iters_out) {
  if (!c || !h || !warm || !hdot || hdot == h) return SCFFT_EINVAL;
  if (!c->have_geom || !c->have_kernel || !c->have_path) return SCFFT_ESTATE;
  c->fsal_valid = false;
  return rhs_any(c, t, left, h, warm, hdot, iters_out);
}

scfft_status scfft_curl(scfft_ctx* c, const double* f, double* out) {
  if (!c || !f || !out || f == out) return SCFFT_EINVAL;
  return by_prec(c, [&](auto z) { return curl_impl<decltype(z)>(c, f, out); });
}

scfft_status scfft_phi(scfft_ctx* c, const double* j, double* out) {
  if (!c || !j || !out || j == out) return SCFFT_EINVAL;
  if (!c->have_kernel) return SCFFT_ESTATE;
  return by_prec(c, [&](auto z) { return phi_impl<decltype(z)>(c, j, out); });
}

scfft_status scfft_step(scfft_ctx* c, double* t, double* dt, double tstop, double* h, double* warm, int* rejected) {
  if (!c || !t || !dt || !h || !warm || !(*dt > 0) || !(tstop > *t)) return SCFFT_EINVAL;
  if (!c->have_geom || !c->have_kernel || !c->have_path) return SCFFT_ESTATE;
  return step_any(c, t, dt, tstop, h, warm, 0.0, rejected);
}

scfft_status scfft_advance(scfft_ctx* c, double* t, double* dt, double tstop, int nsteps, double* h, double* warm,
                           int* steps_done) {
  if (!c || !t || !dt || !h || !warm || !(*dt > 0) || !(tstop > *t) || nsteps < 1) return SCFFT_EINVAL;
  if (!c->have_geom || !c->have_kernel || !c->have_path) return SCFFT_ESTATE;
  int done = 0;
  scfft_status s = SCFFT_OK;
  if (c->opt.precision == SCFFT_PREC_F32 && !c->prof_on) {
    s = advance_f32(c, t, dt, tstop, nsteps, h, warm, &done);
  } else {  // FP64 path, or profiling (per-launch events): the host drives the steps
    const std::vector<double> kinks = kinks_of(c);
    double tlim = tstop;
    for (double v : kinks)
      if (v > *t && v < tlim) tlim = v;
    while (done < nsteps && *t < tlim) {
      s = step_any(c, t, dt, tlim, h, warm, 0.0, nullptr);
      if (s != SCFFT_OK) break;
      ++done;
    }
  }
  if (steps_done) *steps_done = done;
  return s;
}

scfft_status scfft_step_host(scfft_ctx* c, double* t, double* dt, double tstop, double* h_host, double* warm_host,
                             double* h, double* warm, int* rejected) {
  if (!c || !t || !dt || !h_host || !h || !warm || !(*dt > 0) || !(tstop > *t)) return SCFFT_EINVAL;
  if (!c->have_geom || !c->have_kernel || !c->have_path) return SCFFT_ESTATE;
  const size_t bytes = sizeof(double) * 3 * (size_t)c->g.N;
  // the FP32 step reads the caller's warm start only when it starts a trajectory (FSAL below);
  // without warm_host the warm start stays in the device buffer warm
  const bool continues = c->fsal_valid && c->fsal_t == *t && c->fsal_h == h && c->fsal_g == warm;
  const bool reads_warm = warm_host && (c->opt.precision != SCFFT_PREC_F32 || !continues);
  CK(cudaMemcpyAsync(h, h_host, bytes, cudaMemcpyHostToDevice, c->st));
  if (reads_warm) CK(cudaMemcpyAsync(warm, warm_host, bytes, cudaMemcpyHostToDevice, c->st));
  c->stats.h2d_bytes += (long long)(reads_warm ? 2 : 1) * (long long)bytes;
  const scfft_status s = step_any(c, t, dt, tstop, h, warm, 0.0, rejected);
  if (s != SCFFT_OK) return s;
  CK(cudaMemcpyAsync(h_host, h, bytes, cudaMemcpyDeviceToHost, c->st));
  if (warm_host) CK(cudaMemcpyAsync(warm_host, warm, bytes, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->stats.d2h_bytes += (warm_host ? 2 : 1) * (long long)bytes;
  return SCFFT_OK;
}

// ---------------------------------------------------------------- checkpoint / resume
namespace {
struct CkptHeader {
  char magic[8];  // "SCFFTCK1"
  int nx, ny, nz, precision;
  int fsal, pad_;
  double t, dt;
};

size_t ckpt_bytes(const scfft_ctx* c) {
  const size_t n3 = 3 * (size_t)c->g.N;
  const bool f32 = c->opt.precision == SCFFT_PREC_F32;
  // header, h, warm, FSAL stage, FP32-path compensation
  return sizeof(CkptHeader) + 2 * n3 * sizeof(double) + n3 * (f32 ? sizeof(float) : sizeof(double)) +
         (f32 ? n3 * sizeof(double) : 0);
}
}  // namespace

scfft_status scfft_checkpoint_save(scfft_ctx* c, double t, double dt, const double* h, const double* warm, void* buf,
                                   size_t* size) {
  if (!c || !size) return SCFFT_EINVAL;
  const size_t need = ckpt_bytes(c);
  if (!buf) {
    *size = need;
    return SCFFT_OK;
  }
  if (!h || !warm || *size < need) return SCFFT_EINVAL;
  const bool f32 = c->opt.precision == SCFFT_PREC_F32;
  const size_t n3 = 3 * (size_t)c->g.N;
  CK(cudaStreamSynchronize(c->st));
  CkptHeader hd{};
  memcpy(hd.magic, "SCFFTCK1", 8);
  hd.nx = c->g.nx;
  hd.ny = c->g.ny;
  hd.nz = c->g.nz;
  hd.precision = c->opt.precision;
  hd.fsal = (c->fsal_valid && c->fsal_t == t && c->fsal_h == h && c->fsal_g == warm) ? 1 : 0;
  hd.t = t;
  hd.dt = dt;
  char* p = static_cast<char*>(buf);
  memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  CK(cudaMemcpy(p, h, n3 * sizeof(double), cudaMemcpyDeviceToHost));
  p += n3 * sizeof(double);
  CK(cudaMemcpy(p, warm, n3 * sizeof(double), cudaMemcpyDeviceToHost));
  p += n3 * sizeof(double);
  const size_t stage_bytes = n3 * (f32 ? sizeof(float) : sizeof(double));
  if (hd.fsal) {
    CK(cudaMemcpy(p, f32 ? (const void*)c->k32[0] : (const void*)c->k[0], stage_bytes, cudaMemcpyDeviceToHost));
    if (f32) CK(cudaMemcpy(p + stage_bytes, c->comp64, n3 * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    memset(p, 0, stage_bytes + (f32 ? n3 * sizeof(double) : 0));
  }
  *size = need;
  return SCFFT_OK;
}

scfft_status scfft_checkpoint_load(scfft_ctx* c, const void* buf, size_t size, double* t, double* dt, double* h,
                                   double* warm) {
  if (!c || !buf || !t || !dt || !h || !warm) return SCFFT_EINVAL;
  if (size < ckpt_bytes(c)) return SCFFT_EINVAL;
  CkptHeader hd;
  memcpy(&hd, buf, sizeof(hd));
  if (memcmp(hd.magic, "SCFFTCK1", 8) != 0 || hd.nx != c->g.nx || hd.ny != c->g.ny || hd.nz != c->g.nz ||
      hd.precision != c->opt.precision)
    return SCFFT_EINVAL;
  const bool f32 = c->opt.precision == SCFFT_PREC_F32;
  const size_t n3 = 3 * (size_t)c->g.N;
  CK(cudaStreamSynchronize(c->st));
  const char* p = static_cast<const char*>(buf) + sizeof(hd);
  CK(cudaMemcpy(h, p, n3 * sizeof(double), cudaMemcpyHostToDevice));
  p += n3 * sizeof(double);
  CK(cudaMemcpy(warm, p, n3 * sizeof(double), cudaMemcpyHostToDevice));
  p += n3 * sizeof(double);
  c->fsal_valid = false;
  if (hd.fsal) {
    const size_t stage_bytes = n3 * (f32 ? sizeof(float) : sizeof(double));
    if (f32) {
      CS_(ensure_rk32(c));
      CK(cudaMemcpy(c->k32[0], p, stage_bytes, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c->comp64, p + stage_bytes, n3 * sizeof(double), cudaMemcpyHostToDevice));
      c->last32 = c->k32[0];
    } else {
      CS_(ensure_rk(c));
      CK(cudaMemcpy(c->k[0], p, stage_bytes, cudaMemcpyHostToDevice));
    }
    c->fsal_valid = true;
    c->fsal_t = hd.t;
    c->fsal_h = h;
    c->fsal_g = warm;
  }
  *t = hd.t;
  *dt = hd.dt;
  c->stats.t = hd.t;
  c->stats.dt = hd.dt;
  return SCFFT_OK;
}

scfft_status scfft_integrate(scfft_ctx* c, double t0, double t1, double dt0, int nsnap, const double* tsnap, double* h,
                             double* snaps, double* warm, const double* dt_fixed, int nfixed, scfft_stats* stats) {
  if (!c || !h || !(t1 > t0) || !(dt0 > 0) || nsnap < 0 || (nsnap > 0 && (!tsnap || !snaps))) return SCFFT_EINVAL;
  if (dt_fixed && nfixed <= 0) return SCFFT_EINVAL;
  for (int i = 0; i < nsnap; ++i)
    if (!(tsnap[i] > t0 && tsnap[i] <= t1) || (i > 0 && !(tsnap[i] > tsnap[i - 1]))) return SCFFT_EINVAL;
  if (!c->have_geom || !c->have_kernel || !c->have_path) return SCFFT_ESTATE;
  CS_(ensure_rk(c));
  const long long n3 = 3 * c->g.N;
  double* g = warm ? warm : c->ib + 6 * n3;
  if (!warm) {
    double hd[3];
    hedot_at(c, t0, 0, hd);
    CK(run(c, SCFFT_K_RK, [&] {
      fill3_kernel<<<blocks_for(c->g.N), 256, 0, c->st>>>(g, hd[0], hd[1], hd[2], c->g.N);
      return cudaGetLastError();
    }));
  }
  const scfft_stats before = c->stats;
  c->fsal_valid = false;
  double t = t0, dt = dt0;
  int snap_i = 0, nsteps = 0;
  while (t < t1) {
    const double tstop = snap_i < nsnap ? tsnap[snap_i] : t1;
    if (dt_fixed && nsteps >= nfixed) break;
    CS_(step_any(c, &t, &dt, tstop, h, g, dt_fixed ? dt_fixed[nsteps] : 0.0, nullptr));
    ++nsteps;
    if (snap_i < nsnap && t == tsnap[snap_i]) {
      CK(cudaMemcpyAsync(snaps + (size_t)snap_i * n3, h, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->st));
      ++snap_i;
    }
  }
  CK(cudaStreamSynchronize(c->st));
  if (stats) {
    *stats = c->stats;
    stats->accepted = c->stats.accepted - before.accepted;
    stats->rejected = c->stats.rejected - before.rejected;
    stats->rhs_calls = c->stats.rhs_calls - before.rhs_calls;
    stats->iterations = c->stats.iterations - before.iterations;
    stats->launches = c->stats.launches - before.launches;
    stats->h2d_bytes = c->stats.h2d_bytes - before.h2d_bytes;
    stats->d2h_bytes = c->stats.d2h_bytes - before.d2h_bytes;
  }
  return SCFFT_OK;
}

scfft_status scfft_rhs_vjp(scfft_ctx* c, const double* h, const double* lam, double* mu_h, double* mu_g, double* mu_jc,
                           double* mu_a) {
  if (!c || !h || !lam || !mu_h || mu_h == h || mu_h == lam) return SCFFT_EINVAL;
  if (!c->have_geom || !c->have_kernel || c->law || c->curl_kind != SCFFT_CURL_SPECTRAL) return SCFFT_ESTATE;
  c->fsal_valid = false;
  return by_prec(c, [&](auto z) { return vjp_impl<decltype(z)>(c, h, lam, mu_h, mu_g, mu_jc, mu_a); });
}

}  // extern "C"

// Reverse mode of the BS23 map over a recorded, frozen step list (see scfft.h).
namespace {

struct AdjBufs {
  double* base = nullptr;
  double *y, *k1, *k2, *k3, *k4, *Y, *Y2, *yn, *w, *k1b, *k2b, *k3b, *k4b, *mh, *mg, *jct;
  double *cpy, *cpk, *sgy, *sgk;
};

}  // namespace

// A recorded trajectory: step times, kink flags, checkpoints (y_n, k1_n) every C steps, the
// segment currently recomputed, and the cotangent of the next step's first stage.
struct AdjRec {
  AdjBufs b;
  int S = 0, C = 1, ncp = 0;
  std::vector<double> ts;
  std::vector<char> left;  // step n ends on a kink of the path
  int next = -1;           // the step index the next scfft_adjoint_step must take
  int seg = -1;            // checkpoint segment whose states are in sgy / sgk
  bool g0_fill = true;     // the first warm start was dh_e/dt(t_0) (its cotangent goes to the path)
};

namespace {

void free_rec(scfft_ctx* c) {
  if (!c->rec) return;
  cudaFree(c->rec->b.base);
  delete c->rec;
  c->rec = nullptr;
}

scfft_status adj_alloc(scfft_ctx* c, int ncp, int seg, AdjBufs& b) {
  const size_t n3 = 3 * (size_t)c->g.N, N = (size_t)c->g.N;
  const size_t total = 15 * n3 + N + 2 * (size_t)ncp * n3 + 2 * (size_t)seg * n3;
  if (cudaMalloc(&b.base, sizeof(double) * total) != cudaSuccess) {
    cudaGetLastError();
    b.base = nullptr;
    return SCFFT_ENOMEM;
  }
  double* p = b.base;
  double** arr[] = {&b.y,  &b.k1, &b.k2,  &b.k3,  &b.k4,  &b.Y,  &b.Y2, &b.yn,
                    &b.w,  &b.k1b, &b.k2b, &b.k3b, &b.k4b, &b.mh, &b.mg};
  for (double** a : arr) { *a = p; p += n3; }
  b.jct = p; p += N;
  b.cpy = p; p += (size_t)ncp * n3;
  b.cpk = p; p += (size_t)ncp * n3;
  b.sgy = p; p += (size_t)seg * n3;
  b.sgk = p;
  return SCFFT_OK;
}

// out = x + a*y over n values (out may alias x)
cudaError_t axpy(scfft_ctx* c, double* out, const double* x, double a, const double* y, long long n) {
  return run(c, SCFFT_K_RK, [&] {
    combine_kernel<<<blocks_for(n), 256, 0, c->st>>>(out, x, 1.0, a, y, 0, nullptr, 0, nullptr, n);
    return cudaGetLastError();
  });
}

__global__ void scale_kernel(double* __restrict__ out, double a, const double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a * x[i];
}

cudaError_t scal(scfft_ctx* c, double* out, double a, const double* x, long long n) {
  return run(c, SCFFT_K_RK, [&] {
    scale_kernel<<<blocks_for(n), 256, 0, c->st>>>(out, a, x, n);
    return cudaGetLastError();
  });
}

// k_out = F(t, Y; warm = g) (left: the left derivative of h_e at t), leaving g untouched
scfft_status rhs_keep(scfft_ctx* c, AdjBufs& b, double t, int left, const double* Y, const double* g, double* out) {
  const size_t n3 = 3 * (size_t)c->g.N;
  CK(cudaMemcpyAsync(b.w, g, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->st));
  return rhs_any(c, t, left, Y, b.w, out, nullptr);
}

// forward stages of step n from (y, k1): fills Y2, k2, Y (= Y3), k3, yn (= y'), and k4 when
// the step ends on a kink (the last stage, taken with the left derivative there)
scfft_status adj_stages(scfft_ctx* c, AdjRec& r, int n, const double* y, const double* k1) {
  AdjBufs& b = r.b;
  const long long n3 = 3 * c->g.N;
  const double t = r.ts[n], dt = r.ts[n + 1] - r.ts[n];
  CK(axpy(c, b.Y2, y, dt * 0.5, k1, n3));
  CS_(rhs_keep(c, b, t + 0.5 * dt, 0, b.Y2, k1, b.k2));
  CK(axpy(c, b.Y, y, dt * 0.75, b.k2, n3));
  CS_(rhs_keep(c, b, t + 0.75 * dt, 0, b.Y, b.k2, b.k3));
  CK(run(c, SCFFT_K_RK, [&] {
    combine_kernel<<<blocks_for(n3), 256, 0, c->st>>>(b.yn, y, dt, 2.0 / 9.0, k1, 1.0 / 3.0, b.k2, 4.0 / 9.0, b.k3,
                                                      n3);
    return cudaGetLastError();
  }));
  if (r.left[n]) CS_(rhs_keep(c, b, r.ts[n + 1], 1, b.yn, b.k3, b.k4));
  return SCFFT_OK;
}

// the first stage of step n + 1 from the stages of step n: the FSAL stage F(t_{n+1}, y'; g = k3),
// or after a kink F(t_{n+1}, y'; g = k4) with the right derivative
scfft_status adj_next_k1(scfft_ctx* c, AdjRec& r, int n, double* k1_out) {
  return rhs_keep(c, r.b, r.ts[n + 1], 0, r.b.yn, r.left[n] ? r.b.k4 : r.b.k3, k1_out);
}

// dJ/d(path parameters) += (d(dh_e/dt)(t) / d params)^T mu: the knot amplitudes (3 per knot)
// through the rate of the linear piece that holds t (on the side `left` picks at a kink), and
// sin_amp through the rate of the sine inside its window
void path_grad(const scfft_ctx* c, double t, int left, const double mu[3], double* gp) {
  if (!gp) return;
  const int K = (int)c->kt.size();
  for (int s = 0; s + 1 < K; ++s) {
    const double lo = c->kt[s], hi = c->kt[s + 1];
    const bool in = left ? (lo < t && t <= hi) : (lo <= t && t < hi);
    if (in) {
      const double w = 1.0 / (hi - lo);
      for (int a = 0; a < 3; ++a) {
        gp[3 * (s + 1) + a] += w * mu[a];
        gp[3 * s + a] -= w * mu[a];
      }
      break;
    }
  }
  const bool ins = left ? (c->sin_t0 < t && t <= c->sin_t1) : (c->sin_t0 <= t && t < c->sin_t1);
  if (ins && c->sin_period > 0) {
    const double w = 2 * M_PI / c->sin_period;
    gp[3 * K] += w * cos(w * (t - c->sin_t0)) * (c->sin_dir[0] * mu[0] + c->sin_dir[1] * mu[1] + c->sin_dir[2] * mu[2]);
  }
}

// one rhs call's transpose at (t, left): mh = (dF/dh)^T lam, mg = (dF/dg)^T lam; jc and path
// cotangents accumulated
scfft_status adj_call(scfft_ctx* c, AdjRec& r, double t, int left, const double* Y, const double* lam,
                      double* grad_jc, double* grad_path, double* mu_a_acc) {
  AdjBufs& b = r.b;
  double ma[3];
  CS_(by_prec(c, [&](auto z) { return vjp_impl<decltype(z)>(c, Y, lam, b.mh, b.mg, grad_jc ? b.jct : nullptr, ma); }));
  if (grad_jc) CK(axpy(c, grad_jc, grad_jc, 1.0, b.jct, c->g.N));
  path_grad(c, t, left, ma, grad_path);
  if (mu_a_acc)
    for (int q = 0; q < 3; ++q) mu_a_acc[q] += ma[q];
  return SCFFT_OK;
}

// the frozen forward map over ts[0..S] from y0 (warm start warm0, or dh_e/dt(t_0) when NULL)
scfft_status adj_record(scfft_ctx* c, const double* ts, int S, const double* y0, const double* warm0, int C,
                        double* y_end) {
  free_rec(c);
  AdjRec* r = new (std::nothrow) AdjRec();
  if (!r) return SCFFT_ENOMEM;
  r->S = S;
  r->C = std::min(C, S);
  r->ncp = (S + r->C - 1) / r->C;
  r->ts.assign(ts, ts + S + 1);
  const std::vector<double> kinks = kinks_of(c);
  r->left.resize(S);
  for (int n = 0; n < S; ++n) r->left[n] = std::binary_search(kinks.begin(), kinks.end(), ts[n + 1]) ? 1 : 0;
  r->g0_fill = warm0 == nullptr;
  const scfft_status sa = adj_alloc(c, r->ncp, r->C, r->b);
  if (sa != SCFFT_OK) {
    delete r;
    return sa;
  }
  c->rec = r;
  AdjBufs& b = r->b;
  const long long n3 = 3 * c->g.N;
  const size_t bytes = sizeof(double) * n3;
  if (warm0) {
    CK(cudaMemcpyAsync(b.k4b, warm0, bytes, cudaMemcpyDeviceToDevice, c->st));
  } else {
    double g0[3];
    hedot_at(c, ts[0], 0, g0);
    CK(run(c, SCFFT_K_RK, [&] {
      fill3_kernel<<<blocks_for(c->g.N), 256, 0, c->st>>>(b.k4b, g0[0], g0[1], g0[2], c->g.N);
      return cudaGetLastError();
    }));
  }
  // the checkpoint area holds the first warm start until it is consumed by k1_0
  CK(cudaMemcpyAsync(b.y, y0, bytes, cudaMemcpyDeviceToDevice, c->st));
  CS_(rhs_keep(c, b, ts[0], 0, b.y, b.k4b, b.k1));
  for (int n = 0; n < S; ++n) {
    if (n % r->C == 0) {
      CK(cudaMemcpyAsync(b.cpy + (size_t)(n / r->C) * n3, b.y, bytes, cudaMemcpyDeviceToDevice, c->st));
      CK(cudaMemcpyAsync(b.cpk + (size_t)(n / r->C) * n3, b.k1, bytes, cudaMemcpyDeviceToDevice, c->st));
    }
    CS_(adj_stages(c, *r, n, b.y, b.k1));
    CS_(adj_next_k1(c, *r, n, b.k1));
    CK(cudaMemcpyAsync(b.y, b.yn, bytes, cudaMemcpyDeviceToDevice, c->st));
  }
  if (y_end) CK(cudaMemcpyAsync(y_end, b.y, bytes, cudaMemcpyDeviceToDevice, c->st));
  // cotangent of the first stage of the step after the last: none
  CK(cudaMemsetAsync(b.k1b, 0, bytes, c->st));
  CK(cudaStreamSynchronize(c->st));
  r->next = S - 1;
  r->seg = -1;
  return SCFFT_OK;
}

// reverse of step n: lam (device 3N) in: cotangent of y_{n+1}; out: of y_n
scfft_status adj_step(scfft_ctx* c, int n, double* lam, double* grad_jc, double* grad_path, double* mu_a_acc) {
  AdjRec& r = *c->rec;
  AdjBufs& b = r.b;
  const long long n3 = 3 * c->g.N;
  const size_t bytes = sizeof(double) * n3;
  const int m = n / r.C, n0 = m * r.C, n1 = std::min(r.S, n0 + r.C);
  if (r.seg != m) {  // recompute the segment's (y_i, k1_i) from its checkpoint
    CK(cudaMemcpyAsync(b.sgy, b.cpy + (size_t)m * n3, bytes, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(b.sgk, b.cpk + (size_t)m * n3, bytes, cudaMemcpyDeviceToDevice, c->st));
    for (int i = n0; i + 1 < n1; ++i) {
      double* yi = b.sgy + (size_t)(i - n0) * n3;
      double* ki = b.sgk + (size_t)(i - n0) * n3;
      CS_(adj_stages(c, r, i, yi, ki));
      CK(cudaMemcpyAsync(yi + n3, b.yn, bytes, cudaMemcpyDeviceToDevice, c->st));
      CS_(adj_next_k1(c, r, i, ki + n3));
    }
    r.seg = m;
  }
  const double t = r.ts[n], t1 = r.ts[n + 1], dt = t1 - t;
  const double* yi = b.sgy + (size_t)(n - n0) * n3;
  const double* ki = b.sgk + (size_t)(n - n0) * n3;
  CS_(adj_stages(c, r, n, yi, ki));  // Y2, k2, Y (= Y3), k3, yn (= y_{n+1}), k4 at a kink
  if (n + 1 < r.S) {
    // the next step's first stage (cotangent k1b); the last step's is not part of the map
    CS_(adj_call(c, r, t1, 0, b.yn, b.k1b, grad_jc, grad_path, mu_a_acc));
    CK(axpy(c, lam, lam, 1.0, b.mh, n3));
    if (r.left[n]) {  // k1' = F(t1+, y'; g = k4), k4 = F(t1-, y'; g = k3)
      CK(cudaMemcpyAsync(b.k4b, b.mg, bytes, cudaMemcpyDeviceToDevice, c->st));
      CS_(adj_call(c, r, t1, 1, b.yn, b.k4b, grad_jc, grad_path, mu_a_acc));
      CK(axpy(c, lam, lam, 1.0, b.mh, n3));
    }
    CK(cudaMemcpyAsync(b.k3b, b.mg, bytes, cudaMemcpyDeviceToDevice, c->st));
  } else {
    CK(cudaMemsetAsync(b.k3b, 0, bytes, c->st));
  }
  // y' = y + dt (b1 k1 + b2 k2 + b3 k3)
  CK(scal(c, b.k1b, dt * 2.0 / 9.0, lam, n3));
  CK(scal(c, b.k2b, dt / 3.0, lam, n3));
  CK(axpy(c, b.k3b, b.k3b, dt * 4.0 / 9.0, lam, n3));
  // k3 = F(t + 3dt/4, Y3; g = k2), Y3 = y + dt a32 k2
  CS_(adj_call(c, r, t + 0.75 * dt, 0, b.Y, b.k3b, grad_jc, grad_path, mu_a_acc));
  CK(axpy(c, lam, lam, 1.0, b.mh, n3));
  CK(axpy(c, b.k2b, b.k2b, dt * 0.75, b.mh, n3));
  CK(axpy(c, b.k2b, b.k2b, 1.0, b.mg, n3));
  // k2 = F(t + dt/2, Y2; g = k1), Y2 = y + dt a21 k1
  CS_(adj_call(c, r, t + 0.5 * dt, 0, b.Y2, b.k2b, grad_jc, grad_path, mu_a_acc));
  CK(axpy(c, lam, lam, 1.0, b.mh, n3));
  CK(axpy(c, b.k1b, b.k1b, dt * 0.5, b.mh, n3));
  CK(axpy(c, b.k1b, b.k1b, 1.0, b.mg, n3));
  r.next = n - 1;
  if (n == 0) {
    // k1_0 = F(t_0, y_0; g_0)
    CS_(adj_call(c, r, t, 0, b.cpy, b.k1b, grad_jc, grad_path, mu_a_acc));
    CK(axpy(c, lam, lam, 1.0, b.mh, n3));
    if (r.g0_fill && (grad_path || mu_a_acc)) {
      // g_0 = dh_e/dt(t_0) at every node: its cotangent is the node sum of mg
      CK(run(c, SCFFT_K_OTHER, [&] {
        chib_sum_kernel<<<kSumBlocks, 256, 0, c->st>>>(b.mg, c->mask, c->g.N, c->adj_part);
        return cudaGetLastError();
      }));
      CK(cudaMemcpyAsync(c->hadj_part, c->adj_part, sizeof(double) * 3 * kSumBlocks, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      double mg0[3] = {0, 0, 0};
      for (int bk = 0; bk < kSumBlocks; ++bk)
        for (int q = 0; q < 3; ++q) mg0[q] += c->hadj_part[bk * 3 + q];
      path_grad(c, t, 0, mg0, grad_path);
      if (mu_a_acc)
        for (int q = 0; q < 3; ++q) mu_a_acc[q] += mg0[q];
    }
    r.next = -2;  // finished
  }
  CK(cudaStreamSynchronize(c->st));
  return SCFFT_OK;
}

// run f with Eq. 5 frozen at exactly max_iter iterations (the map the reverse mode describes)
template <typename F> scfft_status frozen(scfft_ctx* c, F&& f) {
  const double saved = c->opt.delta_it;
  c->opt.delta_it = 0.0;
  c->fsal_valid = false;
  const scfft_status s = f();
  c->opt.delta_it = saved;
  return s;
}

}  // namespace

extern "C" {

scfft_status scfft_adjoint_record(scfft_ctx* c, const double* ts, int nsteps, const double* y0, const double* warm0,
                                  int checkpoint_every, double* y_end) {
  if (!c || !ts || nsteps < 1 || !y0 || checkpoint_every < 1) return SCFFT_EINVAL;
  for (int n = 0; n < nsteps; ++n)
    if (!(ts[n + 1] > ts[n])) return SCFFT_EINVAL;
  if (!c->have_geom || !c->have_kernel || !c->have_path || c->law || c->curl_kind != SCFFT_CURL_SPECTRAL)
    return SCFFT_ESTATE;
  return frozen(c, [&] { return adj_record(c, ts, nsteps, y0, warm0, checkpoint_every, y_end); });
}

scfft_status scfft_adjoint_step(scfft_ctx* c, int step_index, double* lambda_h, double* grad_jc, double* grad_path) {
  if (!c || !lambda_h) return SCFFT_EINVAL;
  if (!c->rec || c->rec->next != step_index || step_index < 0) return SCFFT_ESTATE;
  return frozen(c, [&] { return adj_step(c, step_index, lambda_h, grad_jc, grad_path, nullptr); });
}

scfft_status scfft_adjoint_integrate(scfft_ctx* c, double t0, const double* dts, int nsteps, const double* y0,
                                     const double* lam_T, double* y_end, double* mu_y0, double* mu_jc, double* mu_a,
                                     int checkpoint_every) {
  if (!c || !dts || nsteps < 1 || !y0 || !lam_T || !mu_y0 || checkpoint_every < 1) return SCFFT_EINVAL;
  for (int n = 0; n < nsteps; ++n)
    if (!(dts[n] > 0)) return SCFFT_EINVAL;
  if (!c->have_geom || !c->have_kernel || !c->have_path || c->law || c->curl_kind != SCFFT_CURL_SPECTRAL)
    return SCFFT_ESTATE;
  std::vector<double> ts(nsteps + 1);
  ts[0] = t0;
  for (int n = 0; n < nsteps; ++n) ts[n + 1] = ts[n] + dts[n];
  const scfft_status s = frozen(c, [&]() -> scfft_status {
    CS_(adj_record(c, ts.data(), nsteps, y0, nullptr, checkpoint_every, y_end));
    const size_t bytes = sizeof(double) * 3 * (size_t)c->g.N;
    CK(cudaMemcpyAsync(mu_y0, lam_T, bytes, cudaMemcpyDeviceToDevice, c->st));
    if (mu_jc) CK(cudaMemsetAsync(mu_jc, 0, sizeof(double) * c->g.N, c->st));
    double ma[3] = {0, 0, 0};
    for (int n = nsteps - 1; n >= 0; --n) CS_(adj_step(c, n, mu_y0, mu_jc, nullptr, ma));
    if (mu_a)
      for (int q = 0; q < 3; ++q) mu_a[q] = ma[q];
    return SCFFT_OK;
  });
  free_rec(c);
  return s;
}

namespace {

// One accepted step of every FP32 instance by one launch of the batch graph (see BatchGraph).
scfft_status batch_graph_step(scfft_ctx** ctxs, int nb, double* t, double* dt, const double* tstop, double** h,
                              double** warm, std::vector<scfft_status>& res) {
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  for (int i = 0; i < nb; ++i) {
    bool need = false;
    if (!(dt[i] > 0) || !(tstop[i] > t[i])) return SCFFT_EINVAL;
    if (!ctxs[i]->have_geom || !ctxs[i]->have_kernel || !ctxs[i]->have_path) return SCFFT_ESTATE;
    CS_(advance_prologue(ctxs[i], t[i], dt[i], tstop[i], 1, h[i], warm[i], &need));
  }
  BatchGraph* b = g_batch;
  bool same = b && (int)b->ctx.size() == nb;
  for (int i = 0; same && i < nb; ++i)
    same = b->ctx[i] == ctxs[i] && b->h[i] == h[i] && b->warm[i] == warm[i] && b->epoch[i] == ctxs[i]->epoch &&
           ctxs[i]->k32[0] == ctxs[i]->step_k[0];
  if (!same) {
    free_batch_graph(g_batch);
    g_batch = nullptr;
    b = new (std::nothrow) BatchGraph();
    if (!b) return SCFFT_ENOMEM;
    bool ok = cudaGraphCreate(&b->g, 0) == cudaSuccess && cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) ==
                                                              cudaSuccess;
    for (int i = 0; ok && i < nb; ++i) {
      scfft_ctx* c = ctxs[i];
      ok = add_step_loop(c, b->g, h[i], warm[i]);
      for (int q = 0; q < 4; ++q) c->step_k[q] = c->k32[q];
      b->ctx.push_back(c);
      b->h.push_back(h[i]);
      b->warm.push_back(warm[i]);
      b->epoch.push_back(c->epoch);
      cudaEvent_t e = nullptr;
      ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
      b->ready.push_back(e);
    }
    if (ok) ok = cudaGraphInstantiate(&b->ex, b->g, 0) == cudaSuccess;
    if (!ok) {
      free_batch_graph(b);
      cudaGetLastError();
      return SCFFT_ECUDA;
    }
    g_batch = b;
  }
  cudaStream_t s0 = ctxs[0]->st;
  for (int i = 0; i < nb; ++i) {
    CK(cudaEventRecord(b->ready[i], ctxs[i]->st));
    CK(cudaStreamWaitEvent(s0, b->ready[i], 0));
  }
  CK(cudaGraphLaunch(b->ex, s0));
  for (int i = 0; i < nb; ++i) CK(advance_readback(ctxs[i], s0));
  CK(cudaStreamSynchronize(s0));
  for (int i = 0; i < nb; ++i) {
    int done = 0;
    res[i] = advance_epilogue(ctxs[i], &t[i], &dt[i], h[i], warm[i], &done);
  }
  return SCFFT_OK;
}

}  // namespace

scfft_status scfft_batch_step(scfft_ctx** ctxs, int nb, double* t, double* dt, const double* tstop, double** h,
                              double** warm, scfft_status* status) {
  if (!ctxs || nb < 1 || !t || !dt || !tstop || !h || !warm) return SCFFT_EINVAL;
  bool graphable = true;
  for (int i = 0; i < nb; ++i) {
    if (!ctxs[i] || !h[i] || !warm[i]) return SCFFT_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return SCFFT_EINVAL;  // one context is one instance
    graphable = graphable && ctxs[i]->opt.precision == SCFFT_PREC_F32 && !ctxs[i]->prof_on;
  }
  std::vector<scfft_status> res(nb, SCFFT_OK);
  if (graphable) {
    const scfft_status s = batch_graph_step(ctxs, nb, t, dt, tstop, h, warm, res);
    if (s != SCFFT_OK) return s;
    scfft_status first = SCFFT_OK;
    for (int i = 0; i < nb; ++i) {
      if (status) status[i] = res[i];
      if (first == SCFFT_OK && res[i] != SCFFT_OK) first = res[i];
    }
    return first;
  }
  std::atomic<int> next(0);
  auto worker = [&]() {
    for (int i = next++; i < nb; i = next++) res[i] = scfft_step(ctxs[i], &t[i], &dt[i], tstop[i], h[i], warm[i], nullptr);
  };
  const int nth = std::min(nb, 64);
  std::vector<std::thread> pool;
  pool.reserve(nth - 1);
  for (int k = 1; k < nth; ++k) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  scfft_status first = SCFFT_OK;
  for (int i = 0; i < nb; ++i) {
    if (status) status[i] = res[i];
    if (first == SCFFT_OK && res[i] != SCFFT_OK) first = res[i];
  }
  return first;
}

const char* scfft_last_cuda_error(void) {
  std::lock_guard<std::mutex> lock(g_err_mutex);
  static thread_local char copy[512];
  memcpy(copy, g_err_text, sizeof(copy));
  return copy;
}

scfft_status scfft_sync(scfft_ctx* c) {
  if (!c) return SCFFT_EINVAL;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(c->hctrl + 2, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
  return (scfft_status)c->hctrl[2].status;
}

scfft_status scfft_inject_fault(scfft_ctx* c, int kind) {
  if (!c || (kind != 0 && kind != SCFFT_FAULT_TMA_WAIT)) return SCFFT_EINVAL;
  if (kind != 0 && c->opt.precision != SCFFT_PREC_F32) return SCFFT_EINVAL;
  c->fault = kind;
  return SCFFT_OK;
}

scfft_status scfft_get_stats(scfft_ctx* c, scfft_stats* out) {
  if (!c || !out) return SCFFT_EINVAL;
  if (flush_pending(c) == SCFFT_ECUDA) return SCFFT_ECUDA;  // a latched device status is the next step's to report
  *out = c->stats;
  return SCFFT_OK;
}

scfft_status scfft_profile(scfft_ctx* c, int enable) {
  if (!c) return SCFFT_EINVAL;
  if (enable && c->pev.empty()) {
    c->pev.resize(2 * kProfPool);
    c->pkind.resize(kProfPool);
    for (auto& e : c->pev) CK(cudaEventCreate(&e));
  }
  if (enable) {
    CK(prof_flush(c));
    for (int k = 0; k < SCFFT_NKINDS; ++k) { c->pms[k] = 0; c->pcnt[k] = 0; }
  }
  c->prof_on = enable != 0;
  return SCFFT_OK;
}

scfft_status scfft_profile_read(scfft_ctx* c, long long* counts, double* ms) {
  if (!c || !counts || !ms) return SCFFT_EINVAL;
  CK(prof_flush(c));
  for (int k = 0; k < SCFFT_NKINDS; ++k) { counts[k] = c->pcnt[k]; ms[k] = c->pms[k]; }
  return SCFFT_OK;
}

}  // extern "C"
