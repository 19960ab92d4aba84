// Host side of the C ABI declared in include/icwf.h: handle life cycle, the rank-k factorisation
// of the interaction, the seeded sampler, initialisation, the per-step kernel schedule,
// observables, diagnostics, per-kernel timing and the serving pool.
//
// Compiled with -ffp-contract=off so that the sampler and the grid formulas round exactly as
// written (the sampler must reproduce the published SplitMix64 stream and the inverse-CDF draw
// bit for bit on every host architecture).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "icwf_internal.h"

namespace icwf {
void jacobi_svd(int m, int n, std::vector<double>& A, std::vector<double>& s,
                std::vector<double>& U, std::vector<double>& Vr);
}

using namespace icwf;

namespace {

thread_local std::string g_err;   // last failure without a handle

// NVTX range around a public call (visible in Nsight timelines; no cost without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

enum Fam {
  F_VELOCITY, F_PROPAGATE, F_ASSEMBLE, F_SHIFT, F_POTRF, F_MATVEC, F_SOLVE, F_RK4, F_OBS,
  F_COUNT
};
const char* kFamNames[F_COUNT] = {"velocity", "propagate", "assemble", "shift",
                                  "cholesky", "rk4_matvec", "chol_solve", "rk4_final",
                                  "observables"};

struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  void* take(size_t bytes) {
    const size_t off = (used + 255) & ~(size_t)255;
    if (off + bytes > size) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

struct icwf_ctx {
  icwf_params p{};
  std::string err;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;              // first RK4 stage, beside the assembly and factorisation
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool mixed = false;
  bool df_solve = false;                    // factorisation and solves in double-float arithmetic
  int N = 0, nx = 0, nR = 0, K = 0, logx = 0, logR = 0;
  double dx = 0, dR = 0;
  double tail_rel = 0, next_rel = 0, sigma_max = 0;
  size_t cwf_elem = 16;   // bytes per complex CWF sample
  // device memory
  Arena arena;
  double *V = nullptr, *U = nullptr, *W = nullptr, *sig = nullptr, *v1 = nullptr, *v2 = nullptr;
  void* Vt = nullptr;
  void *kinx = nullptr, *kinR = nullptr, *twx = nullptr, *twR = nullptr;
  double2 *twx_d = nullptr, *twR_d = nullptr;
  void *psi = nullptr, *chi = nullptr;
  double *x = nullptr, *R = nullptr, *xo = nullptr, *Ro = nullptr;
  double *px = nullptr, *pR = nullptr, *dvec = nullptr;
  double2* C = nullptr;
  double2* kk[4] = {nullptr, nullptr, nullptr, nullptr};
  double2 *y = nullptr, *work = nullptr;
  float* cf32 = nullptr;   // C in FP32 (mixed modes)
  double2 *S[2] = {nullptr, nullptr}, *H[2] = {nullptr, nullptr};
  double2 *L[2] = {nullptr, nullptr}, *Lh = nullptr;
  double *invL[2] = {nullptr, nullptr}, *invLh = nullptr;   // reciprocal Cholesky pivots
  double2 *DL[2] = {nullptr, nullptr}, *DLh = nullptr;       // inverted 32 x 32 diagonal blocks
  unsigned *flags = nullptr, *tickets = nullptr;
  unsigned* cctl = nullptr;                                  // blocked-factorisation tickets/flags
  int* status = nullptr;
  int cur = 0;
  unsigned epoch = 0;
  // observables (allocated on first use)
  double2* Psi = nullptr;
  double* phi = nullptr;
  int n_states = 0;
  double *rho_x = nullptr, *rho_R = nullptr, *part = nullptr, *obs_out = nullptr;
  double *pop = nullptr, *decoh = nullptr;
  double2* proj = nullptr;
  std::vector<void*> extra_allocs;
  size_t obs_bytes = 0;                     // observables work buffers (allocated on first use)
  // tensor-core assembly scratch
  void* tc_scratch = nullptr;
  size_t tc_scratch_bytes = 0;
  // FP64 factorisation: digit planes of the emulated trailing update (allocated when !df_solve)
  void* emu_scratch = nullptr;
  size_t emu_bytes = 0;
  bool emu_update = true;                   // trailing updates on the tensor cores
  // state
  bool initialised = false;
  int64_t steps = 0;
  double t = 0.0;
  int64_t launches = 0;   // kernels launched by icwf_step
  int prop_threads = 256; // CTA size of the CWF propagator (autotuned per shape at create)
  // step_once leaves out the velocity and propagation kernels (a serving pool records the job's
  // step this way when grouped kernels over all live jobs do that part of the step)
  bool traj_grouped = false;
  int64_t version = 0;    // bumped by calls that change captured kernel arguments (eps)
  // icwf_step's captured step graphs (one per parity of the ping-pong buffers)
  bool step_graphs = true;
  cudaGraphExec_t step_exec[2] = {nullptr, nullptr};
  int64_t step_exec_version = -1, step_kernels = 0;
  // profiling
  bool prof_on = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> event_pool;
  double prof_ms[F_COUNT] = {0};
  int64_t prof_n[F_COUNT] = {0};
};

namespace {

icwf_status fail(icwf_ctx* h, icwf_status st, const std::string& msg) {
  if (h) h->err = msg; else g_err = msg;
  return st;
}

#define CK_POOL(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(nullptr, ICWF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, ICWF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

JobView view(icwf_ctx* h) {
  JobView j;
  j.N = h->N; j.nx = h->nx; j.nR = h->nR; j.K = h->K; j.logx = h->logx; j.logR = h->logR;
  j.x_min = h->p.x_min; j.dx = h->dx; j.R_min = h->p.R_min; j.dR = h->dR;
  j.inv_mx = 1.0 / h->p.mass_x; j.inv_mR = 1.0 / h->p.mass_R; j.dt = h->p.dt;
  j.eps = h->p.s_reg_eps;
  j.V = h->V; j.Vt = h->Vt; j.U = h->U; j.W = h->W; j.sig = h->sig; j.v1 = h->v1; j.v2 = h->v2;
  j.psi = h->psi; j.chi = h->chi;
  j.x = h->x; j.R = h->R; j.xo = h->xo; j.Ro = h->Ro;
  j.px = h->px; j.pR = h->pR; j.d = h->dvec;
  j.kinx = h->kinx; j.kinR = h->kinR; j.twx = h->twx; j.twR = h->twR;
  j.status = h->status;
  j.scratch_f32 = h->mixed ? h->cf32 : nullptr;
  return j;
}

// ---- per-kernel timing -----------------------------------------------------------------------

cudaEvent_t take_event(icwf_ctx* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void destroy_streams(icwf_ctx* h) {
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->stream) cudaStreamDestroy(h->stream);
  h->ev_fork = h->ev_join = nullptr;
  h->side = h->stream = nullptr;
}

struct ProfScope {
  icwf_ctx* h;
  int fam;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(icwf_ctx* h_, int f, cudaStream_t s_ = nullptr) : h(h_), fam(f), s(s_ ? s_ : h_->stream) {
    if (h->prof_on) {
      a = take_event(h);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (h->prof_on) {
      cudaEvent_t b = take_event(h);
      cudaEventRecord(b, s);
      h->pending.push_back({fam, {a, b}});
    }
  }
};

void prof_collect(icwf_ctx* h) {
  for (auto& pe : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
      h->prof_ms[pe.first] += ms;
      h->prof_n[pe.first] += 1;
    }
    h->event_pool.push_back(pe.second.first);
    h->event_pool.push_back(pe.second.second);
  }
  h->pending.clear();
}

// ---- host numerics --------------------------------------------------------------------------

struct HStencil { int i0; double w[4]; };

// Same stencil as the device one (4-point cubic Lagrange, start clamped to [0, n-4]).
HStencil h_lagrange4(double p, double lo, double d, int n) {
  HStencil st;
  const double s = (p - lo) / d - 0.5;
  int i0 = (int)std::floor(s) - 1;
  i0 = i0 < 0 ? 0 : (i0 > n - 4 ? n - 4 : i0);
  const double u = s - (double)i0;
  const double u1 = u - 1.0, u2 = u - 2.0, u3 = u - 3.0;
  st.i0 = i0;
  st.w[0] = -(u1 * u2 * u3) / 6.0;
  st.w[1] = (u * u2 * u3) / 2.0;
  st.w[2] = -(u * u1 * u3) / 2.0;
  st.w[3] = (u * u1 * u2) / 6.0;
  return st;
}

// SplitMix64 (Steele, Lea, Flood 2014): state += golden gamma; Stafford variant-13 finaliser.
struct SplitMix64 {
  uint64_t s;
  explicit SplitMix64(uint64_t seed) : s(seed) {}
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// Bit-reversed kinetic phase exp(-i k^2 dt / 2m) / n and twiddles exp(-2 pi i k / n).
void kinetic_tables(int n, double d, double mass, double dt, std::vector<double>& kin,
                    std::vector<double>& tw) {
  const int logn = ilog2(n);
  const double PI = 3.14159265358979323846;
  kin.resize(2 * (size_t)n);
  tw.resize(n);   // n/2 complex
  for (int mp = 0; mp < n; ++mp) {
    int m = 0;
    for (int b = 0; b < logn; ++b) if (mp & (1 << b)) m |= 1 << (logn - 1 - b);
    const int mm = m < n / 2 ? m : m - n;
    const double k = 2.0 * PI * (double)mm / ((double)n * d);
    const double ph = -k * k * dt / (2.0 * mass);
    kin[2 * mp] = std::cos(ph) / n;
    kin[2 * mp + 1] = std::sin(ph) / n;
  }
  for (int k = 0; k < n / 2; ++k) {
    const double a = -2.0 * PI * (double)k / (double)n;
    tw[2 * k] = std::cos(a);
    tw[2 * k + 1] = std::sin(a);
  }
}

template <typename T>
std::vector<T> cast_vec(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}

icwf_status upload(icwf_ctx* h, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream));
  return ICWF_OK;
}

icwf_status sync_status(icwf_ctx* h, const char* where) {
  CK(cudaStreamSynchronize(h->stream));
  if (h->prof_on) prof_collect(h);
  int st[2];
  CK(cudaMemcpy(st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st[0] & ST_TIMEOUT) return fail(h, ICWF_ERR_TIMEOUT, std::string(where) + ": in-kernel wait timed out");
  if (st[0] & (ST_NONFINITE | ST_CHOL)) {
    return fail(h, ICWF_ERR_NUMERIC,
                std::string(where) + ((st[0] & ST_CHOL) ? ": Cholesky pivot <= 0 (S + eps I not positive definite)"
                                                        : ": non-finite velocity or coefficient"));
  }
  return ICWF_OK;
}

// Factor the batch dst[m] = chol((1 - theta_m) S0_m + theta_m S1_m + eps I), m < n <= 2: both
// matrices go through the same launches, so their factorisations overlap on the device.
void factor(icwf_ctx* h, int n, const double2* const* S0, const double2* const* S1,
            const double* theta, double2* const* dst, double* const* inv, double2* const* D) {
  {
    ProfScope ps(h, F_SHIFT);
    for (int m = 0; m < n; ++m) {
      if (h->df_solve) launch_shift_mix_df(h->N, S0[m], S1[m], h->p.s_reg_eps, theta[m], dst[m], h->stream);
      else launch_shift_mix(h->N, S0[m], S1[m], h->p.s_reg_eps, theta[m], dst[m], h->stream);
    }
    h->launches += n;
  }
  ProfScope ps(h, F_POTRF);
  if (h->df_solve) {
    void* a[2] = {dst[0], n > 1 ? dst[1] : dst[0]};
    void* iv[2] = {inv[0], n > 1 ? inv[1] : inv[0]};
    void* dd[2] = {D[0], n > 1 ? D[1] : D[0]};
    h->launches += launch_cholesky_df(h->N, a, iv, dd, n, h->cctl, h->status, h->stream);
  } else {
    h->launches += launch_cholesky(h->N, dst, inv, D, n, h->status, h->stream,
                                   h->emu_update ? h->emu_scratch : nullptr, h->emu_bytes);
  }
}

void solve(icwf_ctx* h, const double2* Lf, const double2* D, const double2* y, double2* out,
           bool minus_i, cudaStream_t s = nullptr) {
  if (!s) s = h->stream;
  ProfScope ps(h, F_SOLVE, s);
  h->epoch = 1;   // the launchers zero the block flags before every solve
  if (h->df_solve)
    launch_chol_solve_df(h->N, Lf, D, y, h->work, out, minus_i, h->flags, h->tickets, h->epoch,
                         h->status, s);
  else
    launch_chol_solve(h->N, Lf, D, y, h->work, out, minus_i, h->flags, h->tickets, h->epoch,
                      h->status, s);
  h->launches += 2;
}

void assemble(icwf_ctx* h, double2* S, double2* Hm) {
  ProfScope ps(h, F_ASSEMBLE);
  // operand planes (two sides) + Grams [+ digit planes (two sides) + exact overlap], or the FP64
  // kernel
  h->launches += h->mixed ? (h->p.overlap_split ? 3 : 6) : 1;
  JobView j = view(h);
  if (h->mixed) {
    launch_assemble_tc(j, h->p.precision, h->p.overlap_split == 0, S, Hm, h->tc_scratch,
                       h->tc_scratch_bytes, h->stream);
  } else {
    launch_assemble_fp64(j, S, Hm, h->stream);
  }
}

// One ICWF step t_n -> t_{n+1}.
// The RK4 stages that need only data of t_n (the first stage; all four with frozen matrices) run on
// a side stream from the start of the step, beside the velocities, propagation, assembly and
// factorisation, which do not touch their inputs or outputs; the main stream joins them before
// the later stages (they share the right-hand-side buffer and the solve scratch).
void step_once(icwf_ctx* h) {
  JobView j = view(h);
  const int cur = h->cur, nxt = 1 - cur;
  const double dt = h->p.dt;
  double2 *Lc = h->L[cur], *Ln = h->L[nxt];
  double *in = h->invL[nxt];
  double2 *Dc = h->DL[cur], *Dn = h->DL[nxt];
  const bool frozen = h->p.coeff_scheme == 1;
  cudaEventRecord(h->ev_fork, h->stream);
  cudaStreamWaitEvent(h->side, h->ev_fork, 0);
  for (int st = 0; st < (frozen ? 4 : 1); ++st) {
    // S, Heff at t_n (frozen over the step) or the first stage of the interpolated scheme
    const double c = st == 0 ? 0.0 : (st == 3 ? dt : 0.5 * dt);
    {
      ProfScope ps(h, F_MATVEC, h->side);
      launch_matvec(h->N, h->H[cur], h->H[cur], 0.0, h->C, st ? h->kk[st - 1] : nullptr, c, h->y,
                    h->side);
      h->launches += 1;
    }
    solve(h, Lc, Dc, h->y, h->kk[st], true, h->side);
  }
  cudaEventRecord(h->ev_join, h->side);
  if (!h->traj_grouped) {
    {
      ProfScope ps(h, F_VELOCITY);
      if (h->mixed) launch_velocity<float>(j, h->C, h->stream);
      else launch_velocity<double>(j, h->C, h->stream);
      h->launches += h->mixed ? 2 : 1;
    }
    {
      ProfScope ps(h, F_PROPAGATE);
      if (h->mixed) launch_propagate<float>(j, h->prop_threads, h->stream);
      else launch_propagate<double>(j, h->prop_threads, h->stream);
      h->launches += 1;
    }
  }
  assemble(h, h->S[nxt], h->H[nxt]);
  if (frozen) {
    const double2* s0[1] = {h->S[nxt]};
    const double th[1] = {1.0};
    double2* d[1] = {Ln};
    double* iv[1] = {in};
    double2* dd[1] = {Dn};
    factor(h, 1, s0, s0, th, d, iv, dd);
    cudaStreamWaitEvent(h->stream, h->ev_join, 0);
  } else {
    const double2* s0[2] = {h->S[cur], h->S[nxt]};
    const double2* s1[2] = {h->S[nxt], h->S[nxt]};
    const double th[2] = {0.5, 1.0};
    double2* d[2] = {h->Lh, Ln};
    double* iv[2] = {h->invLh, in};
    double2* dd[2] = {h->DLh, Dn};
    factor(h, 2, s0, s1, th, d, iv, dd);
    cudaStreamWaitEvent(h->stream, h->ev_join, 0);
    const double thetas[4] = {0.0, 0.5, 0.5, 1.0};
    const double2* Ls[4] = {Lc, h->Lh, h->Lh, Ln};
    const double2* Is[4] = {Dc, h->DLh, h->DLh, Dn};
    for (int st = 1; st < 4; ++st) {
      const double c = st == 3 ? dt : 0.5 * dt;
      {
        ProfScope ps(h, F_MATVEC);
        launch_matvec(h->N, h->H[cur], h->H[nxt], thetas[st], h->C, h->kk[st - 1], c, h->y,
                      h->stream);
        h->launches += 1;
      }
      solve(h, Ls[st], Is[st], h->y, h->kk[st], true);
    }
  }
  {
    ProfScope ps(h, F_RK4);
    launch_rk4_final(h->N, h->C, h->kk[0], h->kk[1], h->kk[2], h->kk[3], dt, h->status,
                     h->stream);
    h->launches += 1;
  }
  h->cur = nxt;
  h->steps += 1;
  h->t += dt;
}

// Record two consecutive steps (not executed) into two graphs, g[p] for ping-pong parity p, and
// restore the host-side step state; *kernels receives the kernels of one step.  Returns false
// (with no graph left) if the capture fails.
bool capture_step(icwf_ctx* h, cudaGraph_t g[2], int64_t* kernels) {
  const bool prof = h->prof_on;
  const int cur0 = h->cur;
  const int64_t steps0 = h->steps, l0 = h->launches;
  const double t0 = h->t;
  h->prof_on = false;
  g[0] = g[1] = nullptr;
  bool ok = true;
  for (int k = 0; k < 2 && ok; ++k) {
    const int par = h->cur;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      ok = false;
      break;
    }
    step_once(h);
    cudaGraph_t gr = nullptr;
    if (cudaStreamEndCapture(h->stream, &gr) != cudaSuccess || !gr) {
      ok = false;
      if (gr) cudaGraphDestroy(gr);
      break;
    }
    g[par] = gr;
  }
  *kernels = (h->launches - l0) / 2;
  h->cur = cur0;
  h->steps = steps0;
  h->t = t0;
  h->launches = l0;
  h->prof_on = prof;
  if (!ok) {
    for (int k = 0; k < 2; ++k)
      if (g[k]) { cudaGraphDestroy(g[k]); g[k] = nullptr; }
    cudaGetLastError();   // the failed capture's own error; the caller launches directly
  }
  return ok;
}

void drop_step_graphs(icwf_ctx* h) {
  for (auto& e : h->step_exec)
    if (e) { cudaGraphExecDestroy(e); e = nullptr; }
  h->step_exec_version = -1;
}

// The handle's instantiated step graphs, (re)built when missing or when a captured argument
// changed; false if they cannot be built (icwf_step then launches directly).
bool step_graphs_ready(icwf_ctx* h) {
  if (h->step_exec[0] && h->step_exec_version == h->version) return true;
  drop_step_graphs(h);
  cudaGraph_t g[2];
  if (!capture_step(h, g, &h->step_kernels)) return false;
  bool ok = true;
  for (int k = 0; k < 2; ++k) {
    if (ok && cudaGraphInstantiate(&h->step_exec[k], g[k], 0) != cudaSuccess) ok = false;
    cudaGraphDestroy(g[k]);
  }
  if (!ok) {
    drop_step_graphs(h);
    cudaGetLastError();
    return false;
  }
  h->step_exec_version = h->version;
  return true;
}

// ---- autotuner ------------------------------------------------------------------------------
// The CWF propagator (one CTA per CWF, radix-2 FFT over the column in shared memory) is launched
// with the CTA size that measured fastest for the problem shape (precision, N, nx, nR): 64, 128,
// 256 or 512 threads, each timed over three launches with CUDA events on the handle's own
// buffers (zeroed first) when the first handle of that shape is created.  Results are cached for
// the process; later handles of the same shape reuse them.

struct TuneKey {
  int prec, N, nx, nR;
  bool operator<(const TuneKey& o) const {
    if (prec != o.prec) return prec < o.prec;
    if (N != o.N) return N < o.N;
    if (nx != o.nx) return nx < o.nx;
    return nR < o.nR;
  }
};
std::mutex g_tune_mutex;
std::map<TuneKey, int> g_tune;

int tune_propagate(icwf_ctx* h) {
  const TuneKey key{h->mixed ? 1 : 0, h->N, h->nx, h->nR};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  const size_t cw = h->cwf_elem;
  cudaMemsetAsync(h->psi, 0, (size_t)h->N * h->nx * cw, h->stream);
  cudaMemsetAsync(h->chi, 0, (size_t)h->N * h->nR * cw, h->stream);
  for (double* q : {h->x, h->R, h->xo, h->Ro}) cudaMemsetAsync(q, 0, (size_t)h->N * 8, h->stream);
  JobView j = view(h);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = 256;
  float best_ms = 1e30f;
  for (int threads : {64, 128, 256, 512}) {
    auto go = [&]() {
      if (h->mixed) launch_propagate<float>(j, threads, h->stream);
      else launch_propagate<double>(j, threads, h->stream);
    };
    go();
    cudaEventRecord(e0, h->stream);
    for (int r = 0; r < 3; ++r) go();
    cudaEventRecord(e1, h->stream);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      continue;
    if (ms < best_ms) { best_ms = ms; best = threads; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune[key] = best;
  return best;
}

icwf_status alloc_obs(icwf_ctx* h) {
  if (h->Psi) return ICWF_OK;
  void* p = nullptr;
  const size_t bytes = align256((size_t)h->nx * h->nR * sizeof(double2)) +
                       align256((size_t)(h->nx + h->nR) * sizeof(double)) * 2 +
                       align256((size_t)(2 * h->nR + h->nx) * sizeof(double)) + align256(64 * sizeof(double)) +
                       align256(8 * sizeof(double)) + align256(64 * sizeof(double)) +
                       align256((size_t)8 * h->nR * sizeof(double2));
  CK(cudaMalloc(&p, bytes));
  h->extra_allocs.push_back(p);
  h->obs_bytes = bytes;
  Arena a{(char*)p, bytes, 0};
  h->Psi = (double2*)a.take((size_t)h->nx * h->nR * sizeof(double2));
  h->rho_x = (double*)a.take((size_t)(h->nx + h->nR) * sizeof(double));
  h->rho_R = (double*)a.take((size_t)(h->nx + h->nR) * sizeof(double));
  h->part = (double*)a.take((size_t)(2 * h->nR + h->nx) * sizeof(double));
  h->obs_out = (double*)a.take(64 * sizeof(double));
  h->pop = (double*)a.take(8 * sizeof(double));
  h->decoh = (double*)a.take(64 * sizeof(double));
  h->proj = (double2*)a.take((size_t)8 * h->nR * sizeof(double2));
  return ICWF_OK;
}

}  // namespace

namespace icwf {

bool handle_obs_view(icwf_handle h, ObsView* v) {
  if (!h || !v) return false;
  v->j = view(h);
  v->C = h->C;
  v->phi = h->phi;
  v->n_states = h->n_states;
  v->mixed = h->mixed;
  v->initialised = h->initialised;
  v->twx_d = h->twx_d;
  v->twR_d = h->twR_d;
  v->stream = h->stream;
  v->device = h->device;
  v->t = h->t;
  return true;
}

void handle_set_error(icwf_handle h, const char* msg) {
  if (h) h->err = msg; else g_err = msg;
}

}  // namespace icwf

// ============================================================================================
// C ABI
// ============================================================================================

extern "C" {

const char* icwf_last_error(icwf_handle h) { return h ? h->err.c_str() : g_err.c_str(); }

icwf_status icwf_create(const icwf_params* pp, const double* Vh, icwf_handle* out) {
  icwf_ctx* h = nullptr;
  if (!out) return fail(nullptr, ICWF_ERR_ARG, "icwf_create: out is NULL");
  *out = nullptr;
  if (!pp || !Vh) return fail(nullptr, ICWF_ERR_ARG, "icwf_create: params or V is NULL");
  const icwf_params& p = *pp;
  if (!pow2(p.nx) || !pow2(p.nR) || p.nx < 8 || p.nR < 8 || p.nx > 4096 || p.nR > 4096)
    return fail(nullptr, ICWF_ERR_ARG, "icwf_create: nx and nR must be powers of two in [8, 4096]");
  if (p.n_traj < 1 || p.n_traj > 16384)
    return fail(nullptr, ICWF_ERR_ARG, "icwf_create: n_traj must be in [1, 16384]");
  if (!(p.x_max > p.x_min) || !(p.R_max > p.R_min) || !(p.mass_x > 0) || !(p.mass_R > 0) ||
      !(p.dt > 0) || !(p.s_reg_eps >= 0) || !(p.svd_rel_cutoff >= 0))
    return fail(nullptr, ICWF_ERR_ARG, "icwf_create: invalid extents, masses, dt, eps or cutoff");
  if (p.precision < 0 || p.precision > 2)
    return fail(nullptr, ICWF_ERR_ARG, "icwf_create: unknown precision");
  if (p.precision != ICWF_FP64 && assemble_tc_scratch_bytes(p.n_traj, p.nx, p.nR, 1) == 0)
    return fail(nullptr, ICWF_ERR_ARG, "icwf_create: mixed precision is not available in this library");
  if (p.coeff_scheme < 0 || p.coeff_scheme > 1)
    return fail(nullptr, ICWF_ERR_ARG, "icwf_create: unknown coeff_scheme");
  if (p.precision != ICWF_FP64 && (p.nx < 64 || p.nR < 64))
    return fail(nullptr, ICWF_ERR_ARG, "icwf_create: mixed precision needs nx, nR >= 64");
  if (p.overlap_split < 0 || p.overlap_split > 1)
    return fail(nullptr, ICWF_ERR_ARG, "icwf_create: overlap_split must be 0 or 1");
  const size_t nV = (size_t)p.nx * p.nR;
  for (size_t e = 0; e < nV; ++e)
    if (!std::isfinite(Vh[e])) return fail(nullptr, ICWF_ERR_ARG, "icwf_create: V has a non-finite entry");

  std::unique_ptr<icwf_ctx> hp(new icwf_ctx);
  h = hp.get();
  h->p = p;
  h->N = p.n_traj; h->nx = p.nx; h->nR = p.nR;
  h->logx = ilog2(p.nx); h->logR = ilog2(p.nR);
  h->dx = (p.x_max - p.x_min) / p.nx;
  h->dR = (p.R_max - p.R_min) / p.nR;
  h->mixed = p.precision != ICWF_FP64;
  h->df_solve = h->mixed && !p.solve_fp64;
  h->cwf_elem = h->mixed ? sizeof(float2) : sizeof(double2);
  cudaGetDevice(&h->device);

  // ---- double-centring and SVD of the interaction (host, FP64) ----
  const int nx = p.nx, nR = p.nR;
  std::vector<double> v1(nx, 0.0), v2(nR, 0.0);
  double grand = 0.0;
  for (int i = 0; i < nx; ++i) {
    double s = 0.0;
    for (int jj = 0; jj < nR; ++jj) s += Vh[(size_t)i * nR + jj];
    v1[i] = s / nR;
  }
  for (int jj = 0; jj < nR; ++jj) {
    double s = 0.0;
    for (int i = 0; i < nx; ++i) s += Vh[(size_t)i * nR + jj];
    v2[jj] = s / nx;
  }
  for (int i = 0; i < nx; ++i) grand += v1[i];
  grand /= nx;
  for (int jj = 0; jj < nR; ++jj) v2[jj] -= grand;
  // V_c column-major in the longer dimension so that m >= n
  const bool tr = nx < nR;
  const int m = tr ? nR : nx, n = tr ? nx : nR;
  std::vector<double> A((size_t)m * n);
  double fro2 = 0.0;
  for (int i = 0; i < nx; ++i)
    for (int jj = 0; jj < nR; ++jj) {
      const double vc = Vh[(size_t)i * nR + jj] - v1[i] - v2[jj];
      fro2 += vc * vc;
      if (!tr) A[(size_t)jj * nx + i] = vc; else A[(size_t)i * nR + jj] = vc;
    }
  std::vector<double> s, Um, Vr;
  jacobi_svd(m, n, A, s, Um, Vr);
  int K = n;
  double tail2 = 0.0;
  {
    // smallest k whose Frobenius tail is within the cutoff
    std::vector<double> tails(n + 1, 0.0);
    for (int k = n - 1; k >= 0; --k) tails[k] = tails[k + 1] + s[k] * s[k];
    const double fro = std::sqrt(tails[0]);
    if (p.svd_rel_cutoff > 0 && fro > 0) {
      K = n;
      for (int k = 0; k < n; ++k)
        if (std::sqrt(tails[k]) <= p.svd_rel_cutoff * fro) { K = k; break; }
    }
    if (p.max_rank > 0 && K > p.max_rank) K = p.max_rank;
    tail2 = tails[K];
    h->tail_rel = fro > 0 ? std::sqrt(tail2) / fro : 0.0;
    h->next_rel = (K < n && s[0] > 0) ? s[K] / s[0] : 0.0;
    h->sigma_max = n > 0 ? s[0] : 0.0;
  }
  if (K < 1) K = 1;   // keep one (possibly zero) term so that the kernels see K >= 1
  h->K = K;
  std::vector<double> Uk((size_t)K * nx), Wk((size_t)K * nR), sk(K);
  for (int k = 0; k < K; ++k) {
    sk[k] = k < n ? s[k] : 0.0;
    for (int i = 0; i < nx; ++i) Uk[(size_t)k * nx + i] = tr ? Vr[(size_t)k * n + i] : Um[(size_t)k * m + i];
    for (int jj = 0; jj < nR; ++jj) Wk[(size_t)k * nR + jj] = tr ? Um[(size_t)k * m + jj] : Vr[(size_t)k * n + jj];
  }

  // ---- device memory ----
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    destroy_streams(h);
    return fail(nullptr, ICWF_ERR_CUDA, "icwf_create: cudaStreamCreate failed");
  }
  const int N = h->N;
  const size_t cw = h->cwf_elem, rw = h->mixed ? sizeof(float) : sizeof(double);
  const size_t NN = (size_t)N * N;
  const int nblk = (N + 31) / 32;
  std::vector<size_t> sizes = {
      nV * sizeof(double), nV * rw, (size_t)K * nx * 8, (size_t)K * nR * 8, (size_t)K * 8,
      (size_t)nx * 8, (size_t)nR * 8,
      (size_t)nx * cw, (size_t)nR * cw, (size_t)nx / 2 * cw, (size_t)nR / 2 * cw,
      (size_t)nx / 2 * 16, (size_t)nR / 2 * 16,
      (size_t)N * nx * cw, (size_t)N * nR * cw,
      (size_t)N * 8 * 4, (size_t)K * N * 8 * 2, (size_t)N * 8,
      (size_t)N * 16 * 8,  // C, k1..k4, y, work(2N)
      (size_t)N * 8,       // C in FP32
      NN * 16 * 7,         // S[2], H[2], L[2], Lh
      (size_t)N * 8, (size_t)N * 8, (size_t)N * 8,   // reciprocal pivots of L[2], Lh
      (size_t)N * 512, (size_t)N * 512, (size_t)N * 512,   // inverted diagonal blocks
      (size_t)2 * nblk * 4 + 64, chol_ctl_words(N) * sizeof(unsigned), 64 * 4};
  size_t total = 0;
  for (size_t b : sizes) total += align256(b);
  if (h->mixed) {
    h->tc_scratch_bytes = assemble_tc_scratch_bytes(N, nx, nR, K);
    total += align256(h->tc_scratch_bytes);
  }
  if (!h->df_solve) {
    h->emu_bytes = herk_emu_scratch_bytes(N);
    total += align256(h->emu_bytes);
    herk_emu_attributes();
  }
  total += 4096;
  if (cudaMalloc(&h->arena.base, total) != cudaSuccess) {
    destroy_streams(h);
    return fail(nullptr, ICWF_ERR_OOM, "icwf_create: cudaMalloc of " + std::to_string(total) + " bytes failed");
  }
  h->arena.size = total;
  Arena& a = h->arena;
  h->V = (double*)a.take(nV * 8);
  h->Vt = a.take(nV * rw);
  h->U = (double*)a.take((size_t)K * nx * 8);
  h->W = (double*)a.take((size_t)K * nR * 8);
  h->sig = (double*)a.take((size_t)K * 8);
  h->v1 = (double*)a.take((size_t)nx * 8);
  h->v2 = (double*)a.take((size_t)nR * 8);
  h->kinx = a.take((size_t)nx * cw);
  h->kinR = a.take((size_t)nR * cw);
  h->twx = a.take((size_t)nx / 2 * cw);
  h->twR = a.take((size_t)nR / 2 * cw);
  h->twx_d = (double2*)a.take((size_t)nx / 2 * 16);
  h->twR_d = (double2*)a.take((size_t)nR / 2 * 16);
  h->psi = a.take((size_t)N * nx * cw);
  h->chi = a.take((size_t)N * nR * cw);
  h->x = (double*)a.take((size_t)N * 8);
  h->R = (double*)a.take((size_t)N * 8);
  h->xo = (double*)a.take((size_t)N * 8);
  h->Ro = (double*)a.take((size_t)N * 8);
  h->px = (double*)a.take((size_t)K * N * 8);
  h->pR = (double*)a.take((size_t)K * N * 8);
  h->dvec = (double*)a.take((size_t)N * 8);
  h->C = (double2*)a.take((size_t)N * 16);
  for (int q = 0; q < 4; ++q) h->kk[q] = (double2*)a.take((size_t)N * 16);
  h->y = (double2*)a.take((size_t)N * 16);
  h->work = (double2*)a.take((size_t)2 * N * 16);
  h->cf32 = (float*)a.take((size_t)N * 8);
  for (int q = 0; q < 2; ++q) {
    h->S[q] = (double2*)a.take(NN * 16);
    h->H[q] = (double2*)a.take(NN * 16);
    h->L[q] = (double2*)a.take(NN * 16);
  }
  h->Lh = (double2*)a.take(NN * 16);
  h->invL[0] = (double*)a.take((size_t)N * 8);
  h->invL[1] = (double*)a.take((size_t)N * 8);
  h->invLh = (double*)a.take((size_t)N * 8);
  h->DL[0] = (double2*)a.take((size_t)N * 512);
  h->DL[1] = (double2*)a.take((size_t)N * 512);
  h->DLh = (double2*)a.take((size_t)N * 512);
  h->flags = (unsigned*)a.take((size_t)2 * nblk * 4 + 64);
  h->tickets = h->flags + 2 * nblk;
  h->cctl = (unsigned*)a.take(chol_ctl_words(N) * sizeof(unsigned));
  h->status = (int*)a.take(64 * 4);
  if (h->mixed) h->tc_scratch = a.take(h->tc_scratch_bytes);
  if (!h->df_solve) h->emu_scratch = a.take(h->emu_bytes);
  if (!h->status || (h->mixed && !h->tc_scratch) || (!h->df_solve && !h->emu_scratch)) {
    cudaFree(h->arena.base);
    destroy_streams(h);
    return fail(nullptr, ICWF_ERR_OOM, "icwf_create: arena layout overflow");
  }

  // ---- tables ----
  std::vector<double> kx, twx, kR, twR;
  kinetic_tables(nx, h->dx, p.mass_x, p.dt, kx, twx);
  kinetic_tables(nR, h->dR, p.mass_R, p.dt, kR, twR);
  icwf_status st;
#define UP(dst, src, bytes) do { st = upload(h, dst, src, bytes); if (st) { g_err = h->err; cudaFree(h->arena.base); destroy_streams(h); return st; } } while (0)
  UP(h->V, Vh, nV * 8);
  std::vector<float> Vf, kxf, kRf, twxf, twRf;
  if (h->mixed) {
    Vf.assign(Vh, Vh + nV);
    kxf = cast_vec<float>(kx); kRf = cast_vec<float>(kR);
    twxf = cast_vec<float>(twx); twRf = cast_vec<float>(twR);
    UP(h->Vt, Vf.data(), nV * 4);
    UP(h->kinx, kxf.data(), kxf.size() * 4);
    UP(h->kinR, kRf.data(), kRf.size() * 4);
    UP(h->twx, twxf.data(), twxf.size() * 4);
    UP(h->twR, twRf.data(), twRf.size() * 4);
  } else {
    UP(h->Vt, Vh, nV * 8);
    UP(h->kinx, kx.data(), kx.size() * 8);
    UP(h->kinR, kR.data(), kR.size() * 8);
    UP(h->twx, twx.data(), twx.size() * 8);
    UP(h->twR, twR.data(), twR.size() * 8);
  }
  UP(h->twx_d, twx.data(), twx.size() * 8);
  UP(h->twR_d, twR.data(), twR.size() * 8);
  UP(h->U, Uk.data(), Uk.size() * 8);
  UP(h->W, Wk.data(), Wk.size() * 8);
  UP(h->sig, sk.data(), sk.size() * 8);
  UP(h->v1, v1.data(), v1.size() * 8);
  UP(h->v2, v2.data(), v2.size() * 8);
#undef UP
  h->prop_threads = tune_propagate(h);
  if (cudaMemsetAsync(h->flags, 0, (size_t)2 * nblk * 4 + 64, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->status, 0, 64 * 4, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaFree(h->arena.base);
    destroy_streams(h);
    return fail(nullptr, ICWF_ERR_CUDA, "icwf_create: initial device transfer failed");
  }
  *out = hp.release();
  return ICWF_OK;
}

icwf_status icwf_destroy(icwf_handle h) {
  if (!h) return ICWF_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_step_graphs(h);
  for (auto& pe : h->pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  for (void* p : h->extra_allocs) cudaFree(p);
  if (h->phi) cudaFree(h->phi);
  if (h->arena.base) cudaFree(h->arena.base);
  destroy_streams(h);
  delete h;
  return ICWF_OK;
}

icwf_status icwf_set_projectors(icwf_handle h, int32_t n_states, const double* phi) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_set_projectors: NULL handle");
  if (n_states < 0 || n_states > 8 || (n_states > 0 && !phi))
    return fail(h, ICWF_ERR_ARG, "icwf_set_projectors: n_states must be in [0, 8] with phi given");
  if (h->phi) { cudaFree(h->phi); h->phi = nullptr; }
  h->n_states = 0;
  if (n_states == 0) return ICWF_OK;
  const size_t bytes = (size_t)n_states * h->nR * h->nx * sizeof(double);
  CK(cudaMalloc(&h->phi, bytes));
  CK(cudaMemcpy(h->phi, phi, bytes, cudaMemcpyHostToDevice));
  h->n_states = n_states;
  return ICWF_OK;
}

static icwf_status init_common(icwf_handle h, const double* psi0, const std::vector<double>& xs,
                               const std::vector<double>& Rs) {
  const int N = h->N, nx = h->nx, nR = h->nR;
  for (int a = 0; a < N; ++a)
    if (!std::isfinite(xs[a]) || !std::isfinite(Rs[a]))
      return fail(h, ICWF_ERR_ARG, "init: non-finite position");
  // slices Psi0(., R_a) and Psi0(x_a, .) by cubic Lagrange interpolation, normalised
  std::vector<double> ps((size_t)2 * N * nx), cs((size_t)2 * N * nR);
  for (int a = 0; a < N; ++a) {
    const HStencil sR = h_lagrange4(Rs[a], h->p.R_min, h->dR, nR);
    double nrm = 0.0;
    for (int i = 0; i < nx; ++i) {
      double re = 0.0, im = 0.0;
      for (int q = 0; q < 4; ++q) {
        const size_t e = 2 * ((size_t)i * nR + sR.i0 + q);
        re += sR.w[q] * psi0[e];
        im += sR.w[q] * psi0[e + 1];
      }
      ps[2 * ((size_t)a * nx + i)] = re;
      ps[2 * ((size_t)a * nx + i) + 1] = im;
      nrm += re * re + im * im;
    }
    nrm = std::sqrt(h->dx * nrm);
    if (!(nrm > 0)) return fail(h, ICWF_ERR_ARG, "init: Psi0 vanishes along a trajectory's slice");
    for (int i = 0; i < 2 * nx; ++i) ps[(size_t)2 * a * nx + i] /= nrm;
    const HStencil sx = h_lagrange4(xs[a], h->p.x_min, h->dx, nx);
    nrm = 0.0;
    for (int jj = 0; jj < nR; ++jj) {
      double re = 0.0, im = 0.0;
      for (int q = 0; q < 4; ++q) {
        const size_t e = 2 * ((size_t)(sx.i0 + q) * nR + jj);
        re += sx.w[q] * psi0[e];
        im += sx.w[q] * psi0[e + 1];
      }
      cs[2 * ((size_t)a * nR + jj)] = re;
      cs[2 * ((size_t)a * nR + jj) + 1] = im;
      nrm += re * re + im * im;
    }
    nrm = std::sqrt(h->dR * nrm);
    if (!(nrm > 0)) return fail(h, ICWF_ERR_ARG, "init: Psi0 vanishes along a trajectory's slice");
    for (int jj = 0; jj < 2 * nR; ++jj) cs[(size_t)2 * a * nR + jj] /= nrm;
  }
  // FP64 scratch for the projection b_a = <phi_a|Psi0>
  void* tmp = nullptr;
  const size_t b_psi = (size_t)N * nx * 16, b_chi = (size_t)N * nR * 16, b_p0 = (size_t)nx * nR * 16;
  CK(cudaMalloc(&tmp, align256(b_psi) + align256(b_chi) + align256(b_p0) + 256));
  Arena a{(char*)tmp, align256(b_psi) + align256(b_chi) + align256(b_p0) + 256, 0};
  double2* dpsi = (double2*)a.take(b_psi);
  double2* dchi = (double2*)a.take(b_chi);
  double2* dp0 = (double2*)a.take(b_p0);
  icwf_status st = ICWF_OK;
  auto cleanup = [&]() { cudaStreamSynchronize(h->stream); cudaFree(tmp); };
#define CKI(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { cleanup(); return fail(h, ICWF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); } } while (0)
  CKI(cudaMemcpyAsync(dpsi, ps.data(), b_psi, cudaMemcpyHostToDevice, h->stream));
  CKI(cudaMemcpyAsync(dchi, cs.data(), b_chi, cudaMemcpyHostToDevice, h->stream));
  CKI(cudaMemcpyAsync(dp0, psi0, b_p0, cudaMemcpyHostToDevice, h->stream));
  CKI(cudaMemcpyAsync(h->x, xs.data(), N * 8, cudaMemcpyHostToDevice, h->stream));
  CKI(cudaMemcpyAsync(h->R, Rs.data(), N * 8, cudaMemcpyHostToDevice, h->stream));
  CKI(cudaMemcpyAsync(h->xo, xs.data(), N * 8, cudaMemcpyHostToDevice, h->stream));
  CKI(cudaMemcpyAsync(h->Ro, Rs.data(), N * 8, cudaMemcpyHostToDevice, h->stream));
  CKI(cudaMemsetAsync(h->status, 0, 64 * 4, h->stream));
  launch_init_projection(N, nx, nR, h->dx, h->dR, dpsi, dchi, dp0, h->y, h->stream);
  if (h->mixed) {
    launch_to_c64((size_t)N * nx, dpsi, (float2*)h->psi, h->stream);
    launch_to_c64((size_t)N * nR, dchi, (float2*)h->chi, h->stream);
  } else {
    CKI(cudaMemcpyAsync(h->psi, dpsi, b_psi, cudaMemcpyDeviceToDevice, h->stream));
    CKI(cudaMemcpyAsync(h->chi, dchi, b_chi, cudaMemcpyDeviceToDevice, h->stream));
  }
  JobView j = view(h);
  launch_velocity<double>(j, nullptr, h->stream);   // pinned factor values at x_0, R_0
  h->cur = 0;
  assemble(h, h->S[0], h->H[0]);
  {
    const double2* s0[1] = {h->S[0]};
    const double th[1] = {1.0};
    double2* d[1] = {h->L[0]};
    double* iv[1] = {h->invL[0]};
    double2* dd[1] = {h->DL[0]};
    factor(h, 1, s0, s0, th, d, iv, dd);
  }
  solve(h, h->L[0], h->DL[0], h->y, h->C, false);
  st = sync_status(h, "init");
  cleanup();
#undef CKI
  if (st != ICWF_OK) return st;
  h->initialised = true;
  h->steps = 0;
  h->t = 0.0;
  return ICWF_OK;
}

icwf_status icwf_init_from_positions(icwf_handle h, const double* psi0, const double* x,
                                     const double* R) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_init_from_positions: NULL handle");
  if (!psi0 || !x || !R) return fail(h, ICWF_ERR_ARG, "icwf_init_from_positions: NULL array");
  std::vector<double> xs(x, x + h->N), Rs(R, R + h->N);
  return init_common(h, psi0, xs, Rs);
}

icwf_status icwf_init_from_density(icwf_handle h, const double* psi0, uint64_t seed) {
  NvtxRange nvtx_("icwf_init_from_density");
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_init_from_density: NULL handle");
  if (!psi0) return fail(h, ICWF_ERR_ARG, "icwf_init_from_density: psi0 is NULL");
  const int nx = h->nx, nR = h->nR, N = h->N;
  const size_t n = (size_t)nx * nR;
  std::vector<double> cum(n);
  double c = 0.0;
  for (size_t e = 0; e < n; ++e) {
    const double re = psi0[2 * e], im = psi0[2 * e + 1];
    if (!std::isfinite(re) || !std::isfinite(im))
      return fail(h, ICWF_ERR_ARG, "icwf_init_from_density: psi0 has a non-finite entry");
    const double pr = re * re;
    const double pi = im * im;
    c = c + (pr + pi);
    cum[e] = c;
  }
  const double total = cum[n - 1];
  if (!(total > 0)) return fail(h, ICWF_ERR_ARG, "icwf_init_from_density: |psi0|^2 sums to zero");
  SplitMix64 rng(seed);
  std::vector<double> xs(N), Rs(N);
  for (int a = 0; a < N; ++a) {
    const double target = rng.uniform() * total;
    size_t idx = (size_t)(std::upper_bound(cum.begin(), cum.end(), target) - cum.begin());
    if (idx > n - 1) idx = n - 1;
    const int i = (int)(idx / nR), jj = (int)(idx % nR);
    const double xi = h->p.x_min + ((double)i + 0.5) * h->dx;
    const double Rj = h->p.R_min + ((double)jj + 0.5) * h->dR;
    xs[a] = xi + (rng.uniform() - 0.5) * h->dx;
    Rs[a] = Rj + (rng.uniform() - 0.5) * h->dR;
  }
  return init_common(h, psi0, xs, Rs);
}

icwf_status icwf_step(icwf_handle h, int32_t n_steps) {
  NvtxRange nvtx_("icwf_step");
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_step: NULL handle");
  if (!h->initialised) return fail(h, ICWF_ERR_STATE, "icwf_step: handle not initialised");
  if (n_steps < 0) return fail(h, ICWF_ERR_ARG, "icwf_step: n_steps < 0");
  if (n_steps > 0 && h->step_graphs && !h->prof_on && step_graphs_ready(h)) {
    // one graph launch per step (the per-family timing events need direct launches)
    for (int s = 0; s < n_steps; ++s) {
      CK(cudaGraphLaunch(h->step_exec[h->cur], h->stream));
      h->cur = 1 - h->cur;
      h->steps += 1;
      h->t += h->p.dt;
      h->launches += h->step_kernels;
    }
  } else {
    for (int s = 0; s < n_steps; ++s) step_once(h);
  }
  CK(cudaGetLastError());
  return sync_status(h, "icwf_step");
}

icwf_status icwf_observables(icwf_handle h, icwf_obs* out) {
  NvtxRange nvtx_("icwf_observables");
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_observables: NULL handle");
  if (!out) return fail(h, ICWF_ERR_ARG, "icwf_observables: out is NULL");
  if (!h->initialised) return fail(h, ICWF_ERR_STATE, "icwf_observables: handle not initialised");
  icwf_status st = alloc_obs(h);
  if (st) return st;
  JobView j = view(h);
  {
    ProfScope ps(h, F_OBS);
    if (h->mixed) launch_reconstruct<float>(j, h->C, h->Psi, h->stream);
    else launch_reconstruct<double>(j, h->C, h->Psi, h->stream);
    launch_obs_lines(j, h->Psi, h->phi, h->n_states, h->rho_x, h->rho_R, h->proj, h->part,
                     h->obs_out, h->pop, h->decoh, h->twx_d, h->twR_d, h->stream);
  }
  double o4[4];
  int cl[2];
  CK(cudaMemcpyAsync(o4, h->obs_out, sizeof(o4), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(cl, h->status, sizeof(cl), cudaMemcpyDeviceToHost, h->stream));
  if (out->rho_x) CK(cudaMemcpyAsync(out->rho_x, h->rho_x, h->nx * 8, cudaMemcpyDeviceToHost, h->stream));
  if (out->rho_R) CK(cudaMemcpyAsync(out->rho_R, h->rho_R, h->nR * 8, cudaMemcpyDeviceToHost, h->stream));
  if (out->pop && h->n_states)
    CK(cudaMemcpyAsync(out->pop, h->pop, h->n_states * 8, cudaMemcpyDeviceToHost, h->stream));
  if (out->decoh && h->n_states)
    CK(cudaMemcpyAsync(out->decoh, h->decoh, h->n_states * h->n_states * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->prof_on) prof_collect(h);
  out->t = h->t;
  out->norm = o4[0];
  out->energy = (o4[1] + o4[2] + o4[3]) / o4[0];
  out->n_states = h->n_states;
  out->n_clamped = cl[1];
  return ICWF_OK;
}

icwf_status icwf_get_state(icwf_handle h, double* C, double* x, double* R, double* psi,
                           double* chi) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_get_state: NULL handle");
  if (!h->initialised) return fail(h, ICWF_ERR_STATE, "icwf_get_state: handle not initialised");
  CK(cudaStreamSynchronize(h->stream));
  const int N = h->N;
  if (C) CK(cudaMemcpy(C, h->C, (size_t)N * 16, cudaMemcpyDeviceToHost));
  if (x) CK(cudaMemcpy(x, h->x, (size_t)N * 8, cudaMemcpyDeviceToHost));
  if (R) CK(cudaMemcpy(R, h->R, (size_t)N * 8, cudaMemcpyDeviceToHost));
  auto grab = [&](const void* src, size_t count, double* dst) -> icwf_status {
    if (!h->mixed) {
      CK(cudaMemcpy(dst, src, count * 16, cudaMemcpyDeviceToHost));
    } else {
      std::vector<float> f(2 * count);
      CK(cudaMemcpy(f.data(), src, count * 8, cudaMemcpyDeviceToHost));
      for (size_t e = 0; e < 2 * count; ++e) dst[e] = f[e];
    }
    return ICWF_OK;
  };
  if (psi) { icwf_status st = grab(h->psi, (size_t)N * h->nx, psi); if (st) return st; }
  if (chi) { icwf_status st = grab(h->chi, (size_t)N * h->nR, chi); if (st) return st; }
  return ICWF_OK;
}

icwf_status icwf_get_matrices(icwf_handle h, double* S, double* Hout, double* Heff) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_get_matrices: NULL handle");
  if (!h->initialised) return fail(h, ICWF_ERR_STATE, "icwf_get_matrices: handle not initialised");
  CK(cudaStreamSynchronize(h->stream));
  const int N = h->N, nx = h->nx, nR = h->nR;
  const size_t NN = (size_t)N * N;
  if (S) CK(cudaMemcpy(S, h->S[h->cur], NN * 16, cudaMemcpyDeviceToHost));
  if (Heff) CK(cudaMemcpy(Heff, h->H[h->cur], NN * 16, cudaMemcpyDeviceToHost));
  if (!Hout) return ICWF_OK;
  // H = T1 o S2 + S1 o T2 + W, W = sum_k s_k A_k o B_k + V1 o S2 + S1 o V2 (diagnostic path)
  void* tmp = nullptr;
  const size_t cw = h->cwf_elem;
  const size_t bytes = align256((size_t)N * nx * cw) + align256((size_t)N * nR * cw) + 9 * align256(NN * 16) + 256;
  CK(cudaMalloc(&tmp, bytes));
  Arena a{(char*)tmp, bytes, 0};
  void* tpsi = a.take((size_t)N * nx * cw);
  void* tchi = a.take((size_t)N * nR * cw);
  double2* G[9];
  for (int q = 0; q < 9; ++q) G[q] = (double2*)a.take(NN * 16);
  double2 *T1 = G[0], *T2 = G[1], *S1 = G[2], *S2 = G[3], *V1 = G[4], *V2 = G[5], *Wm = G[6],
          *Ak = G[7], *Bk = G[8];
  JobView j = view(h);
  cudaStream_t s = h->stream;
  if (h->mixed) {
    launch_kinetic<float>(j, tpsi, tchi, s);
    launch_gram<float>(h->psi, tpsi, nullptr, nx, N, h->dx, T1, s);
    launch_gram<float>(h->chi, tchi, nullptr, nR, N, h->dR, T2, s);
    launch_gram<float>(h->psi, h->psi, nullptr, nx, N, h->dx, S1, s);
    launch_gram<float>(h->chi, h->chi, nullptr, nR, N, h->dR, S2, s);
    launch_gram<float>(h->psi, h->psi, h->v1, nx, N, h->dx, V1, s);
    launch_gram<float>(h->chi, h->chi, h->v2, nR, N, h->dR, V2, s);
  } else {
    launch_kinetic<double>(j, tpsi, tchi, s);
    launch_gram<double>(h->psi, tpsi, nullptr, nx, N, h->dx, T1, s);
    launch_gram<double>(h->chi, tchi, nullptr, nR, N, h->dR, T2, s);
    launch_gram<double>(h->psi, h->psi, nullptr, nx, N, h->dx, S1, s);
    launch_gram<double>(h->chi, h->chi, nullptr, nR, N, h->dR, S2, s);
    launch_gram<double>(h->psi, h->psi, h->v1, nx, N, h->dx, V1, s);
    launch_gram<double>(h->chi, h->chi, h->v2, nR, N, h->dR, V2, s);
  }
  cudaMemsetAsync(Wm, 0, NN * 16, s);
  std::vector<double> sk(h->K);
  cudaMemcpy(sk.data(), h->sig, h->K * 8, cudaMemcpyDeviceToHost);
  for (int k = 0; k < h->K; ++k) {
    if (h->mixed) {
      launch_gram<float>(h->psi, h->psi, h->U + (size_t)k * nx, nx, N, h->dx, Ak, s);
      launch_gram<float>(h->chi, h->chi, h->W + (size_t)k * nR, nR, N, h->dR, Bk, s);
    } else {
      launch_gram<double>(h->psi, h->psi, h->U + (size_t)k * nx, nx, N, h->dx, Ak, s);
      launch_gram<double>(h->chi, h->chi, h->W + (size_t)k * nR, nR, N, h->dR, Bk, s);
    }
    launch_hadamard_acc(N, sk[k], Ak, Bk, Wm, s);
  }
  launch_combine_h(N, T1, T2, S1, S2, V1, V2, Wm, Ak, s);
  cudaError_t e = cudaMemcpyAsync(Hout, Ak, NN * 16, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(h, ICWF_ERR_CUDA, "icwf_get_matrices: copy failed");
  return ICWF_OK;
}

// ---- checkpoint / resume ----------------------------------------------------------------------

namespace {

struct StateHeader {
  char magic[8];          // "ICWFSTA1"
  int32_t version, N, nx, nR, K, precision, coeff_scheme, df_solve, cwf_elem, cur;
  int64_t steps;
  double t;
};

// Device regions that make up the time-stepping state at the current time (in this order).
std::vector<std::pair<void*, size_t>> state_regions(icwf_ctx* h) {
  const size_t N = h->N, NN = N * N, K = h->K, cw = h->cwf_elem;
  const int c = h->cur;
  return {{h->psi, N * h->nx * cw}, {h->chi, N * h->nR * cw},
          {h->x, N * 8}, {h->R, N * 8}, {h->xo, N * 8}, {h->Ro, N * 8},
          {h->px, K * N * 8}, {h->pR, K * N * 8}, {h->dvec, N * 8},
          {h->C, N * 16}, {h->S[c], NN * 16}, {h->H[c], NN * 16}, {h->L[c], NN * 16},
          {h->invL[c], N * 8}, {h->DL[c], N * 512}, {h->status + STATUS_CLAMPED, 4}};
}

size_t state_bytes(icwf_ctx* h) {
  size_t b = sizeof(StateHeader);
  for (auto& r : state_regions(h)) b += r.second;
  return b;
}

}  // namespace

icwf_status icwf_state_bytes(icwf_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(h, ICWF_ERR_ARG, "icwf_state_bytes: NULL argument");
  *bytes = state_bytes(h);
  return ICWF_OK;
}

icwf_status icwf_save_state(icwf_handle h, void* buf, size_t bytes) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_save_state: NULL handle");
  NvtxRange nvtx_("icwf_save_state");
  if (!h->initialised) return fail(h, ICWF_ERR_STATE, "icwf_save_state: handle not initialised");
  if (!buf || bytes < state_bytes(h))
    return fail(h, ICWF_ERR_ARG, "icwf_save_state: buffer smaller than icwf_state_bytes");
  StateHeader hd{};
  std::memcpy(hd.magic, "ICWFSTA1", 8);
  hd.version = 1; hd.N = h->N; hd.nx = h->nx; hd.nR = h->nR; hd.K = h->K;
  hd.precision = h->p.precision; hd.coeff_scheme = h->p.coeff_scheme; hd.df_solve = h->df_solve;
  hd.cwf_elem = (int)h->cwf_elem; hd.cur = h->cur; hd.steps = h->steps; hd.t = h->t;
  CK(cudaStreamSynchronize(h->stream));
  char* p = (char*)buf;
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  for (auto& r : state_regions(h)) {
    CK(cudaMemcpy(p, r.first, r.second, cudaMemcpyDeviceToHost));
    p += r.second;
  }
  return ICWF_OK;
}

icwf_status icwf_load_state(icwf_handle h, const void* buf, size_t bytes) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_load_state: NULL handle");
  NvtxRange nvtx_("icwf_load_state");
  if (!buf || bytes < sizeof(StateHeader)) return fail(h, ICWF_ERR_ARG, "icwf_load_state: buffer too small");
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, "ICWFSTA1", 8) != 0 || hd.version != 1)
    return fail(h, ICWF_ERR_ARG, "icwf_load_state: not a saved ICWF state");
  if (hd.N != h->N || hd.nx != h->nx || hd.nR != h->nR || hd.K != h->K ||
      hd.precision != h->p.precision || hd.coeff_scheme != h->p.coeff_scheme ||
      hd.df_solve != (int)h->df_solve || hd.cwf_elem != (int)h->cwf_elem)
    return fail(h, ICWF_ERR_ARG, "icwf_load_state: state saved from a handle with other parameters");
  CK(cudaStreamSynchronize(h->stream));
  h->cur = hd.cur;
  if (bytes < state_bytes(h)) return fail(h, ICWF_ERR_ARG, "icwf_load_state: buffer too small");
  const char* p = (const char*)buf + sizeof(hd);
  for (auto& r : state_regions(h)) {
    CK(cudaMemcpy(r.first, p, r.second, cudaMemcpyHostToDevice));
    p += r.second;
  }
  const int flags0 = 0;
  CK(cudaMemcpy(h->status + STATUS_FLAGS, &flags0, sizeof(int), cudaMemcpyHostToDevice));
  h->steps = hd.steps;
  h->t = hd.t;
  h->initialised = true;
  return ICWF_OK;
}

icwf_status icwf_get_info(icwf_handle h, icwf_info* out) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_get_info: NULL handle");
  if (!out) return fail(h, ICWF_ERR_ARG, "icwf_get_info: out is NULL");
  out->rank = h->K;
  out->tail_rel = h->tail_rel;
  out->next_rel = h->next_rel;
  out->sigma_max = h->sigma_max;
  out->device_bytes = h->arena.size;
  out->steps_done = h->steps;
  out->t = h->t;
  out->kernel_launches = h->launches;
  out->obs_bytes = h->obs_bytes;
  out->prop_threads = h->prop_threads;
  return ICWF_OK;
}

icwf_status icwf_set_regularisation(icwf_handle h, double eps) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_set_regularisation: NULL handle");
  if (!std::isfinite(eps)) return fail(h, ICWF_ERR_ARG, "icwf_set_regularisation: eps is not finite");
  h->p.s_reg_eps = eps;
  h->version += 1;   // a pool re-captures this job's step graphs
  return ICWF_OK;
}

icwf_status icwf_set_emulated_update(icwf_handle h, int32_t on) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_set_emulated_update: NULL handle");
  h->emu_update = on != 0;
  h->version += 1;   // the step graphs hold the previous update kernels: re-capture them
  return ICWF_OK;
}

icwf_status icwf_set_step_graphs(icwf_handle h, int32_t on) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_set_step_graphs: NULL handle");
  h->step_graphs = on != 0;
  if (!h->step_graphs) drop_step_graphs(h);
  return ICWF_OK;
}

icwf_status icwf_set_wait_limit(icwf_handle h, int64_t polls) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_set_wait_limit: NULL handle");
  if (polls > (int64_t)INT32_MAX - 1) return fail(h, ICWF_ERR_ARG, "icwf_set_wait_limit: polls too large");
  const int v = polls < 0 ? 0 : (int)polls + 1;
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(h->status + STATUS_WAITLIM, &v, sizeof(int), cudaMemcpyHostToDevice));
  return ICWF_OK;
}

icwf_status icwf_get_stream(icwf_handle h, void** stream) {
  if (!h || !stream) return fail(h, ICWF_ERR_ARG, "icwf_get_stream: NULL argument");
  *stream = (void*)h->stream;
  return ICWF_OK;
}

icwf_status icwf_profile_enable(icwf_handle h, int32_t on) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_profile_enable: NULL handle");
  h->prof_on = on != 0;
  return ICWF_OK;
}

icwf_status icwf_profile_reset(icwf_handle h) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_profile_reset: NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  prof_collect(h);
  for (int f = 0; f < F_COUNT; ++f) { h->prof_ms[f] = 0; h->prof_n[f] = 0; }
  return ICWF_OK;
}

icwf_status icwf_profile_read(icwf_handle h, int32_t n, const char** names, double* ms,
                              int64_t* launches, int32_t* n_out) {
  if (!h) return fail(nullptr, ICWF_ERR_ARG, "icwf_profile_read: NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  prof_collect(h);
  for (int f = 0; f < F_COUNT && f < n; ++f) {
    if (names) names[f] = kFamNames[f];
    if (ms) ms[f] = h->prof_ms[f];
    if (launches) launches[f] = h->prof_n[f];
  }
  if (n_out) *n_out = F_COUNT;
  return ICWF_OK;
}

}  // extern "C"

// ============================================================================================
// Serving pool
// ============================================================================================

struct PoolJob {
  icwf_handle h = nullptr;
  int64_t target = 0;
  int state = 0;   // 0 pending, 1 live, 2 finished, 3 failed
  double norm = 0, energy = 0, t = 0;
  std::vector<double> rho_x, rho_R, pop, decoh;
  int n_clamped = 0, n_states = 0;
  // one captured step per ping-pong parity of the job's matrix buffers
  cudaGraph_t g[2] = {nullptr, nullptr};
  bool graphs_tried = false, graphs_ok = false;
  bool grouped = false;   // graphs recorded without velocities and propagation (grouped kernels)
  int64_t kernels_per_step = 0;
  int64_t version = -1;   // handle version the graphs were captured at
};

struct icwf_pool_ctx {
  size_t budget = 0;
  int max_jobs = 0;
  size_t live_bytes = 0;
  std::vector<PoolJob> jobs;
  std::deque<int> pending;
  std::vector<int> live;
  bool use_graphs = true;
  bool use_groups = true;   // grouped velocity and propagation kernels inside the tick graphs
  int group_ctas = 0;       // CTA cap of each grouped kernel (0: one wave at full occupancy)
  cudaStream_t stream = nullptr;
  // instantiated tick graphs of the current live set, keyed by (job id, parity) of every job; each
  // with the device table of its grouped kernels (NULL without grouping)
  struct TickExec {
    cudaGraphExec_t exec = nullptr;
    void* table = nullptr;
    int64_t group_nodes = 0;
  };
  std::map<std::vector<int64_t>, TickExec> ticks_cache;
  std::vector<int> cache_live;   // the live set the cache belongs to
  icwf_pool_stats stats{};
};

namespace {

// Called between ticks only (every tick ends with a synchronisation of the pool's stream), so no
// cached graph or table is in use on the device.
void clear_tick_cache(icwf_pool pool) {
  for (auto& kv : pool->ticks_cache) {
    cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.table) cudaFree(kv.second.table);
  }
  pool->ticks_cache.clear();
}

void destroy_job_graphs(PoolJob& j) {
  for (auto& g : j.g)
    if (g) { cudaGraphDestroy(g); g = nullptr; }
  j.graphs_ok = false;
}

// Capture one step of the job for each parity of its ping-pong buffers (two consecutive steps
// recorded, not executed), then restore the host-side step state; with `grouped` the recorded
// step leaves out the velocities and the propagation, which the tick's grouped kernels run.
// Returns false (and leaves the job to eager stepping) if the capture fails.
bool capture_job_graphs(PoolJob& pj, bool grouped) {
  pj.h->traj_grouped = grouped;
  const bool ok = capture_step(pj.h, pj.g, &pj.kernels_per_step);
  pj.h->traj_grouped = false;
  pj.graphs_ok = ok;
  pj.grouped = grouped;
  pj.version = pj.h->version;
  return ok;
}

// Instantiate the tick graph of the jobs `run` at their current parities: with `grouped`, one
// persistent velocity kernel and one persistent propagation kernel per CWF precision over all of
// those jobs (their entries in one device table), on which every job's recorded step (a child
// graph) depends; else the child graphs alone.  False (nothing kept) on any failure.
bool build_tick(icwf_pool pool, const std::vector<int>& run, bool grouped,
                icwf_pool_ctx::TickExec* out) {
  std::vector<GroupJob> tab[2];   // [0]: FP64 CWFs, [1]: complex64 CWFs
  int traj[2] = {0, 0}, cwfs[2] = {0, 0}, nmax[2] = {0, 0}, thr[2] = {256, 256};
  double work[2] = {0, 0};
  if (grouped) {
    for (int id : run) {
      icwf_ctx* h = pool->jobs[id].h;
      const int t = h->mixed ? 1 : 0;
      GroupJob q = group_job(view(h), h->C);
      q.traj0 = traj[t];
      q.cwf0 = cwfs[t];
      tab[t].push_back(q);
      traj[t] += h->N;
      cwfs[t] += 2 * h->N;
      nmax[t] = std::max(nmax[t], std::max(h->nx, h->nR));
      // CTA size: the autotuned one of the job with the most propagation work
      const double wj = (double)h->N * (double)(h->nx + h->nR);
      if (wj > work[t]) { work[t] = wj; thr[t] = h->prop_threads; }
    }
  }
  const size_t n0 = tab[0].size(), n1 = tab[1].size();
  void* table = nullptr;
  if (n0 + n1 > 0) {
    if (cudaMalloc(&table, (n0 + n1) * sizeof(GroupJob)) != cudaSuccess) { cudaGetLastError(); return false; }
    bool ok = n0 == 0 || cudaMemcpy(table, tab[0].data(), n0 * sizeof(GroupJob),
                                    cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && (n1 == 0 || cudaMemcpy((GroupJob*)table + n0, tab[1].data(), n1 * sizeof(GroupJob),
                                      cudaMemcpyHostToDevice) == cudaSuccess);
    if (!ok) { cudaFree(table); cudaGetLastError(); return false; }
  }
  cudaGraph_t tg = nullptr;
  bool ok = cudaGraphCreate(&tg, 0) == cudaSuccess;
  cudaGraphNode_t deps[2];
  size_t nd = 0;
  int64_t gnodes = 0;
  if (ok && n0 > 0) {
    ok = add_group_nodes<double>(tg, nullptr, 0, (const GroupJob*)table, (int)n0, traj[0], cwfs[0],
                                 nmax[0], thr[0], pool->group_ctas, &deps[nd++]);
    gnodes += 2;
  }
  if (ok && n1 > 0) {
    ok = add_group_nodes<float>(tg, nullptr, 0, (const GroupJob*)table + n0, (int)n1, traj[1],
                                cwfs[1], nmax[1], thr[1], pool->group_ctas, &deps[nd++]);
    gnodes += 2;
  }
  for (size_t k = 0; ok && k < run.size(); ++k) {
    PoolJob& j = pool->jobs[run[k]];
    cudaGraphNode_t node;
    ok = cudaGraphAddChildGraphNode(&node, tg, nd ? deps : nullptr, nd, j.g[j.h->cur]) == cudaSuccess;
  }
  cudaGraphExec_t exec = nullptr;
  ok = ok && cudaGraphInstantiate(&exec, tg, 0) == cudaSuccess;
  if (tg) cudaGraphDestroy(tg);
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    if (table) cudaFree(table);
    cudaGetLastError();
    return false;
  }
  out->exec = exec;
  out->table = table;
  out->group_nodes = gnodes;
  return true;
}

}  // namespace

extern "C" {

icwf_status icwf_pool_create(size_t hbm_budget_bytes, int32_t max_jobs, icwf_pool* out) {
  if (!out || max_jobs < 1 || hbm_budget_bytes == 0)
    return fail(nullptr, ICWF_ERR_ARG, "icwf_pool_create: invalid argument");
  std::unique_ptr<icwf_pool_ctx> p(new icwf_pool_ctx);
  p->budget = hbm_budget_bytes;
  p->max_jobs = max_jobs;
  if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(nullptr, ICWF_ERR_CUDA, "icwf_pool_create: cudaStreamCreate failed");
  *out = p.release();
  return ICWF_OK;
}

icwf_status icwf_pool_set_graphs(icwf_pool pool, int32_t on) {
  if (!pool) return fail(nullptr, ICWF_ERR_ARG, "icwf_pool_set_graphs: NULL pool");
  pool->use_graphs = on != 0;
  return ICWF_OK;
}

icwf_status icwf_pool_set_grouping(icwf_pool pool, int32_t on, int32_t max_ctas) {
  if (!pool || max_ctas < 0)
    return fail(nullptr, ICWF_ERR_ARG, "icwf_pool_set_grouping: invalid argument");
  if ((on != 0) != pool->use_groups || max_ctas != pool->group_ctas) clear_tick_cache(pool);
  pool->use_groups = on != 0;
  pool->group_ctas = max_ctas;
  return ICWF_OK;
}

icwf_status icwf_pool_get_stats(icwf_pool pool, icwf_pool_stats* out) {
  if (!pool || !out) return fail(nullptr, ICWF_ERR_ARG, "icwf_pool_get_stats: NULL argument");
  *out = pool->stats;
  return ICWF_OK;
}

icwf_status icwf_pool_submit(icwf_pool pool, icwf_handle job, int64_t n_steps, int32_t* job_id) {
  if (!pool || !job || n_steps < 0) return fail(nullptr, ICWF_ERR_ARG, "icwf_pool_submit: invalid argument");
  if (!job->initialised) return fail(nullptr, ICWF_ERR_STATE, "icwf_pool_submit: job not initialised");
  if (job->arena.size > pool->budget)
    return fail(nullptr, ICWF_ERR_OOM, "icwf_pool_submit: job footprint exceeds the pool budget");
  PoolJob pj;
  pj.h = job;
  pj.target = job->steps + n_steps;
  pool->jobs.push_back(std::move(pj));
  const int id = (int)pool->jobs.size() - 1;
  pool->pending.push_back(id);
  if (job_id) *job_id = id;
  return ICWF_OK;
}

static void finish_job(icwf_pool pool, int id, bool ok) {
  PoolJob& j = pool->jobs[id];
  icwf_handle h = j.h;
  if (ok) {
    j.rho_x.assign(h->nx, 0.0);
    j.rho_R.assign(h->nR, 0.0);
    j.pop.assign(8, 0.0);
    j.decoh.assign(64, 0.0);
    icwf_obs o{};
    o.rho_x = j.rho_x.data(); o.rho_R = j.rho_R.data(); o.pop = j.pop.data(); o.decoh = j.decoh.data();
    if (icwf_observables(h, &o) == ICWF_OK) {
      j.norm = o.norm; j.energy = o.energy; j.t = o.t; j.n_clamped = o.n_clamped;
      j.n_states = o.n_states;
      j.state = 2;
    } else {
      j.state = 3;
    }
  } else {
    j.state = 3;
  }
  destroy_job_graphs(j);
  pool->live_bytes -= h->arena.size;
  icwf_destroy(h);
  j.h = nullptr;
}

// One tick: admit pending jobs (arrival order, slots and device-memory budget), then advance
// every live job by one step.  With graphs on, each job's step is a captured graph (recorded at
// its first tick, one per buffer parity) and all of them run as child graphs of one tick graph,
// instantiated once per live set and parity pattern and launched with a single cudaGraphLaunch;
// the jobs share nothing, so their kernels overlap freely.  Without graphs (or if a capture
// fails) every job's kernels are launched directly on its own streams.
icwf_status icwf_pool_tick(icwf_pool pool, int32_t* n_live, int32_t* n_finished) {
  NvtxRange nvtx_("icwf_pool_tick");
  if (!pool) return fail(nullptr, ICWF_ERR_ARG, "icwf_pool_tick: NULL pool");
  while (!pool->pending.empty() && (int)pool->live.size() < pool->max_jobs) {
    const int id = pool->pending.front();
    const size_t b = pool->jobs[id].h->arena.size;
    if (pool->live_bytes + b > pool->budget) break;
    pool->pending.pop_front();
    pool->live.push_back(id);
    pool->live_bytes += b;
    pool->jobs[id].state = 1;
  }
  if (pool->live != pool->cache_live) {
    clear_tick_cache(pool);
    pool->cache_live = pool->live;
  }
  std::vector<int> run;
  for (int id : pool->live)
    if (pool->jobs[id].h->steps < pool->jobs[id].target) run.push_back(id);
  bool graphs = pool->use_graphs && !run.empty();
  if (graphs) {
    for (int id : run) {
      PoolJob& j = pool->jobs[id];
      if (j.graphs_tried && (j.version != j.h->version || j.grouped != pool->use_groups)) {
        // captured kernel arguments are stale, or the grouping changed: record the step again
        destroy_job_graphs(j);
        clear_tick_cache(pool);
        j.graphs_tried = false;
      }
      if (!j.graphs_tried) {
        j.graphs_tried = true;
        capture_job_graphs(j, pool->use_groups);
      }
      graphs = graphs && j.graphs_ok;
    }
  }
  bool launched = false;
  if (graphs) {
    std::vector<int64_t> key;
    for (int id : run) key.push_back(2 * (int64_t)id + pool->jobs[id].h->cur);
    icwf_pool_ctx::TickExec te;
    auto it = pool->ticks_cache.find(key);
    if (it != pool->ticks_cache.end()) {
      te = it->second;
    } else if (build_tick(pool, run, pool->use_groups, &te)) {
      pool->ticks_cache[key] = te;
      pool->stats.graph_builds += 1;
    }
    if (te.exec && cudaGraphLaunch(te.exec, pool->stream) == cudaSuccess) {
      launched = true;
      pool->stats.graph_launches += 1;
      pool->stats.group_nodes += te.group_nodes;
      pool->stats.kernel_nodes += te.group_nodes;
      for (int id : run) {
        PoolJob& j = pool->jobs[id];
        icwf_ctx* h = j.h;
        h->cur = 1 - h->cur;
        h->steps += 1;
        h->t += h->p.dt;
        h->launches += j.kernels_per_step;
        pool->stats.kernel_nodes += j.kernels_per_step;
      }
      pool->stats.graph_job_steps += (int64_t)run.size();
    }
  }
  if (!launched) {
    for (int id : run) step_once(pool->jobs[id].h);
    pool->stats.eager_job_steps += (int64_t)run.size();
  }
  pool->stats.ticks += 1;
  if (launched) CK_POOL(cudaStreamSynchronize(pool->stream));
  int fin = 0;
  std::vector<int> still;
  for (int id : pool->live) {
    PoolJob& j = pool->jobs[id];
    const icwf_status st = sync_status(j.h, "icwf_pool_tick");
    if (st != ICWF_OK) { finish_job(pool, id, false); ++fin; continue; }
    if (j.h->steps >= j.target) { finish_job(pool, id, true); ++fin; continue; }
    still.push_back(id);
  }
  pool->live.swap(still);
  if (n_live) *n_live = (int)pool->live.size();
  if (n_finished) *n_finished = fin;
  return ICWF_OK;
}

icwf_status icwf_pool_poll(icwf_pool pool, int32_t job_id, icwf_obs* out, int32_t* state) {
  if (!pool || job_id < 0 || job_id >= (int)pool->jobs.size())
    return fail(nullptr, ICWF_ERR_ARG, "icwf_pool_poll: invalid job id");
  PoolJob& j = pool->jobs[job_id];
  if (state) *state = j.state;
  if (j.state == 2 && out) {
    out->t = j.t; out->norm = j.norm; out->energy = j.energy; out->n_clamped = j.n_clamped;
    out->n_states = j.n_states;
    if (out->rho_x) std::copy(j.rho_x.begin(), j.rho_x.end(), out->rho_x);
    if (out->rho_R) std::copy(j.rho_R.begin(), j.rho_R.end(), out->rho_R);
    if (out->pop) std::copy(j.pop.begin(), j.pop.begin() + j.n_states, out->pop);
    if (out->decoh) std::copy(j.decoh.begin(), j.decoh.begin() + j.n_states * j.n_states, out->decoh);
  }
  return ICWF_OK;
}

icwf_status icwf_pool_destroy(icwf_pool pool) {
  if (!pool) return ICWF_OK;
  if (pool->stream) cudaStreamSynchronize(pool->stream);
  clear_tick_cache(pool);
  for (auto& j : pool->jobs) {
    destroy_job_graphs(j);
    if (j.h) icwf_destroy(j.h);
  }
  if (pool->stream) cudaStreamDestroy(pool->stream);
  delete pool;
  return ICWF_OK;
}

}  // extern "C"
