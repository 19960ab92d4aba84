// Exact propagation of the two-coordinate wavefunction Psi(x, R) (Eq. TDSE without vector
// potential) by the second-order Strang split on the periodic cell-centred grid:
//   Psi <- e^{-i V dt/2} F^-1 e^{-i (kx^2/2m_x + kR^2/2m_R) dt} F e^{-i V dt/2} Psi.
// This is the reference the paper's figures compare the ICWF densities, populations and
// decoherence indicators with.  FP64; Psi row-major nx x nR (x slow).
//
// One step is three kernels:
//   k_rows (forward): per x row, multiply by e^{-i V dt/2}, radix-2 FFT along R (bit-reversed out);
//   k_cols: per group of CB adjacent R columns (coalesced CB-wide loads), FFT along x, multiply by
//           the kinetic phase of (kx, kR) (both tables bit-reversed, 1/n folded in), inverse FFT
//           along x;
//   k_rows (inverse): per x row, inverse FFT along R (natural order out), multiply by the half
//           potential phase.
// Observables use per-row / per-CTA partial sums finished on the host in a fixed order.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/icwf_exact2d.h"
#include "icwf_internal.h"
#include "k_common.cuh"

namespace icwf {
namespace e2d {

constexpr int TPB = 256;
constexpr int MAX_STATES = 8;

// nb transforms of length n = 2^logn stored back to back in shared memory; all threads take part.
__device__ __forceinline__ void fft_dif_b(double2* buf, const double2* __restrict__ tw, int n,
                                          int logn, int nb) {
  const int half = n >> 1;
  for (int s = logn - 1; s >= 0; --s) {
    const int h = 1 << s, tstride = n >> (s + 1);
    for (int idx = threadIdx.x; idx < nb * half; idx += blockDim.x) {
      const int b = idx >> (logn - 1), id = idx & (half - 1);
      const int j = id & (h - 1);
      const int i1 = b * n + ((id >> s) << (s + 1)) + j, i2 = i1 + h;
      const double2 u = buf[i1], v = buf[i2];
      buf[i1] = cadd(u, v);
      buf[i2] = cmul(csub(u, v), tw[j * tstride]);
    }
    __syncthreads();
  }
}
__device__ __forceinline__ void ifft_dit_b(double2* buf, const double2* __restrict__ tw, int n,
                                           int logn, int nb) {
  const int half = n >> 1;
  for (int s = 0; s < logn; ++s) {
    const int h = 1 << s, tstride = n >> (s + 1);
    for (int idx = threadIdx.x; idx < nb * half; idx += blockDim.x) {
      const int b = idx >> (logn - 1), id = idx & (half - 1);
      const int j = id & (h - 1);
      const int i1 = b * n + ((id >> s) << (s + 1)) + j, i2 = i1 + h;
      const double2 u = buf[i1];
      const double2 t = cmul(buf[i2], cconj(tw[j * tstride]));
      buf[i1] = cadd(u, t);
      buf[i2] = csub(u, t);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;   // valid in thread 0
}

// One x row per CTA.  inverse = 0: out = FFT_R(half * in) (half may be null); inverse = 1:
// out = half * IFFT_R(in).  in and out may alias.
__global__ void __launch_bounds__(TPB) k_rows(const double2* in, double2* out,
                                              const double2* __restrict__ half,
                                              const double2* __restrict__ tw, int nR, int logR,
                                              int inverse) {
  extern __shared__ __align__(16) double2 buf[];
  const size_t base = (size_t)blockIdx.x * nR;
  for (int j = threadIdx.x; j < nR; j += blockDim.x) {
    double2 z = in[base + j];
    if (!inverse && half) z = cmul(half[base + j], z);
    buf[j] = z;
  }
  __syncthreads();
  if (inverse) ifft_dit_b(buf, tw, nR, logR, 1);
  else fft_dif_b(buf, tw, nR, logR, 1);
  for (int j = threadIdx.x; j < nR; j += blockDim.x) {
    double2 z = buf[j];
    if (inverse && half) z = cmul(half[base + j], z);
    out[base + j] = z;
  }
}

// CB adjacent R columns per CTA (bit-reversed R frequencies after k_rows).  mode 0: FFT along x,
// multiply by kinx[m] kinR[col], inverse FFT along x, store.  mode 1: FFT along x and
// part[blockIdx.x] = sum |F|^2 (Tx[m] + TR[col]) (kinetic energy, not stored).
__global__ void __launch_bounds__(TPB) k_cols(double2* a, const double2* __restrict__ kinx,
                                              const double2* __restrict__ kinR,
                                              const double2* __restrict__ tw, int nx, int logx,
                                              int nR, int CB, int mode,
                                              const double* __restrict__ Tx,
                                              const double* __restrict__ TR, double* part) {
  extern __shared__ __align__(16) double2 buf[];   // [CB][nx]
  __shared__ double red[TPB / 32];
  const int j0 = blockIdx.x * CB;
  for (int e = threadIdx.x; e < nx * CB; e += blockDim.x) {
    const int i = e / CB, c = e - i * CB;
    buf[c * nx + i] = a[(size_t)i * nR + j0 + c];
  }
  __syncthreads();
  fft_dif_b(buf, tw, nx, logx, CB);
  if (mode == 0) {
    for (int e = threadIdx.x; e < nx * CB; e += blockDim.x) {
      const int c = e / nx, m = e - c * nx;
      buf[e] = cmul(buf[e], cmul(kinx[m], kinR[j0 + c]));
    }
    __syncthreads();
    ifft_dit_b(buf, tw, nx, logx, CB);
    for (int e = threadIdx.x; e < nx * CB; e += blockDim.x) {
      const int i = e / CB, c = e - i * CB;
      a[(size_t)i * nR + j0 + c] = buf[c * nx + i];
    }
  } else {
    double s = 0.0;
    for (int e = threadIdx.x; e < nx * CB; e += blockDim.x) {
      const int c = e / nx, m = e - c * nx;
      const double2 z = buf[e];
      s += (z.x * z.x + z.y * z.y) * (Tx[m] + TR[j0 + c]);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// Per x row: dens[i] = sum_j |Psi|^2, pot[i] = sum_j |Psi|^2 V.
__global__ void __launch_bounds__(TPB) k_dens_rows(const double2* __restrict__ psi,
                                                   const double* __restrict__ V, int nR,
                                                   double* dens, double* pot) {
  __shared__ double red[TPB / 32];
  const size_t base = (size_t)blockIdx.x * nR;
  double s = 0.0, p = 0.0;
  for (int j = threadIdx.x; j < nR; j += blockDim.x) {
    const double2 z = psi[base + j];
    const double d = z.x * z.x + z.y * z.y;
    s += d;
    p += d * V[base + j];
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) dens[blockIdx.x] = s;
  p = block_sum(p, red);
  if (threadIdx.x == 0) pot[blockIdx.x] = p;
}

// Per R column j: dens[j] = sum_i |Psi|^2 and, for n < ns, proj[n][j] = sum_i phi[n][j][i] Psi[i][j].
__global__ void __launch_bounds__(TPB) k_cols_obs(const double2* __restrict__ psi, int nx, int nR,
                                                  const double* __restrict__ phi, int ns,
                                                  double* dens, double2* proj) {
  __shared__ double red[TPB / 32];
  const int j = blockIdx.x;
  double s = 0.0;
  double pr[MAX_STATES], pi[MAX_STATES];
#pragma unroll
  for (int n = 0; n < MAX_STATES; ++n) pr[n] = pi[n] = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double2 z = psi[(size_t)i * nR + j];
    s += z.x * z.x + z.y * z.y;
#pragma unroll
    for (int n = 0; n < MAX_STATES; ++n) {
      if (n < ns) {
        const double f = phi[((size_t)n * nR + j) * nx + i];
        pr[n] += f * z.x;
        pi[n] += f * z.y;
      }
    }
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) dens[j] = s;
#pragma unroll
  for (int n = 0; n < MAX_STATES; ++n) {
    if (n < ns) {   // uniform over the block
      const double a = block_sum(pr[n], red);
      const double b = block_sum(pi[n], red);
      if (threadIdx.x == 0) proj[(size_t)n * nR + j] = make_double2(a, b);
    }
  }
}

int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// kin[mp] = e^{-i k^2 dt / 2m} / n and T[mp] = k^2 / 2m at bit-reversed position mp; tw = e^{-2 pi i k / n}.
void tables(int n, double d, double mass, double dt, std::vector<double2>& kin,
            std::vector<double>& T, std::vector<double2>& tw) {
  const int logn = ilog2i(n);
  const double PI = 3.14159265358979323846;
  kin.resize(n);
  T.resize(n);
  tw.resize(n / 2);
  for (int mp = 0; mp < n; ++mp) {
    int m = 0;
    for (int b = 0; b < logn; ++b)
      if (mp & (1 << b)) m |= 1 << (logn - 1 - b);
    const int mm = m < n / 2 ? m : m - n;
    const double k = 2.0 * PI * (double)mm / ((double)n * d);
    const double e = k * k / (2.0 * mass);
    T[mp] = e;
    kin[mp] = make_double2(std::cos(-e * dt) / n, std::sin(-e * dt) / n);
  }
  for (int k = 0; k < n / 2; ++k) {
    const double a = -2.0 * PI * (double)k / (double)n;
    tw[k] = make_double2(std::cos(a), std::sin(a));
  }
}

}  // namespace e2d
}  // namespace icwf

using namespace icwf;

struct icwf_exact2d_ctx {
  int nx = 0, nR = 0, logx = 0, logR = 0, CB = 1, ns = 0;
  double dx = 0, dR = 0, dt = 0, t = 0;
  bool has_state = false;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  double* V = nullptr;
  double2 *half = nullptr, *psi = nullptr, *work = nullptr;
  double2 *kinx = nullptr, *kinR = nullptr, *twx = nullptr, *twR = nullptr;
  double *Tx = nullptr, *TR = nullptr, *phi = nullptr;
  double *dens_x = nullptr, *pot = nullptr, *dens_R = nullptr, *part = nullptr;
  double2* proj = nullptr;
  std::string err;
};

namespace {

std::string g_err2;

icwf_status fail2(icwf_exact2d h, icwf_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_err2 = msg;
  return st;
}

template <typename T>
bool dalloc(icwf_exact2d h, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return false;
  h->allocs.push_back(q);
  *p = (T*)q;
  return true;
}

void release(icwf_exact2d h) {
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->stream) cudaStreamDestroy(h->stream);
  h->stream = nullptr;
}

icwf_status sync(icwf_exact2d h, const char* what) {
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail2(h, ICWF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  const cudaError_t l = cudaGetLastError();
  if (l != cudaSuccess) return fail2(h, ICWF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(l));
  return ICWF_OK;
}

bool pow2_in(int n) { return n >= 8 && n <= 4096 && (n & (n - 1)) == 0; }

// copies ordered with the handle's (non-blocking) stream, complete on return
bool copy(icwf_exact2d h, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  return cudaMemcpyAsync(dst, src, bytes, kind, h->stream) == cudaSuccess &&
         cudaStreamSynchronize(h->stream) == cudaSuccess;
}

}  // namespace

extern "C" {

icwf_status icwf_exact2d_create(const icwf_params* p, const double* V, icwf_exact2d* out) {
  if (!p || !V || !out) return fail2(nullptr, ICWF_ERR_ARG, "icwf_exact2d_create: null pointer");
  *out = nullptr;
  if (!pow2_in(p->nx) || !pow2_in(p->nR))
    return fail2(nullptr, ICWF_ERR_ARG, "icwf_exact2d_create: nx, nR must be powers of two in [8, 4096]");
  if (!(p->x_max > p->x_min) || !(p->R_max > p->R_min) || !(p->mass_x > 0) || !(p->mass_R > 0) ||
      !(p->dt > 0))
    return fail2(nullptr, ICWF_ERR_ARG, "icwf_exact2d_create: bad extents, masses or dt");
  icwf_exact2d h = new icwf_exact2d_ctx;
  h->nx = p->nx;
  h->nR = p->nR;
  h->logx = e2d::ilog2i(p->nx);
  h->logR = e2d::ilog2i(p->nR);
  h->dx = (p->x_max - p->x_min) / p->nx;
  h->dR = (p->R_max - p->R_min) / p->nR;
  h->dt = p->dt;
  // columns per CTA: as many as fit 96 KB of shared memory, at most 8 (a power of two <= nR)
  h->CB = 8;
  while (h->CB > 1 && (size_t)h->CB * h->nx * sizeof(double2) > 96 * 1024) h->CB >>= 1;
  const size_t NN = (size_t)h->nx * h->nR;
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return fail2(nullptr, ICWF_ERR_CUDA, "icwf_exact2d_create: cudaStreamCreate failed");
  }
  const int ncb = h->nR / h->CB;
  if (!dalloc(h, &h->V, NN) || !dalloc(h, &h->half, NN) || !dalloc(h, &h->psi, NN) ||
      !dalloc(h, &h->work, NN) || !dalloc(h, &h->kinx, h->nx) || !dalloc(h, &h->kinR, h->nR) ||
      !dalloc(h, &h->twx, h->nx / 2) || !dalloc(h, &h->twR, h->nR / 2) ||
      !dalloc(h, &h->Tx, h->nx) || !dalloc(h, &h->TR, h->nR) || !dalloc(h, &h->dens_x, h->nx) ||
      !dalloc(h, &h->pot, h->nx) || !dalloc(h, &h->dens_R, h->nR) || !dalloc(h, &h->part, ncb) ||
      !dalloc(h, &h->proj, (size_t)e2d::MAX_STATES * h->nR)) {
    release(h);
    delete h;
    return fail2(nullptr, ICWF_ERR_OOM, "icwf_exact2d_create: cudaMalloc failed");
  }
  std::vector<double2> half(NN), kx, kR, tx, tR;
  std::vector<double> Tx, TR;
  for (size_t e = 0; e < NN; ++e)
    half[e] = make_double2(std::cos(-0.5 * p->dt * V[e]), std::sin(-0.5 * p->dt * V[e]));
  e2d::tables(h->nx, h->dx, p->mass_x, p->dt, kx, Tx, tx);
  e2d::tables(h->nR, h->dR, p->mass_R, p->dt, kR, TR, tR);
  const auto H2D = cudaMemcpyHostToDevice;
  bool ok = copy(h, h->V, V, NN * 8, H2D) && copy(h, h->half, half.data(), NN * 16, H2D) &&
            copy(h, h->kinx, kx.data(), kx.size() * 16, H2D) &&
            copy(h, h->kinR, kR.data(), kR.size() * 16, H2D) &&
            copy(h, h->twx, tx.data(), tx.size() * 16, H2D) &&
            copy(h, h->twR, tR.data(), tR.size() * 16, H2D) &&
            copy(h, h->Tx, Tx.data(), Tx.size() * 8, H2D) &&
            copy(h, h->TR, TR.data(), TR.size() * 8, H2D);
  if (!ok) {
    release(h);
    delete h;
    return fail2(nullptr, ICWF_ERR_CUDA, "icwf_exact2d_create: upload failed");
  }
  // the largest dynamic shared memory any handle uses (nR <= 4096 rows, CB * nx <= 96 KB), so
  // that handles of different sizes can coexist
  cudaFuncSetAttribute(e2d::k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       4096 * (int)sizeof(double2));
  cudaFuncSetAttribute(e2d::k_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  *out = h;
  return ICWF_OK;
}

icwf_status icwf_exact2d_set_state(icwf_exact2d h, const double* psi) {
  if (!h || !psi) return fail2(h, ICWF_ERR_ARG, "icwf_exact2d_set_state: null pointer");
  const size_t NN = (size_t)h->nx * h->nR;
  if (!copy(h, h->psi, psi, NN * 16, cudaMemcpyHostToDevice))
    return fail2(h, ICWF_ERR_CUDA, "icwf_exact2d_set_state: upload failed");
  h->has_state = true;
  h->t = 0.0;
  return ICWF_OK;
}

icwf_status icwf_exact2d_set_projectors(icwf_exact2d h, int32_t n_states, const double* phi) {
  if (!h || !phi) return fail2(h, ICWF_ERR_ARG, "icwf_exact2d_set_projectors: null pointer");
  if (n_states < 1 || n_states > e2d::MAX_STATES)
    return fail2(h, ICWF_ERR_ARG, "icwf_exact2d_set_projectors: n_states must be in [1, 8]");
  const size_t n = (size_t)n_states * h->nR * h->nx;
  if (!h->phi && !dalloc(h, &h->phi, (size_t)e2d::MAX_STATES * h->nR * h->nx))
    return fail2(h, ICWF_ERR_OOM, "icwf_exact2d_set_projectors: cudaMalloc failed");
  if (!copy(h, h->phi, phi, n * 8, cudaMemcpyHostToDevice))
    return fail2(h, ICWF_ERR_CUDA, "icwf_exact2d_set_projectors: upload failed");
  h->ns = n_states;
  return ICWF_OK;
}

icwf_status icwf_exact2d_step(icwf_exact2d h, int32_t n_steps) {
  if (!h) return fail2(h, ICWF_ERR_ARG, "icwf_exact2d_step: null handle");
  if (n_steps < 0) return fail2(h, ICWF_ERR_ARG, "icwf_exact2d_step: n_steps < 0");
  if (!h->has_state) return fail2(h, ICWF_ERR_STATE, "icwf_exact2d_step: no state set");
  const int smr = h->nR * (int)sizeof(double2), smc = h->CB * h->nx * (int)sizeof(double2);
  for (int s = 0; s < n_steps; ++s) {
    e2d::k_rows<<<h->nx, e2d::TPB, smr, h->stream>>>(h->psi, h->psi, h->half, h->twR, h->nR,
                                                     h->logR, 0);
    e2d::k_cols<<<h->nR / h->CB, e2d::TPB, smc, h->stream>>>(h->psi, h->kinx, h->kinR, h->twx,
                                                             h->nx, h->logx, h->nR, h->CB, 0,
                                                             nullptr, nullptr, nullptr);
    e2d::k_rows<<<h->nx, e2d::TPB, smr, h->stream>>>(h->psi, h->psi, h->half, h->twR, h->nR,
                                                     h->logR, 1);
  }
  const icwf_status st = sync(h, "icwf_exact2d_step");
  if (st == ICWF_OK) h->t += n_steps * h->dt;
  return st;
}

icwf_status icwf_exact2d_get_state(icwf_exact2d h, double* psi) {
  if (!h || !psi) return fail2(h, ICWF_ERR_ARG, "icwf_exact2d_get_state: null pointer");
  if (!h->has_state) return fail2(h, ICWF_ERR_STATE, "icwf_exact2d_get_state: no state set");
  if (!copy(h, psi, h->psi, (size_t)h->nx * h->nR * 16, cudaMemcpyDeviceToHost))
    return fail2(h, ICWF_ERR_CUDA, "icwf_exact2d_get_state: download failed");
  return ICWF_OK;
}

icwf_status icwf_exact2d_observables(icwf_exact2d h, icwf_obs* out) {
  if (!h || !out) return fail2(h, ICWF_ERR_ARG, "icwf_exact2d_observables: null pointer");
  if (!h->has_state) return fail2(h, ICWF_ERR_STATE, "icwf_exact2d_observables: no state set");
  const int nx = h->nx, nR = h->nR, ncb = nR / h->CB;
  const int smr = nR * (int)sizeof(double2), smc = h->CB * nx * (int)sizeof(double2);
  e2d::k_dens_rows<<<nx, e2d::TPB, 0, h->stream>>>(h->psi, h->V, nR, h->dens_x, h->pot);
  e2d::k_cols_obs<<<nR, e2d::TPB, 0, h->stream>>>(h->psi, nx, nR, h->phi, h->ns, h->dens_R, h->proj);
  // kinetic energy: 2D FFT of Psi into work, then sum |F|^2 (Tx + TR) per column group
  e2d::k_rows<<<nx, e2d::TPB, smr, h->stream>>>(h->psi, h->work, nullptr, h->twR, nR, h->logR, 0);
  e2d::k_cols<<<ncb, e2d::TPB, smc, h->stream>>>(h->work, nullptr, nullptr, h->twx, nx, h->logx,
                                                 nR, h->CB, 1, h->Tx, h->TR, h->part);
  icwf_status st = sync(h, "icwf_exact2d_observables");
  if (st != ICWF_OK) return st;
  std::vector<double> dx_(nx), pot(nx), dR_(nR), part(ncb);
  std::vector<double2> proj((size_t)h->ns * nR);
  const auto D2H = cudaMemcpyDeviceToHost;
  bool ok = copy(h, dx_.data(), h->dens_x, nx * 8, D2H) && copy(h, pot.data(), h->pot, nx * 8, D2H) &&
            copy(h, dR_.data(), h->dens_R, nR * 8, D2H) && copy(h, part.data(), h->part, ncb * 8, D2H) &&
            (h->ns == 0 || copy(h, proj.data(), h->proj, proj.size() * 16, D2H));
  if (!ok) return fail2(h, ICWF_ERR_CUDA, "icwf_exact2d_observables: download failed");
  double norm = 0.0, epot = 0.0, ekin = 0.0;
  for (int i = 0; i < nx; ++i) { norm += dx_[i]; epot += pot[i]; }
  for (int c = 0; c < ncb; ++c) ekin += part[c];
  norm *= h->dx * h->dR;
  epot *= h->dx * h->dR;
  ekin *= h->dx * h->dR / ((double)nx * nR);
  out->t = h->t;
  out->norm = norm;
  out->energy = norm > 0 ? (ekin + epot) / norm : 0.0;
  out->n_clamped = 0;
  out->n_states = h->ns;
  if (out->rho_x)
    for (int i = 0; i < nx; ++i) out->rho_x[i] = h->dR * dx_[i];
  if (out->rho_R)
    for (int j = 0; j < nR; ++j) out->rho_R[j] = h->dx * dR_[j];
  if (h->ns > 0) {
    std::vector<double> pn((size_t)h->ns * nR);
    for (int n = 0; n < h->ns; ++n)
      for (int j = 0; j < nR; ++j) {
        const double2 z = proj[(size_t)n * nR + j];
        const double re = h->dx * z.x, im = h->dx * z.y;
        pn[(size_t)n * nR + j] = re * re + im * im;
      }
    if (out->pop)
      for (int n = 0; n < h->ns; ++n) {
        double s = 0.0;
        for (int j = 0; j < nR; ++j) s += pn[(size_t)n * nR + j];
        out->pop[n] = h->dR * s;
      }
    if (out->decoh)
      for (int n = 0; n < h->ns; ++n)
        for (int m = 0; m < h->ns; ++m) {
          double s = 0.0;
          for (int j = 0; j < nR; ++j) s += pn[(size_t)n * nR + j] * pn[(size_t)m * nR + j];
          out->decoh[n * h->ns + m] = h->dR * s;
        }
  }
  return ICWF_OK;
}

icwf_status icwf_exact2d_destroy(icwf_exact2d h) {
  if (!h) return ICWF_OK;
  release(h);
  delete h;
  return ICWF_OK;
}

const char* icwf_exact2d_last_error(icwf_exact2d h) { return h ? h->err.c_str() : g_err2.c_str(); }

}  // extern "C"
