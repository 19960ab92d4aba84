// Observables of the ICWF wavefunction (Eq. ansatz reconstructed on the grid) and the initial
// projection of Psi0 on the product basis.
//   reconstruct  Psi(x_i, R_j) = sum_a C_a psi_a(x_i) chi_a(R_j)
//   obs          reduced densities rho_x, rho_R; <V>; BO projections chi^(n)(R) = int dx phi_n Psi;
//                kinetic energies by Parseval on the FFT of every grid line; final FP64 sums of
//                norm, energy, populations P_n and decoherence indicators D_nm (the quantities
//                the paper monitors in its two applications).
#include <cuda_runtime.h>

#include "icwf_internal.h"
#include "df64.cuh"
#include "k_common.cuh"

namespace icwf {

constexpr int RT = 32;   // reconstruction tile (grid points)
constexpr int RC = 16;   // trajectories per staged chunk (FP64 CWFs)
constexpr int RCF = 32;  // trajectories per staged chunk (complex64 CWFs)

// FP64 CWFs: every product and sum in FP64.
template <typename T>
__device__ __forceinline__ void reconstruct_fp64(const JobView& j, const double2* __restrict__ C,
                                                 double2* __restrict__ Psi) {
  using Z = c_t<T>;
  __shared__ double2 P[RC][RT + 1];
  __shared__ double2 Q[RC][RT + 1];
  const int it = blockIdx.y, jt = blockIdx.x;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const Z* psi = (const Z*)j.psi;
  const Z* chi = (const Z*)j.chi;
  const double2 z = make_double2(0, 0);
  double2 acc[2][2] = {{z, z}, {z, z}};
  const int la = threadIdx.x >> 5;          // 0..7: trajectory within chunk (two passes)
  const int lp = threadIdx.x & 31;          // grid point within tile
  for (int a0 = 0; a0 < j.N; a0 += RC) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int a = a0 + la + 8 * q;
      double2 p = z, w = z;
      const int i = it * RT + lp, jj = jt * RT + lp;
      if (a < j.N) {
        if (i < j.nx) p = cmul(C[a], to_d(psi[(size_t)a * j.nx + i]));
        if (jj < j.nR) w = to_d(chi[(size_t)a * j.nR + jj]);
      }
      P[la + 8 * q][lp] = p;
      Q[la + 8 * q][lp] = w;
    }
    __syncthreads();
#pragma unroll 4
    for (int a = 0; a < RC; ++a) {
      const double2 p0 = P[a][ty], p1 = P[a][ty + 16];
      const double2 q0 = Q[a][tx], q1 = Q[a][tx + 16];
      cfma(acc[0][0], p0, q0); cfma(acc[0][1], p0, q1);
      cfma(acc[1][0], p1, q0); cfma(acc[1][1], p1, q1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = it * RT + ty + 16 * r, jj = jt * RT + tx + 16 * c;
      if (i < j.nx && jj < j.nR) Psi[(size_t)i * j.nR + jj] = acc[r][c];
    }
}

// Complex64 CWFs (mixed modes): the terms C_a psi_a(x_i) chi_a(R_j) and their sums over chunks of
// RCF trajectories in FP32 (C rounded to FP32; the CWFs carry FP32 rounding already), the chunk
// sums added error-free into double-float accumulators (TwoSum), the result written in FP64.
// FP64 arithmetic would bound this GEMM-shaped sum on this GPU (~1/60 of the FP32 rate).  On the
// Shin-Metiu bench grid (N = 256 and 1024, where the terms' magnitudes add up to ~25-50x |Psi|)
// this changes rho_x, rho_R, P_n and the norm by < 2e-7 (L1) against FP64 sums of the same
// complex64 CWFs.
__device__ __forceinline__ void reconstruct_f32(const JobView& j, const double2* __restrict__ C,
                                                double2* __restrict__ Psi) {
  __shared__ float2 P[RCF][RT + 1];
  __shared__ float2 Q[RCF][RT + 1];
  __shared__ float2 Cs[RCF];
  const int it = blockIdx.y, jt = blockIdx.x;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const float2* psi = (const float2*)j.psi;
  const float2* chi = (const float2*)j.chi;
  const float2 z = make_float2(0.f, 0.f);
  df acc[2][2][2];   // [row][column][re, im]
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) acc[r][c][0] = acc[r][c][1] = df_make(0.f, 0.f);
  const int la = threadIdx.x >> 5;          // 0..7: trajectory within chunk (four passes)
  const int lp = threadIdx.x & 31;          // grid point within tile
  const int i = it * RT + lp, jj = jt * RT + lp;
  for (int a0 = 0; a0 < j.N; a0 += RCF) {
    if (threadIdx.x < RCF) {
      const int a = a0 + threadIdx.x;
      Cs[threadIdx.x] = a < j.N ? make_float2((float)C[a].x, (float)C[a].y) : z;
    }
#pragma unroll
    for (int q = 0; q < RCF / 8; ++q) {
      const int a = a0 + la + 8 * q;
      float2 p = z, w = z;
      if (a < j.N) {
        if (i < j.nx) p = psi[(size_t)a * j.nx + i];
        if (jj < j.nR) w = chi[(size_t)a * j.nR + jj];
      }
      P[la + 8 * q][lp] = p;
      Q[la + 8 * q][lp] = w;
    }
    __syncthreads();
    float2 s[2][2] = {{z, z}, {z, z}};
#pragma unroll 8
    for (int a = 0; a < RCF; ++a) {
      const float2 c = Cs[a];
      const float2 p0 = cmul(c, P[a][ty]), p1 = cmul(c, P[a][ty + 16]);
      const float2 q0 = Q[a][tx], q1 = Q[a][tx + 16];
      cfma(s[0][0], p0, q0); cfma(s[0][1], p0, q1);
      cfma(s[1][0], p1, q0); cfma(s[1][1], p1, q1);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        acc[r][c][0] = df_add_f(acc[r][c][0], s[r][c].x);
        acc[r][c][1] = df_add_f(acc[r][c][1], s[r][c].y);
      }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int ii = it * RT + ty + 16 * r, jc = jt * RT + tx + 16 * c;
      if (ii < j.nx && jc < j.nR)
        Psi[(size_t)ii * j.nR + jc] = make_double2(df_to(acc[r][c][0]), df_to(acc[r][c][1]));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_reconstruct(JobView j, const double2* __restrict__ C,
                                                     double2* __restrict__ Psi) {
  if constexpr (sizeof(T) == 4) reconstruct_f32(j, C, Psi);
  else reconstruct_fp64<T>(j, C, Psi);
}

template <typename T>
void launch_reconstruct(const JobView& j, const double2* C, double2* Psi, cudaStream_t s) {
  dim3 g((j.nR + RT - 1) / RT, (j.nx + RT - 1) / RT);
  k_reconstruct<T><<<g, 256, 0, s>>>(j, C, Psi);
}
template void launch_reconstruct<double>(const JobView&, const double2*, double2*, cudaStream_t);
template void launch_reconstruct<float>(const JobView&, const double2*, double2*, cudaStream_t);

// Deterministic block sum of one double per thread (blockDim.x = 256).
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

struct ObsArgs {
  const double2* Psi;
  const double* phi;
  int n_states;
  double* rho_x;
  double* rho_R;
  double2* proj;     // n_states x nR
  double* part;      // [0,nR): kinetic x per column; [nR,2nR): potential per column;
                     // [2nR, 2nR+nx): kinetic R per row
  const double2* twx;
  const double2* twR;
};

// Blocks [0, nR): column j (the x line at R_j); blocks [nR, nR+nx): row i (the R line at x_i).
__global__ void __launch_bounds__(256) k_obs_lines(JobView j, ObsArgs o) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = (double2*)smem_raw;
  __shared__ double red[256];
  const bool col = blockIdx.x < (unsigned)j.nR;
  const int line = col ? blockIdx.x : blockIdx.x - j.nR;
  const int n = col ? j.nx : j.nR;
  const int logn = col ? j.logx : j.logR;
  double dens = 0.0, pot = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const size_t idx = col ? (size_t)e * j.nR + line : (size_t)line * j.nR + e;
    const double2 v = o.Psi[idx];
    buf[e] = v;
    const double d = v.x * v.x + v.y * v.y;
    dens += d;
    if (col) pot += j.V[idx] * d;
  }
  __syncthreads();
  const double sd = block_sum(dens, red);
  if (col) {
    const double sp = block_sum(pot, red);
    if (threadIdx.x == 0) {
      o.rho_R[line] = j.dx * sd;
      o.part[j.nR + line] = j.dx * j.dR * sp;
    }
    for (int ns = 0; ns < o.n_states; ++ns) {
      const double* ph = o.phi + ((size_t)ns * j.nR + line) * j.nx;
      double pr = 0.0, pi = 0.0;
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        pr += ph[e] * buf[e].x;
        pi += ph[e] * buf[e].y;
      }
      const double sr = block_sum(pr, red);
      const double si = block_sum(pi, red);
      if (threadIdx.x == 0) o.proj[(size_t)ns * j.nR + line] = make_double2(j.dx * sr, j.dx * si);
    }
  } else {
    if (threadIdx.x == 0) o.rho_x[line] = j.dR * sd;
  }
  fft_dif(buf, col ? o.twx : o.twR, n, logn);
  double ek = 0.0;
  for (int mp = threadIdx.x; mp < n; mp += blockDim.x) {
    int m = (int)(__brev((unsigned)mp) >> (32 - logn));
    if (m >= n / 2) m -= n;
    ek += (buf[mp].x * buf[mp].x + buf[mp].y * buf[mp].y) * ((double)m * (double)m);
  }
  const double se = block_sum(ek, red);
  if (threadIdx.x == 0) {
    const double PI = 3.14159265358979323846;
    if (col) {
      const double g = 2.0 * PI / (j.nx * j.dx);
      o.part[line] = j.dR * (j.dx / j.nx) * se * g * g * 0.5 * j.inv_mx;
    } else {
      const double g = 2.0 * PI / (j.nR * j.dR);
      o.part[2 * j.nR + line] = j.dx * (j.dR / j.nR) * se * g * g * 0.5 * j.inv_mR;
    }
  }
}

// One block: out = {norm, ekx, ekR, epot}; pop[n]; decoh[n*ns + m].
__global__ void __launch_bounds__(256) k_obs_final(JobView j, ObsArgs o, double* out, double* pop,
                                                   double* decoh) {
  __shared__ double red[256];
  double a = 0, b = 0, c = 0, d = 0;
  for (int e = threadIdx.x; e < j.nR; e += blockDim.x) {
    a += o.rho_R[e];
    b += o.part[e];
    d += o.part[j.nR + e];
  }
  for (int e = threadIdx.x; e < j.nx; e += blockDim.x) c += o.part[2 * j.nR + e];
  const double sa = block_sum(a, red), sb = block_sum(b, red), sc = block_sum(c, red),
               sd = block_sum(d, red);
  if (threadIdx.x == 0) {
    out[0] = j.dR * sa;
    out[1] = sb;
    out[2] = sc;
    out[3] = sd;
  }
  for (int n = 0; n < o.n_states; ++n) {
    double p = 0;
    for (int e = threadIdx.x; e < j.nR; e += blockDim.x) {
      const double2 v = o.proj[(size_t)n * j.nR + e];
      p += v.x * v.x + v.y * v.y;
    }
    const double sp = block_sum(p, red);
    if (threadIdx.x == 0 && pop) pop[n] = j.dR * sp;
    for (int m = 0; m < o.n_states; ++m) {
      double q = 0;
      for (int e = threadIdx.x; e < j.nR; e += blockDim.x) {
        const double2 u = o.proj[(size_t)n * j.nR + e], v = o.proj[(size_t)m * j.nR + e];
        q += (u.x * u.x + u.y * u.y) * (v.x * v.x + v.y * v.y);
      }
      const double sq = block_sum(q, red);
      if (threadIdx.x == 0 && decoh) decoh[n * o.n_states + m] = j.dR * sq;
    }
  }
}

void launch_obs_lines(const JobView& j, const double2* Psi, const double* phi, int n_states,
                      double* rho_x, double* rho_R, double2* proj, double* part, double* out,
                      double* pop, double* decoh, const double2* twx, const double2* twR,
                      cudaStream_t s) {
  ObsArgs o{Psi, phi, n_states, rho_x, rho_R, proj, part, twx, twR};
  const int nmax = j.nx > j.nR ? j.nx : j.nR;
  const size_t sm = (size_t)nmax * sizeof(double2);
  if (sm > 40 * 1024)
    cudaFuncSetAttribute(k_obs_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_obs_lines<<<j.nR + j.nx, 256, sm, s>>>(j, o);
  k_obs_final<<<1, 256, 0, s>>>(j, o, out, pop, decoh);
}

// b_a = dx dR sum_i conj(psi_a(x_i)) sum_j Psi0[i, j] conj(chi_a(R_j)); one CTA per a, one warp
// per grid row i at a time.
__global__ void __launch_bounds__(256) k_init_projection(int N, int nx, int nR, double dx, double dR,
                                                         const double2* __restrict__ psi,
                                                         const double2* __restrict__ chi,
                                                         const double2* __restrict__ Psi0,
                                                         double2* __restrict__ b) {
  __shared__ double red[256];
  const int a = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double2* ca = chi + (size_t)a * nR;
  const double2* pa = psi + (size_t)a * nx;
  double2 acc = make_double2(0, 0);
  for (int i = warp; i < nx; i += 8) {
    double2 t = make_double2(0, 0);
    const double2* row = Psi0 + (size_t)i * nR;
    for (int jj = lane; jj < nR; jj += 32) cfma(t, row[jj], cconj(ca[jj]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
      t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
    }
    if (lane == 0) cfmac(acc, pa[i], t);
  }
  const double sr = block_sum(lane == 0 ? acc.x : 0.0, red);
  const double si = block_sum(lane == 0 ? acc.y : 0.0, red);
  if (threadIdx.x == 0) b[a] = make_double2(dx * dR * sr, dx * dR * si);
}

void launch_init_projection(int N, int nx, int nR, double dx, double dR, const double2* psi,
                            const double2* chi, const double2* Psi0, double2* b, cudaStream_t s) {
  k_init_projection<<<N, 256, 0, s>>>(N, nx, nR, dx, dR, psi, chi, Psi0, b);
}

}  // namespace icwf
