// Per-step kernels of the ICWF update (arXiv 1805.11169):
//   velocity   Eq. v1/v2 at the trajectory positions, explicit Euler positions, and the pinned
//              factor values u_k(x_b), w_k(R_b), V(x_b, R_b) at the new positions;
//   propagate  Hermitian-CWF equations (Eq. conditional_e/n with eta dropped): one Strang
//              split-operator step per CWF, one CTA per CWF, the column staged in shared memory;
//   assemble   FP64 matrix elements (Eq. M, W, W1, W2) from the rank-k factorisation;
//   gram       generic A^H diag(d) B (diagnostics: kinetic and potential Grams for H).
#include <cuda_runtime.h>

#include "icwf_internal.h"
#include "k_common.cuh"

namespace icwf {

// ------------------------------------------------------------------------------ velocities

// One warp per trajectory a (all 32 lanes take part; the caller keeps a warp-uniform).
template <typename T>
__device__ __forceinline__ void velocity_warp(const JobView& j, const double2* __restrict__ C,
                                              double xlo, double xhi, double Rlo, double Rhi,
                                              int a, int lane) {
  using Z = c_t<T>;
  if (a >= j.N) return;
  const double xa = j.x[a], Ra = j.R[a];
  const Stencil sx = lagrange4(xa, j.x_min, j.dx, j.nx);
  const Stencil sR = lagrange4(Ra, j.R_min, j.dR, j.nR);
  const Z* psi = (const Z*)j.psi;
  const Z* chi = (const Z*)j.chi;
  double2 den = make_double2(0, 0), nux = den, nuR = den;
  for (int b = lane; b < j.N; b += 32) {
    const Z* pc = psi + (size_t)b * j.nx + sx.i0;
    const Z* qc = chi + (size_t)b * j.nR + sR.i0;
    double2 E1 = make_double2(0, 0), G1 = E1, E2 = E1, G2 = E1;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const double2 p = to_d(pc[m]);
      const double2 q = to_d(qc[m]);
      E1.x = fma(sx.w[m], p.x, E1.x);  E1.y = fma(sx.w[m], p.y, E1.y);
      G1.x = fma(sx.dw[m], p.x, G1.x); G1.y = fma(sx.dw[m], p.y, G1.y);
      E2.x = fma(sR.w[m], q.x, E2.x);  E2.y = fma(sR.w[m], q.y, E2.y);
      G2.x = fma(sR.dw[m], q.x, G2.x); G2.y = fma(sR.dw[m], q.y, G2.y);
    }
    const double2 cb = C[b];
    const double2 c1 = cmul(cb, E1);
    den = cadd(den, cmul(c1, E2));
    nux = cadd(nux, cmul(cmul(cb, G1), E2));
    nuR = cadd(nuR, cmul(c1, G2));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    den.x += __shfl_xor_sync(0xffffffffu, den.x, off);
    den.y += __shfl_xor_sync(0xffffffffu, den.y, off);
    nux.x += __shfl_xor_sync(0xffffffffu, nux.x, off);
    nux.y += __shfl_xor_sync(0xffffffffu, nux.y, off);
    nuR.x += __shfl_xor_sync(0xffffffffu, nuR.x, off);
    nuR.y += __shfl_xor_sync(0xffffffffu, nuR.y, off);
  }
  // Im(num / den) = (num.y den.x - num.x den.y) / |den|^2
  const double dd = den.x * den.x + den.y * den.y;
  const double vx = (nux.y * den.x - nux.x * den.y) / dd * j.inv_mx;
  const double vR = (nuR.y * den.x - nuR.x * den.y) / dd * j.inv_mR;
  double xn = xa + j.dt * vx;
  double Rn = Ra + j.dt * vR;
  if (lane == 0) {
    if (!isfinite(vx) || !isfinite(vR)) set_flag(j.status, ST_NONFINITE);
    int cl = 0;
    if (xn < xlo) { xn = xlo; ++cl; } else if (xn > xhi) { xn = xhi; ++cl; }
    if (Rn < Rlo) { Rn = Rlo; ++cl; } else if (Rn > Rhi) { Rn = Rhi; ++cl; }
    if (cl) atomicAdd(j.status + STATUS_CLAMPED, cl);
    j.xo[a] = xa; j.Ro[a] = Ra;
    j.x[a] = xn;  j.R[a] = Rn;
  }
  xn = __shfl_sync(0xffffffffu, xn < xlo ? xlo : (xn > xhi ? xhi : xn), 0);
  Rn = __shfl_sync(0xffffffffu, Rn < Rlo ? Rlo : (Rn > Rhi ? Rhi : Rn), 0);
  if (!isfinite(xn)) xn = xa;
  if (!isfinite(Rn)) Rn = Ra;
  // pinned factor values at the new position (used by the assembly at t + dt)
  const Stencil tx = lagrange4(xn, j.x_min, j.dx, j.nx);
  const Stencil tR = lagrange4(Rn, j.R_min, j.dR, j.nR);
  double part = 0.0;
  for (int k = lane; k < j.K; k += 32) {
    const double* u = j.U + (size_t)k * j.nx + tx.i0;
    const double* w = j.W + (size_t)k * j.nR + tR.i0;
    const double uk = tx.w[0] * u[0] + tx.w[1] * u[1] + tx.w[2] * u[2] + tx.w[3] * u[3];
    const double wk = tR.w[0] * w[0] + tR.w[1] * w[1] + tR.w[2] * w[2] + tR.w[3] * w[3];
    j.px[(size_t)k * j.N + a] = uk;
    j.pR[(size_t)k * j.N + a] = wk;
    part += j.sig[k] * (uk * wk);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if (lane == 0) {
    const double* v1 = j.v1 + tx.i0;
    const double* v2 = j.v2 + tR.i0;
    const double a1 = tx.w[0] * v1[0] + tx.w[1] * v1[1] + tx.w[2] * v1[2] + tx.w[3] * v1[3];
    const double a2 = tR.w[0] * v2[0] + tR.w[1] * v2[1] + tR.w[2] * v2[2] + tR.w[3] * v2[3];
    j.d[a] = a1 + a2 + part;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_velocity(JobView j, const double2* __restrict__ C,
                                                  double xlo, double xhi, double Rlo, double Rhi) {
  velocity_warp<T>(j, C, xlo, xhi, Rlo, Rhi, (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5),
                   threadIdx.x & 31);
}

// FP32 version for the mixed modes (complex64 CWFs): stencil weights (lagrange4f), interpolation
// and the three sums in FP32 (FP64 arithmetic is slow and long-latency on this GPU); the position
// update itself stays FP64.  Pinned factor values at the new positions in FP32 as well (the
// tensor-core assembly consumes them in FP32).
// One warp per trajectory a.  The coefficients are read in FP32 from Cf, or, with kFromC, rounded
// from C on the fly (the same values k_coeff_to_f32 stores in Cf).
template <bool kFromC>
__device__ __forceinline__ void velocity_warp_f32(const JobView& j, const double2* __restrict__ C,
                                                  double xlo, double xhi, double Rlo, double Rhi,
                                                  float inv_mx, float inv_mR,
                                                  const float* __restrict__ Cf, int a, int lane) {
  if (a >= j.N) return;
  const double xa = j.x[a], Ra = j.R[a];
  const StencilF sx = lagrange4f(xa, j.x_min, j.dx, j.nx);
  const StencilF sR = lagrange4f(Ra, j.R_min, j.dR, j.nR);
  const float2* psi = (const float2*)j.psi;
  const float2* chi = (const float2*)j.chi;
  float2 den = make_float2(0.f, 0.f), nux = den, nuR = den;
  for (int b = lane; b < j.N; b += 32) {
    const float2* pc = psi + (size_t)b * j.nx + sx.i0;
    const float2* qc = chi + (size_t)b * j.nR + sR.i0;
    float2 E1 = make_float2(0.f, 0.f), G1 = E1, E2 = E1, G2 = E1;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float2 p = pc[m], q = qc[m];
      E1.x = fmaf(sx.w[m], p.x, E1.x);  E1.y = fmaf(sx.w[m], p.y, E1.y);
      G1.x = fmaf(sx.dw[m], p.x, G1.x); G1.y = fmaf(sx.dw[m], p.y, G1.y);
      E2.x = fmaf(sR.w[m], q.x, E2.x);  E2.y = fmaf(sR.w[m], q.y, E2.y);
      G2.x = fmaf(sR.dw[m], q.x, G2.x); G2.y = fmaf(sR.dw[m], q.y, G2.y);
    }
    const float2 cb = kFromC ? make_float2((float)C[b].x, (float)C[b].y)
                             : make_float2(Cf[2 * b], Cf[2 * b + 1]);
    const float2 c1 = cmul(cb, E1);
    den = cadd(den, cmul(c1, E2));
    nux = cadd(nux, cmul(cmul(cb, G1), E2));
    nuR = cadd(nuR, cmul(c1, G2));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    den.x += __shfl_xor_sync(0xffffffffu, den.x, off);
    den.y += __shfl_xor_sync(0xffffffffu, den.y, off);
    nux.x += __shfl_xor_sync(0xffffffffu, nux.x, off);
    nux.y += __shfl_xor_sync(0xffffffffu, nux.y, off);
    nuR.x += __shfl_xor_sync(0xffffffffu, nuR.x, off);
    nuR.y += __shfl_xor_sync(0xffffffffu, nuR.y, off);
  }
  const float dd = den.x * den.x + den.y * den.y;
  const float vx = (nux.y * den.x - nux.x * den.y) / dd * inv_mx;
  const float vR = (nuR.y * den.x - nuR.x * den.y) / dd * inv_mR;
  double xn = xa + j.dt * (double)vx;
  double Rn = Ra + j.dt * (double)vR;
  if (lane == 0) {
    if (!isfinite(vx) || !isfinite(vR)) set_flag(j.status, ST_NONFINITE);
    int cl = 0;
    if (xn < xlo) { xn = xlo; ++cl; } else if (xn > xhi) { xn = xhi; ++cl; }
    if (Rn < Rlo) { Rn = Rlo; ++cl; } else if (Rn > Rhi) { Rn = Rhi; ++cl; }
    if (cl) atomicAdd(j.status + STATUS_CLAMPED, cl);
    j.xo[a] = xa; j.Ro[a] = Ra;
    j.x[a] = xn;  j.R[a] = Rn;
  }
  xn = __shfl_sync(0xffffffffu, xn < xlo ? xlo : (xn > xhi ? xhi : xn), 0);
  Rn = __shfl_sync(0xffffffffu, Rn < Rlo ? Rlo : (Rn > Rhi ? Rhi : Rn), 0);
  if (!isfinite(xn)) xn = xa;
  if (!isfinite(Rn)) Rn = Ra;
  const StencilF tx = lagrange4f(xn, j.x_min, j.dx, j.nx);
  const StencilF tR = lagrange4f(Rn, j.R_min, j.dR, j.nR);
  float part = 0.f;
  for (int k = lane; k < j.K; k += 32) {
    const double* u = j.U + (size_t)k * j.nx + tx.i0;
    const double* w = j.W + (size_t)k * j.nR + tR.i0;
    const float uk = tx.w[0] * (float)u[0] + tx.w[1] * (float)u[1] + tx.w[2] * (float)u[2] + tx.w[3] * (float)u[3];
    const float wk = tR.w[0] * (float)w[0] + tR.w[1] * (float)w[1] + tR.w[2] * (float)w[2] + tR.w[3] * (float)w[3];
    j.px[(size_t)k * j.N + a] = uk;
    j.pR[(size_t)k * j.N + a] = wk;
    part += (float)j.sig[k] * (uk * wk);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if (lane == 0) {
    const double* v1 = j.v1 + tx.i0;
    const double* v2 = j.v2 + tR.i0;
    const float a1 = tx.w[0] * (float)v1[0] + tx.w[1] * (float)v1[1] + tx.w[2] * (float)v1[2] + tx.w[3] * (float)v1[3];
    const float a2 = tR.w[0] * (float)v2[0] + tR.w[1] * (float)v2[1] + tR.w[2] * (float)v2[2] + tR.w[3] * (float)v2[3];
    j.d[a] = (double)(a1 + a2 + part);
  }
}

__global__ void __launch_bounds__(256) k_velocity_f32(JobView j, const double2* __restrict__ C,
                                                      double xlo, double xhi, double Rlo, double Rhi,
                                                      float inv_mx, float inv_mR, float* __restrict__ Cf) {
  velocity_warp_f32<false>(j, C, xlo, xhi, Rlo, Rhi, inv_mx, inv_mR, Cf,
                           (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), threadIdx.x & 31);
}

__global__ void k_coeff_to_f32(int N, const double2* __restrict__ C, float* __restrict__ Cf) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < N) { Cf[2 * b] = (float)C[b].x; Cf[2 * b + 1] = (float)C[b].y; }
}

// Pinned factor values at the current positions without moving them (initialisation).
__global__ void k_pinned_only(JobView j) {
  const int a = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (a >= j.N) return;
  const Stencil tx = lagrange4(j.x[a], j.x_min, j.dx, j.nx);
  const Stencil tR = lagrange4(j.R[a], j.R_min, j.dR, j.nR);
  double part = 0.0;
  for (int k = lane; k < j.K; k += 32) {
    const double* u = j.U + (size_t)k * j.nx + tx.i0;
    const double* w = j.W + (size_t)k * j.nR + tR.i0;
    const double uk = tx.w[0] * u[0] + tx.w[1] * u[1] + tx.w[2] * u[2] + tx.w[3] * u[3];
    const double wk = tR.w[0] * w[0] + tR.w[1] * w[1] + tR.w[2] * w[2] + tR.w[3] * w[3];
    j.px[(size_t)k * j.N + a] = uk;
    j.pR[(size_t)k * j.N + a] = wk;
    part += j.sig[k] * (uk * wk);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if (lane == 0) {
    const double* v1 = j.v1 + tx.i0;
    const double* v2 = j.v2 + tR.i0;
    const double a1 = tx.w[0] * v1[0] + tx.w[1] * v1[1] + tx.w[2] * v1[2] + tx.w[3] * v1[3];
    const double a2 = tR.w[0] * v2[0] + tR.w[1] * v2[1] + tR.w[2] * v2[2] + tR.w[3] * v2[3];
    j.d[a] = a1 + a2 + part;
  }
}

GroupJob group_job(const JobView& j, const double2* C) {
  GroupJob q;
  q.j = j;
  q.C = C;
  q.xlo = j.x_min + 0.5 * j.dx;
  q.xhi = j.x_min + (j.nx - 0.5) * j.dx;
  q.Rlo = j.R_min + 0.5 * j.dR;
  q.Rhi = j.R_min + (j.nR - 0.5) * j.dR;
  q.inv_mx_f = (float)j.inv_mx;
  q.inv_mR_f = (float)j.inv_mR;
  q.traj0 = 0;
  q.cwf0 = 0;
  return q;
}

template <typename T>
void launch_velocity(const JobView& j, const double2* C, cudaStream_t s) {
  const int warps = 8;
  const int grid = (j.N + warps - 1) / warps;
  const GroupJob q = group_job(j, C);
  const double xlo = q.xlo, xhi = q.xhi, Rlo = q.Rlo, Rhi = q.Rhi;
  if (C == nullptr) {
    k_pinned_only<<<grid, warps * 32, 0, s>>>(j);
    return;
  }
  if (sizeof(T) == 4 && j.scratch_f32) {
    k_coeff_to_f32<<<(j.N + 255) / 256, 256, 0, s>>>(j.N, C, j.scratch_f32);
    k_velocity_f32<<<grid, warps * 32, 0, s>>>(j, C, xlo, xhi, Rlo, Rhi, q.inv_mx_f, q.inv_mR_f,
                                               j.scratch_f32);
    return;
  }
  k_velocity<T><<<grid, warps * 32, 0, s>>>(j, C, xlo, xhi, Rlo, Rhi);
}
template void launch_velocity<double>(const JobView&, const double2*, cudaStream_t);
template void launch_velocity<float>(const JobView&, const double2*, cudaStream_t);

// ------------------------------------------------------------------------------ propagation

// One CTA per CWF: CWF index a in [0, N) advances psi_a, a in [N, 2N) advances chi_(a-N).  The
// column and its potential phases live in shared memory buf (2 n complex).  mode 0: Strang step
// in place; mode 1: kinetic operator applied, result to out.  Every thread of the CTA calls it.
template <typename T>
__device__ __forceinline__ void propagate_cta(const JobView& j, const T* __restrict__ Vt, int mode,
                                              void* out_psi, void* out_chi, double kfx, double kfR,
                                              int a, c_t<T>* buf) {
  using Z = c_t<T>;
  const bool xs = a < j.N;
  if (!xs) a -= j.N;
  const int n = xs ? j.nx : j.nR;
  const int logn = xs ? j.logx : j.logR;
  Z* ph = buf + n;
  Z* col = (Z*)(xs ? j.psi : j.chi) + (size_t)a * n;
  const Z* tw = (const Z*)(xs ? j.twx : j.twR);
  if (mode == 0) {
    const Z* kin = (const Z*)(xs ? j.kinx : j.kinR);
    const T hdt = (T)(0.5 * j.dt);
    if (xs) {
      const double Rb = 0.5 * (j.Ro[a] + j.R[a]);
      const Stencil st = lagrange4(Rb, j.R_min, j.dR, j.nR);
      const T w0 = (T)st.w[0], w1 = (T)st.w[1], w2 = (T)st.w[2], w3 = (T)st.w[3];
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const T* vr = Vt + (size_t)i * j.nR + st.i0;
        const T v = w0 * vr[0] + w1 * vr[1] + w2 * vr[2] + w3 * vr[3];
        T sn, cs;
        sincos_t(v * hdt, &sn, &cs);
        const Z p = mk<T>(cs, -sn);
        ph[i] = p;
        buf[i] = cmul(p, col[i]);
      }
    } else {
      const double xb = 0.5 * (j.xo[a] + j.x[a]);
      const Stencil st = lagrange4(xb, j.x_min, j.dx, j.nx);
      const T w0 = (T)st.w[0], w1 = (T)st.w[1], w2 = (T)st.w[2], w3 = (T)st.w[3];
      const T* v0 = Vt + (size_t)st.i0 * j.nR;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const T v = w0 * v0[i] + w1 * v0[i + j.nR] + w2 * v0[i + 2 * j.nR] + w3 * v0[i + 3 * j.nR];
        T sn, cs;
        sincos_t(v * hdt, &sn, &cs);
        const Z p = mk<T>(cs, -sn);
        ph[i] = p;
        buf[i] = cmul(p, col[i]);
      }
    }
    __syncthreads();
    fft_dif(buf, tw, n, logn);
    for (int m = threadIdx.x; m < n; m += blockDim.x) buf[m] = cmul(buf[m], kin[m]);
    __syncthreads();
    ifft_dit(buf, tw, n, logn);
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = cmul(ph[i], buf[i]);
  } else {
    // T f = F^-1 (k^2 / 2m) F f / n; k for the bit-reversed slot m' is that of m = bitrev(m')
    const double kf = xs ? kfx : kfR;     // (2 pi / (n d))^2 / (2 m n)
    Z* out = (Z*)(xs ? out_psi : out_chi) + (size_t)a * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) buf[i] = col[i];
    __syncthreads();
    fft_dif(buf, tw, n, logn);
    for (int mp = threadIdx.x; mp < n; mp += blockDim.x) {
      int m = (int)(__brev((unsigned)mp) >> (32 - logn));
      if (m >= n / 2) m -= n;
      buf[mp] = cscale(buf[mp], (T)(kf * (double)m * (double)m));
    }
    __syncthreads();
    ifft_dit(buf, tw, n, logn);
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = buf[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_propagate(JobView j, const T* __restrict__ Vt, int mode,
                                                   void* out_psi, void* out_chi, double kfx,
                                                   double kfR) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  propagate_cta<T>(j, Vt, mode, out_psi, out_chi, kfx, kfR, blockIdx.x, (c_t<T>*)smem_raw);
}

// The propagator's dynamic shared memory limit, set once (to the largest grid's need) so that no
// launch, captured or not, changes a function attribute.
template <typename T>
void propagate_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_propagate<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * 4096 * sizeof(c_t<T>)));
    done = true;
  }
}

template <typename T>
void launch_propagate(const JobView& j, int threads, cudaStream_t s) {
  const int nmax = j.nx > j.nR ? j.nx : j.nR;
  const size_t sm = 2 * (size_t)nmax * sizeof(c_t<T>);
  propagate_attr<T>();
  k_propagate<T><<<2 * j.N, threads, sm, s>>>(j, (const T*)j.Vt, 0, nullptr, nullptr, 0.0, 0.0);
}

template <typename T>
void launch_kinetic(const JobView& j, void* out_psi, void* out_chi, cudaStream_t s) {
  const int nmax = j.nx > j.nR ? j.nx : j.nR;
  const size_t sm = 2 * (size_t)nmax * sizeof(c_t<T>);
  propagate_attr<T>();
  const double PI = 3.14159265358979323846;
  const double gx = 2.0 * PI / (j.nx * j.dx), gR = 2.0 * PI / (j.nR * j.dR);
  const double kfx = gx * gx * 0.5 * j.inv_mx / j.nx;
  const double kfR = gR * gR * 0.5 * j.inv_mR / j.nR;
  k_propagate<T><<<2 * j.N, 256, sm, s>>>(j, (const T*)j.Vt, 1, out_psi, out_chi, kfx, kfR);
}
template void launch_propagate<double>(const JobView&, int, cudaStream_t);
template void launch_propagate<float>(const JobView&, int, cudaStream_t);
template void launch_kinetic<double>(const JobView&, void*, void*, cudaStream_t);
template void launch_kinetic<float>(const JobView&, void*, void*, cudaStream_t);

// ------------------------------------------------------------------------------ grouped launches

// Velocities, positions and pinned factor values of every trajectory of every job in the group:
// a warp per trajectory, the warps striding over all trajectories of the group.  The mixed modes
// round C to FP32 on the fly (the values launch_velocity's k_coeff_to_f32 would store).
template <typename T>
__global__ void __launch_bounds__(256) k_velocity_group(const GroupJob* __restrict__ g, int njobs,
                                                        int total) {
  const int lane = threadIdx.x & 31;
  const int nw = (int)(gridDim.x * (blockDim.x >> 5));
  for (int item = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); item < total; item += nw) {
    const GroupJob& q = g[group_find(g, njobs, item, false)];
    if constexpr (sizeof(T) == 4)
      velocity_warp_f32<true>(q.j, q.C, q.xlo, q.xhi, q.Rlo, q.Rhi, q.inv_mx_f, q.inv_mR_f,
                              nullptr, item - q.traj0, lane);
    else
      velocity_warp<T>(q.j, q.C, q.xlo, q.xhi, q.Rlo, q.Rhi, item - q.traj0, lane);
  }
}

// Strang step of every CWF of every job in the group: a CTA per CWF, the CTAs striding over all
// CWFs of the group; dynamic shared memory sized for the group's largest grid.
template <typename T>
__global__ void __launch_bounds__(512) k_propagate_group(const GroupJob* __restrict__ g, int njobs,
                                                         int total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const GroupJob& q = g[group_find(g, njobs, item, true)];
    propagate_cta<T>(q.j, (const T*)q.j.Vt, 0, nullptr, nullptr, 0.0, 0.0, item - q.cwf0,
                     (c_t<T>*)smem_raw);
    __syncthreads();   // the next item overwrites the shared column
  }
}

template <typename T>
bool add_group_nodes(cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps,
                     const GroupJob* table, int njobs, int total_traj, int total_cwf, int nmax,
                     int threads, int max_ctas, cudaGraphNode_t* last) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_propagate_group<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * 4096 * sizeof(c_t<T>))) != cudaSuccess)
      return false;
    attr = true;
  }
  if (njobs < 1 || total_traj < 1 || total_cwf < 1 || nmax < 1 || nmax > 4096 || threads < 64 ||
      threads > 512)
    return false;
  int dev = 0, sms = 0, occ_v = 0, occ_p = 0;
  const size_t sm = 2 * (size_t)nmax * sizeof(c_t<T>);
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_v, k_velocity_group<T>, 256, 0) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, k_propagate_group<T>, threads, sm) !=
          cudaSuccess)
    return false;
  if (occ_v < 1 || occ_p < 1) return false;
  long long gv = ((long long)total_traj + 7) / 8, gp = total_cwf;
  if (gv > (long long)occ_v * sms) gv = (long long)occ_v * sms;
  if (gp > (long long)occ_p * sms) gp = (long long)occ_p * sms;
  if (max_ctas > 0 && gv > max_ctas) gv = max_ctas;
  if (max_ctas > 0 && gp > max_ctas) gp = max_ctas;
  cudaKernelNodeParams kp = {};
  void* av[] = {(void*)&table, (void*)&njobs, (void*)&total_traj};
  kp.func = (void*)k_velocity_group<T>;
  kp.gridDim = dim3((unsigned)gv);
  kp.blockDim = dim3(256);
  kp.sharedMemBytes = 0;
  kp.kernelParams = av;
  cudaGraphNode_t nv, np;
  if (cudaGraphAddKernelNode(&nv, graph, deps, ndeps, &kp) != cudaSuccess) return false;
  void* ap[] = {(void*)&table, (void*)&njobs, (void*)&total_cwf};
  kp.func = (void*)k_propagate_group<T>;
  kp.gridDim = dim3((unsigned)gp);
  kp.blockDim = dim3((unsigned)threads);
  kp.sharedMemBytes = (unsigned)sm;
  kp.kernelParams = ap;
  if (cudaGraphAddKernelNode(&np, graph, &nv, 1, &kp) != cudaSuccess) return false;
  *last = np;
  return true;
}
template bool add_group_nodes<double>(cudaGraph_t, const cudaGraphNode_t*, size_t,
                                      const GroupJob*, int, int, int, int, int, int,
                                      cudaGraphNode_t*);
template bool add_group_nodes<float>(cudaGraph_t, const cudaGraphNode_t*, size_t, const GroupJob*,
                                     int, int, int, int, int, int, cudaGraphNode_t*);

// ------------------------------------------------------------------------------ FP64 assembly

constexpr int AT = 32;   // output tile (trajectories)
constexpr int AKC = 16;  // grid points per shared-memory chunk

// Accumulate g[r][c] += sum_i conj(A[i, a_r]) dg[i] B[i, b_c] over the whole grid for the tile
// rows a in [I*AT, I*AT+AT) and columns b in [J*AT, J*AT+AT).  256 threads, 2x2 outputs each.
template <typename T>
__device__ __forceinline__ void gram_tile(const c_t<T>* __restrict__ A, const c_t<T>* __restrict__ B,
                                          const double* __restrict__ dg, int n, int N, int I, int J,
                                          double2 (&As)[AKC][AT + 1], double2 (&Bs)[AKC][AT + 1],
                                          double2 g[2][2]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int la = threadIdx.x >> 3;             // column within tile for loads
  const int li = (threadIdx.x & 7) * 2;        // first of two grid rows for loads
  const int ca = I * AT + la, cb = J * AT + la;
  for (int i0 = 0; i0 < n; i0 += AKC) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = i0 + li + q;
      double2 va = make_double2(0, 0), vb = va;
      if (i < n) {
        if (ca < N) va = to_d(A[(size_t)ca * n + i]);
        if (cb < N) {
          vb = to_d(B[(size_t)cb * n + i]);
          if (dg) vb = cscale(vb, dg[i]);
        }
      }
      As[li + q][la] = va;
      Bs[li + q][la] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < AKC; ++ii) {
      const double2 a0 = As[ii][ty], a1 = As[ii][ty + 16];
      const double2 b0 = Bs[ii][tx], b1 = Bs[ii][tx + 16];
      cfmac(g[0][0], a0, b0); cfmac(g[0][1], a0, b1);
      cfmac(g[1][0], a1, b0); cfmac(g[1][1], a1, b1);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void tri_index(int t, int& I, int& J) {
  int Jc = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (Jc * (Jc + 1) / 2 > t) --Jc;
  while ((Jc + 1) * (Jc + 2) / 2 <= t) ++Jc;
  J = Jc;
  I = t - Jc * (Jc + 1) / 2;
}

// One CTA per upper-triangular tile pair (I <= J): computes S and Heff for the tile (I, J) and,
// off the diagonal, for the mirrored tile (J, I), from the Hermitian Grams of that tile:
//   S1 = dx Psi^H Psi, S2 = dR X^H X, A_k = dx Psi^H diag(u_k) Psi, B_k = dR X^H diag(w_k) X,
//   Heff_ab = sum_k s_k (A_k - u_k(x_b) S1)_ab (B_k - w_k(R_b) S2)_ab - V(x_b,R_b) S_ab.
__global__ void __launch_bounds__(256) k_assemble_fp64(JobView j, double2* __restrict__ S,
                                                        double2* __restrict__ H) {
  __shared__ double2 As[AKC][AT + 1], Bs[AKC][AT + 1];
  int I, J;
  tri_index(blockIdx.x, I, J);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const double2* psi = (const double2*)j.psi;
  const double2* chi = (const double2*)j.chi;
  const int N = j.N;
  int ar[2] = {I * AT + ty, I * AT + ty + 16};
  int bc[2] = {J * AT + tx, J * AT + tx + 16};
  double2 s1[2][2], s2[2][2], h[2][2], ht[2][2];
  const double2 z = make_double2(0, 0);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) { s1[r][c] = z; s2[r][c] = z; h[r][c] = z; ht[r][c] = z; }
  const bool mirror = I != J;
  for (int k = -1; k < j.K; ++k) {
    double2 gx[2][2] = {{z, z}, {z, z}}, gR[2][2] = {{z, z}, {z, z}};
    gram_tile<double>(psi, psi, k < 0 ? nullptr : j.U + (size_t)k * j.nx, j.nx, N, I, J, As, Bs, gx);
    gram_tile<double>(chi, chi, k < 0 ? nullptr : j.W + (size_t)k * j.nR, j.nR, N, I, J, As, Bs, gR);
    if (k < 0) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) { s1[r][c] = cscale(gx[r][c], j.dx); s2[r][c] = cscale(gR[r][c], j.dR); }
      continue;
    }
    const double sk = j.sig[k];
    const double* pxk = j.px + (size_t)k * N;
    const double* pRk = j.pR + (size_t)k * N;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const double uxa = ar[r] < N ? pxk[ar[r]] : 0.0;
      const double wRa = ar[r] < N ? pRk[ar[r]] : 0.0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double uxb = bc[c] < N ? pxk[bc[c]] : 0.0;
        const double wRb = bc[c] < N ? pRk[bc[c]] : 0.0;
        const double2 A = cscale(gx[r][c], j.dx), B = cscale(gR[r][c], j.dR);
        const double2 At = csub(A, cscale(s1[r][c], uxb));
        const double2 Bt = csub(B, cscale(s2[r][c], wRb));
        const double2 p = cmul(At, Bt);
        h[r][c].x = fma(sk, p.x, h[r][c].x);
        h[r][c].y = fma(sk, p.y, h[r][c].y);
        if (mirror) {
          const double2 At2 = csub(cconj(A), cscale(cconj(s1[r][c]), uxa));
          const double2 Bt2 = csub(cconj(B), cscale(cconj(s2[r][c]), wRa));
          const double2 p2 = cmul(At2, Bt2);
          ht[r][c].x = fma(sk, p2.x, ht[r][c].x);
          ht[r][c].y = fma(sk, p2.y, ht[r][c].y);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (ar[r] >= N) continue;
    const double da = j.d[ar[r]];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (bc[c] >= N) continue;
      const double db = j.d[bc[c]];
      const double2 s = cmul(s1[r][c], s2[r][c]);
      S[(size_t)ar[r] * N + bc[c]] = s;
      H[(size_t)ar[r] * N + bc[c]] = csub(h[r][c], cscale(s, db));
      if (mirror) {
        S[(size_t)bc[c] * N + ar[r]] = cconj(s);
        H[(size_t)bc[c] * N + ar[r]] = csub(ht[r][c], cscale(cconj(s), da));
      }
    }
  }
}

void launch_assemble_fp64(const JobView& j, double2* S, double2* H, cudaStream_t s) {
  const int T = (j.N + AT - 1) / AT;
  k_assemble_fp64<<<T * (T + 1) / 2, 256, 0, s>>>(j, S, H);
}

// ------------------------------------------------------------------------------ diagnostics

template <typename T>
__global__ void __launch_bounds__(256) k_gram(const c_t<T>* A, const c_t<T>* B, const double* dg,
                                              int n, int N, double scale, double2* G) {
  __shared__ double2 As[AKC][AT + 1], Bs[AKC][AT + 1];
  const int I = blockIdx.y, J = blockIdx.x;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const double2 z = make_double2(0, 0);
  double2 g[2][2] = {{z, z}, {z, z}};
  gram_tile<T>(A, B, dg, n, N, I, J, As, Bs, g);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int a = I * AT + ty + 16 * r, b = J * AT + tx + 16 * c;
      if (a < N && b < N) G[(size_t)a * N + b] = cscale(g[r][c], scale);
    }
}

template <typename T>
void launch_gram(const void* A, const void* B, const double* dg, int n, int N, double scale,
                 double2* G, cudaStream_t s) {
  const int T_ = (N + AT - 1) / AT;
  k_gram<T><<<dim3(T_, T_), 256, 0, s>>>((const c_t<T>*)A, (const c_t<T>*)B, dg, n, N, scale, G);
}
template void launch_gram<double>(const void*, const void*, const double*, int, int, double, double2*, cudaStream_t);
template void launch_gram<float>(const void*, const void*, const double*, int, int, double, double2*, cudaStream_t);

__global__ void k_combine_h(int NN, const double2* T1, const double2* T2, const double2* S1,
                            const double2* S2, const double2* V1, const double2* V2,
                            const double2* W, double2* H) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NN; e += gridDim.x * blockDim.x) {
    double2 h = cadd(cmul(T1[e], S2[e]), cmul(S1[e], T2[e]));
    h = cadd(h, cadd(cmul(V1[e], S2[e]), cmul(S1[e], V2[e])));
    H[e] = cadd(h, W[e]);
  }
}
void launch_combine_h(int N, const double2* T1, const double2* T2, const double2* S1,
                      const double2* S2, const double2* V1, const double2* V2, const double2* W,
                      double2* H, cudaStream_t s) {
  const int NN = N * N;
  k_combine_h<<<(NN + 255) / 256, 256, 0, s>>>(NN, T1, T2, S1, S2, V1, V2, W, H);
}

__global__ void k_hadamard_acc(int NN, double sig, const double2* A, const double2* B, double2* W) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NN; e += gridDim.x * blockDim.x) {
    const double2 p = cmul(A[e], B[e]);
    W[e].x = fma(sig, p.x, W[e].x);
    W[e].y = fma(sig, p.y, W[e].y);
  }
}
void launch_hadamard_acc(int N, double sig, const double2* A, const double2* B, double2* W,
                         cudaStream_t s) {
  const int NN = N * N;
  k_hadamard_acc<<<(NN + 255) / 256, 256, 0, s>>>(NN, sig, A, B, W);
}

__global__ void k_to_c64(size_t n, const double2* in, float2* out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = make_float2((float)in[e].x, (float)in[e].y);
}
void launch_to_c64(size_t n, const double2* in, float2* out, cudaStream_t s) {
  size_t g = (n + 255) / 256;
  if (g > 65535) g = 65535;
  k_to_c64<<<(unsigned)g, 256, 0, s>>>(n, in, out);
}

}  // namespace icwf
