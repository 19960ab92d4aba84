// Device helpers shared by the ICWF kernels: complex arithmetic on float2/double2 (cplx.cuh and
// the fused multiply-adds below), the 4-point cubic Lagrange stencil, the shared-memory FFT passes
// of the CWF propagator (fft_smem.cuh), status flags and bounded waits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cplx.cuh"
#include "fft_smem.cuh"
#include "icwf_internal.h"

namespace icwf {

// acc += a * b
template <typename Z> __device__ __forceinline__ void cfma(Z& acc, Z a, Z b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename Z> __device__ __forceinline__ void cfmac(Z& acc, Z a, Z b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void sincos_t(double a, double* s, double* c) { sincos(a, s, c); }
__device__ __forceinline__ void sincos_t(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ double2 to_d(double2 z) { return z; }
__device__ __forceinline__ double2 to_d(float2 z) { return make_double2(z.x, z.y); }

// 4-point cubic Lagrange stencil on the cell-centred grid (lo, d, n) at coordinate p:
// f(p) ~ sum_m w[m] f[i0+m], f'(p) ~ sum_m dw[m] f[i0+m]; i0 = floor(s) - 1 clamped to [0, n-4],
// s = (p - lo)/d - 1/2 the fractional cell index.
struct Stencil {
  int i0;
  double w[4];
  double dw[4];
};

__device__ __forceinline__ Stencil lagrange4(double p, double lo, double d, int n) {
  Stencil st;
  double s = (p - lo) / d - 0.5;
  int i0 = (int)floor(s) - 1;
  i0 = i0 < 0 ? 0 : (i0 > n - 4 ? n - 4 : i0);
  double u = s - (double)i0;
  double u1 = u - 1.0, u2 = u - 2.0, u3 = u - 3.0;
  st.i0 = i0;
  st.w[0] = -(u1 * u2 * u3) / 6.0;
  st.w[1] = (u * u2 * u3) / 2.0;
  st.w[2] = -(u * u1 * u3) / 2.0;
  st.w[3] = (u * u1 * u2) / 6.0;
  double inv = 1.0 / d;
  st.dw[0] = -((u2 * u3) + (u1 * u3) + (u1 * u2)) / 6.0 * inv;
  st.dw[1] = ((u2 * u3) + (u * u3) + (u * u2)) / 2.0 * inv;
  st.dw[2] = -((u1 * u3) + (u * u3) + (u * u1)) / 2.0 * inv;
  st.dw[3] = ((u1 * u2) + (u * u2) + (u * u1)) / 6.0 * inv;
  return st;
}

__device__ __forceinline__ void set_flag(int* status, int bit) { atomicOr(status + STATUS_FLAGS, bit); }

// Poll budget of a spin wait on a global flag: the compiled-in default, or the handle's override
// (status word STATUS_WAITLIM, see icwf_set_wait_limit).
__device__ __forceinline__ unsigned wait_budget(const int* status, unsigned dflt) {
  const int v = *((const volatile int*)status + STATUS_WAITLIM);
  return v > 0 ? (unsigned)(v - 1) : dflt;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

}  // namespace icwf
