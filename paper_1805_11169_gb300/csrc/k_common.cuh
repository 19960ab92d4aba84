// Device helpers shared by the ICWF kernels: complex arithmetic on float2/double2 (cplx.cuh and
// the fused multiply-adds below), the 4-point cubic Lagrange stencils (stencil.cuh), the
// shared-memory FFT passes of the CWF propagator (fft_smem.cuh), status flags and bounded waits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cplx.cuh"
#include "fft_smem.cuh"
#include "stencil.cuh"
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
