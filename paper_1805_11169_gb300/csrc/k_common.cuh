// Device helpers shared by the ICWF kernels: complex arithmetic on float2/double2, the 4-point
// cubic Lagrange stencil, and the shared-memory radix-2 FFT passes of the CWF propagator.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "icwf_internal.h"

namespace icwf {

template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <typename T> using c_t = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ c_t<T> mk(T re, T im) {
  c_t<T> z; z.x = re; z.y = im; return z;
}
template <typename Z> __host__ __device__ __forceinline__ Z cadd(Z a, Z b) { a.x += b.x; a.y += b.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z csub(Z a, Z b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z cmul(Z a, Z b) {
  Z r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename Z> __host__ __device__ __forceinline__ Z cmulc(Z a, Z b) {
  Z r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename Z> __host__ __device__ __forceinline__ Z cconj(Z a) { a.y = -a.y; return a; }
template <typename Z, typename S> __host__ __device__ __forceinline__ Z cscale(Z a, S s) { a.x *= s; a.y *= s; return a; }
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

// Forward FFT (decimation in frequency): natural-order input in buf[0..n), bit-reversed output.
// tw[k] = exp(-2 pi i k / n), k < n/2.  All threads of the block take part.
template <typename Z>
__device__ __forceinline__ void fft_dif(Z* buf, const Z* __restrict__ tw, int n, int logn) {
  for (int s = logn - 1; s >= 0; --s) {
    const int h = 1 << s;              // butterfly span
    const int tstride = n >> (s + 1);  // twiddle step n / (2h)
    for (int idx = threadIdx.x; idx < (n >> 1); idx += blockDim.x) {
      const int j = idx & (h - 1);
      const int i1 = ((idx >> s) << (s + 1)) + j;
      const int i2 = i1 + h;
      Z u = buf[i1], v = buf[i2];
      buf[i1] = cadd(u, v);
      buf[i2] = cmul(csub(u, v), tw[j * tstride]);
    }
    __syncthreads();
  }
}

// Inverse FFT without the 1/n factor (decimation in time): bit-reversed input, natural output.
template <typename Z>
__device__ __forceinline__ void ifft_dit(Z* buf, const Z* __restrict__ tw, int n, int logn) {
  for (int s = 0; s < logn; ++s) {
    const int h = 1 << s;
    const int tstride = n >> (s + 1);
    for (int idx = threadIdx.x; idx < (n >> 1); idx += blockDim.x) {
      const int j = idx & (h - 1);
      const int i1 = ((idx >> s) << (s + 1)) + j;
      const int i2 = i1 + h;
      Z u = buf[i1];
      Z t = cmul(buf[i2], cconj(tw[j * tstride]));
      buf[i1] = cadd(u, t);
      buf[i2] = csub(u, t);
    }
    __syncthreads();
  }
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
