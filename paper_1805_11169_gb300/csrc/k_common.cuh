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
// The radix-2 stages s = logn-1, ..., 0 (span 2^s) are taken two at a time: the four elements
// i0, i0 + h/2, i0 + h, i0 + 3h/2 (h = 2^s) that stages s and s-1 combine stay in one thread's
// registers between the two, so a pair of stages costs one pass over shared memory and one
// barrier; each element sees the same operations as in separate radix-2 passes.  An odd last
// stage (span 1) runs alone.
template <typename Z>
__device__ __forceinline__ void fft_dif(Z* buf, const Z* __restrict__ tw, int n, int logn) {
  int s = logn - 1;
  for (; s >= 1; s -= 2) {
    const int h = 1 << s, q = h >> 1;
    const int ts1 = n >> (s + 1);   // twiddle step of stage s:     n / (2h)
    const int ts0 = n >> s;         // twiddle step of stage s - 1: n / h
    for (int g = threadIdx.x; g < (n >> 2); g += blockDim.x) {
      const int j = g & (q - 1);
      const int i0 = ((g >> (s - 1)) << (s + 1)) + j;
      const int i1 = i0 + q, i2 = i0 + h, i3 = i2 + q;
      const Z a0 = buf[i0], a1 = buf[i1], a2 = buf[i2], a3 = buf[i3];
      // stage s: pairs (i0, i2), (i1, i3) with twiddle indices j, j + q
      const Z b0 = cadd(a0, a2), b2 = cmul(csub(a0, a2), tw[j * ts1]);
      const Z b1 = cadd(a1, a3), b3 = cmul(csub(a1, a3), tw[(j + q) * ts1]);
      // stage s - 1: pairs (i0, i1), (i2, i3), both with twiddle index j
      const Z w = tw[j * ts0];
      buf[i0] = cadd(b0, b1);
      buf[i1] = cmul(csub(b0, b1), w);
      buf[i2] = cadd(b2, b3);
      buf[i3] = cmul(csub(b2, b3), w);
    }
    __syncthreads();
  }
  if (s == 0) {
    for (int idx = threadIdx.x; idx < (n >> 1); idx += blockDim.x) {
      const Z u = buf[2 * idx], v = buf[2 * idx + 1];
      buf[2 * idx] = cadd(u, v);
      buf[2 * idx + 1] = cmul(csub(u, v), tw[0]);
    }
    __syncthreads();
  }
}

// Inverse FFT without the 1/n factor (decimation in time): bit-reversed input, natural output.
// Stages s = 0, ..., logn-1 (span 2^s) two at a time as in fft_dif: stages s and s+1 combine the
// elements i0, i0 + h, i0 + 2h, i0 + 3h (h = 2^s); an odd last stage runs alone.
template <typename Z>
__device__ __forceinline__ void ifft_dit(Z* buf, const Z* __restrict__ tw, int n, int logn) {
  int s = 0;
  for (; s + 1 < logn; s += 2) {
    const int h = 1 << s;
    const int ts0 = n >> (s + 1);   // twiddle step of stage s:     n / (2h)
    const int ts1 = n >> (s + 2);   // twiddle step of stage s + 1: n / (4h)
    for (int g = threadIdx.x; g < (n >> 2); g += blockDim.x) {
      const int j = g & (h - 1);
      const int i0 = ((g >> s) << (s + 2)) + j;
      const int i1 = i0 + h, i2 = i0 + 2 * h, i3 = i2 + h;
      const Z a0 = buf[i0], a1 = buf[i1], a2 = buf[i2], a3 = buf[i3];
      // stage s: pairs (i0, i1), (i2, i3), both with twiddle index j
      const Z w = cconj(tw[j * ts0]);
      const Z t1 = cmul(a1, w), t3 = cmul(a3, w);
      const Z b0 = cadd(a0, t1), b1 = csub(a0, t1);
      const Z b2 = cadd(a2, t3), b3 = csub(a2, t3);
      // stage s + 1: pairs (i0, i2), (i1, i3) with twiddle indices j, j + h
      const Z u2 = cmul(b2, cconj(tw[j * ts1]));
      const Z u3 = cmul(b3, cconj(tw[(j + h) * ts1]));
      buf[i0] = cadd(b0, u2);
      buf[i2] = csub(b0, u2);
      buf[i1] = cadd(b1, u3);
      buf[i3] = csub(b1, u3);
    }
    __syncthreads();
  }
  if (s < logn) {
    const int h = 1 << s;
    const int tstride = n >> (s + 1);
    for (int idx = threadIdx.x; idx < (n >> 1); idx += blockDim.x) {
      const int j = idx & (h - 1);
      const int i1 = ((idx >> s) << (s + 1)) + j;
      const int i2 = i1 + h;
      const Z u = buf[i1];
      const Z t = cmul(buf[i2], cconj(tw[j * tstride]));
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
