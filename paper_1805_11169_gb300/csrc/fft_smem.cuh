// In-place FFT passes over a column held in shared memory, run by all threads of a CTA (each pass
// ends with a barrier): the transforms of the CWF propagator's split-operator step and of the
// observables' kinetic energy.  Only the complex helpers of cplx.cuh and the CTA's thread index,
// size and barrier are used, so a host program can compile these passes with a one-thread
// stand-in for threadIdx, blockDim and __syncthreads (the groups of one pass are disjoint, so a
// sequential run is a valid execution).
#pragma once
#include "cplx.cuh"

namespace icwf {

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

}  // namespace icwf
