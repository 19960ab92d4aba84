// Digit planes of the emulated-FP64 trailing update (k_herk_emu.cu), shared by the kernels that
// produce panel rows (the FP64 panel solve writes them as it finishes a row).
//
// A panel row i (32 complex FP64 values) with max |component| < 2^e_i becomes, per component, the
// 64-bit integer X = round(x 2^(63 - e_i)) (integer operations on the FP64 bit pattern), cut from
// the top into seven balanced base-2^8 digits d_1..d_7 (|d_1| <= 256, |d_p| <= 128 after); digit p
// is stored as the exact BF16 value d_p 2^(-8 (p-1)) in four planes (P, -Q, Q, P for the real part
// P and imaginary part Q): planes[((p * 4 + pi) * rpad + i) * 32 + k].
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace icwf {
namespace hemu {

constexpr int NB = 32;                 // block size of the factorisation (panel width = K)
constexpr int DIG = 7;                 // digits per component
constexpr int BETA = 8;                // digit base 2^8
constexpr int PLANES = 4;              // P, -Q, Q, P

// round(|x| 2^(63 - e)) for |x| < 2^e, from the FP64 bit pattern with integer operations only.
__device__ __forceinline__ unsigned long long fixed63(unsigned long long u, int e) {
  const int E = (int)((u >> 52) & 0x7FFu);
  const unsigned long long frac = u & 0xFFFFFFFFFFFFFull;
  const unsigned long long mant = E ? (frac | (1ull << 52)) : frac;   // |x| = mant 2^p2
  const int p2 = E ? E - 1075 : -1074;
  const int s = p2 + 63 - e;              // <= 10 since |x| < 2^e
  if (s >= 0) return mant << s;
  if (s <= -54) return 0;                 // below half a unit
  return (mant + (1ull << (-s - 1))) >> (-s);
}

// Exponent e with max|x| < 2^e (e = 0 for an all-zero row) from the largest |x|'s bit pattern.
__device__ __forceinline__ int row_exponent(unsigned long long mbits) {
  const int E = (int)(mbits >> 52);
  if (E) return E - 1022;
  return mbits ? -1074 + (64 - __clzll((long long)mbits)) : 0;
}

// Called by a full warp, lane = column k, z = L_i,k: writes row i's digit planes and e_i.
__device__ __forceinline__ void emit_row_digits(double2 z, int i, int lane, int rpad,
                                                __nv_bfloat16* __restrict__ planes,
                                                int* __restrict__ ex) {
  const unsigned long long ur = (unsigned long long)__double_as_longlong(z.x);
  const unsigned long long ui = (unsigned long long)__double_as_longlong(z.y);
  const unsigned long long ABS = 0x7FFFFFFFFFFFFFFFull;
  // magnitudes of non-negative doubles order like their bit patterns
  unsigned long long mb = (ur & ABS) > (ui & ABS) ? (ur & ABS) : (ui & ABS);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, mb, off);
    mb = o > mb ? o : mb;
  }
  const int e = row_exponent(mb);
  if (lane == 0) ex[i] = e;
  // signed fixed-point values X = round(x 2^(63 - e)), |X| <= 2^63 - 2^10
  long long xr = (long long)fixed63(ur & ABS, e), xi = (long long)fixed63(ui & ABS, e);
  if (ur >> 63) xr = -xr;
  if (ui >> 63) xi = -xi;
  const size_t pl = (size_t)rpad * NB;
#pragma unroll
  for (int p = 0; p < DIG; ++p) {
    const int sh = 55 - BETA * p;         // digit p weighs 2^sh units of 2^(e - 63)
    // balanced digit: round half up of X / 2^sh, then X -= d 2^sh (the remainder is at most
    // 2^(sh - 1) in magnitude, so the unsigned wrap-around leaves it exact)
    const long long dr = ((xr >> (sh - 1)) + 1) >> 1, di = ((xi >> (sh - 1)) + 1) >> 1;
    xr = (long long)((unsigned long long)xr - ((unsigned long long)dr << sh));
    xi = (long long)((unsigned long long)xi - ((unsigned long long)di << sh));
    const float w = __int_as_float((127 - BETA * p) << 23);   // 2^(-8 p), exact
    const float fr = (float)dr * w, fi = (float)di * w;
    const size_t base = (size_t)(p * PLANES) * pl + (size_t)i * NB + lane;
    planes[base] = __float2bfloat16_rn(fr);            // P
    planes[base + pl] = __float2bfloat16_rn(-fi);      // -Q
    planes[base + 2 * pl] = __float2bfloat16_rn(fi);   // Q
    planes[base + 3 * pl] = __float2bfloat16_rn(fr);   // P
  }
}

}  // namespace hemu
}  // namespace icwf
