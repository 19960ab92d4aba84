// Double-float ("df64") arithmetic: a value is the unevaluated sum h + l of two FP32 numbers,
// |l| <= ulp(h)/2, about 48 significant bits.  Built from the error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum) and the FMA-based exact product (TwoProduct), as in
// Dekker 1971 and the GPU double-float literature (e.g. Thall 2006).
//
// Used where FP64's instruction latency or throughput would bound a dependency chain: inside the
// FP64 mode's 32 x 32 diagonal-block Cholesky (inputs and outputs FP64), and for the whole
// factorisation and triangular solves of the mixed modes (k_linalg_df.cu).  FP32 operations have
// a small fraction of the FP64 latency and ~60x its throughput on this GPU.
//
// Every operation is spelled with explicit round-to-nearest intrinsics on the device so that the
// compiler cannot contract or reassociate them (that would break the error-free transformations);
// the host build (unit tests) relies on -ffp-contract=off.
#pragma once
#include <math.h>

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

#if defined(__CUDA_ARCH__)
#define DF_ADD(a, b) __fadd_rn((a), (b))
#define DF_SUB(a, b) __fsub_rn((a), (b))
#define DF_MUL(a, b) __fmul_rn((a), (b))
#define DF_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#define DF_RSQRT(a) rsqrtf(a)
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#define DF_FMA(a, b, c) fmaf((a), (b), (c))
#define DF_RSQRT(a) (1.0f / sqrtf(a))
#endif

namespace icwf {

struct df {
  float h, l;
};

DF_HD df df_make(float h, float l) { df r; r.h = h; r.l = l; return r; }

// round-to-nearest split of a double: h = fl32(x), l = fl32(x - h)
DF_HD df df_from(double x) {
  const float h = (float)x;
  const float l = (float)(x - (double)h);
  return df_make(h, l);
}
DF_HD double df_to(df a) { return (double)a.h + (double)a.l; }

// Knuth TwoSum: s + e == a + b exactly
DF_HD df two_sum(float a, float b) {
  const float s = DF_ADD(a, b);
  const float v = DF_SUB(s, a);
  const float e = DF_ADD(DF_SUB(a, DF_SUB(s, v)), DF_SUB(b, v));
  return df_make(s, e);
}
// Dekker FastTwoSum (|a| >= |b|): s + e == a + b exactly
DF_HD df fast_two_sum(float a, float b) {
  const float s = DF_ADD(a, b);
  const float e = DF_SUB(b, DF_SUB(s, a));
  return df_make(s, e);
}

DF_HD df df_add(df a, df b) {
  df s = two_sum(a.h, b.h);
  const df t = two_sum(a.l, b.l);
  s.l = DF_ADD(s.l, t.h);
  s = fast_two_sum(s.h, s.l);
  s.l = DF_ADD(s.l, t.l);
  return fast_two_sum(s.h, s.l);
}
// a + b for an FP32 b: TwoSum of the high parts, one renormalisation (error ~2^-48 of |a + b|
// when |a.l| <= ulp(a.h) / 2)
DF_HD df df_add_f(df a, float b) {
  const df s = two_sum(a.h, b);
  return fast_two_sum(s.h, DF_ADD(s.l, a.l));
}
DF_HD df df_neg(df a) { return df_make(-a.h, -a.l); }
DF_HD df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// product: exact h*h by FMA, cross terms to FP32
DF_HD df df_mul(df a, df b) {
  const float p = DF_MUL(a.h, b.h);
  float e = DF_FMA(a.h, b.h, -p);
  e = DF_FMA(a.h, b.l, e);
  e = DF_FMA(a.l, b.h, e);
  return fast_two_sum(p, e);
}

// 1 / sqrt(a), a > 0: FP32 seed, then two Newton steps y <- y + y (1 - a y^2) / 2 in df64
DF_HD df df_rsqrt(df a) {
  df y = df_make(DF_RSQRT(a.h), 0.0f);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df r = df_sub(df_make(1.0f, 0.0f), df_mul(a, df_mul(y, y)));
    y = df_add(y, df_mul(df_make(DF_MUL(0.5f, y.h), DF_MUL(0.5f, y.l)), r));
  }
  return y;
}

// 1 / sqrt(a), a > 0, from an FP32 estimate y0 with relative error |r0| << 1: one correction
// y = y0 (1 + r/2 + 3 r^2/8), r = 1 - a y0^2, which is the binomial series of y0 (1 - r)^(-1/2)
// cut after the r^2 term, so the relative error is O(r^3).  r is formed from exact products
// (1 - t is exact for t in [1/2, 2] by Sterbenz' lemma), so it carries ~46 correct bits.
DF_HD df df_rsqrt_refine(df a, float y0) {
  const float p = DF_MUL(y0, y0);
  const float pe = DF_FMA(y0, y0, -p);       // y0^2 = p + pe exactly
  const float t = DF_MUL(a.h, p);
  const float te = DF_FMA(a.h, p, -t);       // a.h p = t + te exactly
  // the three small terms (each ~2^-24) first, so that r is rounded once
  const float r = DF_SUB(DF_SUB(1.0f, t), DF_FMA(a.h, pe, DF_FMA(a.l, p, te)));
  const float corr = DF_MUL(y0, DF_MUL(r, DF_FMA(0.375f, r, 0.5f)));
  return fast_two_sum(y0, corr);
}
DF_HD df df_rsqrt1(df a) { return df_rsqrt_refine(a, DF_RSQRT(a.h)); }

// Addition without the second renormalisation: the error is bounded relative to |a| + |b|
// (not |a + b|), which is all a normwise backward-stable factorisation needs.
DF_HD df df_add_sloppy(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, DF_ADD(s.l, DF_ADD(a.l, b.l)));
}

// complex double-float
struct cdf {
  df re, im;
};
DF_HD cdf cdf_make(df re, df im) { cdf z; z.re = re; z.im = im; return z; }
DF_HD cdf cdf_add(cdf a, cdf b) { return cdf_make(df_add(a.re, b.re), df_add(a.im, b.im)); }
DF_HD cdf cdf_sub(cdf a, cdf b) { return cdf_make(df_sub(a.re, b.re), df_sub(a.im, b.im)); }
DF_HD cdf cdf_scale(cdf a, df s) { return cdf_make(df_mul(a.re, s), df_mul(a.im, s)); }
DF_HD cdf cdf_mul(cdf a, cdf b) {
  return cdf_make(df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)),
                  df_add(df_mul(a.re, b.im), df_mul(a.im, b.re)));
}
// a * conj(b)
DF_HD cdf cdf_mul_conj(cdf a, cdf b) {
  return cdf_make(df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)),
                  df_sub(df_mul(a.im, b.re), df_mul(a.re, b.im)));
}

}  // namespace icwf
