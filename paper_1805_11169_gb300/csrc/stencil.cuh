// 4-point cubic Lagrange stencils on a cell-centred uniform grid, for values and first derivatives
// at off-grid coordinates (the CWFs at trajectory positions, the potential at pinned coordinates):
// in FP64, and in FP32 for the mixed modes' velocity kernel.  Host and device code.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace icwf {

// 4-point cubic Lagrange stencil on the cell-centred grid (lo, d, n) at coordinate p:
// f(p) ~ sum_m w[m] f[i0+m], f'(p) ~ sum_m dw[m] f[i0+m]; i0 = floor(s) - 1 clamped to [0, n-4],
// s = (p - lo)/d - 1/2 the fractional cell index.
struct Stencil {
  int i0;
  double w[4];
  double dw[4];
};

__host__ __device__ __forceinline__ Stencil lagrange4(double p, double lo, double d, int n) {
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

// FP32 weights: the fractional cell index s is formed in FP64 and rounded once to FP32.
struct StencilF {
  int i0;
  float w[4];
  float dw[4];
};
__host__ __device__ __forceinline__ StencilF lagrange4f(double p, double lo, double d, int n) {
  StencilF st;
  const float s = (float)((p - lo) / d) - 0.5f;
  int i0 = (int)floorf(s) - 1;
  i0 = i0 < 0 ? 0 : (i0 > n - 4 ? n - 4 : i0);
  const float u = s - (float)i0;
  const float u1 = u - 1.f, u2 = u - 2.f, u3 = u - 3.f;
  const float inv = (float)(1.0 / d);
  st.i0 = i0;
  st.w[0] = -(u1 * u2 * u3) * (1.f / 6.f);
  st.w[1] = (u * u2 * u3) * 0.5f;
  st.w[2] = -(u * u1 * u3) * 0.5f;
  st.w[3] = (u * u1 * u2) * (1.f / 6.f);
  st.dw[0] = -((u2 * u3) + (u1 * u3) + (u1 * u2)) * (1.f / 6.f) * inv;
  st.dw[1] = ((u2 * u3) + (u * u3) + (u * u2)) * 0.5f * inv;
  st.dw[2] = -((u1 * u3) + (u * u3) + (u * u1)) * 0.5f * inv;
  st.dw[3] = ((u1 * u2) + (u * u2) + (u * u1)) * (1.f / 6.f) * inv;
  return st;
}

}  // namespace icwf
