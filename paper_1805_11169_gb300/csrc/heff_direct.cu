// icwf_heff_direct: columns of Heff = W - W1 - W2 (Eq. W, W1, W2) by the full double sum over the
// grid, without the rank-k factorisation of the interaction:
//   Heff[a, b] = dx dR sum_i sum_j conj(psi_a(x_i) chi_a(R_j)) D_b(i, j) psi_b(x_i) chi_b(R_j),
//   D_b(i, j) = V(x_i, R_j) - V(x_i, R_b) - V(x_b, R_j),
// the pinned values interpolated from the table with the same 4-point stencil the step uses.
// It is the O(N nx nR)-per-column reference against which the factorised assembly's truncation
// (and, in the mixed modes, rounding) error is reported.  All arithmetic is FP64; the CWFs are
// read in their storage precision and promoted.
//
// Kernels: k_hd_pinned (V(x_i, R_b) and V(x_b, R_j) per requested column), k_hd_tile (one CTA per
// 64 grid points x_i, 64 bras a and one column b: the inner sum over R_j as a tiled real-by-complex
// product staged in shared memory, then the x_i weights conj(psi_a) psi_b and a fixed-order
// reduction over the CTA's x_i), k_hd_final (fixed-order sum over the x_i tiles).  The result does
// not depend on scheduling.
#include <cuda_runtime.h>

#include <vector>

#include "icwf_internal.h"
#include "k_common.cuh"

namespace icwf {
namespace {

constexpr int HD_TI = 64;   // grid points x_i per CTA
constexpr int HD_TA = 64;   // bras a per CTA
constexpr int HD_JC = 16;   // R_j per shared-memory stage

__global__ void k_hd_pinned(JobView j, const int* __restrict__ cols, double* __restrict__ Ve,
                            double* __restrict__ Vn) {
  const int m = blockIdx.x;
  const int b = cols[m];
  const Stencil sR = lagrange4(j.R[b], j.R_min, j.dR, j.nR);
  const Stencil sx = lagrange4(j.x[b], j.x_min, j.dx, j.nx);
  for (int i = threadIdx.x; i < j.nx; i += blockDim.x) {
    const double* v = j.V + (size_t)i * j.nR + sR.i0;
    Ve[(size_t)m * j.nx + i] = sR.w[0] * v[0] + sR.w[1] * v[1] + sR.w[2] * v[2] + sR.w[3] * v[3];
  }
  for (int jj = threadIdx.x; jj < j.nR; jj += blockDim.x) {
    const double* v = j.V + (size_t)sx.i0 * j.nR + jj;
    Vn[(size_t)m * j.nR + jj] = sx.w[0] * v[0] + sx.w[1] * v[j.nR] + sx.w[2] * v[2 * j.nR] +
                                sx.w[3] * v[3 * j.nR];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_hd_tile(JobView j, const int* __restrict__ cols,
                                                 const double* __restrict__ Ve,
                                                 const double* __restrict__ Vn,
                                                 double2* __restrict__ partial) {
  __shared__ double Ds[HD_TI][HD_JC + 1];
  __shared__ double2 Ws[HD_JC * HD_TA];      // also the reduction buffer (16 x 64) at the end
  const int it = blockIdx.x, at = blockIdx.y, m = blockIdx.z;
  const int nit = gridDim.x;
  const int b = cols[m];
  const int N = j.N, nx = j.nx, nR = j.nR;
  const int i0 = it * HD_TI, a0 = at * HD_TA;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const c_t<T>* psi = (const c_t<T>*)j.psi;
  const c_t<T>* chi = (const c_t<T>*)j.chi;
  const double* ve = Ve + (size_t)m * nx;
  const double* vn = Vn + (size_t)m * nR;
  double2 z[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) z[r][c] = make_double2(0.0, 0.0);
  for (int j0 = 0; j0 < nR; j0 += HD_JC) {
    // D_b(i, j) for the CTA's 64 x 16 block (zero outside the grid)
    for (int e = tid; e < HD_TI * HD_JC; e += 256) {
      const int ii = e / HD_JC, jj = e % HD_JC;
      const int i = i0 + ii, jg = j0 + jj;
      Ds[ii][jj] = (i < nx && jg < nR) ? j.V[(size_t)i * nR + jg] - ve[i] - vn[jg] : 0.0;
    }
    // w(j, a) = conj(chi_a(R_j)) chi_b(R_j) (zero outside)
    for (int e = tid; e < HD_JC * HD_TA; e += 256) {
      const int jj = e / HD_TA, aa = e % HD_TA;
      const int jg = j0 + jj, a = a0 + aa;
      double2 w = make_double2(0.0, 0.0);
      if (jg < nR && a < N)
        w = cmulc(to_d(chi[(size_t)a * nR + jg]), to_d(chi[(size_t)b * nR + jg]));
      Ws[jj * HD_TA + aa] = w;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < HD_JC; ++jj) {
      double d[4];
      double2 w[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) d[r] = Ds[ty + 16 * r][jj];
#pragma unroll
      for (int c = 0; c < 4; ++c) w[c] = Ws[jj * HD_TA + tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          z[r][c].x = fma(d[r], w[c].x, z[r][c].x);
          z[r][c].y = fma(d[r], w[c].y, z[r][c].y);
        }
    }
    __syncthreads();
  }
  // x_i weights conj(psi_a(x_i)) psi_b(x_i); sum over this thread's four x_i, then over ty
  double2 acc[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c] = make_double2(0.0, 0.0);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= nx) continue;
    const double2 pb = to_d(psi[(size_t)b * nx + i]);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int a = a0 + tx + 16 * c;
      if (a >= N) continue;
      const double2 wa = cmulc(to_d(psi[(size_t)a * nx + i]), pb);
      acc[c] = cadd(acc[c], cmul(wa, z[r][c]));
    }
  }
  double2* red = Ws;   // [16][64]
#pragma unroll
  for (int c = 0; c < 4; ++c) red[ty * HD_TA + tx + 16 * c] = acc[c];
  __syncthreads();
  if (tid < HD_TA && a0 + tid < N) {
    double2 s = make_double2(0.0, 0.0);
    for (int y = 0; y < 16; ++y) s = cadd(s, red[y * HD_TA + tid]);
    partial[((size_t)m * nit + it) * N + a0 + tid] = s;
  }
}

__global__ void k_hd_final(int N, int M, int nit, double scale, const double2* __restrict__ partial,
                           double2* __restrict__ out) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)M * N) return;
  const int m = (int)(e / N), a = (int)(e % N);
  double2 s = make_double2(0.0, 0.0);
  for (int t = 0; t < nit; ++t) s = cadd(s, partial[((size_t)m * nit + t) * N + a]);
  out[e] = make_double2(scale * s.x, scale * s.y);
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace icwf

extern "C" icwf_status icwf_heff_direct(icwf_handle h, int32_t n_cols, const int32_t* cols,
                                        double* out) {
  using namespace icwf;
  ObsView v;
  if (!h || !handle_obs_view(h, &v)) {
    handle_set_error(nullptr, "icwf_heff_direct: NULL handle");
    return ICWF_ERR_ARG;
  }
  if (!v.initialised) {
    handle_set_error(h, "icwf_heff_direct: handle not initialised");
    return ICWF_ERR_STATE;
  }
  const JobView& j = v.j;
  if (n_cols < 1 || n_cols > j.N || !cols || !out) {
    handle_set_error(h, "icwf_heff_direct: need 1 <= n_cols <= N and non-NULL cols and out");
    return ICWF_ERR_ARG;
  }
  for (int m = 0; m < n_cols; ++m)
    if (cols[m] < 0 || cols[m] >= j.N) {
      handle_set_error(h, "icwf_heff_direct: column index out of range");
      return ICWF_ERR_ARG;
    }
  const int M = n_cols;
  const int nit = (j.nx + HD_TI - 1) / HD_TI;
  const size_t b_cols = up256((size_t)M * 4), b_ve = up256((size_t)M * j.nx * 8),
               b_vn = up256((size_t)M * j.nR * 8), b_part = up256((size_t)M * nit * j.N * 16),
               b_out = up256((size_t)M * j.N * 16);
  cudaStream_t s = v.stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    handle_set_error(h, "icwf_heff_direct: stream synchronisation failed");
    return ICWF_ERR_CUDA;
  }
  char* work = nullptr;
  if (cudaMalloc(&work, b_cols + b_ve + b_vn + b_part + b_out) != cudaSuccess) {
    handle_set_error(h, "icwf_heff_direct: cudaMalloc failed");
    return ICWF_ERR_OOM;
  }
  int* dcols = (int*)work;
  double* Ve = (double*)(work + b_cols);
  double* Vn = (double*)(work + b_cols + b_ve);
  double2* part = (double2*)(work + b_cols + b_ve + b_vn);
  double2* dout = (double2*)(work + b_cols + b_ve + b_vn + b_part);
  bool ok = cudaMemcpyAsync(dcols, cols, (size_t)M * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (ok) {
    k_hd_pinned<<<M, 256, 0, s>>>(j, dcols, Ve, Vn);
    const dim3 grid(nit, (j.N + HD_TA - 1) / HD_TA, M);
    if (v.mixed) k_hd_tile<float><<<grid, 256, 0, s>>>(j, dcols, Ve, Vn, part);
    else k_hd_tile<double><<<grid, 256, 0, s>>>(j, dcols, Ve, Vn, part);
    const size_t n = (size_t)M * j.N;
    k_hd_final<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(j.N, M, nit, j.dx * j.dR, part, dout);
    ok = cudaPeekAtLastError() == cudaSuccess &&
         cudaMemcpyAsync(out, dout, n * 16, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
  }
  cudaFree(work);
  if (!ok) {
    handle_set_error(h, "icwf_heff_direct: a CUDA call failed");
    return ICWF_ERR_CUDA;
  }
  return ICWF_OK;
}
