// FP64 linear algebra of the coefficient update (Eq. coeff, S dC/dt = -i Heff C): the
// Tikhonov-shifted overlap S + eps I, its blocked Cholesky factorisation, the two triangular
// solves, the Heff matrix-vector products of the RK4 stages and the final RK4 combination.
// All arithmetic is FP64 in every precision mode (S is near-singular as CWFs overlap).
#include <cuda_runtime.h>

#include "icwf_internal.h"
#include "k_common.cuh"

namespace icwf {

constexpr int NB = 32;                 // block size of the factorisation and of the solves
constexpr unsigned WAIT_LIMIT = 1u << 22;   // bounded spin (x ~64 ns sleep: well under 1 s)

// ------------------------------------------------------------------------------ S + eps I

__global__ void k_shift_mix(int N, const double2* __restrict__ S0, const double2* __restrict__ S1,
                            double eps, double theta, double2* __restrict__ A) {
  const size_t NN = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < NN;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / N, c = e % N;
    double2 v;
    if (theta == 1.0) {
      v = S1[e];
    } else if (theta == 0.0) {
      v = S0[e];
    } else {
      v = make_double2(0.5 * (S0[e].x + S1[e].x), 0.5 * (S0[e].y + S1[e].y));
    }
    if (r == c) v.x += eps;
    A[e] = v;
  }
}

void launch_shift_mix(int N, const double2* S0, const double2* S1, double eps, double theta,
                      double2* A, cudaStream_t s) {
  const size_t NN = (size_t)N * N;
  size_t g = (NN + 255) / 256;
  if (g > 4096) g = 4096;
  k_shift_mix<<<(unsigned)g, 256, 0, s>>>(N, S0, S1, eps, theta, A);
}

// ------------------------------------------------------------------------------ Cholesky

struct MatBatch { double2* m[2]; double* inv[2]; double2* D[2]; };

// Factor the diagonal block jb of each matrix: one warp per matrix, lane r holds row r of the
// block in registers.  Column c: pivot d = A_cc, 1/sqrt(d) by rsqrt, L_cc = d * rsqrt(d);
// L_rc *= rsqrt(d) for r > c; rank-1 update of the trailing block with column c broadcast by
// shuffles.  The reciprocal pivots are stored for the panel and triangular solves.  Rows and
// columns beyond N are treated as identity so that ragged sizes factor cleanly.
__global__ void __launch_bounds__(32) k_potrf_diag(int N, MatBatch mb, int jb, int* status) {
  double2* A = mb.m[blockIdx.y];
  double* inv = mb.inv[blockIdx.y];
  const int r = threadIdx.x;
  const int r0 = jb * NB;
  const bool rok = r0 + r < N;
  double2 L[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    double2 v = make_double2(c == r ? 1.0 : 0.0, 0.0);
    if (rok && r0 + c < N && c <= r) v = A[(size_t)(r0 + r) * N + r0 + c];
    L[c] = v;
  }
  double my_inv = 1.0;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    double dinv = 0.0;
    if (r == c) {
      double d = L[c].x;
      if (!(d > 0.0)) { set_flag(status, ST_CHOL); d = 1.0; }
      dinv = rsqrt(d);
      L[c] = make_double2(d * dinv, 0.0);
      my_inv = dinv;
    }
    dinv = __shfl_sync(0xffffffffu, dinv, c);
    if (r > c) L[c] = cscale(L[c], dinv);
#pragma unroll
    for (int q = c + 1; q < NB; ++q) {
      double2 lq;
      lq.x = __shfl_sync(0xffffffffu, L[c].x, q);
      lq.y = __shfl_sync(0xffffffffu, L[c].y, q);
      if (r >= q) {
        // L[r][q] -= L[r][c] * conj(L[q][c])
        L[q].x -= L[c].x * lq.x + L[c].y * lq.y;
        L[q].y -= L[c].y * lq.x - L[c].x * lq.y;
      }
    }
  }
  if (rok) {
#pragma unroll
    for (int c = 0; c < NB; ++c)
      if (c <= r && r0 + c < N) A[(size_t)(r0 + r) * N + r0 + c] = L[c];
    inv[r0 + r] = my_inv;
  }
}

constexpr int TR_WARPS = 8;   // rows per panel-solve CTA

// Panel solve A_ib <- A_ib L_bb^-H below the diagonal block jb: one warp per row, lane = column.
// Column-oriented substitution: x_m = a_m / L_mm, then a_c -= x_m conj(L_cm) for c > m.
__global__ void __launch_bounds__(TR_WARPS * 32) k_trsm_panel(int N, MatBatch mb, int jb) {
  __shared__ double2 Ls[NB][NB + 1];
  __shared__ double invs[NB];
  double2* A = mb.m[blockIdx.y];
  const double* inv = mb.inv[blockIdx.y];
  const int c0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    double2 l = make_double2(0.0, 0.0);
    if (c < r && c0 + r < N && c0 + c < N) l = A[(size_t)(c0 + r) * N + c0 + c];
    Ls[r][c] = l;
  }
  if (threadIdx.x < NB) invs[threadIdx.x] = (c0 + threadIdx.x < N) ? inv[c0 + threadIdx.x] : 1.0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = (jb + 1) * NB + blockIdx.x * TR_WARPS + warp;
  if (row >= N) return;
  const bool cok = c0 + lane < N;
  double2 a = cok ? A[(size_t)row * N + c0 + lane] : make_double2(0.0, 0.0);
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    double2 x = cscale(a, invs[m]);
    x.x = __shfl_sync(0xffffffffu, x.x, m);
    x.y = __shfl_sync(0xffffffffu, x.y, m);
    if (lane == m) a = x;
    else if (lane > m) {
      const double2 l = Ls[lane][m];
      a.x -= x.x * l.x + x.y * l.y;   // a -= x conj(l)
      a.y -= x.y * l.x - x.x * l.y;
    }
  }
  if (cok) A[(size_t)row * N + c0 + lane] = a;
}

// Inverse of every diagonal block after the factorisation: D_b = L_bb^-1 (lower triangular,
// 32 x 32), stored row-major per block in D[(b*32 + r)*32 + c].  One warp per block, lane = column
// c of D: D_rc = (delta_rc - sum_{c<=m<r} L_rm D_mc) / L_rr for r >= c.  The triangular solves use
// these blocks as matrix-vector products, which keeps the dependent substitution chain off their
// critical path.
__global__ void __launch_bounds__(32) k_trtri_diag(int N, MatBatch mb) {
  __shared__ double2 Ls[NB][NB + 1];
  __shared__ double invs[NB];
  const double2* A = mb.m[blockIdx.y];
  const double* inv = mb.inv[blockIdx.y];
  double2* D = mb.D[blockIdx.y];
  const int jb = blockIdx.x, r0 = jb * NB, c = threadIdx.x;
  for (int r = 0; r < NB; ++r) {
    double2 l = make_double2(r == c ? 1.0 : 0.0, 0.0);
    if (c < r && r0 + r < N && r0 + c < N) l = A[(size_t)(r0 + r) * N + r0 + c];
    Ls[r][c] = l;
  }
  invs[c] = (r0 + c < N) ? inv[r0 + c] : 1.0;
  __syncwarp();
  double2 d[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    double2 acc = make_double2(r == c ? 1.0 : 0.0, 0.0);
#pragma unroll
    for (int m = 0; m < r; ++m) {
      // only m >= c contributes (D_mc = 0 for m < c); the loop stays uniform across lanes
      const double2 l = Ls[r][m];
      acc.x -= l.x * d[m].x - l.y * d[m].y;
      acc.y -= l.x * d[m].y + l.y * d[m].x;
    }
    d[r] = (r >= c) ? cscale(acc, invs[r]) : make_double2(0.0, 0.0);
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r0 + r < N) D[((size_t)jb * NB + r) * NB + c] = d[r];
}

__device__ __forceinline__ void tri_index_l(int t, int& I, int& J) {
  int Jc = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (Jc * (Jc + 1) / 2 > t) --Jc;
  while ((Jc + 1) * (Jc + 2) / 2 <= t) ++Jc;
  J = Jc;
  I = t - Jc * (Jc + 1) / 2;
}

// Trailing update A_rc -= L_rb L_cb^H for jb < c <= r (one CTA per lower tile).
__global__ void __launch_bounds__(256) k_herk_update(int N, MatBatch mb, int jb) {
  __shared__ double2 Lr[NB][NB + 1];
  __shared__ double2 Lc[NB][NB + 1];
  double2* A = mb.m[blockIdx.y];
  int I, J;
  tri_index_l(blockIdx.x, I, J);
  const int cb = jb + 1 + I, rb = jb + 1 + J;   // cb <= rb
  const int k0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, m = e % NB;
    double2 a = make_double2(0, 0), b = a;
    if (rb * NB + r < N && k0 + m < N) a = A[(size_t)(rb * NB + r) * N + k0 + m];
    if (cb * NB + r < N && k0 + m < N) b = A[(size_t)(cb * NB + r) * N + k0 + m];
    Lr[r][m] = a;
    Lc[r][m] = b;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const double2 z = make_double2(0, 0);
  double2 acc[2][2] = {{z, z}, {z, z}};
#pragma unroll 8
  for (int m = 0; m < NB; ++m) {
    const double2 a0 = Lr[ty][m], a1 = Lr[ty + 16][m];
    const double2 b0 = Lc[tx][m], b1 = Lc[tx + 16][m];
    // acc += a * conj(b)
    cfmac(acc[0][0], b0, a0); cfmac(acc[0][1], b1, a0);
    cfmac(acc[1][0], b0, a1); cfmac(acc[1][1], b1, a1);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int gr = rb * NB + ty + 16 * r, gc = cb * NB + tx + 16 * c;
      if (gr < N && gc < N && gc <= gr) {
        double2* p = A + (size_t)gr * N + gc;
        // conj(b) * a computed by cfmac(b, a) = conj(b)*a; we need a * conj(b): same value.
        p->x -= acc[r][c].x;
        p->y -= acc[r][c].y;
      }
    }
}

int launch_cholesky(int N, double2* const* A, double* const* inv, double2* const* D, int nbatch,
                    int* status, cudaStream_t s) {
  MatBatch mb;
  mb.m[0] = A[0];
  mb.m[1] = nbatch > 1 ? A[1] : A[0];
  mb.inv[0] = inv[0];
  mb.inv[1] = nbatch > 1 ? inv[1] : inv[0];
  mb.D[0] = D[0];
  mb.D[1] = nbatch > 1 ? D[1] : D[0];
  const int T = (N + NB - 1) / NB;
  int launches = 0;
  for (int jb = 0; jb < T; ++jb) {
    k_potrf_diag<<<dim3(1, nbatch), 32, 0, s>>>(N, mb, jb, status);
    ++launches;
    const int rest = T - jb - 1;
    if (rest > 0) {
      const int rows = N - (jb + 1) * NB;
      k_trsm_panel<<<dim3((rows + TR_WARPS - 1) / TR_WARPS, nbatch), TR_WARPS * 32, 0, s>>>(N, mb, jb);
      k_herk_update<<<dim3(rest * (rest + 1) / 2, nbatch), 256, 0, s>>>(N, mb, jb);
      launches += 2;
    }
  }
  k_trtri_diag<<<dim3(T, nbatch), 32, 0, s>>>(N, mb);
  return launches + 1;
}

// ------------------------------------------------------------------------------ matvec

// y_a = sum_b ((1-theta) H0 + theta H1)_ab (C_b + c kp_b); one warp per row.
__global__ void __launch_bounds__(256) k_matvec(int N, const double2* __restrict__ H0,
                                                const double2* __restrict__ H1, double theta,
                                                const double2* __restrict__ C,
                                                const double2* __restrict__ kp, double c,
                                                double2* __restrict__ y) {
  const int a = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (a >= N) return;
  double2 acc = make_double2(0, 0);
  const double2* h0 = H0 + (size_t)a * N;
  const double2* h1 = H1 + (size_t)a * N;
  for (int b = lane; b < N; b += 32) {
    double2 v = C[b];
    if (kp) { const double2 k = kp[b]; v.x += c * k.x; v.y += c * k.y; }
    double2 h;
    if (theta == 0.0) h = h0[b];
    else if (theta == 1.0) h = h1[b];
    else h = make_double2(0.5 * (h0[b].x + h1[b].x), 0.5 * (h0[b].y + h1[b].y));
    cfma(acc, h, v);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  if (lane == 0) y[a] = acc;
}

void launch_matvec(int N, const double2* H0, const double2* H1, double theta, const double2* C,
                   const double2* kp, double c, double2* y, cudaStream_t s) {
  k_matvec<<<(N + 7) / 8, 256, 0, s>>>(N, H0, H1, theta, C, kp, c, y);
}

// ------------------------------------------------------------------------------ triangular solves

__device__ __forceinline__ bool wait_flag(const unsigned* f, unsigned epoch, int* status) {
  for (unsigned it = 0; it < WAIT_LIMIT; ++it) {
    if (ld_acquire(f) == epoch) return true;
    if (it > 4096) __nanosleep(64);   // pure spin first: the expected wait is a few microseconds
  }
  set_flag(status, ST_TIMEOUT);
  return false;
}

constexpr int TW = 8;   // warps per triangular-solve CTA

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Forward solve L z = y with the inverted diagonal blocks D_b = L_bb^-1:
//   z_b = D_b (y_b - sum_{m<b} L_bm z_m).
// CTAs take block rows in ticket order (a CTA only waits on block rows with smaller tickets,
// which are already running or done).  Warp 0 owns the critical product with block b-1 and the
// diagonal product; warps 1.. take the older blocks.  Lane r holds row r; matrix entries are
// loaded into registers before the wait so that only shuffles and FMAs follow the flag.
__global__ void __launch_bounds__(TW * 32) k_trsv_lower(int N, const double2* __restrict__ L,
                                                       const double2* __restrict__ D,
                                                       const double2* __restrict__ y,
                                                       double2* __restrict__ z, unsigned* flags,
                                                       unsigned* ticket, unsigned epoch,
                                                       int* status) {
  __shared__ double2 part[TW][NB];
  __shared__ double2 Ds[NB][NB + 1];
  __shared__ int s_jb;
  if (threadIdx.x == 0) s_jb = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int jb = s_jb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    Ds[r][c] = (r0 + r < N) ? D[((size_t)jb * NB + r) * NB + c] : make_double2(0, 0);
  }
  const bool row_ok = r0 + lane < N;
  const double2* Lrow = L + (size_t)(row_ok ? r0 + lane : 0) * N;
  double2 acc = make_double2(0, 0);
  // warps 1..TW-1: blocks m = 0 .. jb-2, round robin
  for (int m = warp - 1; warp > 0 && m < jb - 1; m += TW - 1) {
    double2 lv[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) lv[c] = __ldg(Lrow + m * NB + c);
    if (lane == 0) wait_flag(flags + m, epoch, status);
    __syncwarp();
    const double2 zm = __ldcg(z + m * NB + lane);
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 zc;
      zc.x = __shfl_sync(0xffffffffu, zm.x, c);
      zc.y = __shfl_sync(0xffffffffu, zm.y, c);
      cfma(acc, lv[c], zc);
    }
  }
  if (warp > 0) part[warp][lane] = row_ok ? acc : make_double2(0, 0);
  __syncthreads();
  if (warp != 0) return;
  // warp 0: prefetch the critical block (jb-1), then wait for z_{jb-1}
  double2 lv[NB];
  const int mc = jb - 1;
#pragma unroll
  for (int c = 0; c < NB; ++c) lv[c] = (mc >= 0) ? __ldg(Lrow + mc * NB + c) : make_double2(0, 0);
  double2 v = row_ok ? y[r0 + lane] : make_double2(0, 0);
  for (int w = 1; w < TW; ++w) v = csub(v, part[w][lane]);
  if (mc >= 0) {
    if (lane == 0) wait_flag(flags + mc, epoch, status);
    __syncwarp();
    const double2 zm = __ldcg(z + mc * NB + lane);
    double2 p = make_double2(0, 0);
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 zc;
      zc.x = __shfl_sync(0xffffffffu, zm.x, c);
      zc.y = __shfl_sync(0xffffffffu, zm.y, c);
      cfma(p, lv[c], zc);
    }
    if (row_ok) v = csub(v, p);
  }
  // z_jb = D_jb v
  double2 out = make_double2(0, 0);
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    double2 vc;
    vc.x = __shfl_sync(0xffffffffu, v.x, c);
    vc.y = __shfl_sync(0xffffffffu, v.y, c);
    cfma(out, Ds[lane][c], vc);
  }
  if (row_ok) z[r0 + lane] = out;
  fence_acq_rel_gpu();
  __syncwarp();
  if (lane == 0) st_release(flags + jb, epoch);
}

// Backward solve L^H w = z, block rows in reverse ticket order:
//   w_b = D_b^H (z_b - sum_{m>b} L_mb^H w_m);  out = w or -i w.
// Lane r of a warp reads column r0 + r of the block rows below (coalesced across lanes).
__global__ void __launch_bounds__(TW * 32) k_trsv_upper(int N, const double2* __restrict__ L,
                                                       const double2* __restrict__ D,
                                                       const double2* __restrict__ z,
                                                       double2* __restrict__ w_out, bool minus_i,
                                                       double2* __restrict__ wbuf, unsigned* flags,
                                                       unsigned* ticket, unsigned epoch,
                                                       int* status) {
  __shared__ double2 part[TW][NB];
  __shared__ double2 Ds[NB][NB + 1];
  __shared__ int s_jb;
  const int nblk = (N + NB - 1) / NB;
  if (threadIdx.x == 0) s_jb = nblk - 1 - (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int jb = s_jb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    Ds[r][c] = (r0 + r < N) ? D[((size_t)jb * NB + r) * NB + c] : make_double2(0, 0);
  }
  const bool col_ok = r0 + lane < N;
  double2 acc = make_double2(0, 0);
  // warps 1..TW-1: blocks m = jb+2 .. nblk-1
  for (int m = jb + 2 + (warp - 1); warp > 0 && m < nblk; m += TW - 1) {
    double2 lv[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 l = make_double2(0, 0);
      if (m * NB + c < N && col_ok) l = __ldg(L + (size_t)(m * NB + c) * N + r0 + lane);
      lv[c] = l;
    }
    if (lane == 0) wait_flag(flags + m, epoch, status);
    __syncwarp();
    const double2 wm = (m * NB + lane < N) ? __ldcg(wbuf + m * NB + lane) : make_double2(0, 0);
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 wc;
      wc.x = __shfl_sync(0xffffffffu, wm.x, c);
      wc.y = __shfl_sync(0xffffffffu, wm.y, c);
      cfmac(acc, lv[c], wc);
    }
  }
  if (warp > 0) part[warp][lane] = acc;
  __syncthreads();
  if (warp != 0) return;
  const int mc = jb + 1;
  double2 lv[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    double2 l = make_double2(0, 0);
    if (mc < nblk && mc * NB + c < N && col_ok) l = __ldg(L + (size_t)(mc * NB + c) * N + r0 + lane);
    lv[c] = l;
  }
  double2 v = col_ok ? z[r0 + lane] : make_double2(0, 0);
  for (int w = 1; w < TW; ++w) v = csub(v, part[w][lane]);
  if (mc < nblk) {
    if (lane == 0) wait_flag(flags + mc, epoch, status);
    __syncwarp();
    const double2 wm = (mc * NB + lane < N) ? __ldcg(wbuf + mc * NB + lane) : make_double2(0, 0);
    double2 p = make_double2(0, 0);
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 wc;
      wc.x = __shfl_sync(0xffffffffu, wm.x, c);
      wc.y = __shfl_sync(0xffffffffu, wm.y, c);
      cfmac(p, lv[c], wc);
    }
    v = csub(v, p);
  }
  // w_jb = D_jb^H v: w_r = sum_c conj(D_cr) v_c
  double2 out = make_double2(0, 0);
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    double2 vc;
    vc.x = __shfl_sync(0xffffffffu, v.x, c);
    vc.y = __shfl_sync(0xffffffffu, v.y, c);
    cfmac(out, Ds[c][lane], vc);
  }
  if (col_ok) {
    wbuf[r0 + lane] = out;
    w_out[r0 + lane] = minus_i ? make_double2(out.y, -out.x) : out;
  }
  fence_acq_rel_gpu();
  __syncwarp();
  if (lane == 0) st_release(flags + jb, epoch);
}

void launch_chol_solve(int N, const double2* L, const double2* D, const double2* y, double2* work,
                       double2* out, bool minus_i, unsigned* flags, unsigned* tickets,
                       unsigned epoch, int* status, cudaStream_t s) {
  const int nblk = (N + NB - 1) / NB;
  cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned), s);
  k_trsv_lower<<<nblk, TW * 32, 0, s>>>(N, L, D, y, work, flags, tickets, epoch, status);
  // work[0, N) holds z; work[N, 2N) holds w for the backward pass's consumers
  k_trsv_upper<<<nblk, TW * 32, 0, s>>>(N, L, D, work, out, minus_i, work + N, flags + nblk,
                                        tickets + 1, epoch, status);
}

// ------------------------------------------------------------------------------ RK4 combination

__global__ void k_rk4_final(int N, double2* C, const double2* k1, const double2* k2,
                            const double2* k3, const double2* k4, double h, int* status) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= N) return;
  double2 s;
  s.x = ((k1[a].x + 2.0 * k2[a].x) + 2.0 * k3[a].x) + k4[a].x;
  s.y = ((k1[a].y + 2.0 * k2[a].y) + 2.0 * k3[a].y) + k4[a].y;
  double2 c = C[a];
  c.x += h * s.x;
  c.y += h * s.y;
  if (!isfinite(c.x) || !isfinite(c.y)) set_flag(status, ST_NONFINITE);
  C[a] = c;
}

void launch_rk4_final(int N, double2* C, const double2* k1, const double2* k2,
                      const double2* k3, const double2* k4, double dt, int* status,
                      cudaStream_t s) {
  k_rk4_final<<<(N + 255) / 256, 256, 0, s>>>(N, C, k1, k2, k3, k4, dt / 6.0, status);
}

__global__ void k_check_finite(int n, const double2* a, int* status) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    if (!isfinite(a[e].x) || !isfinite(a[e].y)) { set_flag(status, ST_NONFINITE); return; }
}
void launch_check_finite(int n, const double2* a, int* status, cudaStream_t s) {
  int g = (n + 255) / 256;
  if (g > 1024) g = 1024;
  k_check_finite<<<g, 256, 0, s>>>(n, a, status);
}

}  // namespace icwf
