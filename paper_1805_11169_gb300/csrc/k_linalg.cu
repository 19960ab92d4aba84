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

struct MatBatch { double2* m[2]; };

// Factor the diagonal block jb of each matrix (one CTA per matrix).  Rows/columns beyond N are
// treated as identity so that ragged sizes factor cleanly.
__global__ void __launch_bounds__(256) k_potrf_diag(int N, MatBatch mb, int jb, int* status) {
  __shared__ double2 L[NB][NB + 1];
  double2* A = mb.m[blockIdx.y];
  const int r0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    double2 v = make_double2(r == c ? 1.0 : 0.0, 0.0);
    if (r0 + r < N && r0 + c < N) v = A[(size_t)(r0 + r) * N + r0 + c];
    L[r][c] = v;
  }
  __syncthreads();
  for (int c = 0; c < NB; ++c) {
    if (threadIdx.x == 0) {
      double d = L[c][c].x;
      if (!(d > 0.0)) { set_flag(status, ST_CHOL); d = 1.0; }
      L[c][c] = make_double2(sqrt(d), 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / L[c][c].x;
    for (int r = c + 1 + threadIdx.x; r < NB; r += blockDim.x) L[r][c] = cscale(L[r][c], inv);
    __syncthreads();
    const int m = NB - 1 - c;   // trailing size
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int r = c + 1 + e / m, q = c + 1 + e % m;
      if (q <= r) {
        // L[r][q] -= L[r][c] * conj(L[q][c])
        const double2 a = L[r][c], b = L[q][c];
        L[r][q].x -= a.x * b.x + a.y * b.y;
        L[r][q].y -= a.y * b.x - a.x * b.y;
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    if (c <= r && r0 + r < N && r0 + c < N) A[(size_t)(r0 + r) * N + r0 + c] = L[r][c];
  }
}

// Panel solve A_ib <- A_ib L_bb^-H for every block row i > jb (one CTA per block row).
__global__ void __launch_bounds__(256) k_trsm_panel(int N, MatBatch mb, int jb) {
  __shared__ double2 L[NB][NB + 1];
  __shared__ double2 X[NB][NB + 1];
  double2* A = mb.m[blockIdx.y];
  const int ib = jb + 1 + blockIdx.x;
  const int r0 = ib * NB, c0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    double2 l = make_double2(r == c ? 1.0 : 0.0, 0.0);
    if (c0 + r < N && c0 + c < N && c <= r) l = A[(size_t)(c0 + r) * N + c0 + c];
    if (c > r) l = make_double2(0.0, 0.0);
    L[r][c] = l;
    double2 x = make_double2(0.0, 0.0);
    if (r0 + r < N && c0 + c < N) x = A[(size_t)(r0 + r) * N + c0 + c];
    X[r][c] = x;
  }
  __syncthreads();
  for (int c = 0; c < NB; ++c) {
    const double inv = 1.0 / L[c][c].x;
    if (threadIdx.x < NB) X[threadIdx.x][c] = cscale(X[threadIdx.x][c], inv);
    __syncthreads();
    const int m = NB - 1 - c;
    for (int e = threadIdx.x; e < NB * m; e += blockDim.x) {
      const int r = e / m, q = c + 1 + e % m;
      // X[r][q] -= X[r][c] * conj(L[q][c])
      const double2 a = X[r][c], b = L[q][c];
      X[r][q].x -= a.x * b.x + a.y * b.y;
      X[r][q].y -= a.y * b.x - a.x * b.y;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    if (r0 + r < N && c0 + c < N) A[(size_t)(r0 + r) * N + c0 + c] = X[r][c];
  }
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

void launch_cholesky(int N, double2* const* A, int nbatch, int* status, cudaStream_t s) {
  MatBatch mb;
  mb.m[0] = A[0];
  mb.m[1] = nbatch > 1 ? A[1] : A[0];
  const int T = (N + NB - 1) / NB;
  for (int jb = 0; jb < T; ++jb) {
    k_potrf_diag<<<dim3(1, nbatch), 256, 0, s>>>(N, mb, jb, status);
    const int rest = T - jb - 1;
    if (rest > 0) {
      k_trsm_panel<<<dim3(rest, nbatch), 256, 0, s>>>(N, mb, jb);
      k_herk_update<<<dim3(rest * (rest + 1) / 2, nbatch), 256, 0, s>>>(N, mb, jb);
    }
  }
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
    __nanosleep(64);
  }
  set_flag(status, ST_TIMEOUT);
  return false;
}

constexpr int TW = 8;   // warps per triangular-solve CTA

// Forward solve L z = y.  CTAs take block rows in ticket order (a CTA only waits on block rows
// with smaller tickets, which are already running or done).  Warp w of the CTA accumulates the
// off-diagonal products of block columns m = w, w + TW, ...; warp 0 then substitutes within the
// diagonal block and publishes z_jb with a release flag.  Each lane first loads its 32 matrix
// entries of a block into registers (independent loads in flight together), then combines them
// with z broadcast by shuffles.
__global__ void __launch_bounds__(TW * 32) k_trsv_lower(int N, const double2* __restrict__ L,
                                                       const double2* __restrict__ y,
                                                       double2* __restrict__ z, unsigned* flags,
                                                       unsigned* ticket, unsigned epoch,
                                                       int* status) {
  __shared__ double2 part[TW][NB];
  __shared__ int s_jb;
  if (threadIdx.x == 0) s_jb = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int jb = s_jb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = jb * NB;
  double2 acc = make_double2(0, 0);
  const bool row_ok = r0 + lane < N;
  const double2* Lrow = L + (size_t)(row_ok ? r0 + lane : 0) * N;
  for (int m = warp; m < jb; m += TW) {
    double2 lv[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) lv[c] = __ldg(Lrow + m * NB + c);   // columns < jb*NB <= N
    if (lane == 0) wait_flag(flags + m, epoch, status);
    __syncwarp();
    const double2 zm = __ldcg(z + m * NB + lane);   // block m < jb is complete: in range
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 zc;
      zc.x = __shfl_sync(0xffffffffu, zm.x, c);
      zc.y = __shfl_sync(0xffffffffu, zm.y, c);
      cfma(acc, lv[c], zc);
    }
  }
  if (!row_ok) acc = make_double2(0, 0);
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    const int r = lane;
    double2 v = make_double2(0, 0);
    if (r0 + r < N) v = y[r0 + r];
    for (int w = 0; w < TW; ++w) v = csub(v, part[w][r]);
    double2 lrow[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 l = make_double2(c == r ? 1.0 : 0.0, 0.0);
      if (r0 + r < N && r0 + c < N && c <= r) l = L[(size_t)(r0 + r) * N + r0 + c];
      lrow[c] = l;
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 zc = v;
      if (r == c) zc = cscale(v, 1.0 / lrow[c].x);
      zc.x = __shfl_sync(0xffffffffu, zc.x, c);
      zc.y = __shfl_sync(0xffffffffu, zc.y, c);
      if (r == c) v = zc;
      else if (r > c) v = csub(v, cmul(lrow[c], zc));
    }
    if (r0 + r < N) z[r0 + r] = v;
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(flags + jb, epoch);
  }
}

// Backward solve L^H w = z, block rows in reverse ticket order; out = w or -i w.  Lane r of a
// warp reads column r0 + r of the block rows below (coalesced across lanes).
__global__ void __launch_bounds__(TW * 32) k_trsv_upper(int N, const double2* __restrict__ L,
                                                       const double2* __restrict__ z,
                                                       double2* __restrict__ w_out, bool minus_i,
                                                       double2* __restrict__ wbuf, unsigned* flags,
                                                       unsigned* ticket, unsigned epoch,
                                                       int* status) {
  __shared__ double2 part[TW][NB];
  __shared__ int s_jb;
  const int nblk = (N + NB - 1) / NB;
  if (threadIdx.x == 0) s_jb = nblk - 1 - (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int jb = s_jb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = jb * NB;
  const bool col_ok = r0 + lane < N;
  double2 acc = make_double2(0, 0);
  for (int m = jb + 1 + warp; m < nblk; m += TW) {
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
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    const int r = lane;
    double2 v = make_double2(0, 0);
    if (r0 + r < N) v = z[r0 + r];
    for (int w = 0; w < TW; ++w) v = csub(v, part[w][r]);
    // column r of the diagonal block: lcol[q] = L[r0 + q][r0 + r] (q >= r)
    double2 lcol[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      double2 l = make_double2(q == r ? 1.0 : 0.0, 0.0);
      if (r0 + r < N && r0 + q < N && q >= r) l = L[(size_t)(r0 + q) * N + r0 + r];
      lcol[q] = l;
    }
    // w_q for q from NB-1 down: w_q = v_q / L_qq; v_r -= conj(L[q][r]) w_q for r < q
#pragma unroll
    for (int q = NB - 1; q >= 0; --q) {
      double2 wq = v;
      if (r == q) wq = cscale(v, 1.0 / lcol[q].x);
      wq.x = __shfl_sync(0xffffffffu, wq.x, q);
      wq.y = __shfl_sync(0xffffffffu, wq.y, q);
      if (r == q) v = wq;
      else if (r < q) v = csub(v, cmulc(lcol[q], wq));
    }
    if (r0 + r < N) {
      wbuf[r0 + r] = v;
      w_out[r0 + r] = minus_i ? make_double2(v.y, -v.x) : v;
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(flags + jb, epoch);
  }
}

void launch_chol_solve(int N, const double2* L, const double2* y, double2* work, double2* out,
                       bool minus_i, unsigned* flags, unsigned* tickets, unsigned epoch,
                       int* status, cudaStream_t s) {
  const int nblk = (N + NB - 1) / NB;
  cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned), s);
  k_trsv_lower<<<nblk, TW * 32, 0, s>>>(N, L, y, work, flags, tickets, epoch, status);
  // work[0, N) holds z; work[N, 2N) holds w for the backward pass's consumers
  k_trsv_upper<<<nblk, TW * 32, 0, s>>>(N, L, work, out, minus_i, work + N, flags + nblk,
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
