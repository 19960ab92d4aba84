// FP64 linear algebra of the coefficient update (Eq. coeff, S dC/dt = -i Heff C): the
// Tikhonov-shifted overlap S + eps I, its blocked Cholesky factorisation, the two triangular
// solves, the Heff matrix-vector products of the RK4 stages and the final RK4 combination.
// All arithmetic here is FP64 (S is near-singular as CWFs overlap); the factorisation's trailing
// updates run either here with FP64 FMAs or in emulated FP64 on the tensor cores (exact integer
// digit products, k_herk_emu.cu).  The FP64 mode and the solve_fp64 option of the mixed modes
// factorise and solve with these kernels; the mixed modes' default solver is the double-float one
// of k_linalg_df.cu.
#include <cuda_runtime.h>

#include "herk_digits.cuh"
#include "icwf_internal.h"
#include "k_common.cuh"

namespace icwf {

constexpr int NB = 32;                 // block size of the factorisation and of the solves
constexpr unsigned WAIT_LIMIT = 1u << 22;   // bounded spin (x ~64 ns sleep: well under 1 s)

// ------------------------------------------------------------------------------ S + eps I

// One CTA per row r (no index division per element).
__global__ void k_shift_mix(int N, const double2* __restrict__ S0, const double2* __restrict__ S1,
                            double eps, double theta, double2* __restrict__ A) {
  const int r = blockIdx.x;
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    const size_t e = (size_t)r * N + c;
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
  k_shift_mix<<<N, 256, 0, s>>>(N, S0, S1, eps, theta, A);
}

// ------------------------------------------------------------------------------ Cholesky

struct MatBatch { double2* m[2]; double* inv[2]; double2* D[2]; };

constexpr int PF_THREADS = 256;


// Factor the diagonal block jb of each matrix (one CTA per matrix) in FP64, right-looking by
// columns.  Column c: its entries below the pivot are scaled, L_rc = A_rc y_c (y_c = 1/sqrt(A_cc),
// computed during the previous column); then the trailing triangle takes the rank-1 update
// A_rq -= L_rc conj(L_qc) for c < q <= r (four FMAs per element).  The update's pairs are read
// from a table sorted by q descending, so those of column c are its first (31-c)(32-c)/2 entries
// and every warp instruction of the update runs on full warps (FP64 instructions issue per warp,
// whatever the number of active lanes).  Thread 0 updates the next pivot, A_{c+1,c+1}, itself and
// computes its reciprocal square root while the others finish the update.  Two barriers per
// column.  Outputs: L in place and the reciprocal pivots.  Rows and columns beyond N are treated
// as identity so that ragged sizes factor cleanly.
//
// FP64 operations wait for one another for a long time on this GPU, so the pivot chain is kept
// short.  The reciprocal square root of a pivot d starts from the FP32 estimate (d narrowed and
// the estimate widened by integer operations on the bit patterns: no FP64 instruction) and takes
// one third-order correction in FP64, y = y0 (1 + r/2 + 3 r^2/8) with r = 1 - d y0^2 (the
// binomial series of (1 - r)^(-1/2) cut after r^2): the estimate's ~2^-22 relative error becomes
// ~2^-64, below FP64 rounding, in five dependent FP64 operations.
__device__ __forceinline__ double rsqrt_fp64(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int E = (int)(u >> 52);   // d > 0
  if (E < 1023 - 120 || E > 1023 + 120) return 1.0 / sqrt(d);   // outside FP32's range
  // d with its mantissa truncated to 23 bits, as an FP32 number (relative error < 2^-23)
  const float f = __uint_as_float(((uint32_t)(E - 1023 + 127) << 23) | (uint32_t)((u >> 29) & 0x7FFFFFu));
  const uint32_t v = __float_as_uint(rsqrtf(f));
  // exact widening of the estimate
  const double y0 = __hiloint2double(
      (int)(((((v >> 23) & 0xFFu) - 127u + 1023u) << 20) | ((v & 0x7FFFFFu) >> 3)), (int)((v & 7u) << 29));
  const double r = fma(-d, y0 * y0, 1.0);
  return fma(y0, r * fma(0.375, r, 0.5), y0);
}
// a pivot is usable when 0 < d < inf (integer test on the bits: no FP64 compare on the chain)
__device__ __forceinline__ bool pivot_ok(double d) {
  const long long b = __double_as_longlong(d);
  return b > 0 && b < 0x7FF0000000000000ll;
}
__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b) { return cmul(a, cconj(b)); }
// a -= t conj(b) in four FMAs
__device__ __forceinline__ double2 csub_mul_conj(double2 a, double2 t, double2 b) {
  a.x = fma(-t.x, b.x, fma(-t.y, b.y, a.x));
  a.y = fma(-t.y, b.x, fma(t.x, b.y, a.y));
  return a;
}

constexpr int PF_PAIRS = (NB - 1) * NB / 2;   // pairs (r, q), 1 <= q <= r <= 31

__global__ void __launch_bounds__(PF_THREADS) k_potrf_diag(int N, MatBatch mb, int jb, int* status) {
  __shared__ double2 L[NB][NB + 1];
  __shared__ double yv[NB];
  __shared__ unsigned char pr[PF_PAIRS], pq[PF_PAIRS];
  double2* A = mb.m[blockIdx.y];
  double* inv = mb.inv[blockIdx.y];
  const int r0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += PF_THREADS) {
    const int r = e / NB, c = e % NB;
    double2 v = make_double2(r == c ? 1.0 : 0.0, 0.0);
    if (c <= r && r0 + r < N && r0 + c < N) v = A[(size_t)(r0 + r) * N + r0 + c];
    L[r][c] = v;
  }
  // pair table: q = 31, 30, ..., 1, and r = q..31 within each q
  for (int i = threadIdx.x; i < PF_PAIRS; i += PF_THREADS) {
    int q = NB - 1, k = i;
    while (k >= NB - q) { k -= NB - q; --q; }
    pr[i] = (unsigned char)(q + k);
    pq[i] = (unsigned char)q;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = L[0][0].x;
    if (!pivot_ok(d)) { set_flag(status, ST_CHOL); d = 1.0; }
    const double y = rsqrt_fp64(d);
    L[0][0] = make_double2(d * y, 0.0);
    yv[0] = y;
  }
  __syncthreads();
  for (int c = 0; c < NB - 1; ++c) {
    double2 l0;   // thread 0: L_{c+1,c}, kept in registers for the next pivot
    {
      const int r = c + 1 + (int)threadIdx.x;
      if (r < NB) L[r][c] = l0 = cscale(L[r][c], yv[c]);
    }
    __syncthreads();
    const int n = (NB - 1 - c) * (NB - c) / 2;
    const int skip = n - (NB - 1 - c);   // the pair (c+1, c+1): thread 0's
    if (threadIdx.x == 0) {
      double d = fma(-l0.x, l0.x, fma(-l0.y, l0.y, L[c + 1][c + 1].x));
      if (!pivot_ok(d)) { set_flag(status, ST_CHOL); d = 1.0; }
      const double y = rsqrt_fp64(d);
      L[c + 1][c + 1] = make_double2(d * y, 0.0);
      yv[c + 1] = y;
    }
    for (int i = (int)threadIdx.x; i < n; i += PF_THREADS) {
      if (i == skip) continue;
      const int r = pr[i], q = pq[i];
      L[r][q] = csub_mul_conj(L[r][q], L[r][c], L[q][c]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NB * NB; e += PF_THREADS) {
    const int r = e / NB, c = e % NB;
    if (c <= r && r0 + r < N && r0 + c < N) A[(size_t)(r0 + r) * N + r0 + c] = L[r][c];
  }
  if (threadIdx.x < NB && r0 + threadIdx.x < N) inv[r0 + threadIdx.x] = yv[threadIdx.x];
}

constexpr int TR_WARPS = 8;   // rows per panel-solve CTA

// Panel solve A_ib <- A_ib L_bb^-H below the diagonal block jb in FP64: one warp per row, lane =
// column, column-oriented substitution on unscaled numerators: a_c -= a_m (conj(L_cm) / L_mm)
// for c > m with the multipliers conj(L_cm) / L_mm staged in shared memory (four FMAs per
// update), and x_c = a_c / L_cc once at the end.  With `emu`, the finished row's digit planes for
// the emulated trailing update are written as well.
__global__ void __launch_bounds__(TR_WARPS * 32) k_trsm_panel(int N, MatBatch mb, int jb,
                                                              EmuPlanes emu) {
  __shared__ double2 Lp[NB][NB + 1];
  const int bm = blockIdx.y;
  double2* A = mb.m[bm];
  const double* inv = mb.inv[bm];
  const int c0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    double2 l = make_double2(0.0, 0.0);
    if (c < r && c0 + r < N) l = cscale(cconj(A[(size_t)(c0 + r) * N + c0 + c]), inv[c0 + c]);
    Lp[r][c] = l;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = (jb + 1) * NB + blockIdx.x * TR_WARPS + warp;
  if (row >= N) return;
  // a block column with rows below it is full: every lane's column is inside the matrix
  double2 a = A[(size_t)row * N + c0 + lane];
#pragma unroll
  for (int m = 0; m < NB - 1; ++m) {
    double2 am;
    am.x = __shfl_sync(0xffffffffu, a.x, m);
    am.y = __shfl_sync(0xffffffffu, a.y, m);
    if (lane > m) {
      const double2 l = Lp[lane][m];
      a.x = fma(-am.x, l.x, fma(am.y, l.y, a.x));
      a.y = fma(-am.x, l.y, fma(-am.y, l.x, a.y));
    }
  }
  a = cscale(a, inv[c0 + lane]);
  A[(size_t)row * N + c0 + lane] = a;
  if (emu.planes[0])
    hemu::emit_row_digits(a, row, lane, emu.rpad, (__nv_bfloat16*)emu.planes[bm], emu.ex[bm]);
}

// Inverse of every diagonal block after the factorisation: D_b = L_bb^-1 (lower triangular),
// row-major per block in D[(b*32 + r)*32 + c], one CTA per block, all blocks at once, in FP64.
// Right-looking elimination: for k = 0..31, row k of D is scaled by 1/L_kk (it is then final) and
// removed from the rows below with the multipliers L_rk.
__global__ void __launch_bounds__(128) k_trtri_diag(int N, MatBatch mb) {
  __shared__ double2 Ls[NB][NB + 1];
  __shared__ double2 Dm[NB][NB + 1];
  __shared__ double ys[NB];
  const double2* A = mb.m[blockIdx.y];
  const double* inv = mb.inv[blockIdx.y];
  double2* D = mb.D[blockIdx.y];
  const int jb = blockIdx.x, r0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    double2 l = make_double2(0.0, 0.0);
    if (c < r && r0 + r < N && r0 + c < N) l = A[(size_t)(r0 + r) * N + r0 + c];
    Ls[r][c] = l;
    Dm[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  if (threadIdx.x < NB) ys[threadIdx.x] = (r0 + threadIdx.x < N) ? inv[r0 + threadIdx.x] : 1.0;
  __syncthreads();
  for (int k = 0; k < NB; ++k) {
    if (threadIdx.x <= k) Dm[k][threadIdx.x] = cscale(Dm[k][threadIdx.x], ys[k]);
    __syncthreads();
    const int rows = NB - 1 - k, cols = k + 1;
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int r = k + 1 + e / cols, c = e % cols;
      Dm[r][c] = csub(Dm[r][c], cmul(Ls[r][k], Dm[k][c]));
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    if (r0 + r < N) D[((size_t)jb * NB + r) * NB + c] = Dm[r][c];
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
  {
    // four independent partial sums per output (FP64 latency), combined at the end
    double2 pa[4][2][2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) pa[q][r][c] = z;
#pragma unroll
    for (int m = 0; m < NB; ++m) {
      const double2 a0 = Lr[ty][m], a1 = Lr[ty + 16][m];
      const double2 b0 = Lc[tx][m], b1 = Lc[tx + 16][m];
      // acc += a * conj(b)
      cfmac(pa[m & 3][0][0], b0, a0); cfmac(pa[m & 3][0][1], b1, a0);
      cfmac(pa[m & 3][1][0], b0, a1); cfmac(pa[m & 3][1][1], b1, a1);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c)
        acc[r][c] = cadd(cadd(pa[0][r][c], pa[1][r][c]), cadd(pa[2][r][c], pa[3][r][c]));
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
                    int* status, cudaStream_t s, void* emu_scratch, size_t emu_bytes) {
  MatBatch mb;
  mb.m[0] = A[0];
  mb.m[1] = nbatch > 1 ? A[1] : A[0];
  mb.inv[0] = inv[0];
  mb.inv[1] = nbatch > 1 ? inv[1] : inv[0];
  mb.D[0] = D[0];
  mb.D[1] = nbatch > 1 ? D[1] : D[0];
  const int T = (N + NB - 1) / NB;
  // the panel solve writes the emulated update's digit planes (scratch checked here, so that a
  // launch_herk_emu refusal cannot leave a panel without its FP64 update)
  EmuPlanes emu{};
  if (emu_scratch && emu_bytes >= herk_emu_scratch_bytes(N)) emu = herk_emu_planes(N, emu_scratch);
  int launches = 0;
  for (int jb = 0; jb < T; ++jb) {
    k_potrf_diag<<<dim3(1, nbatch), PF_THREADS, 0, s>>>(N, mb, jb, status);
    ++launches;
    const int rest = T - jb - 1;
    if (rest > 0) {
      const int rows = N - (jb + 1) * NB;
      k_trsm_panel<<<dim3((rows + TR_WARPS - 1) / TR_WARPS, nbatch), TR_WARPS * 32, 0, s>>>(
          N, mb, jb, emu);
      if (!emu.planes[0] || !launch_herk_emu(N, jb, A, nbatch, emu_scratch, emu_bytes, true, status, s))
        k_herk_update<<<dim3(rest * (rest + 1) / 2, nbatch), 256, 0, s>>>(N, mb, jb);
      launches += 2;
    }
  }
  k_trtri_diag<<<dim3(T, nbatch), 128, 0, s>>>(N, mb);
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
  // four independent partial sums: dependent FP64 operations are long-latency on this GPU
  double2 t[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  const double2* h0 = H0 + (size_t)a * N;
  const double2* h1 = H1 + (size_t)a * N;
  int q = 0;
  for (int b = lane; b < N; b += 32, q = (q + 1) & 3) {
    double2 v = C[b];
    if (kp) { const double2 k = kp[b]; v.x += c * k.x; v.y += c * k.y; }
    double2 h;
    if (theta == 0.0) h = h0[b];
    else if (theta == 1.0) h = h1[b];
    else h = make_double2(0.5 * (h0[b].x + h1[b].x), 0.5 * (h0[b].y + h1[b].y));
    cfma(t[q], h, v);
  }
  double2 acc = cadd(cadd(t[0], t[1]), cadd(t[2], t[3]));
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
  const unsigned lim = wait_budget(status, WAIT_LIMIT);
  for (unsigned it = 0; it < lim; ++it) {
    if (ld_acquire(f) == epoch) return true;
    if (it > 4096) __nanosleep(64);   // pure spin first: the expected wait is a few microseconds
  }
  set_flag(status, ST_TIMEOUT);
  return false;
}

constexpr int TW = 8;   // warps per triangular-solve CTA
constexpr int CW = 4;   // warps sharing the critical block and the diagonal product (one per SM
                        // sub-partition, so the FP64 work on the dependency chain uses all four
                        // FP64 units of the SM)

// Dependent FP64 operations are very slow on this part (hundreds of cycles of latency), so the
// short complex dot products on the solves' dependency chain are evaluated as independent
// products followed by a pairwise tree, never as one running accumulator.
template <int K>
__device__ __forceinline__ double2 tree_sum(double2 (&t)[K]) {
#pragma unroll
  for (int w = 1; w < K; w *= 2)
#pragma unroll
    for (int q = 0; q + w < K; q += 2 * w) t[q] = cadd(t[q], t[q + w]);
  return t[0];
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

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
  __shared__ double2 vsh[NB];
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
  // warps CW..TW-1: blocks m = 0 .. jb-2, round robin (the critical warps 0..CW-1 take jb-1)
  for (int m = warp - CW; warp >= CW && m < jb - 1; m += TW - CW) {
    double2 lv[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) lv[c] = __ldg(Lrow + m * NB + c);
    if (lane == 0) wait_flag(flags + m, epoch, status);
    __syncwarp();
    const double2 zm = __ldcg(z + m * NB + lane);
    double2 t[4] = {acc, make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 zc;
      zc.x = __shfl_sync(0xffffffffu, zm.x, c);
      zc.y = __shfl_sync(0xffffffffu, zm.y, c);
      cfma(t[c & 3], lv[c], zc);
    }
    acc = tree_sum(t);
  }
  if (warp >= CW) part[warp][lane] = row_ok ? acc : make_double2(0, 0);
  // warps 0..CW-1 prefetch their columns of the critical block (jb-1)
  const int mc = jb - 1;
  constexpr int CPW = NB / CW;   // columns per critical warp
  double2 lv[CPW];
#pragma unroll
  for (int q = 0; q < CPW; ++q)
    lv[q] = (warp < CW && mc >= 0) ? __ldg(Lrow + mc * NB + warp * CPW + q) : make_double2(0, 0);
  __syncthreads();   // part[] of warps CW.. complete
  if (warp >= CW) return;
  double2 v = make_double2(0, 0);
  if (warp == 0) {
    v = row_ok ? y[r0 + lane] : make_double2(0, 0);
    for (int w = CW; w < TW; ++w) v = csub(v, part[w][lane]);
  }
  double2 p = make_double2(0, 0);
  if (mc >= 0) {
    if (lane == 0) wait_flag(flags + mc, epoch, status);
    __syncwarp();
    const double2 zm = __ldcg(z + mc * NB + lane);
    double2 t[CPW];
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp * CPW + q;
      double2 zc;
      zc.x = __shfl_sync(0xffffffffu, zm.x, c);
      zc.y = __shfl_sync(0xffffffffu, zm.y, c);
      t[q] = cmul(lv[q], zc);
    }
    p = tree_sum(t);
  }
  part[warp][lane] = p;   // rows' partial products, one per critical warp
  named_sync(1, CW * 32);
  if (warp == 0) {
    double2 t[CW];
#pragma unroll
    for (int w = 0; w < CW; ++w) t[w] = part[w][lane];
    v = csub(v, tree_sum(t));
    if (!row_ok) v = make_double2(0, 0);
    vsh[lane] = v;
  }
  named_sync(1, CW * 32);
  // z_jb = D_jb v, columns split over the critical warps
  double2 out;
  {
    double2 t[CPW];
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp * CPW + q;
      t[q] = cmul(Ds[lane][c], vsh[c]);
    }
    out = tree_sum(t);
  }
  part[warp][lane] = out;
  named_sync(1, CW * 32);
  if (warp == 0) {
    double2 t[CW];
#pragma unroll
    for (int w = 0; w < CW; ++w) t[w] = part[w][lane];
    const double2 zz = tree_sum(t);
    if (row_ok) z[r0 + lane] = zz;
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0) st_release(flags + jb, epoch);
  }
}

// Backward solve L^H w = z, block rows in reverse ticket order:
//   w_b = D_b^H (z_b - sum_{m>b} L_mb^H w_m);  out = w or -i w.
// Lane r of a warp reads column r0 + r of the block rows below (coalesced across lanes).  Warps
// 0..CW-1 share the critical block (jb+1) and the diagonal product; the others take the rest.
__global__ void __launch_bounds__(TW * 32) k_trsv_upper(int N, const double2* __restrict__ L,
                                                       const double2* __restrict__ D,
                                                       const double2* __restrict__ z,
                                                       double2* __restrict__ w_out, bool minus_i,
                                                       double2* __restrict__ wbuf, unsigned* flags,
                                                       unsigned* ticket, unsigned epoch,
                                                       int* status) {
  __shared__ double2 part[TW][NB];
  __shared__ double2 Ds[NB][NB + 1];
  __shared__ double2 vsh[NB];
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
  // warps CW..TW-1: blocks m = nblk-1 .. jb+2, in the order the blocks complete (descending)
  for (int m = nblk - 1 - (warp - CW); warp >= CW && m >= jb + 2; m -= TW - CW) {
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
    double2 t[4] = {acc, make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double2 wc;
      wc.x = __shfl_sync(0xffffffffu, wm.x, c);
      wc.y = __shfl_sync(0xffffffffu, wm.y, c);
      cfmac(t[c & 3], lv[c], wc);
    }
    acc = tree_sum(t);
  }
  if (warp >= CW) part[warp][lane] = acc;
  const int mc = jb + 1;
  constexpr int CPW = NB / CW;
  double2 lv[CPW];
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp * CPW + q;
    double2 l = make_double2(0, 0);
    if (warp < CW && mc < nblk && mc * NB + c < N && col_ok)
      l = __ldg(L + (size_t)(mc * NB + c) * N + r0 + lane);
    lv[q] = l;
  }
  __syncthreads();
  if (warp >= CW) return;
  double2 v = make_double2(0, 0);
  if (warp == 0) {
    v = col_ok ? z[r0 + lane] : make_double2(0, 0);
    for (int w = CW; w < TW; ++w) v = csub(v, part[w][lane]);
  }
  double2 p = make_double2(0, 0);
  if (mc < nblk) {
    if (lane == 0) wait_flag(flags + mc, epoch, status);
    __syncwarp();
    const double2 wm = (mc * NB + lane < N) ? __ldcg(wbuf + mc * NB + lane) : make_double2(0, 0);
    double2 t[CPW];
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp * CPW + q;
      double2 wc;
      wc.x = __shfl_sync(0xffffffffu, wm.x, c);
      wc.y = __shfl_sync(0xffffffffu, wm.y, c);
      t[q] = cmulc(lv[q], wc);
    }
    p = tree_sum(t);
  }
  part[warp][lane] = p;
  named_sync(1, CW * 32);
  if (warp == 0) {
    double2 t[CW];
#pragma unroll
    for (int w = 0; w < CW; ++w) t[w] = part[w][lane];
    v = csub(v, tree_sum(t));
    if (!col_ok) v = make_double2(0, 0);
    vsh[lane] = v;
  }
  named_sync(1, CW * 32);
  // w_jb = D_jb^H v: w_r = sum_c conj(D_cr) v_c, columns split over the critical warps
  double2 out;
  {
    double2 t[CPW];
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp * CPW + q;
      t[q] = cmulc(Ds[c][lane], vsh[c]);
    }
    out = tree_sum(t);
  }
  part[warp][lane] = out;
  named_sync(1, CW * 32);
  if (warp == 0) {
    double2 t[CW];
#pragma unroll
    for (int w = 0; w < CW; ++w) t[w] = part[w][lane];
    const double2 ww = tree_sum(t);
    if (col_ok) {
      wbuf[r0 + lane] = ww;
      w_out[r0 + lane] = minus_i ? make_double2(ww.y, -ww.x) : ww;
    }
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0) st_release(flags + jb, epoch);
  }
}

void launch_chol_solve(int N, const double2* L, const double2* D, const double2* y, double2* work,
                       double2* out, bool minus_i, unsigned* flags, unsigned* tickets,
                       unsigned epoch, int* status, cudaStream_t s) {
  const int nblk = (N + NB - 1) / NB;
  // the block flags start from zero in every solve (one memset with the tickets, which follow
  // them), so a captured launch sequence can be replayed with the same epoch
  cudaMemsetAsync(flags, 0, (2 * (size_t)nblk + 2) * sizeof(unsigned), s);
  (void)tickets;
  k_trsv_lower<<<nblk, TW * 32, 0, s>>>(N, L, D, y, work, flags, flags + 2 * nblk, epoch, status);
  // work[0, N) holds z; work[N, 2N) holds w for the backward pass's consumers
  k_trsv_upper<<<nblk, TW * 32, 0, s>>>(N, L, D, work, out, minus_i, work + N, flags + nblk,
                                        flags + 2 * nblk + 1, epoch, status);
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
