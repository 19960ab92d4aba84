// Coefficient solve of the mixed-precision modes (Eq. coeff) in double-float arithmetic.
//
// The regularised overlap S + eps I is factorised and the RK4 stage systems are solved with
// complex numbers stored as (re_hi, re_lo, im_hi, im_lo) FP32 quadruples (16 bytes, the size of a
// complex128), each part a double-float of ~48 significant bits (csrc/df64.cuh).  On this GPU the
// FP32 pipes have ~64x the FP64 throughput and a far shorter latency, and the Cholesky chain and
// the triangular-solve chains are latency-bound; S itself carries ~1e-6 relative rounding noise in
// these modes, far above the 48-bit arithmetic.  Dot products use compensated accumulation in the
// style of Ogita, Rump and Oishi's Dot2 (TwoProduct + TwoSum, errors summed separately), which
// returns them as accurately as if evaluated in twice the FP32 precision.
//
// Kernels: k_shift_mix_df (S -> S + eps I, converted); k_chol_step_df (the blocked Cholesky, one
// launch per block column with look-ahead: quadrant updates, diagonal factor, panel slabs,
// trailing tiles and the inverses of the diagonal blocks as ticket-ordered tasks; the panel tasks
// also write L^H into the upper triangle); k_chol_solve_cluster (both triangular solves in one
// 8-CTA cluster, N <= 2048) and k_trsv_lower_df / k_trsv_upper_df (per-block kernels with global
// flags, larger N).
#include <cuda_runtime.h>

#include "df64.cuh"
#include "icwf_internal.h"
#include "k_common.cuh"

namespace icwf {
namespace dfs {

constexpr int NB = 32;
constexpr unsigned WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ cdf ld4(const float4 v) {
  return cdf_make(df_make(v.x, v.y), df_make(v.z, v.w));
}
__device__ __forceinline__ float4 st4(cdf z) { return make_float4(z.re.h, z.re.l, z.im.h, z.im.l); }
__device__ __forceinline__ cdf czero() { return cdf_make(df_make(0.f, 0.f), df_make(0.f, 0.f)); }

// Compensated accumulator: value = s + c.
struct acc2 {
  float s, c;
};
__device__ __forceinline__ void acc_prod(acc2& a, float x, float y) {
  const float p = DF_MUL(x, y);
  const float e = DF_FMA(x, y, -p);
  const df t = two_sum(a.s, p);
  a.s = t.h;
  a.c = DF_ADD(a.c, DF_ADD(t.l, e));
}
__device__ __forceinline__ void acc_small(acc2& a, float x) { a.c = DF_ADD(a.c, x); }
__device__ __forceinline__ df acc_val(acc2 a) { return two_sum(a.s, a.c); }
__device__ __forceinline__ acc2 acc_zero() { acc2 a; a.s = 0.f; a.c = 0.f; return a; }
__device__ __forceinline__ acc2 acc_merge(acc2 a, acc2 b) {
  const df t = two_sum(a.s, b.s);
  acc2 r;
  r.s = t.h;
  r.c = DF_ADD(DF_ADD(a.c, b.c), t.l);
  return r;
}

struct cacc {
  acc2 re, im;
};
__device__ __forceinline__ cacc cacc_zero() { cacc z; z.re = acc_zero(); z.im = acc_zero(); return z; }
__device__ __forceinline__ cacc cacc_merge(cacc a, cacc b) {
  cacc r; r.re = acc_merge(a.re, b.re); r.im = acc_merge(a.im, b.im); return r;
}
__device__ __forceinline__ cdf cacc_val(cacc a) { return cdf_make(acc_val(a.re), acc_val(a.im)); }
// a += x * y
__device__ __forceinline__ void cacc_mul(cacc& a, cdf x, cdf y) {
  acc_prod(a.re, x.re.h, y.re.h);
  acc_prod(a.re, -x.im.h, y.im.h);
  acc_small(a.re, DF_FMA(x.re.h, y.re.l, DF_MUL(x.re.l, y.re.h)));
  acc_small(a.re, -DF_FMA(x.im.h, y.im.l, DF_MUL(x.im.l, y.im.h)));
  acc_prod(a.im, x.re.h, y.im.h);
  acc_prod(a.im, x.im.h, y.re.h);
  acc_small(a.im, DF_FMA(x.re.h, y.im.l, DF_MUL(x.re.l, y.im.h)));
  acc_small(a.im, DF_FMA(x.im.h, y.re.l, DF_MUL(x.im.l, y.re.h)));
}
// a += x * conj(y)
__device__ __forceinline__ void cacc_mulc(cacc& a, cdf x, cdf y) {
  acc_prod(a.re, x.re.h, y.re.h);
  acc_prod(a.re, x.im.h, y.im.h);
  acc_small(a.re, DF_FMA(x.re.h, y.re.l, DF_MUL(x.re.l, y.re.h)));
  acc_small(a.re, DF_FMA(x.im.h, y.im.l, DF_MUL(x.im.l, y.im.h)));
  acc_prod(a.im, x.im.h, y.re.h);
  acc_prod(a.im, -x.re.h, y.im.h);
  acc_small(a.im, DF_FMA(x.im.h, y.re.l, DF_MUL(x.im.l, y.re.h)));
  acc_small(a.im, -DF_FMA(x.re.h, y.im.l, DF_MUL(x.re.l, y.im.h)));
}
// a += conj(x) * y
__device__ __forceinline__ void cacc_cmul(cacc& a, cdf x, cdf y) {
  acc_prod(a.re, x.re.h, y.re.h);
  acc_prod(a.re, x.im.h, y.im.h);
  acc_small(a.re, DF_FMA(x.re.h, y.re.l, DF_MUL(x.re.l, y.re.h)));
  acc_small(a.re, DF_FMA(x.im.h, y.im.l, DF_MUL(x.im.l, y.im.h)));
  acc_prod(a.im, x.re.h, y.im.h);
  acc_prod(a.im, -x.im.h, y.re.h);
  acc_small(a.im, DF_FMA(x.re.h, y.im.l, DF_MUL(x.re.l, y.im.h)));
  acc_small(a.im, -DF_FMA(x.im.h, y.re.l, DF_MUL(x.im.l, y.re.h)));
}

struct Batch {
  float4* m[2];
  float2* inv[2];   // 1/L_cc as double-floats
  float4* D[2];     // inverted diagonal blocks
};
// member of a two-entry parameter array without a dynamically indexed (local-memory) copy
template <typename T>
__device__ __forceinline__ T pick2(T const (&a)[2], unsigned i) { return i ? a[1] : a[0]; }

__device__ __forceinline__ cdf shfl_cdf(cdf v, int src) {
  cdf r;
  r.re.h = __shfl_sync(0xffffffffu, v.re.h, src);
  r.re.l = __shfl_sync(0xffffffffu, v.re.l, src);
  r.im.h = __shfl_sync(0xffffffffu, v.im.h, src);
  r.im.l = __shfl_sync(0xffffffffu, v.im.l, src);
  return r;
}

// ---------------------------------------------------------------------------- S + eps I

// One CTA per row r (no index division per element).
__global__ void k_shift_mix_df(int N, const double2* __restrict__ S0, const double2* __restrict__ S1,
                               double eps, double theta, float4* __restrict__ A) {
  const int r = blockIdx.x;
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    const size_t e = (size_t)r * N + c;
    double2 v;
    if (theta == 1.0) v = S1[e];
    else if (theta == 0.0) v = S0[e];
    else v = make_double2(0.5 * (S0[e].x + S1[e].x), 0.5 * (S0[e].y + S1[e].y));
    if (r == c) v.x += eps;
    A[e] = st4(cdf_make(df_from(v.x), df_from(v.y)));
  }
}

__device__ __forceinline__ void tri_index(int t, int& I, int& J) {
  int Jc = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (Jc * (Jc + 1) / 2 > t) --Jc;
  while ((Jc + 1) * (Jc + 2) / 2 <= t) ++Jc;
  J = Jc;
  I = t - Jc * (Jc + 1) / 2;
}

// ---------------------------------------------------------------------------- blocked factorisation
//
// Right-looking blocked Cholesky with one launch per block column and a look-ahead: launch li
// applies panel li - 1 to the trailing matrix and, in the same launch, factors diagonal block li
// and solves panel li.  Its CTAs take tickets in dependency order
//   [3 quadrant updates of diagonal block li] [diagonal factor li] [trailing tiles right of
//   block column li] [panel-li slabs of 8 rows],
// and wait (bounded) only for tasks with smaller tickets, which are already running: the diagonal
// factor waits for its three quadrants, the panel slabs for the diagonal factor.  So the chain
// quadrants -> factor -> slabs overlaps the bulk of the trailing update, and the factor of block
// li + 1 starts as soon as launch li + 1 does.  All arithmetic is double-float with compensated
// (Dot2) accumulation; complex products in the updates use three real products (Karatsuba).

constexpr int CS_THREADS = 256;
constexpr int TS_ROWS = 8;                    // panel rows per slab task
constexpr unsigned CS_WAIT_LIMIT = 1u << 24;
constexpr int CS_SMEM = 6 * NB * NB * 8;      // largest task: trailing tile, 6 double-float planes
// shared memory requested per CTA: more than the tasks use, so that at most two CTAs share an SM
// and the dependency chain (diagonal factor, panel slabs) is not starved by trailing tiles
constexpr int CS_SMEM_LAUNCH = 100 * 1024;
static_assert(CS_SMEM <= CS_SMEM_LAUNCH, "tasks need more shared memory than the launch asks for");

__device__ __forceinline__ cdf ldcg4(const float4* p) { return ld4(__ldcg(p)); }
__device__ __forceinline__ cdf cdf_sub_sloppy(cdf a, cdf b) {
  return cdf_make(df_add_sloppy(a.re, df_neg(b.re)), df_add_sloppy(a.im, df_neg(b.im)));
}
// a += x y for double-float reals (Dot2 step on the high parts, cross terms in FP32)
__device__ __forceinline__ void acc_prod_df(acc2& a, df x, df y) {
  acc_prod(a, x.h, y.h);
  acc_small(a, DF_FMA(x.h, y.l, DF_MUL(x.l, y.h)));
}
__device__ __forceinline__ acc2 acc_neg(acc2 a) { a.s = -a.s; a.c = -a.c; return a; }
// Karatsuba: x conj(w) from P1 = xr wr, P2 = xi wi, P3 = (xr + xi)(wr - wi)
__device__ __forceinline__ cdf kara_val(acc2 p1, acc2 p2, acc2 p3) {
  return cdf_make(acc_val(acc_merge(p1, p2)), acc_val(acc_merge(acc_merge(p3, acc_neg(p1)), p2)));
}

__device__ __forceinline__ bool cs_wait(const unsigned* f, unsigned target, int* status) {
  const unsigned lim = wait_budget(status, CS_WAIT_LIMIT);
  for (unsigned it = 0; it < lim; ++it) {
    if (ld_acquire(f) >= target) return true;
    if (it > 256) __nanosleep(128);
  }
  set_flag(status, ST_TIMEOUT);
  return false;
}
// all of this CTA's global writes, then a release increment of *f
__device__ __forceinline__ void cs_signal(unsigned* f) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(f, 1u);
  }
}

// One output per thread of an R x C block (R C = 256): returns A[orow][ocol] - sum_k X[r][k] conj(Y[c][k])
// with X = rows xrow0.., Y = rows yrow0.. of A over columns k0..k0+31.
template <int R, int C>
__device__ __forceinline__ cdf upd_one(const float4* A, int N, int xrow0, int yrow0, int k0,
                                       int orow, int ocol, bool ok, unsigned char* smem) {
  df(*Xp)[R][NB] = (df(*)[R][NB])smem;                        // [3][R][32]
  df(*Yp)[NB][C] = (df(*)[NB][C])(smem + 3 * R * NB * 8);     // [3][32][C]
  const cdf a = ok ? ldcg4(A + (size_t)orow * N + ocol) : czero();   // issued first, used last
  for (int e = threadIdx.x; e < R * NB; e += CS_THREADS) {
    const int r = e / NB, k = e % NB;
    cdf x = czero();
    if (xrow0 + r < N && k0 + k < N) x = ldcg4(A + (size_t)(xrow0 + r) * N + k0 + k);
    Xp[0][r][k] = x.re;
    Xp[1][r][k] = x.im;
    Xp[2][r][k] = df_add_sloppy(x.re, x.im);
  }
  for (int e = threadIdx.x; e < C * NB; e += CS_THREADS) {
    const int k = e / C, c = e % C;
    cdf y = czero();
    if (yrow0 + c < N && k0 + k < N) y = ldcg4(A + (size_t)(yrow0 + c) * N + k0 + k);
    Yp[0][k][c] = y.re;
    Yp[1][k][c] = y.im;
    Yp[2][k][c] = df_add_sloppy(y.re, df_neg(y.im));
  }
  __syncthreads();
  const int r = threadIdx.x / C, c = threadIdx.x % C;
  acc2 p1 = acc_zero(), p2 = acc_zero(), p3 = acc_zero();
#pragma unroll 8
  for (int k = 0; k < NB; ++k) {
    acc_prod_df(p1, Xp[0][r][k], Yp[0][k][c]);
    acc_prod_df(p2, Xp[1][r][k], Yp[1][k][c]);
    acc_prod_df(p3, Xp[2][r][k], Yp[2][k][c]);
  }
  __syncthreads();
  return cdf_sub(a, kara_val(p1, p2, p3));
}

// Trailing tile (rb, cb), cb <= rb: A_rc -= L_r,jb L_c,jb^H, 2 x 2 outputs per thread.
__device__ __forceinline__ void herk_tile(float4* A, int N, int jb, int rb, int cb,
                                          unsigned char* smem) {
  df(*Rp)[NB][NB] = (df(*)[NB][NB])smem;                      // [plane][row][k]
  df(*Cp)[NB][NB] = (df(*)[NB][NB])(smem + 3 * NB * NB * 8);  // [plane][k][col]
  const int k0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += CS_THREADS) {
    const int r = e / NB, m = e % NB;
    cdf a = czero();
    if (rb * NB + r < N && k0 + m < N) a = ldcg4(A + (size_t)(rb * NB + r) * N + k0 + m);
    Rp[0][r][m] = a.re;
    Rp[1][r][m] = a.im;
    Rp[2][r][m] = df_add_sloppy(a.re, a.im);
    // transposed walk for the column tile: conflict-free shared-memory stores
    const int m2 = e / NB, r2 = e % NB;
    cdf b = czero();
    if (cb * NB + r2 < N && k0 + m2 < N) b = ldcg4(A + (size_t)(cb * NB + r2) * N + k0 + m2);
    Cp[0][m2][r2] = b.re;
    Cp[1][m2][r2] = b.im;
    Cp[2][m2][r2] = df_add_sloppy(b.re, df_neg(b.im));
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  acc2 acc[3][2][2];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) acc[p][r][c] = acc_zero();
#pragma unroll 4
  for (int m = 0; m < NB; ++m) {
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const df a0 = Rp[p][ty][m], a1 = Rp[p][ty + 16][m];
      const df b0 = Cp[p][m][tx], b1 = Cp[p][m][tx + 16];
      acc_prod_df(acc[p][0][0], a0, b0);
      acc_prod_df(acc[p][0][1], a0, b1);
      acc_prod_df(acc[p][1][0], a1, b0);
      acc_prod_df(acc[p][1][1], a1, b1);
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int gr = rb * NB + ty + 16 * r, gc = cb * NB + tx + 16 * c;
      if (gr < N && gc < N && gc <= gr) {
        float4* p = A + (size_t)gr * N + gc;
        *p = st4(cdf_sub(ldcg4(p), kara_val(acc[0][r][c], acc[1][r][c], acc[2][r][c])));
      }
    }
}

// Factor diagonal block jp in place: L L^H = A_jp,jp (lower triangle), reciprocal pivots to inv.
// Warp 7 runs the pivot chain: at step s it takes column s+1 as left by step s-1 (all columns up to
// s-1 applied), applies column s itself, forms the pivot d = a_{s+1,s+1}, y = 1/sqrt(d) (one
// refinement step) and publishes l_{.,s+1} = a_{.,s+1} y.  Warps 0..6 own the entries of columns
// >= 2 in column-descending order, so the entries that step s must update (columns >= s+2) are a
// prefix of that order and idle warps skip the step; each entry keeps A and a compensated
// accumulator of sum_k l_rk conj(l_qk) in registers, and the entries of column s+2 hand their
// value to the pivot warp through a double-buffered shared-memory row.  One barrier per column.
constexpr int PW_BULK = 7 * 32;
constexpr int PW_PAIRS = (NB - 2) * (NB - 1) / 2;                  // entries of columns 2..31
constexpr int PW_SLOTS = (PW_PAIRS + PW_BULK - 1) / PW_BULK;

__device__ __forceinline__ void potrf_task(int N, float4* A, float2* inv, int jp, int* status,
                                           unsigned char* smem) {
  cdf* col = (cdf*)smem;                   // col[c * 32 + r] = l_rc, r >= c
  cdf* pend = col + NB * NB;               // [2][32]: column handed to the pivot warp
  df* yv = (df*)(pend + 2 * NB);           // 1 / sqrt(d_c)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = jp * NB;
  const df zero = df_make(0.f, 0.f), one = df_make(1.f, 0.f);
  auto load = [&](int r, int q) -> cdf {
    if (r0 + r < N) return ldcg4(A + (size_t)(r0 + r) * N + r0 + q);
    return cdf_make(r == q ? one : zero, zero);
  };
  if (warp == 7) {
    // pivot warp: columns 0 and 1 straight from A
    const cdf a0 = load(lane, 0);
    cdf a1 = lane >= 1 ? load(lane, 1) : czero();
    df d;
    d.h = __shfl_sync(0xffffffffu, a0.re.h, 0);
    d.l = __shfl_sync(0xffffffffu, a0.re.l, 0);
    if (!(d.h > 0.f)) {
      if (lane == 0) set_flag(status, ST_CHOL);
      d = one;
    }
    const df y = df_rsqrt1(d);
    col[lane] = lane == 0 ? cdf_make(df_mul(d, y), zero) : cdf_scale(a0, y);
    if (lane == 0) yv[0] = y;
    pend[NB + lane] = a1;                  // column 1, nothing applied yet (parity 1)
  }
  // bulk entries: column-descending order over columns 31..2, column q holds rows q..31
  int er[PW_SLOTS], eq[PW_SLOTS];
  cdf av[PW_SLOTS];
  cacc acc[PW_SLOTS];
#pragma unroll
  for (int i = 0; i < PW_SLOTS; ++i) {
    int e = threadIdx.x + i * PW_BULK, q = NB - 1;
    while (q > 2 && e >= NB - q) { e -= NB - q; --q; }
    const bool on = warp < 7 && threadIdx.x + i * PW_BULK < PW_PAIRS;
    er[i] = on ? q + e : -1;
    eq[i] = q;
    av[i] = on ? load(q + e, q) : czero();
    acc[i] = cacc_zero();
  }
  __syncthreads();
  for (int s = 0; s < NB - 1; ++s) {
    if (warp == 7) {
      // column s+1: v = (value through column s-1) - l_{r,s} conj(l_{s+1,s}), then its pivot
      const int c = s + 1;
      const cdf w = pend[(c & 1) * NB + lane];
      const cdf lr = col[s * NB + lane];
      const cdf lq = col[s * NB + c];
      const cdf v = cdf_sub_sloppy(w, cdf_mul_conj(lr, lq));
      df d;
      d.h = __shfl_sync(0xffffffffu, v.re.h, c);
      d.l = __shfl_sync(0xffffffffu, v.re.l, c);
      if (!(d.h > 0.f)) {
        if (lane == 0) set_flag(status, ST_CHOL);
        d = one;
      }
      const df y = df_rsqrt1(d);
      if (lane > c) col[c * NB + lane] = cdf_scale(v, y);
      else if (lane == c) col[c * NB + c] = cdf_make(df_mul(d, y), zero);
      if (lane == 0) yv[c] = y;
    } else if (warp * 32 < (NB - 2 - s) * (NB - 1 - s) / 2) {
      // entries of columns >= s+2 (the first (30-s)(31-s)/2 of the order) take column s
      const int nact = (NB - 2 - s) * (NB - 1 - s) / 2;
      const cdf* cs = col + s * NB;
#pragma unroll
      for (int i = 0; i < PW_SLOTS; ++i) {
        if (threadIdx.x + i * PW_BULK < nact) {
          const int r = er[i], q = eq[i];
          cacc_mulc(acc[i], cs[r], cs[q]);
          if (q == s + 2) pend[(q & 1) * NB + r] = cdf_sub_sloppy(av[i], cacc_val(acc[i]));
        }
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NB * NB; e += CS_THREADS) {
    const int q = e / NB, r = e % NB;
    if (r >= q && r0 + r < N) A[(size_t)(r0 + r) * N + r0 + q] = st4(col[q * NB + r]);
  }
  if (threadIdx.x < NB && r0 + threadIdx.x < N)
    inv[r0 + threadIdx.x] = make_float2(yv[threadIdx.x].h, yv[threadIdx.x].l);
}

// D = L^{-1} of diagonal block jp (final), by 2 x 2 blocks of 16:
//   D11 = L11^{-1}, D22 = L22^{-1} (forward substitution of the unit vectors, one column per
//   half-warp, compensated accumulation), then D21 = -D22 (L21 D11) as two 16 x 16 products.
__device__ __forceinline__ void trtri_task(int N, const float4* A, const float2* inv, float4* D,
                                           int jp, unsigned char* smem) {
  constexpr int H = NB / 2;
  cdf(*Ls)[NB + 1] = (cdf(*)[NB + 1])smem;                                  // [32][33]
  cdf(*Ds)[NB + 1] = (cdf(*)[NB + 1])(smem + NB * (NB + 1) * 16);           // [32][33]
  cdf(*Ts)[H + 1] = (cdf(*)[H + 1])(smem + 2 * NB * (NB + 1) * 16);         // [16][17]
  df* ys = (df*)(smem + 2 * NB * (NB + 1) * 16 + H * (H + 1) * 16);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = jp * NB;
  const df zero = df_make(0.f, 0.f), one = df_make(1.f, 0.f);
  for (int e = threadIdx.x; e < NB * NB; e += CS_THREADS) {
    const int r = e / NB, c = e % NB;
    Ls[r][c] = (c < r && r0 + r < N) ? ldcg4(A + (size_t)(r0 + r) * N + r0 + c) : czero();
  }
  if (threadIdx.x < NB) {
    const float2 v = r0 + threadIdx.x < N ? __ldcg(inv + r0 + threadIdx.x) : make_float2(1.f, 0.f);
    ys[threadIdx.x] = df_make(v.x, v.y);
  }
  __syncthreads();
  // the 32 unit-vector solves (block b, column j) in two passes of 16 half-warps; rows above j
  // come out as zero by themselves (right-hand side and accumulator are zero there)
  const int hl = lane & (H - 1);
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int sp = 2 * warp + (lane >> 4) + H * pass;
    const int b = sp / H, j = sp % H, o = b * H;
    cacc acc = cacc_zero();
    cdf dv = czero();
    for (int k = 0; k < H; ++k) {
      const cdf v = cdf_scale(cdf_sub(cdf_make(k == j ? one : zero, zero), cacc_val(acc)), ys[o + k]);
      cdf bk;
      bk.re.h = __shfl_sync(0xffffffffu, v.re.h, k, H);
      bk.re.l = __shfl_sync(0xffffffffu, v.re.l, k, H);
      bk.im.h = __shfl_sync(0xffffffffu, v.im.h, k, H);
      bk.im.l = __shfl_sync(0xffffffffu, v.im.l, k, H);
      if (hl == k) dv = bk;
      if (hl > k) cacc_mul(acc, Ls[o + hl][o + k], bk);
    }
    Ds[o + hl][o + j] = dv;
    Ds[o + hl][H - o + j] = czero();      // the other 16 columns of these rows: D12 = 0 / D21 later
  }
  __syncthreads();
  // T = L21 D11, then D21 = -D22 T
  const int r = threadIdx.x / H, c = threadIdx.x % H;
  cacc t = cacc_zero();
#pragma unroll 4
  for (int m = 0; m < H; ++m) cacc_mul(t, Ls[H + r][m], Ds[m][c]);
  Ts[r][c] = cacc_val(t);
  __syncthreads();
  cacc u = cacc_zero();
#pragma unroll 4
  for (int m = 0; m < H; ++m) cacc_mul(u, Ds[H + r][H + m], Ts[m][c]);
  const cdf d21 = cacc_val(u);
  Ds[H + r][c] = cdf_make(df_neg(d21.re), df_neg(d21.im));
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += CS_THREADS) {
    const int rr = e / NB, cc = e % NB;
    if (r0 + rr < N) D[((size_t)jp * NB + rr) * NB + cc] = st4(Ds[rr][cc]);
  }
}

// Control words of one factorisation call (zeroed before its first launch), per matrix m:
//   ctl[li]                          ticket counter of launch li
//   diag  [li][m]  at (T+2) + 2 li   finished quadrant updates of diagonal block li
//   pdone [li][m]  at 3(T+2) + 2 li  diagonal factor of block li published
//   slabdone[m][l][b]                finished 8-row panel slabs of launch l in row block b
//   tilecnt [m][r][c]                trailing updates applied to tile (r, c)
// Tasks wait (bounded) on these rather than on the end of the previous launch, so the chain of
// block column li + 1 (quadrants -> diagonal factor -> panel) overlaps the trailing updates of
// launch li.
struct CholCtl {
  unsigned *slabdone, *tilecnt;
  int T, N;
  __device__ unsigned* sd(int m, int l, int b) const { return slabdone + ((size_t)m * (T + 1) + l) * T + b; }
  __device__ unsigned* tc(int m, int r, int c) const { return tilecnt + ((size_t)m * T + r) * T + c; }
  __device__ unsigned slabs_in(int b) const {
    const int rows = N - b * NB < NB ? N - b * NB : NB;
    return (unsigned)((rows + TS_ROWS - 1) / TS_ROWS);
  }
};

// thread 0 waits (bounded) until *f >= target, then fences; the caller synchronises the CTA
__device__ __forceinline__ void wait_count(const unsigned* f, unsigned target, int* status) {
  if (threadIdx.x == 0 && target > 0) {
    cs_wait(f, target, status);
    __threadfence();
  }
}

__device__ __forceinline__ void chol_task(int N, Batch mb, int nb, int li, unsigned* ctl,
                                          int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ unsigned s_t;
  const int T = (N + NB - 1) / NB;
  const int jp = li, jb = li - 1;
  unsigned* diag = ctl + (T + 2) + 2 * li;     // [li][matrix]: finished quadrants
  unsigned* pdone = ctl + 3 * (T + 2) + 2 * li;  // [li][matrix]: diagonal factor published
  CholCtl cc;
  cc.slabdone = ctl + 5 * (T + 2);
  cc.tilecnt = cc.slabdone + 2 * (size_t)(T + 1) * T;
  cc.T = T;
  cc.N = N;
  if (threadIdx.x == 0) s_t = atomicAdd(ctl + li, 1u);
  __syncthreads();
  int t = (int)s_t;
  const int ndiag = (jb >= 0 && jp < T) ? 3 : 0;
  const int rt = T - jb - 2;
  const int nherk = (jb >= 0 && rt > 0) ? rt * (rt + 1) / 2 : 0;
  const int rows = N - (jp + 1) * NB;
  const int nslab = (jp < T && rows > 0) ? (rows + TS_ROWS - 1) / TS_ROWS : 0;
  if (t < nb * ndiag) {
    // quadrant (rh, ch) of diagonal block jp: A -= L_jp,jb L_jp,jb^H; needs panel jb on the rows
    // of block jp and the jb earlier trailing updates of the diagonal tile
    const int m = t % nb, qd = t / nb;
    const int rh = qd > 0 ? 1 : 0, ch = qd > 1 ? 1 : 0;
    wait_count(cc.sd(m, jb, jp), cc.slabs_in(jp), status);
    wait_count(cc.tc(m, jp, jp), (unsigned)jb, status);
    __syncthreads();
    float4* A = pick2(mb.m, m);
    const int r = threadIdx.x / 16, c = threadIdx.x % 16;
    const int orow = jp * NB + rh * 16 + r, ocol = jp * NB + ch * 16 + c;
    const bool ok = orow < N && ocol < N && (rh != ch || c <= r);
    const cdf v = upd_one<16, 16>(A, N, jp * NB + rh * 16, jp * NB + ch * 16, jb * NB, orow, ocol,
                                  ok, sm);
    if (ok) A[(size_t)orow * N + ocol] = st4(v);
    cs_signal(diag + m);
    return;
  }
  t -= nb * ndiag;
  const int npotrf = jp < T ? 1 : 0;
  if (t < nb * npotrf) {
    const int m = t;
    if (ndiag > 0) {
      if (threadIdx.x == 0) {
        cs_wait(diag + m, 3u, status);
        __threadfence();
      }
      __syncthreads();
    }
    potrf_task(N, pick2(mb.m, m), pick2(mb.inv, m), jp, status, sm);
    cs_signal(pdone + m);
    return;
  }
  t -= nb * npotrf;
  const int ntrtri = jp >= 1 ? 1 : 0;
  if (t < nb * ntrtri) {
    // inverse of the previous diagonal block (final once its factor is published), for the solves
    const int m = t;
    wait_count(ctl + 3 * (T + 2) + 2 * (li - 1) + m, 1u, status);
    __syncthreads();
    trtri_task(N, pick2(mb.m, m), pick2(mb.inv, m), pick2(mb.D, m), jp - 1, sm);
    return;
  }
  t -= nb * ntrtri;
  if (t < nb * nherk) {
    const int m = t % nb;
    int I, J;
    tri_index(t / nb, I, J);
    const int rb = jb + 2 + J, cb = jb + 2 + I;
    // panel jb on both row blocks, and the tile's jb - 1 earlier updates
    wait_count(cc.sd(m, jb, rb), cc.slabs_in(rb), status);
    wait_count(cc.sd(m, jb, cb), cc.slabs_in(cb), status);
    wait_count(cc.tc(m, rb, cb), (unsigned)(jb > 0 ? jb : 0), status);
    __syncthreads();
    herk_tile(pick2(mb.m, m), N, jb, rb, cb, sm);
    cs_signal(cc.tc(m, rb, cb));
    return;
  }
  t -= nb * nherk;
  if (t < nb * nslab) {
    // panel slab: rows i0..i0+7 of block column jp.  a = A - L_i,jb L_jp,jb^H, then x L^H = a by
    // substitution along the row (warp = row, lane = column): x_m = (a_m - sum_k<m x_k conj(L_mk)) / L_mm
    const int m = t % nb, sl = t / nb;
    float4* A = pick2(mb.m, m);
    const float2* inv = pick2(mb.inv, m);
    const int i0 = (jp + 1) * NB + sl * TS_ROWS;
    const int r = threadIdx.x / NB, c = threadIdx.x % NB;
    const bool ok = i0 + r < N;
    const int bi = i0 / NB;
    if (jb >= 0) {
      // panel jb on these rows and on the rows of block jp, and the tile's jb earlier updates
      wait_count(cc.sd(m, jb, bi), cc.slabs_in(bi), status);
      wait_count(cc.sd(m, jb, jp), cc.slabs_in(jp), status);
      wait_count(cc.tc(m, bi, jp), (unsigned)jb, status);
      __syncthreads();
    }
    cdf a;
    if (jb >= 0) a = upd_one<TS_ROWS, NB>(A, N, i0, jp * NB, jb * NB, i0 + r, jp * NB + c, ok, sm);
    else a = ok ? ldcg4(A + (size_t)(i0 + r) * N + jp * NB + c) : czero();
    if (threadIdx.x == 0) {
      cs_wait(pdone + m, 1u, status);
      __threadfence();
    }
    __syncthreads();
    // with L' = L diag(y) (y_k = 1 / L_kk) and x = z diag(y): z_k = a_k - sum_j<k z_j conj(L'_kj),
    // so the chain carries no scaling; L' is formed while staging the block
    cdf(*Ls)[NB + 1] = (cdf(*)[NB + 1])sm;                      // [32][33]
    df* ys = (df*)(sm + NB * (NB + 1) * 16);
    if (threadIdx.x < NB) {
      const float2 v = __ldcg(inv + jp * NB + threadIdx.x);
      ys[threadIdx.x] = df_make(v.x, v.y);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NB * NB; e += CS_THREADS) {
      const int rr = e / NB, cc = e % NB;
      Ls[rr][cc] = cc < rr ? cdf_scale(ldcg4(A + (size_t)(jp * NB + rr) * N + jp * NB + cc), ys[cc])
                           : czero();
    }
    __syncthreads();
    cacc s = cacc_zero();
    cdf z = czero();
    cdf lnext = Ls[c][0];
#pragma unroll 4
    for (int k = 0; k < NB; ++k) {
      const cdf lk = lnext;
      if (k + 1 < NB) lnext = Ls[c][k + 1];   // next step's operand, off the chain
      const cdf zk = shfl_cdf(cdf_sub_sloppy(a, cacc_val(s)), k);
      if (c == k) z = zk;
      if (c > k) cacc_mulc(s, zk, lk);
    }
    if (ok) {
      const cdf x = cdf_scale(z, ys[c]);
      A[(size_t)(i0 + r) * N + jp * NB + c] = st4(x);
      // L^H in the (otherwise unused) upper triangle: the backward solve reads it by rows
      A[(size_t)(jp * NB + c) * N + i0 + r] = st4(cdf_make(x.re, df_neg(x.im)));
    }
    cs_signal(cc.sd(m, li, bi));
  }
}

__global__ void __launch_bounds__(CS_THREADS, 3) k_chol_step_df(int N, Batch mb, int nb, int li,
                                                            unsigned* ctl, int* status) {
  // programmatic dependent launch: the next block column's launch may become resident at once;
  // its tasks wait on the control words for exactly the data they read
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  chol_task(N, mb, nb, li, ctl, status);
  // the grid completes only after its predecessor has, so later work in the stream sees the whole
  // factorisation
  if (threadIdx.x == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------- triangular solves

constexpr int TW = 8;
constexpr int CW = 4;
constexpr int CPW = NB / CW;

__device__ __forceinline__ bool wait_flag(const unsigned* f, unsigned epoch, int* status) {
  const unsigned lim = wait_budget(status, WAIT_LIMIT);
  for (unsigned it = 0; it < lim; ++it) {
    if (ld_acquire(f) == epoch) return true;
    if (it > 4096) __nanosleep(64);
  }
  set_flag(status, ST_TIMEOUT);
  return false;
}
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Forward solve L z = y (z published as double-floats, consumers wait on per-block flags).
// Same schedule as the FP64 kernel: warps CW.. accumulate the older blocks, warps 0..CW-1 share the
// critical block jb-1 and the diagonal product with D_jb.
__global__ void __launch_bounds__(TW * 32) k_trsv_lower_df(int N, const float4* __restrict__ L,
                                                          const float4* __restrict__ D,
                                                          const double2* __restrict__ y,
                                                          float4* __restrict__ z, unsigned* flags,
                                                          unsigned* ticket, unsigned epoch,
                                                          int* status) {
  __shared__ cacc part[TW][NB];
  __shared__ cdf Ds[NB][NB + 1];
  __shared__ cdf vsh[NB];
  __shared__ int s_jb;
  if (threadIdx.x == 0) s_jb = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int jb = s_jb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    Ds[r][c] = (r0 + r < N) ? ld4(D[((size_t)jb * NB + r) * NB + c]) : czero();
  }
  const bool row_ok = r0 + lane < N;
  const float4* Lrow = L + (size_t)(row_ok ? r0 + lane : 0) * N;
  cacc acc = cacc_zero();
  for (int m = warp - CW; warp >= CW && m < jb - 1; m += TW - CW) {
    if (lane == 0) wait_flag(flags + m, epoch, status);
    __syncwarp();
    const cdf zm = ldcg4(z + m * NB + lane);
#pragma unroll 8
    for (int c = 0; c < NB; ++c) cacc_mul(acc, ld4(__ldg(Lrow + m * NB + c)), shfl_cdf(zm, c));
  }
  if (warp >= CW) part[warp][lane] = acc;
  const int mc = jb - 1;
  cdf lv[CPW];
#pragma unroll
  for (int q = 0; q < CPW; ++q)
    lv[q] = (warp < CW && mc >= 0) ? ld4(__ldg(Lrow + mc * NB + warp * CPW + q)) : czero();
  // the right-hand side, converted off the chain
  const double2 yv = (warp == 0 && row_ok) ? y[r0 + lane] : make_double2(0.0, 0.0);
  const cdf yc = cdf_make(df_from(yv.x), df_from(yv.y));
  __syncthreads();
  if (warp >= CW) return;
  cacc p = cacc_zero();
  if (mc >= 0) {
    if (lane == 0) wait_flag(flags + mc, epoch, status);
    __syncwarp();
    const cdf zm = ldcg4(z + mc * NB + lane);
#pragma unroll
    for (int q = 0; q < CPW; ++q) cacc_mul(p, lv[q], shfl_cdf(zm, warp * CPW + q));
  }
  part[warp][lane] = p;
  named_sync(1, CW * 32);
  if (warp == 0) {
    cacc s = part[0][lane];
#pragma unroll
    for (int w = 1; w < TW; ++w) s = cacc_merge(s, part[w][lane]);
    vsh[lane] = row_ok ? cdf_sub(yc, cacc_val(s)) : czero();
  }
  named_sync(1, CW * 32);
  cacc o = cacc_zero();
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp * CPW + q;
    cacc_mul(o, Ds[lane][c], vsh[c]);
  }
  part[warp][lane] = o;
  named_sync(1, CW * 32);
  if (warp == 0) {
    cacc s = part[0][lane];
#pragma unroll
    for (int w = 1; w < CW; ++w) s = cacc_merge(s, part[w][lane]);
    if (row_ok) z[r0 + lane] = st4(cacc_val(s));
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0) st_release(flags + jb, epoch);
  }
}

// Backward solve L^H w = z (double-floats), out = w or -i w in FP64.
__global__ void __launch_bounds__(TW * 32) k_trsv_upper_df(int N, const float4* __restrict__ L,
                                                          const float4* __restrict__ D,
                                                          const float4* __restrict__ z,
                                                          double2* __restrict__ w_out, bool minus_i,
                                                          float4* __restrict__ wbuf, unsigned* flags,
                                                          unsigned* ticket, unsigned epoch,
                                                          int* status) {
  __shared__ cacc part[TW][NB];
  __shared__ cdf Ds[NB][NB + 1];
  __shared__ cdf vsh[NB];
  __shared__ int s_jb;
  const int nblk = (N + NB - 1) / NB;
  if (threadIdx.x == 0) s_jb = nblk - 1 - (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int jb = s_jb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = jb * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    Ds[r][c] = (r0 + r < N) ? ld4(D[((size_t)jb * NB + r) * NB + c]) : czero();
  }
  const bool col_ok = r0 + lane < N;
  cacc acc = cacc_zero();
  for (int m = nblk - 1 - (warp - CW); warp >= CW && m >= jb + 2; m -= TW - CW) {
    if (lane == 0) wait_flag(flags + m, epoch, status);
    __syncwarp();
    const cdf wm = (m * NB + lane < N) ? ldcg4(wbuf + m * NB + lane) : czero();
#pragma unroll 8
    for (int c = 0; c < NB; ++c) {
      const cdf l = (m * NB + c < N && col_ok) ? ld4(__ldg(L + (size_t)(m * NB + c) * N + r0 + lane))
                                                 : czero();
      cacc_cmul(acc, l, shfl_cdf(wm, c));
    }
  }
  if (warp >= CW) part[warp][lane] = acc;
  const int mc = jb + 1;
  cdf lv[CPW];
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp * CPW + q;
    lv[q] = (warp < CW && mc < nblk && mc * NB + c < N && col_ok)
                ? ld4(__ldg(L + (size_t)(mc * NB + c) * N + r0 + lane))
                : czero();
  }
  const cdf zc = (warp == 0 && col_ok) ? ld4(z[r0 + lane]) : czero();
  __syncthreads();
  if (warp >= CW) return;
  cacc p = cacc_zero();
  if (mc < nblk) {
    if (lane == 0) wait_flag(flags + mc, epoch, status);
    __syncwarp();
    const cdf wm = (mc * NB + lane < N) ? ldcg4(wbuf + mc * NB + lane) : czero();
#pragma unroll
    for (int q = 0; q < CPW; ++q) cacc_cmul(p, lv[q], shfl_cdf(wm, warp * CPW + q));
  }
  part[warp][lane] = p;
  named_sync(1, CW * 32);
  if (warp == 0) {
    cacc s = part[0][lane];
#pragma unroll
    for (int w = 1; w < TW; ++w) s = cacc_merge(s, part[w][lane]);
    vsh[lane] = col_ok ? cdf_sub(zc, cacc_val(s)) : czero();
  }
  named_sync(1, CW * 32);
  // w_r = sum_c conj(D_cr) v_c
  cacc o = cacc_zero();
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp * CPW + q;
    cacc_cmul(o, Ds[c][lane], vsh[c]);
  }
  part[warp][lane] = o;
  named_sync(1, CW * 32);
  if (warp == 0) {
    cacc s = part[0][lane];
#pragma unroll
    for (int w = 1; w < CW; ++w) s = cacc_merge(s, part[w][lane]);
    const cdf wv = cacc_val(s);
    if (col_ok) wbuf[r0 + lane] = st4(wv);
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0) st_release(flags + jb, epoch);
    if (col_ok) {
      const double re = df_to(wv.re), im = df_to(wv.im);
      w_out[r0 + lane] = minus_i ? make_double2(im, -re) : make_double2(re, im);
    }
  }
}

// ---------------------------------------------------------------------------- cluster solve

// Both triangular solves of one RK4 stage in a single launch of one 8-CTA thread-block cluster.
// Every CTA keeps the whole forward solution z and backward solution w in its shared memory.
// CTA rank r owns block rows jb = r, r + 8, ...; when it finishes a block, the 32 values go from
// registers into all eight CTAs' shared memory by st.async, completing the transaction count of
// the receiver's per-block mbarrier, so consumers wait on a local barrier instead of polling
// global memory.  The loops are block-major: on the arrival of block m every CTA adds that block's
// products to all of its pending rows, and finishes its own row m + 1 (forward) / m - 1 (backward)
// as soon as the block it depends on is in.  Products use compensated double-float dot products;
// a block is spread as 8 warps x 4 rows, 8 lanes per row with 4 columns each, so the sums over a
// row are 3 shuffle steps and the critical path has a single CTA barrier per block.
constexpr int CL = 8;          // CTAs per cluster
constexpr int CRPC = 8;        // maximum block rows per CTA (N <= CL * CRPC * 32 = 2048)
constexpr int CTH = 256;       // threads per CTA
constexpr unsigned long long CWAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t s_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtime_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init_c(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_c(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test_c(uint64_t* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(s_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for phase 0 of a local block barrier
__device__ __forceinline__ bool block_wait(uint64_t* b, volatile int* abort_flag, int* status) {
  const unsigned long long t0 = gtime_ns();
  while (!mbar_test_c(b, 0u)) {
    if (*abort_flag) return false;
    if (gtime_ns() - t0 > CWAIT_NS) {
      *abort_flag = 1;
      set_flag(status, ST_TIMEOUT);
      return false;
    }
  }
  return true;
}
// store 16 bytes into CTA `rank`'s shared memory (the address is this CTA's twin of it) and
// complete 16 bytes of the transaction count of that CTA's barrier `bar`
__device__ __forceinline__ void st_async16(float4 v, const void* dst_local, uint64_t* bar_local,
                                           uint32_t rank) {
  const uint32_t dst = map_rank(s_u32(dst_local), rank);
  const uint32_t bar = map_rank(s_u32(bar_local), rank);
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
      ::"r"(dst), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
      : "memory");
}

// Shared-memory layout of the cluster solve (per CTA).
struct CLayout {
  float4* zs;        // nblk*32 forward solution
  float4* ws;        // nblk*32 backward solution
  float4* yown;      // CRPC*32 right-hand side of the own rows (double-floats)
  cdf* vsh;          // 32: right-hand side minus products, for the diagonal-block product
  cacc* acc;         // [CRPC][CTH]: each thread's partial sums of the own block rows
  uint64_t* barF;    // nblk
  uint64_t* barB;    // nblk
  int* abort_flag;
};
__host__ __device__ inline size_t clayout_bytes(int nblk) {
  return (size_t)(2 * nblk + CRPC + 1) * NB * 16 + (size_t)CRPC * CTH * sizeof(cacc) +
         (size_t)2 * nblk * 8 + 16;
}
__device__ __forceinline__ CLayout clayout(unsigned char* base, int nblk) {
  CLayout c;
  c.zs = (float4*)base;
  c.ws = c.zs + nblk * NB;
  c.yown = c.ws + nblk * NB;
  c.vsh = (cdf*)(c.yown + CRPC * NB);
  c.acc = (cacc*)(c.vsh + NB);
  c.barF = (uint64_t*)(c.acc + CRPC * CTH);
  c.barB = c.barF + nblk;
  c.abort_flag = (int*)(c.barB + nblk);
  return c;
}

// Sum over the 8 lanes of a row group (lane bits 0..2): every lane gets the same value, since the
// compensated merge is symmetric in its operands.
__device__ __forceinline__ cacc group_sum(cacc a) {
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    cacc b;
    b.re.s = __shfl_xor_sync(0xffffffffu, a.re.s, o);
    b.re.c = __shfl_xor_sync(0xffffffffu, a.re.c, o);
    b.im.s = __shfl_xor_sync(0xffffffffu, a.im.s, o);
    b.im.c = __shfl_xor_sync(0xffffffffu, a.im.c, o);
    a = cacc_merge(a, b);
  }
  return a;
}

// Finish block row m: `mine` is this lane's share (its 4 columns) of the products with all other
// blocks.  The 8 shares of a row are summed by shuffles, subtracted from the right-hand side,
// multiplied by the inverted diagonal block (D_m forward, D_m^H backward; `dk` are this lane's 4
// entries of it, prefetched) and summed again; lane 0 of each row group then stores the value
// straight into all eight CTAs (st.async, completing on their barriers for block m).
template <bool FWD>
__device__ __forceinline__ void finish_block(const CLayout& c, int N, int m, const cacc& mine,
                                             const cdf (&dk)[4], double2* out, bool minus_i) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = warp * 4 + (lane >> 3), c0 = (lane & 7) * 4;
  const int row = m * NB + rb;
  const cdf s = cacc_val(group_sum(mine));
  const cdf rhs = FWD ? ld4(c.yown[(m / CL) * NB + rb]) : ld4(c.zs[row < N ? row : 0]);
  if ((lane & 7) == 0) c.vsh[rb] = row < N ? cdf_sub(rhs, s) : czero();
  __syncthreads();
  cacc o = cacc_zero();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (FWD) cacc_mul(o, dk[q], c.vsh[c0 + q]);
    else cacc_cmul(o, dk[q], c.vsh[c0 + q]);
  }
  const cdf v = cacc_val(group_sum(o));
  if ((lane & 7) == 0) {
    const cdf vv = row < N ? v : czero();
    const float4 f = st4(vv);
    float4* dst = (FWD ? c.zs : c.ws) + row;
    uint64_t* bar = (FWD ? c.barF : c.barB) + m;
    if (!*(volatile int*)c.abort_flag) {
#pragma unroll
      for (uint32_t r = 0; r < CL; ++r) st_async16(f, dst, bar, r);
    }
    if (!FWD && row < N) {
      const double re = df_to(vv.re), im = df_to(vv.im);
      out[row] = minus_i ? make_double2(im, -re) : make_double2(re, im);
    }
  }
}

__device__ __forceinline__ void pf_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Waits for block m on a local barrier; the outcome is made uniform over the CTA.
__device__ __forceinline__ bool cta_wait_block(const CLayout& c, uint64_t* bar, int* status) {
  const bool ok = block_wait(bar, (volatile int*)c.abort_flag, status);
  return !__syncthreads_or(!ok);
}

__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(CTH, 1)
k_chol_solve_cluster(int N, const float4* __restrict__ L, const float4* __restrict__ D,
                     const double2* __restrict__ y, double2* __restrict__ out, bool minus_i,
                     int* status) {
  extern __shared__ __align__(128) unsigned char csm[];
  const int nblk = (N + NB - 1) / NB;
  const CLayout c = clayout(csm, nblk);
  const int rank = (int)cluster_rank();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = warp * 4 + (lane >> 3);     // this lane's row within a block
  const int c0 = (lane & 7) * 4;             // and its 4 columns

  if (threadIdx.x == 0) {
    for (int m = 0; m < nblk; ++m) {
      mbar_init_c(c.barF + m, 1);
      mbar_init_c(c.barB + m, 1);
    }
    *c.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int m = 0; m < nblk; ++m) {
      mbar_expect_c(c.barF + m, 512u);
      mbar_expect_c(c.barB + m, 512u);
    }
  }
  // right-hand side of the own rows, converted to double-floats once
  for (int e = threadIdx.x; e < CRPC * NB; e += CTH) {
    const int row = (rank + CL * (e / NB)) * NB + e % NB;
    const double2 yv = row < N ? y[row] : make_double2(0.0, 0.0);
    c.yown[e] = st4(cdf_make(df_from(yv.x), df_from(yv.y)));
  }
  __syncthreads();
  cluster_sync();

  // the partial sums live in shared memory, so the loops over own rows stay rolled (code size:
  // the critical path must not miss in the instruction cache after each accumulation sweep)
  cacc* acc = c.acc + threadIdx.x;           // acc[i * CTH]
  cdf dk[4], lk[4];
  // ------------------------------------------------ forward: L z = y
  for (int i = 0; i < CRPC; ++i) acc[i * CTH] = cacc_zero();
  bool alive = true;
  // m = -1 only finishes block 0 (no products); each finish has a single call site per pass
  for (int m = -1; m < nblk; ++m) {
    const int mc = m + 1;
    const bool crit = mc < nblk && mc % CL == rank;
    if (crit) {
      // prefetch the critical row's operands before the wait: L[mc, m] and D_mc
      const int row = mc * NB + rb;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        lk[q] = (m >= 0 && row < N) ? ld4(__ldg(L + (size_t)row * N + m * NB + c0 + q)) : czero();
        dk[q] = row < N ? ld4(__ldg(D + (size_t)row * NB + c0 + q)) : czero();
      }
    }
    cdf zc[4];
    if (m >= 0) {
      if (!cta_wait_block(c, c.barF + m, status)) { alive = false; break; }
#pragma unroll
      for (int q = 0; q < 4; ++q) zc[q] = ld4(c.zs[m * NB + c0 + q]);
    }
    if (crit) {
      cacc mine = acc[(mc / CL) * CTH];
      if (m >= 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) cacc_mul(mine, lk[q], zc[q]);
      }
      finish_block<true>(c, N, mc, mine, dk, out, minus_i);
    }
    if (m < 0) continue;
    // the remaining own rows jb > m + 1: acc += L[jb, m] z_m
#pragma unroll 1
    for (int i = (mc + 1 - rank + CL - 1) / CL; i < CRPC; ++i) {
      const int jb = rank + CL * i;
      const int row = jb * NB + rb;
      if (jb >= nblk || row >= N) break;
      const float4* lp = L + (size_t)row * N + m * NB + c0;
      cacc a = acc[i * CTH];
#pragma unroll
      for (int q = 0; q < 4; ++q) cacc_mul(a, ld4(__ldg(lp + q)), zc[q]);
      acc[i * CTH] = a;
      // the next block's operands of this row, into L1 while the CTA waits for that block
      if (jb > mc + 1) pf_l1(lp + NB);
    }
    // operands of this CTA's next critical step (block m + 2 at the next arrival) into L1 now:
    // that step starts right after its block arrives, too soon to wait for L2
    if (m + 2 < nblk && (m + 2) % CL == rank) {
      const int row = (m + 2) * NB + rb;
      if (row < N) {
        pf_l1(L + (size_t)row * N + (m + 1) * NB + c0);
        pf_l1(D + (size_t)row * NB + c0);
      }
    }
  }
  // ------------------------------------------------ backward: L^H w = z
  if (alive) {
    for (int i = 0; i < CRPC; ++i) acc[i * CTH] = cacc_zero();
    // m = nblk only finishes the last block
    for (int m = nblk; m >= 0; --m) {
      const int mc = m - 1;
      const bool crit = mc >= 0 && mc % CL == rank;
      if (crit) {
        // (L^H)[mc, m] from the upper triangle (row mc*32 + rb, columns c0.. of block m) and D_mc^H
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rm = m * NB + c0 + q;
          const int rd = mc * NB + c0 + q;
          lk[q] = (m < nblk && rm < N) ? ld4(__ldg(L + (size_t)(mc * NB + rb) * N + rm)) : czero();
          dk[q] = rd < N ? ld4(__ldg(D + (size_t)rd * NB + rb)) : czero();
        }
      }
      cdf wc[4];
      if (m < nblk) {
        if (!cta_wait_block(c, c.barB + m, status)) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) wc[q] = ld4(c.ws[m * NB + c0 + q]);
      }
      if (crit) {
        cacc mine = acc[(mc / CL) * CTH];
        if (m < nblk) {
#pragma unroll
          for (int q = 0; q < 4; ++q) cacc_mul(mine, lk[q], wc[q]);
        }
        finish_block<false>(c, N, mc, mine, dk, out, minus_i);
      }
      if (m >= nblk) continue;
      // the remaining own rows jb < m - 1: acc += (L^H)[jb, m] w_m, read by rows of the upper triangle
#pragma unroll 1
      for (int i = 0; i < CRPC; ++i) {
        const int jb = rank + CL * i;
        if (jb >= mc) break;
        const float4* up = L + (size_t)(jb * NB + rb) * N + m * NB + c0;
        cacc a = acc[i * CTH];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (m * NB + c0 + q < N) cacc_mul(a, ld4(__ldg(up + q)), wc[q]);
        acc[i * CTH] = a;
        if (jb < mc - 1) pf_l1(up - NB);   // the next block's operands of this row
      }
      // operands of this CTA's next critical step (block m - 2) into L1
      if (m - 2 >= 0 && (m - 2) % CL == rank) {
        pf_l1(L + (size_t)((m - 2) * NB + rb) * N + (m - 1) * NB + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) pf_l1(D + (size_t)((m - 2) * NB + c0 + q) * NB + rb);
      }
    }
  }
  __syncthreads();
  cluster_sync();
  if (*(volatile int*)c.abort_flag) {
    // a wait gave up: stores from other CTAs may still be landing in this CTA's shared memory,
    // which outlives none of them only after they complete; they take microseconds, so linger
    const unsigned long long t0 = gtime_ns();
    while (gtime_ns() - t0 < 200000ull) {
    }
  }
}

size_t cluster_solve_smem(int N) { return clayout_bytes((N + NB - 1) / NB); }

}  // namespace dfs

// ---------------------------------------------------------------------------- launchers

void launch_shift_mix_df(int N, const double2* S0, const double2* S1, double eps, double theta,
                         void* A, cudaStream_t s) {
  dfs::k_shift_mix_df<<<N, 256, 0, s>>>(N, S0, S1, eps, theta, (float4*)A);
}

int launch_cholesky_df(int N, void* const* A, void* const* inv, void* const* D, int nbatch,
                       unsigned* ctl, int* status, cudaStream_t s) {
  using namespace dfs;
  Batch mb;
  for (int q = 0; q < 2; ++q) {
    const int k = (nbatch > 1 && q == 1) ? 1 : 0;
    mb.m[q] = (float4*)A[k];
    mb.inv[q] = (float2*)inv[k];
    mb.D[q] = (float4*)D[k];
  }
  const int T = (N + NB - 1) / NB;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_chol_step_df, cudaFuncAttributeMaxDynamicSharedMemorySize, CS_SMEM_LAUNCH);
    attr = true;
  }
  cudaMemsetAsync(ctl, 0, chol_ctl_words(N) * sizeof(unsigned), s);
  // launches 1.. are programmatic dependents of the previous one (the kernel waits on
  // griddepcontrol before touching data), so a launch's CTAs are resident when its predecessor
  // ends instead of paying the launch latency on the factorisation's critical path
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  for (int li = 0; li <= T; ++li) {
    const int jb = li - 1;
    const int rt = T - jb - 2;
    const int nherk = (jb >= 0 && rt > 0) ? rt * (rt + 1) / 2 : 0;
    const int rows = N - (li + 1) * NB;
    const int nslab = (li < T && rows > 0) ? (rows + TS_ROWS - 1) / TS_ROWS : 0;
    const int per = (jb >= 0 && li < T ? 3 : 0) + (li < T ? 1 : 0) + (li >= 1 ? 1 : 0) + nherk + nslab;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nbatch * per);
    cfg.blockDim = dim3(CS_THREADS);
    cfg.dynamicSmemBytes = CS_SMEM_LAUNCH;
    cfg.stream = s;
    cfg.attrs = pdl;
    cfg.numAttrs = li > 0 ? 1 : 0;   // the first launch follows the memset in stream order
    cudaLaunchKernelEx(&cfg, k_chol_step_df, N, mb, nbatch, li, ctl, status);
  }
  return T + 2;
}

size_t chol_ctl_words(int N) {
  const size_t T = (N + dfs::NB - 1) / dfs::NB;
  return 5 * (T + 2) + 2 * (T + 1) * T + 2 * T * T;
}

void launch_chol_solve_df(int N, const void* L, const void* D, const double2* y, void* work,
                          double2* out, bool minus_i, unsigned* flags, unsigned* tickets,
                          unsigned epoch, int* status, cudaStream_t s) {
  using namespace dfs;
  const int nblk = (N + NB - 1) / NB;
  if (nblk <= CL * CRPC) {
    // one 8-CTA cluster, both passes in one launch
    const size_t sm = cluster_solve_smem(N);
    static size_t sm_set = 0;
    if (sm > sm_set) {
      cudaFuncSetAttribute(k_chol_solve_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cluster_solve_smem(CL * CRPC * NB));
      sm_set = cluster_solve_smem(CL * CRPC * NB);
    }
    k_chol_solve_cluster<<<CL, CTH, sm, s>>>(N, (const float4*)L, (const float4*)D, y, out, minus_i,
                                             status);
    return;
  }
  // block flags and tickets (which follow them) start from zero in every solve, so a captured
  // launch sequence can be replayed with the same epoch
  cudaMemsetAsync(flags, 0, (2 * (size_t)nblk + 2) * sizeof(unsigned), s);
  (void)tickets;
  float4* zb = (float4*)work;
  k_trsv_lower_df<<<nblk, TW * 32, 0, s>>>(N, (const float4*)L, (const float4*)D, y, zb, flags,
                                            flags + 2 * nblk, epoch, status);
  k_trsv_upper_df<<<nblk, TW * 32, 0, s>>>(N, (const float4*)L, (const float4*)D, zb, out, minus_i,
                                            zb + N, flags + nblk, flags + 2 * nblk + 1, epoch, status);
}

}  // namespace icwf
