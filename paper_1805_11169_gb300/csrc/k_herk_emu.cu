// Trailing update of the FP64 blocked Cholesky, A_rc -= L_r,jb L_c,jb^H for the lower triangle
// of the trailing matrix, in emulated FP64 on the sm_103a tensor cores (BF16 digit products with
// exact integer accumulation in TMEM, error-free slicing in the manner of the Ozaki scheme).
//
// Representation.  Every row i of the panel (32 complex FP64 values L_i,k) is scaled by 2^-e_i
// (e_i: the smallest integer with max_k max(|Re|, |Im|) < 2^e_i); each component becomes the
// 64-bit integer X = round(x 2^(63 - e_i)) (integer operations on the FP64 bit pattern, exact up
// to 2^-64 of 2^e_i), and X is cut into D = 7 balanced digits of base B = 2^8 from the top
// (d_1 = round(X / 2^55), then the remainder's next 8 bits, ...), |d_1| <= B, |d_p| <= B/2.
// Digit p is stored as the BF16 value a_p = d_p B^-(p-1) (exact), so
// x = 2^e_i B^-1 sum_p a_p up to 2^-57 of 2^e_i.
//
// Products.  L_r conj(L_c) = 2^(e_r + e_c) B^-2 sum_{p,q} a_p^r conj(a_q^c); the digit pairs of
// levels p + q <= 8 (1-based) are kept: the first dropped level and the digits' own truncation
// together stay below 2^-47 of 2^(e_r + e_c).  A level's sum over K = 32 (64 real products of
// at most 2^15 units each, at most 9 pairs) stays below 2^24 units, so each of the seven kept
// levels is accumulated EXACTLY in its own FP32 accumulator in TMEM.  The epilogue adds the seven
// from the smallest level up, the two smallest in FP32 and the rest in double-float arithmetic
// (about 2^-48 of the result), scales by 2^(e_r + e_c - 16) with integer exponent arithmetic and
// subtracts the result from A in FP64.
//
// Complex products on real MMAs: with P/Q the real/imaginary planes,
//   [Re | Im] += P_r [P_c | -Q_c] + Q_r [Q_c | P_c]
// (M = 128 rows r, N = 64: 32 columns c for Re and Im), so the column operand is stored as the
// planes P, -Q, Q, P (two adjacent 64-row operands) and the row operand as P and Q.  Each digit
// pair takes four MMAs (K = 16 each), 28 pairs in all.
//
// Kernel layout: one CTA per (128-row tile, 32-column tile) of the trailing matrix that meets its
// lower triangle, 576 threads; warp 16 loads the whole K = 32 slice of all digit planes with TMA
// (64-byte rows and swizzle, one stage, 168 KB), warp 17 issues the 112 MMAs, warps 0..15 run the
// epilogue (warp w reads TMEM lanes 32 (w mod 4).. and columns 8 (w div 4)..: four warps per SM
// sub-partition hide each other's dependent chains).  Waits are bounded (2 s): a timeout raises
// the status flag, drains what is in flight and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "df64.cuh"
#include "herk_digits.cuh"
#include "icwf_internal.h"
#include "k_common.cuh"
#include "tc_ptx.cuh"

namespace icwf {
namespace hemu {

using namespace tc;

constexpr int NLEV = 7;                // kept levels p + q = 0..6 (0-based digits)
constexpr int BM = 128;                // rows per CTA (TMEM lanes)
constexpr int BNC = 32;                // columns per CTA
constexpr int ROW = 64;                // bytes per operand row (32 BF16)
constexpr int A_T = BM * ROW;          // 8 KB
constexpr int B_T = PLANES * BNC * ROW;  // 8 KB per digit: P, -Q, Q, P of 32 columns
constexpr int SM_A = DIG * 2 * A_T;    // 112 KB
constexpr int SM_B = DIG * B_T;        // 56 KB
constexpr int SMEM_BYTES = SM_A + SM_B + 1024 + 256;   // + alignment slack, barriers
constexpr int TMEM_COLS = 512;
constexpr int ACC = 2 * BNC;           // [Re | Im]
static_assert(NLEV * ACC <= TMEM_COLS, "accumulators exceed the TMEM allocation");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA exceeded");
constexpr uint32_t IDESC = idesc_mn(0, BM, ACC);
constexpr int EPI_WARPS = 16;          // epilogue warps: 4 TMEM lane quarters x 4 column quarters
constexpr int TMA_WARP = EPI_WARPS, MMA_WARP = EPI_WARPS + 1;
constexpr int EMU_THREADS = (EPI_WARPS + 2) * 32;
constexpr int EPI_COLS = BNC / (EPI_WARPS / 4);   // columns per epilogue warp

struct Maps {
  CUtensorMap a[2], b[2];   // per matrix: 128-row boxes (rows r), 32-row boxes (columns c)
};

struct Args {
  double2* A[2];
  const int* ex[2];         // per-row exponents (absolute row index)
  int N, R0, rpad, nI, nJ;
  int* status;
};

// Digit planes of the panel rows i in [R0, N) of one matrix (one warp per row, lane = column k),
// for panels that were not produced by the FP64 panel solve.
__global__ void __launch_bounds__(256) k_panel_digits(const double2* __restrict__ A0,
                                                      const double2* __restrict__ A1, int N, int jb,
                                                      int rpad, __nv_bfloat16* __restrict__ pl0,
                                                      __nv_bfloat16* __restrict__ pl1,
                                                      int* __restrict__ ex0, int* __restrict__ ex1) {
  const int m = blockIdx.y;
  const double2* A = m ? A1 : A0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = (jb + 1) * NB + blockIdx.x * 8 + warp;
  if (i >= N) return;
  emit_row_digits(A[(size_t)i * N + jb * NB + lane], i, lane, rpad, m ? pl1 : pl0, m ? ex1 : ex0);
}

// x 2^sh as FP64 from an FP32 x by integer arithmetic on the exponent field (FP64 instructions are
// scarce on this GPU): exact while the result is a normal double.  FP32 zeros and subnormals, and
// results below the FP64 normal range, give 0 (such terms sit far below FP64 resolution of the
// products they belong to); NaN and Inf pass through.
__device__ __forceinline__ double f32_scaled(float x, int sh) {
  const uint32_t u = __float_as_uint(x);
  const int ef = (int)((u >> 23) & 0xFFu);
  if (ef == 0xFF) return (double)x;
  const int ed = ef - 127 + 1023 + sh;
  if (ef == 0 || ed <= 0) return 0.0;
  if (ed >= 0x7FF) return x > 0.f ? __longlong_as_double(0x7FF0000000000000ll)
                                  : __longlong_as_double((long long)0xFFF0000000000000ull);
  const uint32_t hi = (u & 0x80000000u) | ((uint32_t)ed << 20) | ((u & 0x7FFFFFu) >> 3);
  const uint32_t lo = (u & 0x7u) << 29;
  return __hiloint2double((int)hi, (int)lo);
}


__global__ void __launch_bounds__(EMU_THREADS, 1) k_herk_emu(Args args, const __grid_constant__ Maps maps) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // linear index over the tiles that meet the lower triangle (some column <= some row): row tile
  // I holds min(4 (I + 1), nJ) column tiles
  const int m = blockIdx.y;
  int I = 0, J = (int)blockIdx.x;
  while (I < args.nI) {
    const int cnt = min((BM / BNC) * (I + 1), args.nJ);
    if (J < cnt) break;
    J -= cnt;
    ++I;
  }
  if (I >= args.nI) return;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + SM_A + SM_B);
  uint64_t* acc_full = full + 1;
  uint64_t* drain = full + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int* ecol = (int*)(tmem_slot + 2);   // exponents of this tile's 32 columns
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = args.N, R0 = args.R0, rpad = args.rpad;
  const int r0 = R0 + I * BM, c0 = R0 + J * BNC;
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(acc_full, 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == TMA_WARP) {
    if (lane == 0) {
      mbar_expect_tx(full, SM_A + SM_B);
      for (int p = 0; p < DIG; ++p) {
        tma_load_2d(smem + (2 * p) * A_T, &maps.a[m], 0, (p * PLANES + 0) * rpad + r0, full);
        tma_load_2d(smem + (2 * p + 1) * A_T, &maps.a[m], 0, (p * PLANES + 2) * rpad + r0, full);
        for (int pi = 0; pi < PLANES; ++pi)
          tma_load_2d(smem + SM_A + p * B_T + pi * BNC * ROW, &maps.b[m], 0,
                      (p * PLANES + pi) * rpad + c0, full);
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      if (mbar_wait(full, 0u, abort_flag, args.status)) {
        fence_after();
        // descriptors of the operand tiles as base + (byte offset >> 4): the start-address field
        // holds address / 16 in its low 14 bits and shared addresses stay below 256 KB
        const uint64_t da = sdesc_sw(smem_u32(smem), 64), db = sdesc_sw(smem_u32(smem + SM_A), 64);
#pragma unroll
        for (int p = 0; p < DIG; ++p) {
#pragma unroll
          for (int q = 0; p + q < NLEV && q < DIG; ++q) {
            const uint32_t acc = tmem + (p + q) * ACC;
            const uint64_t ap = da + ((2 * p) * A_T >> 4), aq = ap + (A_T >> 4);
            const uint64_t bq = db + (q * B_T >> 4);     // rows P | -Q | Q | P of digit q
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint64_t o = kk * 2;                 // 32 bytes (16 BF16 of K) per instruction
              // level p + q starts at its first pair (p = 0)
              mma_desc<0>(acc, ap + o, bq + o, IDESC, (p == 0 && kk == 0) ? 0u : 1u);
              mma_desc<0>(acc, aq + o, bq + (2 * BNC * ROW >> 4) + o, IDESC, 1u);
            }
          }
        }
      }
      mma_commit(acc_full);   // arrives when every issued MMA has completed
      mma_commit(drain);
    }
  } else {
    // epilogue: lane = row r; A[r][c] -= 2^(e_r + e_c - 16) * (sum of the levels)
    const int quarter = warp & 3, cw = (warp >> 2) * EPI_COLS;   // lanes 32 quarter.., columns cw..
    static_assert(EPI_WARPS % 4 == 0 && EPI_COLS % 4 == 0, "epilogue split");
    const int row = quarter * 32 + lane;
    const int r = r0 + row;
    double2* A = args.A[m];
    const int* ex = args.ex[m];
    // lane = row r; GC columns per group.  Loads of A and of the column exponents are issued a
    // group ahead of the stores (a store to A would otherwise order every later load of A behind
    // it), the first group while the MMAs run.
    constexpr int GC = 4;
    double2 av[GC];
    auto load_group = [&](int cg) {
#pragma unroll
      for (int e = 0; e < GC; ++e) {
        const int c = c0 + cw + cg + e;
        const bool in = r < N && c < N && c <= r;
        av[e] = in ? A[(size_t)r * N + c] : make_double2(0.0, 0.0);
      }
    };
    load_group(0);
    const int er = r < N ? ex[r] : 0;
    if (warp == 0) ecol[lane] = c0 + lane < N ? ex[c0 + lane] : 0;   // read after the barrier
    const bool ok = mbar_wait(acc_full, 0u, abort_flag, args.status) && !*abort_flag;
    uint32_t all_ok;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(all_ok)
        : "r"((uint32_t)ok), "n"(EPI_WARPS * 32)
        : "memory");
    if (all_ok) {
      fence_after();
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + cw;
#pragma unroll 1
      for (int cg = 0; cg < EPI_COLS; cg += GC) {
        float v[NLEV][2][GC];
#pragma unroll
        for (int lv = 0; lv < NLEV; ++lv) {
          tmem_ld4(lane_base + lv * ACC + cg, v[lv][0]);
          tmem_ld4(lane_base + lv * ACC + BNC + cg, v[lv][1]);
        }
        tmem_wait_ld();
        double2 out[GC];
#pragma unroll
        for (int e = 0; e < GC; ++e) {
          const int sh = er + ecol[cw + cg + e] - 2 * BETA;
          // the exact level sums, smallest first; the two smallest (below 2^-16 units of level 0)
          // are added in FP32 (rounding below 2^-40 units)
          df re = two_sum(__fadd_rn(v[NLEV - 1][0][e], v[NLEV - 2][0][e]), v[NLEV - 3][0][e]);
          df im = two_sum(__fadd_rn(v[NLEV - 1][1][e], v[NLEV - 2][1][e]), v[NLEV - 3][1][e]);
#pragma unroll
          for (int lv = NLEV - 4; lv >= 0; --lv) {
            re = df_add_f(re, v[lv][0][e]);
            im = df_add_f(im, v[lv][1][e]);
          }
          // hi + lo is exact in FP64 (48 bits), so A - (hi + lo) rounds once
          out[e].x = av[e].x - (f32_scaled(re.h, sh) + f32_scaled(re.l, sh));
          out[e].y = av[e].y - (f32_scaled(im.h, sh) + f32_scaled(im.l, sh));
        }
        if (cg + GC < EPI_COLS) load_group(cg + GC);
#pragma unroll
        for (int e = 0; e < GC; ++e) {
          const int c = c0 + cw + cg + e;
          if (r < N && c < N && c <= r) A[(size_t)r * N + c] = out[e];
        }
      }
    }
  }
  __syncthreads();
  if (warp == MMA_WARP && lane == 0) {
    // an epilogue that gave up early leaves MMAs in flight: let them retire before the dealloc
    const unsigned long long t0 = gtime();
    while (!mbar_test(drain, 0u) && gtime() - t0 < WAIT_NS) {
    }
  }
  if (warp == TMA_WARP && lane == 0 && *abort_flag) {
    // a TMA load that may still be landing: wait (bounded) for the stage's phase
    const unsigned long long t0 = gtime();
    while (!mbar_test(full, 0u) && gtime() - t0 < WAIT_NS) {
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

bool make_map(CUtensorMap* m, void* base, size_t rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)NB, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)NB * 2};
  cuuint32_t box[2] = {(cuuint32_t)NB, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int rpad_for(int N) { return (N + BM - 1) / BM * BM; }

}  // namespace hemu

// The update kernel's shared-memory limit, set once per process by handle creation (outside any
// stream capture, so that no captured launch changes a function attribute).
void herk_emu_attributes() {
  static std::once_flag once;
  std::call_once(once, []() {
    cudaFuncSetAttribute(hemu::k_herk_emu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         hemu::SMEM_BYTES);
  });
}

size_t herk_emu_scratch_bytes(int N) {
  using namespace hemu;
  const size_t rp = (size_t)rpad_for(N);
  const size_t per = ((size_t)DIG * PLANES * rp * NB * 2 + 1023) / 1024 * 1024 + (rp * 4 + 1023) / 1024 * 1024;
  return 2 * per;
}

EmuPlanes herk_emu_planes(int N, void* scratch) {
  using namespace hemu;
  EmuPlanes e;
  e.rpad = rpad_for(N);
  const size_t planes_b = ((size_t)DIG * PLANES * e.rpad * NB * 2 + 1023) / 1024 * 1024;
  const size_t ex_b = ((size_t)e.rpad * 4 + 1023) / 1024 * 1024;
  char* p = (char*)scratch;
  for (int m = 0; m < 2; ++m) {
    e.planes[m] = p; p += planes_b;
    e.ex[m] = (int*)p; p += ex_b;
  }
  return e;
}

bool launch_herk_emu(int N, int jb, double2* const* A, int nbatch, void* scratch, size_t bytes,
                     bool digits_done, int* status, cudaStream_t s) {
  using namespace hemu;
  const int R0 = (jb + 1) * NB;
  const int R = N - R0;
  if (R <= 0) return true;
  if (!scratch || bytes < herk_emu_scratch_bytes(N)) return false;
  const EmuPlanes e = herk_emu_planes(N, scratch);
  const int rp = e.rpad;
  const int nb = nbatch > 1 ? 2 : 1;
  Maps maps;
  for (int m = 0; m < 2; ++m) {
    const int k = m < nb ? m : 0;
    const size_t rows = (size_t)DIG * PLANES * rp;
    if (!make_map(&maps.a[m], e.planes[k], rows, BM) || !make_map(&maps.b[m], e.planes[k], rows, BNC))
      return false;
  }
  if (!digits_done)
    k_panel_digits<<<dim3((R + 7) / 8, nb), 256, 0, s>>>(
        A[0], nb > 1 ? A[1] : A[0], N, jb, rp, (__nv_bfloat16*)e.planes[0],
        (__nv_bfloat16*)e.planes[1], e.ex[0], e.ex[1]);
  Args a;
  a.A[0] = A[0];
  a.A[1] = nb > 1 ? A[1] : A[0];
  a.ex[0] = e.ex[0];
  a.ex[1] = nb > 1 ? e.ex[1] : e.ex[0];
  a.N = N; a.R0 = R0; a.rpad = rp;
  a.nI = (R + BM - 1) / BM;
  a.nJ = (R + BNC - 1) / BNC;
  a.status = status;
  int tiles = 0;
  for (int I = 0; I < a.nI; ++I) tiles += std::min((BM / BNC) * (I + 1), a.nJ);
  k_herk_emu<<<dim3(tiles, nb), EMU_THREADS, SMEM_BYTES, s>>>(a, maps);
  return true;
}

}  // namespace icwf
