// The overlap S = S1 o S2 (Eq. M) of the mixed modes as exact Grams of fixed-point CWFs on the
// sm_103a tensor cores (BF16 operands, FP32 accumulation in TMEM).
//
// Why: S is positive semidefinite, and the coefficient solve factorises S + eps I.  Ordinary split
// products (hi*hi + hi*lo + lo*hi) with FP32 accumulation leave rounding errors whose indefinite
// part reaches ~1e-4 at N = 1024 (S has eigenvalues up to ~N), which forces a large eps.  Here
// each Gram is the exact Gram of a fixed-point representation of the complex64 CWFs, so S stays
// positive semidefinite to FP64 rounding and eps can be as small as in the FP64 mode.
//
// Representation.  Per CWF column b and grid side: m_b = max_i max(|Re|, |Im|), e_b the
// smallest integer with m_b < 2^e_b, and x = psi_b 2^-e_b (components in (-1, 1)).  Each
// component is expanded into D = 4 balanced digits of base B = 2^beta by exact FP32 steps
// (v = x B, d_1 = rint(v), v = (v - d_1) B, d_2 = rint(v), ...), so |d_1| <= B, |d_p| <= B/2;
// digit p is stored as the BF16 value a_p = d_p B^-(p-1) (exact), so x ~ B^-1 sum_p a_p.  With
// beta = 6, four digits carry 24 bits: every component within a factor two of m_b is represented
// exactly; smaller ones to 2^-25 m_b.
//
// Products.  conj(x_a) x_b = B^-2 sum_{p,q} conj(a_p^a) a_q^b over all 16 digit pairs, so the sum
// is the exact Gram of the represented vectors.  Pairs are accumulated by level: p = q = 1
// (integers), p + q = 3 (multiples of 1/B) and p + q >= 4 in three FP32 accumulators.  The first
// two stay below 2^24 units (2 K B^2 <= 2^24: beta = 6 for K <= 2048, beta = 5 for K = 4096), so
// their FP32 sums are exact; the third carries weight B^-2 relative to the first, so its FP32
// rounding is of order 1e-10 of S or below.  The epilogue adds the three (double-float) and scales
// by dx 2^(e_a + e_b) B^-2.
//
// Complex arithmetic on real MMAs: per digit pair, with P/Q the real/imaginary planes,
//   [Re | Im] += P_a [P_b | Q_b] + Q_a [Q_b | -P_b],
// one M = 128, N = 64 accumulator per level and side ([Re | Im] of 32 kets).
//
// Kernel layout (one CTA per 128 bras x 32 kets, upper triangle of 128 x 128 blocks, 192 threads):
//   warp 4       TMA producer: per stage one 16-element K slice (32-byte rows, 32-byte swizzle)
//                of the bra digit planes (4 digits x P, Q, 128 rows) and of the ket digit planes
//                (4 digits x P, Q, -P, 32 rows each), five stages;
//   warp 5       MMA issuer: 16 digit pairs x 2 planes per stage (one K = 16 instruction each);
//   warps 0..3   epilogue: lane = bra a; S1, S2 from TMEM in double-float arithmetic, S = S1 o S2
//                for the block and its Hermitian mirror, stored in FP64.
// Waits are bounded (2 s); a timeout raises the status flag, drains what is in flight and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "df64.cuh"
#include "icwf_internal.h"
#include "k_common.cuh"
#include "tc_ptx.cuh"

namespace icwf {
namespace tcs {

using namespace tc;

constexpr int BM = 128;                  // bras per CTA (TMEM lanes)
constexpr int BNT = 32;                  // kets per CTA
constexpr int DIG = 4;                   // digits per component
constexpr int ROW = 32;                  // bytes per operand row per stage (16 BF16, 32-byte swizzle)
constexpr int KEL = ROW / 2;             // K elements per stage: one MMA instruction's K
constexpr int A_T = BM * ROW;            // one bra plane tile: 4 KB
constexpr int KETROWS = 3 * BNT;         // P, Q, -P of 32 kets
constexpr int B_T = KETROWS * ROW;       // one ket digit block: 3 KB
constexpr int STAGES = 5;                // four slices in flight hide the TMA latency
constexpr int STAGE_BYTES = 2 * DIG * A_T + DIG * B_T;   // 32 KB + 12 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA exceeded");
constexpr int TMEM_COLS = 512;
constexpr int ACC_COLS = 2 * BNT;        // [Re | Im] of 32 kets
constexpr int SIDE_COLS = 3 * ACC_COLS;  // three levels per side
static_assert(2 * SIDE_COLS <= TMEM_COLS, "accumulators exceed the TMEM allocation");
constexpr uint32_t IDESC = idesc_mn(0, BM, ACC_COLS);

struct Args {
  int N, nx, nR;
  int beta_x, beta_R;
  double dx, dR;
  const int* ex;      // N exponents, x side
  const int* eR;      // N exponents, R side
  double2* S;
  int* status;
};

struct Maps {
  CUtensorMap xa, Ra;   // 128-row boxes (bras)
  CUtensorMap xb, Rb;   // 32-row boxes (kets)
};

__device__ __forceinline__ int level_of(int p, int q) { return p + q == 0 ? 0 : (p + q == 1 ? 1 : 2); }

__global__ void __launch_bounds__(192, 1) k_gram_s(Args args, const __grid_constant__ Maps maps) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* drain = acc_full + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int I, J, q4;
  block_index(blockIdx.x, I, J, q4);
  const int N = args.N;
  const int a0 = I * BM;
  const int b0 = J * BM + q4 * BNT;
  const int stx = (args.nx + KEL - 1) / KEL;
  const int stR = (args.nR + KEL - 1) / KEL;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
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

  int last_it[STAGES];
#pragma unroll
  for (int t = 0; t < STAGES; ++t) last_it[t] = -1;
  if (warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int it = 0;
      for (int side = 0; side < 2 && !*abort_flag; ++side) {
        const CUtensorMap* ma = side ? &maps.Ra : &maps.xa;
        const CUtensorMap* mb = side ? &maps.Rb : &maps.xb;
        const int nst = side ? stR : stx;
        for (int s = 0; s < nst; ++s, ++it) {
          const int slot = it % STAGES;
          const unsigned ph = (unsigned)(it / STAGES) & 1u;
          if (!mbar_wait(empty + slot, ph ^ 1u, abort_flag, args.status)) break;
          unsigned char* st = smem + slot * STAGE_BYTES;
          mbar_expect_tx(full + slot, STAGE_BYTES);
          last_it[slot] = it;
          const int kc = s * KEL;
          // plane rows: (3 p + pi) N + b, pi = 0 (P), 1 (Q), 2 (-P)
          for (int p = 0; p < DIG; ++p) {
            tma_load_2d(st + (2 * p + 0) * A_T, ma, kc, (3 * p + 0) * N + a0, full + slot);
            tma_load_2d(st + (2 * p + 1) * A_T, ma, kc, (3 * p + 1) * N + a0, full + slot);
          }
          unsigned char* kb = st + 2 * DIG * A_T;
          for (int p = 0; p < DIG; ++p)
            for (int pi = 0; pi < 3; ++pi)
              tma_load_2d(kb + p * B_T + pi * BNT * ROW, mb, kc, (3 * p + pi) * N + b0, full + slot);
        }
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int it = 0;
      for (int side = 0; side < 2 && !*abort_flag; ++side) {
        const uint32_t acc0 = tmem + side * SIDE_COLS;
        const int nst = side ? stR : stx;
        bool started[3] = {false, false, false};
        for (int s = 0; s < nst; ++s, ++it) {
          const int slot = it % STAGES;
          const unsigned ph = (unsigned)(it / STAGES) & 1u;
          if (!mbar_wait(full + slot, ph, abort_flag, args.status)) break;
          fence_after();
          const uint32_t st = smem_u32(smem + slot * STAGE_BYTES);
          const uint32_t kb = st + 2 * DIG * A_T;
#pragma unroll 1
          for (int p = 0; p < DIG; ++p) {
#pragma unroll 1
            for (int q = 0; q < DIG; ++q) {
              const int lv = level_of(p, q);
              const uint32_t acc = acc0 + lv * ACC_COLS;
              const uint32_t ap = st + (2 * p) * A_T, aq = ap + A_T;
              const uint32_t kq = kb + q * B_T;           // rows P | Q | -P of ket digit q
              const uint32_t first = started[lv] ? 1u : 0u;
              mma_desc<0>(acc, sdesc_sw(ap, ROW), sdesc_sw(kq, ROW), IDESC, first);
              mma_desc<0>(acc, sdesc_sw(aq, ROW), sdesc_sw(kq + BNT * ROW, ROW), IDESC, 1u);
              started[lv] = true;
            }
          }
          mma_commit(empty + slot);
        }
      }
      mma_commit(acc_full);
      mma_commit(drain);
    }
  } else {
    // ---------------- epilogue: warps 0..3, lane = bra row ----------------
    const int row = warp * 32 + lane;
    const int a = a0 + row;
    const bool a_ok = a < N;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const bool mirror = I != J;
    // an aborted producer or issuer still commits acc_full: check the flag as well
    const bool ok = mbar_wait(acc_full, 0u, abort_flag, args.status) && !*abort_flag;
    uint32_t all_ok;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(all_ok)
        : "r"((uint32_t)ok)
        : "memory");
    if (all_ok) {
      fence_after();
      // the levels are combined and S1 o S2 formed in double-float arithmetic (FP32 pairs, ~2^-44
      // relative; FP64 instructions are scarce on this GPU); FP64 only for the stores
      const int ea_x = a_ok ? args.ex[a] : 0, ea_R = a_ok ? args.eR[a] : 0;
      const df dxd = df_from(args.dx), dRd = df_from(args.dR);
#pragma unroll 1
      for (int c8 = 0; c8 < BNT; c8 += 8) {
        cdf sv[2][8];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          float v[3][2][8];
#pragma unroll
          for (int lv = 0; lv < 3; ++lv) {
            tmem_ld8(lane_base + side * SIDE_COLS + lv * ACC_COLS + c8, v[lv][0]);
            tmem_ld8(lane_base + side * SIDE_COLS + lv * ACC_COLS + BNT + c8, v[lv][1]);
          }
          tmem_wait_ld();
          const int beta = side ? args.beta_R : args.beta_x;
          const df dd = side ? dRd : dxd;
          const int* eb = side ? args.eR : args.ex;
          const int ea = side ? ea_R : ea_x;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int b = b0 + c8 + e;
            const int sh = ea + (b < N ? eb[b] : 0) - 2 * beta;   // exact power-of-two scale
            df re = df_add(two_sum(v[0][0][e], v[1][0][e]), df_make(v[2][0][e], 0.f));
            df im = df_add(two_sum(v[0][1][e], v[1][1][e]), df_make(v[2][1][e], 0.f));
            re = df_mul(df_make(ldexpf(re.h, sh), ldexpf(re.l, sh)), dd);
            im = df_mul(df_make(ldexpf(im.h, sh), ldexpf(im.l, sh)), dd);
            sv[side][e] = cdf_make(re, im);
          }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int b = b0 + c8 + e;
          // each pair once, from its a <= b side (diagonal blocks compute both sides; the
          // highest-level sums of the two round differently), so S is exactly Hermitian
          if (b >= N || !a_ok || (!mirror && a > b)) continue;
          const cdf z = cdf_mul(sv[0][e], sv[1][e]);
          const double r = df_to(z.re);
          const double i = a == b ? 0.0 : df_to(z.im);
          args.S[(size_t)a * N + b] = make_double2(r, i);
          if (a != b) args.S[(size_t)b * N + a] = make_double2(r, -i);
        }
      }
    }
  }

  // ---------------- teardown ----------------
  __syncthreads();
  if (warp == 5 && lane == 0) {
    const unsigned long long t0 = gtime();
    while (!mbar_test(drain, 0u) && gtime() - t0 < WAIT_NS) {
    }
  }
  if (warp == 4 && lane == 0 && *abort_flag) {
    for (int t = 0; t < STAGES; ++t) {
      if (last_it[t] < 0) continue;
      const unsigned ph = (unsigned)(last_it[t] / STAGES) & 1u;
      const unsigned long long t0 = gtime();
      while (!mbar_test(full + t, ph) && gtime() - t0 < WAIT_NS) {
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// Digit planes of one grid side: one CTA per column b.  planes[((3 p + pi) N + b) n + i],
// pi = 0: a_p(Re), 1: a_p(Im), 2: -a_p(Re); expo[b] = e_b.
__global__ void __launch_bounds__(256) k_digits(const float2* __restrict__ cwf, int n, int N,
                                                int beta, __nv_bfloat16* __restrict__ planes,
                                                int* __restrict__ expo) {
  __shared__ float red[8];
  const int b = blockIdx.x;
  const float2* col = cwf + (size_t)b * n;
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 z = col[i];
    m = fmaxf(m, fmaxf(fabsf(z.x), fabsf(z.y)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
  const int e = m > 0.f ? ilogbf(m) + 1 : 0;   // m < 2^e
  if (threadIdx.x == 0) expo[b] = e;
  const size_t pl = (size_t)N * n;             // one plane
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 z = col[i];
    float vr = ldexpf(z.x, beta - e), vi = ldexpf(z.y, beta - e);   // x B, exact
#pragma unroll
    for (int p = 0; p < DIG; ++p) {
      const float dr = rintf(vr), di = rintf(vi);
      const __nv_bfloat16 hr = __float2bfloat16_rn(ldexpf(dr, -beta * p));
      const __nv_bfloat16 hi = __float2bfloat16_rn(ldexpf(di, -beta * p));
      const __nv_bfloat16 hn = __float2bfloat16_rn(ldexpf(-dr, -beta * p));
      const size_t base = (size_t)(3 * p) * pl + (size_t)b * n + i;
      planes[base] = hr;
      planes[base + pl] = hi;
      planes[base + 2 * pl] = hn;
      vr = ldexpf(vr - dr, beta);   // remainder in [-1/2, 1/2], exact; next digit
      vi = ldexpf(vi - di, beta);
    }
  }
}

bool make_map64(CUtensorMap* m, void* base, int n, size_t rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)n * 2};
  cuuint32_t box[2] = {(cuuint32_t)KEL, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int beta_for(int n) { return n <= 2048 ? 6 : 5; }

}  // namespace tcs

size_t gram_s_scratch_bytes(int N, int nx, int nR) {
  auto al = [](size_t b) { return (b + 1023) & ~(size_t)1023; };
  const size_t pl = (size_t)3 * tcs::DIG * N * 2;   // bytes per grid point over all planes
  return al(pl * nx) + al(pl * nR) + 2 * al((size_t)N * 4);
}

bool launch_gram_s(const JobView& j, double2* S, void* scratch, size_t bytes, cudaStream_t s) {
  using namespace tcs;
  auto al = [](size_t b) { return (b + 1023) & ~(size_t)1023; };
  const size_t pl = (size_t)3 * DIG * j.N * 2;
  if (gram_s_scratch_bytes(j.N, j.nx, j.nR) > bytes) return false;
  char* p = (char*)scratch;
  __nv_bfloat16* px = (__nv_bfloat16*)p; p += al(pl * j.nx);
  __nv_bfloat16* pR = (__nv_bfloat16*)p; p += al(pl * j.nR);
  int* ex = (int*)p; p += al((size_t)j.N * 4);
  int* eR = (int*)p;
  const int bx = beta_for(j.nx), bR = beta_for(j.nR);
  k_digits<<<j.N, 256, 0, s>>>((const float2*)j.psi, j.nx, j.N, bx, px, ex);
  k_digits<<<j.N, 256, 0, s>>>((const float2*)j.chi, j.nR, j.N, bR, pR, eR);
  Maps m;
  const size_t rows = (size_t)3 * DIG * j.N;
  if (!make_map64(&m.xa, px, j.nx, rows, BM) || !make_map64(&m.Ra, pR, j.nR, rows, BM) ||
      !make_map64(&m.xb, px, j.nx, rows, BNT) || !make_map64(&m.Rb, pR, j.nR, rows, BNT))
    return false;
  Args a;
  a.N = j.N; a.nx = j.nx; a.nR = j.nR;
  a.beta_x = bx; a.beta_R = bR;
  a.dx = j.dx; a.dR = j.dR;
  a.ex = ex; a.eR = eR;
  a.S = S; a.status = j.status;
  const int T = (j.N + BM - 1) / BM;
  const unsigned grid = (unsigned)(4 * T * (T + 1) / 2);
  static bool attr = false;   // set once: no attribute changes inside a captured launch
  if (!attr) {
    cudaFuncSetAttribute(k_gram_s, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  k_gram_s<<<grid, 192, SMEM_BYTES, s>>>(a, m);
  return true;
}

}  // namespace icwf
