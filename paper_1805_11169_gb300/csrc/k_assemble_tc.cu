// Mixed-precision matrix-element assembly (Eq. M, W, W1, W2) on the sm_103a tensor cores.
//
// Each CWF is split into real and imaginary planes, and every plane value v into two pieces of
// the operand type (v ~ hi + lo; BF16 or TF32).  The Grams G_g = Psi^H diag(u_g) Psi (g = 0 is the
// overlap, g >= 1 the rank-k interaction terms) become real products of planar operands:
//   Re G = P^T D P + Q^T D Q,   Im G = P^T D Q - Q^T D P,
// each evaluated as hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory (TMEM).
//
// Kernel layout (one CTA per 128 x 32 block of (bra a, ket b) pairs, 192 threads):
//   warp 4       TMA producer: 128-byte-swizzled tiles of the bra planes (128 rows) and the
//                ket planes scaled by u_g (32 rows), two pipeline stages;
//   warp 5       MMA issuer: tcgen05.mma kind::f16 (BF16) or kind::tf32, M = 128, N = 32, into
//                four accumulators (PP, PQ, QP, QQ) per grid side;
//   warps 0..3   epilogue: lane = bra a.  g = 0 gives S1, S2 (kept in TMEM); every g >= 1 adds
//                s_g (A_g - u_g(x_b) S1)(B_g - w_g(R_b) S2) to Heff (and to the mirrored entry
//                (b, a) for off-diagonal blocks, using u_g(x_a), w_g(R_a)).
// CTAs are launched only for the upper triangle of 128 x 128 trajectory blocks (Hermitian
// symmetry of the Grams), four CTAs per block.
//
// Every wait on an mbarrier is bounded (globaltimer, 2 s); a timeout sets the status flag, stops
// issuing work, drains what is in flight (bounded again), frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "icwf_internal.h"
#include "k_common.cuh"
#include "tc_ptx.cuh"

namespace icwf {

namespace tc {

constexpr int BM = 128;        // bra trajectories per CTA (TMEM lanes)
constexpr int BNT = 32;        // ket trajectories per CTA
constexpr int ROWB = 128;      // bytes of one operand row per stage (one swizzle atom row)
constexpr int STAGES = 2;
constexpr int A_TILE = BM * ROWB;     // 16 KB
constexpr int B_TILE = BNT * ROWB;    // 4 KB
// stage layout: A_P_hi, A_P_lo, A_Q_hi, A_Q_lo, B_P_hi, B_Q_hi, B_P_lo, B_Q_lo (the two hi and the
// two lo ket tiles adjacent: each pair is one 64-row operand)
constexpr int STAGE_BYTES = 4 * A_TILE + 4 * B_TILE;   // 80 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 512 /*barriers, ket factors*/;
constexpr int TMEM_COLS = 512;
// TMEM column map: per side s (0 = x, 1 = R) accumulators PP, PQ, QP, QQ at 32 columns each
constexpr int COL_ACC = 0;       // [0, 256): g accumulators, side-major
constexpr int COL_S = 256;       // [256, 384): S1 (re, im) for 32 kets, then S2 (re, im)
constexpr int COL_H = 384;       // [384, 512): Heff (re, im) and the mirrored entries (re, im)

struct Args {
  int N, nx, nR, K;
  float dx, dR;
  const double* sig;
  const double* px;   // K*N
  const double* pR;
  const double* d;    // N
  double2* S;
  double2* H;
  int* status;
  int kind;           // 0 bf16, 1 tf32
};

// Instruction descriptor of this kernel's MMAs: M = 128, N = 64 (the P and Q planes of 32 kets
// side by side).
constexpr int BN_MMA = 2 * BNT;
__host__ __device__ constexpr uint32_t idesc(int kind) { return idesc_mn(kind, BM, BN_MMA); }
template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  mma_desc<KIND>(d_tmem, a, b, idesc(KIND), acc);
}

struct Maps {
  CUtensorMap xhi_a, xlo_a, Rhi_a, Rlo_a;   // 128-row boxes (bra planes)
  CUtensorMap xhi_b, xlo_b, Rhi_b, Rlo_b;   // 32-row boxes (ket planes)
};

template <int KIND>
__global__ void __launch_bounds__(192, 1) k_gram_tc(Args args, const __grid_constant__ Maps maps) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  float* ket_ux = (float*)(tmem_slot + 4);     // 32 floats
  float* ket_wR = ket_ux + BNT;                // 32 floats

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int I, J, q;
  block_index(blockIdx.x, I, J, q);
  const int N = args.N;
  const int a0 = I * BM;               // bra trajectories a0 .. a0+127
  const int b0 = J * BM + q * BNT;     // ket trajectories b0 .. b0+31
  const int G = args.K + 1;
  const int stx = (args.nx * (KIND ? 4 : 2) + ROWB - 1) / ROWB;   // pipeline stages per Gram
  const int stR = (args.nR * (KIND ? 4 : 2) + ROWB - 1) / ROWB;
  const int kel = ROWB / (KIND ? 4 : 2);                           // K elements per stage

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 128);
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
      for (int g = 0; g < G && !*abort_flag; ++g) {
        for (int side = 0; side < 2 && !*abort_flag; ++side) {
          const CUtensorMap* mha = side ? &maps.Rhi_a : &maps.xhi_a;
          const CUtensorMap* mla = side ? &maps.Rlo_a : &maps.xlo_a;
          const CUtensorMap* mhb = side ? &maps.Rhi_b : &maps.xhi_b;
          const CUtensorMap* mlb = side ? &maps.Rlo_b : &maps.xlo_b;
          const int nst = side ? stR : stx;
          for (int s = 0; s < nst; ++s, ++it) {
            const int slot = it % STAGES;
            const unsigned ph = (unsigned)(it / STAGES) & 1u;
            if (!mbar_wait(empty + slot, ph ^ 1u, abort_flag, args.status)) break;
            unsigned char* st = smem + slot * STAGE_BYTES;
            mbar_expect_tx(full + slot, STAGE_BYTES);
            last_it[slot] = it;
            const int kc = s * kel;
            // bra planes (g = 0 rows): P rows [0, N), Q rows [N, 2N)
            tma_load_2d(st + 0 * A_TILE, mha, kc, a0, full + slot);
            tma_load_2d(st + 1 * A_TILE, mla, kc, a0, full + slot);
            tma_load_2d(st + 2 * A_TILE, mha, kc, N + a0, full + slot);
            tma_load_2d(st + 3 * A_TILE, mla, kc, N + a0, full + slot);
            // ket planes scaled by u_g: rows (2g) N + b and (2g+1) N + b
            unsigned char* sb = st + 4 * A_TILE;
            tma_load_2d(sb + 0 * B_TILE, mhb, kc, 2 * g * N + b0, full + slot);
            tma_load_2d(sb + 1 * B_TILE, mhb, kc, (2 * g + 1) * N + b0, full + slot);
            tma_load_2d(sb + 2 * B_TILE, mlb, kc, 2 * g * N + b0, full + slot);
            tma_load_2d(sb + 3 * B_TILE, mlb, kc, (2 * g + 1) * N + b0, full + slot);
          }
        }
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int it = 0;
      for (int g = 0; g < G && !*abort_flag; ++g) {
        if (g >= 1) {
          // the epilogue must have consumed the previous Gram's accumulators
          if (!mbar_wait(acc_empty, (unsigned)(g - 1) & 1u, abort_flag, args.status)) break;
          fence_after();
        }
        for (int side = 0; side < 2 && !*abort_flag; ++side) {
          const uint32_t acc = tmem + COL_ACC + side * 128;
          const int nst = side ? stR : stx;
          for (int s = 0; s < nst; ++s, ++it) {
            const int slot = it % STAGES;
            const unsigned ph = (unsigned)(it / STAGES) & 1u;
            if (!mbar_wait(full + slot, ph, abort_flag, args.status)) break;
            fence_after();
            const uint32_t st = smem_u32(smem + slot * STAGE_BYTES);
            const uint32_t aph = st, apl = st + A_TILE, aqh = st + 2 * A_TILE, aql = st + 3 * A_TILE;
            const uint32_t bhi = st + 4 * A_TILE, blo = bhi + 2 * B_TILE;   // [P; Q] kets
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t o = kk * 32;   // 32 bytes of K per instruction
              const uint32_t first = (s == 0 && kk == 0) ? 0u : 1u;
              // columns [0, 32) take the P kets, [32, 64) the Q kets: (PP, PQ) and (QP, QQ),
              // each hi*hi + hi*lo + lo*hi
              mma<KIND>(acc + 0, sdesc(aph + o), sdesc(bhi + o), first);
              mma<KIND>(acc + 0, sdesc(aph + o), sdesc(blo + o), 1u);
              mma<KIND>(acc + 0, sdesc(apl + o), sdesc(bhi + o), 1u);
              mma<KIND>(acc + 64, sdesc(aqh + o), sdesc(bhi + o), first);
              mma<KIND>(acc + 64, sdesc(aqh + o), sdesc(blo + o), 1u);
              mma<KIND>(acc + 64, sdesc(aql + o), sdesc(bhi + o), 1u);
            }
            mma_commit(empty + slot);   // frees the stage when these MMAs complete
          }
        }
        mma_commit(acc_full);           // Gram g complete (both sides)
      }
      mma_commit(drain);                // every MMA issued by this CTA
    }
  } else {
    // ---------------- epilogue: warps 0..3, lane = bra row ----------------
    const int row = warp * 32 + lane;
    const int a = a0 + row;
    const bool a_ok = a < N;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const bool mirror = I != J;
    const float dx = args.dx, dR = args.dR;
    for (int g = 0; g < G; ++g) {
      const bool ok = mbar_wait(acc_full, (unsigned)g & 1u, abort_flag, args.status);
      // one decision for all four epilogue warps (they meet at named barriers below)
      uint32_t all_ok;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
          "bar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
          : "=r"(all_ok)
          : "r"((uint32_t)ok)
          : "memory");
      if (!all_ok) break;
      fence_after();
      const float sg = g ? (float)args.sig[g - 1] : 0.f;
      const float uxa = (g && a_ok) ? (float)args.px[(size_t)(g - 1) * N + a] : 0.f;
      const float wRa = (g && a_ok) ? (float)args.pR[(size_t)(g - 1) * N + a] : 0.f;
      if (g) {
        // the kets' factor values for this Gram, staged once in shared memory
        if (row < BNT) {
          const int b = b0 + row;
          ket_ux[row] = b < N ? (float)args.px[(size_t)(g - 1) * N + b] : 0.f;
        } else if (row < 2 * BNT) {
          const int b = b0 + row - BNT;
          ket_wR[row - BNT] = b < N ? (float)args.pR[(size_t)(g - 1) * N + b] : 0.f;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
#pragma unroll 1
      for (int c8 = 0; c8 < BNT; c8 += 8) {
        float xpp[8], xpq[8], xqp[8], xqq[8], rpp[8], rpq[8], rqp[8], rqq[8];
        tmem_ld8(lane_base + COL_ACC + 0 + c8, xpp);
        tmem_ld8(lane_base + COL_ACC + 32 + c8, xpq);
        tmem_ld8(lane_base + COL_ACC + 64 + c8, xqp);
        tmem_ld8(lane_base + COL_ACC + 96 + c8, xqq);
        tmem_ld8(lane_base + COL_ACC + 128 + c8, rpp);
        tmem_ld8(lane_base + COL_ACC + 160 + c8, rpq);
        tmem_ld8(lane_base + COL_ACC + 192 + c8, rqp);
        tmem_ld8(lane_base + COL_ACC + 224 + c8, rqq);
        tmem_wait_ld();
        float Ar[8], Ai[8], Br[8], Bi[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          Ar[e] = dx * (xpp[e] + xqq[e]);
          Ai[e] = dx * (xpq[e] - xqp[e]);
          Br[e] = dR * (rpp[e] + rqq[e]);
          Bi[e] = dR * (rpq[e] - rqp[e]);
        }
        if (g == 0) {
          // S1 = <psi_a|psi_b>, S2 = <chi_a|chi_b>, kept in TMEM for every later Gram;
          // the Heff accumulators start at zero
          float zero[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) zero[e] = 0.f;
          tmem_st8(lane_base + COL_S + c8, Ar);
          tmem_st8(lane_base + COL_S + 32 + c8, Ai);
          tmem_st8(lane_base + COL_S + 64 + c8, Br);
          tmem_st8(lane_base + COL_S + 96 + c8, Bi);
          tmem_st8(lane_base + COL_H + c8, zero);
          tmem_st8(lane_base + COL_H + 32 + c8, zero);
          tmem_st8(lane_base + COL_H + 64 + c8, zero);
          tmem_st8(lane_base + COL_H + 96 + c8, zero);
          tmem_wait_st();
        } else {
          float s1r[8], s1i[8], s2r[8], s2i[8], hr[8], hi[8], tr[8], ti[8];
          tmem_ld8(lane_base + COL_S + c8, s1r);
          tmem_ld8(lane_base + COL_S + 32 + c8, s1i);
          tmem_ld8(lane_base + COL_S + 64 + c8, s2r);
          tmem_ld8(lane_base + COL_S + 96 + c8, s2i);
          tmem_ld8(lane_base + COL_H + c8, hr);
          tmem_ld8(lane_base + COL_H + 32 + c8, hi);
          tmem_ld8(lane_base + COL_H + 64 + c8, tr);
          tmem_ld8(lane_base + COL_H + 96 + c8, ti);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float uxb = ket_ux[c8 + e];
            const float wRb = ket_wR[c8 + e];
            // (A - u(x_b) S1) (B - w(R_b) S2)
            const float atr = Ar[e] - uxb * s1r[e], ati = Ai[e] - uxb * s1i[e];
            const float btr = Br[e] - wRb * s2r[e], bti = Bi[e] - wRb * s2i[e];
            hr[e] = fmaf(sg, atr * btr - ati * bti, hr[e]);
            hi[e] = fmaf(sg, atr * bti + ati * btr, hi[e]);
            if (mirror) {
              // entry (b, a): conj(A) - u(x_a) conj(S1), conj(B) - w(R_a) conj(S2)
              const float mtr = Ar[e] - uxa * s1r[e], mti = -(Ai[e] - uxa * s1i[e]);
              const float ntr = Br[e] - wRa * s2r[e], nti = -(Bi[e] - wRa * s2i[e]);
              tr[e] = fmaf(sg, mtr * ntr - mti * nti, tr[e]);
              ti[e] = fmaf(sg, mtr * nti + mti * ntr, ti[e]);
            }
          }
          tmem_st8(lane_base + COL_H + c8, hr);
          tmem_st8(lane_base + COL_H + 32 + c8, hi);
          tmem_st8(lane_base + COL_H + 64 + c8, tr);
          tmem_st8(lane_base + COL_H + 96 + c8, ti);
          tmem_wait_st();
        }
      }
      fence_before();
      mbar_arrive(acc_empty);
      asm volatile("bar.sync 1, 128;" ::: "memory");   // ket_ux / ket_wR reused by the next Gram
    }
    // final: S = S1 o S2; Heff(a, b) = H - d_b S; Heff(b, a) = HT - d_a conj(S)
    const int aborted = __shfl_sync(0xffffffffu, *abort_flag, 0);
    if (!aborted) {
      const double da = a_ok ? args.d[a] : 0.0;
#pragma unroll 1
      for (int c8 = 0; c8 < BNT; c8 += 8) {
        float s1r[8], s1i[8], s2r[8], s2i[8], hr[8], hi[8], tr[8], ti[8];
        tmem_ld8(lane_base + COL_S + c8, s1r);
        tmem_ld8(lane_base + COL_S + 32 + c8, s1i);
        tmem_ld8(lane_base + COL_S + 64 + c8, s2r);
        tmem_ld8(lane_base + COL_S + 96 + c8, s2i);
        tmem_ld8(lane_base + COL_H + c8, hr);
        tmem_ld8(lane_base + COL_H + 32 + c8, hi);
        tmem_ld8(lane_base + COL_H + 64 + c8, tr);
        tmem_ld8(lane_base + COL_H + 96 + c8, ti);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int b = b0 + c8 + e;
          if (b >= N || !a_ok) continue;
          const double sr = (double)s1r[e] * s2r[e] - (double)s1i[e] * s2i[e];
          const double si = (double)s1r[e] * s2i[e] + (double)s1i[e] * s2r[e];
          const double db = args.d[b];
          if (args.S) args.S[(size_t)a * N + b] = make_double2(sr, si);
          args.H[(size_t)a * N + b] = make_double2(hr[e] - db * sr, hi[e] - db * si);
          if (mirror) {
            if (args.S) args.S[(size_t)b * N + a] = make_double2(sr, -si);
            args.H[(size_t)b * N + a] = make_double2(tr[e] - da * sr, ti[e] + da * si);
          }
        }
      }
    }
  }

  // ---------------- teardown ----------------
  __syncthreads();
  if (warp == 5 && lane == 0) {
    // wait (bounded) until every issued MMA has retired before TMEM is released
    const unsigned long long t0 = gtime();
    while (!mbar_test(drain, 0u) && gtime() - t0 < WAIT_NS) {
    }
  }
  if (warp == 4 && lane == 0 && *abort_flag) {
    // bounded drain of TMA copies that may still be landing in shared memory: wait for the
    // phase of the last copy issued into each stage
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

// ---------------------------------------------------------------------------- operand prep

// Planar split operands for one grid side: rows r = (2g + comp) N + b, K index i contiguous:
// value = comp(psi_b(x_i)) * (g ? u_{g-1}(x_i) : 1), split into hi + lo of the operand type.
// One CTA per (g, b) row; each thread converts 4 consecutive grid points (16-byte loads of the CWF
// and the factor, 16-byte (TF32) or 8-byte (BF16) stores per plane).  n is a multiple of 4.
template <int KIND>
__device__ __forceinline__ void split4(const float (&v)[4], void* hi_out, void* lo_out, size_t at) {
  if (KIND == 0) {
    __nv_bfloat16 h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = __float2bfloat16_rn(v[e]);
      l[e] = __float2bfloat16_rn(v[e] - __bfloat162float(h[e]));
    }
    *(uint2*)((__nv_bfloat16*)hi_out + at) = *(const uint2*)h;
    *(uint2*)((__nv_bfloat16*)lo_out + at) = *(const uint2*)l;
  } else {
    // TF32: keep the top 10 mantissa bits (round to nearest), the remainder as the low piece
    auto r19 = [](float x) {
      uint32_t u32 = __float_as_uint(x);
      u32 = (u32 + 0x1000u) & 0xFFFFE000u;
      return __uint_as_float(u32);
    };
    float4 h, l;
    h.x = r19(v[0]); h.y = r19(v[1]); h.z = r19(v[2]); h.w = r19(v[3]);
    l.x = r19(v[0] - h.x); l.y = r19(v[1] - h.y); l.z = r19(v[2] - h.z); l.w = r19(v[3] - h.w);
    *(float4*)((float*)hi_out + at) = h;
    *(float4*)((float*)lo_out + at) = l;
  }
}

template <int KIND>
__global__ void __launch_bounds__(256) k_prep(const float2* __restrict__ cwf,
                                              const double* __restrict__ U, int n, int N,
                                              void* __restrict__ hi_out, void* __restrict__ lo_out) {
  const int row = blockIdx.x;             // g * N + b
  const int g = row / N, b = row - g * N;
  const float4* src = (const float4*)(cwf + (size_t)b * n);        // 2 complex per float4
  const double2* u = g ? (const double2*)(U + (size_t)(g - 1) * n) : nullptr;
  const size_t rp = ((size_t)(2 * g) * N + b) * n, rq = ((size_t)(2 * g + 1) * N + b) * n;
  for (int i4 = threadIdx.x; 4 * i4 < n; i4 += blockDim.x) {
    const float4 z01 = src[2 * i4], z23 = src[2 * i4 + 1];
    float f[4] = {1.f, 1.f, 1.f, 1.f};
    if (u) {
      const double2 u01 = u[2 * i4], u23 = u[2 * i4 + 1];
      f[0] = (float)u01.x; f[1] = (float)u01.y; f[2] = (float)u23.x; f[3] = (float)u23.y;
    }
    const float vr[4] = {z01.x * f[0], z01.z * f[1], z23.x * f[2], z23.z * f[3]};
    const float vi[4] = {z01.y * f[0], z01.w * f[1], z23.y * f[2], z23.w * f[3]};
    split4<KIND>(vr, hi_out, lo_out, rp + 4 * (size_t)i4);
    split4<KIND>(vi, hi_out, lo_out, rq + 4 * (size_t)i4);
  }
}

// ---------------------------------------------------------------------------- host side

bool make_map(CUtensorMap* m, void* base, int kind, int n, size_t rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const size_t esz = kind ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(n * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(ROWB / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, kind ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace tc

bool launch_assemble_tc(const JobView& j, int precision, bool exact_s, double2* S, double2* H,
                        void* scratch, size_t scratch_bytes, cudaStream_t s) {
  using namespace tc;
  const int kind = precision == ICWF_MIXED_TF32X3 ? 1 : 0;
  const size_t esz = kind ? 4 : 2;
  const int G = j.K + 1;
  const size_t rx = (size_t)2 * G * j.N, nxe = rx * j.nx * esz, nRe = rx * j.nR * esz;
  auto al = [](size_t b) { return (b + 1023) & ~(size_t)1023; };
  const size_t split_bytes = 2 * al(nxe) + 2 * al(nRe);
  if (split_bytes > scratch_bytes) return false;
  if (exact_s &&
      !launch_gram_s(j, S, (char*)scratch + split_bytes, scratch_bytes - split_bytes, s))
    return false;
  char* p = (char*)scratch;
  void* xhi = p; p += al(nxe);
  void* xlo = p; p += al(nxe);
  void* Rhi = p; p += al(nRe);
  void* Rlo = p; p += al(nRe);
  const unsigned rows = (unsigned)(G * j.N);
  const int tx = j.nx / 4 < 256 ? j.nx / 4 : 256, tR = j.nR / 4 < 256 ? j.nR / 4 : 256;
  if (kind) {
    k_prep<1><<<rows, tx, 0, s>>>((const float2*)j.psi, j.U, j.nx, j.N, xhi, xlo);
    k_prep<1><<<rows, tR, 0, s>>>((const float2*)j.chi, j.W, j.nR, j.N, Rhi, Rlo);
  } else {
    k_prep<0><<<rows, tx, 0, s>>>((const float2*)j.psi, j.U, j.nx, j.N, xhi, xlo);
    k_prep<0><<<rows, tR, 0, s>>>((const float2*)j.chi, j.W, j.nR, j.N, Rhi, Rlo);
  }
  Maps m;
  bool ok = make_map(&m.xhi_a, xhi, kind, j.nx, rx, BM) && make_map(&m.xlo_a, xlo, kind, j.nx, rx, BM) &&
            make_map(&m.Rhi_a, Rhi, kind, j.nR, rx, BM) && make_map(&m.Rlo_a, Rlo, kind, j.nR, rx, BM) &&
            make_map(&m.xhi_b, xhi, kind, j.nx, rx, BNT) && make_map(&m.xlo_b, xlo, kind, j.nx, rx, BNT) &&
            make_map(&m.Rhi_b, Rhi, kind, j.nR, rx, BNT) && make_map(&m.Rlo_b, Rlo, kind, j.nR, rx, BNT);
  if (!ok) return false;
  Args a;
  a.N = j.N; a.nx = j.nx; a.nR = j.nR; a.K = j.K;
  a.dx = (float)j.dx; a.dR = (float)j.dR;
  a.sig = j.sig; a.px = j.px; a.pR = j.pR; a.d = j.d;
  a.S = exact_s ? nullptr : S;   // with the exact overlap kernel, S comes from there
  a.H = H; a.status = j.status; a.kind = kind;
  const int T = (j.N + BM - 1) / BM;
  const unsigned grid = (unsigned)(4 * T * (T + 1) / 2);
  if (kind) {
    static bool attr1 = false;   // set once: no attribute changes inside a captured launch
    if (!attr1) {
      cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
      attr1 = true;
    }
    k_gram_tc<1><<<grid, 192, SMEM_BYTES, s>>>(a, m);
  } else {
    static bool attr0 = false;
    if (!attr0) {
      cudaFuncSetAttribute(k_gram_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
      attr0 = true;
    }
    k_gram_tc<0><<<grid, 192, SMEM_BYTES, s>>>(a, m);
  }
  return true;
}

size_t assemble_tc_scratch_bytes(int N, int nx, int nR, int K) {
  // hi + lo planes (P and Q rows for every Gram) for both sides, TF32 (4 bytes) as the larger,
  // then the digit planes of the exact overlap kernel
  const size_t G = (size_t)K + 1;
  return 2 * 4 * G * 2 * (size_t)N * ((size_t)nx + nR) + 4 * 1024 + gram_s_scratch_bytes(N, nx, nR);
}

}  // namespace icwf
