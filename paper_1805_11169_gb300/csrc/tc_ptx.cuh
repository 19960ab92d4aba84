// Inline-PTX wrappers shared by the tcgen05 tensor-core kernels (sm_103a): mbarriers with
// bounded waits, TMA tiled loads, shared-memory and instruction descriptors for K-major BF16/TF32
// operands, tcgen05.mma / commit / fences, TMEM loads and stores, and the triangular block index
// of the Hermitian Gram launches.  Bit layouts follow the public PTX ISA descriptions of the
// tcgen05 shared-memory matrix descriptor and the kind::f16 / kind::tf32 instruction descriptor.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "k_common.cuh"

namespace icwf {
namespace tc {

// every mbarrier wait gives up after this long (globaltimer ns) and raises the timeout flag
constexpr unsigned long long WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and raises the abort flag) on timeout or if another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, volatile int* abort_flag,
                                         int* status) {
  const unsigned long long t0 = gtime();
  while (true) {
    if (mbar_test(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtime() - t0 > WAIT_NS) {
      *abort_flag = 1;
      set_flag(status, ST_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 8 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}
// 4 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = __uint_as_float(r[q]);
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }


// Shared-memory matrix descriptor of a K-major operand tile with rows of `swizzle` bytes (128,
// 64 or 32) in the matching swizzle mode; 8-row groups are 8 * swizzle bytes apart.  The tile base
// is aligned to its swizzle atom; a K offset inside the row is added to the start address.
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr, int swizzle) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                                   // leading-dimension offset (unused)
  d |= (uint64_t)((8 * swizzle) >> 4) << 32;                // stride between 8-row groups
  d |= (uint64_t)1 << 46;                                   // descriptor version
  d |= (uint64_t)(swizzle == 128 ? 2 : (swizzle == 64 ? 4 : 6)) << 61;   // swizzle mode
  return d;
}
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) { return sdesc_sw(saddr, 128); }

// Instruction descriptor: D = F32, A = B = BF16 (kind 0) or TF32 (kind 1), both K-major,
// M x N_ tile.
__host__ __device__ constexpr uint32_t idesc_mn(int kind, int M, int N_) {
  return (1u << 4) | ((kind ? 2u : 1u) << 7) | ((kind ? 2u : 1u) << 10) |
         ((uint32_t)(N_ >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A * B^T with the given instruction descriptor (acc = 0 overwrites).
template <int KIND>
__device__ __forceinline__ void mma_desc(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t acc) {
  if (KIND == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  }
}

// Block (I <= J) of 128 x 128 trajectories and ket quarter q from the linear CTA index.
__device__ __forceinline__ void block_index(int t, int& I, int& J, int& q) {
  q = t & 3;
  t >>= 2;
  int Jc = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (Jc * (Jc + 1) / 2 > t) --Jc;
  while ((Jc + 1) * (Jc + 2) / 2 <= t) ++Jc;
  J = Jc;
  I = t - Jc * (Jc + 1) / 2;
}


// Driver entry point of cuTensorMapEncodeTiled (looked up once).
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}


}  // namespace tc
}  // namespace icwf
