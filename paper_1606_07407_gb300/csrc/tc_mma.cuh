// Fifth-generation tensor-core helpers (tcgen05, sm_103a) as inline PTX: shared-memory matrix
// descriptors for operands without swizzle, the instruction descriptor of a BF16 x BF16 -> FP32
// MMA, tensor-memory allocation, MMA issue and commit to an mbarrier, a bounded wait on that
// mbarrier, and tensor-memory loads of the accumulator.
//
// Operand layout (K-major, no swizzle): a tile of R rows by 64 BF16 elements of K is stored as
// core matrices of 8 rows x 16 bytes (8 elements); core matrix (row / 8, k / 8) sits at byte
// ((row / 8) * 8 + k / 8) * 128, row r % 8 at 16 (r % 8) within it.  So the core matrices next
// to each other along K are 128 bytes apart and those along the rows 1024 bytes apart.
#pragma once

#include <cstdint>

namespace sfft {

constexpr int kTcKTile = 64;                  // BF16 elements of K per staged operand tile
constexpr uint32_t kTcKCoreStride = 128;      // bytes between core matrices along K
constexpr uint32_t kTcRowCoreStride = 1024;   // bytes between core matrices along the rows (8 K-cores)

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k), k < kTcKTile, in a staged operand tile
__device__ __forceinline__ int tc_core_off(int row, int k) {
  return (((row >> 3) * (kTcKTile / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

// Shared-memory matrix descriptor: start address, the byte offsets between core matrices along
// K (leading) and along the rows (stride), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lead, uint32_t stride) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lead >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((stride >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16 with BF16 A and B (both K-major) and an FP32 accumulator.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Tensor-memory columns for the accumulator (a power of two >= 32), by one whole warp.
__device__ __forceinline__ void tc_alloc(uint32_t* smem_result, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(smem_result)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// D (+)= A B^T for one K step of 16, issued by one thread.
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            bool accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u));
}

// The mbarrier's arrival once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      tc_smem_u32(mbar)));
}

__device__ __forceinline__ void tc_mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_u32(mbar)), "r"(count));
}

// Waits for the mbarrier's phase of the given parity with non-blocking tests and a sleep of
// 128 ns between them; gives up after max_iter tests (about max_iter x 0.2 us in all) and returns
// false, so that the caller reports the timeout instead of hanging.
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* mbar, uint32_t parity, int max_iter) {
  for (int it = 0; it < max_iter; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(tc_smem_u32(mbar)), "r"(parity));
    if (done) return true;
    __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void tc_fence_smem() { asm volatile("fence.proxy.async.shared::cta;"); }

// 16 consecutive FP32 accumulator columns of this warp's 32 lanes (warp w of a warpgroup reads
// lanes 32 (w % 4) .. 32 (w % 4) + 31: accumulator rows), then waits for the load.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace sfft
