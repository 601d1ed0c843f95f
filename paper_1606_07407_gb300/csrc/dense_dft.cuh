// Kernel (b) for short primes as a dense contraction on the tensor cores: the length-p DFT
//     Y_n[h] = sum_x y_n[x] e^{-2 pi i h x / p}                                  (Eq. 3)
// of a signal's sample sets is D = A B^T with A the real form of the DFT matrix and B the
// samples.  Row m = 2 h + q of A gives the real (q = 0) or imaginary (q = 1) part of bin h;
// column k = 2 x + q' takes the real (q' = 0) or imaginary (q' = 1) part of sample x:
//     A[2h][2x] = cos t,  A[2h][2x+1] = sin t,  A[2h+1][2x] = -sin t,  A[2h+1][2x+1] = cos t,
// t = 2 pi ((h x) mod p) / p (the root table holds e^{i t} for every residue), and B[n][2x + q']
// the parts of y_n[x].  BF16 keeps 8 bits of each operand, so both are split, v = hi + lo with
// hi = bf16(v) and lo = bf16(v - hi) (8 significant bits each, so v - hi - lo is below 2^-16 |v|),
// and D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 in tensor memory (the dropped
// A_lo B_lo is below 2^-16 of each product).
//
// One block of four warps takes 64 bins (the 128 accumulator rows of a cta_group::1 MMA) of one
// signal and every sample set of it (N = sets rounded up to 16, at most 64); it stages K tiles of
// 32 samples (64 BF16 of K) in two buffers, so the next tile is built while the tensor core
// consumes the last.  One thread issues the MMAs; an mbarrier per buffer, committed after each
// tile's MMAs, tells the block when a buffer is free, with a bounded wait.  Every kDenseFlush
// tiles the accumulator is drained into FP32 registers (see there).
#pragma once

#include <cuda_bf16.h>

#include "engine.cuh"
#include "noise.cuh"
#include "round_steps.cuh"
#include "tc_mma.cuh"

namespace sfft {

constexpr int kDenseBins = 64;        // bins per block (128 accumulator rows)
constexpr int kDenseX = kTcKTile / 2; // samples per K tile
constexpr int kDenseMaxSets = 64;     // sample sets per signal (the MMA's N)
constexpr int kDenseThreads = 128;
constexpr int kDenseWaitPolls = 1 << 16;   // mbarrier tests before a wait gives up (about 15 ms)
// K tiles per accumulation segment: the tensor core's FP32 accumulation rounds each MMA's sum into
// the accumulator, and where the products add coherently (a bin holding one strong mode) those
// roundings add up too, about one unit in the last place of the growing partial sum per MMA; the
// accumulator is drained into registers every kDenseFlush tiles (12 kDenseFlush MMAs), so this
// error stays near 12 kDenseFlush 2^-24 |Y| whatever the length p
constexpr int kDenseFlush = 4;

struct DenseStage {
  unsigned char a_hi[128 * kTcKTile * 2];
  unsigned char a_lo[128 * kTcKTile * 2];
  unsigned char b_hi[kDenseMaxSets * kTcKTile * 2];
  unsigned char b_lo[kDenseMaxSets * kTcKTile * 2];
};
constexpr size_t kDenseSmem = 2 * sizeof(DenseStage) + 1024;   // two buffers, 1 KiB alignment slack

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  *hi = h;
  *lo = __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ void put_split(unsigned char* hi_tile, unsigned char* lo_tile, int row, int k, float v) {
  __nv_bfloat16 h, l;
  split_bf16(v, &h, &l);
  const int off = tc_core_off(row, k);
  *reinterpret_cast<__nv_bfloat16*>(hi_tile + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(lo_tile + off) = l;
}

// blockIdx.x: bin tile; blockIdx.y: signal slot.  Slots whose round does not run dense return.
__global__ void __launch_bounds__(kDenseThreads) k_dft_dense(int n, const SigCfg* __restrict__ cfg, SigRun* run,
                                                             const float2* __restrict__ part,
                                                             const float2* __restrict__ tab,
                                                             float2* __restrict__ Y) {
  extern __shared__ unsigned char dense_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int s = blockIdx.y;
  if (s >= n) return;
  SigRun* rp = run + s;
  const SigRun r = *rp;
  if (!r.active || !r.dense) return;
  const int p = (int)r.p;
  const int h0 = blockIdx.x * kDenseBins;
  if (h0 >= p) return;
  const SigCfg& c = cfg[s];
  const int rows = c.n_sets;
  const int nmma = rows <= 16 ? 16 : rows <= 32 ? 32 : rows <= 48 ? 48 : 64;
  const float2* W = tab + r.tab_at;   // W[m] = e^{2 pi i m / p}
  DenseStage* stage = reinterpret_cast<DenseStage*>(
      (reinterpret_cast<uintptr_t>(dense_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // the set rows past the signal's stay zero in both buffers
  for (int e = tid; e < (nmma - rows) * kTcKTile; e += blockDim.x) {
    const int row = rows + e / kTcKTile, k = e % kTcKTile;
    for (int b = 0; b < 2; ++b) {
      put_split(stage[b].b_hi, stage[b].b_lo, row, k, 0.0f);
    }
  }
  if (warp == 0) tc_alloc(&s_tmem, 64);
  if (tid == 0) {
    tc_mbar_init(&mbar[0], 1);
    tc_mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc_idesc_bf16(128, nmma);

  // A rows 2 hh, 2 hh + 1 of bin h0 + hh, samples xh .. xh + 15 of the tile (two threads a bin)
  const int hh = tid >> 1;
  const int h = h0 + hh;
  const int xh = (tid & 1) * (kDenseX / 2);
  const int n_tiles = (p + kDenseX - 1) / kDenseX;
  // this thread's accumulator row (warp 32 w + lane), summed over segments of kDenseFlush tiles in
  // registers with round-to-nearest additions
  float racc[kDenseMaxSets];
#pragma unroll
  for (int j = 0; j < kDenseMaxSets; ++j) racc[j] = 0.0f;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  bool fail = false;
  int last_commit = -1;
  for (int t = 0; t < n_tiles; ++t) {
    const int b = t & 1;
    DenseStage& S = stage[b];
    if (t >= 2) {   // the MMAs of tile t - 2 read this buffer (already done if a drain waited for them)
      const bool ok = tc_mbar_wait(&mbar[b], (uint32_t)(((t - 2) >> 1) & 1), kDenseWaitPolls);
      if (__syncthreads_or(ok ? 0 : 1)) {
        fail = true;
        break;
      }
    }
    const int x0 = t * kDenseX;
    {
      int64_t x = x0 + xh;
      int idx = h < p ? (int)(((int64_t)h * x) % p) : 0;
#pragma unroll 4
      for (int j = 0; j < kDenseX / 2; ++j, ++x) {
        float cs = 0.0f, sn = 0.0f;
        if (h < p && x < p) {
          const float2 w = __ldg(W + idx);
          cs = w.x;
          sn = w.y;
        }
        idx += h;
        if (idx >= p) idx -= p;
        const int k = 2 * (xh + j);
        put_split(S.a_hi, S.a_lo, 2 * hh, k, cs);
        put_split(S.a_hi, S.a_lo, 2 * hh, k + 1, sn);
        put_split(S.a_hi, S.a_lo, 2 * hh + 1, k, -sn);
        put_split(S.a_hi, S.a_lo, 2 * hh + 1, k + 1, cs);
      }
    }
    for (int e = tid; e < rows * kDenseX; e += blockDim.x) {
      const int row = e / kDenseX, xx = e % kDenseX, x = x0 + xx;
      float2 y = make_float2(0.0f, 0.0f);
      if (x < p) {
        y = sum_splits<float>(part, r, rows, row, x);
        if (r.noise_sigma > 0.0) y = cadd(y, black_box_noise<float>(r.noise_seed, r.round, row, x, r.noise_sigma));
      }
      put_split(S.b_hi, S.b_lo, row, 2 * xx, y.x);
      put_split(S.b_hi, S.b_lo, row, 2 * xx + 1, y.y);
    }
    tc_fence_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = tc_smem_u32(S.a_hi), al = tc_smem_u32(S.a_lo);
      const uint32_t bh = tc_smem_u32(S.b_hi), bl = tc_smem_u32(S.b_lo);
#pragma unroll
      for (int ks = 0; ks < kTcKTile / 16; ++ks) {   // K steps of 16: two core matrices along K
        const uint32_t o = (uint32_t)ks * 2 * kTcKCoreStride;
        const uint64_t dah = tc_desc(ah + o, kTcKCoreStride, kTcRowCoreStride);
        const uint64_t dal = tc_desc(al + o, kTcKCoreStride, kTcRowCoreStride);
        const uint64_t dbh = tc_desc(bh + o, kTcKCoreStride, kTcRowCoreStride);
        const uint64_t dbl = tc_desc(bl + o, kTcKCoreStride, kTcRowCoreStride);
        tc_mma_bf16(tmem, dah, dbh, idesc, (t % kDenseFlush) != 0 || ks > 0);   // a segment starts afresh
        tc_mma_bf16(tmem, dah, dbl, idesc, true);
        tc_mma_bf16(tmem, dal, dbh, idesc, true);
      }
      tc_commit(&mbar[b]);
    }
    last_commit = t;
    if ((t + 1) % kDenseFlush == 0 || t == n_tiles - 1) {
      // drain the segment: its last commit covers every MMA before it; the accumulator's partial
      // sums go into the registers, and the next segment's first MMA overwrites it
      const bool ok = tc_mbar_wait(&mbar[b], (uint32_t)((t >> 1) & 1), kDenseWaitPolls);
      if (__syncthreads_or(ok ? 0 : 1)) {
        fail = true;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int cb = 0; cb < kDenseMaxSets / 16; ++cb) {
        if (cb * 16 < nmma) {
          float v[16];
          tc_ld16(trow + (uint32_t)(cb * 16), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) racc[cb * 16 + j] += v[j];
        }
      }
      tc_fence_before();
      __syncthreads();   // every warp has read the accumulator before the next MMA writes it
    }
  }
  if (!fail) {
    // accumulator row m = 32 warp + lane: part q = m & 1 of bin h0 + m / 2; column n: set n
    const int m = warp * 32 + lane;
    const int hb = h0 + (m >> 1), q = m & 1;
    float* Yf = reinterpret_cast<float*>(Y + c.Y_off);
    const float o = __shfl_xor_sync(0xffffffffu, racc[0], 1);   // the other part of set 0's bin
    const float m2 = hb < p ? racc[0] * racc[0] + o * o : 0.0f;
#pragma unroll
    for (int j = 0; j < kDenseMaxSets; ++j)
      if (j < rows && hb < p) Yf[2 * ((int64_t)j * p + hb) + q] = racc[j];
    max_abs_to<float>(&rp->maxy0_bits, sqrt((double)m2));   // the whole warp: it reduces over the lanes
  } else if (tid == 0) {
    s_fail = 1;
    atomicOr(&rp->err, kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (s_fail && last_commit >= 0) {
    // MMAs may still be in flight: give them one more bounded wait before the columns go back
    (void)tc_mbar_wait(&mbar[last_commit & 1], (uint32_t)((last_commit >> 1) & 1), kDenseWaitPolls);
  }
  if (warp == 0) tc_dealloc(tmem, 64);
}

}  // namespace sfft
