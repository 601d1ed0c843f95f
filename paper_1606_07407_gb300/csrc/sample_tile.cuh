// One tile of the sample-and-residual computation (Alg. 2 sampling; Eq. 41), shared
// by the batched engine and the allocation-free sampling entry point.
//
//   y_n[x] = sum_j C[n][j] W[(alpha_j x) mod p],  x = x0 + 32 row + lane,
//   W[(alpha x) mod p] = W[(alpha (x0 + 32 row)) mod p] * W[(alpha lane) mod p],
//
// the first factor shared by the 32 lanes of a row, the second by the rows of a lane.
#pragma once

#include "engine_kernels.cuh"

namespace sfft {

constexpr int kSampleThreads = kSampleWarps * 32;

template <typename T, int NS>
struct SampleSmem {
  c2<T> Ls[kSampleChunk][32];
  c2<T> Us[kSampleChunk][4 * rows_per_warp(NS)];
  c2<T> Cs[kSampleChunk][NS];
  int al[kSampleChunk], be[kSampleChunk], ga[kSampleChunk];
  int64_t item;
};

// One tile: 32 * 4 * RW samples x the sets of one group x the modes of one split.
// Each 32-mode chunk is summed into fresh accumulators that are then added to the
// running totals (blocked summation), which keeps the float rounding of long mode
// sums near that of the individual terms.
template <typename T, int NS>
__device__ void sample_tile(SampleSmem<T, NS>& sm, const SigCfg& c, const SigRun& r, int xt, int g, int split,
                            const int32_t* __restrict__ alpha, const int32_t* __restrict__ gam,
                            const c2<T>* __restrict__ Cm, const c2<T>* __restrict__ W, c2<T>* __restrict__ part) {
  using C2 = c2<T>;
  constexpr int RW = rows_per_warp(NS);
  constexpr int TX = tile_x(NS);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p = (int)r.p;
  const float inv_p = 1.0f / (float)p;
  const int n0 = g * r.gsize;
  const int ns_valid = min(r.gsize, c.n_sets - n0);
  const int K = r.k_sig + min(r.K_reg, c.reg_cap);
  const int x0 = xt * TX;
  const int j_begin = split * r.jper;
  const int j_end = min(K, j_begin + r.jper);
  const C2 zero = mk2((T)0, (T)0);

  T tot[RW][NS][2];
#pragma unroll
  for (int q = 0; q < RW; ++q)
#pragma unroll
    for (int nn = 0; nn < NS; ++nn) tot[q][nn][0] = tot[q][nn][1] = (T)0;

  for (int jc = j_begin; jc < j_end; jc += kSampleChunk) {
    const int nj = min(kSampleChunk, j_end - jc);
    if (tid < kSampleChunk) {
      const int al = (tid < nj) ? alpha[jc + tid] : 0;
      sm.al[tid] = al;
      sm.ga[tid] = (tid < nj) ? gam[jc + tid] : 0;
      sm.be[tid] = (int)mod_barrett((uint64_t)al * (uint64_t)x0, (uint64_t)p, r.mod_m);
    }
    for (int e = tid; e < kSampleChunk * NS; e += kSampleThreads) {
      const int jj = e / NS, nn = e - jj * NS;
      sm.Cs[jj][nn] = (jj < nj && nn < ns_valid) ? Cm[(int64_t)(n0 + nn) * c.Kmax + jc + jj] : zero;
    }
    __syncthreads();
    for (int e = tid; e < kSampleChunk * 32; e += kSampleThreads) {
      const int jj = e >> 5, ln = e & 31;
      sm.Ls[jj][ln] = W[mod_small((unsigned)sm.al[jj] * (unsigned)ln, p, inv_p)];
    }
    for (int e = tid; e < kSampleChunk * 4 * RW; e += kSampleThreads) {
      const int jj = e / (4 * RW), row = e - jj * (4 * RW);
      sm.Us[jj][row] = W[mod_small((unsigned)sm.be[jj] + (unsigned)row * (unsigned)sm.ga[jj], p, inv_p)];
    }
    __syncthreads();
    T acc[RW][NS][2];
#pragma unroll
    for (int q = 0; q < RW; ++q)
#pragma unroll
      for (int nn = 0; nn < NS; ++nn) acc[q][nn][0] = acc[q][nn][1] = (T)0;
#pragma unroll 2
    for (int jj = 0; jj < kSampleChunk; ++jj) {
      const C2 L = sm.Ls[jj][lane];
      C2 E[RW];
#pragma unroll
      for (int q = 0; q < RW; ++q) E[q] = cmul(sm.Us[jj][warp * RW + q], L);
#pragma unroll
      for (int nn = 0; nn < NS; ++nn) {
        const C2 cc = sm.Cs[jj][nn];
#pragma unroll
        for (int q = 0; q < RW; ++q) {
          acc[q][nn][0] = fma(cc.x, E[q].x, acc[q][nn][0]);
          acc[q][nn][0] = fma(-cc.y, E[q].y, acc[q][nn][0]);
          acc[q][nn][1] = fma(cc.x, E[q].y, acc[q][nn][1]);
          acc[q][nn][1] = fma(cc.y, E[q].x, acc[q][nn][1]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RW; ++q)
#pragma unroll
      for (int nn = 0; nn < NS; ++nn) {
        tot[q][nn][0] += acc[q][nn][0];
        tot[q][nn][1] += acc[q][nn][1];
      }
    __syncthreads();
  }
  C2* out = part + r.part_off;
#pragma unroll
  for (int q = 0; q < RW; ++q) {
    const int x = x0 + (warp * RW + q) * 32 + lane;
    if (x < p) {
#pragma unroll
      for (int nn = 0; nn < NS; ++nn)
        if (nn < ns_valid) out[((int64_t)split * c.n_sets + n0 + nn) * p + x] = mk2(tot[q][nn][0], tot[q][nn][1]);
    }
  }
}

}  // namespace sfft
