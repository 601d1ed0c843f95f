// Host side of the fused short-round kernel: which rounds a slot runs fused, the kernel's
// shared memory, and the launches (the kernel itself is in fused_kernel.cuh, instantiated by
// fused_ns*.cu).
#include <algorithm>
#include <vector>

#include "fused.cuh"
#include "sample_tile.cuh"

namespace sfft {

namespace {

// After each fused launch: whether another one has work (the loop of fused rounds in the graph).
__global__ void k_fused_tail(RoundCtl* ctl, int use_cond, cudaGraphConditionalHandle cond) {
  const unsigned long long v = ctl->n_fused_next;
  ctl->n_fused_next = 0ull;
  ctl->fused_iters += 1;
  if (use_cond) cudaGraphSetConditional(cond, v > 0ull ? 1u : 0u);
}

// Bluestein lengths m 2^a (m in {1, 3, 5}) of the fused path, 32 <= L <= kFusedMaxL, in order
std::vector<int> fused_lengths() {
  std::vector<int> v;
  for (int m = 1; m <= 5; m += 2)
    for (int L = m; L <= kFusedMaxL; L *= 2)
      if (L >= 32) v.push_back(L);
  std::sort(v.begin(), v.end());
  return v;
}

}  // namespace

int fused_max_length(int n_sets) {
  if (n_sets > kFusedMaxSets) return 0;
  int best = 0;
  for (int L : fused_lengths()) {
    if ((n_sets + 1) * fft_threads<float2>(L) > kSampleThreads) break;   // the lengths from here on
    best = L;
  }
  return best;
}

size_t fused_smem_bytes(int max_sets, int max_L) {
  int b = 0;
  for (int L : fused_lengths())
    if (L <= max_L) b = std::max(b, fused_layout(L, max_sets).total);
  return (size_t)b;
}

cudaError_t fused_setup(size_t smem) {
  cudaError_t e;
  if ((e = fused_setup_ns<1>(smem)) != cudaSuccess) return e;
  if ((e = fused_setup_ns<2>(smem)) != cudaSuccess) return e;
  if ((e = fused_setup_ns<3>(smem)) != cudaSuccess) return e;
  if ((e = fused_setup_ns<4>(smem)) != cudaSuccess) return e;
  if ((e = fused_setup_ns<5>(smem)) != cudaSuccess) return e;
  if ((e = fused_setup_ns<6>(smem)) != cudaSuccess) return e;
  return fused_setup_ns<7>(smem);
}

cudaError_t fused_tail(cudaStream_t st, RoundCtl* ctl, int use_cond, cudaGraphConditionalHandle cond) {
  k_fused_tail<<<1, 1, 0, st>>>(ctl, use_cond, cond);
  return cudaGetLastError();
}

cudaError_t fused_launch(int ns, int n_slots, size_t smem, cudaStream_t st, const FusedArgs& a) {
  switch (ns) {
    case 1: return fused_launch_ns<1>(n_slots, smem, st, a);
    case 2: return fused_launch_ns<2>(n_slots, smem, st, a);
    case 3: return fused_launch_ns<3>(n_slots, smem, st, a);
    case 4: return fused_launch_ns<4>(n_slots, smem, st, a);
    case 5: return fused_launch_ns<5>(n_slots, smem, st, a);
    case 6: return fused_launch_ns<6>(n_slots, smem, st, a);
    case 7: return fused_launch_ns<7>(n_slots, smem, st, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sfft
