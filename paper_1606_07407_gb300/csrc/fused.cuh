// Fused short-round kernel: once a signal's line is short, one block runs a round of
// Algorithm 2 end to end (tables, samples, Bluestein DFT, residual, ratio test and read-out,
// registry merge, plan of the next round), instead of a dozen batched launches per round
// that each have little work.  A round runs fused when its Bluestein length is at most the
// slot's limit: the largest length up to kFusedMaxL whose n_sets + 1 transforms (the rows and
// the filter) fit the block at once.  FP32 policies only.  (A 512-thread variant for lengths
// up to 2048 measured slower than the batched kernels on round 2 of the d = 5 workload: one
// block per SM leaves the sampling issue-bound and the batch in two waves.)
#pragma once

#include "fft_reg.cuh"
#include "round_steps.cuh"

namespace sfft {

constexpr int kFusedMaxL = 1024;       // longest Bluestein length of the fused path (half line <= 256)
constexpr int kFusedMaxSets = 7;       // most sample sets: n_sets + 1 transforms of >= 32 threads each
constexpr int kFusedChunk = 512;       // modes staged in shared memory at a time (two per thread)
constexpr int kFusedMaxD = 64;         // directions up to this many coordinates are kept in shared memory
constexpr int kFusedHostRounds = 4;    // fused rounds per round when the host enqueues rounds

// Device buffers and tables of the engine, as the fused kernel reads and writes them.
struct FusedArgs {
  PlanArgs pa;
  PrimeTables pt;
  const SigCfg* cfg;
  SigRun* run;
  RoundCtl* ctl;
  HistRec* hist;
  int64_t* ubuf;
  const int32_t* const* sig_w;
  const double2* const* sig_a;
  const float2* tw;       // the bound modes' twiddles (read only)
  const int32_t* shblk;
  int32_t* regw;
  double2* rega;
  float2* regtw;
  int32_t* hash;
  TwSrc<float2> tws;
  int L_alloc;            // the Bluestein length the shared memory was sized for
};

// Byte offsets of the fused kernel's shared memory for a round of Bluestein length L and
// n_sets sample sets (p <= (L + 1) / 2): the tables W and chirp, the n_sets + 1 padded DFT
// rows of ls values, and the work area (a chunk of modes, then the groups' partial sums, then
// the transforms Y_n).
struct FusedLayout {
  int tab, slots, work, total, ls;
};

__host__ __device__ inline FusedLayout fused_layout(int L, int n_sets) {
  auto up16 = [](int v) { return (v + 15) & ~15; };
  const int p_cap = (L + 1) / 2;
  FusedLayout f;
  f.ls = L + L / 32;
  f.tab = 0;
  f.slots = up16(2 * p_cap * 8);
  f.work = up16(f.slots + (n_sets + 1) * f.ls * 8);
  const int chunk = kFusedChunk * (4 + n_sets * 8);
  const int red = 256 * n_sets * 16;   // (G - 1) H <= 256 positions x n_sets x 4 sums
  const int ys = n_sets * p_cap * 8;
  f.total = up16(f.work + (chunk > red ? (chunk > ys ? chunk : ys) : (red > ys ? red : ys)));
  return f;
}

// Largest Bluestein length a slot of n_sets sample sets runs fused (0: none).
int fused_max_length(int n_sets);

// Dynamic shared memory of the fused kernel for slots of at most max_sets sample sets and
// fused lengths up to max_L.
size_t fused_smem_bytes(int max_sets, int max_L);

// Per set count ns <= kFusedMaxSets (instantiated in fused_ns<ns>.cu): the shared-memory
// attribute and one launch.
template <int NS> cudaError_t fused_setup_ns(size_t smem);
template <int NS> cudaError_t fused_launch_ns(int n_slots, size_t smem, cudaStream_t st, const FusedArgs& a);

// Allows that much dynamic shared memory for every set count.
cudaError_t fused_setup(size_t smem);

// One fused launch for the signals of ns sample sets (one block per signal slot; blocks of
// other signals return at once).
cudaError_t fused_launch(int ns, int n_slots, size_t smem, cudaStream_t st, const FusedArgs& a);

// After the fused launches of a round: counts it and, with use_cond, sets the graph condition
// of the loop of fused rounds to whether some signal has another fused round planned.
cudaError_t fused_tail(cudaStream_t st, RoundCtl* ctl, int use_cond, cudaGraphConditionalHandle cond);

}  // namespace sfft
