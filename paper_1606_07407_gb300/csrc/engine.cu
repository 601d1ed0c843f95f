// Kernels and host driver of the batched round engine (Algorithm 2 for many
// signals at once).  One round, for every active signal s of the batch:
//
//   k_plan_signals, k_plan_scan, k_plan_offsets (grid)
//                            k* = max(k - |R|, 1), p = i-th prime >= c k* (Alg. 2), direction
//                            u of the round reduced mod p, work geometry, mode splits, exclusive
//                            scans of the per-signal work counts; ends the device loop when no
//                            signal is left
//   k_tables                 W[m] = e^{2 pi i m / p} and chirp[x] = e^{-pi i x^2 / p}
//   k_sample    (persistent) y_n[x] = (f - g)(x u / p + e_n / N) for all n (Eq. 41), the modes'
//                            projection alpha = (w . u) mod p fused into the staging
//   k_filter / k_dft         Bluestein DFT (Eq. 3) in shared memory, or the four-step passes
//   k_big{A,B,C}             for lengths above one block
//   k_classify               ratio test, read-out, own-bin check (Eq. 41-42), hash merge into the
//                            registry with pruning, empty-bin flag for the stop rule
//
// The host only enqueues rounds (or launches one CUDA graph whose while-loop the
// planning kernels end), and reads results back once.
#include <algorithm>
#include <cstring>
#include <memory>

#include "engine_kernels.cuh"
#include "fft_reg.cuh"
#include "fft_smem.cuh"
#include "fused.cuh"
#include "noise.cuh"
#include "round_steps.cuh"
#include "sample_tile.cuh"
#include "dense_dft.cuh"

namespace sfft {

namespace {

constexpr int kBindArrays = 8;   // per-signal arrays staged by bind()
// Owner election of the batched signals that share a prime: powner[p] = min over this round's
// claimants of (0xFFFFFFFF - epoch) << 32 | slot.  A later epoch has the smaller high word, so
// keys of earlier rounds never win and the table needs no clearing (all ones at creation).
__device__ __forceinline__ unsigned long long owner_key(unsigned int epoch, int s) {
  return ((unsigned long long)(0xFFFFFFFFu - epoch) << 32) | (unsigned int)s;
}

// round 1 of a slot whose root tables and filter were made with the engine: no owner needed
__device__ __forceinline__ bool uses_engine_tables(const PlanArgs& a, const SigCfg& c, const SigRun& r) {
  return !a.force && r.round == 1 && c.tab0_off >= 0 && r.p == c.p1;
}

inline unsigned long long double_bits(double v) {
  unsigned long long u;
  std::memcpy(&u, &v, sizeof(u));
  return u;
}

// ------------------------------------------------------------------ init / bind

// bindv: the staged per-signal arrays (k at [2n, 3n), noise sigma bits at [6n, 7n), seed at [7n, 8n))
__global__ void k_init(int n, SigRun* run, const int64_t* __restrict__ bindv) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    SigRun r;
    memset(&r, 0, sizeof(r));
    r.active = 1;
    r.k_sig = (int)bindv[2 * n + s];
    r.noise_sigma = __longlong_as_double((long long)bindv[6 * n + s]);
    r.noise_seed = (unsigned long long)bindv[7 * n + s];
    run[s] = r;
  }
}

// A registry to start from (slot 0 of a one-slot engine): entry j takes the seed's key and
// coefficient, its twiddles e^{2 pi i w . s_n} and a hash slot; the slot's state continues after
// round0 rounds with the empty-bin reference of the run that found the entries.  Seed keys are
// distinct (a registry's), so the hash insert compares nothing.
template <typename T>
__global__ void k_seed(const SigCfg* __restrict__ cfg, SigRun* run, const int32_t* __restrict__ seed_w,
                       const double2* __restrict__ seed_a, int n_seed, int round0, double a_ref,
                       const int32_t* __restrict__ shblk, int32_t* regw, double2* rega, c2<T>* regtw, int32_t* hash) {
  const SigCfg& c = cfg[0];
  SigRun* rp = run;
  const int d = c.d, S = c.n_sets - 1;
  const int32_t* blk = shblk + c.blk_off;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_seed; j += gridDim.x * blockDim.x) {
    const int32_t* w = seed_w + (int64_t)j * d;
    int32_t* rw = regw + c.regw_off + (int64_t)j * d;
    for (int l = 0; l < d; ++l) rw[l] = w[l];
    const double2 a = seed_a[j];
    rega[c.rega_off + j] = a;
    for (int n = 1; n <= S; ++n) regtw[c.regtw_off + (int64_t)j * S + n - 1] = shift_root<T>(c, blk, w, n, true);
    int32_t* hs = hash + c.hash_off;
    int slot = (int)(hash_key(w, d) & (unsigned long long)c.hash_mask);
    for (int probe = 0; probe <= c.hash_mask; ++probe, slot = (slot + 1) & c.hash_mask)
      if (atomicCAS(&hs[slot], -1, j) < 0) break;
    if (a.x != 0.0 || a.y != 0.0) atomicAdd(&rp->n_live, 1);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    rp->K_reg = n_seed;
    rp->round = round0;
    rp->a_ref = a_ref;
    rp->any_occupied = 1;   // the round handed over is no empty round of the stop rule
  }
}

// twiddles e^{2 pi i w_j . s_n} of the bound signals' modes, one per shifted set (shift_root)
template <typename T>
__global__ void k_bind_tw(int n, const SigCfg* __restrict__ cfg, const SigRun* __restrict__ run,
                          const int32_t* const* __restrict__ sig_w, const int32_t* __restrict__ shblk,
                          c2<T>* __restrict__ tw) {
  const int s = blockIdx.y;
  if (s >= n) return;
  const SigCfg& c = cfg[s];
  const int S = c.n_sets - 1;
  const int64_t total = (int64_t)run[s].k_sig * S;
  const int32_t* w = sig_w[s];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / S;
    const int nn = (int)(e - j * S) + 1;
    tw[c.tw_off + e] = shift_root<T>(c, shblk + c.blk_off, w + j * c.d, nn, false);
  }
}

// ------------------------------------------------------------------ plan

// Planning: every signal's round (plan_signal; a signal whose next round the fused kernel has
// planned keeps it), the round's totals and the mode splits (k_plan_signals and its last
// block), the work counts of the batched kernels and their exclusive scans over the signals
// (k_plan_scan within blocks, its last block across them; k_plan_offsets).  The last block of
// k_plan_scan sets the graph conditions: some signal active (the round loop), some batched
// work, some fused round planned.
// Rows of one signal that one block of the DFT takes together (they share p, the chirp, the
// filter spectrum and the twiddles): as many as the block has whole-warp groups of the threads a
// row needs, and as the block's shared memory holds padded rows plus one prefetch row of L.
template <typename C2>
__host__ __device__ inline int dft_group_rows(int L, int nthr, int64_t smem_elems, int n_sets, int e = 0) {
  const int need = e == 16 ? fft_threads<C2, 16>(L) : fft_threads<C2>(L);
  int g = nthr / need;
  const int64_t rowpad = (L + L / 32 + 1) & ~1;
  while (g > 1 && (int64_t)g * rowpad + L > smem_elems) --g;
  if (g < 1) g = 1;
  return g < n_sets ? g : n_sets;
}

// The round's mode splits, by the last block of k_plan_signals (all of its threads; the round's
// totals in acc, the blocks' tiles and tail sums in blk).  S (1..64): the persistent sampling
// kernel's 2 n_sm blocks take tiles x S items of 1/S of the modes each; S minimises its waves per
// unit of work, ceil(items / blocks) / S, with 12% per extra split for the partial sums it adds
// and the DFT reads back, then it is halved until the partial sums fit their arena.  Tail: when
// the items (tiles unsplit) leave the last wave mostly empty (rem of 2 n_sm blocks busy), the
// signals whose tiles fall in that wave split their modes q ways, so that their work spreads
// over the idle blocks, if the partial sums still fit.  Also gives each block its exclusive
// offset in the queue of tiles.
__device__ void plan_decide(const PlanArgs& a, const SigCfg* __restrict__ cfg, const SigRun* run, const PlanAcc* acc,
                            PlanBlk* blk, PlanDec* dec, int nblk) {
  __shared__ unsigned long long s_key;
  __shared__ int s_S;
  __shared__ int64_t s_part, s_extra;
  __shared__ int s_bstar;
  const int64_t tot_tiles = (int64_t)__ldcg(&acc->tiles);
  if (threadIdx.x == 0) {
    s_key = ~0ull;
    s_bstar = nblk;
    s_extra = 0;
  }
  __syncthreads();
  if (threadIdx.x < 64 && tot_tiles > 0) {
    const int64_t S = threadIdx.x + 1;
    const int64_t slots = 2LL * a.n_sm;
    const int64_t waves = (tot_tiles * S + slots - 1) / slots;
    const unsigned long long score = (unsigned long long)((waves * (100 + 12 * (S - 1)) << 20) / S);
    atomicMin(&s_key, (score << 6) | (unsigned long long)(S - 1));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // partial-sum elements sum_s min(S, chunks_s) n_sets p_s from the histogram by chunks
    int S = tot_tiles > 0 ? (int)(s_key & 63ull) + 1 : 1;
    for (;;) {
      int64_t tot = 0;
      for (int q = 1; q <= 64; ++q) tot += (int64_t)min(S, q) * (int64_t)__ldcg(&acc->wsum[q]);
      s_part = tot;
      if (tot <= a.part_cap || S == 1) break;
      S /= 2;
    }
    s_S = S;
  }
  __syncthreads();
  const int S = s_S;
  const int64_t slots = 2LL * a.n_sm;
  const int64_t rem = tot_tiles % slots;
  const int64_t tail_from = tot_tiles - rem;   // queue position (in tiles) where the last wave starts
  int q_tail = 1;
  if (S == 1 && rem > 0 && 5 * rem < 4 * slots) {
    const int q = (int)min((int64_t)8, max((int64_t)2, slots / rem));
    // blocks' exclusive tile offsets; the first block whose tiles reach into the last wave
    int64_t carry = 0;
    for (int base = 0; base < nblk; base += blockDim.x) {
      const int b = base + threadIdx.x;
      int64_t tv[1] = {b < nblk ? (int64_t)__ldcg(&blk[b].tiles) : 0}, tt[1];
      const int64_t tb = tv[0];
      block_scan_excl<1>(tv, tt);
      if (b < nblk) {
        blk[b].tile_off = carry + tv[0];
        if (carry + tv[0] + tb > tail_from) atomicMin(&s_bstar, b);
      }
      carry += tt[0];
    }
    __syncthreads();
    const int bstar = s_bstar;
    // the blocks after it are in the tail whole; the boundary block signal by signal
    int64_t extra = 0;
    for (int b = bstar + 1 + (int)threadIdx.x; b < nblk; b += blockDim.x) extra += (int64_t)__ldcg(&blk[b].extra[q - 2]);
    if (bstar < nblk) {
      const int s = bstar * kPlanBlk + (int)threadIdx.x;
      bool batched = false;
      int64_t tv[1] = {0}, tt[1];
      int chunks = 0;
      int64_t w = 0;
      if (threadIdx.x < kPlanBlk && s < a.n) {
        const int active = __ldcg(&run[s].active), fused = __ldcg(&run[s].fused);
        batched = active && !fused;
        if (batched) {
          tv[0] = (int64_t)__ldcg(&run[s].n_xt) * __ldcg(&run[s].groups);
          chunks = __ldcg(&run[s].chunks);
          w = (int64_t)cfg[s].n_sets * __ldcg(&run[s].p);
        }
      }
      const int64_t tiles_s = tv[0];
      block_scan_excl<1>(tv, tt);
      if (batched && __ldcg(&blk[bstar].tile_off) + tv[0] + tiles_s > tail_from)
        extra += (int64_t)max(min(q, chunks) - 1, 0) * w;
    }
    const int64_t tot_extra = block_sum(extra);
    if (s_part + tot_extra <= a.part_cap) q_tail = q;
  }
  if (threadIdx.x == 0) {
    dec->S = S;
    dec->q_tail = q_tail;
    dec->tail_from = tail_from;
  }
}

// The round's parameters of every signal not already planned by the fused kernel (stop rule,
// prime, direction mod p, work geometry: plan_signal), one thread per signal over the whole
// grid.  The same threads then add the round's totals into acc (active and fused signals, batched
// tiles, and the histogram of n_sets p by mode chunks from which the mode splits are sized),
// elect each shared prime's owner, and give their block's batched tiles and, for each tail split
// q = 2..8, the partial sums those splits would add (blk).  The last block to finish (the
// others' results visible to it through the fence before its arrival) then decides the round's
// splits: S for every signal, q_tail for those whose tiles fall in the sampling queue's last
// wave (dec).
template <typename T>
__global__ void __launch_bounds__(kPlanBlk) k_plan_signals(PlanArgs a, const SigCfg* __restrict__ cfg, SigRun* run,
                                                           const int32_t* __restrict__ ptab, int n_ptab,
                                                           const int32_t* __restrict__ pfirst, int64_t pfirst_n,
                                                           const int64_t* __restrict__ dirs,
                                                           const int64_t* __restrict__ plist, int64_t* ubuf,
                                                           HistRec* hist, PlanAcc* acc,
                                                           unsigned long long* __restrict__ powner, PlanBlk* blk,
                                                           PlanDec* dec) {
  __shared__ unsigned long long s_tot[3], s_w[65], s_extra[7];
  __shared__ int s_last;
  for (int i = threadIdx.x; i < 65; i += blockDim.x) s_w[i] = 0ull;
  if (threadIdx.x < 3) s_tot[threadIdx.x] = 0ull;
  if (threadIdx.x < 7) s_extra[threadIdx.x] = 0ull;
  __syncthreads();
  const unsigned int epoch = acc->epoch;
  const PrimeTables pt{ptab, n_ptab, pfirst, pfirst_n, dirs, plist};
  const int s = blockIdx.x * kPlanBlk + threadIdx.x;   // one signal per thread (grid: ceil(n / kPlanBlk))
  if (s < a.n) {
    SigRun r = run[s];
    if (!(r.active && r.fused)) {
      plan_signal<T>(a, cfg[s], r, pt, ubuf, hist, s == 0);
      run[s] = r;
    }
    if (r.active) {
      atomicAdd(&s_tot[1], 1ull);
      if (r.fused) {
        atomicAdd(&s_tot[2], 1ull);
      } else {
        const unsigned long long w = (unsigned long long)cfg[s].n_sets * (unsigned long long)r.p;
        atomicAdd(&s_tot[0], (unsigned long long)r.n_xt * (unsigned long long)r.groups);
        atomicAdd(&s_w[min(r.chunks, 64)], w);
        for (int q = 2; q <= 8; ++q)
          if (min(q, r.chunks) > 1) atomicAdd(&s_extra[q - 2], (unsigned long long)(min(q, r.chunks) - 1) * w);
        if (!uses_engine_tables(a, cfg[s], r)) atomicMin(&powner[r.p], owner_key(epoch, s));
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 3 && s_tot[threadIdx.x]) atomicAdd(&(&acc->tiles)[threadIdx.x], s_tot[threadIdx.x]);
  for (int i = threadIdx.x; i < 65; i += blockDim.x)
    if (s_w[i]) atomicAdd(&acc->wsum[i], s_w[i]);
  if (threadIdx.x == 0) blk[blockIdx.x].tiles = s_tot[0];
  if (threadIdx.x < 7) blk[blockIdx.x].extra[threadIdx.x] = s_extra[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&dec->done1, 1u) == gridDim.x - 1 ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  plan_decide(a, cfg, run, acc, blk, dec, (int)gridDim.x);
  if (threadIdx.x == 0) dec->done1 = 0u;
}

template <typename T>
__global__ void __launch_bounds__(kPlanBlk) k_plan_scan(PlanArgs a, const SigCfg* __restrict__ cfg, SigRun* run,
                                                        RoundCtl* ctl, Scans sc, PlanAcc* acc,
                                                        const unsigned long long* __restrict__ powner, PlanBlk* blk,
                                                        PlanDec* dec) {
  __shared__ int s_last;
  const int n = a.n;
  const int S = dec->S, q_tail = dec->q_tail;
  const int64_t tail_from = dec->tail_from;
  const int s = blockIdx.x * kPlanBlk + threadIdx.x;
  int64_t v[kNumScans + 1];
#pragma unroll
  for (int q = 0; q <= kNumScans; ++q) v[q] = 0;
  SigRun r;
  bool batched = false;   // active and not left to the fused kernel
  if (s < n) {
    r = run[s];
    batched = r.active && !r.fused;
  }
  bool in_tail = false;   // the signal's tiles reach into the last wave (split q_tail ways)
  if (q_tail > 1) {
    int64_t tv[1] = {batched ? (int64_t)r.n_xt * r.groups : 0}, tt[1];
    const int64_t tiles_s = tv[0];
    block_scan_excl<1>(tv, tt);
    in_tail = batched && blk[blockIdx.x].tile_off + tv[0] + tiles_s > tail_from;
  }
  // Batched signals with the same prime share one copy of the tables (W, chirp) and of the filter
  // spectrum: that of the first of them, the owner elected in powner[p] by k_plan_signals.  Round
  // 1 with the tables made with the engine needs no owner.
  if (batched && uses_engine_tables(a, cfg[s], r)) {
    r.tab_at = cfg[s].tab0_off;
    r.bhat_at = cfg[s].bhat0_off;
    r.tab_owner = 0;
  } else if (batched) {
    const int own = (int)(powner[r.p] & 0xFFFFFFFFull);
    r.tab_at = cfg[own].tab_off;
    r.bhat_at = cfg[own].bhat_off;
    r.tab_owner = own == s ? 1 : 0;
  }
  if (batched) {
    const SigCfg& c = cfg[s];
    const int K = a.force ? a.force_K : sampled_modes(c, r);
    const int sp = min(in_tail ? q_tail : S, r.chunks);
    r.jper = ((r.chunks + sp - 1) / sp) * kSampleChunk;
    r.splits = K > 0 ? (K + r.jper - 1) / r.jper : 1;
    v[SC_TAB] = r.tab_owner ? r.p : 0;
    v[SC_MODE] = K;
    // constant indices only: a computed index would put v in local memory
#pragma unroll
    for (int q = 0; q < kMaxSetGroup; ++q)
      if (q == r.gsize - 1) v[SC_SAMP0 + q] = (int64_t)r.n_xt * r.groups * r.splits;
    v[SC_BINS] = r.p;
    if (r.dense) {
      // the dense tensor-core kernel takes the signal's rows (no Bluestein row or filter)
    } else if (!r.big) {
      const bool sm = r.L <= (1 << kSmallFftLog);
      const int g = dft_group_rows<c2<T>>(r.L, sm ? a.dft_thr_s : a.dft_thr_l,
                                         (sm ? a.dft_smem_s : a.dft_smem_l) / (int64_t)sizeof(c2<T>), c.n_sets,
                                         sm ? a.dft_e_s : a.dft_e_l);
      const int64_t groups = (c.n_sets + g - 1) / g;   // row groups
      if (sm) {
        v[SC_ROWS_S] = groups;
        v[SC_FILT_S] = r.tab_owner;
      } else {
        v[SC_ROWS] = groups;
        v[SC_FILT] = r.tab_owner;
      }
    } else {
      int M1, M2, CT, RT;
      big_geom(r.logL, &M1, &M2, &CT, &RT);
      v[SC_BIGA] = (int64_t)(c.n_sets + 1) * (M2 / CT);
      v[SC_BIGB] = (int64_t)c.n_sets * (M1 / RT);
      v[SC_BIGC] = (int64_t)c.n_sets * (M2 / CT);
    }
    v[kNumScans] = (int64_t)r.splits * c.n_sets * r.p;
  }
  int64_t tot[kNumScans + 1];
  block_scan_excl<kNumScans + 1>(v, tot);
  // offsets within the block; k_plan_offsets adds the block's offset
  if (s < n) {
#pragma unroll
    for (int q = 0; q < kNumScans; ++q) sc.v[q][s] = v[q];
    if (batched) {   // the fields this pass sets (the whole record would be 224 bytes of stores)
      SigRun& o = run[s];
      o.tab_at = r.tab_at;
      o.bhat_at = r.bhat_at;
      o.tab_owner = r.tab_owner;
      o.jper = r.jper;
      o.splits = r.splits;
      o.part_off = v[kNumScans];
    }
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q <= kNumScans; ++q) blk[blockIdx.x].tot[q] = tot[q];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&dec->done2, 1u) == gridDim.x - 1 ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last block: exclusive scan of the blocks' totals (kept in blk[b].tot as offsets), the
  // round's totals into the scans' last entries and the round control, the graph conditions
  const int nblk = (int)gridDim.x;
  int64_t carry[kNumScans + 1];
#pragma unroll
  for (int q = 0; q <= kNumScans; ++q) carry[q] = 0;
  for (int base = 0; base < nblk; base += blockDim.x) {
    const int b = base + threadIdx.x;
    int64_t bv[kNumScans + 1];
#pragma unroll
    for (int q = 0; q <= kNumScans; ++q) bv[q] = b < nblk ? __ldcg(&blk[b].tot[q]) : 0;
    int64_t bt[kNumScans + 1];
    block_scan_excl<kNumScans + 1>(bv, bt);
    if (b < nblk) {
#pragma unroll
      for (int q = 0; q <= kNumScans; ++q) blk[b].tot[q] = carry[q] + bv[q];
    }
#pragma unroll
    for (int q = 0; q <= kNumScans; ++q) carry[q] += bt[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int64_t tot_active = (int64_t)acc->active;
    const int64_t tot_fused = (int64_t)acc->fused;
#pragma unroll
    for (int q = 0; q < kNumScans; ++q) sc.v[q][n] = carry[q];
    RoundCtl c;
    c.active = (int)tot_active;
    c.round = ctl->round + 1;
    c.splits = S;
    c.pad = 0;
    c.n_tab = carry[SC_TAB];
    c.n_mode = carry[SC_MODE];
    for (int q = 0; q < kMaxSetGroup; ++q) {
      c.n_samp[q] = carry[SC_SAMP0 + q];
      c.ctr_samp[q] = 0ull;
    }
    c.n_rows = carry[SC_ROWS];
    c.n_filt = carry[SC_FILT];
    c.n_bins = carry[SC_BINS];
    c.n_bigA = carry[SC_BIGA];
    c.n_bigB = carry[SC_BIGB];
    c.n_bigC = carry[SC_BIGC];
    c.n_rows_s = carry[SC_ROWS_S];
    c.n_filt_s = carry[SC_FILT_S];
    c.ctr_rows = c.ctr_filt = 0ull;
    c.n_cand = 0ull;
    c.n_fused_next = 0ull;
    const bool any_batched = tot_active > tot_fused;
    c.bodies_batched = ctl->bodies_batched + (any_batched ? 1 : 0);
    c.fused_iters = ctl->fused_iters;
    *ctl = c;
    if (a.use_cond) {
      cudaGraphSetConditional(a.cond, tot_active > 0 ? 1u : 0u);
      cudaGraphSetConditional(a.cond_batch, any_batched ? 1u : 0u);
      if (a.fuse) cudaGraphSetConditional(a.cond_fused, tot_fused > 0 ? 1u : 0u);   // handle exists
    }
    // the round's totals are read: clear them for the next round
    acc->tiles = acc->active = acc->fused = 0ull;
    acc->epoch += 1;
    dec->done2 = 0u;
  }
  for (int i = threadIdx.x; i < 65; i += blockDim.x) acc->wsum[i] = 0ull;
}

// the blocks' offsets added to the scans and to the partial-sum offsets
__global__ void __launch_bounds__(kPlanBlk) k_plan_offsets(int n, SigRun* run, Scans sc, const PlanBlk* __restrict__ blk) {
  const int s = blockIdx.x * kPlanBlk + threadIdx.x;
  if (s >= n) return;
  const PlanBlk& b = blk[blockIdx.x];
#pragma unroll
  for (int q = 0; q < kNumScans; ++q) sc.v[q][s] += b.tot[q];
  SigRun& r = run[s];
  if (r.active && !r.fused) r.part_off += b.tot[kNumScans];
}

// ------------------------------------------------------------------ tables

// Per-prime tables (W, chirp) and the round's mode projections: for every mode j of f (+a)
// and of the registry (-a): alpha_j = (w_j . u) mod p, ga_j = 32 alpha_j mod p and
// C[n][j] = a_j e^{2 pi i w_{j,n} / N} (n >= 1), C[0][j] = a_j.
template <typename T>
__global__ void k_tables(int n, const SigCfg* __restrict__ cfg, const SigRun* __restrict__ run,
                         const RoundCtl* __restrict__ ctl, Scans sc, c2<T>* __restrict__ tab,
                         const int64_t* __restrict__ ubuf, const int32_t* const* __restrict__ sig_w,
                         const double2* const* __restrict__ sig_a, const c2<T>* __restrict__ tw,
                         const int32_t* __restrict__ regw, const double2* __restrict__ rega,
                         const c2<T>* __restrict__ regtw, int32_t* __restrict__ alpha, int32_t* __restrict__ gam,
                         c2<T>* __restrict__ Cm) {
  const int64_t ntab = ctl->n_tab;
  const int64_t total = ntab + ctl->n_mode;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < ntab) {
      const int s = find_slot(sc.v[SC_TAB], n, e);
      const int64_t m = e - sc.v[SC_TAB][s];
      table_entry<T>(run[s].p, run[s].mod_m, m, tab + cfg[s].tab_off);
      if constexpr (sizeof(T) == 8) {
        // the sampler's roots W[m] in double-float (the chirp, read by the DFT, stays double)
        if (cfg[s].df_sample) df_pack_inplace(tab + cfg[s].tab_off + m);
      }
      continue;
    }
    const int64_t em = e - ntab;
    const int s = find_slot(sc.v[SC_MODE], n, em);
    const int j = (int)(em - sc.v[SC_MODE][s]);
    mode_entry<T>(cfg[s], run[s], s, j, ubuf, sig_w, sig_a, tw, regw, rega, regtw, alpha, gam, Cm);
    if constexpr (sizeof(T) == 8) {
      if (cfg[s].df_sample)
        for (int nn = 0; nn < cfg[s].n_sets; ++nn) df_pack_inplace(Cm + cfg[s].C_off + j + (int64_t)nn * cfg[s].Kmax);
    }
  }
}

// ------------------------------------------------------------------ sampling

// Persistent sampling kernel for the signals whose set groups hold NS sets; DF (double engine
// only) samples in double-float arithmetic, a policy every slot of an engine shares.
template <typename T, int NS, bool DF>
__global__ void __launch_bounds__(kSampleThreads, 2) k_sample(int n, const SigCfg* __restrict__ cfg,
                                                           const SigRun* __restrict__ run, RoundCtl* ctl, Scans sc,
                                                           const int32_t* __restrict__ alpha,
                                                           const int32_t* __restrict__ gam,
                                                           const c2<T>* __restrict__ Cm,
                                                           const c2<T>* __restrict__ tab, c2<T>* __restrict__ part) {
  __shared__ SampleSmem<T, NS> sm;
  const int64_t total = ctl->n_samp[NS - 1];
  const int64_t* scan = sc.v[SC_SAMP0 + NS - 1];
  for (;;) {
    if (threadIdx.x == 0) sm.item = (int64_t)atomicAdd(&ctl->ctr_samp[NS - 1], 1ull);
    __syncthreads();
    const int64_t item = sm.item;
    __syncthreads();
    if (item >= total) break;
    const int s = find_slot(scan, n, item);
    const int64_t local = item - scan[s];
    const SigCfg& c = cfg[s];
    const SigRun r = run[s];
    const int xt = (int)(local % r.n_xt);
    const int64_t rest = local / r.n_xt;
    const int g = (int)(rest % r.groups);
    const int split = (int)(rest / r.groups);
    sample_tile<T, NS, DF>(sm, c, r, xt, g, split, alpha + c.mode_off, gam + c.mode_off, Cm + c.C_off,
                           tab + r.tab_at, part);
  }
}

// sum of the split partials into y (step calls)
template <typename T>
__global__ void k_reduce(const SigCfg* __restrict__ cfg, const SigRun* __restrict__ run, int n_rows,
                         const c2<T>* __restrict__ part, c2<T>* __restrict__ y) {
  const SigRun& r = run[0];
  const int ns = cfg[0].n_sets;
  const int64_t total = (int64_t)n_rows * r.p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    c2<T> acc = part[r.part_off + e];
    for (int q = 1; q < r.splits; ++q) acc = cadd(acc, part[r.part_off + (int64_t)q * ns * r.p + e]);
    y[e] = acc;
  }
}

// ------------------------------------------------------------------ DFT, one block per row

// Spectrum of the Bluestein filter b[m] = conj(chirp[|m|]), |m| < p, by one block into out.
template <typename T>
__device__ __forceinline__ void filter_spectrum(int64_t p, int L, const c2<T>* chirp, const TwSrc<c2<T>>& tws,
                                                c2<T>* out, c2<T>* buf, c2<T>* tw_hi, c2<T>* tw_lo) {
  fft_tables(tw_hi, tw_lo, L, tws);
#pragma unroll 8
  for (int x = threadIdx.x; x < L; x += blockDim.x) buf[fpad(x)] = filter_value<T>(x, p, L, chirp);
  __syncthreads();
  fft_row<c2<T>, false>(buf, L, tw_hi, tw_lo);
#pragma unroll 8
  for (int x = threadIdx.x; x < L; x += blockDim.x) out[x] = buf[fpad(x)];
}

// spectrum of the Bluestein filter of each signal that owns its round's tables, one block each
template <typename T>
__global__ void __launch_bounds__(kFftThreads, 1) k_filter(int n, const SigCfg* __restrict__ cfg, const SigRun* __restrict__ run, RoundCtl* ctl,
                         Scans sc, const c2<T>* __restrict__ tab, TwSrc<c2<T>> tws, c2<T>* __restrict__ bhat,
                         int small) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ C2 tw_lo[kTwLo], tw_hi[kSingleMaxLf / kTwLo];
  C2* buf = reinterpret_cast<C2*>(smem_raw);
  // one block per item (a loop around the unrolled passes would make them spill)
  const int64_t item = blockIdx.x;
  if (item >= (small ? ctl->n_filt_s : ctl->n_filt)) return;
  const int s = find_slot(sc.v[small ? SC_FILT_S : SC_FILT], n, item);
  const SigCfg& c = cfg[s];
  const SigRun& r = run[s];
  filter_spectrum<T>(r.p, r.L, tab + r.tab_at + r.p, tws, bhat + c.bhat_off, buf, tw_hi, tw_lo);
}

// The tables and filter spectrum of round 1's prime, made once when the engine is created (the
// prime is fixed by the plan: the first prime >= max(c k, p_min), or the list's first).
template <typename T>
__global__ void k_tables_one(int64_t p, unsigned long long mod_m, c2<T>* __restrict__ t, int df) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < p; m += (int64_t)gridDim.x * blockDim.x) {
    table_entry<T>(p, mod_m, m, t);
    if constexpr (sizeof(T) == 8) {
      if (df) df_pack_inplace(t + m);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads, 1) k_filter_one(int64_t p, int L, const c2<T>* __restrict__ chirp,
                                                             TwSrc<c2<T>> tws, c2<T>* __restrict__ out) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ C2 tw_lo[kTwLo], tw_hi[kSingleMaxLf / kTwLo];
  filter_spectrum<T>(p, L, chirp, tws, out, reinterpret_cast<C2*>(smem_raw), tw_hi, tw_lo);
}

// E: complex values a thread holds per pass (32 in float: radix-32 passes, 128 registers, one
// 512-thread block or two 256-thread blocks per SM; 16: radix-16 passes, two 512-thread blocks)
template <typename T, int E = fft_per_thread<c2<T>>()>
__global__ void __launch_bounds__(kFftThreads, (E == 16 && sizeof(T) == 4) ? 2 : 1) k_dft(int n, const SigCfg* __restrict__ cfg, SigRun* run, RoundCtl* ctl, Scans sc,
                      const c2<T>* __restrict__ part, const c2<T>* __restrict__ tab,
                      const c2<T>* __restrict__ bhat, TwSrc<c2<T>> tws, c2<T>* __restrict__ Y, int small,
                      int smem_bytes) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ C2 tw_lo[kTwLo], tw_hi[kSingleMaxLf / kTwLo];
  C2* buf = reinterpret_cast<C2*>(smem_raw);
  // one block per group of rows of one signal (a loop around the unrolled passes would make
  // them spill), last groups first: the signals at the end of the sampling queue may carry
  // several mode splits to add.  The block's threads split into g warp-aligned teams of
  // `team` threads, one row each; the rows share p, so the chirp, the filter spectrum and the
  // twiddles serve them all.
  const int64_t n_items = small ? ctl->n_rows_s : ctl->n_rows;
  if ((int64_t)blockIdx.x >= n_items) return;
  const int64_t item = n_items - 1 - blockIdx.x;
  const int64_t* scan = sc.v[small ? SC_ROWS_S : SC_ROWS];
  const int s = find_slot(scan, n, item);
  const SigCfg& c = cfg[s];
  const SigRun r = run[s];
  const int L = r.L;
  const int64_t p = r.p;
  const int g = dft_group_rows<C2>(L, (int)blockDim.x, smem_bytes / (int)sizeof(C2), c.n_sets, E == 16 ? 16 : 0);
  const int row0 = (int)(item - scan[s]) * g;
  const int nrow = min(g, c.n_sets - row0);
  const int team = ((int)blockDim.x / g) & ~31;
  const int sr = (int)threadIdx.x / team, lt = (int)threadIdx.x % team;
  const bool act = sr < nrow;
  const int row = row0 + (act ? sr : 0);
  const int rowpad = (L + L / 32 + 1) & ~1;   // even: every row starts 16-byte aligned
  C2* rb = buf + (act ? sr : 0) * rowpad;
  const C2* chirp = tab + r.tab_at + p;   // the tables and filter of the first signal with this prime
  const C2* B = bhat + r.bhat_at;
  // With room for one more row of L values after the padded rows, the filter spectrum is copied
  // there asynchronously during the forward transform, and then the chirp during the inverse
  // one, so that neither product waits on global memory.
  const int pfo = g * rowpad;
  C2* pf = buf + pfo;
  const bool prefetch = (int64_t)(pfo + L) * (int64_t)sizeof(C2) <= (int64_t)smem_bytes;
  if (prefetch) {
    const int units = L * (int)sizeof(C2) / 16;   // the spectrum's offset is even: 16-byte aligned
    for (int i = threadIdx.x; i < units; i += blockDim.x)
      cp_async<16>(reinterpret_cast<unsigned char*>(pf) + 16 * i, reinterpret_cast<const unsigned char*>(B) + 16 * i);
    cp_async_commit();
  }
  fft_tables(tw_hi, tw_lo, L, tws);
  // loops unrolled so that each thread's global loads are in flight together
  if (act) {
#pragma unroll 8
    for (int x = lt; x < L; x += team) {
      C2 v = mk2((T)0, (T)0);
      if (x < p) {
        C2 y = sum_splits<T>(part, r, c.n_sets, row, x);
        if (r.noise_sigma > 0.0) y = cadd(y, black_box_noise<T>(r.noise_seed, r.round, row, x, r.noise_sigma));
        v = cmul(chirp[x], y);
      }
      rb[fpad(x)] = v;
    }
  }
  __syncthreads();
  fft_row<C2, false, E>(rb, L, tw_hi, tw_lo, lt, team, act);
  if (prefetch) {
    cp_async_wait_all();
    __syncthreads();
    if (act) {
#pragma unroll 8
      for (int k = lt; k < L; k += team) rb[fpad(k)] = cconj(cmul(rb[fpad(k)], pf[k]));
    }
    __syncthreads();   // the spectrum is consumed: the chirp takes its place
    for (int x = threadIdx.x; x < p; x += blockDim.x) cp_async<sizeof(C2)>(pf + x, chirp + x);
    cp_async_commit();
  } else {
    if (act) {
#pragma unroll 8
      for (int k = lt; k < L; k += team) rb[fpad(k)] = cconj(cmul(rb[fpad(k)], B[k]));
    }
    __syncthreads();
  }
  // the inverse transform as conj(FFT(conj(.))): the product was stored conjugated, the forward
  // code runs again, and the read-out below conjugates back, so the kernel holds the code of one
  // direction only (its instruction footprint, with every radix unrolled, is what limits it)
  fft_row<C2, false, E>(rb, L, tw_hi, tw_lo, lt, team, act);
  if (prefetch) {
    cp_async_wait_all();
    __syncthreads();
  }
  const C2* ch = prefetch ? pf : chirp;
  const T invL = (T)1 / (T)L;
  C2* out = Y + c.Y_off + (int64_t)row * p;
  T m2 = (T)0;   // largest |Y_0|^2 of this thread (set 0 only), in the transform's precision
  if (act) {
#pragma unroll 4
    for (int64_t h0 = 0; h0 < p; h0 += team) {
      const int64_t h = h0 + lt;
      if (h < p) {
        const C2 v = cmul(ch[h], cscale(cconj(rb[fpad((int)h)]), invL));
        out[h] = v;
        m2 = fmax(m2, v.x * v.x + v.y * v.y);
      }
    }
  }
  // whole warps only (teams are warp-aligned): the team of set 0 reports its largest bin
  if (act && row == 0) max_abs_to<T>(&run[s].maxy0_bits, sqrt((double)m2));
}

// ------------------------------------------------------------------ DFT, four-step passes for long lengths

template <typename T>
__global__ void k_bigA(int n, const SigCfg* __restrict__ cfg, const SigRun* __restrict__ run,
                       const RoundCtl* __restrict__ ctl, Scans sc, const c2<T>* __restrict__ part,
                       const c2<T>* __restrict__ tab, const c2<T>* __restrict__ twG, int64_t Lmax,
                       c2<T>* __restrict__ Z) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* buf = reinterpret_cast<C2*>(smem_raw);
  const int64_t total = ctl->n_bigA;
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = find_slot(sc.v[SC_BIGA], n, item);
    const int64_t local = item - sc.v[SC_BIGA][s];
    const SigCfg& c = cfg[s];
    const SigRun r = run[s];
    int M1, M2, CT, RT;
    big_geom(r.logL, &M1, &M2, &CT, &RT);
    const int logM1 = r.logL / 2;
    const int64_t L = 1LL << r.logL;
    const int ntile = M2 / CT;
    const int row = (int)(local / ntile);
    const int x2_0 = (int)(local % ntile) * CT;
    const int ls = M1 + 1;
    C2* tw = buf + CT * ls;
    const C2* chirp = tab + r.tab_at + r.p;
    for (int j = threadIdx.x; j < M1 / 2; j += blockDim.x) tw[j] = twG[(int64_t)j * (Lmax >> logM1)];
    for (int e = threadIdx.x; e < CT * M1; e += blockDim.x) {
      const int x1 = e / CT, cc = e - x1 * CT;
      const int64_t x = (int64_t)x1 * M2 + x2_0 + cc;
      C2 v;
      if (row < c.n_sets) {
        v = mk2((T)0, (T)0);
        if (x < r.p) {
          C2 y = sum_splits<T>(part, r, c.n_sets, row, x);
          if (r.noise_sigma > 0.0) y = cadd(y, black_box_noise<T>(r.noise_seed, r.round, row, x, r.noise_sigma));
          v = cmul(chirp[x], y);
        }
      } else {
        v = filter_value<T>(x, r.p, L, chirp);
      }
      buf[cc * ls + brev_bits(x1, logM1)] = v;
    }
    __syncthreads();
    fft_dit(buf, ls, logM1, CT, tw, false);
    C2* z = Z + c.z_off + (int64_t)row * L;
    const int64_t tstep = Lmax >> r.logL;
    for (int e = threadIdx.x; e < CT * M1; e += blockDim.x) {
      const int k1 = e / CT, cc = e - k1 * CT;
      const int64_t x2 = x2_0 + cc;
      const int64_t m = (x2 * k1) & (L - 1);
      z[(int64_t)k1 * M2 + x2] = cmul(buf[cc * ls + k1], twG[m * tstep]);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_bigB(int n, const SigCfg* __restrict__ cfg, const SigRun* __restrict__ run,
                       const RoundCtl* __restrict__ ctl, Scans sc, const c2<T>* __restrict__ twG, int64_t Lmax,
                       c2<T>* __restrict__ Z) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* buf = reinterpret_cast<C2*>(smem_raw);
  const int64_t total = ctl->n_bigB;
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = find_slot(sc.v[SC_BIGB], n, item);
    const int64_t local = item - sc.v[SC_BIGB][s];
    const SigCfg& c = cfg[s];
    const SigRun r = run[s];
    int M1, M2, CT, RT;
    big_geom(r.logL, &M1, &M2, &CT, &RT);
    const int logM2 = r.logL - r.logL / 2;
    const int64_t L = 1LL << r.logL;
    const int ntile = M1 / RT;
    const int row = (int)(local / ntile);
    const int k1_0 = (int)(local % ntile) * RT;
    const int ls = M2 + 1;
    C2* bufF = buf + RT * ls;
    C2* tw = buf + 2 * RT * ls;
    for (int j = threadIdx.x; j < M2 / 2; j += blockDim.x) tw[j] = twG[(int64_t)j * (Lmax >> logM2)];
    C2* zr = Z + c.z_off + (int64_t)row * L;
    const C2* zf = Z + c.z_off + (int64_t)c.n_sets * L;
    for (int e = threadIdx.x; e < RT * M2; e += blockDim.x) {
      const int rr = e / M2, x2 = e - rr * M2;
      const int64_t off = (int64_t)(k1_0 + rr) * M2 + x2;
      buf[rr * ls + brev_bits(x2, logM2)] = zr[off];
      bufF[rr * ls + brev_bits(x2, logM2)] = zf[off];
    }
    __syncthreads();
    fft_dit(buf, ls, logM2, 2 * RT, tw, false);
    for (int e = threadIdx.x; e < RT * M2; e += blockDim.x) {
      const int rr = e / M2, k2 = e - rr * M2;
      buf[rr * ls + k2] = cmul(buf[rr * ls + k2], bufF[rr * ls + k2]);
    }
    __syncthreads();
    fft_dif(buf, ls, logM2, RT, tw, true);
    const int64_t tstep = Lmax >> r.logL;
    for (int e = threadIdx.x; e < RT * M2; e += blockDim.x) {
      const int rr = e / M2, x2 = e - rr * M2;
      const int64_t k1 = k1_0 + rr;
      const int64_t m = ((int64_t)x2 * k1) & (L - 1);
      zr[k1 * M2 + x2] = cmul(buf[rr * ls + brev_bits(x2, logM2)], cconj(twG[m * tstep]));
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_bigC(int n, const SigCfg* __restrict__ cfg, SigRun* run, const RoundCtl* __restrict__ ctl, Scans sc,
                       const c2<T>* __restrict__ tab, const c2<T>* __restrict__ twG, int64_t Lmax,
                       const c2<T>* __restrict__ Z, c2<T>* __restrict__ Y) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* buf = reinterpret_cast<C2*>(smem_raw);
  const int64_t total = ctl->n_bigC;
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = find_slot(sc.v[SC_BIGC], n, item);
    const int64_t local = item - sc.v[SC_BIGC][s];
    const SigCfg& c = cfg[s];
    const SigRun r = run[s];
    int M1, M2, CT, RT;
    big_geom(r.logL, &M1, &M2, &CT, &RT);
    const int logM1 = r.logL / 2;
    const int64_t L = 1LL << r.logL;
    const int ntile = M2 / CT;
    const int row = (int)(local / ntile);
    const int x2_0 = (int)(local % ntile) * CT;
    const int ls = M1 + 1;
    C2* tw = buf + CT * ls;
    const C2* chirp = tab + r.tab_at + r.p;
    for (int j = threadIdx.x; j < M1 / 2; j += blockDim.x) tw[j] = twG[(int64_t)j * (Lmax >> logM1)];
    const C2* z = Z + c.z_off + (int64_t)row * L;
    for (int e = threadIdx.x; e < CT * M1; e += blockDim.x) {
      const int k1 = e / CT, cc = e - k1 * CT;
      buf[cc * ls + k1] = z[(int64_t)k1 * M2 + x2_0 + cc];
    }
    __syncthreads();
    fft_dif(buf, ls, logM1, CT, tw, true);
    const T invL = (T)1 / (T)L;
    C2* out = Y + c.Y_off + (int64_t)row * r.p;
    const int tot = CT * M1;
    T m2 = (T)0;
    for (int e0 = 0; e0 < tot; e0 += blockDim.x) {
      const int e = e0 + threadIdx.x;
      if (e < tot) {
        const int x1 = e / CT, cc = e - x1 * CT;
        const int64_t x = (int64_t)x1 * M2 + x2_0 + cc;
        if (x < r.p) {
          const C2 v = cmul(chirp[x], cscale(buf[cc * ls + brev_bits(x1, logM1)], invL));
          out[x] = v;
          m2 = fmax(m2, v.x * v.x + v.y * v.y);
        }
      }
    }
    if (row == 0) max_abs_to<T>(&run[s].maxy0_bits, sqrt((double)m2));
    __syncthreads();
  }
}

// ------------------------------------------------------------------ registry removed in the bin domain

// Residual BINS (peel_entry): every live registry mode of an active signal leaves its bin of
// each set, one thread per mode.
template <typename T>
__global__ void k_peel(int n, const SigCfg* __restrict__ cfg, const SigRun* __restrict__ run,
                       const int64_t* __restrict__ ubuf, const int32_t* __restrict__ regw,
                       const double2* __restrict__ rega, const c2<T>* __restrict__ regtw, c2<T>* __restrict__ Ybuf) {
  const int s = blockIdx.y;
  if (s >= n) return;
  const SigCfg& c = cfg[s];
  const SigRun& r = run[s];
  if (!r.active || r.fused || !c.peel_bins) return;
  const int nr = min(r.K_reg, c.reg_cap);
  const int64_t* u = ubuf + c.u_off;
  T* Y = reinterpret_cast<T*>(Ybuf + c.Y_off);
  for (int jr = blockIdx.x * blockDim.x + threadIdx.x; jr < nr; jr += gridDim.x * blockDim.x)
    peel_entry<T>(c, r, jr, u, regw, rega, regtw, [&](int64_t e, T gx, T gy) { peel_add(Y + 2 * e, gx, gy); });
}

// ------------------------------------------------------------------ classification and registry merge

// Bins of the round whose set-0 magnitude is above the empty-bin level, appended to the
// candidate list; also the first round's reference amplitude A_ref and the flag that some bin of
// some set is above that level (the stop rule reads it).  A block takes a contiguous range of bins and gathers its
// candidates in shared memory, with one atomic on the list's counter per kCandBuf of them; a
// warp whose 32 bins belong to one signal reads that signal's level once.
constexpr int kCandBuf = 2048;
template <typename T>
__global__ void __launch_bounds__(256) k_occupied(int n, const SigCfg* __restrict__ cfg, SigRun* run, RoundCtl* ctl,
                                                  Scans sc, const c2<T>* __restrict__ Ybuf, int2* __restrict__ cand,
                                                  double eta_override) {
  __shared__ int2 buf[kCandBuf];
  __shared__ int s_cnt;
  __shared__ unsigned long long s_base;
  const int64_t total = ctl->n_bins;
  const int lane = threadIdx.x & 31;
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;   // bins of this block
  const int64_t lo = blockIdx.x * per, hi = min(total, lo + per);
  __shared__ int s_from;   // slot of the first bin of the current tile of 256 bins
  if (threadIdx.x == 0) {
    s_cnt = 0;
    s_from = lo < hi ? find_slot(sc.v[SC_BINS], n, lo) : 0;
  }
  __syncthreads();
  auto flush = [&]() {   // all threads: copy the gathered candidates out, one atomic
    __syncthreads();
    const int m = min(s_cnt, kCandBuf);
    if (threadIdx.x == 0) s_base = m > 0 ? atomicAdd(&ctl->n_cand, (unsigned long long)m) : 0ull;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) cand[s_base + i] = buf[i];
    __syncthreads();
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
  };
  for (int64_t b0 = lo; b0 < hi; b0 += blockDim.x) {
    const int64_t e = b0 + threadIdx.x;
    const bool valid = e < hi;
    // the block's bins are contiguous: search from the slot of the tile's first bin
    const int s = valid ? find_slot_from(sc.v[SC_BINS], n, e, s_from) : -1;
    const int s0 = __shfl_sync(0xffffffffu, s, 0);
    const bool uni = __all_sync(0xffffffffu, !valid || s == s0);
    bool occ = false;     // set 0 above the level: a candidate for the ratio test
    bool resid = false;   // some set above the level: the residual is not empty
    int64_t h = 0;
    // the signal's level: by lane 0 for the warp when its bins share the signal, else per lane
    T lvl = (T)0;   // squared level in float, the level itself in double
    auto level = [&](int ss) -> T {
      const SigCfg& c = cfg[ss];
      SigRun* rp = run + ss;
      const int64_t p = rp->p;
      const bool first = rp->round == 1;
      const double maxy0 = __longlong_as_double((long long)rp->maxy0_bits);
      if (sizeof(T) == 4) {
        // float policy: the squared level in float (the double pipe of this GPU is narrow, and
        // the level is a heuristic far from any mode's size)
        const float a_ref = first ? (float)maxy0 / (float)p : (float)rp->a_ref;
        const float eta = eta_override >= 0.0 ? (float)eta_override
                                               : fmaxf((float)c.rho * (float)p * a_ref,
                                                       6.0f * (float)c.sigma * sqrtf((float)p));
        return (T)(eta * eta);
      }
      const double a_ref = first ? maxy0 / (double)p : rp->a_ref;
      return (T)(eta_override >= 0.0 ? eta_override : fmax(c.rho * (double)p * a_ref, 6.0 * c.sigma * sqrt((double)p)));
    };
    if (uni) {
      T l0 = (T)0;
      if (lane == 0 && s0 >= 0) l0 = level(s0);
      lvl = __shfl_sync(0xffffffffu, l0, 0);
    } else if (valid) {
      lvl = level(s);
    }
    if (valid) {
      const SigCfg& c = cfg[s];
      SigRun* rp = run + s;
      h = e - sc.v[SC_BINS][s];
      if (h == 0) {
        // once per signal: A_ref (first round) and the prune level of the round's merges
        const int64_t p = rp->p;
        const bool first = rp->round == 1;
        const double maxy0 = __longlong_as_double((long long)rp->maxy0_bits);
        const double a_ref = first ? maxy0 / (double)p : rp->a_ref;
        if (first) rp->a_ref = a_ref;
        rp->eta_prune = fmax(c.rho * a_ref, 6.0 * c.sigma / sqrt((double)p));
      }
      auto above = [&](const c2<T> y) -> bool {
        if (sizeof(T) == 4) return y.x * y.x + y.y * y.y > lvl;
        return sqrt((double)y.x * (double)y.x + (double)y.y * (double)y.y) > (double)lvl;
      };
      occ = above(Ybuf[c.Y_off + h]);
      // The residual is empty only when every set is: two modes w, w' of opposite coefficients
      // whose difference the line does not see ((w - w') . u = 0 mod p; a read-out that
      // slipped in a coordinate outside the round's block leaves such a pair in the registry)
      // cancel in set 0 but not in the set of that coordinate.  Such a bin is no candidate (no
      // single mode passes the ratio test there), but it keeps the signal's rounds going.
      // (skipped once the signal is known to be occupied this round)
      resid = occ;
      if (!resid && !rp->any_occupied)
        for (int n = 1; n < c.n_sets && !resid; ++n) resid = above(Ybuf[c.Y_off + (int64_t)n * rp->p + h]);
    }
    // the occupied flag: once per warp for a one-signal warp
    const unsigned mask = __ballot_sync(0xffffffffu, occ);
    const unsigned rmask = __ballot_sync(0xffffffffu, resid);
    if (uni) {
      if (lane == 0 && rmask != 0u && !run[s0].any_occupied) run[s0].any_occupied = 1;
    } else if (resid && !run[s].any_occupied) {
      run[s].any_occupied = 1;
    }
    // gather: warp offsets by one shared atomic per warp
    int wbase = 0;
    if (lane == 0 && mask != 0u) wbase = atomicAdd(&s_cnt, __popc(mask));
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    if (occ) {
      const int slot = wbase + __popc(mask & ((1u << lane) - 1u));
      if (slot < kCandBuf) buf[slot] = make_int2(s, (int)h);
    }
    __syncthreads();
    // the next tile starts at or after the slot of this tile's last bin
    if (threadIdx.x == blockDim.x - 1) s_from = valid ? s : s_from;
    if (s_cnt > kCandBuf - (int)blockDim.x) {
      // (kCandBuf >= 2 blockDim: the last tile always fitted)
      flush();
    }
    __syncthreads();
  }
  flush();
}

// three blocks per SM (80 registers): one candidate per thread is a chain of global loads and
// atomics, so more warps hide more of it
template <typename T>
__global__ void __launch_bounds__(256, 3) k_classify(int n, const SigCfg* __restrict__ cfg, SigRun* run,
                                                     const RoundCtl* __restrict__ ctl,
                           const int2* __restrict__ cand, const c2<T>* __restrict__ Ybuf,
                           const int64_t* __restrict__ ubuf, const int32_t* __restrict__ shblk, int32_t* regw,
                           double2* rega, c2<T>* regtw, int32_t* hash, ClassifyOut co) {
  const int64_t total = (int64_t)ctl->n_cand;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 sh = cand[e];
    const int s = sh.x;
    classify_candidate<T>(cfg[s], run + s, s, sh.y, Ybuf + cfg[s].Y_off, ubuf, shblk, regw, rega, regtw, hash, co);
  }
}

// ------------------------------------------------------------------ outputs

__global__ void k_output(int n, const SigCfg* __restrict__ cfg, SigRun* run, const int32_t* __restrict__ regw,
                         const double2* __restrict__ rega, const int64_t* __restrict__ bindv, int32_t* out_w,
                         double2* out_a, int64_t* n_found, int* status, HistRec* hist) {
  __shared__ int warp_sums[32];
  __shared__ int64_t base_s;
  const int s = blockIdx.x;
  if (s >= n) return;
  const SigCfg& c = cfg[s];
  SigRun* rp = run + s;
  const int nr = min(rp->K_reg, c.reg_cap);
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int32_t* rw = regw + c.regw_off;
  const double2* ra = rega + c.rega_off;
  const int64_t cap = bindv[3 * n + s];
  int32_t* ow = out_w + bindv[5 * n + s];
  double2* oa = out_a + bindv[4 * n + s];
  for (int c0 = 0; c0 < nr; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    const bool live = i < nr && (ra[i].x != 0.0 || ra[i].y != 0.0);
    const unsigned bal = __ballot_sync(0xffffffffu, live);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[wid] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int q = 0; q < nw; ++q) {
      if (q < wid) off += warp_sums[q];
      tot += warp_sums[q];
    }
    const int64_t pos = base_s + off + before;
    if (live && pos < cap) {
      for (int l = 0; l < c.d; ++l) ow[pos * c.d + l] = rw[(int64_t)i * c.d + l];
      oa[pos] = ra[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) base_s += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    n_found[s] = base_s;
    int st = rp->active ? (int)SFFT_ERR_NOT_CONVERGED : rp->status;
    if (rp->err) st = (rp->err & kErrTimeout) ? SFFT_ERR_TIMEOUT : SFFT_ERR_CAPACITY;
    if (st == SFFT_OK && base_s > cap) st = SFFT_ERR_CAPACITY;
    if (st == SFFT_OK && base_s > c.k) st = SFFT_ERR_INCONSISTENT;
    status[s] = st;
    if (s == 0 && hist != nullptr && rp->round >= 1 && rp->round <= SFFT_STATS_MAX_ROUNDS) {
      hist[rp->round - 1].accepted = rp->n_acc;
      hist[rp->round - 1].live = rp->n_live;
    }
  }
}

// e^{2 pi i j / 1024}, j = 0..1023, in double: the reference points of the float engine's
// double read-out and coefficient roots (classification)
__global__ void k_root1k(double2* t) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 1024; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi((double)j / 512.0, &s, &c);
    t[j] = make_double2(c, s);
  }
}

__global__ void k_twiddles(int64_t Lmax, void* twG, int fp64) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < Lmax; m += (int64_t)gridDim.x * blockDim.x) {
    const int64_t mm = (2 * m > Lmax) ? m - Lmax : m;
    double s, c;
    sincospi(-2.0 * (double)mm / (double)Lmax, &s, &c);
    if (fp64) reinterpret_cast<double2*>(twG)[m] = make_double2(c, s);
    else reinterpret_cast<float2*>(twG)[m] = make_float2((float)c, (float)s);
  }
}

// ------------------------------------------------------------------ host side

// the smallest prime >= v (trial division; v below 2^40)
int64_t first_prime_at_least(int64_t v) {
  for (int64_t q = std::max<int64_t>(v, 2);; ++q) {
    bool prime = true;
    for (int64_t f = 2; f * f <= q; ++f)
      if (q % f == 0) {
        prime = false;
        break;
      }
    if (prime) return q;
  }
}

std::vector<int32_t> sieve_primes(int64_t lim) {
  std::vector<char> comp((size_t)lim + 1, 0);
  std::vector<int32_t> out;
  for (int64_t q = 2; q <= lim; ++q) {
    if (comp[q]) continue;
    out.push_back((int32_t)q);
    for (int64_t m = q * q; m <= lim; m += q) comp[m] = 1;
  }
  return out;
}

int64_t next_pow2(int64_t v) {
  int64_t r = 1;
  while (r < v) r <<= 1;
  return r;
}

int log2i(int64_t v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}

#define ECHK(x)                          \
  do {                                   \
    cudaError_t _e = (x);                \
    if (_e != cudaSuccess) return _e;    \
  } while (0)

template <typename T>
class Engine final : public EngineBase {
 public:
  using C2 = c2<T>;

  ~Engine() override {
    if (graph_exec_) cudaGraphExecDestroy(graph_exec_);
    if (graph_) cudaGraphDestroy(graph_);
    for (cudaEvent_t e : events_) cudaEventDestroy(e);
    if (fork_ev_) cudaEventDestroy(fork_ev_);
    if (join_ev_) cudaEventDestroy(join_ev_);
    if (side_) cudaStreamDestroy(side_);
    for (int q = 0; q < kMaxSetGroup - 1; ++q) {
      if (samp_join_[q]) cudaEventDestroy(samp_join_[q]);
      if (samp_st_[q]) cudaStreamDestroy(samp_st_[q]);
    }
    if (samp_fork_) cudaEventDestroy(samp_fork_);
    for (void* q : allocs_) cudaFree(q);
    if (host_stage_) cudaFreeHost(host_stage_);
  }

  cudaError_t init(const std::vector<SlotDesc>& slots, cudaStream_t st, bool profile, bool use_graph) {
    n_ = (int)slots.size();
    st_ = st;
    profile_ = profile;
    use_graph_ = use_graph;
    ECHK(cudaGetDevice(&dev_));
    ECHK(cudaDeviceGetAttribute(&n_sm_, cudaDevAttrMultiProcessorCount, dev_));
    std::vector<SigCfg> cfg(n_);
    std::vector<int64_t> dirs, plist;
    std::vector<int32_t> shblk;   // (start, size) of every shift block, block form
    int64_t tw = 0, regw = 0, rega = 0, hashn = 0, tab = 0, bhat = 0, Y = 0, z = 0, u = 0, part_min = 0;
    int64_t bins = 0;   // candidate-list entries: every bin of every slot at its largest prime
    int64_t modes = 0, cm = 0;
    int64_t pmax_all = 2;
    const int single_logL = log2i(single_max_L<T>());
    for (int s = 0; s < n_; ++s) {
      const SlotDesc& d = slots[s];
      SigCfg& c = cfg[s];
      std::memset(&c, 0, sizeof(c));
      c.d = d.d;
      c.shift_block = d.shift_block;
      c.shift_tilt = d.shift_tilt;
      c.tilt_base = d.tilt_base;
      c.tilt_height = d.tilt_height;
      c.tilt_hypo = d.tilt_hypo;
      c.n_sets = d.shift_block ? 1 + (int)d.shift_blocks.size() : d.d + 1;
      c.fuse_L = (sizeof(T) == 4 && d.fuse) ? fused_max_length(c.n_sets) : 0;
      if (d.fuse_max_len > 0) c.fuse_L = std::min(c.fuse_L, d.fuse_max_len);
      if (c.fuse_L < 32) c.fuse_L = 0;   // below the shortest Bluestein length: nothing is fused
      if (c.fuse_L > 0) {
        // the shortest Bluestein length any round of the slot can have is that of the smallest
        // prime its rule (k* = 1) or list gives; a slot whose rounds are all longer never fuses,
        // and an engine without fusable slots launches no fused kernel
        int64_t p_reach;
        if (!d.primes.empty()) p_reach = *std::min_element(d.primes.begin(), d.primes.end());
        else p_reach = first_prime_at_least(std::max<int64_t>(std::max<int64_t>((d.c8 + 7) / 8, d.p_min), 2));
        if (p_reach < 2 || bluestein_length(2 * p_reach - 1) > c.fuse_L) c.fuse_L = 0;
      }
      c.blk_off = (int64_t)shblk.size();
      if (d.shift_block) {
        int start = 0;
        for (int size : d.shift_blocks) {
          shblk.push_back(start);
          shblk.push_back(size);
          start += size;
        }
      }
      c.k = (int)d.k;
      c.c8 = d.c8;
      c.empty_rounds = std::max(1, d.empty_rounds);
      c.dense_dft = (sizeof(T) == 4 && d.dense_dft) ? 1 : 0;
      c.stall_div = d.stall_div;
      c.df_sample = (sizeof(T) == 8 && d.df_sample) ? 1 : 0;
      if (c.df_sample) any_df_ = true;
      if (c.dense_dft) any_dense_ = true;
      c.max_rounds = d.max_rounds;
      c.n_dirs = d.n_dirs;
      c.n_primes = (int)d.primes.size();
      c.box_lo = d.box_lo;
      c.ratio64 = d.ratio64;
      c.coef_mean = d.coef_mean;
      c.peel_bins = d.peel_bins;
      c.N = d.N;
      c.p_max = d.p_max;
      c.p_min = d.p_min;
      c.tau = d.tau;
      c.rho = d.rho;
      c.delta = d.delta;
      c.sigma = d.sigma;
      c.reg_cap = (int)std::min<int64_t>(2 * d.k + 256, 1LL << 30);
      c.hash_mask = (int)next_pow2(2 * (int64_t)c.reg_cap) - 1;
      const int64_t Lmax = std::max<int64_t>(next_pow2(2 * d.p_max - 1), 32);
      c.logL_max = log2i(Lmax);
      c.dirs_off = (int64_t)dirs.size();
      dirs.insert(dirs.end(), d.dirs.begin(), d.dirs.end());
      c.primes_off = (int64_t)plist.size();
      plist.insert(plist.end(), d.primes.begin(), d.primes.end());
      c.tw_off = tw;
      tw += std::max<int64_t>(d.k, 1) * d.d;
      c.regw_off = regw;
      c.regtw_off = regw;
      regw += (int64_t)c.reg_cap * d.d;
      c.rega_off = rega;
      rega += c.reg_cap;
      c.hash_off = hashn;
      hashn += (int64_t)c.hash_mask + 1;
      c.tab_off = tab;
      tab += 2 * d.p_max;
      c.bhat_off = bhat;
      bhat += std::min<int64_t>(Lmax, single_max_L<T>());
      c.Y_off = Y;
      Y += (int64_t)c.n_sets * d.p_max;
      bins += d.p_max;
      if (c.logL_max > single_logL) {
        c.z_off = z;
        z += (int64_t)(c.n_sets + 1) * Lmax;
        any_big_ = true;
        logL_big_max_ = std::max(logL_big_max_, c.logL_max);
      } else {
        c.z_off = -1;
      }
      c.u_off = u;
      u += d.d;
      c.Kmax = (int)(d.k + (c.peel_bins ? 0 : c.reg_cap));   // modes the round's tables hold
      if (c.peel_bins) {
        any_peel_ = true;
        peel_gx_ = std::max(peel_gx_, (int)std::min<int64_t>((c.reg_cap + 255) / 256, 32));
      }
      c.mode_off = modes;
      modes += c.Kmax;
      c.C_off = cm;
      cm += (int64_t)c.n_sets * c.Kmax;
      {
        const int groups = (c.n_sets + kMaxSetGroup - 1) / kMaxSetGroup;
        const int gsize = (c.n_sets + groups - 1) / groups;
        ns_mask_ |= 1u << (gsize - 1);
      }
      part_min += (int64_t)c.n_sets * d.p_max;
      rows_max_ += c.n_sets;
      pmax_all = std::max(pmax_all, d.p_max);
      if (c.fuse_L > 0) {
        any_fuse_ = true;
        fuse_ns_mask_ |= 1u << (c.n_sets - 1);
        fuse_sets_max_ = std::max(fuse_sets_max_, c.n_sets);
        fuse_L_max_ = std::max(fuse_L_max_, c.fuse_L);
      }
      small_logL_max_ = std::max(small_logL_max_, std::min(c.logL_max, single_logL));
      k_max_ = std::max<int64_t>(k_max_, d.k);
      kd_max_ = std::max<int64_t>(kd_max_, d.k * d.d);
      reg_cap_max_ = std::max<int64_t>(reg_cap_max_, c.reg_cap);
    }
    cfg_host_ = cfg;
    Lmax_ = std::max<int64_t>(next_pow2(2 * pmax_all - 1), 32);
    p_max_ = pmax_all;
    // a signal takes at most 64 mode splits (the planner's S), so 64 part_min holds any split choice;
    // small engines (one short signal) stay small, large batches stop at 128 MiB
    part_cap_ = std::max<int64_t>(part_min, std::min<int64_t>((int64_t)(128ll << 20) / (int64_t)sizeof(C2),
                                                              64 * part_min));
    hash_total_ = hashn;
    // prime table up to the largest p any slot can reach
    std::vector<int32_t> ptab = sieve_primes(pmax_all + 2);
    n_ptab_ = (int)ptab.size();
    // pfirst[v]: index in ptab of the smallest prime >= v, for v <= pmax_all + 1
    std::vector<int32_t> pfirst((size_t)pmax_all + 2);
    {
      size_t q = 0;
      for (int64_t v = 0; v <= pmax_all + 1; ++v) {
        while (q < ptab.size() && ptab[q] < v) ++q;
        pfirst[(size_t)v] = (int32_t)q;
      }
    }
    pfirst_n_ = (int64_t)pfirst.size();
    // Round 1's prime is fixed by the plan (k* = k): the first prime >= max(c k, p_min), or the
    // list's first.  Where its transform is one block, its tables and filter spectrum are made
    // here once, shared by the slots with that prime, and the rounds reuse them every execute.
    std::vector<int64_t> pre_p, pre_tab, pre_bhat;
    for (int s = 0; s < n_; ++s) {
      const SlotDesc& d = slots[s];
      SigCfg& c = cfg[s];
      c.tab0_off = c.bhat0_off = -1;
      c.p1 = 0;
      int64_t p1 = -1;
      if (!d.primes.empty()) {
        p1 = d.primes[0];
      } else {
        const int64_t lo = std::max<int64_t>(std::max<int64_t>(prime_floor_ck(d.c8, std::max<int64_t>(d.k, 1)), d.p_min), 2);
        if (lo < (int64_t)pfirst.size() && pfirst[(size_t)lo] < (int32_t)ptab.size()) p1 = ptab[pfirst[(size_t)lo]];
      }
      if (p1 < 2 || p1 > d.p_max || bluestein_length(2 * p1 - 1) > single_max_L<T>()) continue;
      size_t q = 0;
      while (q < pre_p.size() && pre_p[q] != p1) ++q;
      if (q == pre_p.size()) {
        pre_p.push_back(p1);
        pre_tab.push_back(tab);
        pre_bhat.push_back(bhat);
        tab += 2 * p1;
        bhat += bluestein_length(2 * p1 - 1);
      }
      c.p1 = p1;
      c.tab0_off = pre_tab[q];
      c.bhat0_off = pre_bhat[q];
    }
    cfg_host_ = cfg;

    ECHK(alloc(&cfg_, cfg.size() * sizeof(SigCfg)));
    ECHK(alloc(&run_, n_ * sizeof(SigRun)));
    ECHK(alloc(&ctl_, sizeof(RoundCtl)));
    for (int q = 0; q < kNumScans; ++q) ECHK(alloc(&scans_.v[q], (size_t)(n_ + 1) * sizeof(int64_t)));
    ECHK(alloc(&ptab_, ptab.size() * sizeof(int32_t)));
    ECHK(alloc(&pfirst_, pfirst.size() * sizeof(int32_t)));
    ECHK(alloc(&powner_, (size_t)(pmax_all + 1) * sizeof(unsigned long long)));
    ECHK(cudaMemsetAsync(powner_, 0xFF, (size_t)(pmax_all + 1) * sizeof(unsigned long long), st_));
    ECHK(alloc(&pacc_, sizeof(PlanAcc)));
    ECHK(cudaMemsetAsync(pacc_, 0, sizeof(PlanAcc), st_));
    ECHK(alloc(&pblk_, (size_t)((n_ + kPlanBlk - 1) / kPlanBlk) * sizeof(PlanBlk)));
    ECHK(alloc(&pdec_, sizeof(PlanDec)));
    ECHK(cudaMemsetAsync(pdec_, 0, sizeof(PlanDec), st_));
    ECHK(alloc(&dirs_, std::max<size_t>(dirs.size(), 1) * sizeof(int64_t)));
    ECHK(alloc(&shblk_, std::max<size_t>(shblk.size(), 1) * sizeof(int32_t)));
    ECHK(alloc(&plist_, std::max<size_t>(plist.size(), 1) * sizeof(int64_t)));
    ECHK(alloc(&tw_, (size_t)tw * sizeof(C2)));
    ECHK(alloc(&regw_, (size_t)regw * sizeof(int32_t)));
    ECHK(alloc(&regtw_, (size_t)regw * sizeof(C2)));
    ECHK(alloc(&rega_, (size_t)rega * sizeof(double2)));
    ECHK(alloc(&hash_, (size_t)hashn * sizeof(int32_t)));
    ECHK(alloc(&tab_, (size_t)tab * sizeof(C2)));
    ECHK(alloc(&bhat_, (size_t)bhat * sizeof(C2)));
    ECHK(alloc(&Y_, (size_t)Y * sizeof(C2)));
    ECHK(alloc(&cand_, (size_t)bins * sizeof(int2)));
    if (z > 0) ECHK(alloc(&Z_, (size_t)z * sizeof(C2)));
    ECHK(alloc(&u_, (size_t)u * sizeof(int64_t)));
    ECHK(alloc(&alpha_, (size_t)modes * sizeof(int32_t)));
    ECHK(alloc(&gam_, (size_t)modes * sizeof(int32_t)));
    ECHK(alloc(&Cm_, (size_t)cm * sizeof(C2)));
    ECHK(alloc(&part_, (size_t)part_cap_ * sizeof(C2)));
    ECHK(alloc(&twG_, (size_t)Lmax_ * sizeof(C2)));
    ECHK(alloc(&twG3_, (size_t)len3_ * sizeof(C2)));
    ECHK(alloc(&twG5_, (size_t)len5_ * sizeof(C2)));
    ECHK(alloc(&hist_, SFFT_STATS_MAX_ROUNDS * sizeof(HistRec)));
    ECHK(alloc(&bind_, (size_t)n_ * kBindArrays * sizeof(int64_t)));
    ECHK(alloc(&outn_, (size_t)n_ * sizeof(int64_t)));
    ECHK(alloc(&outst_, (size_t)n_ * sizeof(int)));
    ECHK(alloc(&stepc_, 2 * sizeof(int)));
    stage_ctl_ = align16((size_t)n_ * kBindArrays * sizeof(int64_t) + (size_t)64 * sizeof(int64_t));
    stage_n_ = align16(stage_ctl_ + sizeof(RoundCtl));
    stage_st_ = align16(stage_n_ + (size_t)n_ * sizeof(int64_t));
    stage_hist_ = align16(stage_st_ + (size_t)n_ * sizeof(int));
    host_stage_bytes_ = stage_hist_ + SFFT_STATS_MAX_ROUNDS * sizeof(HistRec);
    ECHK(cudaMallocHost(&host_stage_, host_stage_bytes_));
    ECHK(alloc(&root1k_, 1024 * sizeof(double2)));
    k_root1k<<<4, 256, 0, st_>>>((double2*)root1k_);
    ECHK(cudaGetLastError());
    for (SigCfg& c : cfg) c.root1k = (const double2*)root1k_;
    cfg_host_ = cfg;
    ECHK(cudaMemcpyAsync(cfg_, cfg.data(), cfg.size() * sizeof(SigCfg), cudaMemcpyHostToDevice, st_));
    ECHK(cudaMemcpyAsync(ptab_, ptab.data(), ptab.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
    ECHK(cudaMemcpyAsync(pfirst_, pfirst.data(), pfirst.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
    ECHK(cudaStreamSynchronize(st_));   // host vectors go out of scope
    if (!dirs.empty())
      ECHK(cudaMemcpyAsync(dirs_, dirs.data(), dirs.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st_));
    if (!plist.empty())
      ECHK(cudaMemcpyAsync(plist_, plist.data(), plist.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st_));
    if (!shblk.empty())
      ECHK(cudaMemcpyAsync(shblk_, shblk.data(), shblk.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
    k_twiddles<<<(int)std::min<int64_t>((Lmax_ + 255) / 256, 4096), 256, 0, st_>>>(Lmax_, twG_, sizeof(T) == 8);
    ECHK(cudaGetLastError());
    k_twiddles<<<(int)std::min<int64_t>((len3_ + 255) / 256, 4096), 256, 0, st_>>>(len3_, twG3_, sizeof(T) == 8);
    ECHK(cudaGetLastError());
    k_twiddles<<<(int)std::min<int64_t>((len5_ + 255) / 256, 4096), 256, 0, st_>>>(len5_, twG5_, sizeof(T) == 8);
    ECHK(cudaGetLastError());
    // launch shapes
    small_threads_ = std::max(32, (1 << small_logL_max_) / fft_per_thread<C2>());
    smem_small_ = (size_t)((1 << small_logL_max_) + (1 << small_logL_max_) / 32) * sizeof(C2);
    ECHK(cudaFuncSetAttribute(k_filter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_small_));
    ECHK(cudaFuncSetAttribute(k_filter_one<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_small_));
    for (size_t q = 0; q < pre_p.size(); ++q) {
      const int64_t p1 = pre_p[q];
      const int L1 = bluestein_length(2 * p1 - 1);
      C2* t0 = (C2*)tab_ + pre_tab[q];
      k_tables_one<T><<<(int)std::min<int64_t>((p1 + 255) / 256, 1024), 256, 0, st_>>>(p1, ~0ull / (uint64_t)p1, t0,
                                                                                        any_df_ ? 1 : 0);
      ECHK(cudaGetLastError());
      k_filter_one<T><<<1, std::max(32, fft_threads<C2>(L1)), (size_t)(L1 + L1 / 32) * sizeof(C2), st_>>>(
          p1, L1, t0 + p1, tw_src(), (C2*)bhat_ + pre_bhat[q]);
      ECHK(cudaGetLastError());
    }
    // The long-row DFT blocks take several rows of a signal at a time when they are short enough
    // (dft_group_rows), plus the prefetch row where it fits.  Their shared memory leaves room for
    // two blocks per SM (which the registers allow up to 256 threads) unless one row of the
    // batch's longest length needs more; blocks of 512 threads (lengths above 8192) are one per
    // SM by registers and take all of it.  The short-row blocks hold one row of 2^kSmallFftLog
    // and its prefetch row (six blocks per SM by shared memory, eight by registers), or two
    // shorter rows.
    {
      int optin = 0, per_sm = 0;
      ECHK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev_));
      ECHK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev_));
      const size_t kStatic = (size_t)(kTwLo + kSingleMaxLf / kTwLo) * sizeof(C2);   // k_dft's static tables
      const size_t room = (size_t)optin > kStatic + 1024 ? (size_t)optin - kStatic - 1024 : 0;
      const size_t half = (size_t)per_sm / 2 > kStatic + 2048 ? (size_t)per_sm / 2 - kStatic - 2048 : 0;
      // float batches with rows up to 8192: radix-16 passes in 512-thread blocks, two per SM
      dft_e_l_ = (sizeof(T) == 4 && small_logL_max_ <= 13 && kDftE16) ? 16 : 0;
      dft_thr_l_ = dft_e_l_ == 16 ? std::max(32, (1 << small_logL_max_) / 16) : small_threads_;
      const size_t cap = (small_threads_ <= 256 || dft_e_l_ == 16) ? std::min(room, half) : room;
      smem_dft_ = std::max(smem_small_, cap & ~(size_t)15);
      const int ls = std::min(small_logL_max_, kSmallFftLog);
      dft_e_s_ = (sizeof(T) == 4 && kDftE16) ? 16 : 0;   // short rows in radix-16 passes as well
      dft_thr_s_ = std::max(32, (1 << ls) / (dft_e_s_ == 16 ? 16 : fft_per_thread<C2>()));
      dft_smem_s_ = (size_t)((((1 << ls) + (1 << ls) / 32 + 1) & ~1) + (1 << ls)) * sizeof(C2);
    }
    ECHK(cudaFuncSetAttribute(k_dft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dft_));
    if constexpr (sizeof(T) == 4)
      ECHK(cudaFuncSetAttribute(k_dft<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dft_));
    if (any_big_) {
      size_t sa = 0, sb = 0;
      for (int lg = single_logL + 1; lg <= logL_big_max_; ++lg) {
        const int l1 = lg / 2, l2 = lg - l1, M1 = 1 << l1, M2 = 1 << l2;
        const int CT = std::min(M2, std::max(1, kBigColElems / M1));
        const int RT = std::min(M1, std::max(1, kBigRowElems / M2));
        sa = std::max(sa, (size_t)(CT * (M1 + 1) + M1 / 2) * sizeof(C2));
        sb = std::max(sb, (size_t)(2 * RT * (M2 + 1) + M2 / 2) * sizeof(C2));
      }
      smem_bigA_ = sa;
      smem_bigB_ = sb;
      ECHK(cudaFuncSetAttribute(k_bigA<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
      ECHK(cudaFuncSetAttribute(k_bigB<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
      ECHK(cudaFuncSetAttribute(k_bigC<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
    }
    if (any_fuse_) {
      smem_fused_ = fused_smem_bytes(fuse_sets_max_, fuse_L_max_);
      ECHK(fused_setup(smem_fused_));
    }
    if (any_dense_) ECHK(cudaFuncSetAttribute(k_dft_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem));
    if (profile_) {
      events_.resize((size_t)(SFFT_STATS_MAX_ROUNDS + 4) * 8);
      for (auto& e : events_) ECHK(cudaEventCreate(&e));
    }
    ECHK(cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking));
    ECHK(cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming));
    ECHK(cudaEventCreateWithFlags(&join_ev_, cudaEventDisableTiming));
    ECHK(cudaEventCreateWithFlags(&samp_fork_, cudaEventDisableTiming));
    for (int q = 0; q < kMaxSetGroup - 1; ++q) {
      ECHK(cudaStreamCreateWithFlags(&samp_st_[q], cudaStreamNonBlocking));
      ECHK(cudaEventCreateWithFlags(&samp_join_[q], cudaEventDisableTiming));
    }
    ECHK(cudaStreamSynchronize(st_));
    return cudaSuccess;
  }

  size_t device_bytes() const override { return bytes_; }
  int64_t max_prime() const override { return p_max_; }
  int64_t mode_capacity() const override { return k_max_ + reg_cap_max_; }

  cudaError_t launch_tables() {
    k_tables<T><<<4 * n_sm_, 256, 0, st_>>>(n_, cfg_, run_, ctl_, scans_, (C2*)tab_, u_, sig_w_, sig_a_, (C2*)tw_,
                                            regw_, rega_, (C2*)regtw_, alpha_, gam_, (C2*)Cm_);
    return cudaGetLastError();
  }

  // Bluestein rows of one block each, in two classes: short rows (L <= 2^kSmallFftLog) in
  // small-memory blocks, so many fit on an SM, and the longer rows
  // The Bluestein filter spectra of the round's owners (short and long class) on stream s.
  cudaError_t launch_filters(cudaStream_t s) {
    const int ls = std::min(small_logL_max_, kSmallFftLog);
    const int thr_s = std::max(32, (1 << ls) / fft_per_thread<C2>());
    const size_t smem_s = (size_t)((1 << ls) + (1 << ls) / 32) * sizeof(C2);
    const TwSrc<C2> tws = tw_src();
    k_filter<T><<<n_, thr_s, smem_s, s>>>(n_, cfg_, run_, ctl_, scans_, (C2*)tab_, tws, (C2*)bhat_, 1);
    ECHK(cudaGetLastError());
    if (small_logL_max_ > kSmallFftLog) {
      k_filter<T><<<n_, small_threads_, smem_small_, s>>>(n_, cfg_, run_, ctl_, scans_, (C2*)tab_, tws, (C2*)bhat_, 0);
      ECHK(cudaGetLastError());
    }
    return cudaSuccess;
  }

  // with_filters: the filter spectra first, on the same stream (else they were made beside the
  // sampling, see enqueue_batched)
  // The short- and long-row launches take different rows: with both present, the short one runs
  // on a stream of its own beside the long one.
  cudaError_t launch_dft_rows(bool with_filters = true) {
    const TwSrc<C2> tws = tw_src();
    if (with_filters) ECHK(launch_filters(st_));
    const bool both = small_logL_max_ > kSmallFftLog;
    cudaStream_t s_short = st_;
    if (both) {
      ECHK(cudaEventRecord(samp_fork_, st_));
      s_short = samp_st_[0];
      ECHK(cudaStreamWaitEvent(s_short, samp_fork_, 0));
    }
    if (sizeof(T) == 4 && dft_e_s_ == 16)
      k_dft<T, 16><<<(unsigned)rows_max_, dft_thr_s_, dft_smem_s_, s_short>>>(n_, cfg_, run_, ctl_, scans_, (C2*)part_,
                                                                              (C2*)tab_, (C2*)bhat_, tws, (C2*)Y_, 1,
                                                                              (int)dft_smem_s_);
    else
      k_dft<T><<<(unsigned)rows_max_, dft_thr_s_, dft_smem_s_, s_short>>>(n_, cfg_, run_, ctl_, scans_, (C2*)part_,
                                                                         (C2*)tab_, (C2*)bhat_, tws, (C2*)Y_, 1,
                                                                         (int)dft_smem_s_);
    ECHK(cudaGetLastError());
    if (both) {
      ECHK(cudaEventRecord(samp_join_[0], s_short));
      if (sizeof(T) == 4 && dft_e_l_ == 16)
        k_dft<T, 16><<<(unsigned)rows_max_, dft_thr_l_, smem_dft_, st_>>>(n_, cfg_, run_, ctl_, scans_, (C2*)part_,
                                                                          (C2*)tab_, (C2*)bhat_, tws, (C2*)Y_, 0,
                                                                          (int)smem_dft_);
      else
        k_dft<T><<<(unsigned)rows_max_, small_threads_, smem_dft_, st_>>>(n_, cfg_, run_, ctl_, scans_, (C2*)part_,
                                                                           (C2*)tab_, (C2*)bhat_, tws, (C2*)Y_, 0,
                                                                           (int)smem_dft_);
      ECHK(cudaGetLastError());
      ECHK(cudaStreamWaitEvent(st_, samp_join_[0], 0));
    }
    return cudaSuccess;
  }

  // the dense tensor-core DFT of the rounds that take it: a block per 64 bins of each such signal
  cudaError_t launch_dense() {
    if constexpr (sizeof(T) == 4) {
      if (!any_dense_) return cudaSuccess;
      const int64_t pm = std::min<int64_t>(p_max_, kDenseMaxP);
      const dim3 grid((unsigned)((pm + kDenseBins - 1) / kDenseBins), (unsigned)n_);
      k_dft_dense<<<grid, kDenseThreads, kDenseSmem, st_>>>(n_, cfg_, run_, (const float2*)part_, (const float2*)tab_,
                                                           (float2*)Y_);
      return cudaGetLastError();
    }
    return cudaSuccess;
  }

  // one persistent sampling launch per set-group size present in the batch
  // The launches are independent (each takes its own queue of tiles): the first runs on the
  // engine's stream, the others on streams of their own forked from it and joined back, so that
  // each persistent launch's last, partly empty wave overlaps the next one's blocks.
  cudaError_t launch_samples(int64_t* launches) {
    int forked = 0;
    bool first = true;
    for (int ns = 1; ns <= kMaxSetGroup; ++ns) {
      if (!(ns_mask_ & (1u << (ns - 1)))) continue;
      cudaStream_t s = st_;
      if (!first) {
        if (forked == 0) ECHK(cudaEventRecord(samp_fork_, st_));
        s = samp_st_[forked];
        ECHK(cudaStreamWaitEvent(s, samp_fork_, 0));
      }
#define SFFT_SAMPLE(NSV)                                                                                      \
  case NSV:                                                                                                   \
    if constexpr (sizeof(T) == 8) {                                                                           \
      if (any_df_) {                                                                                          \
        k_sample<T, NSV, true><<<2 * n_sm_, kSampleThreads, 0, s>>>(n_, cfg_, run_, ctl_, scans_, alpha_,     \
                                                                    gam_, (C2*)Cm_, (C2*)tab_, (C2*)part_);   \
        break;                                                                                                \
      }                                                                                                       \
    }                                                                                                         \
    k_sample<T, NSV, false><<<2 * n_sm_, kSampleThreads, 0, s>>>(n_, cfg_, run_, ctl_, scans_, alpha_, gam_,   \
                                                                 (C2*)Cm_, (C2*)tab_, (C2*)part_);           \
    break;
      switch (ns) {
        SFFT_SAMPLE(1)
        SFFT_SAMPLE(2)
        SFFT_SAMPLE(3)
        SFFT_SAMPLE(4)
        SFFT_SAMPLE(5)
        SFFT_SAMPLE(6)
        SFFT_SAMPLE(7)
        SFFT_SAMPLE(8)
        default: break;
      }
#undef SFFT_SAMPLE
      ECHK(cudaGetLastError());
      if (launches) launches[2] += 1;
      if (!first) {
        ECHK(cudaEventRecord(samp_join_[forked], s));
        ++forked;
      }
      first = false;
    }
    for (int q = 0; q < forked; ++q) ECHK(cudaStreamWaitEvent(st_, samp_join_[q], 0));
    return cudaSuccess;
  }

  // One fused round: a launch per set count present (the signals whose round is marked
  // fused run it and plan the next), then the tail that counts it and sets the loop condition.
  cudaError_t launch_fused(const PlanArgs& pa, int64_t* launches) {
    if constexpr (sizeof(T) == 4) {
      FusedArgs fa;
      fa.pa = pa;
      fa.pt = PrimeTables{ptab_, n_ptab_, pfirst_, pfirst_n_, dirs_, plist_};
      fa.cfg = cfg_;
      fa.run = run_;
      fa.ctl = ctl_;
      fa.hist = hist_;
      fa.ubuf = u_;
      fa.sig_w = sig_w_;
      fa.sig_a = sig_a_;
      fa.tw = (const float2*)tw_;
      fa.shblk = shblk_;
      fa.regw = regw_;
      fa.rega = rega_;
      fa.regtw = (float2*)regtw_;
      fa.hash = hash_;
      fa.tws = tw_src();
      fa.L_alloc = fuse_L_max_;
      for (int ns = 1; ns <= kFusedMaxSets; ++ns) {
        if (!(fuse_ns_mask_ & (1u << (ns - 1)))) continue;
        ECHK(fused_launch(ns, n_, smem_fused_, st_, fa));
        launches[6] += 1;
      }
      ECHK(fused_tail(st_, ctl_, pa.use_cond, pa.cond_fused));
      launches[6] += 1;
    }
    return cudaSuccess;
  }

  // ---------------------------------------------------------------- one round
  // occupied bins into the candidate list, then the ratio test, read-out and merge over it
  cudaError_t launch_classify(const ClassifyOut& co) {
    k_occupied<T><<<8 * n_sm_, 256, 0, st_>>>(n_, cfg_, run_, ctl_, scans_, (const C2*)Y_, cand_, co.eta_override);
    ECHK(cudaGetLastError());
    k_classify<T><<<8 * n_sm_, 256, 0, st_>>>(n_, cfg_, run_, ctl_, cand_, (const C2*)Y_, u_, shblk_, regw_, rega_,
                                             (C2*)regtw_, hash_, co);
    return cudaGetLastError();
  }

  // The round's plan: every signal's parameters and the round's totals over the grid (its last
  // block decides the mode splits), the work counts and their scans within blocks (its last
  // block scans the blocks' totals and writes the round control), then the blocks' offsets.
  cudaError_t launch_plan_kernels(const PlanArgs& pa, HistRec* hist, int64_t* launches) {
    const int nblk = (n_ + kPlanBlk - 1) / kPlanBlk;
    k_plan_signals<T><<<nblk, kPlanBlk, 0, st_>>>(pa, cfg_, run_, ptab_, n_ptab_, pfirst_, pfirst_n_, dirs_, plist_, u_,
                                                  hist, pacc_, powner_, pblk_, pdec_);
    ECHK(cudaGetLastError());
    k_plan_scan<T><<<nblk, kPlanBlk, 0, st_>>>(pa, cfg_, run_, ctl_, scans_, pacc_, powner_, pblk_, pdec_);
    ECHK(cudaGetLastError());
    k_plan_offsets<<<nblk, kPlanBlk, 0, st_>>>(n_, run_, scans_, pblk_);
    ECHK(cudaGetLastError());
    if (launches) launches[0] += 3;
    return cudaSuccess;
  }

  cudaError_t launch_plan(const PlanArgs& pa, int64_t* launches) {
    return launch_plan_kernels(pa, hist_, launches);
  }

  // The batched kernels of a round, over the signals not left to the fused kernel; mark(q)
  // records the profile events between the kernel classes.
  template <class Mark>
  cudaError_t enqueue_batched(int64_t* launches, Mark mark) {
    ECHK(launch_tables());
    launches[0] += 1;
    ECHK(mark(1));
    ECHK(mark(2));
    // the filter spectra depend only on the round's primes: they are made on a side stream beside
    // the sampling, whose persistent blocks take their tiles from a queue and so absorb the SMs
    // the filters hold for a while
    ECHK(cudaEventRecord(fork_ev_, st_));
    ECHK(cudaStreamWaitEvent(side_, fork_ev_, 0));
    ECHK(launch_filters(side_));
    ECHK(cudaEventRecord(join_ev_, side_));
    ECHK(launch_samples(launches));
    ECHK(cudaStreamWaitEvent(st_, join_ev_, 0));
    ECHK(mark(3));
    ECHK(launch_dft_rows(false));
    launches[3] += small_logL_max_ > kSmallFftLog ? 4 : 2;
    if (any_dense_) {
      ECHK(launch_dense());
      launches[3] += 1;
    }
    if (any_big_) {
      k_bigA<T><<<4 * n_sm_, 256, smem_bigA_, st_>>>(n_, cfg_, run_, ctl_, scans_, (C2*)part_, (C2*)tab_, (C2*)twG_,
                                                     Lmax_, (C2*)Z_);
      ECHK(cudaGetLastError());
      k_bigB<T><<<4 * n_sm_, 256, smem_bigB_, st_>>>(n_, cfg_, run_, ctl_, scans_, (C2*)twG_, Lmax_, (C2*)Z_);
      ECHK(cudaGetLastError());
      k_bigC<T><<<4 * n_sm_, 256, smem_bigA_, st_>>>(n_, cfg_, run_, ctl_, scans_, (C2*)tab_, (C2*)twG_, Lmax_,
                                                     (C2*)Z_, (C2*)Y_);
      ECHK(cudaGetLastError());
      launches[3] += 3;
    }
    ECHK(mark(4));
    if (any_peel_) {
      k_peel<T><<<dim3(peel_gx_, n_), 256, 0, st_>>>(n_, cfg_, run_, u_, regw_, rega_, (const C2*)regtw_, (C2*)Y_);
      ECHK(cudaGetLastError());
      launches[5] += 1;
    }
    ECHK(mark(6));
    ClassifyOut co{nullptr, nullptr, nullptr, 0, nullptr, nullptr, -1.0};
    ECHK(launch_classify(co));
    launches[4] += 2;
    ECHK(mark(5));
    return cudaSuccess;
  }

  // One round enqueued from the host: plan, batched kernels, then kFusedHostRounds fused rounds
  // (launches without work return at once).
  cudaError_t enqueue_round(const PlanArgs& pa, int64_t* launches, int round_idx, bool record) {
    auto mark = [&](int q) -> cudaError_t {
      if (!record) return cudaSuccess;
      return cudaEventRecord(events_[(size_t)round_idx * 8 + q], st_);
    };
    ECHK(mark(0));
    ECHK(launch_plan(pa, launches));
    ECHK(enqueue_batched(launches, mark));
    if (any_fuse_)
      for (int q = 0; q < kFusedHostRounds; ++q) ECHK(launch_fused(pa, launches));
    ECHK(mark(7));
    return cudaSuccess;
  }

  cudaError_t bind(const int32_t* const* sig_w, const double2* const* sig_a, const int64_t* k_sig,
                   const int64_t* caps, const double* noise_sigma = nullptr, const uint64_t* noise_seed = nullptr) {
    // pinned staging: sig_w pointers, sig_a pointers, k_sig, capacities, output row offsets,
    // output element offsets (rows of d_s ints)
    int64_t* h = reinterpret_cast<int64_t*>(host_stage_);
    int64_t rows = 0, elems = 0;
    for (int s = 0; s < n_; ++s) {
      const int64_t cap = caps ? caps[s] : 0;
      h[s] = (int64_t)(uintptr_t)sig_w[s];
      h[n_ + s] = (int64_t)(uintptr_t)sig_a[s];
      h[2 * n_ + s] = k_sig[s];
      h[3 * n_ + s] = cap;
      h[4 * n_ + s] = rows;
      h[5 * n_ + s] = elems;
      h[6 * n_ + s] = noise_sigma ? (int64_t)double_bits(noise_sigma[s]) : 0;
      h[7 * n_ + s] = noise_seed ? (int64_t)noise_seed[s] : 0;
      rows += cap;
      elems += cap * cfg_host_[s].d;
    }
    ECHK(cudaMemcpyAsync(bind_, h, (size_t)n_ * kBindArrays * sizeof(int64_t), cudaMemcpyHostToDevice, st_));
    sig_w_ = reinterpret_cast<const int32_t* const*>(bind_);
    sig_a_ = reinterpret_cast<const double2* const*>(reinterpret_cast<int64_t*>(bind_) + n_);
    ksig_dev_ = reinterpret_cast<int64_t*>(bind_) + 2 * n_;
    k_init<<<(n_ + 255) / 256, 256, 0, st_>>>(n_, run_, reinterpret_cast<const int64_t*>(bind_));
    ECHK(cudaGetLastError());
    ECHK(cudaMemsetAsync(hash_, 0xFF, (size_t)hash_total_ * sizeof(int32_t), st_));
    ECHK(cudaMemsetAsync(ctl_, 0, sizeof(RoundCtl), st_));
    const int gx = (int)std::min<int64_t>(std::max<int64_t>((kd_max_ + 255) / 256, 1), 64);
    k_bind_tw<T><<<dim3(gx, n_), 256, 0, st_>>>(n_, cfg_, run_, sig_w_, shblk_, (C2*)tw_);
    ECHK(cudaGetLastError());
    if (seed_n_ > 0 && n_ == 1) {
      const int n_seed = (int)std::min<int64_t>(seed_n_, cfg_host_[0].reg_cap);
      k_seed<T><<<(n_seed + 255) / 256, 256, 0, st_>>>(cfg_, run_, seed_w_, seed_a_, n_seed, seed_round_, seed_aref_,
                                                       shblk_, regw_, rega_, (C2*)regtw_, hash_);
      seed_n_ = 0;   // one run only
    }
    return cudaGetLastError();
  }

  void set_seed(const int32_t* w, const double2* a, int64_t n, int round0, double a_ref) override {
    seed_w_ = w;
    seed_a_ = a;
    seed_n_ = n;
    seed_round_ = round0;
    seed_aref_ = a_ref;
  }

  cudaError_t last_state(int* rounds, double* a_ref) override {
    SigRun r;
    ECHK(cudaMemcpyAsync(&r, run_, sizeof(SigRun), cudaMemcpyDeviceToHost, st_));
    ECHK(cudaStreamSynchronize(st_));
    *rounds = r.round;
    *a_ref = r.a_ref;
    return cudaSuccess;
  }

  // Adds a conditional node of the given type after the work captured so far on cs, and
  // captures fill() (launches on st_) into its body.
  template <class Fill>
  cudaError_t capture_conditional(cudaStream_t cs, cudaGraphConditionalNodeType type,
                                  cudaGraphConditionalHandle handle, Fill fill) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    ECHK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd));
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
    cp->type = cudaGraphNodeTypeConditional;
    cp->conditional.handle = handle;
    cp->conditional.type = type;
    cp->conditional.size = 1;
    cudaGraphNode_t node;
    ECHK(cudaGraphAddNode(&node, cg, deps, nullptr, nd, cp));
    ECHK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t inner;
    ECHK(cudaStreamCreateWithFlags(&inner, cudaStreamNonBlocking));
    cudaStream_t saved = st_;
    st_ = inner;
    cudaError_t e = cudaStreamBeginCaptureToGraph(inner, cp->conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = fill();
      cudaGraph_t captured;
      const cudaError_t e2 = cudaStreamEndCapture(inner, &captured);
      if (e == cudaSuccess) e = e2;
    }
    st_ = saved;
    cudaStreamDestroy(inner);
    return e;
  }

  cudaError_t build_graph(int hard_rounds) {
    // while (some signal active) {
    //   plan;
    //   if (some signal has batched work) { the batched kernels }
    //   while (some signal has a fused round planned) { fused round }
    // }
    cudaGraph_t g;
    ECHK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle handle;
    ECHK(cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault));
    // the parameter block has union members without default constructors: zeroed raw storage
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
    cp->type = cudaGraphNodeTypeConditional;
    cp->conditional.handle = handle;
    cp->conditional.type = cudaGraphCondTypeWhile;
    cp->conditional.size = 1;
    cudaGraphNode_t node;
    ECHK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, cp));
    cudaGraph_t body = cp->conditional.phGraph_out[0];
    PlanArgs pa = plan_args(hard_rounds);
    pa.use_cond = 1;
    pa.cond = handle;
    ECHK(cudaGraphConditionalHandleCreate(&pa.cond_batch, body, 0, cudaGraphCondAssignDefault));
    if (any_fuse_) ECHK(cudaGraphConditionalHandleCreate(&pa.cond_fused, body, 0, cudaGraphCondAssignDefault));
    cudaStream_t cs;
    ECHK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = st_;
    st_ = cs;
    int64_t dplan[SFFT_NKCLASS] = {};
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = launch_plan(pa, dplan);
      if (e == cudaSuccess)
        e = capture_conditional(cs, cudaGraphCondTypeIf, pa.cond_batch, [&]() {
          return enqueue_batched(launch_batched_, [](int) { return cudaSuccess; });
        });
      if (e == cudaSuccess && any_fuse_)
        e = capture_conditional(cs, cudaGraphCondTypeWhile, pa.cond_fused,
                                [&]() { return launch_fused(pa, launch_fused_); });
      cudaGraph_t captured;
      const cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
      if (e == cudaSuccess) e = e2;
    }
    st_ = saved;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return e;
    }
    ECHK(cudaGraphInstantiate(&graph_exec_, g, 0));
    graph_ = g;
    return cudaSuccess;
  }

  PlanArgs plan_args(int hard_rounds) const {
    PlanArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.n = n_;
    pa.part_cap = part_cap_;
    pa.n_sm = n_sm_;
    pa.single_max_logL = log2i(single_max_L<T>());
    pa.hard_rounds = hard_rounds;
    pa.fuse = any_fuse_ ? 1 : 0;
    pa.dft_thr_s = dft_thr_s_;
    pa.dft_smem_s = (int64_t)dft_smem_s_;
    pa.dft_thr_l = dft_thr_l_;
    pa.dft_e_l = dft_e_l_;
    pa.dft_e_s = dft_e_s_;
    pa.dft_smem_l = (int64_t)smem_dft_;
    return pa;
  }

  int hard_rounds() const {
    int m = 1;
    for (const SigCfg& c : cfg_host_) m = std::max(m, c.max_rounds);
    return std::min(m, SFFT_STATS_MAX_ROUNDS);
  }

  // ---------------------------------------------------------------- execute
  cudaError_t run(const int32_t* const* sig_w, const double2* const* sig_a, const int64_t* k_sig, const int64_t* caps,
                  const double* noise_sigma, const uint64_t* noise_seed, int32_t* out_w, double2* out_a,
                  int64_t* n_found, int* status, sfft_stats* stats) override {
    int64_t launches[SFFT_NKCLASS] = {};
    const int hard = hard_rounds();
    ECHK(bind(sig_w, sig_a, k_sig, caps, noise_sigma, noise_seed));
    launches[5] += 2;
    int rounds_enqueued = 0;
    const bool record = profile_ && stats != nullptr;
    if (use_graph_ && !record) {
      if (!graph_exec_) ECHK(build_graph(hard));
      ECHK(cudaGraphLaunch(graph_exec_, st_));
    } else {
      RoundCtl* hctl = reinterpret_cast<RoundCtl*>(reinterpret_cast<char*>(host_stage_) + stage_ctl_);
      const PlanArgs pa = plan_args(hard);
      for (;;) {
        const int G = rounds_enqueued < 4 ? 4 : 2;
        for (int q = 0; q < G && rounds_enqueued <= hard; ++q) {
          ECHK(enqueue_round(pa, launches, rounds_enqueued, record));
          ++rounds_enqueued;
        }
        ECHK(cudaMemcpyAsync(hctl, ctl_, sizeof(RoundCtl), cudaMemcpyDeviceToHost, st_));
        ECHK(cudaStreamSynchronize(st_));
        if (hctl->active == 0 || rounds_enqueued > hard) break;
      }
    }
    k_output<<<n_, 1024, 0, st_>>>(n_, cfg_, run_, regw_, rega_, reinterpret_cast<const int64_t*>(bind_), out_w,
                                   out_a, outn_, outst_, stats ? hist_ : nullptr);
    ECHK(cudaGetLastError());
    launches[5] += 1;
    char* hb = reinterpret_cast<char*>(host_stage_);
    int64_t* hn = reinterpret_cast<int64_t*>(hb + stage_n_);
    int* hst = reinterpret_cast<int*>(hb + stage_st_);
    ECHK(cudaMemcpyAsync(hn, outn_, n_ * sizeof(int64_t), cudaMemcpyDeviceToHost, st_));
    ECHK(cudaMemcpyAsync(hst, outst_, n_ * sizeof(int), cudaMemcpyDeviceToHost, st_));
    RoundCtl* hctl_end = reinterpret_cast<RoundCtl*>(hb + stage_ctl_);
    if (stats) ECHK(cudaMemcpyAsync(hctl_end, ctl_, sizeof(RoundCtl), cudaMemcpyDeviceToHost, st_));
    HistRec* hh = nullptr;
    std::vector<SigRun> runs;
    if (stats) {
      hh = reinterpret_cast<HistRec*>(hb + stage_hist_);
      ECHK(cudaMemcpyAsync(hh, hist_, SFFT_STATS_MAX_ROUNDS * sizeof(HistRec), cudaMemcpyDeviceToHost, st_));
      runs.resize(n_);
      ECHK(cudaMemcpyAsync(runs.data(), run_, n_ * sizeof(SigRun), cudaMemcpyDeviceToHost, st_));
    }
    ECHK(cudaStreamSynchronize(st_));
    for (int s = 0; s < n_; ++s) {
      n_found[s] = hn[s];
      status[s] = hst[s];
    }
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      int rounds = 0;
      bool conv = true;
      for (int s = 0; s < n_; ++s) {
        rounds = std::max(rounds, runs[s].round);
        stats->samples += runs[s].samples;
        stats->terms += runs[s].terms;
        stats->terms_fused += runs[s].terms_fused;
        conv = conv && (hst[s] == SFFT_OK || hst[s] == SFFT_ERR_INCONSISTENT || hst[s] == SFFT_ERR_CAPACITY) &&
               !runs[s].active;
      }
      stats->rounds = rounds;
      stats->converged = conv ? 1 : 0;
      const int r0 = std::min(runs[0].round, SFFT_STATS_MAX_ROUNDS);
      for (int i = 0; i < r0; ++i) {
        stats->p[i] = hh[i].p;
        stats->K[i] = hh[i].K;
        stats->accepted[i] = hh[i].accepted;
        stats->registry[i] = hh[i].live;
      }
      if (use_graph_ && !record) {
        // bodies of the device loop (three plan launches each), those with batched work, and fused rounds
        launches[0] += 3 * hctl_end->round;
        for (int q = 0; q < SFFT_NKCLASS; ++q)
          launches[q] += launch_batched_[q] * hctl_end->bodies_batched + launch_fused_[q] * hctl_end->fused_iters;
      }
      for (int q = 0; q < SFFT_NKCLASS; ++q) stats->kernel_launches[q] = launches[q];
      if (record) {
        for (int i = 0; i < rounds_enqueued; ++i) {
          float ms;
          const size_t b = (size_t)i * 8;
          ECHK(cudaEventElapsedTime(&ms, events_[b + 0], events_[b + 1]));
          stats->kernel_ms[0] += ms;
          ECHK(cudaEventElapsedTime(&ms, events_[b + 2], events_[b + 3]));
          stats->kernel_ms[2] += ms;
          ECHK(cudaEventElapsedTime(&ms, events_[b + 3], events_[b + 4]));
          stats->kernel_ms[3] += ms;
          ECHK(cudaEventElapsedTime(&ms, events_[b + 4], events_[b + 6]));
          stats->kernel_ms[5] += ms;
          ECHK(cudaEventElapsedTime(&ms, events_[b + 6], events_[b + 5]));
          stats->kernel_ms[4] += ms;
          ECHK(cudaEventElapsedTime(&ms, events_[b + 5], events_[b + 7]));
          stats->kernel_ms[6] += ms;
        }
      }
    }
    return cudaSuccess;
  }

  // ---------------------------------------------------------------- step calls (slot 0)
  cudaError_t prepare_step(int64_t p, const int64_t* u, int K, const int32_t* w, const double2* a) {
    if (u) {
      std::vector<int64_t> um((size_t)cfg_host_[0].d);
      for (int l = 0; l < cfg_host_[0].d; ++l) {
        int64_t v = u[l] % p;
        um[l] = v < 0 ? v + p : v;
      }
      ECHK(cudaMemcpyAsync(u_ + cfg_host_[0].u_off, um.data(), um.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                           st_));
      ECHK(cudaStreamSynchronize(st_));
    }
    const int32_t* wp[1] = {w};
    const double2* ap[1] = {a};
    int64_t ks[1] = {K};
    int64_t cp[1] = {0};
    ECHK(bind(wp, ap, ks, cp));
    PlanArgs pa = plan_args(1 << 20);
    pa.fuse = 0;   // a step call runs its stage in the batched kernels
    pa.force = 1;
    pa.force_p = p;
    pa.force_K = K;
    ECHK(launch_plan_kernels(pa, nullptr, nullptr));
    return launch_tables();
  }

  cudaError_t step_sample(int64_t p, const int64_t* u, int64_t K, const int32_t* w, const double2* a,
                          void* y_out) override {
    ECHK(prepare_step(p, u, (int)K, w, a));
    ECHK(launch_samples(nullptr));
    k_reduce<T><<<2 * n_sm_, 256, 0, st_>>>(cfg_, run_, cfg_host_[0].n_sets, (C2*)part_, (C2*)y_out);
    ECHK(cudaGetLastError());
    return cudaStreamSynchronize(st_);
  }

  cudaError_t step_dft(int64_t p, int n_rows, const void* y, void* Y_out) override {
    ECHK(prepare_step(p, nullptr, 0, nullptr, nullptr));
    // the rows enter as a single split at the start of the partial arena
    const int ns = cfg_host_[0].n_sets;
    ECHK(cudaMemsetAsync(part_, 0, (size_t)ns * p * sizeof(C2), st_));
    ECHK(cudaMemcpyAsync(part_, y, (size_t)n_rows * p * sizeof(C2), cudaMemcpyDeviceToDevice, st_));
    ECHK(launch_dft_rows());
    ECHK(launch_dense());
    if (any_big_) {
      k_bigA<T><<<4 * n_sm_, 256, smem_bigA_, st_>>>(n_, cfg_, run_, ctl_, scans_, (C2*)part_, (C2*)tab_, (C2*)twG_,
                                                     Lmax_, (C2*)Z_);
      k_bigB<T><<<4 * n_sm_, 256, smem_bigB_, st_>>>(n_, cfg_, run_, ctl_, scans_, (C2*)twG_, Lmax_, (C2*)Z_);
      k_bigC<T><<<4 * n_sm_, 256, smem_bigA_, st_>>>(n_, cfg_, run_, ctl_, scans_, (C2*)tab_, (C2*)twG_, Lmax_,
                                                     (C2*)Z_, (C2*)Y_);
      ECHK(cudaGetLastError());
    }
    ECHK(cudaMemcpyAsync(Y_out, (C2*)Y_ + cfg_host_[0].Y_off, (size_t)n_rows * p * sizeof(C2),
                         cudaMemcpyDeviceToDevice, st_));
    return cudaStreamSynchronize(st_);
  }

  cudaError_t step_classify(int64_t p, const int64_t* u, const void* Y, double eta, int64_t cap, int32_t* h_out,
                            int32_t* w_out, double2* a_out, int64_t* n_out, int* err) override {
    ECHK(prepare_step(p, u, 0, nullptr, nullptr));
    const int ns = cfg_host_[0].n_sets;
    ECHK(cudaMemcpyAsync((C2*)Y_ + cfg_host_[0].Y_off, Y, (size_t)ns * p * sizeof(C2), cudaMemcpyDeviceToDevice, st_));
    ECHK(cudaMemsetAsync(stepc_, 0, 2 * sizeof(int), st_));
    int* cnt = reinterpret_cast<int*>(stepc_);
    ClassifyOut co{h_out, w_out, a_out, (int)cap, cnt, cnt + 1, eta};
    ECHK(launch_classify(co));
    int* h = reinterpret_cast<int*>(reinterpret_cast<char*>(host_stage_) + stage_st_);
    ECHK(cudaMemcpyAsync(h, stepc_, 2 * sizeof(int), cudaMemcpyDeviceToHost, st_));
    ECHK(cudaStreamSynchronize(st_));
    *n_out = h[0];
    *err = h[1];
    return cudaSuccess;
  }

 private:
  template <typename P>
  cudaError_t alloc(P** out, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes == 0 ? 16 : bytes);
    if (e == cudaSuccess) {
      allocs_.push_back(q);
      bytes_ += bytes;
      *out = reinterpret_cast<P*>(q);
    }
    return e;
  }

  static size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

  int n_ = 0, dev_ = 0, n_sm_ = 148;
  cudaStream_t st_ = nullptr;
  bool profile_ = false, use_graph_ = false, any_big_ = false;
  bool any_peel_ = false;   // some slot removes its registry in the bin domain
  bool any_fuse_ = false;   // some slot may run short rounds in the fused kernel (FP32 engines)
  int fuse_sets_max_ = 0;      // most sample sets of such a slot
  unsigned fuse_ns_mask_ = 0;  // set counts of such slots
  int fuse_L_max_ = 0;         // and its longest fused Bluestein length
  size_t smem_fused_ = 0;      // dynamic shared memory of the fused kernel
  int2* cand_ = nullptr;    // (slot, bin) of the round's occupied bins, sum of p_max entries
  int peel_gx_ = 1;         // k_peel blocks per signal
  int logL_big_max_ = 0, small_logL_max_ = 1, small_threads_ = 256, n_ptab_ = 0;
  size_t smem_small_ = 0, smem_bigA_ = 0, smem_bigB_ = 0, bytes_ = 0, host_stage_bytes_ = 0;
  size_t smem_dft_ = 0;   // the long-row DFT kernel's dynamic shared memory (rows + prefetch row)
  int dft_thr_s_ = 32;     // the short-row DFT launch's block size
  int dft_thr_l_ = 256;    // the long-row DFT launch's block size
  int dft_e_l_ = 0;        // its values per thread and pass (16, or 0: the precision's default)
  int dft_e_s_ = 0;        // the same for the short-row launch
  size_t dft_smem_s_ = 0;  // and dynamic shared memory
  int64_t rows_max_ = 0;
  int64_t Lmax_ = 2, p_max_ = 2, part_cap_ = 0, hash_total_ = 0, k_max_ = 0, kd_max_ = 0, reg_cap_max_ = 0;
  bool any_dense_ = false;   // some slot takes short rounds' DFT on the tensor cores
  bool any_df_ = false;      // the slots sample in double-float (tables and coefficients packed for it)
  // registry seed for the next run (set_seed)
  const int32_t* seed_w_ = nullptr;
  const double2* seed_a_ = nullptr;
  int64_t seed_n_ = 0;
  int seed_round_ = 0;
  double seed_aref_ = 0.0;
  std::vector<SigCfg> cfg_host_;
  std::vector<void*> allocs_;
  std::vector<cudaEvent_t> events_;
  cudaStream_t side_ = nullptr;                            // filter spectra beside the sampling
  cudaEvent_t fork_ev_ = nullptr, join_ev_ = nullptr;
  // the sampling launches of the set-group sizes after the first run on streams of their own
  cudaStream_t samp_st_[kMaxSetGroup - 1] = {};
  cudaEvent_t samp_fork_ = nullptr, samp_join_[kMaxSetGroup - 1] = {};
  void* host_stage_ = nullptr;
  SigCfg* cfg_ = nullptr;
  SigRun* run_ = nullptr;
  RoundCtl* ctl_ = nullptr;
  Scans scans_;
  int32_t* ptab_ = nullptr;
  int32_t* pfirst_ = nullptr;
  unsigned long long* powner_ = nullptr;   // [p_max + 1] owner election keys (owner_key), all ones at creation
  PlanAcc* pacc_ = nullptr;                // the round's totals between the planning kernels
  PlanBlk* pblk_ = nullptr;                // [ceil(n / kPlanBlk)] per-block planning results
  PlanDec* pdec_ = nullptr;                // the round's split decision and arrival counters
  int64_t pfirst_n_ = 0;
  int64_t* dirs_ = nullptr;
  int32_t* shblk_ = nullptr;   // (start, size) per shift block of every slot (block form)
  int64_t* plist_ = nullptr;
  void* tw_ = nullptr;
  int32_t* regw_ = nullptr;
  void* regtw_ = nullptr;
  double2* rega_ = nullptr;
  int32_t* hash_ = nullptr;
  void* tab_ = nullptr;
  void* bhat_ = nullptr;
  void* Y_ = nullptr;
  void* Z_ = nullptr;
  int64_t* u_ = nullptr;
  int32_t* alpha_ = nullptr;
  int32_t* gam_ = nullptr;
  void* Cm_ = nullptr;
  void* root1k_ = nullptr;   // double2 [1024]: e^{2 pi i j / 1024}
  unsigned ns_mask_ = 0;   // set-group sizes present among the slots
  void* part_ = nullptr;
  void* twG_ = nullptr;
  void* twG3_ = nullptr;   // e^{-2 pi i j / len3_}, len3_ = 3 2^A: lengths 3 2^a of the one-block path
  void* twG5_ = nullptr;   // the same for 5 2^a
  // the one-block path's largest lengths 3 2^a and 5 2^a (and a table for the power-of-two ones)
  static constexpr int64_t len3_ = 3 * (single_max_L<T>() / 4);
  static constexpr int64_t len5_ = 5 * (single_max_L<T>() / 8);
  TwSrc<C2> tw_src() const {
    TwSrc<C2> t;
    t.t[0] = (const C2*)twG_;
    t.t[1] = (const C2*)twG3_;
    t.t[2] = (const C2*)twG5_;
    t.len[0] = Lmax_;
    t.len[1] = len3_;
    t.len[2] = len5_;
    return t;
  }
  HistRec* hist_ = nullptr;
  void* bind_ = nullptr;
  int64_t* outn_ = nullptr;
  int* outst_ = nullptr;
  void* stepc_ = nullptr;
  const int32_t* const* sig_w_ = nullptr;
  const double2* const* sig_a_ = nullptr;
  int64_t* ksig_dev_ = nullptr;
  size_t stage_ctl_ = 0, stage_n_ = 0, stage_st_ = 0, stage_hist_ = 0;
  cudaGraph_t graph_ = nullptr;
  cudaGraphExec_t graph_exec_ = nullptr;
  // launches per class of one batched round body and of one fused round (graph mode counts)
  int64_t launch_batched_[SFFT_NKCLASS] = {};
  int64_t launch_fused_[SFFT_NKCLASS] = {};
};

}  // namespace

cudaError_t engine_create(bool fp64, const std::vector<SlotDesc>& slots, cudaStream_t st, bool profile,
                          bool use_graph, EngineBase** out) {
  *out = nullptr;
  if (fp64) {
    auto* e = new Engine<double>();
    cudaError_t r = e->init(slots, st, profile, use_graph);
    if (r != cudaSuccess) {
      delete e;
      return r;
    }
    *out = e;
  } else {
    auto* e = new Engine<float>();
    cudaError_t r = e->init(slots, st, profile, use_graph);
    if (r != cudaSuccess) {
      delete e;
      return r;
    }
    *out = e;
  }
  return cudaSuccess;
}

}  // namespace sfft
