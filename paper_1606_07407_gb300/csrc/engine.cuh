// Batched round engine: per-signal configuration and round state live on the
// device, so every kernel of a round serves all signals of a batch and the
// host only launches rounds (or one CUDA graph whose loop the device ends).
#pragma once

#include <vector>

#include "sfft_internal.cuh"

namespace sfft {

constexpr int kPlanBlk = 128;        // signals per block of the planning kernels
#ifndef SFFT_DFT_E16
#define SFFT_DFT_E16 1
#endif
constexpr bool kDftE16 = SFFT_DFT_E16 != 0;   // long-row DFT in radix-16 passes (float, L <= 8192)
constexpr int kSingleMaxLf = 16384;   // one-block Bluestein length, FP32 (data + twiddles in shared memory)
constexpr int kSingleMaxLd = 8192;    // same for FP64
constexpr int kBigColElems = 4096;    // elements of one column tile of the four-step passes
constexpr int kBigRowElems = 2048;    // elements of one row tile

template <typename T> constexpr int single_max_L() { return sizeof(T) == 4 ? kSingleMaxLf : kSingleMaxLd; }

// Row pairs per warp for a set group of ns sets: 32 positions x of the half line, each with its
// mirror p - x.  Chunk and running sums (4 reals per position and set, twice) stay within about
// 80 registers in float, and the staged roots within 48 KiB of shared memory.
__host__ __device__ constexpr int row_pairs(int ns) { return ns <= 2 ? 5 : ns <= 4 ? 3 : ns <= 6 ? 2 : 1; }
// positions of the half line per sampling tile
__host__ __device__ constexpr int tile_x(int ns) { return 32 * kSampleWarps * row_pairs(ns); }

// Static description of one signal slot of a batch.
struct SigCfg {
  int d, n_sets, k, c8, max_rounds, n_dirs, n_primes, box_lo;   // c8: the prime factor c in eighths
  int ratio64;        // phase ratio and coefficient in double
  int coef_mean;      // coefficient = mean over the d + 1 sets (else Y_0[h] / p)
  int peel_bins;      // the registry leaves the transform bin by bin (else it is sampled with f)
  int shift_block;    // shifted sets move along block unwrap vectors (Alg. 2 as printed), else e_n / N
  int fuse_L;         // rounds of Bluestein length up to this run in the fused kernel (0: none)
  int shift_tilt;     // Alg. 3 (d = 2): set n shifted by (axis n) / Q, Q = (base + height) N, the
  int tilt_base, tilt_height, tilt_hypo;   // axes (base, -height) and (height, base)
  int reg_cap, hash_mask, logL_max;
  int empty_rounds;   // rounds in a row with no bin of any set occupied that end the recovery
  int dense_dft;      // rounds of primes up to kDenseMaxP take the tensor-core dense DFT
  int stall_div;      // > 0: stop (NOT_CONVERGED) after a round that accepted fewer than k* / stall_div bins
  int df_sample;      // FP64 engine: sampling in double-float on the FP32 pipe (roots, coefficients packed)
  int64_t N, p_max;
  int64_t p_min;      // floor of the prime rule: the i-th prime >= max(ceil(c k*), p_min)
  double tau, rho, delta, sigma;
  int64_t dirs_off, primes_off;  // into the direction / prime-list arrays
  int64_t blk_off;    // int32 [2 (n_sets - 1)]: start and size of each shift block (block form)
  int64_t tw_off;     // T2 [k * d]        unit twiddles e^{2 pi i w_n / N} of the signal's modes
  int64_t regw_off;   // int32 [reg_cap * d]
  int64_t rega_off;   // double2 [reg_cap]
  int64_t regtw_off;  // T2 [reg_cap * d]
  int64_t hash_off;   // int32 [hash_mask + 1]
  int64_t tab_off;    // T2 [2 * p_max]     W[m] = e^{2 pi i m / p}, then chirp[x] = e^{-pi i x^2 / p}
  int64_t bhat_off;   // T2 [L_max]         spectrum of the Bluestein filter
  int64_t p1;         // round 1's prime when its tables below were made with the engine (else 0)
  int64_t tab0_off, bhat0_off;   // those tables and filter spectrum (-1: none)
  int64_t Y_off;      // T2 [n_sets * p_max]
  int64_t z_off;      // T2 [(n_sets + 1) * L_max] four-step work space, -1 if never needed
  int64_t u_off;      // int64 [d]           direction of the round, reduced mod p
  int64_t mode_off;   // int32 [Kmax]        alpha_j = (w_j . u) mod p and 32 alpha_j mod p of the round
  int64_t C_off;      // T2 [n_sets * Kmax]  a_j e^{2 pi i w_{j,n} / N} of the round (registry: -a)
  int Kmax;           // k, plus reg_cap when the registry is sampled
  const double2* root1k;   // e^{2 pi i j / 1024}, j < 1024, in double (the engine's; shared by its slots)
};

// Dynamic state of one signal, updated by the kernels of each round.
struct SigRun {
  int active, round, status, err;
  int K_reg;          // registry entries ever created (pruned ones have a = 0)
  int n_live;         // entries with a != 0
  int any_occupied;   // some bin above the empty-bin level this round
  int n_acc;          // bins accepted this round
  int k_sig;          // modes of the bound black box
  int logL, big;      // power-of-two Bluestein length of the round (four-step path when big)
  int L;              // Bluestein length of the one-block path: m 2^a >= 2p - 1, m in {1, 3, 5}
  int fused;          // the round runs in the fused short-round kernel (one block for the signal)
  int dense;          // the round's DFT is the dense tensor-core contraction (k_dft_dense)
  int n_xt, groups, gsize, chunks, jper, splits;
  int mgroups;        // mode groups per sampling tile (warps sharing rows when p is small)
  int reg_start;      // registry entries at the start of the round
  int64_t p;
  unsigned long long mod_m;   // floor((2^64 - 1) / p), Barrett reduction
  unsigned long long proj_off;   // (box_lo mod p)(sum of u mod p) mod p, for project_mod
  unsigned int mod32;            // floor((2^32 - 1) / p) when (N + 1) p < 2^32, else 0
  unsigned int pad32;
  int64_t part_off;
  int64_t tab_at, bhat_at;   // this round's W / chirp table and filter spectrum (shared by equal primes)
  int tab_owner;             // 1: this signal computes them
  int empty_streak;   // rounds in a row, up to the last one run, with no bin of any set occupied
  unsigned long long maxy0_bits;
  double a_ref;
  double eta_prune;   // the round's prune level: max(rho A_ref, 6 sigma / sqrt(p))
  double noise_sigma;              // noise of the bound black box (0: none)
  unsigned long long noise_seed;
  int64_t samples, terms;
  int64_t terms_fused;  // of the terms, those of fused rounds
  int64_t n_out;
};

// Work totals of the round (exclusive scans over signals are in Scans).
struct RoundCtl {
  int active, round, splits, pad;
  int64_t n_tab, n_mode, n_rows, n_filt, n_bins, n_bigA, n_bigB, n_bigC, n_rows_s, n_filt_s;
  int64_t n_samp[kMaxSetGroup];               // sampling tiles, per set-group size
  unsigned long long ctr_samp[kMaxSetGroup], ctr_rows, ctr_filt;
  unsigned long long n_cand;                  // occupied bins found this round (classification)
  unsigned long long n_fused_next;            // signals with another fused round planned
  int64_t bodies_batched;                     // round bodies that had batched work (whole run)
  int64_t fused_iters;                        // fused rounds launched (whole run)
};

// The round's totals, gathered over the grid while the signals are planned (k_plan_signals)
// and read by the last blocks of the planning kernels; the last block of k_plan_scan clears
// them for the next round.  epoch numbers the plan launches of
// the engine (never cleared): the owner election of round e keys powner[p] by e.
struct PlanAcc {
  unsigned long long tiles, active, fused;   // batched tiles; active and fused signals
  unsigned long long wsum[65];               // sum of n_sets p over batched signals with min(chunks, 64) = c
  unsigned int epoch, pad;
};

// The round's split decision (the last block of k_plan_signals) and the arrival counters by
// which the last block of each planning kernel knows it is last (cleared by that block).
struct PlanDec {
  int S, q_tail;
  int64_t tail_from;
  unsigned int done1, done2;
};

// exclusive scans over signals: tables, modes, DFT rows, filters, bins, four-step passes, DFT
// rows and filters of short lengths, then sampling tiles for each set-group size 1..kMaxSetGroup
constexpr int kNumScans = 10 + kMaxSetGroup;
struct Scans {
  int64_t* v[kNumScans];       // each [n + 1]
};

// Per block of kPlanBlk signals: batched tiles, the partial sums tail splits q = 2..8 would add,
// the block's offset in the queue of tiles, and its work totals (then exclusive offsets).
struct PlanBlk {
  unsigned long long tiles;
  unsigned long long extra[7];
  int64_t tile_off;
  int64_t tot[kNumScans + 1];
};
enum { SC_TAB = 0, SC_MODE, SC_ROWS, SC_FILT, SC_BINS, SC_BIGA, SC_BIGB, SC_BIGC, SC_ROWS_S, SC_FILT_S, SC_SAMP0 };

constexpr int kSmallFftLog = 11;   // Bluestein rows up to 2048 points run in small-memory blocks
constexpr int kDenseMaxP = 8191;   // longest prime whose DFT the dense tensor-core kernel takes
constexpr int kErrTimeout = 4;     // SigRun::err bit: a bounded device wait ran out (1, 2: capacity)

struct HistRec {
  int64_t p;
  int32_t K, accepted, live, pad;
};

// Host-side description of one signal slot.
// Modes the sampling kernel sums for a signal this round: the black box's, plus the
// registry's when the residual is sampled rather than removed in the bin domain.
__host__ __device__ inline int sampled_modes(const SigCfg& c, const SigRun& r) {
  const int reg = r.K_reg < c.reg_cap ? r.K_reg : c.reg_cap;
  return r.k_sig + (c.peel_bins ? 0 : reg);
}

struct SlotDesc {
  int d;
  int64_t N;
  int64_t k;
  int c8;                          // prime factor c of the rule p >= c k*, in eighths (40: c = 5)
  int box_lo;
  int ratio64;
  int coef_mean;
  int peel_bins;
  int shift_block;
  int shift_tilt = 0;              // Alg. 3 (d = 2): sets shifted along the rotated axes
  int tilt_base = 0, tilt_height = 0, tilt_hypo = 0;
  int fuse = 1;                    // short rounds may run in the fused kernel
  int fuse_max_len = 0;            // longest Bluestein length run fused (0: the kernel's limit)
  int empty_rounds = 1;            // empty rounds in a row that end the recovery
  int dense_dft = 0;               // short rounds' DFT on the tensor cores (split BF16)
  int stall_div = 0;               // stop when a round accepts fewer than k* / stall_div bins
  int df_sample = 0;               // FP64 engine: double-float sampling
  std::vector<int> shift_blocks;   // block sizes of the shifted sets (block form)
  double tau, rho, delta, sigma;
  int max_rounds;
  std::vector<int64_t> dirs;     // n_dirs x d
  int n_dirs;
  std::vector<int64_t> primes;   // prime-list override (empty: rule)
  int64_t p_min = 0;             // floor of the rule
  int64_t p_max;
};

// ceil(c k) for the prime factor c = c8 / 8, in exact integer arithmetic
__host__ __device__ inline int64_t prime_floor_ck(int c8, int64_t k) { return ((int64_t)c8 * k + 7) / 8; }

// Engine interface, instantiated for float (FP32 bulk) and double (FP64).
class EngineBase {
 public:
  virtual ~EngineBase() {}
  // noise_sigma / noise_seed: per-signal noise of the black boxes (null: none)
  virtual cudaError_t run(const int32_t* const* sig_w, const double2* const* sig_a, const int64_t* k_sig,
                          const int64_t* caps, const double* noise_sigma, const uint64_t* noise_seed,
                          int32_t* out_w, double2* out_a, int64_t* n_found, int* status, sfft_stats* stats) = 0;
  virtual cudaError_t step_sample(int64_t p, const int64_t* u, int64_t K, const int32_t* w, const double2* a,
                                  void* y_out) = 0;
  virtual cudaError_t step_dft(int64_t p, int n_rows, const void* y, void* Y_out) = 0;
  virtual cudaError_t step_classify(int64_t p, const int64_t* u, const void* Y, double eta, int64_t cap,
                                    int32_t* h_out, int32_t* w_out, double2* a_out, int64_t* n_out, int* err) = 0;
  // The next run() of a one-slot engine starts from a registry of n entries (w int32 [n x d],
  // a complex128 [n], device, read by that run before it writes its outputs), after round0
  // rounds, with the empty-bin reference a_ref of the run that found them.
  virtual void set_seed(const int32_t* w, const double2* a, int64_t n, int round0, double a_ref) = 0;
  // slot 0's rounds run and empty-bin reference A_ref after the last run()
  virtual cudaError_t last_state(int* rounds, double* a_ref) = 0;
  virtual size_t device_bytes() const = 0;
  virtual int64_t max_prime() const = 0;
  virtual int64_t mode_capacity() const = 0;
};

// Creates an engine for the slots (all slots share T).  profile: CUDA-event timing per kernel class.
cudaError_t engine_create(bool fp64, const std::vector<SlotDesc>& slots, cudaStream_t st, bool profile,
                          bool use_graph, EngineBase** out);

}  // namespace sfft
