// Internal declarations shared by the CUDA translation units of the sparse-FFT
// library: complex helpers, the device round state, kernel argument blocks and
// the host launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sfft.h"

namespace sfft {

// ---------------------------------------------------------------- complex types
template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <typename T> using c2 = typename V2<T>::t;

__host__ __device__ inline float2 mk2(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 mk2(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk2(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk2(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk2(a.x, -a.y); }
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) {
  return mk2(a.x * s, a.y * s);
}

// ---------------------------------------------------------------- limits
constexpr int kMaxSetGroup = 8;     // sample sets accumulated per thread (register tile)
constexpr int kSampleWarps = 4;     // warps per sampling block
constexpr int kSampleRowsPerWarp = 4;
constexpr int kSampleRows = kSampleWarps * kSampleRowsPerWarp;   // 16 rows of 32 samples
constexpr int kSampleTileX = kSampleRows * 32;                    // 512 samples per block tile
constexpr int kSampleChunk = 32;    // modes staged in shared memory per step
constexpr int kFftSmemElems = 4096; // complex elements of one in-shared-memory FFT tile
constexpr int kSingleMaxL = 4096;   // largest Bluestein length done by one block per row

// Error bits of DevState::err
constexpr int kErrAccCapacity = 1;
constexpr int kErrRegCapacity = 2;
constexpr int kErrHashFull = 4;

// ---------------------------------------------------------------- device state
// One per plan; the host reads it back after every round.
struct DevState {
  unsigned long long max_y0_bits;  // largest |Y_0[h]| of the round, as double bits
  double a_ref;                    // first-round largest bin / p (empty-bin scale)
  int n_acc;                       // bins accepted this round
  int n_reg;                       // registry entries ever created (live or pruned)
  int n_live;                      // registry entries with a nonzero coefficient
  int any_occupied;                // some bin above the empty-bin level this round
  int err;                         // kErr* bits
  int pad;
};

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `st` and returns the launch error (cudaGetLastError).

// Per-round setup: u_mod[l] = dirs[dir_index][l] mod p; resets the round counters.
cudaError_t launch_round_begin(cudaStream_t st, DevState* state, const int64_t* dirs, int dir_index,
                               int d, int64_t p, int64_t* u_mod);

// Per-prime tables: W[i] = e^{2 pi i i/p}, chirp[x] = e^{-pi i x^2/p}, computed in double.
template <typename T>
cudaError_t launch_prime_tables(cudaStream_t st, int64_t p, c2<T>* W, c2<T>* chirp);

// Twiddles twG[m] = e^{-2 pi i m / Lmax}, m < Lmax, computed in double.
template <typename T>
cudaError_t launch_twiddles(cudaStream_t st, int64_t Lmax, c2<T>* twG);

// a-2: per-round mode projection.  Modes j < K_sig come from the signal (+a), the
// next K_reg from the registry (-a).  alpha[j] = (w_j . u) mod p;
// C[n * Kpad + j] = a_j e^{2 pi i w_{j,n-1} / N} (n >= 1), C[j] = a_j.
template <typename T>
cudaError_t launch_project(cudaStream_t st, int K_sig, int K_reg, int d, int64_t N, int64_t p,
                           const int64_t* u_mod, const int32_t* sig_w, const double2* sig_a,
                           const int32_t* reg_w, const double2* reg_a, int n_sets, int Kpad,
                           int32_t* alpha, c2<T>* C);

// a-3: partial samples part[(s * n_sets + n) * p + x] over mode split s.
struct SampleGeom {
  int n_xt;      // tiles of 512 samples
  int splits;    // mode splits
  int jper;      // modes per split (multiple of kSampleChunk)
  int groups;    // set groups
  int gsize;     // sets per group (<= kMaxSetGroup)
};
SampleGeom sample_geometry(int64_t p, int K, int n_sets, int64_t part_capacity_elems, int n_sm);
template <typename T>
cudaError_t launch_sample(cudaStream_t st, const SampleGeom& g, int64_t p, int K, int n_sets, int Kpad,
                          const int32_t* alpha, const c2<T>* C, const c2<T>* W, c2<T>* part);
// Sum of the split partials into y[n * p + x].
template <typename T>
cudaError_t launch_reduce_partials(cudaStream_t st, int64_t p, int n_sets, int splits,
                                   const c2<T>* part, c2<T>* y);

// a-4: Bluestein DFT of n_rows rows of length p held as `splits` partial sums.
struct DftGeom {
  int64_t L;
  int logL, logM1, logM2;
  bool single;
};
DftGeom dft_geometry(int64_t p);
template <typename T>
cudaError_t launch_bluestein(cudaStream_t st, const DftGeom& g, int64_t p, int n_rows, int splits,
                             const c2<T>* part, const c2<T>* chirp, const c2<T>* twG, int64_t Lmax,
                             c2<T>* Z, c2<T>* Y, DevState* state_maxy0);

// a-5: classification of the p bins.
struct ClassifyArgs {
  int64_t p;
  int64_t N;
  int d;
  int box_lo;
  int round;          // 1-based; round 1 fixes a_ref from the largest bin
  double rho, tau, delta, sigma;
  double eta_override;  // >= 0: use this level instead of the rho / sigma rule
  int acc_cap;
};
template <typename T, typename R>
cudaError_t launch_classify(cudaStream_t st, const ClassifyArgs& a, const c2<T>* Y, const int64_t* u_mod,
                            DevState* state, int32_t* acc_h, int32_t* acc_w, double2* acc_a);

// a-6: merge the accepted list into the registry hash, then prune.
cudaError_t launch_merge(cudaStream_t st, int d, int acc_cap, const int32_t* acc_w, const double2* acc_a,
                         DevState* state, int32_t* reg_w, double2* reg_a, int reg_cap, int32_t* hash,
                         int hash_mask);
cudaError_t launch_prune(cudaStream_t st, int64_t p, double rho, double sigma, int reg_cap,
                         DevState* state, double2* reg_a);
// Compaction of live entries (registry order) into the outputs; writes *count_dev.
cudaError_t launch_output(cudaStream_t st, int d, int reg_cap, const DevState* state,
                          const int32_t* reg_w, const double2* reg_a, int64_t capacity,
                          int32_t* freqs_out, double2* coeffs_out, int64_t* count_dev);

}  // namespace sfft
