// Per-signal steps of one round of Algorithm 2, as device functions: the batched kernels of
// the round engine call them for many signals at once, and the fused short-round kernel calls
// them for one signal per block.
//
//   plan_signal         stop rule, the round's prime (Alg. 2), line direction and geometry
//   table_entry         W[m] = e^{2 pi i m / p} and chirp[m] = e^{-pi i m^2 / p}
//   mode_entry          a mode's projection (w . u) mod p and per-set coefficients
//   peel_entry          a registry mode taken off its bin of every set (residual in the bin domain)
//   classify_candidate  Eq. 42 ratio test, Eq. 7 read-out, own-bin check, registry merge
#pragma once

#include "engine_kernels.cuh"

namespace sfft {

// ------------------------------------------------------------------ plan

struct PlanArgs {
  int n;
  int64_t part_cap;
  int n_sm;
  int single_max_logL;
  int force;            // step calls: slot 0 uses force_p and the direction already in its u slot
  int64_t force_p;
  int force_K;          // modes bound for the step call
  int use_cond;
  cudaGraphConditionalHandle cond;
  int hard_rounds;      // stop the device loop after this many rounds
  int fuse;             // 0: no round runs fused (step calls)
  cudaGraphConditionalHandle cond_batch;   // graph condition: some signal has batched work
  cudaGraphConditionalHandle cond_fused;   // graph condition: some signal has a fused round planned
  int dft_thr_s, dft_thr_l;                // block sizes of the short- and long-row DFT launches
  int64_t dft_smem_s, dft_smem_l;          // and their dynamic shared memory, bytes
  int dft_e_l, dft_e_s;                    // values per thread and pass of the long- and short-row launches (0: default)
};

__host__ __device__ inline int ceil_log2(int64_t v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}

// Smallest length m 2^a >= max(n, 32) with m in {1, 3, 5}: the cyclic convolution of Bluestein's
// DFT only needs n = 2p - 1 points, and these lengths factor into the FFT's radices.
__host__ __device__ inline int bluestein_length(int64_t n) {
  n = n < 32 ? 32 : n;
  int64_t best = (int64_t)1 << ceil_log2(n);
  for (int m = 3; m <= 5; m += 2) {
    const int64_t L = (int64_t)m << ceil_log2((n + m - 1) / m);
    if (L < best) best = L;
  }
  return (int)best;
}

__device__ __forceinline__ void big_geom(int logL, int* M1, int* M2, int* CT, int* RT) {
  const int l1 = logL / 2, l2 = logL - l1;
  *M1 = 1 << l1;
  *M2 = 1 << l2;
  *CT = min(*M2, max(1, kBigColElems / *M1));
  *RT = min(*M1, max(1, kBigRowElems / *M2));
}

// Tables of the prime rule and the line directions.
struct PrimeTables {
  const int32_t* ptab;
  int n_ptab;
  const int32_t* pfirst;
  int64_t pfirst_n;
  const int64_t* dirs;
  const int64_t* plist;
};

// Round setup of one signal (Alg. 2): the stop rule, then for an active signal the next round's
// prime, line direction (written to its u slot), Bluestein lengths and sampling geometry, and
// the statistics of the round just finished (first slot only).
template <typename T>
__device__ void plan_signal(const PlanArgs& a, const SigCfg& c, SigRun& r, const PrimeTables& pt, int64_t* ubuf,
                            HistRec* hist, bool first_slot) {
  if (first_slot && hist != nullptr && r.round >= 1 && r.round <= SFFT_STATS_MAX_ROUNDS) {
    hist[r.round - 1].accepted = r.n_acc;
    hist[r.round - 1].live = r.n_live;
  }
  if (r.active && !a.force) {
    // The residual is empty when c.empty_rounds rounds in a row, on successive line directions,
    // find no bin of any set above the empty-bin level: a wrong read-out that passed the own-bin
    // check (wrong outside the round's block, or by a multiple of p inside it) leaves a pair w,
    // w' that lines not separating them put in one bin, whose shifted sets differ by only about
    // 2 pi |w_n - w'_n| / N in phase, below the level; a later line of the block where they
    // differ, with another prime, splits the pair.
    if (r.round > 0) r.empty_streak = r.any_occupied ? 0 : r.empty_streak + 1;
    if (r.round > 0 && r.empty_streak >= c.empty_rounds) {
      r.active = 0;                        // the residual is empty: done
      r.status = SFFT_OK;
    } else if (r.err) {
      r.active = 0;
      r.status = (r.err & kErrTimeout) ? SFFT_ERR_TIMEOUT : SFFT_ERR_CAPACITY;
    } else if (c.stall_div > 0 && r.round >= 2 &&
               (int64_t)r.n_acc * c.stall_div < max((int64_t)c.k - r.n_live, (int64_t)1)) {
      r.active = 0;   // the round found almost none of the modes left: hand over (see stall_div)
      r.status = SFFT_ERR_NOT_CONVERGED;
    } else if (r.round >= c.max_rounds || r.round >= a.hard_rounds) {
      r.active = 0;
      r.status = SFFT_ERR_NOT_CONVERGED;
    }
  }
  r.fused = 0;
  if (r.active) {
    const int i = r.round + 1;
    int64_t p;
    if (a.force) {
      p = a.force_p;
    } else if (c.n_primes > 0) {
      p = pt.plist[c.primes_off + (i - 1) % c.n_primes];
    } else {
      const int64_t kstar = max((int64_t)c.k - r.n_live, (int64_t)1);
      const int64_t lo = max(max(prime_floor_ck(c.c8, kstar), c.p_min), (int64_t)2);
      // pfirst[v] = index of the smallest prime >= v, so the i-th prime >= lo is one lookup away
      const int64_t idx = lo < pt.pfirst_n ? (int64_t)pt.pfirst[lo] + i - 1 : (int64_t)pt.n_ptab;
      p = idx < pt.n_ptab ? pt.ptab[idx] : -1;
    }
    if (p < 2 || p > c.p_max) {
      r.active = 0;
      r.status = SFFT_ERR_INVALID_ARG;
    } else {
      r.p = p;
      r.mod_m = ~0ull / (uint64_t)p;
      r.round = i;
      if (!a.force) {
        const int di = i % c.n_dirs;
        for (int l = 0; l < c.d; ++l) {
          int64_t v = pt.dirs[c.dirs_off + (int64_t)di * c.d + l] % p;
          ubuf[c.u_off + l] = v < 0 ? v + p : v;
        }
      }
      r.proj_off = proj_offset(c.d, ubuf + c.u_off, c.box_lo, p, r.mod_m);
      r.mod32 = (uint64_t)(c.N + 1) * (uint64_t)p < (1ull << 32) ? 0xFFFFFFFFu / (uint32_t)p : 0u;
      const int K = a.force ? a.force_K : sampled_modes(c, r);
      r.logL = max(ceil_log2(2 * p - 1), 5);   // at least 32 points
      r.L = bluestein_length(2 * p - 1);
      r.big = r.L > (1 << a.single_max_logL);
      // fused rounds: short lines, and 2p < L (true of every prime) so that the half line of
      // a fused round has at most L / 4 positions
      r.fused = a.fuse && !r.big && r.L <= c.fuse_L && 2 * p < r.L;
      r.dense = c.dense_dft && p <= kDenseMaxP && sizeof(T) == 4;
      if (r.dense) r.fused = 0;
      r.groups = (c.n_sets + kMaxSetGroup - 1) / kMaxSetGroup;
      r.gsize = (c.n_sets + r.groups - 1) / r.groups;
      {
        // tiles cover the half line 0 <= x < H (each x also gives p - x); a tile's warps
        // split into mode groups when H is shorter than the tile
        const int64_t H = p / 2 + 1;
        const int rowx = 32 * row_pairs(r.gsize);
        r.mgroups = (sizeof(T) != 4) ? 1 : (H <= rowx ? 8 : H <= 2 * rowx ? 4 : H <= 4 * rowx ? 2 : 1);
        const int tx = tile_x(r.gsize) / r.mgroups;
        r.n_xt = (int)((H + tx - 1) / tx);
      }
      r.chunks = K > 0 ? (K + kSampleChunk - 1) / kSampleChunk : 1;
      r.any_occupied = 0;
      r.n_acc = 0;
      r.reg_start = r.K_reg;
      r.maxy0_bits = 0ull;
      r.samples += (int64_t)c.n_sets * p;
      r.terms += (int64_t)c.n_sets * p * K;
      if (r.fused) r.terms_fused += (int64_t)c.n_sets * p * K;
      if (first_slot && hist != nullptr && i <= SFFT_STATS_MAX_ROUNDS) {
        hist[i - 1].p = p;
        hist[i - 1].K = K;
        hist[i - 1].accepted = 0;
        hist[i - 1].live = r.n_live;
      }
    }
  }
}

// ------------------------------------------------------------------ tables

// W[m] = e^{2 pi i m / p} and chirp[m] = e^{-pi i m^2 / p} of one index m < p of a signal's tables
template <typename T>
__device__ __forceinline__ void table_entry(int64_t p, unsigned long long mod_m, int64_t m, c2<T>* t) {
  t[m] = unit_root<T>(m, p);
  // x^2 mod 2p from x^2 mod p: of r and r + p the one with the parity of x (p odd)
  uint64_t r2;
  if (p == 2) {
    r2 = ((uint64_t)m * (uint64_t)m) % 4u;
  } else {
    const uint64_t r = mod_barrett((uint64_t)m * (uint64_t)m, (uint64_t)p, mod_m);
    r2 = ((r ^ (uint64_t)m) & 1u) ? r + (uint64_t)p : r;
  }
  t[p + m] = cconj(unit_root<T>((int64_t)r2, 2 * p));
}

// Mode j of a signal this round (black box for j < k, with frequencies sw and coefficients sa;
// registry with -a after): returns its frequency vector, with its coefficient in *a0 and its
// row of twiddles e^{2 pi i w_j . s_n}, n = 1 .. n_sets - 1, in *twr.
template <typename T>
__device__ __forceinline__ const int32_t* mode_source(const SigCfg& c, const SigRun& r, int j,
                                                      const int32_t* __restrict__ sw, const double2* __restrict__ sa,
                                                      const c2<T>* __restrict__ tw, const int32_t* __restrict__ regw,
                                                      const double2* __restrict__ rega,
                                                      const c2<T>* __restrict__ regtw, c2<T>* a0, const c2<T>** twr) {
  const int d = c.d;
  const int32_t* w;
  double2 a;
  const int S = c.n_sets - 1;   // twiddles per mode: one per shifted set
  if (j < r.k_sig) {
    w = sw + (int64_t)j * d;
    a = sa[j];
    *twr = tw + c.tw_off + (int64_t)j * S;
  } else {
    const int jr = j - r.k_sig;
    w = regw + c.regw_off + (int64_t)jr * d;
    a = rega[c.rega_off + jr];
    a.x = -a.x;   // registry modes: f - g
    a.y = -a.y;
    *twr = regtw + c.regtw_off + (int64_t)jr * S;
  }
  *a0 = mk2((T)a.x, (T)a.y);
  return w;
}

// The round's tables entry of mode j: alpha_j = (w_j . u) mod p, ga_j = 32 alpha_j mod p and
// C[n][j] = a_j e^{2 pi i w_j . s_n}.
template <typename T>
__device__ __forceinline__ void mode_entry(const SigCfg& c, const SigRun& r, int s, int j, const int64_t* __restrict__ ubuf,
                                           const int32_t* const* __restrict__ sig_w,
                                           const double2* const* __restrict__ sig_a, const c2<T>* __restrict__ tw,
                                           const int32_t* __restrict__ regw, const double2* __restrict__ rega,
                                           const c2<T>* __restrict__ regtw, int32_t* __restrict__ alpha,
                                           int32_t* __restrict__ gam, c2<T>* __restrict__ Cm) {
  c2<T> a0;
  const c2<T>* twr;
  const int32_t* w = mode_source<T>(c, r, j, sig_w[s], sig_a[s], tw, regw, rega, regtw, &a0, &twr);
  const uint64_t acc = project_mod(w, c.d, ubuf + c.u_off, c.box_lo, r.p, r.mod_m, r.proj_off, r.mod32);
  alpha[c.mode_off + j] = (int32_t)acc;
  gam[c.mode_off + j] = (int32_t)mod_barrett(acc * 32u, (uint64_t)r.p, r.mod_m);
  c2<T>* crow = Cm + c.C_off + j;
  crow[0] = a0;
  for (int nn = 1; nn < c.n_sets; ++nn) crow[(int64_t)nn * c.Kmax] = cmul(a0, twr[nn - 1]);
}

// ------------------------------------------------------------------ Bluestein DFT helpers

// filter b[x] = conj(chirp[|x|]) of the cyclic convolution, |x| < p (x > L - p wraps to -x)
template <typename T>
__device__ __forceinline__ c2<T> filter_value(int64_t x, int64_t p, int64_t L, const c2<T>* chirp) {
  if (x < p) return cconj(chirp[x]);
  if (x > L - p) return cconj(chirp[L - x]);
  return mk2((T)0, (T)0);
}

// sample x of row `row`: the sum of the mode splits' partial sums
template <typename T>
__device__ __forceinline__ c2<T> sum_splits(const c2<T>* __restrict__ part, const SigRun& r, int n_sets, int row,
                                            int64_t x) {
  c2<T> acc = part[r.part_off + (int64_t)row * r.p + x];
  for (int q = 1; q < r.splits; ++q) acc = cadd(acc, part[r.part_off + ((int64_t)q * n_sets + row) * r.p + x]);
  return acc;
}

// *dst = max(*dst, largest v of the warp), as the bits of a non-negative double (all 32 lanes)
template <typename T>
__device__ __forceinline__ void max_abs_to(unsigned long long* dst, double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > 0.0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

// ------------------------------------------------------------------ registry removed in the bin domain

// Residual BINS: each live registry mode (w, a) of an active signal takes p a e^{2 pi i w_n / N}
// off bin (w . u) mod p of set n (p a off set 0).  That is the transform of the mode's samples
// (sum over x of W^{(alpha - h) x} is p at h = alpha and 0 elsewhere), so f's transform minus
// these is the transform of f - g (Alg. 2, by linearity).  Modes sharing a bin add in any order.
// y += (gx, gy) atomically: one 64-bit vector atomic in float, two in double
__device__ __forceinline__ void peel_add(float* y, float gx, float gy) {
  atomicAdd(reinterpret_cast<float2*>(y), make_float2(gx, gy));
}
__device__ __forceinline__ void peel_add(double* y, double gx, double gy) {
  atomicAdd(y, gx);
  atomicAdd(y + 1, gy);
}

// Registry mode jr of a signal: add(e, gx, gy) receives -p a e^{2 pi i w . s_n} for bin
// e = n p + (w . u) mod p of every set n (pruned modes add nothing).
template <typename T, class Add>
__device__ __forceinline__ void peel_entry(const SigCfg& c, const SigRun& r, int jr, const int64_t* u,
                                           const int32_t* __restrict__ regw, const double2* __restrict__ rega,
                                           const c2<T>* __restrict__ regtw, Add add) {
  const double2 a = rega[c.rega_off + jr];
  if (a.x == 0.0 && a.y == 0.0) return;   // pruned
  const int64_t p = r.p;
  const int64_t h = (int64_t)project_mod(regw + c.regw_off + (int64_t)jr * c.d, c.d, u, c.box_lo, p, r.mod_m,
                                         r.proj_off, r.mod32);
  // -p a, then -p a e^{2 pi i w . s_n} for n >= 1, in T (float policy: the double pipe is narrow)
  const T px = (T)(-(double)p * a.x), py = (T)(-(double)p * a.y);
  add(h, px, py);
  const c2<T>* tw = regtw + c.regtw_off + (int64_t)jr * (c.n_sets - 1);
  for (int nn = 1; nn < c.n_sets; ++nn) {
    const c2<T> t = tw[nn - 1];
    add((int64_t)nn * p + h, px * t.x - py * t.y, px * t.y + py * t.x);
  }
}

// ------------------------------------------------------------------ classification and registry merge

__device__ __forceinline__ unsigned long long hash_key(const int32_t* w, int d) {
  unsigned long long h = 0x9E3779B97F4A7C15ull ^ (unsigned long long)d;
  for (int l = 0; l < d; ++l) {
    h ^= (unsigned long long)(uint32_t)w[l];
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 32;
  }
  h ^= h >> 29;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 32;
  return h;
}

// Arg(Y_n / Y_0) in [-pi, pi) read as N Arg / (2 pi); false when farther than delta from an integer.
template <typename R>
__device__ __forceinline__ bool read_coord(R ynx, R yny, R y0x, R y0y, int64_t N, int box_lo, R delta,
                                           int64_t* w_out) {
  const R re = ynx * y0x + yny * y0y;   // Y_n conj(Y_0)
  const R im = yny * y0x - ynx * y0y;
  const R pi = (R)3.14159265358979323846;
  R phi = atan2(im, re);
  if (phi >= pi) phi -= (R)2 * pi;
  const R v = (R)N * phi / ((R)2 * pi);
  const R rr = rint(v);
  if (!(fabs(v - rr) <= delta)) return false;
  // |rr| <= N / 2 and -N <= box_lo <= 0, so rr - box_lo lies in [-N/2, 3N/2]: one wrap
  int64_t wn = (int64_t)rr - box_lo;
  if (wn < 0) wn += N;
  else if (wn >= N) wn -= N;
  *w_out = wn + box_lo;
  return true;
}

// ---- the float engine's double read-out and coefficient roots without double transcendentals
// (GB300's FP64 pipe runs at 1/64 of the FP32 rate, and a double atan2 or sincospi costs tens of
// its operations).  Both reduce the angle against a table of e^{2 pi i j / 1024} in double:
// what is left is below about pi / 1024, where short series are exact to double rounding.

// Arg(z) / (2 pi) for z = re + i im != 0, given af, a float estimate of Arg(z) (within about
// 1e-3 of it, any multiple of 2 pi apart): k = af's nearest 1024th of a turn in [-512, 512),
// z e^{-2 pi i k / 1024} has the angle a = atan(t), t = Im / Re, |t| < 4e-3, whose series stops at
// t^7 (t^9 / 9 < 1e-22); the quotient through a float reciprocal and one Newton step (relative
// error about 2^-46; a double division where Re is outside float's range).  Turns in
// [-1/2 - 1e-3, 1/2 + 1e-3].
__device__ __forceinline__ double arg_turns_fx(const double2* __restrict__ root1k, double re, double im, float af) {
  int k = __float2int_rn(af * (float)(512.0 / 3.14159265358979323846)) & 1023;
  if (k >= 512) k -= 1024;
  const double2 w = root1k[k & 1023];
  const double re2 = re * w.x + im * w.y;   // z conj(w)
  const double im2 = im * w.x - re * w.y;
  double y;
  if (fabs(re2) > 1e-30 && fabs(re2) < 1e30) {
    y = (double)__frcp_rn((float)re2);
    y = y * (2.0 - re2 * y);
  } else {
    y = 1.0 / re2;
  }
  const double t = im2 * y;
  const double t2 = t * t;
  const double a = t * (1.0 + t2 * (-1.0 / 3.0 + t2 * (1.0 / 5.0 + t2 * (-1.0 / 7.0))));
  return (double)k * (1.0 / 1024.0) + a * (0.5 / 3.14159265358979323846);
}

// read_coord for float transforms with the read-out in double (the ratio Y_n conj(Y_0) is formed
// from exact double products of the floats, its angle by arg_turns_fx)
__device__ __forceinline__ bool read_coord_fx(const double2* __restrict__ root1k, float ynx, float yny, float y0x,
                                              float y0y, int64_t N, int box_lo, double delta, int64_t* w_out) {
  const double re = (double)ynx * (double)y0x + (double)yny * (double)y0y;   // Y_n conj(Y_0)
  const double im = (double)yny * (double)y0x - (double)ynx * (double)y0y;
  const float af = atan2f(yny, ynx) - atan2f(y0y, y0x);
  const double v = (double)N * arg_turns_fx(root1k, re, im, af);
  const double rr = rint(v);
  if (!(fabs(v - rr) <= delta)) return false;
  // |rr| <= N / 2 + 1 and -N <= box_lo <= 0: one wrap
  int64_t wn = (int64_t)rr - box_lo;
  if (wn < 0) wn += N;
  else if (wn >= N) wn -= N;
  *w_out = wn + box_lo;
  return true;
}

// e^{2 pi i m / q} in double (0 <= m < q < 2^31, inv_q = 1 / q in double, sc = 1024 / q in
// float): j = the nearest 1024th of a turn (within one), then the angle left,
// e = 2 pi (1024 m - j q) / (1024 q), |e| < 0.01, by the Taylor series of cos and sin to e^6 / e^7
// (the next terms are below 1e-20).
__device__ __forceinline__ double2 unit_root_fx(const double2* __restrict__ root1k, int64_t m, int64_t q,
                                                double inv_q, float sc) {
  const int64_t j = (int64_t)__float2int_rn((float)m * sc);
  const double e = (double)(1024 * m - j * q) * (inv_q * (3.14159265358979323846 / 512.0));
  const double e2 = e * e;
  const double cs = 1.0 + e2 * (-1.0 / 2.0 + e2 * (1.0 / 24.0 + e2 * (-1.0 / 720.0)));
  const double sn = e * (1.0 + e2 * (-1.0 / 6.0 + e2 * (1.0 / 120.0 + e2 * (-1.0 / 5040.0))));
  const double2 w = root1k[j & 1023];
  return make_double2(w.x * cs - w.y * sn, w.x * sn + w.y * cs);
}

// Block form: Arg(Y_n / Y_0) read as the block's unwrapped frequency w~ = 2 N^{d1} Arg / (2 pi),
// taken in the window [W_lo, W_lo + N^{d1}) of the box's unwrapped values (W_lo that of
// (box_lo, ..., box_lo)) and split into its d1 base-N digits, lowest first; false when farther
// than delta from an integer or outside the window.
template <typename R>
__device__ __forceinline__ bool read_block(R ynx, R yny, R y0x, R y0y, int64_t N, int size, int box_lo, R delta,
                                           int32_t* digits) {
  const R re = ynx * y0x + yny * y0y;
  const R im = yny * y0x - ynx * y0y;
  const R pi = (R)3.14159265358979323846;
  R phi = atan2(im, re);
  if (phi >= pi) phi -= (R)2 * pi;
  int64_t span = 1, ones = 0;   // N^{d1} and 1 + N + ... + N^{d1-1}
  for (int r = 0; r < size; ++r) {
    ones += span;
    span *= N;
  }
  const int64_t q = 2 * span;
  const R v = (R)q * phi / ((R)2 * pi);
  const R rr = rint(v);
  if (!(fabs(v - rr) <= delta)) return false;
  int64_t t = ((int64_t)rr - (int64_t)box_lo * ones) % q;
  if (t < 0) t += q;
  if (t >= span) return false;
  for (int r = 0; r < size; ++r) {
    digits[r] = (int32_t)(t % N) + box_lo;
    t /= N;
  }
  return true;
}

// Tilted form (Alg. 3, d = 2): sets 1 and 2 read the rotated coordinates w~_n =
// Q Arg(Y_n / Y_0) / (2 pi), Q = (base + height) N, each in the window of the box's values
// (lowest: base lo - height (lo + N - 1), then (base + height) lo); the pair is turned back by
// [cos sin; -sin cos] times hypo, which gives hypo^2 w (the rotated frequencies carry the factor
// hypo, Eq. 27).  False when a phase is farther than delta from an integer, the turned pair is
// not a multiple of hypo^2, or w leaves the box.
template <typename R>
__device__ __forceinline__ bool read_tilt(const SigCfg& c, R y1x, R y1y, R y2x, R y2y, R y0x, R y0y, int32_t* w) {
  const int64_t b = c.tilt_base, h = c.tilt_height, hy = c.tilt_hypo;
  const int64_t N = c.N, lo = c.box_lo;
  const int64_t q = (b + h) * N;
  const R pi = (R)3.14159265358979323846;
  int64_t wt[2];
#pragma unroll
  for (int n = 0; n < 2; ++n) {
    const R ynx = n == 0 ? y1x : y2x, yny = n == 0 ? y1y : y2y;
    const R re = ynx * y0x + yny * y0y;   // Y_n conj(Y_0)
    const R im = yny * y0x - ynx * y0y;
    R phi = atan2(im, re);
    if (phi >= pi) phi -= (R)2 * pi;
    const R v = (R)q * phi / ((R)2 * pi);
    const R rr = rint(v);
    if (!(fabs(v - rr) <= (R)c.delta)) return false;
    const int64_t wlo = n == 0 ? b * lo - h * (lo + N - 1) : (b + h) * lo;
    int64_t t = ((int64_t)rr - wlo) % q;
    if (t < 0) t += q;
    wt[n] = wlo + t;
  }
  const int64_t c2 = hy * hy;
  const int64_t x1 = b * wt[0] + h * wt[1], x2 = b * wt[1] - h * wt[0];
  if (x1 % c2 != 0 || x2 % c2 != 0) return false;
  const int64_t w1 = x1 / c2, w2 = x2 / c2;
  if (w1 < lo || w1 >= lo + N || w2 < lo || w2 >= lo + N) return false;
  w[0] = (int32_t)w1;
  w[1] = (int32_t)w2;
  return true;
}

// Read-out of shifted set n (1-based) of an occupied bin: the coordinate it fixes (coordinate
// form) or the d1 coordinates of block n (block form) go to w (if not null), and their
// (w_l - box_lo) u_l are added to *bin mod p.
// FX: the transforms are float and the read-out double (read_coord_fx).
template <typename R, bool FX = false>
__device__ __forceinline__ bool read_set(const SigCfg& c, const SigRun& r, const int32_t* __restrict__ blk, int n,
                                         R ynx, R yny, R y0x, R y0y, const int64_t* u, uint64_t* bin, int32_t* w) {
  const uint64_t up = (uint64_t)r.p;
  if (!c.shift_block) {
    int64_t wn;
    if constexpr (FX) {
      if (!read_coord_fx(c.root1k, (float)ynx, (float)yny, (float)y0x, (float)y0y, c.N, c.box_lo, c.delta, &wn))
        return false;
    } else {
      if (!read_coord<R>(ynx, yny, y0x, y0y, c.N, c.box_lo, (R)c.delta, &wn)) return false;
    }
    if (w) w[n - 1] = (int32_t)wn;
    *bin = mod_barrett((uint64_t)(wn - c.box_lo) * (uint64_t)u[n - 1] + *bin, up, r.mod_m);
    return true;
  }
  const int b = blk[2 * (n - 1)], size = blk[2 * (n - 1) + 1];
  int32_t dg[32];
  if (size > 32 || !read_block<R>(ynx, yny, y0x, y0y, c.N, size, c.box_lo, (R)c.delta, dg)) return false;
  for (int t = 0; t < size; ++t) {
    if (w) w[b + t] = dg[t];
    *bin = mod_barrett((uint64_t)(dg[t] - c.box_lo) * (uint64_t)u[b + t] + *bin, up, r.mod_m);
  }
  return true;
}

struct ClassifyOut {   // step calls: accepted bins are appended here instead of merged
  int32_t* h;
  int32_t* w;
  double2* a;
  int cap;
  int* count;
  int* err;
  double eta_override;
};

// The tilted form's ratio test (Eq. 42) and read-out of an occupied bin: both sets, then
// read_tilt; *bin gets sum_l (w_l - box_lo) u_l mod p.
template <typename T, typename R>
__device__ __forceinline__ bool decode_tilt(const SigCfg& c, const SigRun& r, const c2<T>* Y, const int64_t* u,
                                            int64_t h, R y0x, R y0y, R m0, int32_t* w_out, uint64_t* bin) {
  const uint64_t up = (uint64_t)r.p;
  const c2<T> y1 = Y[r.p + h], y2 = Y[2 * r.p + h];
  const R y1x = (R)y1.x, y1y = (R)y1.y, y2x = (R)y2.x, y2y = (R)y2.y;
  if (!(fabs(sqrt(y1x * y1x + y1y * y1y) / m0 - (R)1) < (R)c.tau)) return false;   // Eq. 42
  if (!(fabs(sqrt(y2x * y2x + y2y * y2y) / m0 - (R)1) < (R)c.tau)) return false;
  int32_t wt[2];
  if (!read_tilt<R>(c, y1x, y1y, y2x, y2y, y0x, y0y, wt)) return false;
  if (w_out) {
    w_out[0] = wt[0];
    w_out[1] = wt[1];
  }
  uint64_t b = mod_barrett((uint64_t)(wt[0] - c.box_lo) * (uint64_t)u[0], up, r.mod_m);
  *bin = mod_barrett((uint64_t)(wt[1] - c.box_lo) * (uint64_t)u[1] + b, up, r.mod_m);
  return true;
}

// Eq. 42 ratio test and Eq. 7 read-out of sets 1..d of an occupied bin (the tilted form:
// decode_tilt).  The sets' values are fetched eight at a time so that their loads
// overlap.  Writes w_n to w_out (if not null) and returns whether every set passes and
// (w . u) mod p is the bin itself.
template <typename T, typename R>
__device__ bool decode_bin(const SigCfg& c, const SigRun& r, const int32_t* __restrict__ blk, const c2<T>* Y,
                           const int64_t* u, int64_t h, R y0x, R y0y, R m0, int32_t* w_out) {
  constexpr int kB = 8;
  constexpr bool FX = sizeof(T) == 4 && sizeof(R) == 8;   // float transforms, double read-out
  const int64_t p = r.p;
  const uint64_t up = (uint64_t)p;
  const int S = c.n_sets - 1;
  uint64_t bin = 0;
  if (c.shift_tilt) {
    if (!decode_tilt<T, R>(c, r, Y, u, h, y0x, y0y, m0, w_out, &bin)) return false;
  }
  for (int n0 = 1; n0 <= S && !c.shift_tilt; n0 += kB) {
    c2<T> yv[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) yv[i] = n0 + i <= S ? Y[(int64_t)(n0 + i) * p + h] : mk2((T)0, (T)0);
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const int n = n0 + i;
      if (n > S) break;
      const R ynx = (R)yv[i].x, yny = (R)yv[i].y;
      if constexpr (FX) {   // the magnitudes of float values in float (tau >> float rounding)
        const float mn = sqrtf(yv[i].x * yv[i].x + yv[i].y * yv[i].y);
        if (!(fabsf(mn / (float)m0 - 1.0f) < (float)c.tau)) return false;   // Eq. 42
      } else {
        const R mn = sqrt(ynx * ynx + yny * yny);
        if (!(fabs(mn / m0 - (R)1) < (R)c.tau)) return false;   // Eq. 42
      }
      if (!read_set<R, FX>(c, r, blk, n, ynx, yny, y0x, y0y, u, &bin, w_out)) return false;
    }
  }
  uint64_t usum = 0;
  for (int l = 0; l < c.d; ++l) usum += (uint64_t)u[l];
  const int64_t blm = ((int64_t)c.box_lo % p + p) % p;
  bin = mod_barrett(bin + mod_barrett((uint64_t)blm * mod_barrett(usum, up, r.mod_m), up, r.mod_m), up, r.mod_m);
  return (int64_t)bin == h;
}

// The read-out vector of an accepted bin, computed again (for vectors longer than the
// decoder's register copy).
template <typename T, typename R>
__device__ void read_coords(const SigCfg& c, const SigRun& r, const int32_t* __restrict__ blk, const c2<T>* Y,
                            const int64_t* u, int64_t h, R y0x, R y0y, int32_t* w_out) {
  if (c.shift_tilt) {
    const c2<T> y1 = Y[r.p + h], y2 = Y[2 * r.p + h];
    read_tilt<R>(c, (R)y1.x, (R)y1.y, (R)y2.x, (R)y2.y, y0x, y0y, w_out);
    return;
  }
  uint64_t bin = 0;
  for (int n = 1; n < c.n_sets; ++n) {
    const c2<T> yn = Y[(int64_t)n * r.p + h];
    read_set<R, sizeof(T) == 4 && sizeof(R) == 8>(c, r, blk, n, (R)yn.x, (R)yn.y, y0x, y0y, u, &bin, w_out);
  }
}

// Coefficient estimate of an accepted bin with read-out vector w (Eq. 41).  With coef_mean
// the estimate is the mean over the sets of Y_n[h] e^{-2 pi i w . s_n} / p: for a bin
// holding one mode every term equals a exactly, and the mean averages the sets' independent
// rounding (and the leakage of other modes' residuals, whose phases differ across the sets).
template <typename T, typename R>
__device__ double2 coefficient(const SigCfg& c, const SigRun& r, const int32_t* __restrict__ blk, const c2<T>* Y,
                               int64_t h, R y0x, R y0y, const int32_t* w, const c2<T>* tn) {
  if (!c.coef_mean) {
    if (sizeof(R) == 4) {
      const float scale = 1.0f / (float)r.p;
      return make_double2((double)((float)y0x * scale), (double)((float)y0y * scale));
    }
    const double scale = 1.0 / (double)r.p;
    return make_double2((double)y0x * scale, (double)y0y * scale);
  }
  R ax = y0x, ay = y0y;
  // float transforms, double estimate, coordinate form: the roots from the table (unit_root_fx)
  constexpr bool FX = sizeof(T) == 4 && sizeof(R) == 8;
  const bool fx = FX && !c.shift_block && !c.shift_tilt && c.N < (1LL << 31);
  const double inv_N = fx ? 1.0 / (double)c.N : 0.0;
  const float sc_N = fx ? 1024.0f / (float)c.N : 0.0f;
  for (int n = 1; n < c.n_sets; ++n) {
    const c2<T> yn = Y[(int64_t)n * r.p + h];
    c2<R> t;   // e^{2 pi i w . s_n}
    if (sizeof(R) == sizeof(T) && tn != nullptr) {
      t = mk2((R)tn[n - 1].x, (R)tn[n - 1].y);
    } else if (FX && fx) {
      const int64_t m = w[n - 1] < 0 ? (int64_t)w[n - 1] + c.N : (int64_t)w[n - 1];   // w in the box
      const double2 q = unit_root_fx(c.root1k, m, c.N, inv_N, sc_N);
      t = mk2((R)q.x, (R)q.y);
    } else {
      t = shift_root<R>(c, blk, w, n, true);
    }
    ax += (R)yn.x * t.x + (R)yn.y * t.y;     // Y_n conj(t)
    ay += (R)yn.y * t.x - (R)yn.x * t.y;
  }
  if (sizeof(R) == 4) {   // float read-out: scale in float (the double pipe of this GPU is narrow)
    const float scale = 1.0f / ((float)r.p * (float)c.n_sets);
    return make_double2((double)((float)ax * scale), (double)((float)ay * scale));
  }
  const double scale = 1.0 / ((double)r.p * (double)c.n_sets);
  return make_double2((double)ax * scale, (double)ay * scale);
}

// *ctr += v from every active lane, one atomic per group of lanes that share key (a signal)
__device__ __forceinline__ void warp_add(int* ctr, int v, int key) {
  const unsigned grp = __match_any_sync(__activemask(), key);
  const int leader = __ffs(grp) - 1;
  int sum = 0;
  for (unsigned m = grp; m; m &= m - 1) sum += __shfl_sync(grp, v, __ffs(m) - 1);
  if ((threadIdx.x & 31) == leader) atomicAdd(ctr, sum);
}

// Ratio test, read-out, own-bin check and registry merge of one occupied bin h of signal s
// (Eq. 41-42, Alg. 2 registry update); Y holds the signal's d + 1 transforms (global memory or
// the fused kernel's shared copy).
template <typename T>
__device__ void classify_candidate(const SigCfg& c, SigRun* rp, int s, int64_t h, const c2<T>* Y,
                                   const int64_t* __restrict__ ubuf, const int32_t* __restrict__ shblk,
                                   int32_t* regw, double2* rega, c2<T>* regtw, int32_t* hash, const ClassifyOut& co) {
  const SigRun& r = *rp;
  const c2<T> y0 = Y[h];
  const int64_t* u = ubuf + c.u_off;
  const int32_t* blk = shblk + c.blk_off;
  const int dd = c.d;
  const int S = c.n_sets - 1;   // shifted sets: twiddles per set
  int32_t wk[64];
  int32_t* wreg = dd <= 64 ? wk : nullptr;   // decoded vector kept for the read-out
  bool ok;
  if (c.ratio64) {
    const double m0d = sizeof(T) == 4 ? (double)sqrtf((float)(y0.x * y0.x + y0.y * y0.y))
                                      : sqrt((double)y0.x * (double)y0.x + (double)y0.y * (double)y0.y);
    ok = decode_bin<T, double>(c, r, blk, Y, u, h, (double)y0.x, (double)y0.y, m0d, wreg);
  } else {
    ok = decode_bin<T, T>(c, r, blk, Y, u, h, y0.x, y0.y, sqrt(y0.x * y0.x + y0.y * y0.y), wreg);
  }
  if (!ok) return;
  warp_add(&rp->n_acc, 1, s);
  if (co.count != nullptr) {
    const int idx = atomicAdd(co.count, 1);
    if (idx >= co.cap) {
      atomicOr(co.err, 1);
      return;
    }
    co.h[idx] = (int32_t)h;
    int32_t* wo = co.w + (int64_t)idx * dd;
    if (wreg) {
      for (int l = 0; l < dd; ++l) wo[l] = wk[l];
    } else if (c.ratio64) {
      read_coords<T, double>(c, r, blk, Y, u, h, (double)y0.x, (double)y0.y, wo);
    } else {
      read_coords<T, T>(c, r, blk, Y, u, h, (T)y0.x, (T)y0.y, wo);
    }
    if (c.ratio64) co.a[idx] = coefficient<T, double>(c, r, blk, Y, h, (double)y0.x, (double)y0.y, wo, nullptr);
    else co.a[idx] = coefficient<T, T>(c, r, blk, Y, h, (T)y0.x, (T)y0.y, wo, nullptr);
    return;
  }
  // ---- merge into the registry: keys accepted in one round are distinct (each lands in its
  // own bin) and the table never deletes, so a key is present iff met before the first
  // empty slot of its probe sequence; one writer per key per round.
  int32_t* rw = regw + c.regw_off;
  double2* ra = rega + c.rega_off;
  c2<T>* rt = regtw + c.regtw_off;
  int32_t* hs = hash + c.hash_off;
  const double eta_prune2 = r.eta_prune * r.eta_prune;
  // decoded vector: up to 64 coordinates in registers, else read back from the registry slot
  int32_t* wv = wk;
  int scratch_idx = -1;
  if (dd > 64) {
    scratch_idx = atomicAdd(&rp->K_reg, 1);
    if (scratch_idx >= c.reg_cap) {
      atomicOr(&rp->err, 1);
      return;
    }
    wv = rw + (int64_t)scratch_idx * dd;
  }
  if (!wreg) {
    if (c.ratio64) read_coords<T, double>(c, r, blk, Y, u, h, (double)y0.x, (double)y0.y, wv);
    else read_coords<T, T>(c, r, blk, Y, u, h, (T)y0.x, (T)y0.y, wv);
  }
  // e^{2 pi i w . s_n} of the decoded vector: the registry keeps them (and the float read-out
  // uses them) so they are formed once
  c2<T> tn[64];
  const bool keep_tn = S <= 64;
  if (keep_tn) {
    for (int n = 1; n <= S; ++n) tn[n - 1] = shift_root<T>(c, blk, wv, n, true);
  }
  double2 a;
  if (c.ratio64) a = coefficient<T, double>(c, r, blk, Y, h, (double)y0.x, (double)y0.y, wv, nullptr);
  else a = coefficient<T, T>(c, r, blk, Y, h, (T)y0.x, (T)y0.y, wv, keep_tn ? tn : nullptr);
  int slot = (int)(hash_key(wv, dd) & (unsigned long long)c.hash_mask);
  int mine = scratch_idx;
  bool placed = false, merged = false, past_empty = false;
  for (int probe = 0; probe <= c.hash_mask; ++probe, slot = (slot + 1) & c.hash_mask) {
    int cur = __ldcg(&hs[slot]);   // a stale -1 only makes the CAS below fail
    if (cur < 0) {
      past_empty = true;   // the key is not in the table
      if (mine < 0) {
        mine = atomicAdd(&rp->K_reg, 1);
        if (mine >= c.reg_cap) {
          atomicOr(&rp->err, 1);
          break;
        }
        for (int l = 0; l < dd; ++l) rw[(int64_t)mine * dd + l] = wv[l];
      }
      ra[mine] = a;
      for (int n = 1; n <= S; ++n)
        rt[(int64_t)mine * S + n - 1] = keep_tn ? tn[n - 1] : shift_root<T>(c, blk, wv, n, true);
      // no fence: nobody reads this entry before the next kernel (see the probe rule below)
      cur = atomicCAS(&hs[slot], -1, mine);
      if (cur < 0) {
        placed = true;
        break;
      }
      continue;   // slot taken by another new key of this round
    }
    // keys accepted in one round are distinct (each decodes in its own bin), so a slot claimed
    // this round (index from the round's start on, or any slot beyond an empty one) holds
    // another key: only keys of earlier rounds, complete since the last kernel, are compared
    if (past_empty || cur >= r.reg_start) continue;
    const int32_t* ow = rw + (int64_t)cur * dd;
    bool same = true;
    for (int l = 0; l < dd && same; ++l) same = (ow[l] == wv[l]);
    if (same) {
      const double2 old = ra[cur];
      double2 nw = make_double2(old.x + a.x, old.y + a.y);   // duplicate key: a_R += a
      const bool was_live = (old.x != 0.0 || old.y != 0.0);
      const bool live = nw.x * nw.x + nw.y * nw.y >= eta_prune2;   // prune small coefficients
      if (!live) nw = make_double2(0.0, 0.0);
      ra[cur] = nw;
      if (was_live && !live) atomicSub(&rp->n_live, 1);
      if (!was_live && live) atomicAdd(&rp->n_live, 1);
      merged = true;
      break;
    }
  }
  if (merged && scratch_idx >= 0) {
    // the slot that held the decoded vector stays a zero mode
    ra[scratch_idx] = make_double2(0.0, 0.0);
    for (int l = 0; l < S; ++l) rt[(int64_t)scratch_idx * S + l] = mk2((T)0, (T)0);
  }
  if (placed) warp_add(&rp->n_live, 1, s);
  else if (!merged && mine >= 0 && mine < c.reg_cap) atomicOr(&rp->err, 2);   // table full
}

}  // namespace sfft
