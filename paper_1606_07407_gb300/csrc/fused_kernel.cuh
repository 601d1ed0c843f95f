// Fused short-round kernel (see fused.cuh).  Each launch runs one round of Algorithm 2 for
// every signal whose plan marks it fused, one block of kSampleThreads threads per signal, with
// the round's data in shared memory:
//
//   tables      W[m] = e^{2 pi i m / p} and chirp[m] = e^{-pi i m^2 / p} (table_entry)
//   samples     y_n[x] = sum_j C[n][j] W[(alpha_j x) mod p] for every set n (Eq. 41), thread
//               x of the half line taking x and p - x (their exponentials are conjugate), the
//               modes staged kFusedChunk at a time (mode_source) and split over mode groups of
//               threads when the half line is short, summed in blocks of 32; written times the
//               chirp into the rows
//   DFT         Bluestein (Eq. 3) of the n_sets rows and the filter at once, one row per
//               fft_threads(L) threads (radix-16 passes where they fit), out into Y_n
//   residual    when the registry is removed in the bin domain: every entry's bin and its set-0
//               term first; after the empty-bin test, the other sets' terms at the occupied bins
//               only (or the whole peel, peel_entry's, for a registry beyond the shared list)
//   classify    empty-bin test, then the ratio test, read-out and registry merge of every
//               occupied bin (classify_candidate)
//   plan        the next round (plan_signal): the next launch runs it while it stays short,
//               else the batched kernels plan it again the same way
//
// Shared memory (offsets from fused_layout at the allocation's length): the tables (2p), the
// n_sets + 1 rows of the DFT (padded; afterwards the candidate list, occupied-bin flags and the
// entries' bins), and a work area that holds in turn a chunk of modes, the groups' partial sums
// and the transforms Y_n.  The registry's probe rule (entries of earlier rounds are complete)
// holds as in the batched path, since each round is a launch of its own.
//
// Included by the translation units that instantiate the kernel, one set count each (they
// compile in parallel).
#pragma once

#include "fused.cuh"
#include "noise.cuh"
#include "sample_tile.cuh"

namespace sfft {

namespace {

// Samples of every set into the DFT rows: slot n + 1 gets chirp[x] y_n[x] at x < p.
template <int NS>
__device__ __forceinline__ void fused_sample(const FusedArgs& a, const SigCfg& c, const SigRun& r, int s,
                                             const int64_t* u_s, const float2* tab_s, float2* slots, int ls,
                                             unsigned char* work) {
  using C2 = float2;
  const int tid = threadIdx.x;
  const int p = (int)r.p;
  const int H = p / 2 + 1;                        // positions of the half line (<= 256)
  // mode groups: thread (g, x) = (tid / H, tid mod H); positions x < extra have G + 1 groups, the
  // others G, so that every thread of the block has work
  const int G = max(1, (int)blockDim.x / H);
  const int extra = (int)blockDim.x - G * H;
  const int g = tid / H, x = tid - g * H;
  const int Gx = G + (x < extra ? 1 : 0);          // this position's groups
  const bool on = g < Gx;
  const int Gmax = G + (extra > 0 ? 1 : 0);
  const float inv_p = 1.0f / (float)p;
  const int32_t* sw = a.sig_w[s];   // the black box's modes
  const double2* sa = a.sig_a[s];
  int* m_al = reinterpret_cast<int*>(work);
  C2* m_C = reinterpret_cast<C2*>(work + kFusedChunk * sizeof(int));
  // each chunk's sums go to fresh accumulators that are then added to the running totals
  // (blocked summation, as in the batched kernel): with many modes a single float sum per
  // sample would carry the rounding of all K terms
  float acc[NS][4], tot[NS][4];
#pragma unroll
  for (int n = 0; n < NS; ++n) tot[n][0] = tot[n][1] = tot[n][2] = tot[n][3] = 0.0f;
  const int K = sampled_modes(c, r);
  for (int j0 = 0; j0 < K; j0 += kFusedChunk) {
    const int cnt = min(kFusedChunk, K - j0);
    if (j0 > 0) __syncthreads();   // every thread is done with the previous chunk
#pragma unroll 2
    for (int jj = tid; jj < cnt; jj += blockDim.x) {
      C2 a0;
      const C2* twr;
      const int32_t* w = mode_source<float>(c, r, j0 + jj, sw, sa, a.tw, a.regw, a.rega, a.regtw, &a0, &twr);
      C2 t[NS > 1 ? NS - 1 : 1];   // loaded with w, before the projection's chain
#pragma unroll
      for (int n = 1; n < NS; ++n) t[n - 1] = twr[n - 1];
      m_al[jj] = (int)project_mod(w, c.d, u_s, c.box_lo, r.p, r.mod_m, r.proj_off, r.mod32);
      m_C[jj * NS] = a0;
#pragma unroll
      for (int n = 1; n < NS; ++n) m_C[jj * NS + n] = cmul(a0, t[n - 1]);
    }
    __syncthreads();
    // blocks of 32 of the thread's modes (every Gx-th of the chunk)
    for (int j1 = g; j1 < cnt; j1 += 32 * Gx) {
#pragma unroll
      for (int n = 0; n < NS; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.0f;
      if (on) {
        const int j_end = min(cnt, j1 + 32 * Gx);
        // unrolled so that several modes' index chains (load, product, reduction, table load) overlap
#pragma unroll 4
        for (int jj = j1; jj < j_end; jj += Gx) {
          const C2 E = tab_s[mod_small((unsigned)m_al[jj] * (unsigned)x, p, inv_p)];
          auto term = [&](int n, float cr, float ci) {
            acc[n][0] = fmaf(cr, E.x, acc[n][0]);   // P1: c_r e_r
            acc[n][1] = fmaf(ci, E.y, acc[n][1]);   // P2: c_i e_i
            acc[n][2] = fmaf(cr, E.y, acc[n][2]);   // P3: c_r e_i
            acc[n][3] = fmaf(ci, E.x, acc[n][3]);   // P4: c_i e_r
          };
          if constexpr (NS % 2 == 0) {
            // two sets' coefficients per 16-byte load (jj NS is even, so the pair is aligned)
            const float4* c4 = reinterpret_cast<const float4*>(m_C + jj * NS);
#pragma unroll
            for (int n = 0; n < NS; n += 2) {
              const float4 cc = c4[n / 2];
              term(n, cc.x, cc.y);
              term(n + 1, cc.z, cc.w);
            }
          } else {
#pragma unroll
            for (int n = 0; n < NS; ++n) {
              const C2 cc = m_C[jj * NS + n];
              term(n, cc.x, cc.y);
            }
          }
        }
      }
#pragma unroll
      for (int n = 0; n < NS; ++n)
#pragma unroll
        for (int k = 0; k < 4; ++k) tot[n][k] += acc[n][k];
    }
  }
  if (Gmax > 1) {
    // groups 1..Gx-1 hand their sums to group 0 through the work area
    float* red = reinterpret_cast<float*>(work);
    __syncthreads();   // the last chunk is consumed
    if (on && g > 0) {
#pragma unroll
      for (int n = 0; n < NS; ++n)
#pragma unroll
        for (int k = 0; k < 4; ++k) red[(((g - 1) * H + x) * NS + n) * 4 + k] = tot[n][k];
    }
    __syncthreads();
    if (g == 0) {
      for (int gg = 1; gg < Gx; ++gg)
#pragma unroll
        for (int n = 0; n < NS; ++n)
#pragma unroll
          for (int k = 0; k < 4; ++k) tot[n][k] += red[(((gg - 1) * H + x) * NS + n) * 4 + k];
    }
  }
  if (g == 0) {
    const C2* chirp = tab_s + p;
    const bool mirror = x >= 1 && p - x >= H;   // p - x is a distinct sample of the other half
    const bool noisy = r.noise_sigma > 0.0;
#pragma unroll
    for (int n = 0; n < NS; ++n) {
      const float P1 = tot[n][0], P2 = tot[n][1], P3 = tot[n][2], P4 = tot[n][3];
      C2* rb = slots + (n + 1) * ls;
      C2 y = mk2(P1 - P2, P3 + P4);
      if (noisy) y = cadd(y, black_box_noise<float>(r.noise_seed, r.round, n, x, r.noise_sigma));
      rb[fpad(x)] = cmul(chirp[x], y);
      if (mirror) {
        C2 ym = mk2(P1 + P2, P4 - P3);
        if (noisy) ym = cadd(ym, black_box_noise<float>(r.noise_seed, r.round, n, p - x, r.noise_sigma));
        rb[fpad(p - x)] = cmul(chirp[p - x], ym);
      }
    }
  }
}

// Bluestein DFT (Eq. 3) of the rows in the slots, all at once: the forward transforms of slot
// 0 (the filter) and slots 1..n_sets (the rows, times the chirp), the products with the
// filter's spectrum, the inverse transforms, and Y_n[h] = chirp[h] (...)[h] / L into Ys.  The
// largest |Y_0| goes to *maxy0 (the first round's A_ref).  A function of its own, called once:
// the compiler keeps the unrolled passes in registers only where they are neither in a loop
// nor at several call sites.
// E bounds the values a thread holds per pass: 16 (shorter register chains, more passes) where
// the rows and the filter still fit the block at fft_threads<16>(L) threads each, else 32.
template <int E>
__device__ __noinline__ void fused_convolve(const SigCfg& c, const SigRun& r, const float2* tab_s, float2* slots,
                                            int ls, float2* tw_hi, float2* tw_lo, float2* Ys,
                                            unsigned long long* maxy0) {
  using C2 = float2;
  const int p = (int)r.p;
  const int L = r.L;
  const int nthr = fft_threads<C2, E>(L);
  const int slot = threadIdx.x / nthr, lt = threadIdx.x - slot * nthr;
  const int row = slot - 1;
  const bool data = slot >= 1 && row < c.n_sets;
  const bool act = slot == 0 || data;
  C2* rb = slots + slot * ls;
  fft_row<C2, false, E>(rb, L, tw_hi, tw_lo, lt, nthr, act);
  // the inverse as conj(FFT(conj(.))): one direction's code in the kernel
  if (data)
    for (int k = lt; k < L; k += nthr) rb[fpad(k)] = cconj(cmul(rb[fpad(k)], slots[fpad(k)]));
  __syncthreads();
  fft_row<C2, false, E>(rb, L, tw_hi, tw_lo, lt, nthr, data);
  float m2 = 0.0f;   // largest |Y_0|^2 seen by this thread
  if (data) {
    const C2* chirp = tab_s + p;
    const float invL = 1.0f / (float)L;
    for (int h = lt; h < p; h += nthr) {
      const C2 v = cmul(chirp[h], cscale(cconj(rb[fpad(h)]), invL));
      Ys[row * p + h] = v;
      m2 = fmaxf(m2, v.x * v.x + v.y * v.y);
    }
  }
  // row 0 is slot 1: whole warps, as nthr is a multiple of 32
  if (slot == 1) max_abs_to<float>(maxy0, sqrt((double)m2));
}

// The registry of the round's start off its bins of Ys (residual in the bin domain, as
// peel_entry): -p a e^{2 pi i w . s_n} to bin (w . u) mod p of set n.  Each thread takes four
// entries at a time and loads all of them before its shared-memory atomics, so that the loads
// overlap; the products are formed in float (the double pipe of this GPU is narrow).
template <int NS>
__device__ __forceinline__ void fused_peel(const SigCfg& c, const SigRun& r, float2* Ys, const int64_t* u,
                                           const int32_t* regw, const double2* rega, const float2* regtw) {
  constexpr int U = 4;
  constexpr int S = NS - 1 > 0 ? NS - 1 : 1;
  const int nr = min(r.K_reg, c.reg_cap);
  const int p = (int)r.p;
  const float pf = (float)p;
  float* Yt = reinterpret_cast<float*>(Ys);
  const int32_t* rw = regw + c.regw_off;
  const double2* ra = rega + c.rega_off;
  const float2* rt = regtw + c.regtw_off;
  for (int j0 = threadIdx.x; j0 < nr; j0 += U * blockDim.x) {
    double2 av[U];
    float2 tv[U][S];
    int h[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int jr = j0 + q * blockDim.x;
      av[q] = jr < nr ? ra[jr] : make_double2(0.0, 0.0);
#pragma unroll
      for (int n = 0; n < NS - 1; ++n) tv[q][n] = jr < nr ? rt[(int64_t)jr * (NS - 1) + n] : make_float2(0.f, 0.f);
      h[q] = jr < nr ? (int)project_mod(rw + (int64_t)jr * c.d, c.d, u, c.box_lo, r.p, r.mod_m, r.proj_off, r.mod32) : -1;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (h[q] < 0 || (av[q].x == 0.0 && av[q].y == 0.0)) continue;   // past the end, or pruned
      const float px = -pf * (float)av[q].x, py = -pf * (float)av[q].y;
      atomicAdd(Yt + 2 * h[q], px);
      atomicAdd(Yt + 2 * h[q] + 1, py);
#pragma unroll
      for (int n = 1; n < NS; ++n) {
        const float2 t = tv[q][n - 1];
        const int e = n * p + h[q];
        atomicAdd(Yt + 2 * e, px * t.x - py * t.y);
        atomicAdd(Yt + 2 * e + 1, px * t.y + py * t.x);
      }
    }
  }
}

// Residual in the bin domain, set 0 only: every registry entry of the round's start gets its
// bin h = (w . u) mod p in hreg (-1 when pruned) and takes -p a off Y_0[h].  The other sets are
// corrected later at the occupied bins only (fused_peel_bins): the candidates come from set 0
// alone, and the ratio test and read-out read the other sets at occupied bins only (a round
// without candidates corrects them at every registry entry's bin to test them for the stop rule).
template <int NS>
__device__ __forceinline__ void fused_peel_set0(const SigCfg& c, const SigRun& r, float2* Ys, const int64_t* u,
                                                const int32_t* regw, const double2* rega, int16_t* hreg) {
  constexpr int U = 4;
  const int nr = min(r.K_reg, c.reg_cap);
  const float pf = (float)r.p;
  float* Yt = reinterpret_cast<float*>(Ys);
  const int32_t* rw = regw + c.regw_off;
  const double2* ra = rega + c.rega_off;
  for (int j0 = threadIdx.x; j0 < nr; j0 += U * blockDim.x) {
    double2 av[U];
    int h[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int jr = j0 + q * blockDim.x;
      av[q] = jr < nr ? ra[jr] : make_double2(0.0, 0.0);
      h[q] = jr < nr ? (int)project_mod(rw + (int64_t)jr * c.d, c.d, u, c.box_lo, r.p, r.mod_m, r.proj_off, r.mod32)
                     : -1;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int jr = j0 + q * blockDim.x;
      if (jr >= nr) continue;
      const bool live = av[q].x != 0.0 || av[q].y != 0.0;
      hreg[jr] = live ? (int16_t)h[q] : (int16_t)-1;
      if (!live) continue;
      atomicAdd(Yt + 2 * h[q], -pf * (float)av[q].x);
      atomicAdd(Yt + 2 * h[q] + 1, -pf * (float)av[q].y);
    }
  }
}

// The other sets' residual at the occupied bins (occ[h] != 0): the entries whose bin is
// occupied add -p a e^{2 pi i w . s_n} to Y_n[h], n >= 1 (four entries per thread, their loads
// first; a few entries per occupied bin, so few atomics).
template <int NS>
__device__ __forceinline__ void fused_peel_bins(const SigCfg& c, const SigRun& r, float2* Ys, const uint8_t* occ,
                                                const double2* rega, const float2* regtw, const int16_t* hreg) {
  constexpr int U = 4;
  constexpr int S = NS - 1 > 0 ? NS - 1 : 1;
  const int nr = min(r.K_reg, c.reg_cap);
  const int p = (int)r.p;
  const float pf = (float)p;
  float* Yt = reinterpret_cast<float*>(Ys);
  const double2* ra = rega + c.rega_off;
  const float2* rt = regtw + c.regtw_off;
  for (int j0 = threadIdx.x; j0 < nr; j0 += U * blockDim.x) {
    int h[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int jr = j0 + q * blockDim.x;
      h[q] = jr < nr ? (int)hreg[jr] : -1;
      if (h[q] >= 0 && !occ[h[q]]) h[q] = -1;
    }
    double2 av[U];
    float2 tv[U][S];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (h[q] < 0) continue;
      const int jr = j0 + q * blockDim.x;
      av[q] = ra[jr];
#pragma unroll
      for (int n = 0; n < NS - 1; ++n) tv[q][n] = rt[(int64_t)jr * (NS - 1) + n];
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (h[q] < 0) continue;
      const float px = -pf * (float)av[q].x, py = -pf * (float)av[q].y;
#pragma unroll
      for (int n = 1; n < NS; ++n) {
        const float2 t = tv[q][n - 1];
        const int e = n * p + h[q];
        atomicAdd(Yt + 2 * e, px * t.x - py * t.y);
        atomicAdd(Yt + 2 * e + 1, px * t.y + py * t.x);
      }
    }
  }
}

// ratio test, read-out and registry merge of the occupied bins cand[0..n_cand)
__device__ __noinline__ void fused_classify(const SigCfg& c, SigRun* rp, int s, const int* cand, int n_cand,
                                            const float2* Ys, const int64_t* ubuf, const int32_t* shblk,
                                            int32_t* regw, double2* rega, float2* regtw, int32_t* hash) {
  const ClassifyOut co{nullptr, nullptr, nullptr, 0, nullptr, nullptr, -1.0};
  for (int e = threadIdx.x; e < n_cand; e += blockDim.x)
    classify_candidate<float>(c, rp, s, cand[e], Ys, ubuf, shblk, regw, rega, regtw, hash, co);
}

// Plans the signal's next round (one thread); returns 1 when it runs fused too.  A round left
// to the batched kernels is not stored: their plan kernel makes the same one.
__device__ __noinline__ int fused_next(const PlanArgs& pa, const PrimeTables& pt, const SigCfg& c, SigRun* rp, int s,
                                       int64_t* ubuf, HistRec* hist) {
  SigRun nx = *rp;
  plan_signal<float>(pa, c, nx, pt, ubuf, hist, s == 0);
  if (!nx.active) {
    *rp = nx;   // done, or stopped by the round limit
    return 0;
  }
  if (nx.fused) {
    *rp = nx;
    return 1;
  }
  rp->fused = 0;   // the round just run is finished and the next one not yet planned
  return 0;
}

// One round of every signal of NS sample sets whose plan marks it fused (blocks of other
// signals return).
template <int NS>
__global__ void __launch_bounds__(kSampleThreads, 2) k_fused(FusedArgs a) {
  using C2 = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ C2 tw_lo[kTwLo], tw_hi[kFusedMaxL / kTwLo];
  __shared__ SigRun rs;   // the round being run
  __shared__ int s_cnt;
  __shared__ PlanArgs s_pa;
  __shared__ PrimeTables s_pt;
  __shared__ int64_t s_u[kFusedMaxD];   // the round's direction (d <= kFusedMaxD)
  const int s = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  if (s >= a.pa.n) return;
  SigRun* rp = a.run + s;
  const SigCfg& c = a.cfg[s];
  {
    const SigRun& r0 = *rp;   // every thread reads the same fields: a uniform exit
    if (!r0.active || !r0.fused || c.n_sets != NS) return;
  }
  if (tid == 0) {
    rs = *rp;
    s_pa = a.pa;
    s_pt = a.pt;
    s_cnt = 0;
  }
  if (c.d <= kFusedMaxD && tid < c.d) s_u[tid] = a.ubuf[c.u_off + tid];
  const int64_t* u_s = c.d <= kFusedMaxD ? s_u : a.ubuf + c.u_off;
  __syncthreads();
  const SigRun& r = rs;
  const int p = (int)r.p;
  const int L = r.L;
  const FusedLayout lay = fused_layout(a.L_alloc, NS);   // every area at its largest
  C2* tab_s = reinterpret_cast<C2*>(smem_raw + lay.tab);
  C2* slots = reinterpret_cast<C2*>(smem_raw + lay.slots);
  unsigned char* work = smem_raw + lay.work;
  const int ls = lay.ls;

  // tables, the DFT's twiddles, then the filter (slot 0) and the rows' zero tails
  for (int m = tid; m < p; m += blockDim.x) table_entry<float>(r.p, r.mod_m, m, tab_s);
  fft_tables(tw_hi, tw_lo, L, a.tws);
  __syncthreads();
  for (int e = tid; e < L; e += blockDim.x) slots[fpad(e)] = filter_value<float>(e, p, L, tab_s + p);
  for (int e = tid; e < NS * (L - p); e += blockDim.x) {
    const int n = e / (L - p), x = p + (e - n * (L - p));
    slots[(n + 1) * ls + fpad(x)] = mk2(0.0f, 0.0f);
  }
  fused_sample<NS>(a, c, r, s, u_s, tab_s, slots, ls, work);
  __syncthreads();

  C2* Ys = reinterpret_cast<C2*>(work);   // the modes and partial sums are consumed
  if ((NS + 1) * fft_threads<C2, 16>(L) <= (int)blockDim.x)
    fused_convolve<16>(c, r, tab_s, slots, ls, tw_hi, tw_lo, Ys, &rp->maxy0_bits);
  else
    fused_convolve<32>(c, r, tab_s, slots, ls, tw_hi, tw_lo, Ys, &rp->maxy0_bits);
  __syncthreads();
  // the DFT rows are consumed: their area takes the candidate list (p <= kFusedMaxL / 2 entries),
  // occupied-bin flags (bytes) and the registry entries' bins (int16)
  int* cand = reinterpret_cast<int*>(slots);
  uint8_t* occf = reinterpret_cast<uint8_t*>(slots) + 2 * kFusedMaxL;
  int16_t* hreg = reinterpret_cast<int16_t*>(slots) + 3 * kFusedMaxL / 2;
  const int hcap = (lay.work - lay.slots) / 2 - 3 * kFusedMaxL / 2;
  const bool lazy = min(r.K_reg, c.reg_cap) <= hcap;
  for (int h = tid; h < p; h += blockDim.x) occf[h] = 0;
  if (c.peel_bins) {
    if (lazy) fused_peel_set0<NS>(c, r, Ys, u_s, a.regw, a.rega, hreg);
    else fused_peel<NS>(c, r, Ys, u_s, a.regw, a.rega, a.regtw);
    __syncthreads();
  }

  // empty-bin test, as in the batched path (A_ref from the first round's largest bin)
  const bool first = r.round == 1;
  const double maxy0 = __longlong_as_double((long long)rp->maxy0_bits);
  if (tid == 0) {
    const double a_ref = first ? maxy0 / (double)p : r.a_ref;
    if (first) rp->a_ref = a_ref;
    rp->eta_prune = fmax(c.rho * a_ref, 6.0 * c.sigma / sqrt((double)p));
  }
  const float a_ref_f = first ? (float)maxy0 / (float)p : (float)r.a_ref;
  const float eta = fmaxf((float)c.rho * (float)p * a_ref_f, 6.0f * (float)c.sigma * sqrtf((float)p));
  for (int h0 = 0; h0 < p; h0 += blockDim.x) {
    const int h = h0 + tid;
    bool occ = false;
    if (h < p) {
      const C2 y0 = Ys[h];
      occ = y0.x * y0.x + y0.y * y0.y > eta * eta;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, occ);
    int base = 0;
    if (lane == 0 && mask != 0u) base = atomicAdd(&s_cnt, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (occ) {
      cand[base + __popc(mask & ((1u << lane) - 1u))] = h;
      occf[h] = 1;
    }
  }
  __syncthreads();
  const int n_cand = s_cnt;
  if (tid == 0 && n_cand > 0) rp->any_occupied = 1;
  if (c.peel_bins && lazy && n_cand > 0) {
    fused_peel_bins<NS>(c, r, Ys, occf, a.rega, a.regtw, hreg);
    __syncthreads();
  }
  if (NS > 1 && n_cand == 0) {
    // Set 0 is empty, so the signal would stop; the residual is empty only when the other sets
    // are too.  Two registry entries of opposite coefficients whose difference this line does
    // not see cancel in set 0 alone (a read-out that slipped in a coordinate outside the round's
    // block leaves such a pair).  The other sets' residual differs from f's transform only at
    // the bins of registry entries: those take their peel first.
    if (c.peel_bins && lazy) {
      const int nr = min(r.K_reg, c.reg_cap);
      for (int j = tid; j < nr; j += blockDim.x)
        if (hreg[j] >= 0) occf[hreg[j]] = 1;
      __syncthreads();
      fused_peel_bins<NS>(c, r, Ys, occf, a.rega, a.regtw, hreg);
      __syncthreads();
    }
    int any = 0;
    for (int e = tid; e < (NS - 1) * p; e += blockDim.x) {
      const C2 y = Ys[p + e];
      any |= y.x * y.x + y.y * y.y > eta * eta ? 1 : 0;
    }
    any = __syncthreads_or(any);
    if (tid == 0 && any) rp->any_occupied = 1;
  }
  fused_classify(c, rp, s, cand, n_cand, Ys, a.ubuf, a.shblk, a.regw, a.rega, a.regtw, a.hash);
  __syncthreads();

  // the next round: fused again while its line stays short
  if (tid == 0 && fused_next(s_pa, s_pt, c, rp, s, a.ubuf, a.hist)) atomicAdd(&a.ctl->n_fused_next, 1ull);
}

}  // namespace

template <int NS>
cudaError_t fused_setup_ns(size_t smem) {
  return cudaFuncSetAttribute(k_fused<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int NS>
cudaError_t fused_launch_ns(int n_slots, size_t smem, cudaStream_t st, const FusedArgs& a) {
  k_fused<NS><<<n_slots, kSampleThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sfft
