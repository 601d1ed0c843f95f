// One tile of the sample-and-residual computation (Alg. 2 sampling; Eq. 41), shared
// by the batched engine and the allocation-free sampling entry point.
//
//   y_n[x] = sum_j C[n][j] W[(alpha_j x) mod p],  W[m] = e^{2 pi i m / p}.
//
// The points x and p - x of the line have conjugate exponentials, W[(alpha (p - x)) mod p] =
// conj(W[(alpha x) mod p]) = conj(E).  With C = c_r + i c_i and E = e_r + i e_i, the four sums
//   P1 = sum c_r e_r,  P2 = sum c_i e_i,  P3 = sum c_r e_i,  P4 = sum c_i e_r
// give both samples: y[x] = (P1 - P2, P3 + P4) and y[p - x] = (P1 + P2, P4 - P3), so every term
// of the two samples costs four fused multiply-adds instead of eight.  A tile therefore runs
// over the positions 0 <= x < H = floor(p / 2) + 1 (x and p - x coincide only for p = 2), and
//   E = W[(alpha (x0 + 32 row)) mod p] * W[(alpha lane) mod p],  x = x0 + 32 row + lane,
// the first factor shared by the 32 lanes of a row, the second by the rows of a lane.
#pragma once

#include <type_traits>

#include "engine_kernels.cuh"

namespace sfft {

constexpr int kSampleThreads = kSampleWarps * 32;

// Asynchronous global -> shared copies (cp.async): the gathers of the next chunk's unit
// roots land in shared memory while the current chunk is being accumulated.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (BYTES == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// staging buffers: two in float (the next chunk is gathered during the current one), one in double
template <typename T> constexpr int sample_stages() { return sizeof(T) == 4 ? 2 : 1; }

// Staged data of one or two 32-mode chunks, overlaid at the end of a tile by the buffer that
// adds the mode groups' sums (half of the warps' sums at a time).
// In float the per-set coefficients of a mode are padded to an even count, so that the
// accumulation reads two sets' values with one 16-byte shared-memory load.
template <typename T, int NS>
struct alignas(16) SampleSmem {
  static constexpr int S = sample_stages<T>();
  static constexpr int RP = row_pairs(NS);
  static constexpr int NSP = sizeof(T) == 4 ? ((NS + 1) & ~1) : NS;
  struct Stage {
    c2<T> Ls[S][kSampleChunk][32];
    c2<T> Us[S][kSampleChunk][kSampleWarps * RP];
    c2<T> Cs[S][kSampleChunk][NSP];
  };
  static constexpr int kRedValues = (kSampleWarps / 2) * RP * NS * 4 * 32;
  union {
    Stage st;
    T red[kRedValues];
  };
  int al[S][kSampleChunk], be[S][kSampleChunk], ga[S][kSampleChunk];
  int64_t item;
};

// Sums one staged 32-mode chunk (modes grp, grp + G, ...) into the first Q row pairs of the
// totals: E = U_row L_lane, then the four products of every set's coefficient with E.
template <typename T, int NS, int RP, int Q>
__device__ __forceinline__ void accumulate_chunk(const SampleSmem<T, NS>& sm, int b, int grp, int G, int lane,
                                                 int wrow, T (&tot)[RP][NS][4]) {
  using C2 = c2<T>;
  T acc[Q][NS][4];
#pragma unroll
  for (int qq = 0; qq < Q; ++qq)
#pragma unroll
    for (int nn = 0; nn < NS; ++nn) acc[qq][nn][0] = acc[qq][nn][1] = acc[qq][nn][2] = acc[qq][nn][3] = (T)0;
#pragma unroll 2
  for (int jj = grp; jj < kSampleChunk; jj += G) {
    const C2 L = sm.st.Ls[b][jj][lane];
    C2 E[Q];
    if constexpr (sizeof(T) == 4 && RP % 2 == 0 && Q % 2 == 0) {   // two rows per 16-byte load
#pragma unroll
      for (int qq = 0; qq < Q; qq += 2) {
        const float4 u4 = *reinterpret_cast<const float4*>(&sm.st.Us[b][jj][wrow * RP + qq]);
        E[qq] = cmul(mk2(u4.x, u4.y), L);
        E[qq + 1] = cmul(mk2(u4.z, u4.w), L);
      }
    } else {
#pragma unroll
      for (int qq = 0; qq < Q; ++qq) E[qq] = cmul(sm.st.Us[b][jj][wrow * RP + qq], L);
    }
    auto term = [&](int nn, C2 cc) {
#pragma unroll
      for (int qq = 0; qq < Q; ++qq) {
        acc[qq][nn][0] = fma(cc.x, E[qq].x, acc[qq][nn][0]);   // P1: c_r e_r
        acc[qq][nn][1] = fma(cc.y, E[qq].y, acc[qq][nn][1]);   // P2: c_i e_i
        acc[qq][nn][2] = fma(cc.x, E[qq].y, acc[qq][nn][2]);   // P3: c_r e_i
        acc[qq][nn][3] = fma(cc.y, E[qq].x, acc[qq][nn][3]);   // P4: c_i e_r
      }
    };
    if constexpr (sizeof(T) == 4) {   // two sets per 16-byte load (rows padded to even)
#pragma unroll
      for (int nn = 0; nn < NS; nn += 2) {
        const float4 c4 = *reinterpret_cast<const float4*>(&sm.st.Cs[b][jj][nn]);
        term(nn, mk2(c4.x, c4.y));
        if (nn + 1 < NS) term(nn + 1, mk2(c4.z, c4.w));
      }
    } else {
#pragma unroll
      for (int nn = 0; nn < NS; ++nn) term(nn, sm.st.Cs[b][jj][nn]);
    }
  }
#pragma unroll
  for (int qq = 0; qq < Q; ++qq)
#pragma unroll
    for (int nn = 0; nn < NS; ++nn)
#pragma unroll
      for (int k = 0; k < 4; ++k) tot[qq][nn][k] += acc[qq][nn][k];
}

// The same for 1 <= nq < RP row pairs (the rows of a warp that reach past the half line are skipped).
template <typename T, int NS, int RP>
__device__ __forceinline__ void accumulate_rows(const SampleSmem<T, NS>& sm, int b, int grp, int G, int lane,
                                                int wrow, int nq, T (&tot)[RP][NS][4]) {
  switch (nq) {
    case 1: if constexpr (RP > 1) accumulate_chunk<T, NS, RP, 1>(sm, b, grp, G, lane, wrow, tot); break;
    case 2: if constexpr (RP > 2) accumulate_chunk<T, NS, RP, 2>(sm, b, grp, G, lane, wrow, tot); break;
    case 3: if constexpr (RP > 3) accumulate_chunk<T, NS, RP, 3>(sm, b, grp, G, lane, wrow, tot); break;
    case 4: if constexpr (RP > 4) accumulate_chunk<T, NS, RP, 4>(sm, b, grp, G, lane, wrow, tot); break;
    case 5: if constexpr (RP > 5) accumulate_chunk<T, NS, RP, 5>(sm, b, grp, G, lane, wrow, tot); break;
    case 6: if constexpr (RP > 6) accumulate_chunk<T, NS, RP, 6>(sm, b, grp, G, lane, wrow, tot); break;
    case 7: if constexpr (RP > 7) accumulate_chunk<T, NS, RP, 7>(sm, b, grp, G, lane, wrow, tot); break;
    default: break;
  }
}

// ---- double-float arithmetic on the FP32 pipe: a value is hi + lo with |lo| <= ulp(hi) / 2 (a
// float2 (hi, lo)), about 48 significant bits.  Products are exact through an FMA (a b - fl(a b)
// is a float), sums through Knuth's two-sum; the round-to-nearest intrinsics keep the compiler
// from contracting the error terms away.
__device__ __forceinline__ float2 df_quick(float s, float e) {   // |e| <= |s|: renormalise
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  return df_quick(s, e);
}
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ double df_value(float2 a) { return (double)a.x + (double)a.y; }
// a complex value staged as double-float: (re hi, re lo, im hi, im lo) in the 16 bytes of a double2
__device__ __forceinline__ float4 df_pack(double2 v) {
  const float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

__device__ __forceinline__ void df_pack_inplace(double2* v) {
  *reinterpret_cast<float4*>(v) = df_pack(*v);
}
// a b as an unnormalised pair (fl(a.hi b.hi), the rest): 4 operations
__device__ __forceinline__ float2 df_prod(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return make_float2(p, e);
}
// acc += a b with acc left unnormalised: the high parts by two-sum, every low-order term into
// acc.y (8 operations after the product).  Within a 32-mode chunk acc.y stays below about 32
// ulps of the largest partial sum, so its own rounding costs no more than renormalising.
__device__ __forceinline__ void df_mac(float2& acc, float2 a, float2 b) {
  const float2 q = df_prod(a, b);
  const float t = __fadd_rn(acc.x, q.x);
  const float bb = __fsub_rn(t, acc.x);
  const float err = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(t, bb)), __fsub_rn(q.x, bb));
  acc.y = __fadd_rn(acc.y, __fadd_rn(err, q.y));
  acc.x = t;
}

// accumulate_chunk in double-float (the FP64 engine's double-float sampling): the staged roots and
// coefficients hold df_pack values, the sums P1..P4 are double-float
template <int NS, int RP, int Q>
__device__ __forceinline__ void accumulate_chunk_df(const SampleSmem<double, NS>& sm, int lane, int wrow,
                                                    float2 (&tot)[RP][NS][4]) {
  float2 acc[Q][NS][4];
#pragma unroll
  for (int qq = 0; qq < Q; ++qq)
#pragma unroll
    for (int nn = 0; nn < NS; ++nn)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[qq][nn][k] = make_float2(0.0f, 0.0f);
  for (int jj = 0; jj < kSampleChunk; ++jj) {
    const float4 L = reinterpret_cast<const float4&>(sm.st.Ls[0][jj][lane]);
    float2 Er[Q], Ei[Q];   // E = U L, unnormalised (|E| = 1: absolute error about 2^-48)
#pragma unroll
    for (int qq = 0; qq < Q; ++qq) {
      const float4 U = reinterpret_cast<const float4&>(sm.st.Us[0][jj][wrow * RP + qq]);
      const float2 ur = make_float2(U.x, U.y), ui = make_float2(U.z, U.w);
      const float2 lr = make_float2(L.x, L.y), li = make_float2(L.z, L.w);
      Er[qq] = df_prod(ur, lr);
      df_mac(Er[qq], make_float2(-ui.x, -ui.y), li);
      Ei[qq] = df_prod(ur, li);
      df_mac(Ei[qq], ui, lr);
    }
#pragma unroll
    for (int nn = 0; nn < NS; ++nn) {
      const float4 C = reinterpret_cast<const float4&>(sm.st.Cs[0][jj][nn]);
      const float2 cr = make_float2(C.x, C.y), ci = make_float2(C.z, C.w);
#pragma unroll
      for (int qq = 0; qq < Q; ++qq) {
        df_mac(acc[qq][nn][0], cr, Er[qq]);   // P1: c_r e_r
        df_mac(acc[qq][nn][1], ci, Ei[qq]);   // P2: c_i e_i
        df_mac(acc[qq][nn][2], cr, Ei[qq]);   // P3: c_r e_i
        df_mac(acc[qq][nn][3], ci, Er[qq]);   // P4: c_i e_r
      }
    }
  }
#pragma unroll
  for (int qq = 0; qq < Q; ++qq)
#pragma unroll
    for (int nn = 0; nn < NS; ++nn)
#pragma unroll
      for (int k = 0; k < 4; ++k) tot[qq][nn][k] = df_add(tot[qq][nn][k], acc[qq][nn][k]);
}

template <int NS, int RP>
__device__ __forceinline__ void accumulate_rows_df(const SampleSmem<double, NS>& sm, int lane, int wrow, int nq,
                                                   float2 (&tot)[RP][NS][4]) {
  switch (nq) {
    case 1: if constexpr (RP > 1) accumulate_chunk_df<NS, RP, 1>(sm, lane, wrow, tot); break;
    case 2: if constexpr (RP > 2) accumulate_chunk_df<NS, RP, 2>(sm, lane, wrow, tot); break;
    case 3: if constexpr (RP > 3) accumulate_chunk_df<NS, RP, 3>(sm, lane, wrow, tot); break;
    case 4: if constexpr (RP > 4) accumulate_chunk_df<NS, RP, 4>(sm, lane, wrow, tot); break;
    default: break;
  }
}

// One tile: 32 * kSampleWarps * RP positions of the half line (each giving the samples x and
// p - x) x the sets of one group x the modes of one split.  Each 32-mode chunk is summed into
// fresh accumulators that are then added to the running totals (blocked summation), which
// keeps the float rounding of long mode sums near that of the individual terms.
// DF (T = double only): the staged data hold df_pack values and the sums run in double-float on
// the FP32 pipe (one mode group, one stage, as in double); the samples are written in double.
template <typename T, int NS, bool DF = false>
__device__ void sample_tile(SampleSmem<T, NS>& sm, const SigCfg& c, const SigRun& r, int xt, int g, int split,
                            const int32_t* __restrict__ alpha, const int32_t* __restrict__ gam,
                            const c2<T>* __restrict__ Cm, const c2<T>* __restrict__ W, c2<T>* __restrict__ part) {
  using C2 = c2<T>;
  constexpr int RP = row_pairs(NS);
  constexpr int S = sample_stages<T>();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // G mode groups of kSampleWarps / G warps: a group covers all rows of the tile and takes
  // every G-th mode
  const int G = r.mgroups;
  const int wpg = kSampleWarps / G;
  const int grp = warp / wpg, wrow = warp - grp * wpg;
  const int TX = 32 * RP * wpg;
  const int rows = RP * wpg;   // rows of 32 positions in the tile
  const int p = (int)r.p;
  const int H = p / 2 + 1;   // positions of the half line
  const float inv_p = 1.0f / (float)p;
  const int n0 = g * r.gsize;
  const int ns_valid = min(r.gsize, c.n_sets - n0);
  const int K = sampled_modes(c, r);
  const int x0 = xt * TX;
  const int nq = min(RP, max(0, (H - (x0 + wrow * RP * 32) + 31) / 32));   // row pairs of this warp below H
  const int j_begin = split * r.jper;
  const int j_end = min(K, j_begin + r.jper);
  const int nchunks = j_end > j_begin ? (j_end - j_begin + kSampleChunk - 1) / kSampleChunk : 0;
  const C2 zero = mk2((T)0, (T)0);

  // mode indices of chunk q into stage b (threads < 32)
  auto put_index = [&](int b, int al, int ga) {
    sm.al[b][tid] = al;
    sm.ga[b][tid] = ga;
    sm.be[b][tid] = (int)mod_barrett((uint64_t)al * (uint64_t)x0, (uint64_t)p, r.mod_m);
  };
  auto load_index = [&](int q, int* al, int* ga) {
    const int j = j_begin + q * kSampleChunk + tid;
    *al = (j < j_end) ? alpha[j] : 0;
    *ga = (j < j_end) ? gam[j] : 0;
  };
  // unit roots and per-set coefficients of chunk q into stage b (all threads)
  auto issue_data = [&](int q, int b) {
    const int jc = j_begin + q * kSampleChunk;
    const int nj = min(kSampleChunk, j_end - jc);
    for (int e = tid; e < kSampleChunk * 32; e += kSampleThreads) {
      const int jj = e >> 5, ln = e & 31;
      cp_async<sizeof(C2)>(&sm.st.Ls[b][jj][ln], W + mod_small((unsigned)sm.al[b][jj] * (unsigned)ln, p, inv_p));
    }
    for (int e = tid; e < kSampleChunk * rows; e += kSampleThreads) {   // the rows a mode group covers
      const int jj = e / rows, row = e - jj * rows;
      cp_async<sizeof(C2)>(&sm.st.Us[b][jj][row],
                           W + mod_small((unsigned)sm.be[b][jj] + (unsigned)row * (unsigned)sm.ga[b][jj], p, inv_p));
    }
    constexpr int NSP = SampleSmem<T, NS>::NSP;
    for (int e = tid; e < kSampleChunk * NSP; e += kSampleThreads) {
      const int jj = e / NSP, nn = e - jj * NSP;
      if (jj < nj && nn < ns_valid) cp_async<sizeof(C2)>(&sm.st.Cs[b][jj][nn], Cm + (int64_t)(n0 + nn) * c.Kmax + jc + jj);
      else sm.st.Cs[b][jj][nn] = zero;
    }
    cp_async_commit();
  };

  using Acc = std::conditional_t<DF, float2, T>;
  Acc tot[RP][NS][4];
#pragma unroll
  for (int q = 0; q < RP; ++q)
#pragma unroll
    for (int nn = 0; nn < NS; ++nn)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if constexpr (DF) tot[q][nn][k] = make_float2(0.0f, 0.0f);
        else tot[q][nn][k] = (T)0;
      }

  if (nchunks > 0) {
    if (tid < kSampleChunk) {
      int al, ga;
      load_index(0, &al, &ga);
      put_index(0, al, ga);
      if (S == 2 && nchunks > 1) {
        load_index(1, &al, &ga);
        put_index(1, al, ga);
      }
    }
    __syncthreads();
    issue_data(0, 0);
    cp_async_wait_all();
    __syncthreads();
  }
  for (int q = 0; q < nchunks; ++q) {
    const int b = (S == 2) ? (q & 1) : 0;
    int al_n = 0, ga_n = 0;
    if (S == 2) {
      if (q + 1 < nchunks) issue_data(q + 1, b ^ 1);                     // gathers of the next chunk
      if (tid < kSampleChunk && q + 2 < nchunks) load_index(q + 2, &al_n, &ga_n);   // indices two ahead
    }
    if constexpr (DF) {
      if (nq == RP) accumulate_chunk_df<NS, RP, RP>(sm, lane, wrow, tot);
      else if (nq > 0) accumulate_rows_df<NS, RP>(sm, lane, wrow, nq, tot);
    } else {
      if (nq == RP) accumulate_chunk<T, NS, RP, RP>(sm, b, grp, G, lane, wrow, tot);
      else if (nq > 0) accumulate_rows<T, NS, RP>(sm, b, grp, G, lane, wrow, nq, tot);
    }
    if (S == 2) {
      // stage b is free again: it takes the indices of chunk q + 2
      if (tid < kSampleChunk && q + 2 < nchunks) put_index(b, al_n, ga_n);
      cp_async_wait_all();
      __syncthreads();
    } else if (q + 1 < nchunks) {
      __syncthreads();   // every thread is done with the single stage
      if (tid < kSampleChunk) {
        int al, ga;
        load_index(q + 1, &al, &ga);
        put_index(0, al, ga);
      }
      __syncthreads();
      issue_data(q + 1, 0);
      cp_async_wait_all();
      __syncthreads();
    }
  }
  if constexpr (!DF) {
  if (G > 1) {
    // add the mode groups' sums pairwise into group 0 through the (now free) staging memory:
    // at each step the upper half of the remaining groups hands its sums to the lower half
    constexpr int KK = RP * NS * 4;
    __syncthreads();
    for (int half = G / 2; half >= 1; half /= 2) {
      if (grp >= half && grp < 2 * half) {
        const int slot = (grp - half) * wpg + wrow;   // < kSampleWarps / 2
#pragma unroll
        for (int q = 0; q < RP; ++q)
#pragma unroll
          for (int nn = 0; nn < NS; ++nn)
#pragma unroll
            for (int k = 0; k < 4; ++k) sm.red[(slot * KK + (q * NS + nn) * 4 + k) * 32 + lane] = tot[q][nn][k];
      }
      __syncthreads();
      if (grp < half) {
        const int slot = grp * wpg + wrow;
#pragma unroll
        for (int q = 0; q < RP; ++q)
#pragma unroll
          for (int nn = 0; nn < NS; ++nn)
#pragma unroll
            for (int k = 0; k < 4; ++k) tot[q][nn][k] += sm.red[(slot * KK + (q * NS + nn) * 4 + k) * 32 + lane];
      }
      __syncthreads();
    }
    if (grp > 0) return;
  }
  }
  C2* out = part + r.part_off;
#pragma unroll
  for (int q = 0; q < RP; ++q) {
    const int x = x0 + (wrow * RP + q) * 32 + lane;
    if (x < H) {
      const bool mirror = x >= 1 && p - x >= H;   // p - x is a distinct sample of the other half
#pragma unroll
      for (int nn = 0; nn < NS; ++nn) {
        if (nn < ns_valid) {
          C2* row = out + ((int64_t)split * c.n_sets + n0 + nn) * p;
          if constexpr (DF) {
            const float2 P1 = tot[q][nn][0], P2 = tot[q][nn][1], P3 = tot[q][nn][2], P4 = tot[q][nn][3];
            row[x] = mk2((T)df_value(df_sub(P1, P2)), (T)df_value(df_add(P3, P4)));
            if (mirror) row[p - x] = mk2((T)df_value(df_add(P1, P2)), (T)df_value(df_sub(P4, P3)));
          } else {
            const T P1 = tot[q][nn][0], P2 = tot[q][nn][1], P3 = tot[q][nn][2], P4 = tot[q][nn][3];
            row[x] = mk2(P1 - P2, P3 + P4);
            if (mirror) row[p - x] = mk2(P1 + P2, P4 - P3);
          }
        }
      }
    }
  }
}

}  // namespace sfft
