// Device helpers of the batched round engine: modular arithmetic, unit roots,
// block scans and work-item lookup.
#pragma once

#include "engine.cuh"

namespace sfft {

// x mod p for x < 2^64 by Barrett reduction with m = floor((2^64 - 1) / p):
// q = floor(x m / 2^64) is floor(x / p) or one less, so one correction suffices.
__device__ __forceinline__ uint64_t mod_barrett(uint64_t x, uint64_t p, uint64_t m) {
  const uint64_t q = __umul64hi(x, m);
  uint64_t r = x - q * p;
  return r >= p ? r - p : r;
}

// (w . u) mod p for w in the box [box_lo, box_lo + N)^d and u reduced mod p, as
// sum_l (w_l - box_lo) u_l + box_lo sum_l u_l with every step reduced (w_l - box_lo < 2^31, u_l < p).
// off = (box_lo mod p) (sum_l u_l mod p) mod p, a constant of the round (proj_offset)
// Up to 8 coordinates are loaded together before the reduction chain (their loads overlap).
// m32 = floor((2^32 - 1) / p) when (N + 1) p < 2^32 (every partial sum fits 32 bits: 32-bit
// Barrett steps), else 0 (64-bit steps).
__device__ __forceinline__ uint64_t project_mod(const int32_t* w, int d, const int64_t* u, int box_lo, int64_t p,
                                                uint64_t mm, uint64_t off, uint32_t m32) {
  const uint64_t up = (uint64_t)p;
  uint64_t acc = 0;
  if (d <= 8) {
    int32_t wv[8];
    int64_t uv[8];
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      wv[l] = l < d ? w[l] : box_lo;
      uv[l] = l < d ? u[l] : 0;
    }
    if (m32 != 0u) {
      const uint32_t p32 = (uint32_t)p;
      uint32_t a32 = 0;
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        if (l < d) {
          const uint32_t x = (uint32_t)(wv[l] - box_lo) * (uint32_t)uv[l] + a32;
          const uint32_t r = x - __umulhi(x, m32) * p32;
          a32 = r >= p32 ? r - p32 : r;
        }
      }
      acc = a32;
    } else {
#pragma unroll
      for (int l = 0; l < 8; ++l)
        if (l < d) acc = mod_barrett((uint64_t)(int64_t)(wv[l] - box_lo) * (uint64_t)uv[l] + acc, up, mm);
    }
  } else {
    for (int l = 0; l < d; ++l) acc = mod_barrett((uint64_t)(int64_t)(w[l] - box_lo) * (uint64_t)u[l] + acc, up, mm);
  }
  acc += off;   // < 2p
  return acc >= up ? acc - up : acc;
}

// The offset of project_mod for the direction u (reduced mod p) of a round: w . u = sum_l
// (w_l - box_lo) u_l + box_lo sum_l u_l, the first sum over non-negative terms.
__device__ __forceinline__ uint64_t proj_offset(int d, const int64_t* u, int box_lo, int64_t p, uint64_t mm) {
  const uint64_t up = (uint64_t)p;
  uint64_t usum = 0;
  for (int l = 0; l < d; ++l) usum = mod_barrett(usum + (uint64_t)u[l], up, mm);
  const int64_t blm = ((int64_t)box_lo % p + p) % p;
  return mod_barrett((uint64_t)blm * usum, up, mm);
}

// a mod p for 0 <= a < 64 p < 2^31, via a float reciprocal and one correction.
__device__ __forceinline__ int mod_small(unsigned a, int p, float inv_p) {
  int q = __float2int_rz(__uint2float_rn(a) * inv_p);
  int r = (int)a - q * p;
  if (r < 0) r += p;
  else if (r >= p) r -= p;
  return r;
}

// e^{2 pi i m / q} for integers 0 <= m < q.  The angle is folded to (-pi, pi]
// as 2 (m - q [2m > q]) / q half-turns; in float the half-turn count is split
// into a rounded head and an exactly computed tail, and the tail enters by a
// first-order rotation, so the only rounding left is that of sincospif itself.
template <typename T> __device__ __forceinline__ c2<T> unit_root(int64_t m, int64_t q);
template <> __device__ __forceinline__ float2 unit_root<float>(int64_t m, int64_t q) {
  const int64_t mm = (2 * m > q) ? m - q : m;
  const float num = (float)(2 * mm);   // exact: |2 mm| <= q < 2^24
  const float qf = (float)q;
  const float xh = num / qf;
  const float xl = fmaf(-xh, qf, num) / qf;
  float s, c;
  sincospif(xh, &s, &c);
  const float dl = 3.14159265358979f * xl;
  return make_float2(fmaf(-s, dl, c), fmaf(c, dl, s));
}
template <> __device__ __forceinline__ double2 unit_root<double>(int64_t m, int64_t q) {
  const int64_t mm = (2 * m > q) ? m - q : m;
  double s, c;
  sincospi(2.0 * (double)mm / (double)q, &s, &c);
  return make_double2(c, s);
}

// e^{2 pi i w . s_n} of shifted set n (1-based).  Coordinate form: s_n = e_n / N, the root of
// w_n mod N of order N.  Block form: s_n = v_n / (2 N^{d1}) along the unwrap vector of block n
// (start blk[2n - 2], size d1 = blk[2n - 1]), the root of w~_n mod 2 N^{d1} of order 2 N^{d1},
// w~_n = sum_r w_{start + r} N^r.  in_box: w lies in the box (one conditional wrap suffices).
// Tilted form (Alg. 3, d = 2): s_n = (axis n) / Q, the root of w~_n mod Q of order Q, with
// w~_1 = base w_1 - height w_2, w~_2 = height w_1 + base w_2 and Q = (base + height) N.
template <typename T>
__device__ __forceinline__ c2<T> shift_root(const SigCfg& c, const int32_t* __restrict__ blk, const int32_t* w,
                                            int n, bool in_box) {
  if (c.shift_tilt) {
    const int64_t b = c.tilt_base, h = c.tilt_height, w1 = w[0], w2 = w[1];
    const int64_t q = (b + h) * c.N;
    int64_t m = (n == 1 ? b * w1 - h * w2 : h * w1 + b * w2) % q;
    if (m < 0) m += q;
    return unit_root<T>(m, q);
  }
  if (!c.shift_block) {
    int64_t m = w[n - 1];
    if (in_box) {
      if (m < 0) m += c.N;
    } else {
      m %= c.N;
      if (m < 0) m += c.N;
    }
    return unit_root<T>(m, c.N);
  }
  const int b = blk[2 * (n - 1)], size = blk[2 * (n - 1) + 1];
  int64_t wt = 0, pw = 1;
  for (int r = 0; r < size; ++r) {
    wt += (int64_t)w[b + r] * pw;
    pw *= c.N;
  }
  const int64_t q = 2 * pw;
  int64_t m = in_box ? wt : wt % q;
  if (m < 0) m += q;
  return unit_root<T>(m, q);
}

// chirp[x] = e^{-pi i x^2 / p} = conj(e^{2 pi i (x^2 mod 2p) / (2p)})
template <typename T>
__device__ __forceinline__ c2<T> chirp_at(int64_t x, int64_t p) {
  const uint64_t q = ((uint64_t)x * (uint64_t)x) % (uint64_t)(2 * p);
  return cconj(unit_root<T>((int64_t)q, 2 * p));
}

// index s with scan[s] <= item < scan[s + 1] (scan non-decreasing, scan[0] = 0)
__device__ __forceinline__ int find_slot(const int64_t* __restrict__ scan, int n, int64_t item) {
  int lo = 0, hi = n;   // invariant scan[lo] <= item < scan[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(scan + mid) <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

// find_slot for an item known to lie at or after slot `from` (scan[from] <= item): the item is
// most often in that slot itself (one load); else a galloping search from it, then a binary one.
__device__ __forceinline__ int find_slot_from(const int64_t* __restrict__ scan, int n, int64_t item, int from) {
  int lo = from;
  if (__ldg(scan + lo + 1) > item) return lo;
  int hi = lo + 1, step = 1;   // scan[hi] <= item
  for (;;) {
    lo = hi;
    const int nxt = min(lo + step, n);
    if (nxt == n || __ldg(scan + nxt) > item) {
      hi = nxt;
      break;
    }
    hi = nxt;
    step *= 2;
  }
  // scan[lo] <= item < scan[hi] (scan[n] is the total, above every item)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(scan + mid) <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Exclusive scan of V values per thread over the block (a multiple of 32 threads, at most 1024).
template <int V>
__device__ __forceinline__ void block_scan_excl(int64_t (&v)[V], int64_t (&tot)[V]) {
  __shared__ int64_t ws[32][V];
  __shared__ int64_t wt[V];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int64_t incl[V];
#pragma unroll
  for (int q = 0; q < V; ++q) {
    int64_t x = v[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    incl[q] = x;
    if (lane == 31) ws[wid][q] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < V; ++q) {
      int64_t x = lane < nwarps ? ws[lane][q] : 0;
      const int64_t own = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      ws[lane][q] = x - own;
      if (lane == 31) wt[q] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < V; ++q) {
    v[q] = incl[q] - v[q] + ws[wid][q];
    tot[q] = wt[q];
  }
  __syncthreads();
}

__device__ __forceinline__ int64_t block_sum(int64_t x) {
  int64_t v[1] = {x}, t[1];
  block_scan_excl<1>(v, t);
  return t[0];
}

}  // namespace sfft
