// Stockham auto-sort FFT of one row held in shared memory, with each pass's radix-R
// butterflies done in registers, for lengths L = m 2^a with m in {1, 3, 5}.
//
// Passes use radix E (32 in float, 16 in double) while E points remain in the power-of-two
// part; the rest of it goes with the odd factor m into one pass of radix m 2^b when that is at
// most E points, else into a radix-2^b pass followed by a radix-m pass.  The pass with stride Ns
// (product of the earlier radices, always a power of two) and radix R computes, for the
// butterflies j = 0..L/R-1:
//     v[r] = x[j + r L/R] * w^(r k),  k = j mod Ns,  w = e^{-+2 pi i / (Ns R)}
//     v    = DFT_R(v)
//     x'[(j div Ns) Ns R + k + r Ns] = v[r]
// which leaves the transform in natural order after the last pass.  The block's threads take
// the butterflies in turn, at most E / R each (the block sizes and lengths in use keep L / R
// within that); all of a pass's values are read before a barrier and written after it, so one
// buffer suffices.  Rows use the padded index e + e / 32: the only pass whose writes stride by
// 32 (Ns = 1) then hits distinct banks.  Twiddles e^{-2 pi i m / L} come from two tables,
// e^{-2 pi i m / L} = hi[m >> 7] * lo[m & 127], filled from a global table of a multiple of L.
#pragma once

#include "sfft_internal.cuh"

namespace sfft {

constexpr int kTwLo = 128;          // entries of the low twiddle table
constexpr int kFftThreads = 512;    // block size of the one-row FFT kernels

// complex values per thread and pass: 32 in float, 16 in double (same register bytes)
template <typename C2> __host__ __device__ constexpr int fft_per_thread() { return sizeof(C2) == 8 ? 32 : 16; }

__device__ __forceinline__ int fpad(int e) { return e + (e >> 5); }

// cos(pi m / 16), m = 0..16: the unit roots of order 32 used inside the power-of-two register DFTs
__host__ __device__ __forceinline__ double cos_pi16(int m) {
  constexpr double c[17] = {1.0,
                            0.98078528040323044912618223613424,
                            0.92387953251128675612818318939679,
                            0.83146961230254523707878837761791,
                            0.70710678118654752440084436210485,
                            0.55557023301960222474283081394853,
                            0.38268343236508977172845998403040,
                            0.19509032201612826784828486847702,
                            0.0,
                            -0.19509032201612826784828486847702,
                            -0.38268343236508977172845998403040,
                            -0.55557023301960222474283081394853,
                            -0.70710678118654752440084436210485,
                            -0.83146961230254523707878837761791,
                            -0.92387953251128675612818318939679,
                            -0.98078528040323044912618223613424,
                            -1.0};
  return c[m];
}

// cos(pi j / 60), j = 0..60: the unit roots of order dividing 120 used by the radix-3 and
// radix-5 factors
__host__ __device__ constexpr double cos_pi60(int j) {
  constexpr double c[61] = {
      +1.000000000000000000000, +0.998629534754573873784, +0.994521895368273336923,
      +0.987688340595137726190, +0.978147600733805637929, +0.965925826289068286750,
      +0.951056516295153572116, +0.933580426497201748990, +0.913545457642600895502,
      +0.891006524188367862360, +0.866025403784438646764, +0.838670567945424029638,
      +0.809016994374947424102, +0.777145961456970879980, +0.743144825477394235015,
      +0.707106781186547524401, +0.669130606358858213826, +0.629320391049837452706,
      +0.587785252292473129169, +0.544639035015027082224, +0.500000000000000000000,
      +0.453990499739546791560, +0.406736643075800207754, +0.358367949545300273484,
      +0.309016994374947424102, +0.258819045102520762349, +0.207911690817759337102,
      +0.156434465040230869010, +0.104528463267653471400, +0.052335956242943832722,
      +0.0,                     -0.052335956242943832722, -0.104528463267653471400,
      -0.156434465040230869010, -0.207911690817759337102, -0.258819045102520762349,
      -0.309016994374947424102, -0.358367949545300273484, -0.406736643075800207754,
      -0.453990499739546791560, -0.500000000000000000000, -0.544639035015027082224,
      -0.587785252292473129169, -0.629320391049837452706, -0.669130606358858213826,
      -0.707106781186547524401, -0.743144825477394235015, -0.777145961456970879980,
      -0.809016994374947424102, -0.838670567945424029638, -0.866025403784438646764,
      -0.891006524188367862360, -0.913545457642600895502, -0.933580426497201748990,
      -0.951056516295153572116, -0.965925826289068286750, -0.978147600733805637929,
      -0.987688340595137726190, -0.994521895368273336923, -0.998629534754573873784,
      -1.000000000000000000000};
  return c[j];
}

// cos and sin of pi j / 60 for 0 <= j < 120
__host__ __device__ constexpr double cos_pi60_any(int j) { return j <= 60 ? cos_pi60(j) : cos_pi60(120 - j); }
__host__ __device__ constexpr double sin_pi60_any(int j) {
  return j <= 60 ? cos_pi60(j <= 30 ? 30 - j : j - 30) : -cos_pi60(j <= 90 ? 90 - j : j - 90);
}

// e^{-+2 pi i e / N} (forward: minus) for N dividing 120
template <typename C2, int N, bool INV>
__host__ __device__ __forceinline__ C2 root_n(int e) {
  using T = decltype(C2().x);
  const int j = ((120 / N) * e) % 120;
  const double s = sin_pi60_any(j);
  return mk2((T)cos_pi60_any(j), (T)(INV ? s : -s));
}

// In-register DFT of R points, R a power of two <= 32, forward (e^{-2 pi i}) or inverse.
// Radix-2 decimation in time on the bit-reversed register order; all indices are
// compile-time constants, so the permutation costs nothing.
template <typename C2, int R, bool INV>
__host__ __device__ __forceinline__ void dft_reg(C2 (&v)[R]) {
  using T = decltype(C2().x);
  constexpr int LG = R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int j = 0;
#pragma unroll
    for (int b = 0; b < LG; ++b) j |= ((i >> b) & 1) << (LG - 1 - b);
    if (i < j) {
      const C2 t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int s = 1; s < R; s *= 2) {
#pragma unroll
    for (int g = 0; g < R; g += 2 * s) {
#pragma unroll
      for (int t = 0; t < s; ++t) {
        // w = e^{-+2 pi i t / (2 s)} = e^{-+ i pi (16 t / s) / 16}
        const int m = (16 * t) / s;   // 0..15 in units of pi / 16
        const C2 a = v[g + t];
        C2 b = v[g + t + s];
        if (t != 0) {
          // cos(pi m / 16) and sin(pi m / 16) = cos(pi |8 - m| / 16)
          const T c = (T)cos_pi16(m);
          const T sn = (T)cos_pi16(m <= 8 ? 8 - m : m - 8);
          const T wy = INV ? sn : -sn;
          b = mk2(b.x * c - b.y * wy, b.x * wy + b.y * c);
        }
        v[g + t] = cadd(a, b);
        v[g + t + s] = csub(a, b);
      }
    }
  }
}

// 3-point DFT: X0 = a + t, X1,2 = a - t / 2 -+ i sin(2 pi / 3) (b - c), t = b + c
template <typename C2, bool INV>
__host__ __device__ __forceinline__ void dft3(C2 (&v)[3]) {
  using T = decltype(C2().x);
  const T sn = (T)cos_pi60(10);   // sin(2 pi / 3)
  const C2 t = cadd(v[1], v[2]);
  const C2 d = csub(v[1], v[2]);
  const C2 m = mk2(v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y);
  const C2 q = INV ? mk2(-sn * d.y, sn * d.x) : mk2(sn * d.y, -sn * d.x);   // -+ i sn d
  v[0] = cadd(v[0], t);
  v[1] = cadd(m, q);
  v[2] = csub(m, q);
}

// 5-point DFT from the symmetric pairs t1 = x1 + x4, t2 = x2 + x3, t3 = x1 - x4, t4 = x2 - x3:
// X1,4 = x0 + c1 t1 + c2 t2 -+ i (s1 t3 + s2 t4), X2,3 = x0 + c2 t1 + c1 t2 -+ i (s2 t3 - s1 t4),
// c_k = cos(2 pi k / 5), s_k = sin(2 pi k / 5); the inverse swaps the signs of the i terms.
template <typename C2, bool INV>
__host__ __device__ __forceinline__ void dft5(C2 (&v)[5]) {
  using T = decltype(C2().x);
  const T c1 = (T)cos_pi60(24), c2 = (T)cos_pi60(48);   // cos(2 pi / 5), cos(4 pi / 5)
  const T s1 = (T)cos_pi60(6), s2 = (T)cos_pi60(18);    // sin(2 pi / 5), sin(4 pi / 5)
  const C2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  const C2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  const C2 a1 = mk2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
  const C2 a2 = mk2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
  const C2 b1 = mk2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
  const C2 b2 = mk2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
  // -+ i b
  const C2 q1 = INV ? mk2(-b1.y, b1.x) : mk2(b1.y, -b1.x);
  const C2 q2 = INV ? mk2(-b2.y, b2.x) : mk2(b2.y, -b2.x);
  v[0] = cadd(v[0], cadd(t1, t2));
  v[1] = cadd(a1, q1);
  v[4] = csub(a1, q1);
  v[2] = cadd(a2, q2);
  v[3] = csub(a2, q2);
}

template <typename C2, int R, bool INV>
__host__ __device__ __forceinline__ void dft_any(C2 (&v)[R]);

// DFT of N = M P points (M = 3 or 5, P a power of two) by one Cooley-Tukey step: with
// n = P n1 + n2 and k = k1 + M k2, X[k] = sum_{n2} W_N^{n2 k1} W_P^{n2 k2} sum_{n1} x[n] W_M^{n1 k1}.
template <typename C2, int M, int P, bool INV>
__host__ __device__ __forceinline__ void dft_mixed(C2 (&v)[M * P]) {
  constexpr int N = M * P;
#pragma unroll
  for (int n2 = 0; n2 < P; ++n2) {
    C2 t[M];
#pragma unroll
    for (int n1 = 0; n1 < M; ++n1) t[n1] = v[P * n1 + n2];
    dft_any<C2, M, INV>(t);
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) v[P * k1 + n2] = t[k1];
  }
#pragma unroll
  for (int k1 = 1; k1 < M; ++k1)
#pragma unroll
    for (int n2 = 1; n2 < P; ++n2) v[P * k1 + n2] = cmul(v[P * k1 + n2], root_n<C2, N, INV>(n2 * k1));
  C2 out[N];
#pragma unroll
  for (int k1 = 0; k1 < M; ++k1) {
    C2 t[P];
#pragma unroll
    for (int n2 = 0; n2 < P; ++n2) t[n2] = v[P * k1 + n2];
    dft_reg<C2, P, INV>(t);
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) out[k1 + M * k2] = t[k2];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = out[i];
}

template <typename C2, int R, bool INV>
__host__ __device__ __forceinline__ void dft_any(C2 (&v)[R]) {
  if constexpr ((R & (R - 1)) == 0) dft_reg<C2, R, INV>(v);
  else if constexpr (R == 3) dft3<C2, INV>(v);
  else if constexpr (R == 5) dft5<C2, INV>(v);
  else if constexpr (R % 3 == 0) dft_mixed<C2, 3, R / 3, INV>(v);
  else dft_mixed<C2, 5, R / 5, INV>(v);
}

// e^{-+2 pi i m / L} from the two tables (m < L)
template <typename C2>
__device__ __forceinline__ C2 tw_at(const C2* hi, const C2* lo, int m, bool inv) {
  const C2 a = hi[m >> 7], b = lo[m & (kTwLo - 1)];
  C2 w = cmul(a, b);
  if (inv) w.y = -w.y;
  return w;
}

// Global twiddle tables e^{-2 pi i j / len} for lengths 2^A, 3 2^A3 and 5 2^A5; a length
// m 2^a reads the table of its odd factor m with stride len / L.
template <typename C2>
struct TwSrc {
  const C2* t[3];
  int64_t len[3];
};

__device__ __forceinline__ int odd_slot(int L) {
  const int m = L >> (__ffs(L) - 1);
  return m == 1 ? 0 : (m == 3 ? 1 : 2);
}

// Fills the hi / lo tables for length L (one block, all threads).
template <typename C2>
__device__ void fft_tables(C2* hi, C2* lo, int L, const TwSrc<C2>& src) {
  const int q = odd_slot(L);
  const C2* __restrict__ tw = src.t[q];
  const int64_t step = src.len[q] / L;
  for (int i = threadIdx.x; i < kTwLo; i += blockDim.x) lo[i] = tw[(int64_t)(i % L) * step];
  for (int i = threadIdx.x; i * kTwLo < L; i += blockDim.x) hi[i] = tw[(int64_t)i * kTwLo * step];
}

// One pass over a row by the nthr threads t = 0..nthr-1 given to it (act false: the thread has
// no row this time and only takes part in the barriers); E bounds the values a thread holds.
template <typename C2, int R, bool INV, int E = fft_per_thread<C2>()>
__device__ __forceinline__ void stockham_pass(C2* buf, int L, int Ns, const C2* hi, const C2* lo, int t, int nthr,
                                              bool act) {
  constexpr int J = E / R > 0 ? E / R : 1;   // butterflies per thread at most
  const int B = act ? L / R : 0;             // butterflies of the pass
  const int tstride = L / (Ns * R);          // twiddle index scale: w^(r k) = e^{-2 pi i r k tstride / L}
  C2 v[J][R];
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int j = t + q * nthr;
    if (j < B) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = buf[fpad(j + r * B)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int j = t + q * nthr;
    if (j < B) {
      const int k = j & (Ns - 1);
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], tw_at(hi, lo, r * k * tstride, INV));
      }
      dft_any<C2, R, INV>(v[q]);
      const int base = (j - k) * R + k;   // (j div Ns) Ns R + k
#pragma unroll
      for (int r = 0; r < R; ++r) buf[fpad(base + r * Ns)] = v[q][r];
    }
  }
  __syncthreads();
}

// a pass of radix 2^b (1 <= b < log2 E)
template <typename C2, bool INV, int E = fft_per_thread<C2>()>
__device__ __forceinline__ void pow2_pass(C2* buf, int L, int Ns, int b, const C2* hi, const C2* lo, int t, int nthr,
                                          bool act) {
  switch (b) {
    case 1: stockham_pass<C2, 2, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
    case 2: stockham_pass<C2, 4, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
    case 3: stockham_pass<C2, 8, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
    case 4:
      if constexpr (E > 16) stockham_pass<C2, 16, INV, E>(buf, L, Ns, hi, lo, t, nthr, act);
      break;
    default: break;
  }
}

// Radix plan of a row of length L = m 2^a (m in {1, 3, 5}, L >= 32): `pass(R)` for each pass in
// order.  Radix E while E points remain in the power-of-two part, then the rest of it with m in
// one pass of radix m 2^b if that is at most E points, else a radix-2^b pass and a radix-m pass.
template <int E, class F>
__host__ __device__ __forceinline__ void fft_plan(int L, F pass) {
  constexpr int LE = E == 32 ? 5 : E == 16 ? 4 : 3;
  int a = 0;
  while (((L >> a) & 1) == 0) ++a;
  const int m = L >> a;
  int rem = a;
  while (rem >= LE) {
    pass(E);
    rem -= LE;
  }
  if (m == 1) {
    if (rem > 0) pass(1 << rem);
    return;
  }
  if ((m << rem) <= E) {
    pass(m << rem);
    return;
  }
  if (rem > 0) pass(1 << rem);
  pass(m);
}

// Threads one row of length L needs so that no thread has more than E / R butterflies of a
// radix-R pass, rounded up to whole warps.
template <typename C2, int E = fft_per_thread<C2>()>
__host__ __device__ inline int fft_threads(int L) {
  int need = 32;
  fft_plan<E>(L, [&](int R) {
    const int J = E / R > 0 ? E / R : 1;
    const int q = (L / R + J - 1) / J;
    if (q > need) need = q;
  });
  return (need + 31) / 32 * 32;
}

// Full transform of one row of length L = m 2^a (m in {1, 3, 5}, L >= 32) in buf (padded
// layout) by threads t = 0..nthr-1, nthr >= fft_threads(L); threads with act false take part
// in the barriers only.  (inlined: the caller must leave it about 100 registers)
template <typename C2, bool INV, int E = fft_per_thread<C2>()>
__device__ __forceinline__ void fft_row(C2* buf, int L, const C2* hi, const C2* lo, int t, int nthr, bool act) {
  constexpr int LE = E == 32 ? 5 : E == 16 ? 4 : 3;
  const int a = __ffs(L) - 1;
  const int m = L >> a;
  int Ns = 1, rem = a;
  while (rem >= LE) {
    stockham_pass<C2, E, INV, E>(buf, L, Ns, hi, lo, t, nthr, act);
    Ns <<= LE;
    rem -= LE;
  }
  if (m == 1) {
    pow2_pass<C2, INV, E>(buf, L, Ns, rem, hi, lo, t, nthr, act);
    return;
  }
  const int mp = m << rem;
  if (mp <= E) {
    switch (mp) {
      case 3: stockham_pass<C2, 3, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
      case 5: stockham_pass<C2, 5, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
      case 6: stockham_pass<C2, 6, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
      case 10: stockham_pass<C2, 10, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
      case 12: stockham_pass<C2, 12, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
      case 20: if constexpr (E >= 20) stockham_pass<C2, 20, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
      case 24: if constexpr (E >= 24) stockham_pass<C2, 24, INV, E>(buf, L, Ns, hi, lo, t, nthr, act); break;
      default: break;
    }
    return;
  }
  pow2_pass<C2, INV, E>(buf, L, Ns, rem, hi, lo, t, nthr, act);
  Ns <<= rem;
  if (m == 3) stockham_pass<C2, 3, INV, E>(buf, L, Ns, hi, lo, t, nthr, act);
  else stockham_pass<C2, 5, INV, E>(buf, L, Ns, hi, lo, t, nthr, act);
}

// the same by the whole block
template <typename C2, bool INV>
__device__ __forceinline__ void fft_row(C2* buf, int L, const C2* hi, const C2* lo) {
  fft_row<C2, INV>(buf, L, hi, lo, (int)threadIdx.x, (int)blockDim.x, true);
}

}  // namespace sfft
