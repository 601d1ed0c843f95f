// Stockham auto-sort FFT of one row held in shared memory, with each pass's
// radix-R butterflies done in registers.
//
// For a length L = 2^n (n >= 5) the passes use radix E (32 in float, 16 in
// double) while E points remain per transform, then one smaller power of two.  Pass with
// stride Ns (product of the earlier radices) and radix R, for j = 0..L/R-1:
//     v[r] = x[j + r L/R] * w^(r k),  k = j mod Ns,  w = e^{-+2 pi i / (Ns R)}
//     v    = DFT_R(v)
//     x'[(j div Ns) Ns R + k + r Ns] = v[r]
// which leaves the transform in natural order after the last pass.  Every thread
// handles E values per pass (E / R indices j), so L / E threads take part; all
// of a pass's values are read before the barrier and written after it, so one
// buffer suffices.  Rows use the padded index e + e / 32: the only pass whose
// writes stride by 32 (Ns = 1) then hits distinct banks.  Twiddles e^{-2 pi i m / L}
// come from two 128-entry tables, e^{-2 pi i m / L} = hi[m >> 7] * lo[m & 127].
#pragma once

#include "sfft_internal.cuh"

namespace sfft {

constexpr int kTwLo = 128;          // entries of the low twiddle table
constexpr int kFftThreads = 512;    // block size of the one-row FFT kernels

// complex values per thread and pass: 32 in float, 16 in double (same register bytes)
template <typename C2> __host__ __device__ constexpr int fft_per_thread() { return sizeof(C2) == 8 ? 32 : 16; }

__device__ __forceinline__ int fpad(int e) { return e + (e >> 5); }

// cos(pi m / 16), m = 0..16: the unit roots of order 32 used inside the register DFTs
__device__ __forceinline__ double cos_pi16(int m) {
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

// In-register DFT of R points (R a power of two <= 32), forward (e^{-2 pi i}) or inverse.
// Radix-2 decimation in time on the bit-reversed register order; all indices are
// compile-time constants, so the permutation costs nothing.
template <typename C2, int R, bool INV>
__device__ __forceinline__ void dft_reg(C2 (&v)[R]) {
  using T = decltype(C2().x);
  constexpr int LG = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5;
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
        const int m = (16 * t) / s;   // 0..31 in units of pi / 16
        const C2 a = v[g + t];
        C2 b = v[g + t + s];
        if (t != 0) {
          // m < 16: cos(pi m / 16) and sin(pi m / 16) = cos(pi |8 - m| / 16)
          const T c = (T)cos_pi16(m);
          const T sn = (T)cos_pi16(m <= 8 ? 8 - m : m - 8);
          // w = c - i sn (forward) or c + i sn (inverse), sn = sin(pi m / 16)
          const T wy = INV ? sn : -sn;
          b = mk2(b.x * c - b.y * wy, b.x * wy + b.y * c);
        }
        v[g + t] = cadd(a, b);
        v[g + t + s] = csub(a, b);
      }
    }
  }
}

// e^{-+2 pi i m / L} from the two tables (m < L)
template <typename C2>
__device__ __forceinline__ C2 tw_at(const C2* hi, const C2* lo, int m, bool inv) {
  const C2 a = hi[m >> 7], b = lo[m & (kTwLo - 1)];
  C2 w = cmul(a, b);
  if (inv) w.y = -w.y;
  return w;
}

// Builds the twiddle tables for length L from twG (e^{-2 pi i m / Lmax}, m < Lmax).
template <typename C2>
__device__ void fft_tables(C2* hi, C2* lo, int logL, const C2* __restrict__ twG, int64_t Lmax) {
  const int L = 1 << logL;
  const int64_t step = Lmax >> logL;
  for (int i = threadIdx.x; i < kTwLo; i += blockDim.x) lo[i] = twG[(int64_t)(i & (L - 1)) * step];
  for (int i = threadIdx.x; i * kTwLo < L; i += blockDim.x) hi[i] = twG[(int64_t)i * kTwLo * step];
}

template <typename C2, int R, bool INV>
__device__ __forceinline__ void stockham_pass(C2* buf, int L, int Ns, const C2* hi, const C2* lo) {
  constexpr int E = fft_per_thread<C2>();
  constexpr int J = E / R;
  const int nthr = L / E;
  const int t = threadIdx.x;
  const int LR = L / R;
  const int tstride = L / (Ns * R);   // twiddle index scale: w^(r k) = e^{-2 pi i r k tstride / L}
  C2 v[J][R];
  if (t < nthr) {
#pragma unroll
    for (int q = 0; q < J; ++q) {
      const int j = t + q * nthr;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = buf[fpad(j + r * LR)];
    }
  }
  __syncthreads();
  if (t < nthr) {
#pragma unroll
    for (int q = 0; q < J; ++q) {
      const int j = t + q * nthr;
      const int k = j & (Ns - 1);
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], tw_at(hi, lo, r * k * tstride, INV));
      }
      dft_reg<C2, R, INV>(v[q]);
      const int base = (j - k) * R + k;   // (j div Ns) Ns R + k
#pragma unroll
      for (int r = 0; r < R; ++r) buf[fpad(base + r * Ns)] = v[q][r];
    }
  }
  __syncthreads();
}

// Full transform of one row of length L = 2^logL (5 <= logL) in buf (padded layout).
// (inlined: the caller must leave it about 100 registers)
template <typename C2, bool INV>
__device__ __forceinline__ void fft_row(C2* buf, int logL, const C2* hi, const C2* lo) {
  constexpr int E = fft_per_thread<C2>();
  constexpr int LE = E == 32 ? 5 : 4;
  const int L = 1 << logL;
  int Ns = 1, rem = logL;
  while (rem >= LE) {
    stockham_pass<C2, E, INV>(buf, L, Ns, hi, lo);
    Ns <<= LE;
    rem -= LE;
  }
  switch (rem) {
    case 1: stockham_pass<C2, 2, INV>(buf, L, Ns, hi, lo); break;
    case 2: stockham_pass<C2, 4, INV>(buf, L, Ns, hi, lo); break;
    case 3: stockham_pass<C2, 8, INV>(buf, L, Ns, hi, lo); break;
    case 4: stockham_pass<C2, 16, INV>(buf, L, Ns, hi, lo); break;
    default: break;
  }
}

}  // namespace sfft
