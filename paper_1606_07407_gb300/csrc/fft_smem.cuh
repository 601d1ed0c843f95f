// Radix-2 FFT stages on lines held in shared memory, shared by the DFT kernels.
//
// Forward transforms use decimation in time (bit-reversed input, natural
// output); inverse transforms decimation in frequency (natural input,
// bit-reversed output), so a forward-multiply-inverse sequence needs no
// permutation pass.  tw[j] = e^{-2 pi i j / M}, j < M/2, for a line of length M.
#pragma once

#include "sfft_internal.cuh"

namespace sfft {

__device__ __forceinline__ int brev_bits(int x, int logM) {
  return logM == 0 ? 0 : (int)(__brev((unsigned)x) >> (32 - logM));
}

// In-place radix-2 DIT over `nlines` lines of length 2^logM at buf + l * ls.
template <typename C2>
__device__ void fft_dit(C2* buf, int ls, int logM, int nlines, const C2* tw, bool inv) {
  const int half = 1 << (logM - 1);
  const int nbf = half * nlines;
  for (int s = 0; s < logM; ++s) {
    const int hs = 1 << s;
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
      const int line = b >> (logM - 1);
      const int t = b & (half - 1);
      const int j = t & (hs - 1);
      const int i = ((t >> s) << (s + 1)) | j;
      C2 w = tw[j << (logM - 1 - s)];
      if (inv) w.y = -w.y;
      C2* base = buf + line * ls;
      const C2 a = base[i];
      const C2 c = cmul(w, base[i + hs]);
      base[i] = cadd(a, c);
      base[i + hs] = csub(a, c);
    }
    __syncthreads();
  }
}

// In-place radix-2 DIF: natural input, bit-reversed output.
template <typename C2>
__device__ void fft_dif(C2* buf, int ls, int logM, int nlines, const C2* tw, bool inv) {
  const int half = 1 << (logM - 1);
  const int nbf = half * nlines;
  for (int s = logM - 1; s >= 0; --s) {
    const int hs = 1 << s;
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
      const int line = b >> (logM - 1);
      const int t = b & (half - 1);
      const int j = t & (hs - 1);
      const int i = ((t >> s) << (s + 1)) | j;
      C2 w = tw[j << (logM - 1 - s)];
      if (inv) w.y = -w.y;
      C2* base = buf + line * ls;
      const C2 a = base[i];
      const C2 c = base[i + hs];
      base[i] = cadd(a, c);
      base[i + hs] = cmul(w, csub(a, c));
    }
    __syncthreads();
  }
}

}  // namespace sfft
