// Batched prime-length DFT (Eq. 3) by Bluestein's chirp-z identity over
// power-of-two FFTs held in shared memory.
//
//   Y[h] = sum_{x<p} y[x] e^{-2 pi i h x / p}
//        = e^{-pi i h^2/p} sum_{x<p} (y[x] e^{-pi i x^2/p}) e^{+pi i (h-x)^2/p},
// a cyclic convolution of length L = 2^ceil(log2(2p-1)) of a[x] = y[x] chirp[x]
// (zero for x >= p) with b[m] = conj(chirp[|m|]) on |m| < p (wrapped mod L),
// where chirp[x] = e^{-pi i (x^2 mod 2p)/p} comes from the per-prime table.
//
// L <= 4096: one block per row does FFT(a), FFT(b), product, inverse FFT.
// L  > 4096: four-step split L = M1 * M2, x = M2 x1 + x2, k = k1 + M1 k2:
//   pass A (per column x2):  Z[k1][x2] = e^{-2 pi i x2 k1 / L} FFT_{M1}(a[M2 x1 + x2])[k1]
//                            (the filter b rides along as one extra row)
//   pass B (per row k1):     X = FFT_{M2}(Z[k1][.]), X *= B^[k1][.],
//                            Z[k1][x2] = e^{+2 pi i x2 k1 / L} IFFT_{M2}(X)[x2]
//   pass C (per column x2):  c[M2 x1 + x2] = IFFT_{M1}(Z[.][x2])[x1],  Y[h] = chirp[h] c[h] / L
// Forward FFTs are radix-2 decimation in time (bit-reversed in, natural out),
// inverse FFTs decimation in frequency (natural in, bit-reversed out), so no
// explicit permutation pass is needed.  Twiddles come from one table
// twG[m] = e^{-2 pi i m / Lmax}, built in double and rounded once.
#include "sfft_internal.cuh"

namespace sfft {

namespace {

__device__ __forceinline__ int brev(int x, int logM) {
  return logM == 0 ? 0 : (int)(__brev((unsigned)x) >> (32 - logM));
}

// In-place radix-2 DIT over `nlines` lines of length 2^logM, line l at buf + l * ls.
// Input bit-reversed, output natural.  tw[j] = e^{-2 pi i j / M}, j < M/2.
template <typename C2>
__device__ void dit_stages(C2* buf, int ls, int logM, int nlines, const C2* tw, bool inv) {
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
__device__ void dif_stages(C2* buf, int ls, int logM, int nlines, const C2* tw, bool inv) {
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

template <typename C2>
__device__ __forceinline__ C2 sum_partials(const C2* __restrict__ part, int splits, int64_t stride, int64_t off) {
  C2 acc = part[off];
  for (int s = 1; s < splits; ++s) acc = cadd(acc, part[(int64_t)s * stride + off]);
  return acc;
}

// value of the Bluestein filter b at position x of the length-L convolution
template <typename C2>
__device__ __forceinline__ C2 filter_at(int64_t x, int64_t p, int64_t L, const C2* __restrict__ chirp) {
  if (x < p) return cconj(chirp[x]);
  if (x > L - p) return cconj(chirp[L - x]);
  return mk2(decltype(C2().x)(0), decltype(C2().x)(0));
}

__device__ __forceinline__ void atomic_max_abs(DevState* st, double v) {
  atomicMax(&st->max_y0_bits, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__device__ __forceinline__ void warp_max_to_state(DevState* st, double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > 0.0) atomic_max_abs(st, v);
}

template <typename T>
__global__ void bluestein_single_kernel(int64_t p, int logL, int n_rows, int splits, const c2<T>* __restrict__ part,
                                        const c2<T>* __restrict__ chirp, const c2<T>* __restrict__ twG, int64_t Lmax,
                                        c2<T>* __restrict__ Y, DevState* st) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* buf = reinterpret_cast<C2*>(smem_raw);   // [0, L): data, [L, 2L): filter
  const int L = 1 << logL;
  C2* tw = buf + 2 * L;
  const int row = blockIdx.x;
  const int64_t tstep = Lmax >> logL;
  const int64_t pstride = (int64_t)n_rows * p;
  for (int j = threadIdx.x; j < L / 2; j += blockDim.x) tw[j] = twG[j * tstep];
  for (int x = threadIdx.x; x < L; x += blockDim.x) {
    const int r = brev(x, logL);
    C2 a = mk2((T)0, (T)0);
    if (x < p) a = cmul(chirp[x], sum_partials(part, splits, pstride, (int64_t)row * p + x));
    buf[r] = a;
    buf[L + r] = filter_at(x, p, L, chirp);
  }
  __syncthreads();
  dit_stages(buf, L, logL, 2, tw, false);
  for (int k = threadIdx.x; k < L; k += blockDim.x) buf[k] = cmul(buf[k], buf[L + k]);
  __syncthreads();
  dif_stages(buf, L, logL, 1, tw, true);
  const T invL = (T)1 / (T)L;
  for (int h0 = 0; h0 < p; h0 += blockDim.x) {
    const int h = h0 + threadIdx.x;
    double m = 0.0;
    if (h < p) {
      const C2 v = cmul(chirp[h], cscale(buf[brev(h, logL)], invL));
      Y[(int64_t)row * p + h] = v;
      m = hypot((double)v.x, (double)v.y);
    }
    if (row == 0 && st != nullptr) warp_max_to_state<T>(st, m);
  }
}

// pass A: column FFTs of the chirp-multiplied data (rows < n_rows) and of the filter (row n_rows)
template <typename T>
__global__ void bluestein_colfwd_kernel(int64_t p, int logM1, int logM2, int CT, int n_rows, int splits,
                                        const c2<T>* __restrict__ part, const c2<T>* __restrict__ chirp,
                                        const c2<T>* __restrict__ twG, int64_t Lmax, c2<T>* __restrict__ Z) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M1 = 1 << logM1, M2 = 1 << logM2, logL = logM1 + logM2;
  const int64_t L = (int64_t)M1 * M2;
  const int ls = M1 + 1;
  C2* buf = reinterpret_cast<C2*>(smem_raw);
  C2* tw = buf + CT * ls;
  const int row = blockIdx.y;
  const int x2_0 = blockIdx.x * CT;
  const int64_t pstride = (int64_t)n_rows * p;
  for (int j = threadIdx.x; j < M1 / 2; j += blockDim.x) tw[j] = twG[(int64_t)j * (Lmax >> logM1)];
  for (int e = threadIdx.x; e < CT * M1; e += blockDim.x) {
    const int x1 = e / CT, c = e - x1 * CT;
    const int64_t x = (int64_t)x1 * M2 + x2_0 + c;
    C2 v;
    if (row < n_rows) {
      v = mk2((T)0, (T)0);
      if (x < p) v = cmul(chirp[x], sum_partials(part, splits, pstride, (int64_t)row * p + x));
    } else {
      v = filter_at(x, p, L, chirp);
    }
    buf[c * ls + brev(x1, logM1)] = v;
  }
  __syncthreads();
  dit_stages(buf, ls, logM1, CT, tw, false);
  const int64_t tstep = Lmax >> logL;
  for (int e = threadIdx.x; e < CT * M1; e += blockDim.x) {
    const int k1 = e / CT, c = e - k1 * CT;
    const int64_t x2 = x2_0 + c;
    const int64_t m = (x2 * k1) & (L - 1);
    Z[(int64_t)row * L + (int64_t)k1 * M2 + x2] = cmul(buf[c * ls + k1], twG[m * tstep]);
  }
}

// pass B: row FFT, product with the filter spectrum, inverse row FFT
template <typename T>
__global__ void bluestein_rows_kernel(int logM1, int logM2, int RT, int n_rows, const c2<T>* __restrict__ twG,
                                      int64_t Lmax, c2<T>* __restrict__ Z) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M2 = 1 << logM2, logL = logM1 + logM2;
  const int64_t L = (int64_t)M2 << logM1;
  const int ls = M2 + 1;
  C2* bufA = reinterpret_cast<C2*>(smem_raw);   // RT data rows then RT filter rows
  C2* bufF = bufA + RT * ls;
  C2* tw = bufA + 2 * RT * ls;
  const int row = blockIdx.y;
  const int k1_0 = blockIdx.x * RT;
  for (int j = threadIdx.x; j < M2 / 2; j += blockDim.x) tw[j] = twG[(int64_t)j * (Lmax >> logM2)];
  for (int e = threadIdx.x; e < RT * M2; e += blockDim.x) {
    const int r = e / M2, x2 = e - r * M2;
    const int64_t off = (int64_t)(k1_0 + r) * M2 + x2;
    bufA[r * ls + brev(x2, logM2)] = Z[(int64_t)row * L + off];
    bufF[r * ls + brev(x2, logM2)] = Z[(int64_t)n_rows * L + off];
  }
  __syncthreads();
  dit_stages(bufA, ls, logM2, 2 * RT, tw, false);
  for (int e = threadIdx.x; e < RT * M2; e += blockDim.x) {
    const int r = e / M2, k2 = e - r * M2;
    bufA[r * ls + k2] = cmul(bufA[r * ls + k2], bufF[r * ls + k2]);
  }
  __syncthreads();
  dif_stages(bufA, ls, logM2, RT, tw, true);
  const int64_t tstep = Lmax >> logL;
  for (int e = threadIdx.x; e < RT * M2; e += blockDim.x) {
    const int r = e / M2, x2 = e - r * M2;
    const int64_t k1 = k1_0 + r;
    const int64_t m = ((int64_t)x2 * k1) & (L - 1);
    Z[(int64_t)row * L + k1 * M2 + x2] = cmul(bufA[r * ls + brev(x2, logM2)], cconj(twG[m * tstep]));
  }
}

// pass C: inverse column FFTs, chirp post-multiply, first p outputs
template <typename T>
__global__ void bluestein_colinv_kernel(int64_t p, int logM1, int logM2, int CT, const c2<T>* __restrict__ chirp,
                                        const c2<T>* __restrict__ twG, int64_t Lmax, const c2<T>* __restrict__ Z,
                                        c2<T>* __restrict__ Y, DevState* st) {
  using C2 = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M1 = 1 << logM1, M2 = 1 << logM2;
  const int64_t L = (int64_t)M1 * M2;
  const int ls = M1 + 1;
  C2* buf = reinterpret_cast<C2*>(smem_raw);
  C2* tw = buf + CT * ls;
  const int row = blockIdx.y;
  const int x2_0 = blockIdx.x * CT;
  for (int j = threadIdx.x; j < M1 / 2; j += blockDim.x) tw[j] = twG[(int64_t)j * (Lmax >> logM1)];
  for (int e = threadIdx.x; e < CT * M1; e += blockDim.x) {
    const int k1 = e / CT, c = e - k1 * CT;
    buf[c * ls + k1] = Z[(int64_t)row * L + (int64_t)k1 * M2 + x2_0 + c];
  }
  __syncthreads();
  dif_stages(buf, ls, logM1, CT, tw, true);
  const T invL = (T)1 / (T)L;
  const int total = CT * M1;
  for (int e0 = 0; e0 < total; e0 += blockDim.x) {
    const int e = e0 + threadIdx.x;
    double m = 0.0;
    if (e < total) {
      const int x1 = e / CT, c = e - x1 * CT;
      const int64_t x = (int64_t)x1 * M2 + x2_0 + c;
      if (x < p) {
        const C2 v = cmul(chirp[x], cscale(buf[c * ls + brev(x1, logM1)], invL));
        Y[(int64_t)row * p + x] = v;
        m = hypot((double)v.x, (double)v.y);
      }
    }
    if (row == 0 && st != nullptr) warp_max_to_state<T>(st, m);
  }
}

int pow2_floor(int64_t v) {
  int r = 1;
  while ((int64_t)r * 2 <= v) r *= 2;
  return r;
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

DftGeom dft_geometry(int64_t p) {
  DftGeom g;
  g.L = 2;
  g.logL = 1;
  while (g.L < 2 * p - 1) {
    g.L *= 2;
    g.logL += 1;
  }
  g.single = g.L <= kSingleMaxL;
  g.logM1 = g.logL / 2;
  g.logM2 = g.logL - g.logM1;
  return g;
}

template <typename T>
cudaError_t launch_bluestein(cudaStream_t st, const DftGeom& g, int64_t p, int n_rows, int splits,
                             const c2<T>* part, const c2<T>* chirp, const c2<T>* twG, int64_t Lmax, c2<T>* Z,
                             c2<T>* Y, DevState* state) {
  using C2 = c2<T>;
  cudaError_t e;
  if (g.single) {
    const int L = (int)g.L;
    const size_t smem = (size_t)(2 * L + L / 2) * sizeof(C2);
    if ((e = allow_smem(bluestein_single_kernel<T>, smem)) != cudaSuccess) return e;
    const int threads = L >= 512 ? 256 : 128;
    bluestein_single_kernel<T><<<n_rows, threads, smem, st>>>(p, g.logL, n_rows, splits, part, chirp, twG, Lmax, Y,
                                                               state);
    return cudaGetLastError();
  }
  const int M1 = 1 << g.logM1, M2 = 1 << g.logM2;
  // column tile: enough blocks to spread over the GPU, at most kFftSmemElems elements per block
  int CT = pow2_floor(std::max<int64_t>(1, (int64_t)M2 * (n_rows + 1) / 296));
  CT = std::min(CT, std::max(1, kFftSmemElems / M1));
  CT = std::max(CT, std::min(4, M2));
  CT = std::min(CT, M2);
  int RT = pow2_floor(std::max<int64_t>(1, (int64_t)M1 * n_rows / 296));
  RT = std::min(RT, std::max(1, (kFftSmemElems / 2) / M2));
  RT = std::min(RT, M1);
  const size_t smemA = (size_t)(CT * (M1 + 1) + M1 / 2) * sizeof(C2);
  const size_t smemB = (size_t)(2 * RT * (M2 + 1) + M2 / 2) * sizeof(C2);
  if ((e = allow_smem(bluestein_colfwd_kernel<T>, smemA)) != cudaSuccess) return e;
  if ((e = allow_smem(bluestein_rows_kernel<T>, smemB)) != cudaSuccess) return e;
  if ((e = allow_smem(bluestein_colinv_kernel<T>, smemA)) != cudaSuccess) return e;
  const int thrA = std::min(256, std::max(32, CT * M1 / 2));
  const int thrB = std::min(256, std::max(32, RT * M2));
  bluestein_colfwd_kernel<T><<<dim3(M2 / CT, n_rows + 1), thrA, smemA, st>>>(p, g.logM1, g.logM2, CT, n_rows, splits,
                                                                             part, chirp, twG, Lmax, Z);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bluestein_rows_kernel<T><<<dim3(M1 / RT, n_rows), thrB, smemB, st>>>(g.logM1, g.logM2, RT, n_rows, twG, Lmax, Z);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bluestein_colinv_kernel<T><<<dim3(M2 / CT, n_rows), thrA, smemA, st>>>(p, g.logM1, g.logM2, CT, chirp, twG, Lmax,
                                                                         Z, Y, state);
  return cudaGetLastError();
}

template cudaError_t launch_bluestein<float>(cudaStream_t, const DftGeom&, int64_t, int, int, const float2*,
                                             const float2*, const float2*, int64_t, float2*, float2*, DevState*);
template cudaError_t launch_bluestein<double>(cudaStream_t, const DftGeom&, int64_t, int, int, const double2*,
                                              const double2*, const double2*, int64_t, double2*, double2*,
                                              DevState*);

}  // namespace sfft
