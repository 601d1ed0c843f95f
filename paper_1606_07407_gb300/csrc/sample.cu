// Round setup, per-prime tables, mode projection and the sample-and-residual
// kernel (the black-box sampling of f - g along the line and its shifted copies).
//
// Sampling (Alg. 2 sampling lines; Eq. 41, general form): for x < p and n <= d
//     y_n[x] = sum_j C[n][j] * exp(2 pi i ((alpha_j x) mod p) / p),
//     alpha_j = (w_j . u) mod p,  C[0][j] = a_j,  C[n][j] = a_j exp(2 pi i w_{j,n} / N),
// which is f(x u/p + s_n) with s_n = e_n / N, because f is 1-periodic in every
// coordinate and w_j . (x u / p + s_n) = x (w_j . u) / p + w_{j,n} / N.  Registry
// modes carry -a, so one pass gives f - g.  The phase index (alpha_j x) mod p is
// reduced exactly in integers; the unit root it selects is the product of two
// entries of the table W[i] = exp(2 pi i i / p) (built in double, rounded once):
//     x = x_tile + 32 row + lane:  W[(alpha x) mod p] = W[(alpha (x_tile + 32 row)) mod p] * W[(alpha lane) mod p].
// The first factor is the same for the 32 lanes of a row, the second for every
// row of a lane, so each (mode, sample) term costs one complex product to form
// the unit root and one complex multiply-add per sample set.
#include "sfft_internal.cuh"

namespace sfft {

namespace {

// a mod p for 0 <= a < 64 p < 2^31, via a float reciprocal and one correction.
__device__ __forceinline__ int mod_small(unsigned a, int p, float inv_p) {
  int q = __float2int_rz(__uint2float_rn(a) * inv_p);
  int r = (int)a - q * p;
  if (r < 0) r += p;
  else if (r >= p) r -= p;
  return r;
}

__global__ void round_begin_kernel(DevState* st, const int64_t* dirs, int dir_index, int d, int64_t p,
                                   int64_t* u_mod) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->max_y0_bits = 0ull;
    st->n_acc = 0;
    st->n_live = 0;
    st->any_occupied = 0;
  }
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < d; l += gridDim.x * blockDim.x) {
    int64_t v = dirs[(int64_t)dir_index * d + l] % p;
    u_mod[l] = v < 0 ? v + p : v;
  }
}

template <typename T>
__global__ void prime_tables_kernel(int64_t p, c2<T>* W, c2<T>* chirp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
    // W[i] = exp(2 pi i i / p), argument folded into (-1, 1] half-turns
    int64_t ii = (2 * i > p) ? i - p : i;
    double s, c;
    sincospi(2.0 * (double)ii / (double)p, &s, &c);
    W[i] = mk2((T)c, (T)s);
    // chirp[x] = exp(-pi i x^2 / p) with x^2 reduced mod 2p exactly
    unsigned long long q = ((unsigned long long)i * (unsigned long long)i) % (unsigned long long)(2 * p);
    int64_t qq = (int64_t)q > p ? (int64_t)q - 2 * p : (int64_t)q;
    sincospi(-(double)qq / (double)p, &s, &c);
    chirp[i] = mk2((T)c, (T)s);
  }
}

template <typename T>
__global__ void twiddle_kernel(int64_t Lmax, c2<T>* twG) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < Lmax; m += (int64_t)gridDim.x * blockDim.x) {
    int64_t mm = (2 * m > Lmax) ? m - Lmax : m;
    double s, c;
    sincospi(-2.0 * (double)mm / (double)Lmax, &s, &c);
    twG[m] = mk2((T)c, (T)s);
  }
}

template <typename T>
__global__ void project_kernel(int K_sig, int K_reg, int d, int64_t N, int64_t p, const int64_t* __restrict__ u_mod,
                               const int32_t* __restrict__ sig_w, const double2* __restrict__ sig_a,
                               const int32_t* __restrict__ reg_w, const double2* __restrict__ reg_a, int n_sets,
                               int Kpad, int32_t* __restrict__ alpha, c2<T>* __restrict__ C) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K_sig + K_reg) return;
  const int32_t* w;
  double2 a;
  if (j < K_sig) {
    w = sig_w + (int64_t)j * d;
    a = sig_a[j];
  } else {
    w = reg_w + (int64_t)(j - K_sig) * d;
    a = reg_a[j - K_sig];
    a.x = -a.x;   // g is subtracted: f - g
    a.y = -a.y;
  }
  int64_t acc = 0;
  for (int l = 0; l < d; ++l) {
    int64_t wm = (int64_t)w[l] % p;
    if (wm < 0) wm += p;
    acc = (acc + wm * u_mod[l]) % p;
  }
  alpha[j] = (int32_t)acc;
  C[j] = mk2((T)a.x, (T)a.y);
  for (int n = 1; n < n_sets; ++n) {
    int64_t wn = (int64_t)w[n - 1] % N;
    if (wn < 0) wn += N;
    int64_t wf = (2 * wn > N) ? wn - N : wn;   // half-turns folded into (-1, 1]
    double s, c;
    sincospi(2.0 * (double)wf / (double)N, &s, &c);
    C[(int64_t)n * Kpad + j] = mk2((T)(a.x * c - a.y * s), (T)(a.x * s + a.y * c));
  }
}

template <typename T, int NS>
__global__ void __launch_bounds__(kSampleWarps * 32)
sample_kernel(int p, int K, int n_sets, int Kpad, int jper, int gsize, const int32_t* __restrict__ alpha,
              const c2<T>* __restrict__ C, const c2<T>* __restrict__ W, c2<T>* __restrict__ part) {
  using C2 = c2<T>;
  constexpr int RW = kSampleRowsPerWarp;
  constexpr int NT = kSampleWarps * 32;
  __shared__ C2 Ls[kSampleChunk][32];
  __shared__ C2 Us[kSampleChunk][kSampleRows];
  __shared__ C2 Cs[kSampleChunk][NS];
  __shared__ int al_s[kSampleChunk], be_s[kSampleChunk], ga_s[kSampleChunk];

  const int xt = blockIdx.x, s = blockIdx.y, g = blockIdx.z;
  const int n0 = g * gsize;
  const int ns_valid = min(gsize, n_sets - n0);
  const int x0 = xt * kSampleTileX;
  const int j_begin = s * jper;
  const int j_end = min(K, j_begin + jper);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float inv_p = 1.0f / (float)p;
  const C2 zero = mk2((T)0, (T)0);

  T acc[RW][NS][2];
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int n = 0; n < NS; ++n) acc[r][n][0] = acc[r][n][1] = (T)0;

  for (int jc = j_begin; jc < j_end; jc += kSampleChunk) {
    const int nj = min(kSampleChunk, j_end - jc);
    if (tid < kSampleChunk) {
      const int a = (tid < nj) ? alpha[jc + tid] : 0;
      al_s[tid] = a;
      be_s[tid] = (int)(((unsigned long long)a * (unsigned long long)x0) % (unsigned long long)p);
      ga_s[tid] = mod_small((unsigned)a * 32u, p, inv_p);
    }
    for (int e = tid; e < kSampleChunk * NS; e += NT) {
      const int jj = e / NS, n = e - jj * NS;
      Cs[jj][n] = (jj < nj && n < ns_valid) ? C[(int64_t)(n0 + n) * Kpad + jc + jj] : zero;
    }
    __syncthreads();
    for (int e = tid; e < kSampleChunk * 32; e += NT) {
      const int jj = e >> 5, ln = e & 31;
      Ls[jj][ln] = W[mod_small((unsigned)al_s[jj] * (unsigned)ln, p, inv_p)];
    }
    for (int e = tid; e < kSampleChunk * kSampleRows; e += NT) {
      const int jj = e / kSampleRows, row = e - jj * kSampleRows;
      Us[jj][row] = W[mod_small((unsigned)be_s[jj] + (unsigned)row * (unsigned)ga_s[jj], p, inv_p)];
    }
    __syncthreads();
#pragma unroll 2
    for (int jj = 0; jj < kSampleChunk; ++jj) {
      const C2 L = Ls[jj][lane];
      C2 E[RW];
#pragma unroll
      for (int r = 0; r < RW; ++r) E[r] = cmul(Us[jj][warp * RW + r], L);
#pragma unroll
      for (int n = 0; n < NS; ++n) {
        const C2 c = Cs[jj][n];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
          acc[r][n][0] = fma(c.x, E[r].x, acc[r][n][0]);
          acc[r][n][0] = fma(-c.y, E[r].y, acc[r][n][0]);
          acc[r][n][1] = fma(c.x, E[r].y, acc[r][n][1]);
          acc[r][n][1] = fma(c.y, E[r].x, acc[r][n][1]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    const int x = x0 + (warp * RW + r) * 32 + lane;
    if (x < p) {
#pragma unroll
      for (int n = 0; n < NS; ++n)
        if (n < ns_valid) part[((int64_t)s * n_sets + n0 + n) * p + x] = mk2(acc[r][n][0], acc[r][n][1]);
    }
  }
}

template <typename T>
__global__ void reduce_partials_kernel(int64_t p, int n_sets, int splits, const c2<T>* __restrict__ part,
                                       c2<T>* __restrict__ y) {
  const int64_t total = (int64_t)n_sets * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    c2<T> acc = part[e];
    for (int s = 1; s < splits; ++s) acc = cadd(acc, part[(int64_t)s * total + e]);
    y[e] = acc;
  }
}

int grid_for(int64_t n, int threads, int cap = 65535 * 4) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace

cudaError_t launch_round_begin(cudaStream_t st, DevState* state, const int64_t* dirs, int dir_index, int d,
                               int64_t p, int64_t* u_mod) {
  round_begin_kernel<<<grid_for(d, 128, 64), 128, 0, st>>>(state, dirs, dir_index, d, p, u_mod);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prime_tables(cudaStream_t st, int64_t p, c2<T>* W, c2<T>* chirp) {
  prime_tables_kernel<T><<<grid_for(p, 256, 2048), 256, 0, st>>>(p, W, chirp);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_twiddles(cudaStream_t st, int64_t Lmax, c2<T>* twG) {
  twiddle_kernel<T><<<grid_for(Lmax, 256, 4096), 256, 0, st>>>(Lmax, twG);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project(cudaStream_t st, int K_sig, int K_reg, int d, int64_t N, int64_t p, const int64_t* u_mod,
                           const int32_t* sig_w, const double2* sig_a, const int32_t* reg_w, const double2* reg_a,
                           int n_sets, int Kpad, int32_t* alpha, c2<T>* C) {
  const int K = K_sig + K_reg;
  if (K == 0) return cudaSuccess;
  project_kernel<T><<<(K + 127) / 128, 128, 0, st>>>(K_sig, K_reg, d, N, p, u_mod, sig_w, sig_a, reg_w, reg_a,
                                                     n_sets, Kpad, alpha, C);
  return cudaGetLastError();
}

SampleGeom sample_geometry(int64_t p, int K, int n_sets, int64_t part_capacity_elems, int n_sm) {
  SampleGeom g;
  g.groups = (n_sets + kMaxSetGroup - 1) / kMaxSetGroup;
  g.gsize = (n_sets + g.groups - 1) / g.groups;
  g.n_xt = (int)((p + kSampleTileX - 1) / kSampleTileX);
  const int chunks = K > 0 ? (K + kSampleChunk - 1) / kSampleChunk : 1;
  const int64_t base = (int64_t)g.n_xt * g.groups;
  const int64_t target = 4LL * n_sm;
  int64_t splits = (target + base - 1) / base;
  if (splits > chunks) splits = chunks;
  const int64_t fit = part_capacity_elems / ((int64_t)n_sets * p);
  if (splits > fit) splits = fit;
  if (splits < 1) splits = 1;
  const int per = (int)((chunks + splits - 1) / splits);
  g.jper = per * kSampleChunk;
  g.splits = K > 0 ? (K + g.jper - 1) / g.jper : 1;
  return g;
}

template <typename T>
cudaError_t launch_sample(cudaStream_t st, const SampleGeom& g, int64_t p, int K, int n_sets, int Kpad,
                          const int32_t* alpha, const c2<T>* C, const c2<T>* W, c2<T>* part) {
  dim3 grid(g.n_xt, g.splits, g.groups);
  dim3 block(kSampleWarps * 32);
  const int ip = (int)p;
#define SFFT_SAMPLE_CASE(NS)                                                                          \
  case NS:                                                                                            \
    sample_kernel<T, NS><<<grid, block, 0, st>>>(ip, K, n_sets, Kpad, g.jper, g.gsize, alpha, C, W, part); \
    break;
  switch (g.gsize) {
    SFFT_SAMPLE_CASE(1)
    SFFT_SAMPLE_CASE(2)
    SFFT_SAMPLE_CASE(3)
    SFFT_SAMPLE_CASE(4)
    SFFT_SAMPLE_CASE(5)
    SFFT_SAMPLE_CASE(6)
    SFFT_SAMPLE_CASE(7)
    SFFT_SAMPLE_CASE(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef SFFT_SAMPLE_CASE
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce_partials(cudaStream_t st, int64_t p, int n_sets, int splits, const c2<T>* part, c2<T>* y) {
  reduce_partials_kernel<T><<<grid_for((int64_t)n_sets * p, 256, 4096), 256, 0, st>>>(p, n_sets, splits, part, y);
  return cudaGetLastError();
}

#define SFFT_INST(T)                                                                                          \
  template cudaError_t launch_prime_tables<T>(cudaStream_t, int64_t, c2<T>*, c2<T>*);                        \
  template cudaError_t launch_twiddles<T>(cudaStream_t, int64_t, c2<T>*);                                     \
  template cudaError_t launch_project<T>(cudaStream_t, int, int, int, int64_t, int64_t, const int64_t*,       \
                                         const int32_t*, const double2*, const int32_t*, const double2*, int, \
                                         int, int32_t*, c2<T>*);                                              \
  template cudaError_t launch_sample<T>(cudaStream_t, const SampleGeom&, int64_t, int, int, int,              \
                                        const int32_t*, const c2<T>*, const c2<T>*, c2<T>*);                  \
  template cudaError_t launch_reduce_partials<T>(cudaStream_t, int64_t, int, int, const c2<T>*, c2<T>*);
SFFT_INST(float)
SFFT_INST(double)
#undef SFFT_INST

}  // namespace sfft
