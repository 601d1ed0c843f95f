// Bin classification and read-out (Eq. 7-8, Eq. 41-42), registry merge into a
// device hash table, pruning, and compaction of the live registry.
//
// Per bin h (one thread):
//   empty        |Y_0[h]| <= eta_bin
//   ratio test   | |Y_n[h]| / |Y_0[h]| - 1 | < tau        for every n = 1..d   (Eq. 42)
//   read-out     v_n = N Arg(Y_n[h] / Y_0[h]) / (2 pi), Arg in [-pi, pi)    (Eq. 41, eps = 1/N)
//                |v_n - round(v_n)| <= delta, w_n = round(v_n) folded into the box
//   own bin      (w . u) mod p == h
//   coefficient  a = Y_0[h] / p                                            (Eq. 41)
// The phase ratio and everything after it run in the ratio type R (double under
// the FP32-bulk policy).  Accepted bins are appended through an atomic counter.
#include "sfft_internal.cuh"

namespace sfft {

namespace {

template <typename R> __device__ __forceinline__ R two_pi();
template <> __device__ __forceinline__ float two_pi<float>() { return 6.28318530717958647692f; }
template <> __device__ __forceinline__ double two_pi<double>() { return 6.28318530717958647692; }
template <typename R> __device__ __forceinline__ R pi_r();
template <> __device__ __forceinline__ float pi_r<float>() { return 3.14159265358979323846f; }
template <> __device__ __forceinline__ double pi_r<double>() { return 3.14159265358979323846; }

__device__ __forceinline__ float my_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double my_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float my_hypot(float y, float x) { return hypotf(y, x); }
__device__ __forceinline__ double my_hypot(double y, double x) { return hypot(y, x); }
__device__ __forceinline__ float my_rint(float v) { return rintf(v); }
__device__ __forceinline__ float my_fabs(float v) { return fabsf(v); }
__device__ __forceinline__ double my_fabs(double v) { return ::fabs(v); }
__device__ __forceinline__ double my_rint(double v) { return rint(v); }

// Read-out of coordinate n-1 from Y_n and Y_0; returns false when it is not within delta
// of an integer.  Identical arithmetic in both passes of the classifier.
template <typename R>
__device__ __forceinline__ bool read_coordinate(R ynx, R yny, R y0x, R y0y, int64_t N, int box_lo, R delta,
                                                int64_t* w_out) {
  const R re = ynx * y0x + yny * y0y;   // Y_n conj(Y_0)
  const R im = yny * y0x - ynx * y0y;
  R phi = my_atan2(im, re);
  if (phi >= pi_r<R>()) phi -= two_pi<R>();   // Arg in [-pi, pi)
  const R v = (R)N * phi / two_pi<R>();
  const R r = my_rint(v);
  if (!(my_fabs(v - r) <= delta)) return false;
  int64_t wn = ((int64_t)r - box_lo) % N;
  if (wn < 0) wn += N;
  *w_out = wn + box_lo;
  return true;
}

template <typename T, typename R>
__global__ void classify_kernel(ClassifyArgs a, const c2<T>* __restrict__ Y, const int64_t* __restrict__ u_mod,
                                DevState* st, int32_t* __restrict__ acc_h, int32_t* __restrict__ acc_w,
                                double2* __restrict__ acc_a) {
  const int64_t p = a.p;
  double a_ref;
  if (a.round == 1) {
    a_ref = __longlong_as_double((long long)st->max_y0_bits) / (double)p;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->a_ref = a_ref;
  } else {
    a_ref = st->a_ref;
  }
  const double eta = a.eta_override >= 0.0 ? a.eta_override
                                           : fmax(a.rho * (double)p * a_ref, 6.0 * a.sigma * sqrt((double)p));
  const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (h >= p) return;
  const c2<T> y0 = Y[h];
  const R y0x = (R)y0.x, y0y = (R)y0.y;
  const R m0 = my_hypot(y0x, y0y);
  if (!((double)m0 > eta)) return;
  st->any_occupied = 1;
  const R tau = (R)a.tau, delta = (R)a.delta;
  int64_t bin = 0;
  for (int n = 1; n <= a.d; ++n) {
    const c2<T> yn = Y[(int64_t)n * p + h];
    const R ynx = (R)yn.x, yny = (R)yn.y;
    const R mn = my_hypot(ynx, yny);
    if (!(my_fabs(mn / m0 - (R)1) < tau)) return;   // Eq. 42
    int64_t wn;
    if (!read_coordinate<R>(ynx, yny, y0x, y0y, a.N, a.box_lo, delta, &wn)) return;
    int64_t wm = wn % p;
    if (wm < 0) wm += p;
    bin = (bin + wm * u_mod[n - 1]) % p;
  }
  if (bin != h) return;
  const int idx = atomicAdd(&st->n_acc, 1);
  if (idx >= a.acc_cap) {
    atomicOr(&st->err, kErrAccCapacity);
    return;
  }
  acc_h[idx] = (int32_t)h;
  acc_a[idx] = make_double2((double)y0.x / (double)p, (double)y0.y / (double)p);
  for (int n = 1; n <= a.d; ++n) {
    const c2<T> yn = Y[(int64_t)n * p + h];
    int64_t wn = 0;
    read_coordinate<R>((R)yn.x, (R)yn.y, y0x, y0y, a.N, a.box_lo, delta, &wn);
    acc_w[(int64_t)idx * a.d + n - 1] = (int32_t)wn;
  }
}

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

// One thread per accepted entry.  Keys accepted in one round are distinct (each
// lands in its own bin), and the table never deletes, so a key is present iff it
// is met before the first empty slot of its probe sequence.
__global__ void merge_kernel(int d, int acc_cap, const int32_t* __restrict__ acc_w,
                             const double2* __restrict__ acc_a, DevState* st, int32_t* reg_w, double2* reg_a,
                             int reg_cap, int32_t* hash, int hash_mask) {
  const int n = min(st->n_acc, acc_cap);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t* w = acc_w + (int64_t)i * d;
  const double2 a = acc_a[i];
  int slot = (int)(hash_key(w, d) & (unsigned long long)hash_mask);
  int mine = -1;   // registry index once allocated
  for (int probe = 0; probe <= hash_mask; ++probe, slot = (slot + 1) & hash_mask) {
    int cur = atomicAdd(&hash[slot], 0);
    if (cur < 0) {
      if (mine < 0) {
        mine = atomicAdd(&st->n_reg, 1);
        if (mine >= reg_cap) {
          atomicOr(&st->err, kErrRegCapacity);
          return;
        }
        for (int l = 0; l < d; ++l) reg_w[(int64_t)mine * d + l] = w[l];
        reg_a[mine] = a;
        __threadfence();
      }
      cur = atomicCAS(&hash[slot], -1, mine);
      if (cur < 0) return;   // inserted
      continue;              // slot taken by another new key of this round
    }
    if (mine >= 0) continue; // past the first empty slot: only new keys of this round follow
    __threadfence();
    const volatile int32_t* rw = reg_w + (int64_t)cur * d;
    bool same = true;
    for (int l = 0; l < d && same; ++l) same = (rw[l] == w[l]);
    if (same) {
      atomicAdd(&reg_a[cur].x, a.x);   // duplicate key: a_R += a (merge)
      atomicAdd(&reg_a[cur].y, a.y);
      return;
    }
  }
  atomicOr(&st->err, kErrHashFull);
}

// Entries with |a| below the prune level get a = 0 (they no longer contribute to g);
// the rest are counted as live.
__global__ void prune_kernel(int64_t p, double rho, double sigma, int reg_cap, DevState* st, double2* reg_a) {
  const int n = min(st->n_reg, reg_cap);
  const double eta = fmax(rho * st->a_ref, 6.0 * sigma / sqrt((double)p));
  int live = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 a = reg_a[i];
    if (hypot(a.x, a.y) < eta) {
      reg_a[i] = make_double2(0.0, 0.0);
    } else {
      live += 1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) live += __shfl_xor_sync(0xffffffffu, live, o);
  if ((threadIdx.x & 31) == 0 && live) atomicAdd(&st->n_live, live);
}

// One block: ordered compaction of the live registry entries.
__global__ void output_kernel(int d, int reg_cap, const DevState* st, const int32_t* __restrict__ reg_w,
                              const double2* __restrict__ reg_a, int64_t capacity, int32_t* freqs_out,
                              double2* coeffs_out, int64_t* count_dev) {
  __shared__ int warp_sums[32];
  __shared__ int64_t base_s;
  const int n = min(st->n_reg, reg_cap);
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c0 = 0; c0 < n; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    const bool live = i < n && (reg_a[i].x != 0.0 || reg_a[i].y != 0.0);
    const unsigned bal = __ballot_sync(0xffffffffu, live);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[wid] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int q = 0; q < nw; ++q) {
      if (q < wid) off += warp_sums[q];
      tot += warp_sums[q];
    }
    const int64_t pos = base_s + off + before;
    if (live && pos < capacity) {
      for (int l = 0; l < d; ++l) freqs_out[pos * d + l] = reg_w[(int64_t)i * d + l];
      coeffs_out[pos] = reg_a[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) base_s += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count_dev = base_s;
}

}  // namespace

template <typename T, typename R>
cudaError_t launch_classify(cudaStream_t st, const ClassifyArgs& a, const c2<T>* Y, const int64_t* u_mod,
                            DevState* state, int32_t* acc_h, int32_t* acc_w, double2* acc_a) {
  const int threads = 128;
  const int64_t blocks = (a.p + threads - 1) / threads;
  classify_kernel<T, R><<<(unsigned)blocks, threads, 0, st>>>(a, Y, u_mod, state, acc_h, acc_w, acc_a);
  return cudaGetLastError();
}

cudaError_t launch_merge(cudaStream_t st, int d, int acc_cap, const int32_t* acc_w, const double2* acc_a,
                         DevState* state, int32_t* reg_w, double2* reg_a, int reg_cap, int32_t* hash,
                         int hash_mask) {
  const int threads = 128;
  const int blocks = (acc_cap + threads - 1) / threads;
  merge_kernel<<<blocks > 0 ? blocks : 1, threads, 0, st>>>(d, acc_cap, acc_w, acc_a, state, reg_w, reg_a, reg_cap,
                                                            hash, hash_mask);
  return cudaGetLastError();
}

cudaError_t launch_prune(cudaStream_t st, int64_t p, double rho, double sigma, int reg_cap, DevState* state,
                         double2* reg_a) {
  const int threads = 256;
  int blocks = (reg_cap + threads - 1) / threads;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  prune_kernel<<<blocks, threads, 0, st>>>(p, rho, sigma, reg_cap, state, reg_a);
  return cudaGetLastError();
}

cudaError_t launch_output(cudaStream_t st, int d, int reg_cap, const DevState* state, const int32_t* reg_w,
                          const double2* reg_a, int64_t capacity, int32_t* freqs_out, double2* coeffs_out,
                          int64_t* count_dev) {
  output_kernel<<<1, 1024, 0, st>>>(d, reg_cap, state, reg_w, reg_a, capacity, freqs_out, coeffs_out, count_dev);
  return cudaGetLastError();
}

template cudaError_t launch_classify<float, double>(cudaStream_t, const ClassifyArgs&, const float2*, const int64_t*,
                                                    DevState*, int32_t*, int32_t*, double2*);
template cudaError_t launch_classify<float, float>(cudaStream_t, const ClassifyArgs&, const float2*, const int64_t*,
                                                   DevState*, int32_t*, int32_t*, double2*);
template cudaError_t launch_classify<double, double>(cudaStream_t, const ClassifyArgs&, const double2*,
                                                     const int64_t*, DevState*, int32_t*, int32_t*, double2*);

}  // namespace sfft
