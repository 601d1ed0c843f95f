// C ABI of the sparse-FFT library: plans, synthetic signals, the round driver of
// Algorithm 2 (MultiPhaseshift) and the per-step entry points.
//
// Round i (Alg. 2 loop body, general form):
//   k* = max(k - |R|, 1); p = i-th prime >= c k* (or the caller's list)
//   u  = direction (i mod count): partial unwrap of a block (Eq. 35-38) or a given tilt
//   kernels: round setup -> per-prime tables -> projection (a-2) -> sampling (a-3)
//            -> Bluestein DFT (a-4) -> classification (a-5) -> merge + prune (a-6)
//   the host reads the round counters back and stops when no bin was occupied (a-7).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "sfft_internal.cuh"

using namespace sfft;

namespace {

thread_local int g_last_cuda_error = 0;

#define SFFT_CUDA(call)                                   \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) {                              \
      g_last_cuda_error = (int)_e;                        \
      return SFFT_ERR_CUDA;                               \
    }                                                     \
  } while (0)

int64_t next_pow2(int64_t v) {
  int64_t r = 1;
  while (r < v) r <<= 1;
  return r;
}

// Primes by a sieve of Eratosthenes up to `lim`.
std::vector<int64_t> primes_up_to(int64_t lim) {
  std::vector<char> comp((size_t)lim + 1, 0);
  std::vector<int64_t> out;
  for (int64_t q = 2; q <= lim; ++q) {
    if (comp[q]) continue;
    out.push_back(q);
    for (int64_t m = q * q; m <= lim; m += q) comp[m] = 1;
  }
  return out;
}

}  // namespace

struct sfft_signal_s {
  int d = 0;
  int64_t N = 0;
  int64_t k = 0;
  int32_t* w = nullptr;   // device [k x d]
  double2* a = nullptr;   // device [k]
};

struct sfft_plan_s {
  int d = 0;
  int64_t N = 0;
  int64_t k = 0;
  int c = 5;
  int prec = SFFT_PREC_FP32_FP64RATIO;
  int box_lo = 0;
  double tau = 0, rho = 0, delta = 0, sigma = 0;
  int max_rounds = 0;
  std::vector<int64_t> prime_list;   // caller's schedule, empty = rule
  std::vector<int64_t> primes;       // sieve, for the rule
  int n_dirs = 0;
  cudaStream_t stream = nullptr;
  int n_sets = 0;
  int64_t p_max = 0, L_max = 0;
  int reg_cap = 0, acc_cap = 0, K_max = 0, Kpad = 0, hash_cap = 0;
  int64_t part_cap = 0;
  int n_sm = 148;
  size_t bytes = 0;
  size_t csize = 8;   // bytes of one complex element of the bulk type
  // device
  DevState* state = nullptr;
  DevState* state_host = nullptr;   // pinned
  int64_t* dirs = nullptr;
  int64_t* u_mod = nullptr;
  int32_t* alpha = nullptr;
  void* C = nullptr;
  void* W = nullptr;
  void* chirp = nullptr;
  void* twG = nullptr;
  void* part = nullptr;
  void* Z = nullptr;
  void* Y = nullptr;
  int32_t* acc_h = nullptr;
  int32_t* acc_w = nullptr;
  double2* acc_a = nullptr;
  int32_t* reg_w = nullptr;
  double2* reg_a = nullptr;
  int32_t* hash = nullptr;
  int64_t* count_dev = nullptr;
  int64_t* count_host = nullptr;   // pinned
  std::vector<void*> allocs;

  ~sfft_plan_s() {
    for (void* q : allocs) cudaFree(q);
    if (state_host) cudaFreeHost(state_host);
    if (count_host) cudaFreeHost(count_host);
  }

  cudaError_t alloc(void** out, size_t bytes_) {
    cudaError_t e = cudaMalloc(out, bytes_ == 0 ? 16 : bytes_);
    if (e == cudaSuccess) {
      allocs.push_back(*out);
      bytes += bytes_;
    }
    return e;
  }

  int64_t ith_prime_at_least(int i, int64_t lo) const {
    auto it = std::lower_bound(primes.begin(), primes.end(), std::max<int64_t>(lo, 2));
    const size_t idx = (size_t)(it - primes.begin()) + (size_t)(i - 1);
    return idx < primes.size() ? primes[idx] : -1;
  }

  int64_t round_prime(int i, int64_t k_star) const {
    if (!prime_list.empty()) return prime_list[(size_t)(i - 1) % prime_list.size()];
    return ith_prime_at_least(i, (int64_t)c * k_star);
  }
};

extern "C" {

int sfft_last_cuda_error(void) { return g_last_cuda_error; }

const char* sfft_status_string(sfft_status s) {
  switch (s) {
    case SFFT_OK: return "ok";
    case SFFT_ERR_INVALID_ARG: return "invalid argument";
    case SFFT_ERR_NOT_CONVERGED: return "not converged";
    case SFFT_ERR_CAPACITY: return "capacity exceeded";
    case SFFT_ERR_PRECISION: return "beyond phase resolution";
    case SFFT_ERR_INCONSISTENT: return "more modes than k";
    case SFFT_ERR_CUDA: return "cuda error";
    case SFFT_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown";
}

sfft_status sfft_plan_create(int d, int64_t N, int64_t k, const sfft_pschedule* ps, const sfft_tilts* tilts,
                             const sfft_opts* opts, void* stream, sfft_plan* plan_out) {
  if (!plan_out) return SFFT_ERR_INVALID_ARG;
  *plan_out = nullptr;
  if (d < 1 || d > 4096 || N < 2 || N > (1LL << 30) || k < 0 || k > (1LL << 26)) return SFFT_ERR_INVALID_ARG;
  sfft_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.precision < 0 || o.precision > SFFT_PREC_FP64) return SFFT_ERR_INVALID_ARG;
  if (o.box_lo > 0 || o.box_lo < -N) return SFFT_ERR_INVALID_ARG;
  if (o.precision != SFFT_PREC_FP64 && N > (1LL << 24)) return SFFT_ERR_PRECISION;
  if (o.tau < 0 || o.rho < 0 || o.delta < 0 || o.delta >= 0.5 || o.noise_sigma < 0 || o.max_rounds < 0)
    return SFFT_ERR_INVALID_ARG;

  sfft_plan_s* P = new sfft_plan_s();
  std::unique_ptr<sfft_plan_s> guard(P);
  P->d = d;
  P->N = N;
  P->k = k;
  P->prec = o.precision;
  P->box_lo = o.box_lo;
  const bool fp64 = o.precision == SFFT_PREC_FP64;
  P->tau = o.tau > 0 ? o.tau : (fp64 ? 1e-7 : 1e-3);
  P->rho = o.rho > 0 ? o.rho : (fp64 ? std::ldexp(1.0, -40) : std::ldexp(1.0, -17));
  P->delta = o.delta > 0 ? o.delta : (fp64 ? 0.1 : 0.25);
  P->sigma = o.noise_sigma;
  int lg = 1;
  while ((1LL << lg) < std::max<int64_t>(k, 2)) ++lg;
  P->max_rounds = o.max_rounds > 0 ? o.max_rounds : 64 + 4 * lg;
  if (P->max_rounds > SFFT_STATS_MAX_ROUNDS) P->max_rounds = SFFT_STATS_MAX_ROUNDS;
  P->stream = (cudaStream_t)stream;
  P->n_sets = d + 1;
  P->csize = fp64 ? sizeof(double2) : sizeof(float2);

  // ---- prime schedule
  if (ps) {
    if (ps->c_prime < 0 || ps->n_primes < 0) return SFFT_ERR_INVALID_ARG;
    if (ps->c_prime > 0) P->c = ps->c_prime;
    if (ps->n_primes > 0) {
      if (!ps->primes) return SFFT_ERR_INVALID_ARG;
      for (int i = 0; i < ps->n_primes; ++i) {
        const int64_t q = ps->primes[i];
        if (q < 2 || q > (1LL << 26)) return SFFT_ERR_INVALID_ARG;
        for (int64_t f = 2; f * f <= q; ++f)
          if (q % f == 0) return SFFT_ERR_INVALID_ARG;
        P->prime_list.push_back(q);
      }
    }
  }
  if (P->prime_list.empty()) {
    const int64_t lo = (int64_t)P->c * std::max<int64_t>(k, 1);
    int64_t lim = lo + 64LL * P->max_rounds + 1000;
    for (;;) {
      P->primes = primes_up_to(lim);
      if (P->ith_prime_at_least(P->max_rounds, lo) > 0) break;
      lim *= 2;
    }
    P->p_max = P->ith_prime_at_least(P->max_rounds, lo);
  } else {
    P->p_max = *std::max_element(P->prime_list.begin(), P->prime_list.end());
  }
  if (P->p_max > (1LL << 26)) return SFFT_ERR_INVALID_ARG;

  // ---- line directions
  std::vector<int64_t> dirs;
  if (tilts && tilts->n_dirs > 0) {
    if (!tilts->dirs) return SFFT_ERR_INVALID_ARG;
    dirs.assign(tilts->dirs, tilts->dirs + (size_t)tilts->n_dirs * d);
    P->n_dirs = tilts->n_dirs;
  } else {
    std::vector<int> blocks;
    if (tilts && tilts->n_blocks > 0) {
      if (!tilts->block_sizes) return SFFT_ERR_INVALID_ARG;
      int tot = 0;
      for (int q = 0; q < tilts->n_blocks; ++q) {
        if (tilts->block_sizes[q] < 1) return SFFT_ERR_INVALID_ARG;
        blocks.push_back(tilts->block_sizes[q]);
        tot += tilts->block_sizes[q];
      }
      if (tot != d) return SFFT_ERR_INVALID_ARG;
    } else {
      // default: smallest b with N^b >= 4 c k, d / b blocks, earlier blocks take the remainder
      int b = 1;
      double range = (double)N;
      while (range < 4.0 * P->c * std::max<int64_t>(k, 1) && b < d) {
        ++b;
        range *= (double)N;
      }
      const int nb = std::max(1, d / b);
      for (int q = 0; q < nb; ++q) blocks.push_back(d / nb + (q < d % nb ? 1 : 0));
    }
    P->n_dirs = (int)blocks.size();
    dirs.assign((size_t)P->n_dirs * d, 0);
    int start = 0;
    for (int q = 0; q < P->n_dirs; ++q) {
      int64_t pw = 1;
      for (int r = 0; r < blocks[q]; ++r) {
        dirs[(size_t)q * d + start + r] = pw;   // N^r on the block's r-th coordinate (Eq. 35)
        if (r + 1 < blocks[q]) {
          if (pw > (int64_t)(9.0e18 / (double)N)) return SFFT_ERR_INVALID_ARG;
          pw *= N;
        }
      }
      start += blocks[q];
    }
  }

  // ---- sizes
  P->reg_cap = (int)std::min<int64_t>(2 * k + 256, (1LL << 30));
  P->acc_cap = (int)std::min<int64_t>(P->p_max, (int64_t)P->reg_cap);
  P->K_max = (int)(k + P->reg_cap);
  P->Kpad = ((P->K_max + 31) / 32) * 32;
  P->hash_cap = (int)next_pow2(2 * (int64_t)P->reg_cap);
  P->L_max = next_pow2(2 * P->p_max - 1);
  const int64_t one_split = (int64_t)P->n_sets * P->p_max;
  P->part_cap = std::max<int64_t>(one_split, (int64_t)(64ll << 20) / (int64_t)P->csize);
  int dev = 0;
  SFFT_CUDA(cudaGetDevice(&dev));
  SFFT_CUDA(cudaDeviceGetAttribute(&P->n_sm, cudaDevAttrMultiProcessorCount, dev));

  void* q = nullptr;
#define SFFT_ALLOC(field, bytes_)                \
  SFFT_CUDA(P->alloc(&q, (size_t)(bytes_)));     \
  P->field = reinterpret_cast<decltype(P->field)>(q);
  SFFT_ALLOC(state, sizeof(DevState));
  SFFT_ALLOC(dirs, dirs.size() * sizeof(int64_t));
  SFFT_ALLOC(u_mod, (size_t)d * sizeof(int64_t));
  SFFT_ALLOC(alpha, (size_t)P->Kpad * sizeof(int32_t));
  SFFT_ALLOC(C, (size_t)P->n_sets * P->Kpad * P->csize);
  SFFT_ALLOC(W, (size_t)P->p_max * P->csize);
  SFFT_ALLOC(chirp, (size_t)P->p_max * P->csize);
  SFFT_ALLOC(twG, (size_t)P->L_max * P->csize);
  SFFT_ALLOC(part, (size_t)P->part_cap * P->csize);
  SFFT_ALLOC(Z, (size_t)(P->n_sets + 1) * P->L_max * P->csize);
  SFFT_ALLOC(Y, (size_t)P->n_sets * P->p_max * P->csize);
  SFFT_ALLOC(acc_h, (size_t)P->acc_cap * sizeof(int32_t));
  SFFT_ALLOC(acc_w, (size_t)P->acc_cap * d * sizeof(int32_t));
  SFFT_ALLOC(acc_a, (size_t)P->acc_cap * sizeof(double2));
  SFFT_ALLOC(reg_w, (size_t)P->reg_cap * d * sizeof(int32_t));
  SFFT_ALLOC(reg_a, (size_t)P->reg_cap * sizeof(double2));
  SFFT_ALLOC(hash, (size_t)P->hash_cap * sizeof(int32_t));
  SFFT_ALLOC(count_dev, sizeof(int64_t));
#undef SFFT_ALLOC
  SFFT_CUDA(cudaMallocHost((void**)&P->state_host, sizeof(DevState)));
  SFFT_CUDA(cudaMallocHost((void**)&P->count_host, sizeof(int64_t)));
  SFFT_CUDA(cudaMemcpyAsync(P->dirs, dirs.data(), dirs.size() * sizeof(int64_t), cudaMemcpyHostToDevice, P->stream));
  if (fp64) {
    SFFT_CUDA(launch_twiddles<double>(P->stream, P->L_max, (double2*)P->twG));
  } else {
    SFFT_CUDA(launch_twiddles<float>(P->stream, P->L_max, (float2*)P->twG));
  }
  SFFT_CUDA(cudaStreamSynchronize(P->stream));
  *plan_out = guard.release();
  return SFFT_OK;
}

void sfft_plan_destroy(sfft_plan plan) {
  if (!plan) return;
  cudaStreamSynchronize(plan->stream);
  delete plan;
}

int64_t sfft_plan_max_prime(sfft_plan plan) { return plan ? plan->p_max : -1; }
int64_t sfft_plan_mode_capacity(sfft_plan plan) { return plan ? plan->K_max : -1; }
int64_t sfft_plan_device_bytes(sfft_plan plan) { return plan ? (int64_t)plan->bytes : -1; }

sfft_status sfft_signal_synthetic(int d, int64_t N, int64_t k, const int32_t* freqs_dev, const double* coeffs_dev,
                                  double noise_sigma, uint64_t noise_seed, sfft_signal* signal_out) {
  (void)noise_seed;
  if (!signal_out) return SFFT_ERR_INVALID_ARG;
  *signal_out = nullptr;
  if (d < 1 || N < 2 || k < 0 || (k > 0 && (!freqs_dev || !coeffs_dev))) return SFFT_ERR_INVALID_ARG;
  if (noise_sigma != 0.0) return SFFT_ERR_INVALID_ARG;
  sfft_signal_s* S = new sfft_signal_s();
  S->d = d;
  S->N = N;
  S->k = k;
  cudaError_t e = cudaMalloc((void**)&S->w, (size_t)std::max<int64_t>(k, 1) * d * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->a, (size_t)std::max<int64_t>(k, 1) * sizeof(double2));
  if (e == cudaSuccess && k > 0)
    e = cudaMemcpy(S->w, freqs_dev, (size_t)k * d * sizeof(int32_t), cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && k > 0)
    e = cudaMemcpy(S->a, coeffs_dev, (size_t)k * sizeof(double2), cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) {
    g_last_cuda_error = (int)e;
    cudaFree(S->w);
    cudaFree(S->a);
    delete S;
    return SFFT_ERR_CUDA;
  }
  *signal_out = S;
  return SFFT_OK;
}

void sfft_signal_destroy(sfft_signal signal) {
  if (!signal) return;
  cudaFree(signal->w);
  cudaFree(signal->a);
  delete signal;
}

}  // extern "C"

namespace {

// One round's kernels, on the plan's stream.
template <typename T, typename R>
cudaError_t enqueue_round(sfft_plan_s* P, const sfft_signal_s* S, int round, int64_t p, int K_reg,
                          SampleGeom* geom_out) {
  using C2 = c2<T>;
  cudaError_t e;
  const int dir_index = round % P->n_dirs;
  if ((e = launch_round_begin(P->stream, P->state, P->dirs, dir_index, P->d, p, P->u_mod)) != cudaSuccess) return e;
  if ((e = launch_prime_tables<T>(P->stream, p, (C2*)P->W, (C2*)P->chirp)) != cudaSuccess) return e;
  const int K = (int)S->k + K_reg;
  if ((e = launch_project<T>(P->stream, (int)S->k, K_reg, P->d, P->N, p, P->u_mod, S->w, S->a, P->reg_w, P->reg_a,
                             P->n_sets, P->Kpad, P->alpha, (C2*)P->C)) != cudaSuccess)
    return e;
  const SampleGeom g = sample_geometry(p, K, P->n_sets, P->part_cap, P->n_sm);
  *geom_out = g;
  if ((e = launch_sample<T>(P->stream, g, p, K, P->n_sets, P->Kpad, P->alpha, (const C2*)P->C, (const C2*)P->W,
                            (C2*)P->part)) != cudaSuccess)
    return e;
  const DftGeom dg = dft_geometry(p);
  if ((e = launch_bluestein<T>(P->stream, dg, p, P->n_sets, g.splits, (const C2*)P->part, (const C2*)P->chirp,
                               (const C2*)P->twG, P->L_max, (C2*)P->Z, (C2*)P->Y, P->state)) != cudaSuccess)
    return e;
  ClassifyArgs ca;
  ca.p = p;
  ca.N = P->N;
  ca.d = P->d;
  ca.box_lo = P->box_lo;
  ca.round = round;
  ca.rho = P->rho;
  ca.tau = P->tau;
  ca.delta = P->delta;
  ca.sigma = P->sigma;
  ca.eta_override = -1.0;
  ca.acc_cap = P->acc_cap;
  if ((e = launch_classify<T, R>(P->stream, ca, (const C2*)P->Y, P->u_mod, P->state, P->acc_h, P->acc_w,
                                 P->acc_a)) != cudaSuccess)
    return e;
  if ((e = launch_merge(P->stream, P->d, P->acc_cap, P->acc_w, P->acc_a, P->state, P->reg_w, P->reg_a, P->reg_cap,
                        P->hash, P->hash_cap - 1)) != cudaSuccess)
    return e;
  return launch_prune(P->stream, p, P->rho, P->sigma, P->reg_cap, P->state, P->reg_a);
}

template <typename T, typename R>
sfft_status execute_impl(sfft_plan_s* P, const sfft_signal_s* S, int64_t capacity, int32_t* freqs_out,
                         double* coeffs_out, int64_t* n_found, sfft_stats* stats) {
  SFFT_CUDA(cudaMemsetAsync(P->state, 0, sizeof(DevState), P->stream));
  SFFT_CUDA(cudaMemsetAsync(P->hash, 0xFF, (size_t)P->hash_cap * sizeof(int32_t), P->stream));
  if (stats) std::memset(stats, 0, sizeof(*stats));
  int n_live = 0, n_reg = 0;
  bool converged = false;
  int rounds = 0;
  for (int i = 1; i <= P->max_rounds; ++i) {
    const int64_t k_star = std::max<int64_t>(P->k - n_live, 1);
    const int64_t p = P->round_prime(i, k_star);
    if (p < 2 || p > P->p_max) return SFFT_ERR_INVALID_ARG;
    SampleGeom g;
    SFFT_CUDA((enqueue_round<T, R>(P, S, i, p, n_reg, &g)));
    SFFT_CUDA(cudaMemcpyAsync(P->state_host, P->state, sizeof(DevState), cudaMemcpyDeviceToHost, P->stream));
    SFFT_CUDA(cudaStreamSynchronize(P->stream));
    const DevState hs = *P->state_host;
    rounds = i;
    if (stats && i <= SFFT_STATS_MAX_ROUNDS) {
      stats->p[i - 1] = p;
      stats->K[i - 1] = (int32_t)(S->k + n_reg);
      stats->accepted[i - 1] = hs.n_acc;
      stats->registry[i - 1] = hs.n_live;
      stats->samples += (int64_t)P->n_sets * p;
      stats->terms += (int64_t)P->n_sets * p * (S->k + n_reg);
    }
    if (hs.err) return SFFT_ERR_CAPACITY;
    n_live = hs.n_live;
    n_reg = std::min(hs.n_reg, P->reg_cap);
    if (!hs.any_occupied) {
      converged = true;
      break;
    }
  }
  if (stats) {
    stats->rounds = rounds;
    stats->converged = converged ? 1 : 0;
  }
  SFFT_CUDA(launch_output(P->stream, P->d, P->reg_cap, P->state, P->reg_w, P->reg_a, capacity, freqs_out,
                          (double2*)coeffs_out, P->count_dev));
  SFFT_CUDA(cudaMemcpyAsync(P->count_host, P->count_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, P->stream));
  SFFT_CUDA(cudaStreamSynchronize(P->stream));
  *n_found = *P->count_host;
  if (*n_found > capacity) return SFFT_ERR_CAPACITY;
  if (!converged) return SFFT_ERR_NOT_CONVERGED;
  if (*n_found > P->k) return SFFT_ERR_INCONSISTENT;
  return SFFT_OK;
}

}  // namespace

extern "C" {

sfft_status sfft_execute(sfft_plan plan, sfft_signal signal, int64_t capacity, int32_t* freqs_out_dev,
                         double* coeffs_out_dev, int64_t* n_found, sfft_stats* stats) {
  if (!plan || !signal || !n_found || capacity < 0) return SFFT_ERR_INVALID_ARG;
  if (capacity > 0 && (!freqs_out_dev || !coeffs_out_dev)) return SFFT_ERR_INVALID_ARG;
  if (signal->d != plan->d || signal->N != plan->N || signal->k > plan->k) return SFFT_ERR_INVALID_ARG;
  *n_found = 0;
  switch (plan->prec) {
    case SFFT_PREC_FP32_FP64RATIO:
      return execute_impl<float, double>(plan, signal, capacity, freqs_out_dev, coeffs_out_dev, n_found, stats);
    case SFFT_PREC_FP32:
      return execute_impl<float, float>(plan, signal, capacity, freqs_out_dev, coeffs_out_dev, n_found, stats);
    default:
      return execute_impl<double, double>(plan, signal, capacity, freqs_out_dev, coeffs_out_dev, n_found, stats);
  }
}

sfft_status sfft_sample(sfft_plan P, int64_t p, const int64_t* u, int64_t K, const int32_t* freqs_dev,
                        const double* coeffs_dev, void* y_out_dev) {
  if (!P || !u || !y_out_dev || p < 2 || p > P->p_max || K < 0 || K > P->K_max) return SFFT_ERR_INVALID_ARG;
  if (K > 0 && (!freqs_dev || !coeffs_dev)) return SFFT_ERR_INVALID_ARG;
  std::vector<int64_t> um((size_t)P->d);
  for (int l = 0; l < P->d; ++l) {
    int64_t v = u[l] % p;
    um[l] = v < 0 ? v + p : v;
  }
  SFFT_CUDA(cudaMemcpyAsync(P->u_mod, um.data(), um.size() * sizeof(int64_t), cudaMemcpyHostToDevice, P->stream));
  const int iK = (int)K;
  const SampleGeom g = sample_geometry(p, iK, P->n_sets, P->part_cap, P->n_sm);
  if (P->prec == SFFT_PREC_FP64) {
    SFFT_CUDA(launch_prime_tables<double>(P->stream, p, (double2*)P->W, (double2*)P->chirp));
    SFFT_CUDA(launch_project<double>(P->stream, iK, 0, P->d, P->N, p, P->u_mod, freqs_dev, (const double2*)coeffs_dev,
                                     nullptr, nullptr, P->n_sets, P->Kpad, P->alpha, (double2*)P->C));
    SFFT_CUDA(launch_sample<double>(P->stream, g, p, iK, P->n_sets, P->Kpad, P->alpha, (const double2*)P->C,
                                    (const double2*)P->W, (double2*)P->part));
    SFFT_CUDA(launch_reduce_partials<double>(P->stream, p, P->n_sets, g.splits, (const double2*)P->part,
                                             (double2*)y_out_dev));
  } else {
    SFFT_CUDA(launch_prime_tables<float>(P->stream, p, (float2*)P->W, (float2*)P->chirp));
    SFFT_CUDA(launch_project<float>(P->stream, iK, 0, P->d, P->N, p, P->u_mod, freqs_dev, (const double2*)coeffs_dev,
                                    nullptr, nullptr, P->n_sets, P->Kpad, P->alpha, (float2*)P->C));
    SFFT_CUDA(launch_sample<float>(P->stream, g, p, iK, P->n_sets, P->Kpad, P->alpha, (const float2*)P->C,
                                   (const float2*)P->W, (float2*)P->part));
    SFFT_CUDA(launch_reduce_partials<float>(P->stream, p, P->n_sets, g.splits, (const float2*)P->part,
                                            (float2*)y_out_dev));
  }
  SFFT_CUDA(cudaStreamSynchronize(P->stream));
  return SFFT_OK;
}

sfft_status sfft_dft(sfft_plan P, int64_t p, int n_rows, const void* y_dev, void* Y_out_dev) {
  if (!P || !y_dev || !Y_out_dev || p < 2 || p > P->p_max || n_rows < 1 || n_rows > P->n_sets)
    return SFFT_ERR_INVALID_ARG;
  const DftGeom dg = dft_geometry(p);
  if (P->prec == SFFT_PREC_FP64) {
    SFFT_CUDA(launch_prime_tables<double>(P->stream, p, (double2*)P->W, (double2*)P->chirp));
    SFFT_CUDA(launch_bluestein<double>(P->stream, dg, p, n_rows, 1, (const double2*)y_dev, (const double2*)P->chirp,
                                       (const double2*)P->twG, P->L_max, (double2*)P->Z, (double2*)Y_out_dev,
                                       nullptr));
  } else {
    SFFT_CUDA(launch_prime_tables<float>(P->stream, p, (float2*)P->W, (float2*)P->chirp));
    SFFT_CUDA(launch_bluestein<float>(P->stream, dg, p, n_rows, 1, (const float2*)y_dev, (const float2*)P->chirp,
                                      (const float2*)P->twG, P->L_max, (float2*)P->Z, (float2*)Y_out_dev, nullptr));
  }
  SFFT_CUDA(cudaStreamSynchronize(P->stream));
  return SFFT_OK;
}

sfft_status sfft_classify(sfft_plan P, int64_t p, const int64_t* u, const void* Y_dev, double eta_bin,
                          int64_t capacity, int32_t* h_out_dev, int32_t* freqs_out_dev, double* coeffs_out_dev,
                          int64_t* n_out) {
  if (!P || !u || !Y_dev || !n_out || p < 2 || p > P->p_max || eta_bin < 0 || capacity < 0 ||
      capacity > (int64_t)1 << 30)
    return SFFT_ERR_INVALID_ARG;
  if (capacity > 0 && (!h_out_dev || !freqs_out_dev || !coeffs_out_dev)) return SFFT_ERR_INVALID_ARG;
  std::vector<int64_t> um((size_t)P->d);
  for (int l = 0; l < P->d; ++l) {
    int64_t v = u[l] % p;
    um[l] = v < 0 ? v + p : v;
  }
  SFFT_CUDA(cudaMemcpyAsync(P->u_mod, um.data(), um.size() * sizeof(int64_t), cudaMemcpyHostToDevice, P->stream));
  SFFT_CUDA(cudaMemsetAsync(P->state, 0, sizeof(DevState), P->stream));
  ClassifyArgs ca;
  ca.p = p;
  ca.N = P->N;
  ca.d = P->d;
  ca.box_lo = P->box_lo;
  ca.round = 0;
  ca.rho = P->rho;
  ca.tau = P->tau;
  ca.delta = P->delta;
  ca.sigma = P->sigma;
  ca.eta_override = eta_bin;
  ca.acc_cap = (int)capacity;
  switch (P->prec) {
    case SFFT_PREC_FP32_FP64RATIO:
      SFFT_CUDA((launch_classify<float, double>(P->stream, ca, (const float2*)Y_dev, P->u_mod, P->state, h_out_dev,
                                                freqs_out_dev, (double2*)coeffs_out_dev)));
      break;
    case SFFT_PREC_FP32:
      SFFT_CUDA((launch_classify<float, float>(P->stream, ca, (const float2*)Y_dev, P->u_mod, P->state, h_out_dev,
                                               freqs_out_dev, (double2*)coeffs_out_dev)));
      break;
    default:
      SFFT_CUDA((launch_classify<double, double>(P->stream, ca, (const double2*)Y_dev, P->u_mod, P->state, h_out_dev,
                                                 freqs_out_dev, (double2*)coeffs_out_dev)));
  }
  SFFT_CUDA(cudaMemcpyAsync(P->state_host, P->state, sizeof(DevState), cudaMemcpyDeviceToHost, P->stream));
  SFFT_CUDA(cudaStreamSynchronize(P->stream));
  *n_out = P->state_host->n_acc;
  if (P->state_host->err) {
    *n_out = std::min<int64_t>(*n_out, capacity);
    return SFFT_ERR_CAPACITY;
  }
  return SFFT_OK;
}

}  // extern "C"
