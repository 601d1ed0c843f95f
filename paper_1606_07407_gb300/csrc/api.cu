// C ABI of the sparse-FFT library: plans, synthetic signals, single and batched
// execution of Algorithm 2 (MultiPhaseshift) and the per-step entry points.
// Every call runs through the batched round engine; a single-signal plan is a
// batch of one.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "engine.cuh"

using namespace sfft;

namespace {

thread_local int g_last_cuda_error = 0;

sfft_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SFFT_OK;
  g_last_cuda_error = (int)e;
  return SFFT_ERR_CUDA;
}

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

int64_t ith_prime_at_least(const std::vector<int64_t>& primes, int i, int64_t lo) {
  auto it = std::lower_bound(primes.begin(), primes.end(), std::max<int64_t>(lo, 2));
  const size_t idx = (size_t)(it - primes.begin()) + (size_t)(i - 1);
  return idx < primes.size() ? primes[idx] : -1;
}

__global__ void k_signal_copy(int64_t nw, const int32_t* w_src, int32_t* w_dst, int64_t na, const double2* a_src,
                              double2* a_dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nw; e += (int64_t)gridDim.x * blockDim.x)
    w_dst[e] = w_src[e];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < na; e += (int64_t)gridDim.x * blockDim.x)
    a_dst[e] = a_src[e];
}

// Copies for sfft_signal_assign_many, passed by value: block row y copies signal y's modes.
constexpr int kAssignPerLaunch = 256;
struct AssignDesc {
  int32_t* w_dst;
  double2* a_dst;
  int64_t w_src, a_src;   // offsets into the packed arrays
  int64_t nw, na;         // int32 frequency entries and coefficients to copy
};
struct AssignArgs {
  AssignDesc d[kAssignPerLaunch];
};

__global__ void k_signal_copy_many(AssignArgs args, int count, const int32_t* __restrict__ w_src,
                                   const double2* __restrict__ a_src) {
  const int y = blockIdx.y;
  if (y >= count) return;
  const AssignDesc& c = args.d[y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < c.nw; e += (int64_t)gridDim.x * blockDim.x)
    c.w_dst[e] = w_src[c.w_src + e];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < c.na; e += (int64_t)gridDim.x * blockDim.x)
    c.a_dst[e] = a_src[c.a_src + e];
}

}  // namespace

void sfft::sfft_record_cuda_error(int e) { g_last_cuda_error = e; }

struct sfft_signal_s {
  int d = 0;
  int64_t N = 0;
  int64_t k = 0;
  int64_t k_cap = 0;
  double noise_sigma = 0.0;    // complex Gaussian noise of every sample (E|z|^2 = sigma^2)
  uint64_t noise_seed = 0;
  int32_t* w = nullptr;   // device [k x d]
  double2* a = nullptr;   // device [k]
};

struct sfft_plan_s {
  SlotDesc desc;
  int prec = SFFT_PREC_AUTO;
  cudaStream_t stream = nullptr;
  bool profile = false, graph = false;
  std::unique_ptr<EngineBase> eng;
  std::unique_ptr<EngineBase> eng64;   // FP32_THEN_FP64: the double rounds after the float ones
};

struct sfft_batch_s {
  int n = 0;
  int prec = 0;
  std::vector<int> d;
  std::vector<int64_t> k;
  std::vector<int64_t> N;
  std::unique_ptr<EngineBase> eng;
};

// policies whose plans run on the double engine
inline bool double_engine(int prec) { return prec == SFFT_PREC_FP64 || prec == SFFT_PREC_DF64; }

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
  if (o.precision < SFFT_PREC_AUTO || o.precision > SFFT_PREC_DF64) return SFFT_ERR_INVALID_ARG;
  if (o.box_lo > 0 || o.box_lo < -N) return SFFT_ERR_INVALID_ARG;
  const bool fp64 = o.precision == SFFT_PREC_FP64 || o.precision == SFFT_PREC_DF64;
  if (!fp64 && N > (1LL << 23)) return SFFT_ERR_PRECISION;
  if (o.tau < 0 || o.rho < 0 || o.delta < 0 || o.delta >= 0.5 || o.noise_sigma < 0 || o.max_rounds < 0)
    return SFFT_ERR_INVALID_ARG;
  if (o.residual != SFFT_RESIDUAL_BINS && o.residual != SFFT_RESIDUAL_SAMPLES) return SFFT_ERR_INVALID_ARG;
  if (o.shift != SFFT_SHIFT_COORD && o.shift != SFFT_SHIFT_BLOCK && o.shift != SFFT_SHIFT_TILT)
    return SFFT_ERR_INVALID_ARG;
  if (o.shift == SFFT_SHIFT_TILT) {
    // Alg. 3 is two-dimensional; sin and cos rational with one denominator (Eq. 25)
    const int64_t b = o.tilt_base, h = o.tilt_height, hy = o.tilt_hypo;
    if (d != 2 || b < 1 || h < 1 || b > (1 << 20) || h > (1 << 20) || b * b + h * h != hy * hy)
      return SFFT_ERR_INVALID_ARG;
    int64_t x = b, y = h;
    while (y != 0) {
      const int64_t t = x % y;
      x = y;
      y = t;
    }
    if (x != 1) return SFFT_ERR_INVALID_ARG;
    if ((double)(b + h) * (double)N > std::ldexp(1.0, 40)) return SFFT_ERR_INVALID_ARG;
  }

  std::unique_ptr<sfft_plan_s> P(new sfft_plan_s());
  SlotDesc& D = P->desc;
  D.d = d;
  D.N = N;
  D.k = k;
  D.c8 = 40;   // c = 5 (Sec. 5)
  D.box_lo = o.box_lo;
  P->prec = o.precision;
  const bool auto_ratio = o.precision == SFFT_PREC_AUTO || o.precision == SFFT_PREC_FP32_BF16DFT ||
                          o.precision == SFFT_PREC_FP32_THEN_FP64;
  D.ratio64 = (o.precision == SFFT_PREC_FP32_FP64RATIO || fp64 || (auto_ratio && N > (1LL << 14))) ? 1 : 0;
  D.dense_dft = o.precision == SFFT_PREC_FP32_BF16DFT ? 1 : 0;
  D.df_sample = o.precision == SFFT_PREC_DF64 ? 1 : 0;
  D.coef_mean = o.coef_set0 ? 0 : 1;
  D.peel_bins = o.residual == SFFT_RESIDUAL_BINS ? 1 : 0;
  D.tau = o.tau > 0 ? o.tau : (fp64 ? 1e-7 : 1e-3);
  D.rho = o.rho > 0 ? o.rho : (fp64 ? std::ldexp(1.0, -40) : std::ldexp(1.0, -17));
  D.delta = o.delta > 0 ? o.delta : (fp64 ? 0.1 : 0.25);
  D.sigma = o.noise_sigma;
  int lg = 1;
  while ((1LL << lg) < std::max<int64_t>(k, 2)) ++lg;
  D.max_rounds = o.max_rounds > 0 ? o.max_rounds : 64 + 4 * lg;
  if (D.max_rounds > SFFT_STATS_MAX_ROUNDS) D.max_rounds = SFFT_STATS_MAX_ROUNDS;
  P->stream = (cudaStream_t)stream;
  P->profile = o.profile != 0;
  P->graph = o.graph != 0;
  D.fuse = (o.unfused || D.dense_dft) ? 0 : 1;   // the fused kernel has its own (Bluestein) DFT
  if (o.fuse_max_len < 0 || o.empty_rounds < 0) return SFFT_ERR_INVALID_ARG;
  D.fuse_max_len = o.fuse_max_len;

  // ---- prime schedule
  if (ps) {
    if (ps->c_prime < 0 || ps->c_prime > 4096 || ps->c_eighths < 0 || ps->c_eighths > 8 * 4096 || ps->n_primes < 0 ||
        ps->p_min < 0 || ps->p_min > (1LL << 26))
      return SFFT_ERR_INVALID_ARG;
    if (ps->c_prime > 0) D.c8 = 8 * ps->c_prime;
    if (ps->c_eighths > 0) D.c8 = ps->c_eighths;
    D.p_min = ps->p_min;
    if (ps->n_primes > 0) {
      if (!ps->primes) return SFFT_ERR_INVALID_ARG;
      for (int i = 0; i < ps->n_primes; ++i) {
        const int64_t q = ps->primes[i];
        if (q < 2 || q > (1LL << 26)) return SFFT_ERR_INVALID_ARG;
        for (int64_t f = 2; f * f <= q; ++f)
          if (q % f == 0) return SFFT_ERR_INVALID_ARG;
        D.primes.push_back(q);
      }
    }
  }
  if (D.primes.empty()) {
    const int64_t lo = std::max<int64_t>(prime_floor_ck(D.c8, std::max<int64_t>(k, 1)), D.p_min);
    int64_t lim = lo + 64LL * D.max_rounds + 1000;
    for (;;) {
      std::vector<int64_t> pr = primes_up_to(lim);
      const int64_t pm = ith_prime_at_least(pr, D.max_rounds, lo);
      if (pm > 0) {
        D.p_max = pm;
        break;
      }
      lim *= 2;
    }
  } else {
    D.p_max = *std::max_element(D.primes.begin(), D.primes.end());
  }
  if (D.p_max > (1LL << 26) || (!fp64 && D.p_max >= (1LL << 22))) return SFFT_ERR_INVALID_ARG;

  // ---- blocks (partial unwrapping, Sec. 4.1; also the shifted sets of the block form)
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
    while (range < 4.0 * (D.c8 / 8.0) * std::max<int64_t>(k, 1) && b < d) {
      ++b;
      range *= (double)N;
    }
    const int nb = std::max(1, d / b);
    for (int q = 0; q < nb; ++q) blocks.push_back(d / nb + (q < d % nb ? 1 : 0));
  }

  // ---- line directions (the tilted form: its two rotated axes unless directions are given)
  if (o.shift == SFFT_SHIFT_TILT && !(tilts && tilts->n_dirs > 0)) {
    D.n_dirs = 2;
    D.dirs = {(int64_t)o.tilt_base, -(int64_t)o.tilt_height, (int64_t)o.tilt_height, (int64_t)o.tilt_base};
  } else if (tilts && tilts->n_dirs > 0) {
    if (!tilts->dirs) return SFFT_ERR_INVALID_ARG;
    D.dirs.assign(tilts->dirs, tilts->dirs + (size_t)tilts->n_dirs * d);
    D.n_dirs = tilts->n_dirs;
  } else {
    D.n_dirs = (int)blocks.size();
    D.dirs.assign((size_t)D.n_dirs * d, 0);
    int start = 0;
    for (int q = 0; q < D.n_dirs; ++q) {
      int64_t pw = 1;
      for (int r = 0; r < blocks[q]; ++r) {
        D.dirs[(size_t)q * d + start + r] = pw;   // N^r on the block's r-th coordinate (Eq. 35)
        if (r + 1 < blocks[q]) {
          if (pw > (int64_t)(9.0e18 / (double)N)) return SFFT_ERR_INVALID_ARG;
          pw *= N;
        }
      }
      start += blocks[q];
    }
  }

  // ---- stop rule: empty rounds in a row that end the recovery (see sfft.h)
  D.empty_rounds = o.empty_rounds > 0 ? o.empty_rounds : (fp64 ? 1 : D.n_dirs);

  // ---- shifted sets: e_n / N per coordinate, or v_n / (2 N^{d1}) per block (Alg. 2 as printed).
  // The block form reads a block's unwrapped frequency (up to N^{d1}) from one phase, so the
  // precision policy follows N^{d1}: float ratio up to 2^14, float samples up to 2^20, FP64 beyond.
  D.shift_block = o.shift == SFFT_SHIFT_BLOCK ? 1 : 0;
  if (D.shift_block) {
    double span_max = 0.0;
    for (int size : blocks) {
      if (size > 32) return SFFT_ERR_INVALID_ARG;
      const double span = std::pow((double)N, (double)size);
      if (span > std::ldexp(1.0, 40)) return SFFT_ERR_INVALID_ARG;
      span_max = std::max(span_max, span);
    }
    if (!fp64 && span_max > std::ldexp(1.0, 20)) return SFFT_ERR_PRECISION;
    if (auto_ratio) D.ratio64 = span_max > std::ldexp(1.0, 14) ? 1 : 0;
    D.shift_blocks = blocks;
  }
  // the tilted form reads a rotated coordinate (Q = (base + height) N values) from one phase:
  // the same policy as the block form's 2 N^{d1}
  D.shift_tilt = o.shift == SFFT_SHIFT_TILT ? 1 : 0;
  if (D.shift_tilt) {
    D.tilt_base = o.tilt_base;
    D.tilt_height = o.tilt_height;
    D.tilt_hypo = o.tilt_hypo;
    const double q = (double)(o.tilt_base + o.tilt_height) * (double)N;
    if (!fp64 && q > std::ldexp(1.0, 21)) return SFFT_ERR_PRECISION;
    if (auto_ratio) D.ratio64 = q > std::ldexp(1.0, 15) ? 1 : 0;
  }

  // the dense DFT takes every sample set of a signal as the N of one MMA (at most 64)
  if (D.dense_dft && (D.shift_block ? 1 + (int)D.shift_blocks.size() : d + 1) > 64) return SFFT_ERR_INVALID_ARG;
  if (o.precision == SFFT_PREC_FP32_THEN_FP64) D.stall_div = 64;
  std::vector<SlotDesc> slots(1, D);
  EngineBase* e = nullptr;
  sfft_status st = cuda_status(engine_create(fp64, slots, P->stream, P->profile, P->graph, &e));
  if (st != SFFT_OK) return st;
  P->eng.reset(e);
  if (o.precision == SFFT_PREC_FP32_THEN_FP64) {
    // the double rounds: FP64 ratio test and read-out, one empty round ends them, no stall
    // hand-over, nothing fused.  They keep the float rounds' empty-bin level: the float
    // coefficients' own errors (about 2^-20 relative) stay below it, so the double rounds end once
    // every mode is found instead of trying to isolate hundreds of residuals of that size.
    SlotDesc D64 = D;
    D64.stall_div = 0;
    D64.ratio64 = 1;
    D64.fuse = 0;
    D64.dense_dft = 0;
    D64.tau = 1e-7;
    D64.delta = 0.1;
    D64.empty_rounds = o.empty_rounds > 0 ? o.empty_rounds : 1;
    std::vector<SlotDesc> s64(1, D64);
    EngineBase* e64 = nullptr;
    st = cuda_status(engine_create(true, s64, P->stream, P->profile, P->graph, &e64));
    if (st != SFFT_OK) return st;
    P->eng64.reset(e64);
  }
  *plan_out = P.release();
  return SFFT_OK;
}

void sfft_plan_destroy(sfft_plan plan) {
  if (!plan) return;
  cudaStreamSynchronize(plan->stream);
  delete plan;
}

int64_t sfft_plan_max_prime(sfft_plan plan) { return plan ? plan->eng->max_prime() : -1; }
int64_t sfft_plan_mode_capacity(sfft_plan plan) { return plan ? plan->eng->mode_capacity() : -1; }
int sfft_plan_sets(sfft_plan plan) {
  if (!plan) return -1;
  return plan->desc.shift_block ? 1 + (int)plan->desc.shift_blocks.size() : plan->desc.d + 1;
}
int64_t sfft_plan_device_bytes(sfft_plan plan) {
  if (!plan) return -1;
  return (int64_t)(plan->eng->device_bytes() + (plan->eng64 ? plan->eng64->device_bytes() : 0));
}

sfft_status sfft_signal_synthetic(int d, int64_t N, int64_t k, const int32_t* freqs_dev, const double* coeffs_dev,
                                  double noise_sigma, uint64_t noise_seed, sfft_signal* signal_out) {
  if (!signal_out) return SFFT_ERR_INVALID_ARG;
  *signal_out = nullptr;
  if (d < 1 || N < 2 || k < 0 || (k > 0 && (!freqs_dev || !coeffs_dev))) return SFFT_ERR_INVALID_ARG;
  if (!(noise_sigma >= 0.0) || !std::isfinite(noise_sigma)) return SFFT_ERR_INVALID_ARG;
  std::unique_ptr<sfft_signal_s> S(new sfft_signal_s());
  S->noise_sigma = noise_sigma;
  S->noise_seed = noise_seed;
  S->d = d;
  S->N = N;
  S->k = k;
  S->k_cap = k;
  cudaError_t e = cudaMalloc((void**)&S->w, (size_t)std::max<int64_t>(k, 1) * d * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->a, (size_t)std::max<int64_t>(k, 1) * sizeof(double2));
  if (e == cudaSuccess && k > 0) {
    const int64_t nw = k * d;
    const int blocks = (int)std::min<int64_t>((nw + 255) / 256, 1024);
    k_signal_copy<<<blocks, 256>>>(nw, freqs_dev, S->w, k, (const double2*)coeffs_dev, S->a);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  }
  if (e != cudaSuccess) {
    cudaFree(S->w);
    cudaFree(S->a);
    return cuda_status(e);
  }
  *signal_out = S.release();
  return SFFT_OK;
}

void sfft_signal_destroy(sfft_signal signal) {
  if (!signal) return;
  cudaFree(signal->w);
  cudaFree(signal->a);
  delete signal;
}

sfft_status sfft_signal_assign(sfft_signal S, int64_t k, const int32_t* freqs_dev, const double* coeffs_dev) {
  if (!S || k < 0 || k > S->k_cap || (k > 0 && (!freqs_dev || !coeffs_dev))) return SFFT_ERR_INVALID_ARG;
  if (k > 0) {
    const int64_t nw = k * S->d;
    const int blocks = (int)std::min<int64_t>((nw + 255) / 256, 1024);
    k_signal_copy<<<blocks, 256>>>(nw, freqs_dev, S->w, k, (const double2*)coeffs_dev, S->a);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return cuda_status(e);
  }
  S->k = k;
  return SFFT_OK;
}

sfft_status sfft_signal_assign_many(int n, const sfft_signal* signals, const int64_t* ks, const int32_t* freqs_dev,
                                    const double* coeffs_dev, void* stream) {
  if (n < 0 || (n > 0 && (!signals || !ks))) return SFFT_ERR_INVALID_ARG;
  int64_t tot_w = 0, tot_a = 0, max_w = 0;
  for (int s = 0; s < n; ++s) {
    const sfft_signal_s* S = signals[s];
    if (!S || ks[s] < 0 || ks[s] > S->k_cap) return SFFT_ERR_INVALID_ARG;
    tot_w += ks[s] * S->d;
    tot_a += ks[s];
    max_w = std::max(max_w, ks[s] * S->d);
  }
  if (tot_a > 0 && (!freqs_dev || !coeffs_dev)) return SFFT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int gx = (int)std::min<int64_t>(std::max<int64_t>((max_w + 255) / 256, 1), 16);
  int64_t w_off = 0, a_off = 0;
  for (int s0 = 0; s0 < n; s0 += kAssignPerLaunch) {
    const int cnt = std::min(kAssignPerLaunch, n - s0);
    AssignArgs args;
    std::memset(&args, 0, sizeof(args));
    for (int i = 0; i < cnt; ++i) {
      sfft_signal_s* S = signals[s0 + i];
      args.d[i] = AssignDesc{S->w, S->a, w_off, a_off, ks[s0 + i] * S->d, ks[s0 + i]};
      w_off += ks[s0 + i] * S->d;
      a_off += ks[s0 + i];
    }
    k_signal_copy_many<<<dim3(gx, cnt), 256, 0, st>>>(args, cnt, freqs_dev, (const double2*)coeffs_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
  }
  for (int s = 0; s < n; ++s) signals[s]->k = ks[s];
  return SFFT_OK;
}

sfft_status sfft_execute(sfft_plan plan, sfft_signal signal, int64_t capacity, int32_t* freqs_out_dev,
                         double* coeffs_out_dev, int64_t* n_found, sfft_stats* stats) {
  if (!plan || !signal || !n_found || capacity < 0) return SFFT_ERR_INVALID_ARG;
  if (capacity > 0 && (!freqs_out_dev || !coeffs_out_dev)) return SFFT_ERR_INVALID_ARG;
  if (signal->d != plan->desc.d || signal->N != plan->desc.N || signal->k > plan->desc.k)
    return SFFT_ERR_INVALID_ARG;
  *n_found = 0;
  const int32_t* w[1] = {signal->w};
  const double2* a[1] = {signal->a};
  int64_t ks[1] = {signal->k};
  int64_t caps[1] = {capacity};
  const double ns[1] = {signal->noise_sigma};
  const uint64_t nseed[1] = {signal->noise_seed};
  int st = 0;
  sfft_stats s1;
  sfft_stats* st1 = (plan->eng64 && stats) ? &s1 : stats;
  sfft_status cs = cuda_status(
      plan->eng->run(w, a, ks, caps, ns, nseed, freqs_out_dev, (double2*)coeffs_out_dev, n_found, &st, st1));
  if (cs != SFFT_OK) return cs;
  if (!plan->eng64 || st == SFFT_OK || st == SFFT_ERR_TIMEOUT) {
    if (st1 != stats && stats) *stats = s1;
    return (sfft_status)st;
  }
  // FP32_THEN_FP64: the double rounds continue from the float registry (the outputs just written)
  int r0 = 0;
  double a_ref = 0.0;
  cs = cuda_status(plan->eng->last_state(&r0, &a_ref));
  if (cs != SFFT_OK) return cs;
  plan->eng64->set_seed(freqs_out_dev, (const double2*)coeffs_out_dev, std::min(*n_found, capacity), r0, a_ref);
  sfft_stats s2;
  cs = cuda_status(plan->eng64->run(w, a, ks, caps, ns, nseed, freqs_out_dev, (double2*)coeffs_out_dev, n_found,
                                    &st, stats ? &s2 : nullptr));
  if (cs != SFFT_OK) return cs;
  if (stats) {
    // rounds 1..r0 from the float run, the rest from the double one
    *stats = s2;
    stats->samples += s1.samples;
    stats->terms += s1.terms;
    stats->terms_fused += s1.terms_fused;
    for (int i = 0; i < std::min(r0, SFFT_STATS_MAX_ROUNDS); ++i) {
      stats->p[i] = s1.p[i];
      stats->K[i] = s1.K[i];
      stats->accepted[i] = s1.accepted[i];
      stats->registry[i] = s1.registry[i];
    }
    for (int q = 0; q < SFFT_NKCLASS; ++q) {
      stats->kernel_launches[q] += s1.kernel_launches[q];
      stats->kernel_ms[q] += s1.kernel_ms[q];
    }
  }
  return (sfft_status)st;
}

sfft_status sfft_batch_create(int n, const sfft_plan* plans, void* stream, int graph, sfft_batch* batch_out) {
  if (!batch_out || n < 1 || !plans || graph < 0 || graph > (SFFT_BATCH_GRAPH | SFFT_BATCH_PROFILE))
    return SFFT_ERR_INVALID_ARG;
  *batch_out = nullptr;
  std::unique_ptr<sfft_batch_s> B(new sfft_batch_s());
  B->n = n;
  std::vector<SlotDesc> slots;
  slots.reserve(n);
  bool profile = (graph & SFFT_BATCH_PROFILE) != 0;
  for (int s = 0; s < n; ++s) {
    if (!plans[s] || plans[s]->eng64) return SFFT_ERR_INVALID_ARG;   // FP32_THEN_FP64: plain form only
    const bool fp64 = double_engine(plans[s]->prec);
    if (s == 0) B->prec = plans[s]->prec;
    if (double_engine(B->prec) != fp64) return SFFT_ERR_INVALID_ARG;
    if (fp64 && plans[s]->prec != B->prec) return SFFT_ERR_INVALID_ARG;   // DF64 with DF64 only
    slots.push_back(plans[s]->desc);
    B->d.push_back(plans[s]->desc.d);
    B->k.push_back(plans[s]->desc.k);
    B->N.push_back(plans[s]->desc.N);
    profile = profile || plans[s]->profile;
  }
  EngineBase* e = nullptr;
  sfft_status st = cuda_status(
      engine_create(double_engine(B->prec), slots, (cudaStream_t)stream, profile, (graph & SFFT_BATCH_GRAPH) != 0,
                    &e));
  if (st != SFFT_OK) return st;
  B->eng.reset(e);
  *batch_out = B.release();
  return SFFT_OK;
}

void sfft_batch_destroy(sfft_batch batch) { delete batch; }

int64_t sfft_batch_device_bytes(sfft_batch batch) { return batch ? (int64_t)batch->eng->device_bytes() : -1; }

sfft_status sfft_batch_execute(sfft_batch batch, const sfft_signal* signals, const int64_t* capacities,
                               int32_t* freqs_out_dev, double* coeffs_out_dev, int64_t* n_found, int32_t* status,
                               sfft_stats* stats) {
  if (!batch || !signals || !capacities || !n_found || !status) return SFFT_ERR_INVALID_ARG;
  const int n = batch->n;
  std::vector<const int32_t*> w(n);
  std::vector<const double2*> a(n);
  std::vector<int64_t> ks(n);
  std::vector<double> nsig(n);
  std::vector<uint64_t> nseed(n);
  int64_t total_cap = 0;
  for (int s = 0; s < n; ++s) {
    const sfft_signal_s* S = signals[s];
    if (!S || S->d != batch->d[s] || S->N != batch->N[s] || S->k > batch->k[s] || capacities[s] < 0)
      return SFFT_ERR_INVALID_ARG;
    w[s] = S->w;
    a[s] = S->a;
    ks[s] = S->k;
    nsig[s] = S->noise_sigma;
    nseed[s] = S->noise_seed;
    total_cap += capacities[s];
  }
  if (total_cap > 0 && (!freqs_out_dev || !coeffs_out_dev)) return SFFT_ERR_INVALID_ARG;
  std::vector<int> st(n, 0);
  sfft_status cs = cuda_status(batch->eng->run(w.data(), a.data(), ks.data(), capacities, nsig.data(), nseed.data(),
                                               freqs_out_dev,
                                               (double2*)coeffs_out_dev, n_found, st.data(), stats));
  if (cs != SFFT_OK) return cs;
  int worst = SFFT_OK;
  for (int s = 0; s < n; ++s) {
    status[s] = st[s];
    if (st[s] != SFFT_OK && worst == SFFT_OK) worst = st[s];
  }
  return (sfft_status)worst;
}

sfft_status sfft_sample(sfft_plan P, int64_t p, const int64_t* u, int64_t K, const int32_t* freqs_dev,
                        const double* coeffs_dev, void* y_out_dev) {
  if (!P || !u || !y_out_dev || p < 2 || p > P->eng->max_prime() || K < 0) return SFFT_ERR_INVALID_ARG;
  if (K > 0 && (!freqs_dev || !coeffs_dev)) return SFFT_ERR_INVALID_ARG;
  if (K > P->desc.k) return SFFT_ERR_CAPACITY;
  return cuda_status(P->eng->step_sample(p, u, K, freqs_dev, (const double2*)coeffs_dev, y_out_dev));
}

sfft_status sfft_dft(sfft_plan P, int64_t p, int n_rows, const void* y_dev, void* Y_out_dev) {
  if (!P || !y_dev || !Y_out_dev || p < 2 || p > P->eng->max_prime() || n_rows < 1 || n_rows > P->desc.d + 1)
    return SFFT_ERR_INVALID_ARG;
  return cuda_status(P->eng->step_dft(p, n_rows, y_dev, Y_out_dev));
}

sfft_status sfft_classify(sfft_plan P, int64_t p, const int64_t* u, const void* Y_dev, double eta_bin,
                          int64_t capacity, int32_t* h_out_dev, int32_t* freqs_out_dev, double* coeffs_out_dev,
                          int64_t* n_out) {
  if (!P || !u || !Y_dev || !n_out || p < 2 || p > P->eng->max_prime() || eta_bin < 0 || capacity < 0 ||
      capacity > ((int64_t)1 << 30))
    return SFFT_ERR_INVALID_ARG;
  if (capacity > 0 && (!h_out_dev || !freqs_out_dev || !coeffs_out_dev)) return SFFT_ERR_INVALID_ARG;
  int err = 0;
  sfft_status st = cuda_status(P->eng->step_classify(p, u, Y_dev, eta_bin, capacity, h_out_dev, freqs_out_dev,
                                                     (double2*)coeffs_out_dev, n_out, &err));
  if (st != SFFT_OK) return st;
  if (err) {
    *n_out = std::min<int64_t>(*n_out, capacity);
    return SFFT_ERR_CAPACITY;
  }
  return SFFT_OK;
}

}  // extern "C"
