// Allocation-free variant of the sampling step (kernel (a)).
//
// Some callers cannot allocate device memory when they want samples: code that
// runs under an allocator it does not own (a memory pool that must not grow, a
// host that forbids cudaMalloc after start-up), or code that is not allowed to
// create a plan and keep its buffers.  This entry point serves them: it computes
// the same samples as sfft_sample, on the caller's stream, from the caller's
// input and output buffers, and keeps its scratch (the root-of-unity table, the
// modes' projections and their per-set coefficients) in one file-scope device
// array that the library holds on every GPU it is loaded on until the process
// exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
#include <algorithm>
#include <mutex>

#include "sample_tile.cuh"

namespace sfft {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB on every device
constexpr int kNoAllocMaxD = 32;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_sample_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_dev[kNoAllocMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct NoAllocArgs {
  int d, n_sets, K, Kpad, gsize, groups, n_xt, box_lo;
  int64_t N, p;
  unsigned long long mod_m;
  int64_t u[kNoAllocMaxD];   // direction reduced mod p
};

// W[m] = e^{2 pi i m / p}; for each mode: alpha = (w . u) mod p, ga = 32 alpha mod p and
// C[n][j] = a_j e^{2 pi i w_{j,n} / N} (n >= 1), C[0][j] = a_j.
__global__ void k_na_tables(NoAllocArgs a, const int32_t* __restrict__ w, const double2* __restrict__ coeff,
                            float2* __restrict__ W, int32_t* __restrict__ alpha, int32_t* __restrict__ gam,
                            float2* __restrict__ Cm) {
  const int64_t total = a.p + a.K;
  const uint64_t up = (uint64_t)a.p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < a.p) {
      W[e] = unit_root<float>(e, a.p);
      continue;
    }
    const int j = (int)(e - a.p);
    const int32_t* wj = w + (int64_t)j * a.d;
    uint64_t acc = 0, usum = 0;
    for (int l = 0; l < a.d; ++l) {
      acc = mod_barrett((uint64_t)(int64_t)(wj[l] - a.box_lo) * (uint64_t)a.u[l] + acc, up, a.mod_m);
      usum += (uint64_t)a.u[l];
    }
    const int64_t blm = ((int64_t)a.box_lo % a.p + a.p) % a.p;
    acc = mod_barrett(acc + mod_barrett((uint64_t)blm * mod_barrett(usum, up, a.mod_m), up, a.mod_m), up, a.mod_m);
    alpha[j] = (int32_t)acc;
    gam[j] = (int32_t)mod_barrett(acc * 32u, up, a.mod_m);
    const float2 a0 = make_float2((float)coeff[j].x, (float)coeff[j].y);
    Cm[j] = a0;
    for (int n = 1; n < a.n_sets; ++n) {
      int64_t m = (int64_t)wj[n - 1] % a.N;
      if (m < 0) m += a.N;
      Cm[(int64_t)n * a.Kpad + j] = cmul(a0, unit_root<float>(m, a.N));
    }
  }
}

// one block per (sample tile, set group); every block sums all K modes
template <int NS>
__global__ void __launch_bounds__(kSampleThreads, 2)
k_na_sample(NoAllocArgs a, const int32_t* __restrict__ alpha, const int32_t* __restrict__ gam,
            const float2* __restrict__ Cm, const float2* __restrict__ W, float2* __restrict__ y) {
  __shared__ SampleSmem<float, NS> sm;
  SigCfg c;
  memset(&c, 0, sizeof(c));
  c.d = a.d;
  c.n_sets = a.n_sets;
  c.Kmax = a.Kpad;
  SigRun r;
  memset(&r, 0, sizeof(r));
  r.p = a.p;
  r.mod_m = a.mod_m;
  r.k_sig = a.K;
  r.gsize = a.gsize;
  r.groups = a.groups;
  r.n_xt = a.n_xt;
  r.splits = 1;
  r.mgroups = 1;
  r.jper = a.Kpad > 0 ? a.Kpad : kSampleChunk;
  const int xt = blockIdx.x, g = blockIdx.y;
  sample_tile<float, NS>(sm, c, r, xt, g, 0, alpha, gam, Cm, W, y);
}

cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_dev[dev] == nullptr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_sample_scratch);   // the array's device address on this device
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = ptr;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace sfft

using namespace sfft;

extern "C" sfft_status sfft_sample_noalloc(int d, int64_t N, int64_t p, const int64_t* u, int64_t K,
                                           const int32_t* freqs_dev, const double* coeffs_dev, void* y_out_dev,
                                           int box_lo, void* stream) {
  if (d < 1 || d > kNoAllocMaxD || N < 2 || N > (1LL << 23) || p < 2 || p >= (1LL << 22) || K < 0 || !u ||
      !y_out_dev || (K > 0 && (!freqs_dev || !coeffs_dev)) || box_lo > 0 || box_lo < -N)
    return SFFT_ERR_INVALID_ARG;
  // every mode takes at least 4 bytes of scratch: a K beyond that count cannot fit, and this
  // check, in 64 bits, comes before K is narrowed to int below
  if (K > (int64_t)(kNoAllocScratchBytes / sizeof(int32_t))) return SFFT_ERR_CAPACITY;
  NoAllocArgs a;
  memset(&a, 0, sizeof(a));
  a.d = d;
  a.n_sets = d + 1;
  a.K = (int)K;
  a.Kpad = (int)((K + kSampleChunk - 1) / kSampleChunk) * kSampleChunk;
  a.N = N;
  a.p = p;
  a.box_lo = box_lo;
  a.mod_m = ~0ull / (uint64_t)p;
  a.groups = (a.n_sets + kMaxSetGroup - 1) / kMaxSetGroup;
  a.gsize = (a.n_sets + a.groups - 1) / a.groups;
  a.n_xt = (int)((p / 2 + 1 + tile_x(a.gsize) - 1) / tile_x(a.gsize));   // tiles of the half line
  for (int l = 0; l < d; ++l) {
    int64_t v = u[l] % p;
    a.u[l] = v < 0 ? v + p : v;
  }
  // scratch layout: W [p] | alpha [Kpad] | ga [Kpad] | C [(d+1) x Kpad], each 256-byte aligned
  const size_t offW = 0;
  const size_t offA = align256(offW + (size_t)p * sizeof(float2));
  const size_t offG = align256(offA + (size_t)a.Kpad * sizeof(int32_t));
  const size_t offC = align256(offG + (size_t)a.Kpad * sizeof(int32_t));
  const size_t need = offC + (size_t)a.n_sets * a.Kpad * sizeof(float2);
  if (need > kNoAllocScratchBytes) return SFFT_ERR_CAPACITY;
  void* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) {
    sfft_record_cuda_error((int)e);
    return SFFT_ERR_CUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  float2* W = reinterpret_cast<float2*>(b + offW);
  int32_t* alpha = reinterpret_cast<int32_t*>(b + offA);
  int32_t* gam = reinterpret_cast<int32_t*>(b + offG);
  float2* Cm = reinterpret_cast<float2*>(b + offC);
  cudaStream_t st = (cudaStream_t)stream;
  int n_sm = 148, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tab_entries = p + K;
  const int tb = (int)std::min<int64_t>((tab_entries + 255) / 256, 4LL * n_sm);
  k_na_tables<<<tb, 256, 0, st>>>(a, freqs_dev, (const double2*)coeffs_dev, W, alpha, gam, Cm);
  const dim3 grid(a.n_xt, a.groups);
  float2* y = static_cast<float2*>(y_out_dev);
  switch (a.gsize) {
    case 1: k_na_sample<1><<<grid, kSampleThreads, 0, st>>>(a, alpha, gam, Cm, W, y); break;
    case 2: k_na_sample<2><<<grid, kSampleThreads, 0, st>>>(a, alpha, gam, Cm, W, y); break;
    case 3: k_na_sample<3><<<grid, kSampleThreads, 0, st>>>(a, alpha, gam, Cm, W, y); break;
    case 4: k_na_sample<4><<<grid, kSampleThreads, 0, st>>>(a, alpha, gam, Cm, W, y); break;
    case 5: k_na_sample<5><<<grid, kSampleThreads, 0, st>>>(a, alpha, gam, Cm, W, y); break;
    case 6: k_na_sample<6><<<grid, kSampleThreads, 0, st>>>(a, alpha, gam, Cm, W, y); break;
    case 7: k_na_sample<7><<<grid, kSampleThreads, 0, st>>>(a, alpha, gam, Cm, W, y); break;
    default: k_na_sample<8><<<grid, kSampleThreads, 0, st>>>(a, alpha, gam, Cm, W, y); break;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    sfft_record_cuda_error((int)e);
    return SFFT_ERR_CUDA;
  }
  return SFFT_OK;
}
