// Internal declarations shared by the CUDA translation units of the sparse-FFT
// library: complex helpers and tile constants.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sfft.h"

namespace sfft {

// Stores a cudaError_t for sfft_last_cuda_error() of the calling thread.
void sfft_record_cuda_error(int e);

// ---------------------------------------------------------------- complex types
template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <typename T> using c2 = typename V2<T>::t;

__host__ __device__ inline float2 mk2(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 mk2(double a, double b) { return make_double2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk2(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk2(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk2(a.x, -a.y); }
template <typename C, typename S> __host__ __device__ __forceinline__ C cscale(C a, S s) {
  return mk2(a.x * s, a.y * s);
}

// ---------------------------------------------------------------- limits
constexpr int kMaxSetGroup = 8;     // sample sets accumulated per thread (register tile)
constexpr int kSampleWarps = 8;     // warps per sampling block
constexpr int kSampleChunk = 32;    // modes staged in shared memory per step

}  // namespace sfft
