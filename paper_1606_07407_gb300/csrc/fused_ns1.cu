// The fused short-round kernel for signals of 1 sample set.
#include "fused_kernel.cuh"

namespace sfft {

template cudaError_t fused_setup_ns<1>(size_t);
template cudaError_t fused_launch_ns<1>(int, size_t, cudaStream_t, const FusedArgs&);

}  // namespace sfft
