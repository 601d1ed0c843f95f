// The fused short-round kernel for signals of 2 sample sets.
#include "fused_kernel.cuh"

namespace sfft {

template cudaError_t fused_setup_ns<2>(size_t);
template cudaError_t fused_launch_ns<2>(int, size_t, cudaStream_t, const FusedArgs&);

}  // namespace sfft
