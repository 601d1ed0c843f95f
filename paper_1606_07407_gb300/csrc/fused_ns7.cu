// The fused short-round kernel for signals of 7 sample sets.
#include "fused_kernel.cuh"

namespace sfft {

template cudaError_t fused_setup_ns<7>(size_t);
template cudaError_t fused_launch_ns<7>(int, size_t, cudaStream_t, const FusedArgs&);

}  // namespace sfft
