// The fused short-round kernel for signals of 3 sample sets.
#include "fused_kernel.cuh"

namespace sfft {

template cudaError_t fused_setup_ns<3>(size_t);
template cudaError_t fused_launch_ns<3>(int, size_t, cudaStream_t, const FusedArgs&);

}  // namespace sfft
