// batch_uni.cu -- the persistent multi-instance kernel specialised for launches
// whose instances all share one model and one cost (see batch.cu): compiled
// apart from the general kernel so that the two build in parallel.
#include "batch_kernel.cuh"

namespace mppi {

template cudaError_t launch_k_batch<64, true>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<128, true>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<256, true>(const BatchArgs&, int, cudaStream_t);

}  // namespace mppi
