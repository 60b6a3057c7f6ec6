// batch_uni_box.cu -- the shared-model variants of the persistent
// multi-instance kernel for models with the free box (flat ground, or a
// heightfield / static boxes); see batch_uni.cu.
#include "batch_kernel.cuh"

namespace mppi {

template cudaError_t launch_k_batch<64, UNI_FLAT_BOX>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<128, UNI_FLAT_BOX>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<256, UNI_FLAT_BOX>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<64, UNI_TERRAIN_BOX>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<128, UNI_TERRAIN_BOX>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<256, UNI_TERRAIN_BOX>(const BatchArgs&, int, cudaStream_t);

}  // namespace mppi
