// batch_uni.cu -- the persistent multi-instance kernel specialised for launches
// whose instances all share one model and one cost (see batch.cu), for models
// without the free box (flat ground, or a heightfield / static boxes): each
// variant holds only its model's rollout code.  Compiled apart from the general
// kernel and the free-box variants (batch_uni_box.cu) so that they build in
// parallel.
#include "batch_kernel.cuh"

namespace mppi {

template cudaError_t launch_k_batch<64, UNI_FLAT>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<128, UNI_FLAT>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<256, UNI_FLAT>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<64, UNI_TERRAIN>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<128, UNI_TERRAIN>(const BatchArgs&, int, cudaStream_t);
template cudaError_t launch_k_batch<256, UNI_TERRAIN>(const BatchArgs&, int, cudaStream_t);

}  // namespace mppi
