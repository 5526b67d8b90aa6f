// persistent_14.cu -- fused persistent matmul kernels for N = 2^14.
#include "persistent_impl.cuh"

namespace sfhe {
template int persistent_occupancy<14>(int);
template cudaError_t persistent_launch<14>(const RnsConsts&, const PersistentArgs&, cudaStream_t);
}  // namespace sfhe
