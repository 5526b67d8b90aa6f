// persistent_12.cu -- fused persistent matmul kernels for N = 2^12.
#include "persistent_impl.cuh"

namespace sfhe {
template int persistent_occupancy<12>(int);
template cudaError_t persistent_launch<12>(const RnsConsts&, const PersistentArgs&, cudaStream_t);
}  // namespace sfhe
