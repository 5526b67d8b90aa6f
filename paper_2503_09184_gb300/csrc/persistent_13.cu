// persistent_13.cu -- fused persistent matmul kernels for N = 2^13.
#include "persistent_impl.cuh"

namespace sfhe {
template int persistent_occupancy<13>(int);
template cudaError_t persistent_launch<13>(const RnsConsts&, const PersistentArgs&, cudaStream_t);
}  // namespace sfhe
