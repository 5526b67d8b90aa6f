// persistent_13.cu -- fused persistent matmul kernels for N = 2^13.
#include "persistent_impl.cuh"

namespace sfhe {
template int persistent_occupancy<13>(int);
template cudaError_t persistent_launch<13>(const RnsConsts&, const MmDesc*, const Entry*, int, const int2*, const u64*,
                                           const u64*, u64*, size_t, unsigned*, int, bool, cudaStream_t);
}  // namespace sfhe
