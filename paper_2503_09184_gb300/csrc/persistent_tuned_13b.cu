// persistent_tuned_13b.cu -- the NTT-form variants 3 and 4 of the
// per-product persistent kernel at N = 2^13, L = 4 (a separate unit, compiled
// in parallel with the others).
#define SFHE_TUNED_TU
#include "persistent_impl.cuh"

namespace sfhe {
template cudaError_t persistent_launch_variant<13, 4, 3>(const RnsConsts&, const PersistentArgs&, cudaStream_t);
template cudaError_t persistent_launch_variant<13, 4, 4>(const RnsConsts&, const PersistentArgs&, cudaStream_t);
}  // namespace sfhe
