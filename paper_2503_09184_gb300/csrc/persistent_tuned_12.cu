// persistent_tuned_12.cu -- the tuned stage-S variants 1 and 2 of the
// per-product persistent kernel at N = 2^12, L = 2 (a separate unit, compiled
// in parallel with persistent_12.cu).
#define SFHE_TUNED_TU
#include "persistent_impl.cuh"

namespace sfhe {
template cudaError_t persistent_launch_variant<12, 2, 1>(const RnsConsts&, const PersistentArgs&, cudaStream_t);
template cudaError_t persistent_launch_variant<12, 2, 2>(const RnsConsts&, const PersistentArgs&, cudaStream_t);
}  // namespace sfhe
