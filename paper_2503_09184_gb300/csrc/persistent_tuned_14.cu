// persistent_tuned_14.cu -- the tuned stage-S variants 1 and 2 of the
// per-product persistent kernel at N = 2^14, L = 8 (a separate unit, compiled
// in parallel with persistent_14.cu).
#define SFHE_TUNED_TU
#include "persistent_impl.cuh"

namespace sfhe {
template cudaError_t persistent_launch_variant<14, 8, 1>(const RnsConsts&, const PersistentArgs&, cudaStream_t);
template cudaError_t persistent_launch_variant<14, 8, 2>(const RnsConsts&, const PersistentArgs&, cudaStream_t);
}  // namespace sfhe
