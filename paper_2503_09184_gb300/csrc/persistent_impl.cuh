// persistent_impl.cuh -- launchers of the fused persistent matmul kernel,
// instantiated per ring degree in persistent_<logN>.cu (parallel compiles);
// the tuned stage-S variants of the main rings in persistent_tuned_<logN>.cu.
#pragma once
#include "launch.h"
#include "launch_util.cuh"

namespace sfhe {

// rings with tuned variants 1 and 2 of the per-product kernel: the tiny, the
// sweep / layer and the mixed ring
constexpr bool has_variants(int logN, int L)
{
    return (logN == 12 && L == 2) || (logN == 13 && L == 4) || (logN == 14 && L == 8);
}

// rings with the NTT-form variants 3 and 4 (persistent_tuned_13b.cu)
constexpr bool has_ntt_variants(int logN, int L) { return logN == 13 && L == 4; }

template <int LOGN, int L>
static int occupancy_of()
{
    int blocks = 0;
    const size_t smem = PersistentPlan<LOGN, L>::SMEM;
    if (allow_smem(k_matmul_persistent<LOGN, L, false, 0>, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_matmul_persistent<LOGN, L, false, 0>, nt_of<LOGN>(),
                                                      smem) != cudaSuccess)
        return 0;
    return blocks;
}

template <int LOGN>
int persistent_occupancy(int L)
{
    switch (L) {
    case 2: return occupancy_of<LOGN, 2>();
    case 3: return occupancy_of<LOGN, 3>();
    case 4: return occupancy_of<LOGN, 4>();
    case 8: return occupancy_of<LOGN, 8>();
    default: return 0;
    }
}

// one launch of one instance, with the persisting-L2 window as a launch
// attribute (it is captured into a graph's kernel node with the launch)
template <int LOGN, int L, bool GROUPED, int V>
static cudaError_t launch_instance(const RnsConsts& rc, const PersistentArgs& a, cudaStream_t s)
{
    const size_t smem = PersistentPlan<LOGN, L>::SMEM;
    auto kern = k_matmul_persistent<LOGN, L, GROUPED, V>;
    cudaError_t e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.grid);
    cfg.blockDim = dim3((unsigned)nt_of<LOGN>());
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (a.l2_bytes) {
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[0].val.accessPolicyWindow.base_ptr = const_cast<void*>(a.l2_base);
        attr[0].val.accessPolicyWindow.num_bytes = a.l2_bytes;
        attr[0].val.accessPolicyWindow.hitRatio = a.l2_hit_ratio;
        attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, rc, a.mms, a.entries, a.n_entries, a.rowlist, a.rlk, a.rlk_sh, a.scratch,
                              a.scratch_stride, a.queue, a.stop);
}

template <int LOGN, int L>
static cudaError_t launch_one(const RnsConsts& rc, const PersistentArgs& a, cudaStream_t s)
{
    if (a.grouped) return launch_instance<LOGN, L, true, 0>(rc, a, s);
    if constexpr (has_variants(LOGN, L)) {
        if (a.variant == 1) return persistent_launch_variant<LOGN, L, 1>(rc, a, s);
        if (a.variant == 2) return persistent_launch_variant<LOGN, L, 2>(rc, a, s);
    }
    if constexpr (has_ntt_variants(LOGN, L)) {
        if (a.variant == 3) return persistent_launch_variant<LOGN, L, 3>(rc, a, s);
        if (a.variant == 4) return persistent_launch_variant<LOGN, L, 4>(rc, a, s);
    }
    if (a.variant != 0) return cudaErrorInvalidValue;
    return launch_instance<LOGN, L, false, 0>(rc, a, s);
}

template <int LOGN>
cudaError_t persistent_launch(const RnsConsts& rc, const PersistentArgs& a, cudaStream_t s)
{
    switch (rc.L) {
    case 2: return launch_one<LOGN, 2>(rc, a, s);
    case 3: return launch_one<LOGN, 3>(rc, a, s);
    case 4: return launch_one<LOGN, 4>(rc, a, s);
    case 8: return launch_one<LOGN, 8>(rc, a, s);
    default: return cudaErrorInvalidValue;
    }
}

#ifdef SFHE_TUNED_TU
// defined only in the units that instantiate the tuned variants, so that
// persistent_<logN>.cu does not compile them a second time
template <int LOGN, int L, int V>
cudaError_t persistent_launch_variant(const RnsConsts& rc, const PersistentArgs& a, cudaStream_t s)
{
    return launch_instance<LOGN, L, false, V>(rc, a, s);
}
#endif

}  // namespace sfhe
