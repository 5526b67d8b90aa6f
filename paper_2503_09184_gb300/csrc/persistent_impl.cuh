// persistent_impl.cuh -- launchers of the fused persistent matmul kernel,
// instantiated per ring degree in persistent_<logN>.cu (parallel compiles).
#pragma once
#include "launch.h"
#include "launch_util.cuh"

namespace sfhe {

template <int LOGN, int L>
static int occupancy_of()
{
    int blocks = 0;
    const size_t smem = PersistentPlan<LOGN, L>::SMEM;
    if (allow_smem(k_matmul_persistent<LOGN, L, false>, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_matmul_persistent<LOGN, L, false>, nt_of<LOGN>(),
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

template <int LOGN, int L, bool GROUPED>
static cudaError_t launch_variant(const RnsConsts& rc, const MmDesc* mms, const Entry* entries, int n_entries,
                                  const int2* rowlist, const u64* rlk, const u64* rlk_sh, u64* scratch,
                                  size_t scratch_stride, unsigned* queue, int grid, cudaStream_t s)
{
    const size_t smem = PersistentPlan<LOGN, L>::SMEM;
    cudaError_t e = allow_smem(k_matmul_persistent<LOGN, L, GROUPED>, smem);
    if (e != cudaSuccess) return e;
    k_matmul_persistent<LOGN, L, GROUPED><<<grid, nt_of<LOGN>(), smem, s>>>(rc, mms, entries, n_entries, rowlist, rlk,
                                                                           rlk_sh, scratch, scratch_stride, queue);
    return cudaGetLastError();
}

// grouped: the grouped accumulate-then-round kernel (MmDesc::group products
// per rounding) instead of the per-product one
template <int LOGN, int L>
static cudaError_t launch_one(const RnsConsts& rc, const MmDesc* mms, const Entry* entries, int n_entries,
                              const int2* rowlist, const u64* rlk, const u64* rlk_sh, u64* scratch,
                              size_t scratch_stride, unsigned* queue, int grid, bool grouped, cudaStream_t s)
{
    return grouped ? launch_variant<LOGN, L, true>(rc, mms, entries, n_entries, rowlist, rlk, rlk_sh, scratch,
                                                   scratch_stride, queue, grid, s)
                   : launch_variant<LOGN, L, false>(rc, mms, entries, n_entries, rowlist, rlk, rlk_sh, scratch,
                                                    scratch_stride, queue, grid, s);
}

template <int LOGN>
cudaError_t persistent_launch(const RnsConsts& rc, const MmDesc* mms, const Entry* entries, int n_entries,
                              const int2* rowlist, const u64* rlk, const u64* rlk_sh, u64* scratch,
                              size_t scratch_stride, unsigned* queue, int grid, bool grouped, cudaStream_t s)
{
    switch (rc.L) {
    case 2: return launch_one<LOGN, 2>(rc, mms, entries, n_entries, rowlist, rlk, rlk_sh, scratch, scratch_stride, queue, grid, grouped, s);
    case 3: return launch_one<LOGN, 3>(rc, mms, entries, n_entries, rowlist, rlk, rlk_sh, scratch, scratch_stride, queue, grid, grouped, s);
    case 4: return launch_one<LOGN, 4>(rc, mms, entries, n_entries, rowlist, rlk, rlk_sh, scratch, scratch_stride, queue, grid, grouped, s);
    case 8: return launch_one<LOGN, 8>(rc, mms, entries, n_entries, rowlist, rlk, rlk_sh, scratch, scratch_stride, queue, grid, grouped, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sfhe
