// launch_util.cuh -- small helpers shared by the launcher translation units.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "kernels.cuh"

namespace sfhe {
namespace {

// opt a kernel into more than 48 KB of dynamic shared memory (once per kernel)
template <typename K>
cudaError_t allow_smem(K* kernel, size_t bytes)
{
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> done;
    if (bytes <= 48 * 1024) return cudaSuccess;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find((const void*)kernel);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done[(const void*)kernel] = bytes;
    return e;
}

template <int LOGN>
constexpr size_t smem_of() { return (size_t)NttGeom<LOGN>::T::SMEM_WORDS * sizeof(u64); }
template <int LOGN>
constexpr int nt_of() { return NttGeom<LOGN>::T::NT; }

}  // namespace
}  // namespace sfhe
