// chunk_launch.h -- launchers of the chunked product's gathers (slots.cu).
#pragma once
#include <cuda_runtime.h>

#include "rns.h"

namespace sfhe {

// out[q] = in[src[q]] over whole ciphertexts [2][L][N]
cudaError_t launch_gather_ct(const RnsConsts& rc, const u64* in, const int* src, long long n, u64* out, cudaStream_t s);
// C[chunk[j]] += x[list[t]] for t in ptr[j] .. ptr[j+1], in list order, for
// j < m (the additions of the single-ciphertext add)
cudaError_t launch_add_lists(const RnsConsts& rc, u64* C, const u64* x, const int* chunk, const int* ptr,
                             const int* list, long long m, cudaStream_t s);

}  // namespace sfhe
