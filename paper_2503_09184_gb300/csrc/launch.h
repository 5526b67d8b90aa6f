// launch.h -- host launchers of the kernels (kernels.cu); every launcher
// dispatches on the ring degree (and, where it matters, on L) and returns
// the launch's cudaError_t.
#pragma once
#include <cuda_runtime.h>
#include "rns.h"
#include "worklist.h"

namespace sfhe {

bool supported_ring(int logN, int L);
int ntt_threads(int logN);
size_t ntt_smem_bytes(int logN);

// batches of NTTs: polynomial (g, l) at in + g * in_gstride + (in_l0 + l) N
// -> out + g * out_gstride + (out_l0 + l) N, prime prime0 + l (of Q, or of B
// for the 32-bit version)
cudaError_t launch_ntt(const RnsConsts& rc, bool inverse, const u64* in, size_t in_gstride, int in_l0, u64* out,
                       size_t out_gstride, int out_l0, int prime0, int nlimbs, long long ngroups, cudaStream_t s);
// R of the lane-interleaved layout of lifted operands at ring degree 2^logN
int ext_interleave(int logN);
// interleaved: the NTT-form side is in the lane-interleaved layout of lifted
// operands (NttT::lane_idx) instead of natural slot order
cudaError_t launch_ntt32(const RnsConsts& rc, bool inverse, const u32* in, size_t in_gstride, int in_l0, u32* out,
                         size_t out_gstride, int out_l0, int prime0, int nlimbs, long long ngroups, bool interleaved,
                         cudaStream_t s);
cudaError_t launch_keygen(const RnsConsts& rc, u64* s_ntt, signed char* s_coeff, u64* rlk, u64* rlk_sh, int* err,
                          cudaStream_t s);
cudaError_t launch_encrypt(const RnsConsts& rc, const u64* s_ntt, const long long* vals, const int* coords, long long n,
                           u64 matrix_id, u64* ct, int* err, cudaStream_t s);
cudaError_t launch_decrypt(const RnsConsts& rc, const u64* s_ntt, const u64* ct, long long n, long long* out,
                           cudaStream_t s);
cudaError_t launch_lift_extend(const RnsConsts& rc, const u64* in, u32* out, long long ngroups, cudaStream_t s);
// plain per-product path
cudaError_t launch_tensor_intt(const RnsConsts& rc, const u32* a, const u32* b, u32* T, cudaStream_t s);
cudaError_t launch_scale_round(const RnsConsts& rc, const u32* T, u64* D, cudaStream_t s);
cudaError_t launch_relin_ntt(const RnsConsts& rc, const u64* D, u64* U, cudaStream_t s);
cudaError_t launch_relin_accum(const RnsConsts& rc, const u64* U, const u64* rlk, const u64* rlk_sh, u64* C,
                               cudaStream_t s);
// fused persistent path (persistent_<logN>.cu).  One launch: the work list,
// the key, the per-CTA scratch, the grid, the mode, the tile variant and a
// persisting-L2 access-policy window (over the relinearisation key and its
// companions; l2_bytes = 0: none).
struct PersistentArgs {
    const MmDesc* mms;
    const Entry* entries;
    int n_entries;
    const int2* rowlist;
    const u64* rlk;
    const u64* rlk_sh;
    u64* scratch;
    size_t scratch_stride;
    unsigned* queue;
    const unsigned* stop;  // nullable: once *stop != 0, no CTA takes another entry
    int grid;
    bool grouped;
    int variant;
    const void* l2_base;
    size_t l2_bytes;
    float l2_hit_ratio;
};
template <int LOGN>
int persistent_occupancy(int L);
template <int LOGN>
cudaError_t persistent_launch(const RnsConsts& rc, const PersistentArgs& a, cudaStream_t s);
// the tuned stage-S variants 1 and 2 of the rings that have them
// (persistent_tuned_<logN>.cu)
template <int LOGN, int L, int V>
cudaError_t persistent_launch_variant(const RnsConsts& rc, const PersistentArgs& a, cudaStream_t s);
// words of the per-CTA scratch of the persistent kernel (uint64 units)
size_t persistent_scratch_words(const RnsConsts& rc);
int persistent_ctas_per_sm(const RnsConsts& rc);
// tile variants of the per-product persistent kernel at this ring (1: the
// default only; 3 where the tuner has candidates) and a name for each
int persistent_variants(const RnsConsts& rc);
const char* persistent_variant_name(const RnsConsts& rc, int v);
cudaError_t launch_persistent(const RnsConsts& rc, const PersistentArgs& a, cudaStream_t s);
// slot-packed ciphertexts (slots.cu)
cudaError_t launch_galois_keygen(const RnsConsts& rc, const u64* s_ntt, u32 g, u64* key, u64* key_sh, int* err,
                                 cudaStream_t s);
cudaError_t launch_encrypt_poly(const RnsConsts& rc, const u64* s_ntt, const long long* polys, const int* coords,
                                long long n, u64 matrix_id, u64* ct, int* err, cudaStream_t s);
// w: n L N words of scratch; out: n N message digits in [0, t) (device)
cudaError_t launch_decrypt_poly(const RnsConsts& rc, const u64* s_ntt, const u64* ct, long long n, u64* w,
                                long long* out, cudaStream_t s);
cudaError_t launch_galois_apply(const RnsConsts& rc, const u64* in, long long n, u32 g, u64* out, cudaStream_t s);
cudaError_t launch_mul_plain(const RnsConsts& rc, u64* ct, long long n, const u64* pt, cudaStream_t s);
cudaError_t launch_add_ct(const RnsConsts& rc, u64* acc, const u64* x, long long n, cudaStream_t s);
size_t rotate_work_words(const RnsConsts& rc);
size_t rotate_batch_words(const RnsConsts& rc, long long n);
cudaError_t launch_rotate_batch(const RnsConsts& rc, const u64* in, size_t in_stride, long long n, u32 g,
                                const u64* key, const u64* key_sh, u64* out, size_t out_stride, u64* work,
                                long long batch, cudaStream_t s);
cudaError_t launch_rotate(const RnsConsts& rc, const u64* in, u32 g, const u64* key, const u64* key_sh, u64* out,
                          u64* work, cudaStream_t s);
// a bounded wait that runs out: sets queue[1] = 1 (selftest.cu)
cudaError_t launch_wait_selftest(unsigned* queue, u32 tries, u64 limit_ns, cudaStream_t s);
// multiplies per second of shoup32_lazy over all SMs (8 independent chains
// per thread, full occupancy), timed with events on s; synchronises s
cudaError_t measure_mulmod32(u32 b, u32 w, u32 ws, double* per_s, cudaStream_t s);
cudaError_t launch_prng(u64 seed, u64 dom, u64 o0, u64 o1, u64 o2, u64 idx0, long long n, u64* out, cudaStream_t s);

}  // namespace sfhe
