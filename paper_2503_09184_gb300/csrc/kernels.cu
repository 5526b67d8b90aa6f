// kernels.cu -- template instantiations and launchers of the device code.
#define SFHE_KERNELS_TU
#include <stdio.h>
#include "launch.h"
#include "launch_util.cuh"

namespace sfhe {

namespace {

#define SFHE_DISPATCH_LOGN(logN, ...)               \
    switch (logN) {                                 \
    case 12: { constexpr int LG = 12; __VA_ARGS__; } \
    case 13: { constexpr int LG = 13; __VA_ARGS__; } \
    case 14: { constexpr int LG = 14; __VA_ARGS__; } \
    default: return cudaErrorInvalidValue;          \
    }

#define SFHE_DISPATCH_L(L, ...)                    \
    switch (L) {                                   \
    case 2: { constexpr int LL = 2; __VA_ARGS__; } \
    case 3: { constexpr int LL = 3; __VA_ARGS__; } \
    case 4: { constexpr int LL = 4; __VA_ARGS__; } \
    case 8: { constexpr int LL = 8; __VA_ARGS__; } \
    default: return cudaErrorInvalidValue;         \
    }

const long long kMaxGridY = 65535;

template <int LOGN>
constexpr size_t smem32_of() { return (size_t)NttGeom<LOGN>::T32::SMEM_WORDS * sizeof(u32); }
template <int LOGN>
constexpr int nt32_of() { return NttGeom<LOGN>::T32::NT; }

}  // namespace

bool supported_ring(int logN, int L)
{
    return (logN >= 12 && logN <= 14) && (L == 2 || L == 3 || L == 4 || L == 8);
}

int ntt_threads(int logN)
{
    switch (logN) {
    case 12: return nt_of<12>();
    case 13: return nt_of<13>();
    case 14: return nt_of<14>();
    default: return 0;
    }
}

size_t ntt_smem_bytes(int logN)
{
    switch (logN) {
    case 12: return smem_of<12>();
    case 13: return smem_of<13>();
    case 14: return smem_of<14>();
    default: return 0;
    }
}

template <int LOGN>
static cudaError_t ntt_impl(const RnsConsts& rc, bool inverse, const u64* in, size_t in_gstride, int in_l0, u64* out,
                            size_t out_gstride, int out_l0, int prime0, int nlimbs, long long ngroups, cudaStream_t s)
{
    const size_t smem = smem_of<LOGN>();
    cudaError_t e = inverse ? allow_smem(k_ntt_inv<LOGN>, smem) : allow_smem(k_ntt_fwd<LOGN>, smem);
    if (e != cudaSuccess) return e;
    for (long long g0 = 0; g0 < ngroups; g0 += kMaxGridY) {
        const long long ng = ngroups - g0 < kMaxGridY ? ngroups - g0 : kMaxGridY;
        dim3 grid(nlimbs, (unsigned)ng);
        const u64* src = in + g0 * in_gstride;
        u64* dst = out + g0 * out_gstride;
        if (inverse)
            k_ntt_inv<LOGN><<<grid, nt_of<LOGN>(), smem, s>>>(rc, src, in_gstride, in_l0, dst, out_gstride, out_l0, prime0);
        else
            k_ntt_fwd<LOGN><<<grid, nt_of<LOGN>(), smem, s>>>(rc, src, in_gstride, in_l0, dst, out_gstride, out_l0, prime0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_ntt(const RnsConsts& rc, bool inverse, const u64* in, size_t in_gstride, int in_l0, u64* out,
                       size_t out_gstride, int out_l0, int prime0, int nlimbs, long long ngroups, cudaStream_t s)
{
    if (ngroups <= 0 || nlimbs <= 0) return cudaSuccess;
    SFHE_DISPATCH_LOGN(rc.logN, return ntt_impl<LG>(rc, inverse, in, in_gstride, in_l0, out, out_gstride, out_l0,
                                                    prime0, nlimbs, ngroups, s));
}

template <int LOGN, bool ILV>
static cudaError_t ntt32_impl(const RnsConsts& rc, bool inverse, const u32* in, size_t in_gstride, int in_l0, u32* out,
                              size_t out_gstride, int out_l0, int prime0, int nlimbs, long long ngroups, cudaStream_t s)
{
    const size_t smem = smem32_of<LOGN>();
    cudaError_t e = inverse ? allow_smem(k_ntt32_inv<LOGN, ILV>, smem) : allow_smem(k_ntt32_fwd<LOGN, ILV>, smem);
    if (e != cudaSuccess) return e;
    for (long long g0 = 0; g0 < ngroups; g0 += kMaxGridY) {
        const long long ng = ngroups - g0 < kMaxGridY ? ngroups - g0 : kMaxGridY;
        dim3 grid(nlimbs, (unsigned)ng);
        const u32* src = in + g0 * in_gstride;
        u32* dst = out + g0 * out_gstride;
        if (inverse)
            k_ntt32_inv<LOGN, ILV><<<grid, nt32_of<LOGN>(), smem, s>>>(rc, src, in_gstride, in_l0, dst, out_gstride, out_l0,
                                                                  prime0);
        else
            k_ntt32_fwd<LOGN, ILV><<<grid, nt32_of<LOGN>(), smem, s>>>(rc, src, in_gstride, in_l0, dst, out_gstride, out_l0,
                                                                  prime0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int ext_interleave(int logN)
{
    switch (logN) {
    case 12: return NttGeom<12>::T32::R;
    case 13: return NttGeom<13>::T32::R;
    case 14: return NttGeom<14>::T32::R;
    default: return 0;
    }
}

cudaError_t launch_ntt32(const RnsConsts& rc, bool inverse, const u32* in, size_t in_gstride, int in_l0, u32* out,
                         size_t out_gstride, int out_l0, int prime0, int nlimbs, long long ngroups, bool interleaved,
                         cudaStream_t s)
{
    if (ngroups <= 0 || nlimbs <= 0) return cudaSuccess;
    if (interleaved)
        SFHE_DISPATCH_LOGN(rc.logN, return ntt32_impl<LG, true>(rc, inverse, in, in_gstride, in_l0, out, out_gstride,
                                                                out_l0, prime0, nlimbs, ngroups, s));
    SFHE_DISPATCH_LOGN(rc.logN, return ntt32_impl<LG, false>(rc, inverse, in, in_gstride, in_l0, out, out_gstride,
                                                             out_l0, prime0, nlimbs, ngroups, s));
}

template <int LOGN>
static cudaError_t keygen_impl(const RnsConsts& rc, u64* s_ntt, signed char* s_coeff, u64* rlk, u64* rlk_sh, int* err,
                               cudaStream_t s)
{
    const size_t smem = smem_of<LOGN>();
    cudaError_t e = allow_smem(k_keygen_secret<LOGN>, smem);
    if (e == cudaSuccess) e = allow_smem(k_keygen_rlk<LOGN>, smem);
    if (e != cudaSuccess) return e;
    k_keygen_secret<LOGN><<<rc.L, nt_of<LOGN>(), smem, s>>>(rc, s_ntt, s_coeff, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_keygen_rlk<LOGN><<<dim3(rc.L, rc.L), nt_of<LOGN>(), smem, s>>>(rc, s_ntt, rlk, rlk_sh, err);
    return cudaGetLastError();
}

cudaError_t launch_keygen(const RnsConsts& rc, u64* s_ntt, signed char* s_coeff, u64* rlk, u64* rlk_sh, int* err,
                          cudaStream_t s)
{
    SFHE_DISPATCH_LOGN(rc.logN, return keygen_impl<LG>(rc, s_ntt, s_coeff, rlk, rlk_sh, err, s));
}

template <int LOGN>
static cudaError_t encrypt_impl(const RnsConsts& rc, const u64* s_ntt, const long long* vals, const int* coords,
                                long long n, u64 mid, u64* ct, int* err, cudaStream_t s)
{
    const size_t smem = smem_of<LOGN>();
    cudaError_t e = allow_smem(k_encrypt<LOGN>, smem);
    if (e != cudaSuccess) return e;
    const size_t ctw = (size_t)2 * rc.L * rc.N;
    for (long long n0 = 0; n0 < n; n0 += kMaxGridY) {
        const long long nn = n - n0 < kMaxGridY ? n - n0 : kMaxGridY;
        k_encrypt<LOGN><<<dim3(rc.L, (unsigned)nn), nt_of<LOGN>(), smem, s>>>(rc, s_ntt, vals + n0, coords + 2 * n0, mid,
                                                                              ct + n0 * ctw, err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_encrypt(const RnsConsts& rc, const u64* s_ntt, const long long* vals, const int* coords, long long n,
                           u64 matrix_id, u64* ct, int* err, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    SFHE_DISPATCH_LOGN(rc.logN, return encrypt_impl<LG>(rc, s_ntt, vals, coords, n, matrix_id, ct, err, s));
}

cudaError_t launch_decrypt(const RnsConsts& rc, const u64* s_ntt, const u64* ct, long long n, long long* out,
                           cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    SFHE_DISPATCH_LOGN(rc.logN, k_decrypt<LG><<<(unsigned)n, 256, 0, s>>>(rc, s_ntt, ct, out); return cudaGetLastError());
}

cudaError_t launch_lift_extend(const RnsConsts& rc, const u64* in, u32* out, long long ngroups, cudaStream_t s)
{
    const long long total = ngroups * rc.N;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    SFHE_DISPATCH_LOGN(rc.logN, SFHE_DISPATCH_L(rc.L, {
        k_lift_extend<LL, Cfg<LG, LL>::K><<<blocks, 256, 0, s>>>(rc, in, out, (int)ngroups);
        return cudaGetLastError();
    }));
}

cudaError_t launch_tensor_intt(const RnsConsts& rc, const u32* a, const u32* b, u32* T, cudaStream_t s)
{
    SFHE_DISPATCH_LOGN(rc.logN, SFHE_DISPATCH_L(rc.L, {
        cudaError_t e = allow_smem(k_tensor_intt<LG, LL>, smem32_of<LG>());
        if (e != cudaSuccess) return e;
        k_tensor_intt<LG, LL><<<dim3(rc.K, 3), nt32_of<LG>(), smem32_of<LG>(), s>>>(rc, a, b, T);
        return cudaGetLastError();
    }));
}

cudaError_t launch_scale_round(const RnsConsts& rc, const u32* T, u64* D, cudaStream_t s)
{
    dim3 grid((rc.N + 127) / 128, 3);
    SFHE_DISPATCH_LOGN(rc.logN, SFHE_DISPATCH_L(rc.L, {
        k_scale_round<LG, LL><<<grid, 128, 0, s>>>(rc, T, D);
        return cudaGetLastError();
    }));
}

cudaError_t launch_relin_ntt(const RnsConsts& rc, const u64* D, u64* U, cudaStream_t s)
{
    SFHE_DISPATCH_LOGN(rc.logN, {
        cudaError_t e = allow_smem(k_relin_ntt<LG>, smem_of<LG>());
        if (e != cudaSuccess) return e;
        k_relin_ntt<LG><<<dim3(rc.L, rc.L + 2), nt_of<LG>(), smem_of<LG>(), s>>>(rc, D, U);
        return cudaGetLastError();
    });
}

cudaError_t launch_relin_accum(const RnsConsts& rc, const u64* U, const u64* rlk, const u64* rlk_sh, u64* C,
                               cudaStream_t s)
{
    k_relin_accum<<<dim3((rc.N + 255) / 256, rc.L), 256, 0, s>>>(rc, U, rlk, rlk_sh, C);
    return cudaGetLastError();
}

size_t persistent_scratch_words(const RnsConsts& rc)
{
    const size_t N = rc.N, L = rc.L, K = rc.K;
    const size_t w = 3 * L * N + 2 * N + (3 * K * N + 1) / 2;
    return (w + 31) & ~(size_t)31;  // 256-byte aligned slots
}

int persistent_ctas_per_sm(const RnsConsts& rc)
{
    switch (rc.logN) {
    case 12: return persistent_occupancy<12>(rc.L);
    case 13: return persistent_occupancy<13>(rc.L);
    case 14: return persistent_occupancy<14>(rc.L);
    default: return 0;
    }
}

cudaError_t launch_persistent(const RnsConsts& rc, const PersistentArgs& a, cudaStream_t s)
{
    switch (rc.logN) {
    case 12: return persistent_launch<12>(rc, a, s);
    case 13: return persistent_launch<13>(rc, a, s);
    case 14: return persistent_launch<14>(rc, a, s);
    default: return cudaErrorInvalidValue;
    }
}

int persistent_variants(const RnsConsts& rc)
{
    if (rc.logN == 13 && rc.L == 4) return 5;  // three stage-S tiles, two NTT forms
    const bool v = (rc.logN == 12 && rc.L == 2) || (rc.logN == 14 && rc.L == 8);
    return v ? 3 : 1;
}

// the tiles of PersistentTile, as the host names them
static_assert(PersistentTile<13, 4, 0>::SM == 2 && PersistentTile<13, 4, 0>::LS == 4, "tile table");
static_assert(PersistentTile<13, 4, 1>::SM == 2 && PersistentTile<13, 4, 1>::LS == 2, "tile table");
static_assert(PersistentTile<13, 4, 2>::SM == 1 && PersistentTile<13, 4, 2>::LS == 4, "tile table");
static_assert(PersistentTile<13, 4, 3>::SM == 2 && PersistentTile<13, 4, 3>::LS == 2 &&
                  PersistentTile<13, 4, 3>::NB::LEAN, "tile table");
static_assert(PersistentTile<13, 4, 4>::SM == 2 && PersistentTile<13, 4, 4>::LS == 2 &&
                  PersistentTile<13, 4, 4>::NB::SHUF, "tile table");
static_assert(!PersistentTile<13, 4, 1>::NB::LEAN && !PersistentTile<13, 4, 1>::NB::SHUF, "tile table");
static_assert(PersistentTile<14, 8, 0>::SM == 1 && PersistentTile<14, 8, 0>::LS == 8, "tile table");
static_assert(PersistentTile<14, 8, 1>::SM == 1 && PersistentTile<14, 8, 1>::LS == 4, "tile table");
static_assert(PersistentTile<14, 8, 2>::SM == 1 && PersistentTile<14, 8, 2>::LS == 2, "tile table");
static_assert(PersistentTile<12, 2, 0>::SM == 2 && PersistentTile<12, 2, 0>::LS == 2, "tile table");
static_assert(PersistentTile<12, 2, 1>::SM == 2 && PersistentTile<12, 2, 1>::LS == 1, "tile table");
static_assert(PersistentTile<12, 2, 2>::SM == 1 && PersistentTile<12, 2, 2>::LS == 2, "tile table");

const char* persistent_variant_name(const RnsConsts& rc, int v)
{
    static const char* names[][5] = {
        {"2 coefficients per thread, 4 primes per pass", "2 coefficients per thread, 2 primes per pass",
         "1 coefficient per thread, 4 primes per pass",
         "2 coefficients per thread, 2 primes per pass; lean NTT exchange addresses and reductions",
         "2 coefficients per thread, 2 primes per pass; inverse NTT with a warp-shuffle stage"},
        {"1 coefficient per thread, 8 primes per pass", "1 coefficient per thread, 4 primes per pass",
         "1 coefficient per thread, 2 primes per pass", "", ""},
        {"2 coefficients per thread, 2 primes per pass", "2 coefficients per thread, 1 prime per pass",
         "1 coefficient per thread, 2 primes per pass", "", ""},
    };
    if (v < 0 || v >= persistent_variants(rc)) return "";
    if (persistent_variants(rc) == 1) return "default stage-S tile";
    return names[rc.logN == 13 ? 0 : (rc.logN == 14 ? 1 : 2)][v];
}

cudaError_t launch_prng(u64 seed, u64 dom, u64 o0, u64 o1, u64 o2, u64 idx0, long long n, u64* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_prng_words<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seed, dom, o0, o1, o2, idx0, n, out);
    return cudaGetLastError();
}

}  // namespace sfhe
