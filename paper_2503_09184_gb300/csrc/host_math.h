// host_math.h -- host-side number theory and table construction for the
// RNS bases (primes, roots of unity, twiddles, base-conversion constants).
#pragma once
#include <stdint.h>
#include <vector>
#include "rns.h"

namespace sfhe {

bool is_prime_u64(uint64_t n);
// The `count` largest primes below 2^bits that are 1 mod 2N, descending.
bool ntt_primes(uint32_t N, int count, std::vector<uint64_t>& out, int bits = 54);
// Smallest primitive 2N-th root of unity mod q.
uint64_t min_primitive_2n_root(uint64_t q, uint32_t N);
// Slot packing over Z_t[X]/(X^N + 1), t prime and 1 mod 2N: slot s of m is
// m(zeta^e_s), s = (r, j) = (s / (N/2), s mod (N/2)), e_s = 3^j (r = 0) or
// -3^j (r = 1) mod 2N, zeta the smallest primitive 2N-th root of unity mod
// t.  Outputs in [0, t); false if t or N does not fit.
bool slots_encode(uint32_t N, uint64_t t, const int64_t* vals, int64_t* poly);
bool slots_decode(uint32_t N, uint64_t t, const int64_t* poly, int64_t* vals);
// Rounded-Gaussian |e| table (20 entries) for width sigma.
void cdt_table(double sigma, uint64_t* T);
// Twiddle tables of one prime: [4][N] = psi_rev, psi_rev_shoup, ipsi_rev,
// ipsi_rev_shoup; also N^-1 and the merged last-stage multiplier.  The
// 64-bit version is for the 54-bit primes (Shoup companions over 2^64), the
// 32-bit one for the 30-bit primes (companions over 2^32).
void twiddles(uint64_t q, uint32_t N, uint64_t* out4N, ShoupC* ninv, ShoupC* wlast);
void twiddles32(uint32_t b, uint32_t N, uint32_t* out4N, Shoup32* ninv, Shoup32* wlast);
// Fills every base-conversion constant of rc from its primes (rc.m[].q,
// rc.mb[].b, rc.L, rc.K, rc.t, rc.N set).  Returns false if a size
// margin does not hold.
bool fill_constants(RnsConsts& rc);
// ninv_bx / wlast_bx = ninv_b, wlast_b (twiddles32) times 2^32 bhat_inv
// (fill_constants): the tensor stage's inverse NTT takes its input in
// Montgomery form and outputs x~_k.
void fold_tensor_scaling(RnsConsts& rc);

}  // namespace sfhe
