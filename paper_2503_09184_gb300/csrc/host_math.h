// host_math.h -- host-side number theory and table construction for the
// RNS bases (primes, roots of unity, twiddles, base-conversion constants).
#pragma once
#include <stdint.h>
#include <vector>
#include "rns.h"

namespace sfhe {

bool is_prime_u64(uint64_t n);
// The `count` largest primes below 2^54 that are 1 mod 2N, descending.
bool ntt_primes(uint32_t N, int count, std::vector<uint64_t>& out);
// Smallest primitive 2N-th root of unity mod q.
uint64_t min_primitive_2n_root(uint64_t q, uint32_t N);
// Rounded-Gaussian |e| table (20 entries) for width sigma.
void cdt_table(double sigma, uint64_t* T);
// Twiddle tables of one prime: [4][N] = psi_rev, psi_rev_shoup, ipsi_rev,
// ipsi_rev_shoup; also N^-1 and the merged last-stage multiplier.
void twiddles(uint64_t q, uint32_t N, uint64_t* out4N, ShoupC* ninv, ShoupC* wlast);
// Fills every base-conversion constant of rc from its primes (rc.m[].q,
// rc.L, rc.Lp, rc.t, rc.N already set).
void fill_constants(RnsConsts& rc);

}  // namespace sfhe
