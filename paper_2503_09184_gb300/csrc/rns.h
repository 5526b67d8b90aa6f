// rns.h -- parameter and constant tables shared by the host code and the
// kernels of the encrypted sparse matmul (RNS BFV, one ciphertext per matrix
// element).  Plain structs only; filled on the host, passed to kernels by
// value (__grid_constant__).
//
// Two RNS bases:
//   Q = q_0 .. q_{L-1}: the ciphertext modulus, primes 2^53 < q < 2^54
//       (64-bit words);
//   B = b_0 .. b_{K-1}: the tensor base, primes 2^29 < b < 2^30 (32-bit
//       words), at least twice the range of the exact integer tensor of
//       two ciphertexts (B > 2 N Q^2).
#pragma once
#include <stdint.h>

#define SFHE_MAX_L 8   // ciphertext primes
#define SFHE_MAX_K 32  // tensor-base primes

typedef uint64_t u64;
typedef uint32_t u32;

// Size of the tensor base B (K primes of 30 bits) for ring degree 2^logN and
// L ciphertext primes: B > 2 N Q^2 holds with every prime above 2^29.9 and
// Q below 2^(54 L) (the host re-checks it exactly).
constexpr int tensor_base_size(int logN, int L) { return (10 * (logN + 108 * L + 1) + 298) / 299; }

// A 54-bit modulus q and its Barrett constant floor(2^114 / q).
struct Mod {
    u64 q;
    u64 mu;
};

// A constant multiplier w < q with its Shoup companion floor(w 2^64 / q).
struct ShoupC {
    u64 w;
    u64 ws;
};

// A 30-bit modulus b with floor(2^61 / b) (values below 2^61) and
// floor(2^64 / b) (any 64-bit value).
struct Mod32 {
    u32 b;
    u32 mu61;
    u64 mu64;
    u32 binv;  // -b^-1 mod 2^32 (Montgomery reduction)
    u32 pad;
};

// A constant multiplier w < b with its Shoup companion floor(w 2^32 / b).
struct Shoup32 {
    u32 w;
    u32 ws;
};

struct RnsConsts {
    int N, logN, L, K;
    int Qwords;
    u64 t;
    u64 seed;
    Mod m[SFHE_MAX_L];
    Mod32 mb[SFHE_MAX_K];
    // NTT twiddles in device memory: Q primes [L][4][N] u64, B primes
    // [K][4][N] u32; rows psi_rev, psi_rev_shoup, ipsi_rev, ipsi_rev_shoup
    // (psi^(+-bitrev(k)), psi the smallest primitive 2N-th root).
    const u64* tw;
    const u32* twb;
    ShoupC ninv[SFHE_MAX_L], wlast[SFHE_MAX_L];
    Shoup32 ninv_b[SFHE_MAX_K], wlast_b[SFHE_MAX_K];
    // the same multiplied by 2^32 (B/b_k)^-1: an inverse NTT of the tensor in
    // Montgomery form with these outputs x~_k = [x_k (B/b_k)^-1]_{b_k}
    // directly (the tensor stage)
    Shoup32 ninv_bx[SFHE_MAX_K], wlast_bx[SFHE_MAX_K];

    // centred lift Q -> B:  a = sum_i a~_i (Q/q_i) - v Q,
    // a~_i = [a_i (Q/q_i)^-1]_{q_i}; the 54-bit a~_i is split at bit 27.
    ShoupC qhat_inv[SFHE_MAX_L];           // [(Q/q_i)^-1]_{q_i}
    u32 qhat_b[SFHE_MAX_L][SFHE_MAX_K];     // [Q/q_i]_{b_k}
    u32 qhat_b27[SFHE_MAX_L][SFHE_MAX_K];   // [2^27 Q/q_i]_{b_k}
    u32 negQ_b[SFHE_MAX_K];                 // [-Q]_{b_k}
    // exact decision of round(sum_i y_i / q_i): Q and Q/q_i as words
    u64 Qw[SFHE_MAX_L + 1];
    u64 Qhat_w[SFHE_MAX_L][SFHE_MAX_L + 1];

    // tensor x from B:  x = sum_k x~_k (B/b_k) - v B, |x| < B / 4
    Shoup32 bhat_inv[SFHE_MAX_K];           // [(B/b_k)^-1]_{b_k}
    u32 bfrac[SFHE_MAX_K];                  // floor(2^43 / b_k)

    // scale and round by t/Q, directly from B: with t (B/b_k) = alpha_k Q + r_k
    // and t B = alpha_B Q + r_B,
    //   round(t x / Q) = sum_k x~_k alpha_k - v alpha_B + round(F),
    //   F = (sum_k x~_k r_k - v r_B) / Q,
    // F estimated with rho = floor(r 2^64 / Q), decided exactly near a half.
    u32 rho_s[SFHE_MAX_K][2];                     // rho_k bits 6..34 and 35..63
    u32 rhoB_lo, rhoB_hi;                         // rho_B split in 32-bit halves
    u32 alpha_q_lo[SFHE_MAX_K][SFHE_MAX_L];       // [alpha_k]_{q_i} mod 2^27
    u32 alpha_q_hi[SFHE_MAX_K][SFHE_MAX_L];       // [alpha_k]_{q_i} >> 27
    u64 negalphaB_q[SFHE_MAX_L];                  // [-alpha_B]_{q_i}
    u64 negK_q[SFHE_MAX_L];                       // [-K]_{q_i} (removes the offset K added to F)
    u64 r_w[SFHE_MAX_K][SFHE_MAX_L + 1];          // r_k as words (exact decision)
    u64 rB_w[SFHE_MAX_L + 1];                     // r_B as words

    // products per rounding in the grouped accumulate-then-round mode:
    // floor(B / (2 N Q^2)), at most 1024
    int lazy_group;

    // encryption / decryption
    u64 delta_q[SFHE_MAX_L];                // floor(Q/t) mod q_i
    ShoupC t_q[SFHE_MAX_L];                 // t mod q_i
    u64 cdt[20];                            // Gaussian |e| table
};

// Domains of the counter-based generator (shared written definition).
enum { SFHE_DOM_SECRET = 1, SFHE_DOM_RLK_A = 2, SFHE_DOM_RLK_E = 3, SFHE_DOM_ENC_A = 4, SFHE_DOM_ENC_E = 5 };
