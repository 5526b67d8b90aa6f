// rns.h -- parameter and constant tables shared by the host code and the
// kernels of the encrypted sparse matmul (RNS BFV, one ciphertext per matrix
// element).  Plain structs only; filled on the host, passed to kernels by
// value (__grid_constant__).
#pragma once
#include <stdint.h>

#define SFHE_MAX_L 8               // ciphertext primes (Q base)
#define SFHE_MAX_P (SFHE_MAX_L + 1)  // extension primes (P base), L + 1 of them
#define SFHE_MAX_QP (SFHE_MAX_L + SFHE_MAX_P)

typedef uint64_t u64;
typedef uint32_t u32;

// A modulus q with 2^53 < q < 2^54 and its Barrett constant floor(2^114 / q).
struct Mod {
    u64 q;
    u64 mu;
};

// A constant multiplier w < q with its Shoup companion floor(w 2^64 / q).
struct ShoupC {
    u64 w;
    u64 ws;
};

// Everything a kernel needs about the RNS bases Q = q_0..q_{L-1} and
// P = p_0..p_{L}.  Index convention for prime arrays over Q u P: 0..L-1 are
// the q_i, L..L+Lp-1 the p_j.
struct RnsConsts {
    int N, logN, L, Lp;
    u64 t;
    u64 seed;
    Mod m[SFHE_MAX_QP];
    // NTT: twiddle tables live in device memory, [prime][4][N]:
    // psi_rev, psi_rev_shoup, ipsi_rev, ipsi_rev_shoup (psi^(+-bitrev(k)))
    const u64* tw;
    ShoupC ninv[SFHE_MAX_QP];    // N^-1
    ShoupC wlast[SFHE_MAX_QP];   // ipsi_rev[1] * N^-1 (last inverse stage)

    // centred lift Q -> P
    ShoupC qhat_inv[SFHE_MAX_L];                 // [(Q/q_i)^-1]_{q_i}
    u64 qhat_mod_p[SFHE_MAX_L][SFHE_MAX_P];      // [Q/q_i]_{p_j}
    u64 negQ_mod_p[SFHE_MAX_P];                  // [-Q]_{p_j}
    // exact fallback of round(sum_i y_i / q_i): Q and Q/q_i as words
    int Qwords;
    u64 Qw[SFHE_MAX_L + 1];
    u64 Qhat_w[SFHE_MAX_L][SFHE_MAX_L + 1];

    // scale and round by t/Q from Q u P, result first in base P
    ShoupC qphat_inv[SFHE_MAX_L];                // [(QP/q_i)^-1]_{q_i}
    ShoupC tP_q[SFHE_MAX_L];                     // [t P]_{q_i}
    u64 omega[SFHE_MAX_L][SFHE_MAX_P];           // [floor(t P / q_i)]_{p_j}
    ShoupC tQinv_p[SFHE_MAX_P];                  // [t Q^-1]_{p_j}
    // base P -> Q (centred)
    ShoupC phat_inv[SFHE_MAX_P];                 // [(P/p_j)^-1]_{p_j}
    u64 phat_mod_q[SFHE_MAX_P][SFHE_MAX_L];      // [P/p_j]_{q_i}
    u64 negP_mod_q[SFHE_MAX_L];                  // [-P]_{q_i}

    // encryption / decryption
    u64 delta_q[SFHE_MAX_L];                     // floor(Q/t) mod q_i
    ShoupC t_q[SFHE_MAX_L];                      // t mod q_i
    u64 cdt[20];                                 // Gaussian |e| table
};

// Domains of the counter-based generator (shared written definition).
enum { SFHE_DOM_SECRET = 1, SFHE_DOM_RLK_A = 2, SFHE_DOM_RLK_E = 3, SFHE_DOM_ENC_A = 4, SFHE_DOM_ENC_E = 5 };
