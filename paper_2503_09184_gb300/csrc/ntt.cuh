// ntt.cuh -- negacyclic NTT of one polynomial by one CTA.
//
// NTT form: slot i holds the evaluation at psi^(2 bitrev(i) + 1), psi the
// smallest primitive 2N-th root of unity of the prime.  Forward is
// Cooley-Tukey (natural order in, bit-reversed out), inverse is
// Gentleman-Sande (bit-reversed in, natural out) with N^-1 merged into the
// last stage.
//
// Each of the NT = N / R threads keeps R = 2^LOGR elements in registers and
// runs up to LOGR butterfly stages on them (a "pass"); between passes the
// CTA exchanges elements through shared memory, padded by one word every R
// words so that both access patterns are (nearly) free of bank conflicts.
//
// Register slot v of thread tid in a pass that starts at butterfly distance
// 2^S and spans RR stages holds global index
//   G = (v >> RR) * NT + tid,  e = (G >> S) << (S + RR) | (v & (2^RR-1)) << S | (G & (2^S-1)).
// The inverse's first pass has S = 0, RR = LOGR: thread tid holds the
// contiguous run tid*R .. tid*R + R-1 (loads fuse with producers); the
// forward's last pass is the same layout (stores are contiguous runs).
//
// Arithmetic policies (Harvey's lazy butterflies):
//   Arith64, primes 2^53 < q < 2^54 in 64-bit words: forward accepts any
//     input below 2^63 and adds less than 2q per stage (no reductions);
//     inverse keeps [0, 2q).
//   Arith32, primes 2^29 < b < 2^30 in 32-bit words: forward keeps [0, 4b)
//     (input below 4b), inverse keeps [0, 2b).
#pragma once
#include "device_math.cuh"

struct Arith64 {
    using W = u64;
    SFHE_DEV static void fwd(W& X, W& Y, W w, W ws, W q)
    {
        const W T = shoup_lazy(Y, w, ws, q);
        Y = X - T + 2 * q;
        X = X + T;
    }
    SFHE_DEV static void inv(W& X, W& Y, W w, W ws, W q)
    {
        const W s = X + Y;
        const W d = X - Y + 2 * q;
        X = s >= 2 * q ? s - 2 * q : s;
        Y = shoup_lazy(d, w, ws, q);
    }
    SFHE_DEV static void inv_last(W& X, W& Y, W ni, W nis, W wl, W wls, W q)
    {
        const W s = X + Y, d = X - Y + 2 * q;
        X = shoup_lazy(s, ni, nis, q);
        Y = shoup_lazy(d, wl, wls, q);
    }
};

struct Arith32 {
    using W = u32;
    SFHE_DEV static void fwd(W& X, W& Y, W w, W ws, W b)
    {
        const W X1 = X >= 2 * b ? X - 2 * b : X;
        const W T = shoup32_lazy(Y, w, ws, b);
        Y = X1 - T + 2 * b;
        X = X1 + T;
    }
    SFHE_DEV static void inv(W& X, W& Y, W w, W ws, W b)
    {
        const W s = X + Y;
        const W d = X - Y + 2 * b;
        X = s >= 2 * b ? s - 2 * b : s;
        Y = shoup32_lazy(d, w, ws, b);
    }
    SFHE_DEV static void inv_last(W& X, W& Y, W ni, W nis, W wl, W wls, W b)
    {
        const W s = X + Y, d = X - Y + 2 * b;
        X = shoup32_lazy(s, ni, nis, b);
        Y = shoup32_lazy(d, wl, wls, b);
    }
};

template <int LOGN_, int LOGR_, typename A>
struct NttT {
    using W = typename A::W;
    static constexpr int LOGN = LOGN_;
    static constexpr int LOGR = LOGR_;
    static constexpr int N = 1 << LOGN;
    static constexpr int R = 1 << LOGR;
    static constexpr int NT = N >> LOGR;
    static constexpr int NFULL = LOGN / LOGR;
    static constexpr int REM = LOGN % LOGR;
    static constexpr int SMEM_WORDS = N + (N >> LOGR);

    SFHE_DEV static int pad(int e) { return e + (e >> LOGR); }

    template <int S, int RR>
    SFHE_DEV static int idx(int v, int tid)
    {
        const int g = v >> RR, u = v & ((1 << RR) - 1);
        const int G = g * NT + tid;
        return ((G >> S) << (S + RR)) | (u << S) | (G & ((1 << S) - 1));
    }

    // layouts seen by callers
    SFHE_DEV static int run_idx(int v, int tid) { return tid * R + v; }  // inverse input / forward output
    SFHE_DEV static int fwd_in_idx(int v, int tid)
    {
        if constexpr (REM > 0) return idx<LOGN - REM, REM>(v, tid);
        else return idx<(NFULL - 1) * LOGR, LOGR>(v, tid);
    }
    SFHE_DEV static int inv_out_idx(int v, int tid)
    {
        if constexpr (REM > 0) return idx<NFULL * LOGR, REM>(v, tid);
        else return idx<(NFULL - 1) * LOGR, LOGR>(v, tid);
    }

    template <int S, int RR>
    SFHE_DEV static void store(const W (&x)[R], W* sm, int tid)
    {
#pragma unroll
        for (int v = 0; v < R; v++) sm[pad(idx<S, RR>(v, tid))] = x[v];
    }
    template <int S, int RR>
    SFHE_DEV static void load(W (&x)[R], const W* sm, int tid)
    {
#pragma unroll
        for (int v = 0; v < R; v++) x[v] = sm[pad(idx<S, RR>(v, tid))];
    }

    // ------------------------------------------------------------ forward ---
    template <int S, int RR>
    SFHE_DEV static void fwd_pass(W (&x)[R], int tid, const W* __restrict__ w, const W* __restrict__ ws, W q)
    {
#pragma unroll
        for (int d = 0; d < RR; d++) {
            const int h = 1 << (RR - 1 - d);
            const int lvl = LOGN - (S + RR) + d;
#pragma unroll
            for (int v = 0; v < R; v++) {
                const int u = v & ((1 << RR) - 1);
                if (u & h) continue;
                const int G = (v >> RR) * NT + tid;
                const int ti = (1 << lvl) + (((G >> S) << d) | (u >> (RR - d)));
                A::fwd(x[v], x[v + h], __ldg(w + ti), __ldg(ws + ti), q);
            }
        }
    }

    template <int P>
    SFHE_DEV static void fwd_full(W (&x)[R], W* sm, int tid, const W* w, const W* ws, W q)
    {
        // full pass P (S = P*LOGR) after pass P+1 (or the remainder pass)
        if constexpr (P == NFULL - 1 && REM > 0) {
            __syncthreads();
            store<LOGN - REM, REM>(x, sm, tid);
            __syncthreads();
            load<P * LOGR, LOGR>(x, sm, tid);
        } else if constexpr (P < NFULL - 1) {
            __syncthreads();
            store<(P + 1) * LOGR, LOGR>(x, sm, tid);
            __syncthreads();
            load<P * LOGR, LOGR>(x, sm, tid);
        }
        fwd_pass<P * LOGR, LOGR>(x, tid, w, ws, q);
        if constexpr (P > 0) fwd_full<P - 1>(x, sm, tid, w, ws, q);
    }

    // x: fwd_in_idx layout in, run_idx layout out.  tw points at the prime's
    // table [4][N].
    SFHE_DEV static void forward(W (&x)[R], W* sm, int tid, const W* tw, W q)
    {
        const W* w = tw;
        const W* ws = tw + N;
        if constexpr (REM > 0) fwd_pass<LOGN - REM, REM>(x, tid, w, ws, q);
        fwd_full<NFULL - 1>(x, sm, tid, w, ws, q);
    }

    // ------------------------------------------------------------ inverse ---
    template <int S, int RR, bool LAST>
    SFHE_DEV static void inv_pass(W (&x)[R], int tid, const W* __restrict__ w, const W* __restrict__ ws, W q, W ni,
                                  W nis, W wl, W wls)
    {
#pragma unroll
        for (int d = 0; d < RR; d++) {
            const bool final_stage = LAST && (d == RR - 1);
#pragma unroll
            for (int v = 0; v < R; v++) {
                const int u = v & ((1 << RR) - 1);
                if (u & (1 << d)) continue;
                const int v2 = v + (1 << d);
                if (final_stage) {
                    A::inv_last(x[v], x[v2], ni, nis, wl, wls, q);
                } else {
                    const int G = (v >> RR) * NT + tid;
                    const int ti = (N >> (S + d + 1)) + (((G >> S) << (RR - d - 1)) | (u >> (d + 1)));
                    A::inv(x[v], x[v2], __ldg(w + ti), __ldg(ws + ti), q);
                }
            }
        }
    }

    template <int P>
    SFHE_DEV static void inv_rest(W (&x)[R], W* sm, int tid, const W* w, const W* ws, W q, W ni, W nis, W wl, W wls)
    {
        if constexpr (P < NFULL) {
            __syncthreads();
            store<(P - 1) * LOGR, LOGR>(x, sm, tid);
            __syncthreads();
            load<P * LOGR, LOGR>(x, sm, tid);
            inv_pass<P * LOGR, LOGR, (P == NFULL - 1 && REM == 0)>(x, tid, w, ws, q, ni, nis, wl, wls);
            inv_rest<P + 1>(x, sm, tid, w, ws, q, ni, nis, wl, wls);
        } else if constexpr (P == NFULL && REM > 0) {
            __syncthreads();
            store<(NFULL - 1) * LOGR, LOGR>(x, sm, tid);
            __syncthreads();
            load<NFULL * LOGR, REM>(x, sm, tid);
            inv_pass<NFULL * LOGR, REM, true>(x, tid, w, ws, q, ni, nis, wl, wls);
        }
    }

    // x: run_idx layout in ([0, 2q)), inv_out_idx layout out ([0, 2q)).
    // (ni, nis) = N^-1 and its Shoup companion; (wl, wls) = ipsi_rev[1] N^-1.
    SFHE_DEV static void inverse(W (&x)[R], W* sm, int tid, const W* tw, W q, W ni, W nis, W wl, W wls)
    {
        const W* w = tw + 2 * N;
        const W* ws = tw + 3 * N;
        inv_pass<0, LOGR, (NFULL == 1 && REM == 0)>(x, tid, w, ws, q, ni, nis, wl, wls);
        inv_rest<1>(x, sm, tid, w, ws, q, ni, nis, wl, wls);
    }
};

// Geometry per ring degree: 64-bit (ciphertext primes) and 32-bit (tensor
// base) transforms; R elements per thread, N / R threads per CTA.
template <int LOGN>
struct NttGeom {
    using T = NttT<LOGN, 4, Arith64>;
    using T32 = NttT<LOGN, 4, Arith32>;
};
template <>
struct NttGeom<14> {
    using T = NttT<14, 5, Arith64>;
    using T32 = NttT<14, 5, Arith32>;
};
