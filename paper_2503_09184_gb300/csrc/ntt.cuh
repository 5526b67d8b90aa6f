// ntt.cuh -- negacyclic NTT of one polynomial by one CTA.
//
// NTT form: slot i holds the evaluation at psi^(2 bitrev(i) + 1), psi the
// primitive 2N-th root of unity of the prime.  Forward is Cooley-Tukey
// (natural order in, bit-reversed out), inverse is Gentleman-Sande
// (bit-reversed in, natural out) with N^-1 merged into the last stage.
//
// Each of the NT = N / R threads keeps R = 2^LOGR elements in registers and
// runs up to LOGR butterfly stages on them (a "pass"); between passes the
// CTA exchanges elements through shared memory, padded by one word every R
// words so that both access patterns are free of bank conflicts.
//
// Register slot v of thread tid in a pass that starts at butterfly distance
// 2^S and spans RR stages holds global index
//   G = (v >> RR) * NT + tid,  e = (G >> S) << (S + RR) | (v & (2^RR-1)) << S | (G & (2^S-1)).
// The inverse's first pass has S = 0, RR = LOGR: thread tid holds the
// contiguous run tid*R .. tid*R + R-1 (loads fuse with producers); the
// forward's last pass is the same layout (stores are contiguous runs).
//
// Value ranges (Harvey's lazy reduction): forward accepts any input below
// 2^63 and adds less than 2q per stage; inverse accepts [0, 2q) and returns
// [0, 2q).
#pragma once
#include "device_math.cuh"

template <int LOGN_, int LOGR_>
struct Ntt {
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
    SFHE_DEV static int run_idx(int v, int tid) { return tid * R + v; }      // inverse input / forward output
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
    SFHE_DEV static void store(const u64 (&x)[R], u64* sm, int tid)
    {
#pragma unroll
        for (int v = 0; v < R; v++) sm[pad(idx<S, RR>(v, tid))] = x[v];
    }
    template <int S, int RR>
    SFHE_DEV static void load(u64 (&x)[R], const u64* sm, int tid)
    {
#pragma unroll
        for (int v = 0; v < R; v++) x[v] = sm[pad(idx<S, RR>(v, tid))];
    }

    // ------------------------------------------------------------ forward ---
    template <int S, int RR>
    SFHE_DEV static void fwd_pass(u64 (&x)[R], int tid, const u64* __restrict__ w, const u64* __restrict__ ws, u64 q)
    {
        const u64 two_q = 2 * q;
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
                const u64 T = shoup_lazy(x[v + h], __ldg(w + ti), __ldg(ws + ti), q);
                const u64 X = x[v];
                x[v + h] = X - T + two_q;
                x[v] = X + T;
            }
        }
    }

    template <int P>
    SFHE_DEV static void fwd_full(u64 (&x)[R], u64* sm, int tid, const u64* w, const u64* ws, u64 q)
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
    // table [4][N].  Output below (input bound) + 2 q LOGN.
    SFHE_DEV static void forward(u64 (&x)[R], u64* sm, int tid, const u64* tw, u64 q)
    {
        const u64* w = tw;
        const u64* ws = tw + N;
        if constexpr (REM > 0) fwd_pass<LOGN - REM, REM>(x, tid, w, ws, q);
        fwd_full<NFULL - 1>(x, sm, tid, w, ws, q);
    }

    // ------------------------------------------------------------ inverse ---
    template <int S, int RR, bool LAST>
    SFHE_DEV static void inv_pass(u64 (&x)[R], int tid, const u64* __restrict__ w, const u64* __restrict__ ws, u64 q,
                                  ShoupC ninv, ShoupC wlast)
    {
        const u64 two_q = 2 * q;
#pragma unroll
        for (int d = 0; d < RR; d++) {
            const bool final_stage = LAST && (d == RR - 1);
#pragma unroll
            for (int v = 0; v < R; v++) {
                const int u = v & ((1 << RR) - 1);
                if (u & (1 << d)) continue;
                const int v2 = v + (1 << d);
                const u64 X = x[v], Y = x[v2];
                if (final_stage) {
                    x[v] = shoup_lazy(X + Y, ninv, q);
                    x[v2] = shoup_lazy(X - Y + two_q, wlast, q);
                } else {
                    const int G = (v >> RR) * NT + tid;
                    const int ti = (N >> (S + d + 1)) + (((G >> S) << (RR - d - 1)) | (u >> (d + 1)));
                    u64 s = X + Y;
                    x[v] = s >= two_q ? s - two_q : s;
                    x[v2] = shoup_lazy(X - Y + two_q, __ldg(w + ti), __ldg(ws + ti), q);
                }
            }
        }
    }

    template <int P>
    SFHE_DEV static void inv_rest(u64 (&x)[R], u64* sm, int tid, const u64* w, const u64* ws, u64 q, ShoupC ninv,
                                  ShoupC wlast)
    {
        if constexpr (P < NFULL) {
            __syncthreads();
            store<(P - 1) * LOGR, LOGR>(x, sm, tid);
            __syncthreads();
            load<P * LOGR, LOGR>(x, sm, tid);
            inv_pass<P * LOGR, LOGR, (P == NFULL - 1 && REM == 0)>(x, tid, w, ws, q, ninv, wlast);
            inv_rest<P + 1>(x, sm, tid, w, ws, q, ninv, wlast);
        } else if constexpr (P == NFULL && REM > 0) {
            __syncthreads();
            store<(NFULL - 1) * LOGR, LOGR>(x, sm, tid);
            __syncthreads();
            load<NFULL * LOGR, REM>(x, sm, tid);
            inv_pass<NFULL * LOGR, REM, true>(x, tid, w, ws, q, ninv, wlast);
        }
    }

    // x: run_idx layout in ([0, 2q)), inv_out_idx layout out ([0, 2q)).
    SFHE_DEV static void inverse(u64 (&x)[R], u64* sm, int tid, const u64* tw, u64 q, ShoupC ninv, ShoupC wlast)
    {
        const u64* w = tw + 2 * N;
        const u64* ws = tw + 3 * N;
        inv_pass<0, LOGR, (NFULL == 1 && REM == 0)>(x, tid, w, ws, q, ninv, wlast);
        inv_rest<1>(x, sm, tid, w, ws, q, ninv, wlast);
    }
};

// Geometry per ring degree: threads per CTA and elements per thread.
template <int LOGN>
struct NttGeom { using T = Ntt<LOGN, 4>; };
template <>
struct NttGeom<14> { using T = Ntt<14, 5>; };
