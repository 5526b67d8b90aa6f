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
// CTA exchanges elements through shared memory.  The exchange layout keeps
// every warp access free of bank conflicts for all pass layouts: 64-bit words
// are padded by one word every R words; 32-bit words are XOR-swizzled within
// each 32-word row (no padding, so three polynomials' buffers fit beside the
// staged operands of the persistent kernel).
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
    template <bool LEAN>
    SFHE_DEV static void fwd(W& X, W& Y, W w, W ws, W q)
    {
        const W T = shoup_lazy(Y, w, ws, q);
        Y = X - T + 2 * q;
        X = X + T;
    }
    template <bool LEAN>
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
    // LEAN: min(s, s - 2b) reduces s < 4b to [0, 2b) (below 2b the
    // difference wraps above 2^31 > s); otherwise a compare and select
    SFHE_DEV static W red2(W s, W b) { return s >= 2 * b ? s - 2 * b : s; }
    SFHE_DEV static W red2_lean(W s, W b) { return min(s, s - 2 * b); }
    template <bool LEAN>
    SFHE_DEV static void fwd(W& X, W& Y, W w, W ws, W b)
    {
        const W X1 = LEAN ? red2_lean(X, b) : red2(X, b);
        const W T = shoup32_lazy(Y, w, ws, b);
        Y = X1 - T + 2 * b;
        X = X1 + T;
    }
    template <bool LEAN>
    SFHE_DEV static void inv(W& X, W& Y, W w, W ws, W b)
    {
        const W s = X + Y;
        const W d = X - Y + 2 * b;
        X = LEAN ? red2_lean(s, b) : red2(s, b);
        Y = shoup32_lazy(d, w, ws, b);
    }
    SFHE_DEV static void inv_last(W& X, W& Y, W ni, W nis, W wl, W wls, W b)
    {
        const W s = X + Y, d = X - Y + 2 * b;
        X = shoup32_lazy(s, ni, nis, b);
        Y = shoup32_lazy(d, wl, wls, b);
    }
};

// FORM_ picks code forms of the same transform (the run-time tuner's NTT
// candidates; every form computes the same values): 0 the default, 1 the
// lean forms at every size, 2 the inverse's shuffle stage where it applies.
template <int LOGN_, int LOGR_, typename A, int FORM_ = 0>
struct NttT {
    using W = typename A::W;
    static constexpr int LOGN = LOGN_;
    static constexpr int LOGR = LOGR_;
    static constexpr int N = 1 << LOGN;
    static constexpr int R = 1 << LOGR;
    static constexpr int NT = N >> LOGR;
    static constexpr int NFULL = LOGN / LOGR;
    static constexpr int REM = LOGN % LOGR;
    static constexpr bool SWIZZLE = sizeof(W) == 4;
    // Lean forms (exchange addresses as a base and per-slot constants, the
    // 32-bit reductions by an unsigned minimum): measured faster inside the
    // persistent kernel at N = 16384 and slower at N = 8192, where the
    // kernel sits at the register limit; so by default they are taken from
    // N = 16384 (form 1 takes them everywhere).
    static constexpr int FORM = FORM_;
    static constexpr bool LEAN = LOGN >= 14 || FORM == 1;
    // Inverse with one stage more than whole passes (32-bit words, form 2):
    // the stage after the first pass pairs each thread with its neighbour
    // (tid ^ 1) and runs on warp shuffles, so the passes are LOGR + 1, LOGR,
    // ... stages with one shared-memory exchange fewer.
    static constexpr bool SHUF = FORM == 2 && SWIZZLE && REM == 1;
    static constexpr int SMEM_WORDS = SWIZZLE ? N : N + (N >> LOGR);
    static_assert(!SWIZZLE || LOGR == 4 || LOGR == 5, "swizzle defined for R = 16 and 32");

    // shared-memory word of element e.  R = 16: a warp's lanes vary element
    // bits 4..8 (first pass), 0..3 and 8 (second) or 0..4 (later passes);
    // XOR-ing bits 5..8 into bank bits 0..3 and bit 8 into bank bit 4 makes
    // all 32 banks distinct in each case.  R = 32: lanes vary bits 5..9 or
    // 0..4, and XOR-ing bits 5..9 into bits 0..4 does the same.
    SFHE_DEV static int pad(int e)
    {
        if constexpr (!SWIZZLE) return e + (e >> LOGR);
        else if constexpr (LOGR == 4) return e ^ (((e >> 5) & 15) | (((e >> 8) & 1) << 4));
        else return e ^ ((e >> 5) & 31);
    }

    template <int S, int RR>
    SFHE_DEV static int idx(int v, int tid)
    {
        const int g = v >> RR, u = v & ((1 << RR) - 1);
        const int G = g * NT + tid;
        return ((G >> S) << (S + RR)) | (u << S) | (G & ((1 << S) - 1));
    }

    // layouts seen by callers
    SFHE_DEV static int run_idx(int v, int tid) { return tid * R + v; }  // inverse input / forward output
    // lane-interleaved storage of the run layout: element tid * R + v is kept
    // at v * NT + tid, so a warp's accesses to one v are consecutive words
    SFHE_DEV static int lane_idx(int v, int tid) { return v * NT + tid; }
    SFHE_DEV static int fwd_in_idx(int v, int tid)
    {
        if constexpr (REM > 0) return idx<LOGN - REM, REM>(v, tid);
        else return idx<(NFULL - 1) * LOGR, LOGR>(v, tid);
    }
    SFHE_DEV static int inv_out_idx(int v, int tid)
    {
        if constexpr (SHUF) return idx<LOGN - LOGR, LOGR>(v, tid);
        else if constexpr (REM > 0) return idx<NFULL * LOGR, REM>(v, tid);
        else return idx<(NFULL - 1) * LOGR, LOGR>(v, tid);
    }

    // Exchange addresses.  idx(v, tid) places the bits of v and of tid in
    // disjoint fields, so idx(v, tid) = idx(0, tid) | idx(v, 0); the swizzle
    // is XOR-linear and the padding additive on disjoint fields, so the word
    // of slot v is the thread's base word combined with a per-slot constant:
    // one XOR per slot (swizzled) or an immediate offset (padded).
    template <int S, int RR>
    SFHE_DEV static int slot_addr(int base, int v)
    {
        if constexpr (SWIZZLE) return base ^ pad(idx<S, RR>(v, 0));
        else return base + pad(idx<S, RR>(v, 0));
    }
    template <int S, int RR>
    SFHE_DEV static void store(const W (&x)[R], W* sm, int tid)
    {
        const int base = pad(idx<S, RR>(0, tid));
#pragma unroll
        for (int v = 0; v < R; v++) sm[LEAN ? slot_addr<S, RR>(base, v) : pad(idx<S, RR>(v, tid))] = x[v];
    }
    template <int S, int RR>
    SFHE_DEV static void load(W (&x)[R], const W* sm, int tid)
    {
        const int base = pad(idx<S, RR>(0, tid));
#pragma unroll
        for (int v = 0; v < R; v++) x[v] = sm[LEAN ? slot_addr<S, RR>(base, v) : pad(idx<S, RR>(v, tid))];
    }

    // The C twiddles (and Shoup companions) at w[ti0 .. ti0+C-1]; ti0 is a
    // multiple of C, so they come in as 16-byte (or 8-byte) vector loads.
    template <int C>
    SFHE_DEV static void tw_fetch(W (&wv)[C], W (&wsv)[C], const W* __restrict__ w, const W* __restrict__ ws, int ti0)
    {
        constexpr int V = (16 / (int)sizeof(W)) < C ? (16 / (int)sizeof(W)) : C;  // words per load
#pragma unroll
        for (int i = 0; i < C; i += V) {
            if constexpr (V == 4) {
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(w + ti0 + i));
                const uint4 b = __ldg(reinterpret_cast<const uint4*>(ws + ti0 + i));
                wv[i] = a.x, wv[i + 1] = a.y, wv[i + 2] = a.z, wv[i + 3] = a.w;
                wsv[i] = b.x, wsv[i + 1] = b.y, wsv[i + 2] = b.z, wsv[i + 3] = b.w;
            } else if constexpr (V == 2 && sizeof(W) == 4) {
                const uint2 a = __ldg(reinterpret_cast<const uint2*>(w + ti0 + i));
                const uint2 b = __ldg(reinterpret_cast<const uint2*>(ws + ti0 + i));
                wv[i] = a.x, wv[i + 1] = a.y;
                wsv[i] = b.x, wsv[i + 1] = b.y;
            } else if constexpr (V == 2) {
                const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(w + ti0 + i));
                const ulonglong2 b = __ldg(reinterpret_cast<const ulonglong2*>(ws + ti0 + i));
                wv[i] = a.x, wv[i + 1] = a.y;
                wsv[i] = b.x, wsv[i + 1] = b.y;
            } else {
                wv[i] = __ldg(w + ti0 + i);
                wsv[i] = __ldg(ws + ti0 + i);
            }
        }
    }
    // twiddles held in registers at a time: 64 bytes of each table (32 when
    // a thread holds 32 elements)
    static constexpr int TWB = (R >= 32 ? 32 : 64) / (int)sizeof(W);

    // ------------------------------------------------------------ forward ---
    // Stage D of a pass: butterflies at distance h = 2^(RR-1-D).  Register
    // slot v = g 2^RR + u, u = t 2^(RR-D) + r (r < h), uses twiddle
    // 2^lvl + ((G >> S) << D) + t, lvl = LOGN - (S+RR) + D: per group the 2^D
    // twiddles are consecutive; they are fetched TWB at a time.
    template <int S, int RR, int D>
    SFHE_DEV static void fwd_stages(W (&x)[R], int tid, const W* __restrict__ w, const W* __restrict__ ws, W q)
    {
        if constexpr (D < RR) {
            constexpr int h = 1 << (RR - 1 - D);
            constexpr int lvl = LOGN - (S + RR) + D;
            constexpr int C = 1 << D;
            constexpr int CB = C < TWB ? C : TWB;
#pragma unroll
            for (int g = 0; g < (R >> RR); g++) {
                const int G = g * NT + tid;
                const int ti0 = (1 << lvl) + ((G >> S) << D);
#pragma unroll
                for (int t0 = 0; t0 < C; t0 += CB) {
                    W wv[CB], wsv[CB];
                    tw_fetch<CB>(wv, wsv, w, ws, ti0 + t0);
#pragma unroll
                    for (int t = 0; t < CB; t++) {
#pragma unroll
                        for (int r = 0; r < h; r++) {
                            const int v = (g << RR) + ((t0 + t) << (RR - D)) + r;
                            A::template fwd<LEAN>(x[v], x[v + h], wv[t], wsv[t], q);
                        }
                    }
                }
            }
            fwd_stages<S, RR, D + 1>(x, tid, w, ws, q);
        }
    }

    template <int S, int RR>
    SFHE_DEV static void fwd_pass(W (&x)[R], int tid, const W* __restrict__ w, const W* __restrict__ ws, W q)
    {
        fwd_stages<S, RR, 0>(x, tid, w, ws, q);
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

    // Forward transform kept in shared memory, VT virtual threads of this
    // geometry per physical thread (the CTA has NT / VT threads): each pass
    // loads one virtual thread's R elements, runs its stages in registers and
    // stores them back in place, so only R elements are live per thread at a
    // time (the register-resident forward above keeps all of a thread's
    // elements across the passes).  in(e) returns input element e (natural
    // order, below 2^63); out(vt, x) receives the R outputs of virtual
    // thread vt, slots vt R .. vt R + R - 1 (the run layout).  sm holds
    // SMEM_WORDS words.
    template <int VT, typename In, typename Out>
    SFHE_DEV static void forward_looped(W* sm, int tid, const W* tw, W q, In in, Out out)
    {
        constexpr int NTP = NT / VT;
        static_assert(NTP * VT == NT, "whole virtual threads");
        const W* w = tw;
        const W* ws = tw + N;
        __syncthreads();  // earlier users of sm are done
#pragma unroll 1
        for (int j = 0; j < VT; j++) {
            const int vt = tid + j * NTP;
            W x[R];
#pragma unroll
            for (int v = 0; v < R; v++) x[v] = in(fwd_in_idx(v, vt));
            if constexpr (REM > 0) {
                fwd_pass<LOGN - REM, REM>(x, vt, w, ws, q);
                store<LOGN - REM, REM>(x, sm, vt);
            } else {
                fwd_pass<(NFULL - 1) * LOGR, LOGR>(x, vt, w, ws, q);
                if constexpr (NFULL == 1) out(vt, x);
                else store<(NFULL - 1) * LOGR, LOGR>(x, sm, vt);
            }
        }
        looped_rest<VT, (REM > 0 ? NFULL - 1 : NFULL - 2)>(sm, tid, w, ws, q, out);
    }
    template <int VT, int P, typename Out>
    SFHE_DEV static void looped_rest(W* sm, int tid, const W* w, const W* ws, W q, Out out)
    {
        if constexpr (P >= 0) {
            constexpr int NTP = NT / VT;
            __syncthreads();  // the previous pass has stored every element
#pragma unroll 1
            for (int j = 0; j < VT; j++) {
                const int vt = tid + j * NTP;
                W x[R];
                load<P * LOGR, LOGR>(x, sm, vt);
                fwd_pass<P * LOGR, LOGR>(x, vt, w, ws, q);
                if constexpr (P > 0) store<P * LOGR, LOGR>(x, sm, vt);
                else out(vt, x);
            }
            looped_rest<VT, P - 1>(sm, tid, w, ws, q, out);
        }
    }

    // ------------------------------------------------------------ inverse ---
    // The inverse transforms NP polynomials modulo the same prime at once:
    // x[j] holds polynomial j, every twiddle is fetched once for all of them,
    // and each exchange costs one pair of barriers (polynomial j exchanges
    // through sm + j * SMEM_WORDS).
    //
    // Stage D of a pass: butterflies at distance 2^D.  Register slot
    // v = g 2^RR + u, u = t 2^(D+1) + r (r < 2^D), uses twiddle
    // N / 2^(S+D+1) + ((G >> S) << (RR-D-1)) + t: per group the 2^(RR-D-1)
    // twiddles are consecutive; they are fetched TWB at a time.  The
    // transform's last stage multiplies by N^-1 (and the last twiddle) instead.
    template <int NP, int S, int RR, bool LAST, int D>
    SFHE_DEV static void inv_stages(W (&x)[NP][R], int tid, const W* __restrict__ w, const W* __restrict__ ws, W q,
                                    W ni, W nis, W wl, W wls)
    {
        if constexpr (D < RR) {
            constexpr int C = 1 << (RR - D - 1);
            constexpr int CB = C < TWB ? C : TWB;
#pragma unroll
            for (int g = 0; g < (R >> RR); g++) {
                const int G = g * NT + tid;
                const int ti0 = (N >> (S + D + 1)) + ((G >> S) << (RR - D - 1));
#pragma unroll
                for (int t0 = 0; t0 < C; t0 += CB) {
                    W wv[CB], wsv[CB];
                    if constexpr (!(LAST && D == RR - 1)) tw_fetch<CB>(wv, wsv, w, ws, ti0 + t0);
#pragma unroll
                    for (int t = 0; t < CB; t++) {
#pragma unroll
                        for (int r = 0; r < (1 << D); r++) {
                            const int v = (g << RR) + ((t0 + t) << (D + 1)) + r;
#pragma unroll
                            for (int j = 0; j < NP; j++) {
                                if constexpr (LAST && D == RR - 1)
                                    A::inv_last(x[j][v], x[j][v + (1 << D)], ni, nis, wl, wls, q);
                                else
                                    A::template inv<LEAN>(x[j][v], x[j][v + (1 << D)], wv[t], wsv[t], q);
                            }
                        }
                    }
                }
            }
            inv_stages<NP, S, RR, LAST, D + 1>(x, tid, w, ws, q, ni, nis, wl, wls);
        }
    }

    // one exchange: store in the layout of pass (S0, RR0), load in (S1, RR1)
    template <int NP, int S0, int RR0, int S1, int RR1>
    SFHE_DEV static void exchange(W (&x)[NP][R], W* sm, int tid)
    {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NP; j++) store<S0, RR0>(x[j], sm + (size_t)j * SMEM_WORDS, tid);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NP; j++) load<S1, RR1>(x[j], sm + (size_t)j * SMEM_WORDS, tid);
    }

    template <int NP, int PS>
    SFHE_DEV static void inv_rest(W (&x)[NP][R], W* sm, int tid, const W* w, const W* ws, W q, W ni, W nis, W wl,
                                  W wls)
    {
        if constexpr (PS < NFULL) {
            exchange<NP, (PS - 1) * LOGR, LOGR, PS * LOGR, LOGR>(x, sm, tid);
            inv_stages<NP, PS * LOGR, LOGR, (PS == NFULL - 1 && REM == 0), 0>(x, tid, w, ws, q, ni, nis, wl, wls);
            inv_rest<NP, PS + 1>(x, sm, tid, w, ws, q, ni, nis, wl, wls);
        } else if constexpr (PS == NFULL && REM > 0) {
            exchange<NP, (NFULL - 1) * LOGR, LOGR, NFULL * LOGR, REM>(x, sm, tid);
            inv_stages<NP, NFULL * LOGR, REM, true, 0>(x, tid, w, ws, q, ni, nis, wl, wls);
        }
    }

    // The shuffle stage (distance R, the stage after the first pass): element
    // tid R + v pairs with (tid + 1) R + v for even tid; the even thread
    // takes slots v < R/2, the odd one the others, each receiving the half it
    // lacks from its neighbour.  Afterwards slot v of thread t holds element
    // 2R (t >> 1) + (R/2) (t & 1) + (v mod R/2) + R (v div R/2).
    SFHE_DEV static int shuf_elem(int v, int tid)
    {
        return 2 * R * (tid >> 1) + (R / 2) * (tid & 1) + (v & (R / 2 - 1)) + R * (v >> (LOGR - 1));
    }
    template <int NP>
    SFHE_DEV static void shuffle_stage(W (&x)[NP][R], int tid, const W* __restrict__ w, const W* __restrict__ ws, W q)
    {
        // twiddle of the pair: N / 2^(LOGR+1) + (e >> (LOGR+1)) = ... + (tid >> 1)
        const int ti = (N >> (LOGR + 1)) + (tid >> 1);
        const W tw = __ldg(w + ti), tws = __ldg(ws + ti);
        const bool odd = tid & 1;
#pragma unroll
        for (int j = 0; j < NP; j++) {
#pragma unroll
            for (int k = 0; k < R / 2; k++) {
                const W send = odd ? x[j][k] : x[j][R / 2 + k];
                const W recv = __shfl_xor_sync(0xffffffffu, send, 1);
                W X = odd ? recv : x[j][k];
                W Y = odd ? x[j][R / 2 + k] : recv;
                A::template inv<LEAN>(X, Y, tw, tws, q);
                x[j][k] = X;
                x[j][R / 2 + k] = Y;
            }
        }
    }
    // the passes after the shuffle stage: pass PS starts at S = LOGR + 1 +
    // (PS - 1) LOGR
    template <int NP, int PS>
    SFHE_DEV static void inv_rest_shuf(W (&x)[NP][R], W* sm, int tid, const W* w, const W* ws, W q, W ni, W nis,
                                       W wl, W wls)
    {
        if constexpr (PS < NFULL) {
            constexpr int S = LOGR + 1 + (PS - 1) * LOGR;
            if constexpr (PS == 1) {
                __syncthreads();
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    W* smj = sm + (size_t)j * SMEM_WORDS;
#pragma unroll
                    for (int v = 0; v < R; v++) smj[pad(shuf_elem(v, tid))] = x[j][v];
                }
                __syncthreads();
#pragma unroll
                for (int j = 0; j < NP; j++) load<S, LOGR>(x[j], sm + (size_t)j * SMEM_WORDS, tid);
            } else {
                exchange<NP, S - LOGR, LOGR, S, LOGR>(x, sm, tid);
            }
            inv_stages<NP, S, LOGR, PS == NFULL - 1, 0>(x, tid, w, ws, q, ni, nis, wl, wls);
            inv_rest_shuf<NP, PS + 1>(x, sm, tid, w, ws, q, ni, nis, wl, wls);
        }
    }

    // x: run_idx layout in ([0, 2q)), inv_out_idx layout out ([0, 2q)).
    // (ni, nis) = N^-1 and its Shoup companion; (wl, wls) = ipsi_rev[1] N^-1.
    // sm holds NP * SMEM_WORDS words.
    template <int NP>
    SFHE_DEV static void inverse_m(W (&x)[NP][R], W* sm, int tid, const W* tw, W q, W ni, W nis, W wl, W wls)
    {
        const W* w = tw + 2 * N;
        const W* ws = tw + 3 * N;
        if constexpr (SHUF) {
            static_assert(NFULL >= 2, "the shuffle form needs two whole passes");
            inv_stages<NP, 0, LOGR, false, 0>(x, tid, w, ws, q, ni, nis, wl, wls);
            shuffle_stage<NP>(x, tid, w, ws, q);
            inv_rest_shuf<NP, 1>(x, sm, tid, w, ws, q, ni, nis, wl, wls);
        } else {
            inv_stages<NP, 0, LOGR, (NFULL == 1 && REM == 0), 0>(x, tid, w, ws, q, ni, nis, wl, wls);
            inv_rest<NP, 1>(x, sm, tid, w, ws, q, ni, nis, wl, wls);
        }
    }
    SFHE_DEV static void inverse(W (&x)[R], W* sm, int tid, const W* tw, W q, W ni, W nis, W wl, W wls)
    {
        inverse_m<1>(reinterpret_cast<W(&)[1][R]>(x), sm, tid, tw, q, ni, nis, wl, wls);
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
