/*
 * sfhe.h -- C ABI of the GB300 encrypted sparse matrix multiplication.
 *
 * The operation is the paper's encrypted matrix product (Ferguson et al.,
 * "Exploiting Unstructured Sparsity in Fully Homomorphic Encrypted DNNs",
 * Alg. 1 and Sec. 3.3): C[i][j] = sum over k of Relin(A[i][k] x B[k][j]),
 * every matrix element encrypted in its own ciphertext (chunk size c = 1),
 * with the k-loop running over every k (naive dense) or only over the
 * nonzeros of A listed by one of the three sparse encodings (naive sparse
 * mask, CSR, ELLPACK; Sec. 3.3.2).  The scheme is RNS BFV: ring
 * Z[X]/(X^N + 1), ciphertext modulus Q = q_0 ... q_{L-1} (the L largest
 * primes below 2^54 with q = 1 mod 2N), plaintext modulus t, ternary secret,
 * rounded Gaussian errors, relinearisation key with one digit per prime.
 * Each message is placed in the constant coefficient.
 *
 * Conventions for every entry point:
 *  - Status codes only; no exception crosses the ABI.  sfhe_last_error()
 *    returns a message for the calling thread's last failure.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on it unless stated; arguments are
 *    validated on the host before anything is launched.
 *  - "device" pointers are CUDA device memory owned by the caller (for
 *    example torch tensors); "host" pointers are ordinary host memory owned
 *    by the caller and only read during the call.  The library owns only
 *    what a handle holds (sfhe_ctx, sfhe_matrix, sfhe_plan,
 *    sfhe_host_plan, sfhe_rotkeys); the caller releases each with its
 *    *_destroy call.
 *  - Two ways to hold operands: sfhe_matrix, an opaque handle whose device
 *    memory the library allocates and frees (the calls of the paper's
 *    problem statement: encrypted inputs A and B with their matrix
 *    structure in, the encrypted product out), and sfhe_matrix_view, a
 *    plain descriptor over device buffers the caller allocated (for callers
 *    that manage device memory themselves: plans, CUDA graphs, serving).
 *  - Ciphertext layouts (uint64 words, canonical residues):
 *      ciphertext  [2 (c0, c1)][L][N], NTT form (slot i = evaluation at
 *                  psi^(2 bitrev(i) + 1), psi the smallest primitive 2N-th
 *                  root of unity mod the limb's prime);
 *      lifted      [2][K][N] uint32, NTT form over the tensor base
 *                  B = b_0 .. b_{K-1}: the K largest primes below 2^30 with
 *                  b = 1 mod 2N, enough that B > 2 N Q^2 (twice the range
 *                  of the exact integer tensor of two ciphertexts), stored
 *                  lane-interleaved: slot i at (i mod R) (N / R) + i / R,
 *                  R = sfhe_info.ext_interleave (the layout the kernels
 *                  read with consecutive addresses across a warp);
 *      coefficient [2][L][N] in coefficient form (sfhe_to_coeff).
 */
#ifndef SFHE_H
#define SFHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFHE_OK = 0,
    SFHE_EINVAL = 1,       /* malformed argument (null pointer, bad index array) */
    SFHE_ESHAPE = 2,       /* operand shapes do not match */
    SFHE_ENOMEM = 3,       /* device allocation failed or workspace too small */
    SFHE_ECUDA = 4,        /* a CUDA runtime call failed */
    SFHE_ETIMEOUT = 5,     /* a bounded device wait gave up (sfhe_matmul_check) */
    SFHE_EBUDGET = 6,      /* reserved: request over a memory budget */
    SFHE_EUNSUPPORTED = 7, /* parameters outside what the kernels implement */
    SFHE_EDEVICE = 8       /* a kernel reported a failure through the status word */
} sfhe_status;

/* Sec. 3.3: naive dense (Alg. 1), naive sparse (plaintext zero mask), CSR, ELLPACK */
typedef enum { SFHE_ENC_DENSE = 0, SFHE_ENC_MASK = 1, SFHE_ENC_CSR = 2, SFHE_ENC_ELL = 3 } sfhe_encoding;

/* execution modes of a matmul.  SFHE_EXEC_LAZY is not the paper's order of
 * operations: an output entry's products (ascending k) are taken in groups of
 * G = sfhe_info.lazy_group; each group's exact tensors are summed, scaled and
 * rounded once and relinearised once, and the groups are added.  The result
 * is a different ciphertext with the same decryption (the rounding and
 * relinearisation noise is added once per group instead of once per
 * product); G = 1 would be Alg. 1's per-product order. */
enum {
    SFHE_EXEC_PLAIN = 1,      /* one short launch sequence per ciphertext product */
    SFHE_EXEC_PERSISTENT = 2, /* all products of all matmuls in one persistent launch */
    SFHE_EXEC_GRAPH = 4,      /* with PERSISTENT: replay the launch as a CUDA graph */
    SFHE_EXEC_LAZY = 8        /* with PERSISTENT: grouped accumulate-then-round (below) */
};

typedef struct {
    uint32_t N;    /* ring degree: 4096, 8192 or 16384 */
    uint32_t L;    /* ciphertext primes: 2, 3, 4 or 8 */
    uint64_t t;    /* plaintext modulus, 2 <= t < 2^32 */
    double sigma;  /* error width; the rounded Gaussian is cut at 19 */
} sfhe_params;

typedef struct {
    uint32_t N, L;
    uint32_t K;             /* tensor-base primes */
    uint64_t t;
    uint64_t q[8];          /* ciphertext primes, descending */
    uint32_t b[32];         /* tensor-base primes, descending */
    uint64_t ct_words;      /* 2 L N (uint64 words) */
    uint64_t ext_words;     /* 2 K N (uint32 words) */
    int32_t num_sms;
    uint32_t ext_interleave; /* R of the lifted layout (16, or 32 at N = 16384) */
    int32_t lazy_group;      /* G of SFHE_EXEC_LAZY: floor(B / (2 N Q^2)), at most 1024 */
    uint64_t l2_window;      /* bytes of the persisting-L2 window over the relinearisation key (0: none) */
    float l2_hit_ratio;      /* its hit ratio (the persisting limit over the window) */
} sfhe_info;

typedef struct sfhe_ctx sfhe_ctx;
typedef struct sfhe_plan sfhe_plan;
/* an encoded, encrypted matrix in device memory the library owns */
typedef struct sfhe_matrix sfhe_matrix;
/* a matmul with host-resident operands (sfhe_matmul_host) */
typedef struct sfhe_host_plan sfhe_host_plan;

/*
 * Encoded left or right operand (Sec. 3.3.2).  Plaintext structure arrays
 * are host memory; ciphertext storage is device memory.
 *   DENSE: nct = rows*cols, ciphertext r*cols + c encrypts element (r, c).
 *   MASK:  as DENSE plus mask[rows*cols], 1 where the element is zero
 *          (B_ik = [M_ik = 0]); products with a set mask are skipped.  A
 *          right operand may be MASK-encoded too: the sparse matmuls then
 *          skip k wherever A[i][k] or B[k][j] is zero, the naive sparse
 *          condition of Sec. 3.3.2 over both operands (the dense loop of
 *          Alg. 1 still takes every k).
 *   CSR:   row_ptr[rows+1], col_idx[nct]; ciphertext t encrypts the t-th
 *          nonzero in row-major order.
 *   ELL:   ell_width slots per row, ell_col[rows*ell_width] (-1 = padding);
 *          ciphertext r*ell_width + s encrypts slot s of row r (padding slots
 *          hold encryptions of zero and are skipped).
 * `ct` [nct][2][L][N] (uint64) and `ext` [nct][2][K][N] (uint32) are device
 * buffers; the matmul reads `ext` of A and B (fill it with sfhe_lift) and
 * writes `ct` of C (which must be DENSE, rows*cols ciphertexts).
 */
typedef struct {
    int32_t rows, cols, encoding, nct, ell_width;
    const uint8_t* mask;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const int32_t* ell_col;
    uint64_t* ct;
    uint32_t* ext;
} sfhe_matrix_view;

/* ------------------------------------------------------------ context --- */
/* Parameters and keys.  Selects the primes, builds the NTT and base
 * conversion tables, and runs key generation on the current device from
 * `seed` (secret and relinearisation key never leave the device unless
 * exported).  Synchronous.  The key and its Shoup companions share one
 * allocation, over which every persistent launch carries a persisting-L2
 * access-policy window: the context raises its persisting-L2 limit (a limit
 * of this process's CUDA context, gone with it) up to the key's size.  The
 * environment variable SFHE_L2_PERSIST=0 leaves the limit alone and launches
 * without the window.  Errors: EINVAL (null), EUNSUPPORTED (N, L or t
 * outside the list above), ECUDA / ENOMEM (device), EDEVICE (sampling). */
sfhe_status sfhe_ctx_create(const sfhe_params* params, uint64_t seed, sfhe_ctx** out);
void sfhe_ctx_destroy(sfhe_ctx* ctx);
sfhe_status sfhe_ctx_info(const sfhe_ctx* ctx, sfhe_info* out);
/* Synchronises `stream` and reads the context's device status word (set by
 * encryption / key generation when a sampler exhausted its retries). */
sfhe_status sfhe_ctx_check(sfhe_ctx* ctx, void* stream);
const char* sfhe_last_error(void);

/* Host-only helpers (no device needed).  Primes: q[L] the L largest primes
 * below 2^54 that are 1 mod 2N; b[*K] the *K largest below 2^30 of the same
 * form (the tensor base); primality by deterministic Miller-Rabin with the
 * bases 2..37.  CDT: T[k] = floor(2^63 P(|e| <= k)) of the rounded Gaussian
 * of width sigma, k < 19, T[19] = 2^63. */
sfhe_status sfhe_select_primes(uint32_t N, uint32_t L, uint64_t* q, uint32_t* b, int32_t* K);
sfhe_status sfhe_cdt_table(double sigma, uint64_t* T20);

/* ---------------------------------------------------------- operands --- */
/* Structure of a plaintext matrix (host values[rows*cols], row-major) under
 * an encoding (Sec. 3.3.2: the naive sparse mask, CSR, ELLPACK): fills *nct
 * and *ell_width. */
sfhe_status sfhe_encode_count(const int64_t* values, int32_t rows, int32_t cols, int32_t encoding, int32_t* nct,
                              int32_t* ell_width);
/* Fills the structure arrays (each may be NULL when the encoding has none)
 * and, per stored ciphertext, the value it encrypts (ct_values[nct]) and its
 * stream coordinates (ct_coords[2*nct]: row, col; ELL padding slot s of row
 * r has col = cols + s). */
sfhe_status sfhe_encode_fill(const int64_t* values, int32_t rows, int32_t cols, int32_t encoding, uint8_t* mask,
                             int32_t* row_ptr, int32_t* col_idx, int32_t* ell_col, int64_t* ct_values,
                             int32_t* ct_coords);

/* Memory an encoded operand holds (the per-scheme ciphertext memory of
 * Sec. 4.6, Fig. 4), host only: *ct_bytes = nct * 2 * L * N * 8 (the
 * ciphertexts), *ext_bytes = nct * 2 * K * N * 4 (their lift to the tensor
 * base), *meta_bytes = the plaintext structure: 0 (DENSE), rows*cols (MASK,
 * one byte per element), (rows + 1 + nct) * 4 (CSR), rows * ell_width * 4
 * (ELL).  Reads only the descriptor's sizes and encoding.  Errors: EINVAL
 * (null, bad encoding), EUNSUPPORTED (N, L), ESHAPE (negative sizes). */
sfhe_status sfhe_matrix_bytes(uint32_t N, uint32_t L, const sfhe_matrix_view* M, uint64_t* ct_bytes,
                              uint64_t* ext_bytes, uint64_t* meta_bytes);

/* Secret-key BFV encryption (the scheme of Sec. 3.1, one element per
 * ciphertext as in the c = 1 setting of Sec. 3.2): ct[n] (device, [n][2][L][N], NTT form) encrypts
 * values[n] (host) in the constant coefficient; the randomness of
 * ciphertext n is drawn from the stream (matrix_id, coords[2n], coords[2n+1]). */
sfhe_status sfhe_encrypt(sfhe_ctx* ctx, const int64_t* values, const int32_t* coords, int64_t n, uint64_t matrix_id,
                         uint64_t* ct, void* stream);
/* Exact centred lift to the tensor base (the first step of the BFV multiply
 * of Alg. 1, done once per ciphertext): ext[n] (device, uint32) from ct[n]
 * (device): every coefficient's representative in (-Q/2, Q/2) reduced mod
 * each b_k, NTT form.  Needs sfhe_lift_workspace_size() bytes of device
 * workspace (a smaller workspace processes the ciphertexts in chunks). */
sfhe_status sfhe_lift_workspace_size(const sfhe_ctx* ctx, int64_t n, size_t* bytes);
sfhe_status sfhe_lift(sfhe_ctx* ctx, const uint64_t* ct, int64_t n, uint32_t* ext, void* work, size_t work_bytes,
                      void* stream);
/* Decryption of the constant coefficient of ct[n] (device) into out[n]
 * (device int64), centred in (-t/2, t/2]. */
sfhe_status sfhe_decrypt(sfhe_ctx* ctx, const uint64_t* ct, int64_t n, int64_t* out, void* stream);
/* NTT form <-> coefficient form of npoly ciphertext polynomials laid out
 * as [npoly][L][N] (a ciphertext is two of them: npoly = 2 n). */
sfhe_status sfhe_to_coeff(sfhe_ctx* ctx, const uint64_t* in, int64_t npoly, uint64_t* out, void* stream);
sfhe_status sfhe_from_coeff(sfhe_ctx* ctx, const uint64_t* in, int64_t npoly, uint64_t* out, void* stream);
/* Keys in coefficient form: secret (host int8[N]); relinearisation key
 * (device [L digit][2 (b, a)][L limb][N]). */
sfhe_status sfhe_export_secret(sfhe_ctx* ctx, int8_t* s_host);
sfhe_status sfhe_export_relin_key(sfhe_ctx* ctx, uint64_t* out, void* stream);

/* ------------------------------------------------ slot-packed chunks --- */
/* Alg. 1 with chunk size c > 1 (Sec. 3.2): a chunk ciphertext holds c
 * consecutive row-major matrix elements in its slots 0 .. c-1 (BFV batching,
 * t prime and 1 mod 2N).  Slot s = (r, j) = (s / (N/2), s mod (N/2)) of a
 * plaintext polynomial m is m(zeta^e) with e = 3^j (r = 0) or -3^j (r = 1)
 * mod 2N, zeta the smallest primitive 2N-th root of unity mod t, so the
 * automorphism X -> X^(3^k) rotates each row of N/2 slots left by k.
 *
 * Host only: slots <-> plaintext polynomial (values and coefficients mod t;
 * outputs in [0, t)).  EUNSUPPORTED if t is not a prime 1 mod 2N. */
sfhe_status sfhe_slots_encode(uint32_t N, uint64_t t, const int64_t* values, int64_t* poly);
sfhe_status sfhe_slots_decode(uint32_t N, uint64_t t, const int64_t* poly, int64_t* values);
/* Galois element of a left rotation by k (right for k < 0): 3^(k mod N/2)
 * mod 2N; 0 if N is not a power of two >= 4.  Host only. */
uint32_t sfhe_rotation_element(uint32_t N, int32_t k);
/* Secret-key encryption of whole plaintext polynomials polys[n][N] (host,
 * coefficients mod t): c0 = -a s + e + Delta m, the stream as sfhe_encrypt
 * (a polynomial with only a constant coefficient gives sfhe_encrypt's
 * ciphertext). ct: device [n][2][L][N], NTT form. */
sfhe_status sfhe_encrypt_poly(sfhe_ctx* ctx, const int64_t* polys, const int32_t* coords, int64_t n,
                              uint64_t matrix_id, uint64_t* ct, void* stream);
/* Every coefficient of the messages: out (device [n][N]) in [0, t). */
sfhe_status sfhe_decrypt_poly(sfhe_ctx* ctx, const uint64_t* ct, int64_t n, int64_t* out, void* stream);
/* Galois key for g (odd, < 2N): key and key_sh (device, [L digit][2 (b,
 * a)][L limb][N] each, NTT form and Shoup companions): b_j = -a_j s + e_j +
 * g_j s(X^g), the gadget of the relinearisation key; randomness from its
 * own stream (domains 6 and 7, objects (g, j)). */
sfhe_status sfhe_galois_keygen(sfhe_ctx* ctx, uint32_t g, uint64_t* key, uint64_t* key_sh, void* stream);
/* Rotation (fhe_rotate of Alg. 1): out[n] = the key switch back to s of
 * (c0(X^g), c1(X^g)): (c0' + sum_j D_j b_j, sum_j D_j a_j), unsigned digits
 * D_j = [c1']_{q_j}.  in and out device, distinct; needs
 * sfhe_rotate_workspace_size() bytes of device workspace per ciphertext
 * switched at once (a larger workspace batches more). */
sfhe_status sfhe_rotate_workspace_size(const sfhe_ctx* ctx, size_t* bytes);
sfhe_status sfhe_rotate(sfhe_ctx* ctx, const uint64_t* in, int64_t n, uint32_t g, const uint64_t* key,
                        const uint64_t* key_sh, uint64_t* out, void* work, size_t work_bytes, void* stream);
/* A plaintext polynomial (host [N] mod t, lifted to its centred
 * representatives) in NTT form over Q: pt device [L][N].  Synchronous. */
sfhe_status sfhe_plain_ntt(sfhe_ctx* ctx, const int64_t* poly, uint64_t* pt, void* stream);
/* ct[n] *= pt (Alg. 1's multiply by the slot-zero mask): decrypts to the
 * slot-wise product.  In place, device. */
sfhe_status sfhe_mul_plain(sfhe_ctx* ctx, uint64_t* ct, int64_t n, const uint64_t* pt, void* stream);
/* acc[n] += x[n] (mod q_i), device. */
sfhe_status sfhe_add(sfhe_ctx* ctx, uint64_t* acc, const uint64_t* x, int64_t n, void* stream);
/* Rotation keys for chunk size c: left and right rotations by 1 .. c-1
 * (2 (c - 1) Galois keys, device memory owned by the object). */
typedef struct sfhe_rotkeys sfhe_rotkeys;
sfhe_status sfhe_rotkeys_create(sfhe_ctx* ctx, int32_t c, void* stream, sfhe_rotkeys** out);
void sfhe_rotkeys_destroy(sfhe_rotkeys* rk);
/* The encrypted matrix product over chunks (Sec. 3.2; the operations of
 * Alg. 1 with c > 1).  A holds ceil(M K / c) chunk ciphertexts of the M x K
 * matrix (row-major, element e in slot e mod c of chunk e / c), B ceil(K Nc /
 * c) of the K x Nc one, C receives ceil(M Nc / c).  Entry (i, j) of C is the
 * sum, over its products k, of the term Relin(a x b), where a is A's chunk
 * holding element (i, k) turned so that the element sits in slot 0 and b
 * likewise for B's element (k, j) (the BFV multiply's exact scale-and-round
 * stands in for CKKS's rescale; a turn by 0 is no operation), placed at slot
 * (i Nc + j) mod c of chunk (i Nc + j) / c by the slot-0 mask and a turn
 * right.  This call places every term on its own, as Alg. 1 does, one short
 * launch sequence per product.  a_zero / b_zero (host, may be NULL): the
 * naive sparse masks; a product is skipped where either is set.  The
 * product sets come from the work-list builder of the per-element matmul.
 * *products (may be NULL) receives the count.  The workspace (device) holds
 * the per-product temporaries. */
sfhe_status sfhe_matmul_chunked_workspace_size(const sfhe_ctx* ctx, size_t* bytes);
sfhe_status sfhe_matmul_chunked(sfhe_ctx* ctx, const sfhe_rotkeys* rk, int32_t M, int32_t K, int32_t Nc,
                                const uint64_t* A, const uint64_t* B, uint64_t* C, const uint8_t* a_zero,
                                const uint8_t* b_zero, void* work, size_t work_bytes, void* stream, int64_t* products);
/* The same terms with the placement applied to each entry's sum instead
 * of to each term (another ciphertext with the same decryption): every
 * operand element is turned to slot 0 once (M K + K Nc key switches,
 * batched by turn amount), the entries' sums of relinearised products run
 * on the persistent kernel, and each sum is masked and turned to its offset
 * (M Nc key switches) before it is added into its chunk.  Workspace
 * (device) from the size call, which needs the same chunk size and masks. */
sfhe_status sfhe_matmul_chunked_fused_workspace_size(const sfhe_ctx* ctx, int32_t c, int32_t M, int32_t K, int32_t Nc,
                                                     const uint8_t* a_zero, const uint8_t* b_zero, size_t* bytes);
sfhe_status sfhe_matmul_chunked_fused(sfhe_ctx* ctx, const sfhe_rotkeys* rk, int32_t M, int32_t K, int32_t Nc,
                                      const uint64_t* A, const uint64_t* B, uint64_t* C, const uint8_t* a_zero,
                                      const uint8_t* b_zero, void* work, size_t work_bytes, void* stream,
                                      int64_t* products);

/* ------------------------------------------------------------- CKKS --- */
/* The scheme and parameter set the paper runs (Sec. 3.1): ring degree
 * p = 8192, a coefficient modulus of 50, 40, 40 and 40 bits plus a 40-bit
 * prime for key switching, initial scale 2^40; the chunked product of Alg. 1
 * over it with its rescales.  (N = 64 is accepted for small tests.)
 * Primes: per bit size, the largest primes below 2^bits that are 1 mod 2N,
 * in the order of the list, the key-switching prime P last.  Slots: slot
 * j < N/2 of a real-coefficient polynomial m is m(zeta^(3^j)), zeta =
 * exp(i pi / N); X -> X^(3^k) turns the slots left by k (sfhe_rotation_element).
 * Ciphertexts: [2][L][N] uint64, NTT form; at level l only limbs 0 .. l
 * (primes q_0 .. q_l) are used.  Key switching (relinearisation, rotations)
 * takes one digit per prime: digits D_j = [d]_{q_j}, the sum of D_j times
 * key digit j over q_0 .. q_l and P, then the rounded division by P.  A key
 * digit for w = s^2 or s(X^g) is (-a_j s + e_j + P g_j w, a_j), g_j = 1 mod
 * q_j and 0 mod the other q_i.  Rescaling from level l: round(c / q_l) in
 * every limb below l; the scale is divided by q_l.  Randomness: the secret
 * from the same stream as the BFV context's (ternary, domain 1); encryption
 * domains 11 / 12 with the stream object (matrix id, row, col); key
 * domains 9 / 10 with objects (g, j, 0), g = 0 for relinearisation. */
typedef struct {
    uint32_t N;             /* 8192 (64 for tests) */
    uint32_t L;             /* data primes, 3 .. 8 for the chunked product */
    uint32_t bits[8];       /* their sizes, e.g. 50, 40, 40, 40 */
    uint32_t special_bits;  /* the key-switching prime, e.g. 40 */
    uint32_t log_scale;     /* initial scale 2^log_scale, e.g. 40 */
    double sigma;           /* error width (3.2) */
} sfhe_ckks_params;
typedef struct sfhe_ckks_ctx sfhe_ckks_ctx;
typedef struct sfhe_ckks_rotkeys sfhe_ckks_rotkeys;
/* Primes, tables, the secret and the relinearisation key on the current
 * device.  Synchronous.  Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA, EDEVICE. */
sfhe_status sfhe_ckks_ctx_create(const sfhe_ckks_params* params, uint64_t seed, sfhe_ckks_ctx** out);
void sfhe_ckks_ctx_destroy(sfhe_ckks_ctx* ctx);
/* q[L] the data primes, *p the key-switching prime, *scale the initial scale (any may be NULL) */
sfhe_status sfhe_ckks_ctx_primes(const sfhe_ckks_ctx* ctx, uint64_t* q, uint64_t* p, double* scale);
/* Host only.  Encoding of n <= N/2 real values (the other slots 0) at
 * `scale`: poly[k] = round((2 scale / N) sum_j values[j] cos(pi 3^j k / N))
 * in double precision.  Decoding of a plaintext given as coefficient-form
 * residues coeff[level + 1][N] (limbs of the primes q_0 .. q_level; the
 * centred integer is rebuilt by CRT): values[j] = (1 / scale)
 * sum_k m_k cos(pi 3^j k / N), j < n. */
sfhe_status sfhe_ckks_encode(const sfhe_ckks_ctx* ctx, const double* values, int32_t n, double scale, int64_t* poly);
sfhe_status sfhe_ckks_decode(const sfhe_ckks_ctx* ctx, const uint64_t* coeff, int32_t level, double scale, int32_t n,
                             double* values);
/* Secret-key encryption of n integer plaintext polynomials polys[n][N]
 * (host) at the top level: c = (-a s + e + m, a); ct device [n][2][L][N]. */
sfhe_status sfhe_ckks_encrypt(sfhe_ckks_ctx* ctx, const int64_t* polys, const int32_t* coords, int64_t n,
                              uint64_t matrix_id, uint64_t* ct, void* stream);
/* Decryption and decoding of n ciphertexts at `level`: values[n][slots]
 * (host).  Synchronises `stream`. */
sfhe_status sfhe_ckks_decrypt(sfhe_ckks_ctx* ctx, const uint64_t* ct, int32_t level, int64_t n, double scale,
                              int32_t slots, double* values, void* stream);
/* limbs 0 .. level of n ciphertexts to coefficient form (device [n][2][L][N], other limbs 0) */
sfhe_status sfhe_ckks_to_coeff(sfhe_ckks_ctx* ctx, const uint64_t* ct, int32_t level, int64_t n, uint64_t* out,
                               void* stream);
/* Device workspace of one key switch (sfhe_ckks_rotate); sfhe_ckks_mul_relin
 * needs L N words more, sfhe_ckks_rescale (2 n + 2 n level) N words. */
sfhe_status sfhe_ckks_workspace_size(const sfhe_ckks_ctx* ctx, size_t* bytes);
/* out = a x b relinearised, at `level` (out distinct from a and b) */
sfhe_status sfhe_ckks_mul_relin(sfhe_ckks_ctx* ctx, const uint64_t* a, const uint64_t* b, int32_t level, uint64_t* out,
                                void* work, size_t work_bytes, void* stream);
/* n ciphertexts from `level` to level - 1 (in may equal out) */
sfhe_status sfhe_ckks_rescale(sfhe_ckks_ctx* ctx, const uint64_t* in, int32_t level, int64_t n, uint64_t* out,
                              void* work, size_t work_bytes, void* stream);
/* Galois keys of the left and right turns by 1 .. c-1 (domains 9 / 10, object (g, j, 0)) */
sfhe_status sfhe_ckks_rotkeys_create(sfhe_ckks_ctx* ctx, int32_t c, void* stream, sfhe_ckks_rotkeys** out);
void sfhe_ckks_rotkeys_destroy(sfhe_ckks_rotkeys* rk);
/* out = the slots of in turned left by k (right for k < 0), 0 < |k| < c; in, out distinct */
sfhe_status sfhe_ckks_rotate(sfhe_ckks_ctx* ctx, const sfhe_ckks_rotkeys* rk, const uint64_t* in, int32_t level,
                             int32_t k, uint64_t* out, void* work, size_t work_bytes, void* stream);
/* A plaintext polynomial (host, signed coefficients) in NTT form over limbs
 * 0 .. level: pt device [L][N].  Synchronous.  sfhe_ckks_mul_plain: ct[n]
 * *= pt; sfhe_ckks_add: acc[n] += x[n]; both over limbs 0 .. level. */
sfhe_status sfhe_ckks_plain_ntt(sfhe_ckks_ctx* ctx, const int64_t* poly, int32_t level, uint64_t* pt, void* stream);
sfhe_status sfhe_ckks_mul_plain(sfhe_ckks_ctx* ctx, uint64_t* ct, int32_t level, int64_t n, const uint64_t* pt,
                                void* stream);
sfhe_status sfhe_ckks_add(sfhe_ckks_ctx* ctx, uint64_t* acc, const uint64_t* x, int32_t level, int64_t n, void* stream);
/* The chunked product of Alg. 1 with chunk size rk->c: A holds ceil(M K / c)
 * chunks at the top level (element e in slot e mod c of chunk e / c, scale
 * D), B ceil(K Nc / c); C receives ceil(M Nc / c) chunks two levels lower at
 * the scale *result_scale = D^2 / q_top.  Entry (i, j) is the sum over its
 * products k of: the chunks holding A[i][k] and B[k][j] turned to slot 0,
 * multiplied, relinearised, rescaled; times the slot-0 mask encoded at the
 * scale q_{top-1}; rescaled; turned right to (i Nc + j) mod c.  (Alg. 1's
 * relinearisation after the mask product has nothing to do with a
 * plaintext.)  a_zero / b_zero (host, may be NULL): the naive sparse masks.
 * Workspace from the size call. */
sfhe_status sfhe_ckks_matmul_chunked_workspace_size(const sfhe_ckks_ctx* ctx, size_t* bytes);
sfhe_status sfhe_ckks_matmul_chunked(sfhe_ckks_ctx* ctx, const sfhe_ckks_rotkeys* rk, int32_t M, int32_t K, int32_t Nc,
                                     const uint64_t* A, const uint64_t* B, uint64_t* C, const uint8_t* a_zero,
                                     const uint8_t* b_zero, void* work, size_t work_bytes, void* stream,
                                     int64_t* products, double* result_scale);

/* Measured rate of the 32-bit Shoup modular multiply a w mod b (three
 * 32-bit multiplies: the high product with the precomputed companion and two
 * low products; the butterfly multiply of the tensor stage's inverse NTTs)
 * on the current device, all SMs at full occupancy, eight independent chains
 * per thread: *per_s = multiplies per second.  A measured reference for the
 * integer roofline beside the peak derived from unit counts and clocks.
 * Uses the context's first tensor-base prime; synchronises `stream`.
 * Errors: EINVAL (null), ECUDA. */
sfhe_status sfhe_measure_mulmod32(sfhe_ctx* ctx, double* per_s, void* stream);

/* --------------------------------------- library-owned matrices (handles) --- */
/* The paper states the problem as: encrypted inputs A and B with the matrix
 * information of the left and right operands in, the encrypted product R out
 * (Alg. 1's input and output lines; the three sparse encodings of
 * Sec. 3.3.2).  These calls take and return that: sfhe_matrix handles own
 * their ciphertexts (NTT form, [nct][2][L][N]) and their lift to the tensor
 * base in device memory allocated here (cudaMalloc) and released by
 * sfhe_matrix_destroy; the plaintext structure (mask, CSR or ELLPACK arrays)
 * is copied into the handle.  Every call validates its arguments before it
 * launches; errors leave *out NULL.  A handle belongs to the context that
 * made it and must be destroyed before the context. */

/* Primes of the context: q[L] the ciphertext primes (descending), p[K] the
 * primes of the extended base the multiply runs in (the tensor base B of
 * 30-bit primes, K = sfhe_info.K <= 32; the paper's scheme leaves the
 * auxiliary base to the library).  Host memory.  Errors: EINVAL (null). */
sfhe_status sfhe_ctx_get_primes(const sfhe_ctx* ctx, uint64_t* q, uint64_t* p);

/* Encodes the plaintext matrix vals[rows*cols] (host, row-major) under
 * `encoding` (Sec. 3.3.2), encrypts every stored element in its own
 * ciphertext (secret-key BFV, the value in the constant coefficient;
 * randomness from the stream (matrix_id, row, col) as sfhe_encrypt) and lifts
 * the ciphertexts to the tensor base, on `stream`.  ELLPACK padding slots
 * hold encryptions of zero.  Errors: EINVAL (null, bad encoding), ESHAPE
 * (negative shape), ENOMEM (device), ECUDA. */
sfhe_status sfhe_matrix_encrypt(sfhe_ctx* ctx, const int64_t* vals, int32_t rows, int32_t cols, sfhe_encoding encoding,
                                uint64_t matrix_id, void* stream, sfhe_matrix** out);
/* A matrix from ciphertexts already encrypted elsewhere: coeff_limbs (host,
 * [nct][2][L][N], coefficient form, canonical residues: limb i below q_i)
 * and the structure `idx` (host int32):
 *   DENSE: unused (may be NULL), nct = rows*cols;
 *   MASK:  idx[rows*cols], nonzero where the element is zero, nct = rows*cols;
 *   CSR:   row_ptr[rows+1] followed by col_idx[nct], nct = row_ptr[rows];
 *   ELL:   idx[0] = ell_width, then ell_col[rows*ell_width] (-1 = padding),
 *          nct = rows*ell_width.
 * The ciphertexts are copied to the device, taken to NTT form and lifted on
 * `stream`; the host arrays may be reused once the call returns.  Errors:
 * EINVAL (null, bad structure, a residue >= its prime), ESHAPE, ENOMEM,
 * ECUDA. */
sfhe_status sfhe_matrix_import(sfhe_ctx* ctx, const uint64_t* coeff_limbs, const int32_t* idx, int32_t rows,
                               int32_t cols, sfhe_encoding encoding, void* stream, sfhe_matrix** out);
/* The ciphertexts in coefficient form, canonical residues, into host
 * coeff_limbs[nct][2][L][N] (nct from sfhe_matrix_info).  Synchronises
 * `stream`.  Errors: EINVAL (null), ECUDA. */
sfhe_status sfhe_matrix_export(const sfhe_matrix* M, uint64_t* coeff_limbs, void* stream);
/* Decryption into host out[rows*cols] (row-major), centred in (-t/2, t/2]:
 * every stored element decrypted, elements the encoding does not store
 * (CSR / ELLPACK zeros) are 0.  Synchronises `stream`.  Errors: EINVAL (null,
 * a handle of another context), ECUDA. */
sfhe_status sfhe_matrix_decrypt(sfhe_ctx* ctx, const sfhe_matrix* M, int64_t* out, void* stream);
/* Releases the handle's device memory (synchronises the device).  NULL is a no-op. */
void sfhe_matrix_destroy(sfhe_matrix* M);
/* Shape, encoding and stored ciphertext count of a handle (any may be NULL). */
sfhe_status sfhe_matrix_info(const sfhe_matrix* M, int32_t* rows, int32_t* cols, int32_t* encoding, int32_t* nct);
/* A descriptor of the handle's storage for the calls that take views
 * (plans, graphs).  The view points into the handle (ct, ext and the
 * structure arrays) and is valid until sfhe_matrix_destroy; a result
 * handle not yet used as an operand is lifted here first (on `stream`). */
sfhe_status sfhe_matrix_view_of(sfhe_matrix* M, sfhe_matrix_view* out, void* stream);

/* *C = A x B over every k (the naive dense loop of Alg. 1; A must store
 * every element: DENSE or MASK), all products in one persistent launch.  C
 * is a new DENSE handle of A.rows x B.cols ciphertexts, written on `stream`;
 * the transient workspace is allocated and freed on the stream
 * (cudaMallocAsync).  An operand that is itself a result is lifted first.
 * Errors: EINVAL (null, handles of another context, encodings), ESHAPE
 * (A.cols != B.rows), EUNSUPPORTED (more than 1024 products in one entry),
 * ENOMEM, ECUDA. */
sfhe_status sfhe_matmul_dense(sfhe_ctx* ctx, const sfhe_matrix* A, const sfhe_matrix* B, sfhe_matrix** C, void* stream);
/* *C = A x B with the k-loop over the nonzeros of A as `encoding` lists
 * them (Sec. 3.3.2; A must carry that encoding: EINVAL otherwise); a
 * MASK-encoded B also skips the k where B[k][j] is zero.  Otherwise as
 * sfhe_matmul_dense. */
sfhe_status sfhe_matmul_sparse(sfhe_ctx* ctx, const sfhe_matrix* A, const sfhe_matrix* B, sfhe_encoding encoding,
                               sfhe_matrix** C, void* stream);
/* n independent products C[m] = A[m] x B[m] (each A over the k its own
 * encoding lists) in one execution under `flags` (SFHE_EXEC_PLAIN, or
 * SFHE_EXEC_PERSISTENT optionally with SFHE_EXEC_LAZY; SFHE_EXEC_GRAPH is
 * for plans).  C[0..n-1] receive new handles (all NULL on error).  No
 * counterpart in the paper, whose Sec. 3.4 spreads one matmul's output
 * entries over CPU threads. */
sfhe_status sfhe_matmul_batch(sfhe_ctx* ctx, int32_t n, const sfhe_matrix* const* A, const sfhe_matrix* const* B,
                              sfhe_matrix** C, uint32_t flags, void* stream);

/* -------------------------------------------- host-resident operands --- */
/* A matmul whose ciphertexts live in host memory: every call copies A's and
 * B's ciphertexts to the device, lifts them, runs the matmul and copies C
 * back (Alg. 1's input and output at the host).  The plan is built once from
 * descriptors of the n matmuls' structure (their ct / ext fields are
 * ignored) and owns `depth` (1 or 2) sets of device buffers.  With depth 2
 * consecutive calls overlap: call i+1's upload and call i-1's download run
 * on the plan's own copy streams while call i computes.  flags as
 * sfhe_matmul_batch.  Errors: EINVAL, ESHAPE, EUNSUPPORTED, ENOMEM, ECUDA. */
sfhe_status sfhe_host_plan_create(sfhe_ctx* ctx, int32_t n, const sfhe_matrix_view* A, const sfhe_matrix_view* B,
                                  uint32_t flags, int32_t depth, sfhe_host_plan** out);
/* One matmul: A_ct[m] (host, [nct_A][2][L][N] NTT form), B_ct[m] likewise,
 * into C_ct[m] (host, [rows_A * cols_B][2][L][N] NTT form).  Asynchronous:
 * the inputs are read from host memory at some time after the call (write
 * them before calling; the uploads do not wait for work on `stream`), and
 * work enqueued on `stream` after the call waits for C_ct to be written; the
 * host buffers must stay valid and unchanged until then.  Page-locked
 * (pinned) host buffers let the copies overlap with computation.  Errors:
 * EINVAL (null), ECUDA. */
sfhe_status sfhe_matmul_host(sfhe_host_plan* hp, const uint64_t* const* A_ct, const uint64_t* const* B_ct,
                             uint64_t* const* C_ct, void* stream);
/* products per call, bytes copied host->device and device->host per call,
 * and the library's kernel launches per call. */
sfhe_status sfhe_host_plan_stats(const sfhe_host_plan* hp, int64_t* products, uint64_t* h2d_bytes,
                                 uint64_t* d2h_bytes, int64_t* launches);
/* Waits for the plan's work and releases it.  NULL is a no-op. */
void sfhe_host_plan_destroy(sfhe_host_plan* hp);

/* ------------------------------------------- matmul over views --- */
/* The same products over caller-owned device memory (sfhe_matrix_view):
 * the caller allocates C's ciphertexts and the workspace, and picks the
 * execution mode.  Workspace (device bytes) for n matmuls A[m] x B[m] under
 * `flags`: */
sfhe_status sfhe_matmul_workspace_size(const sfhe_ctx* ctx, int32_t n, const sfhe_matrix_view* A,
                                       const sfhe_matrix_view* B, uint32_t flags, size_t* bytes);
/* An upper bound of sfhe_matmul_workspace_size for any n <= max_matmuls
 * matmuls with at most max_entries output entries and max_products
 * products in all (a workspace a serving loop allocates once and reuses for
 * every batch).  Host only.  Errors: EINVAL, ESHAPE (negative bounds). */
sfhe_status sfhe_matmul_workspace_bound(const sfhe_ctx* ctx, int32_t max_matmuls, int64_t max_entries,
                                        int64_t max_products, uint32_t flags, size_t* bytes);
/* C = A x B with the k-loop over every k: the naive dense loop of Alg. 1
 * (Sec. 3.3.1), each product multiplied, relinearised and added (A must
 * store every element: DENSE or MASK; masks are ignored). */
sfhe_status sfhe_matmul_dense_view(sfhe_ctx* ctx, const sfhe_matrix_view* A, const sfhe_matrix_view* B,
                                   sfhe_matrix_view* C, uint32_t flags, void* work, size_t work_bytes, void* stream);
/* C = A x B with the k-loop over the nonzeros of A as `encoding` lists them
 * (Sec. 3.3.2; A must carry that encoding; EINVAL otherwise); a MASK-encoded
 * B also skips the k where B[k][j] is zero. */
sfhe_status sfhe_matmul_sparse_view(sfhe_ctx* ctx, const sfhe_matrix_view* A, const sfhe_matrix_view* B,
                                    int32_t encoding, sfhe_matrix_view* C, uint32_t flags, void* work,
                                    size_t work_bytes, void* stream);
/* n independent matmuls C[m] = A[m] x B[m] (each A in its own encoding) in
 * one execution.  No counterpart in the paper, whose Sec. 3.4 spreads one
 * matmul's output entries over CPU threads; here the entries of all n
 * matmuls share one persistent launch. */
sfhe_status sfhe_matmul_batch_view(sfhe_ctx* ctx, int32_t n, const sfhe_matrix_view* A, const sfhe_matrix_view* B,
                                   sfhe_matrix_view* C, uint32_t flags, void* work, size_t work_bytes, void* stream);

/* Plans: the work list is built and uploaded once (into `work`), then
 * sfhe_plan_execute only launches (with SFHE_EXEC_GRAPH, one graph launch),
 * so it can be replayed and captured.  The plan keeps the pointers of A, B,
 * C and `work`; they must stay valid until sfhe_plan_destroy. */
sfhe_status sfhe_plan_create(sfhe_ctx* ctx, int32_t n, const sfhe_matrix_view* A, const sfhe_matrix_view* B,
                             sfhe_matrix_view* C, uint32_t flags, void* work, size_t work_bytes, void* stream,
                             sfhe_plan** out);
sfhe_status sfhe_plan_execute(sfhe_plan* plan, void* stream);
/* Synchronises `stream` and reads the status word of a matmul workspace
 * after a PERSISTENT execution: SFHE_ETIMEOUT if one of the kernel's bounded
 * waits for an operand copy ran out (the kernel then stopped early and C is
 * incomplete). */
sfhe_status sfhe_matmul_check(void* work, void* stream);
/* Preemption of a persistent plan: the serving loop's continuous admission
 * (a request that arrives while a plan runs need not wait for the whole
 * launch; the paper's Sec. 3.4 runs one matmul at a time and has no
 * counterpart).
 * sfhe_plan_set_stop: `word` is the device address of one uint32 (NULL
 * clears it), which the caller owns and writes, e.g. with a copy on another
 * stream while the launch runs.  Every CTA of the plan's persistent launches
 * reads it before it takes its next output entry and takes none once it is
 * nonzero; no CTA waits on it, so a launch ends within one entry's time of
 * the word being set, the entries it took complete, C of the others is
 * untouched.  Errors: EINVAL (null plan, a PLAIN or GRAPH plan, misaligned).
 * sfhe_plan_progress: synchronises `stream` and reports how many output
 * entries, in the plan's execution order, the launches so far completed
 * (all of them after an execution that was not stopped).
 * sfhe_plan_resume: launches the plan again from its first entry not taken
 * (clear the word first); a stopped execution plus its resumptions write
 * the same C, limb for limb, as one execution.  sfhe_plan_execute restarts
 * from the first entry.  Errors: EINVAL (null plan, a PLAIN plan, resume
 * before the first execution), ECUDA. */
sfhe_status sfhe_plan_set_stop(sfhe_plan* plan, const uint32_t* word);
sfhe_status sfhe_plan_progress(const sfhe_plan* plan, int64_t* done, void* stream);
sfhe_status sfhe_plan_resume(sfhe_plan* plan, void* stream);
/* Self-test of the bounded device waits (no fault is involved): one thread
 * waits on an mbarrier that nothing arrives at, gives up after `tries`
 * attempts (1 .. 2^30) or `limit_us` microseconds of the GPU's clock
 * (1 .. 10^6), whichever comes first, and sets the status word of `work`
 * (device, at least 256 bytes, its first 8 bytes zeroed by the caller) as
 * the persistent kernel does; sfhe_matmul_check(work) then reports
 * SFHE_ETIMEOUT.  The persistent kernel's own bound is one second or 2^26
 * attempts.  Errors: EINVAL (null, bounds out of range), ECUDA. */
sfhe_status sfhe_selftest_wait_bound(void* work, uint32_t tries, uint32_t limit_us, void* stream);
/* Tile tuning of the per-product persistent kernel.  Where a ring has
 * several tiles (stage-S tiles of the exact scale-and-round: how many
 * coefficients a thread rounds at a time and how many output primes it
 * reconstructs per pass; and code forms of the tensor's inverse NTT: lean
 * exchange addresses and reductions, a warp-shuffle stage; N = 4096 with
 * L = 2 and N = 16384 with L = 8 have three tiles, N = 8192 with L = 4
 * five), the first per-product persistent plan of a context times every
 * tile on the plan's first entries (one per
 * CTA, at most four products each; this writes their C, which every
 * execution writes again, and synchronises the stream) and the context
 * keeps the fastest for all its later plans.  sfhe_ctx_tuning: the tile in
 * use (-1 before the first plan), how many there are, and the calibration
 * time of each (ms[n_variants], at most 8, may be NULL; zeros while untuned).
 * sfhe_ctx_set_variant: use tile `variant` from now on (-1: tune as above).
 * sfhe_ctx_variant_name: a description of a tile ("" if out of range). */
sfhe_status sfhe_ctx_tuning(const sfhe_ctx* ctx, int32_t* variant, int32_t* n_variants, float* ms);
sfhe_status sfhe_ctx_set_variant(sfhe_ctx* ctx, int32_t variant);
const char* sfhe_ctx_variant_name(const sfhe_ctx* ctx, int32_t variant);
/* products performed, output entries, own kernel launches per execute, CTAs */
sfhe_status sfhe_plan_stats(const sfhe_plan* plan, int64_t* products, int64_t* entries, int64_t* launches,
                            int64_t* ctas);
void sfhe_plan_destroy(sfhe_plan* plan);

/* ------------------------------------------------- stage entry points --- */
/* One product's tensor and exact scale-and-round (the multiply of Alg. 1):
 * d[3][L][N] (uint64, coefficient form) from lifted a, b (device).
 * Workspace: 3 K N uint32 words. */
sfhe_status sfhe_ct_tensor_scale(sfhe_ctx* ctx, const uint32_t* a_ext, const uint32_t* b_ext, uint64_t* d, void* work,
                                 size_t work_bytes, void* stream);
/* One product multiplied and relinearised (Alg. 1's multiply and relinearisation),
 * NTT form [2][L][N] (plain path).  Workspace: 3 K N uint32 words (rounded up
 * to 256 bytes) + (3 L + (L+2) L) N uint64 words. */
sfhe_status sfhe_ct_mul_relin(sfhe_ctx* ctx, const uint32_t* a_ext, const uint32_t* b_ext, uint64_t* out, void* work,
                              size_t work_bytes, void* stream);

/* Bytes of the library's static device scratch (one copy per device). */
#define SFHE_STATIC_SCRATCH_BYTES (8u << 20)
/* sfhe_ct_mul_relin without a workspace argument: the same computation and
 * the same result, with its scratch in a fixed device array of
 * SFHE_STATIC_SCRATCH_BYTES inside the library, so the call allocates no
 * memory.  The paper has no counterpart: it is for callers that cannot
 * hand over device memory (a plain C caller without a device allocator,
 * code running during stream capture, a serving loop that must not enter an
 * allocator).  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) and should precede any stream capture; later
 * calls only launch.  Destroying a context of the device forgets the
 * address, so the first call after it looks the address up again (after a
 * device reset the array lives at a new address).  The context's device must be the current device.
 * Rings whose scratch, 3 K N uint32 words (rounded up to 256 bytes) +
 * (3 L + (L+2) L) N uint64 words, exceeds the array are rejected with
 * SFHE_ENOMEM (N = 8192, L = 4 needs 3.8 MB and fits; N = 16384, L = 8
 * needs 19.5 MB and does not).  Nothing in the scratch has to start at
 * zero; `out` is cleared by the call.  All calls on one device share the
 * array: calls that overlap in time (other streams, other threads) race
 * and must be serialised by the caller. */
sfhe_status sfhe_ct_mul_relin_static(sfhe_ctx* ctx, const uint32_t* a_ext, const uint32_t* b_ext, uint64_t* out,
                                     void* stream);
/* Forward / inverse NTT of npoly polynomials (device, [npoly][N]) modulo
 * prime `prime_index`: 0..L-1 the q_i (uint64 words), L..L+K-1 the b_k
 * (uint32 words). */
sfhe_status sfhe_ntt(sfhe_ctx* ctx, int32_t prime_index, int32_t inverse, const void* in, int64_t npoly, void* out,
                     void* stream);
/* Words idx0 .. idx0+n-1 of the generator stream (seed, domain, o0, o1, o2)
 * into out (device). */
sfhe_status sfhe_prng_words(uint64_t seed, uint32_t domain, uint64_t o0, uint64_t o1, uint64_t o2, uint64_t idx0,
                            int64_t n, uint64_t* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SFHE_H */
