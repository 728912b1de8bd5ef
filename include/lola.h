/*
 * lola.h -- C-ABI of the GB300 LoLa library: RNS-BFV ciphertext arithmetic on
 * one GPU and the LoLa message representations / matrix-vector algorithms on
 * top of it.
 *
 * Problem statement (paper Sec. 1 and Sec. 3.1): a client encrypts its data
 * with a homomorphic encryption scheme (BFV), a server evaluates a network on
 * the ciphertexts without the secret key, and the client decrypts the
 * result.  The network is a layer list; each layer consumes one message
 * representation and produces another (Sec. 4.2, Tables 1 and 3).
 *
 * Conventions for every call:
 *  - Return value: LOLA_OK (0) or a negative LOLA_E_* code.  Nothing aborts
 *    the process.  lola_last_error() returns a thread-local message for the
 *    last failing call on the calling thread.
 *  - Handles (lola_ctx, lola_keys, lola_ct, lola_net) are created and owned by
 *    the library and released with the matching *_destroy call.  Destroying
 *    NULL is a no-op.
 *  - "host" pointers are caller-owned CPU memory, read or written during the
 *    call only.  "device" pointers are caller-owned GPU memory on the
 *    context's device; the library never frees them.
 *  - Residues are uint64 words holding canonical values in [0, q).  A
 *    ciphertext in the device layout is [2][L][n] words, limb-major: limb j
 *    (prime q_j) of each of its two polynomials is n contiguous words.  A
 *    batch of ciphertexts is those blocks back to back.  Between operations
 *    ciphertexts are kept in NTT (evaluation) form; import/export calls
 *    convert from/to coefficient form.  After modulus switching a
 *    ciphertext keeps the first L' primes: [2][L'][n] (lola_mod_switch,
 *    lola_ct_level).
 *  - A "message" is one plaintext slot vector; the library encrypts each
 *    message once per plaintext modulus t_i (CRT pipelines, Sec. 4.4), so a
 *    lola_ct holding m messages holds m * k_t ciphertexts ordered
 *    [message][t_i].
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    that take a stream are asynchronous with respect to the host unless
 *    they read or write host memory.
 */
#ifndef LOLA_H
#define LOLA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LOLA_OK 0
#define LOLA_E_PARAM (-1)   /* invalid argument or parameter set */
#define LOLA_E_NOMEM (-2)   /* device or host allocation failed */
#define LOLA_E_NOKEY (-3)   /* a needed Galois / relinearisation key is missing */
#define LOLA_E_REPR (-4)    /* a layer's input representation does not match */
#define LOLA_E_CUDA (-5)    /* a CUDA runtime call failed */
#define LOLA_E_TIMEOUT (-6) /* a bounded wait expired */
#define LOLA_E_STATE (-7)   /* object used in the wrong state (e.g. secret key missing) */

typedef struct lola_ctx lola_ctx;
typedef struct lola_keys lola_keys;
typedef struct lola_ct lola_ct;
typedef struct lola_net lola_net;

/* ------------------------------------------------------------------ context
 * BFV parameters (Sec. 3.1: ring Z_t[x]/(x^n+1), n a power of two, with an
 * order-2n root of unity mod t for batching).
 *   n      ring degree, power of two, 16 <= n <= 16384
 *   L      number of ciphertext primes (Q = q_0 ... q_{L-1}), 1 <= L <= 12
 *   K      special primes for key switching: 0, 1 or 2 (P = their product,
 *          q_L q_{L+1})
 *   q      L + K distinct primes, each = 1 mod 2n and < 2^61 - 2^30
 *   k_t    number of plaintext moduli (CRT pipelines), 1 <= k_t <= 4
 *   t      k_t distinct primes = 1 mod 2n, < 2^31, coprime to all q
 *   alpha  ciphertext primes per key-switching digit: 0 or 1 (one digit per
 *          prime), or 2 (digits of two consecutive primes, the last one
 *          single when L is odd; needs K > 0, and P above every digit's
 *          modulus for a small switching error, e.g. K = 2 with primes of
 *          one size).  A digit is the residue of the switched polynomial
 *          modulo its primes' product, in [0, that product).
 * The library adds its own auxiliary primes for exact ct x ct scaling.
 * Errors: LOLA_E_PARAM for an invalid set, LOLA_E_CUDA / LOLA_E_NOMEM. */
typedef struct {
  uint32_t n;
  uint32_t L;
  uint32_t K;
  const uint64_t* q; /* host, L + K entries, special prime last */
  uint32_t k_t;
  const uint64_t* t; /* host, k_t entries */
  uint32_t alpha;
} lola_params;

int lola_ctx_create(const lola_params* params, int device, lola_ctx** out);
void lola_ctx_destroy(lola_ctx* ctx);
/* The auxiliary prime basis chosen by the context (count, then primes). */
int lola_ctx_aux_primes(const lola_ctx* ctx, uint64_t* primes_out, uint32_t* count_out);

/* --------------------------------------------------------------------- keys
 * Key generation from a seed (secret key ternary, errors discrete Gaussian
 * sigma = 3.2, uniform masks; Philox4x64-10 streams).  rot_steps lists the
 * column-rotation steps k (0 < k < n/2, right shift within each row of the
 * 2 x n/2 slot matrix, Sec. 3.1) that need Galois keys; flags add the
 * relinearisation key and the row-swap key.  *secret_out receives a handle
 * holding the secret, public and evaluation keys; *eval_out (may be NULL)
 * a handle holding only the evaluation keys (what the server gets).
 * Errors: LOLA_E_PARAM (bad step), LOLA_E_NOMEM, LOLA_E_CUDA. */
#define LOLA_KEY_RELIN 1u
#define LOLA_KEY_ROW_SWAP 2u
int lola_keygen(lola_ctx* ctx, uint64_t seed, const int32_t* rot_steps, size_t n_steps, uint32_t flags,
                lola_keys** secret_out, lola_keys** eval_out);
void lola_keys_destroy(lola_keys* keys);
/* Key material in coefficient form, for parity checks.  what: 0 = secret s
 * (n int64 words written as uint64 two's complement), 1 = public key
 * ([2][L][n]), 2 = relinearisation key, 3 = Galois key for rotation `step`
 * (step = 0 selects the row swap).  Switching keys are [2 (b, a)][L digits]
 * [L+K primes][n].  words_out receives the size; host may be NULL to query.
 * Errors: LOLA_E_NOKEY, LOLA_E_STATE (secret missing), LOLA_E_PARAM. */
int lola_keys_export(lola_ctx* ctx, const lola_keys* keys, int what, int32_t step, uint64_t* host,
                     size_t* words_out);

/* -------------------------------------------------------------- ciphertexts
 * Encrypt n_msg slot vectors (host, n_msg x n int64, any sign; reduced mod
 * each t_i).  Ciphertext c = (Delta m + p0 u + e1, p1 u + e2) mod Q with
 * Delta = floor(Q / t_i); the randomness of ciphertext (message i, modulus
 * j) comes from stream id i * k_t + j under `seed`.
 * Errors: LOLA_E_STATE (no public key), LOLA_E_PARAM, LOLA_E_NOMEM. */
int lola_encrypt(lola_ctx* ctx, const lola_keys* keys, const int64_t* slots, size_t n_msg, uint64_t seed,
                 lola_ct** out);
/* Seeded symmetric encryption (a library facility; the paper's E is
 * public-key BFV): the client holds the secret key (Sec. 1: it encrypts and
 * decrypts), so it can encrypt with it, c1 = a, c0 = Delta m + e - a s, and
 * draw a from a seed; the server regenerates c1 from the seed
 * (lola_ct_upload_seeded), so only c0 crosses the wire and the host-device
 * link.  a on prime q_j: its evaluation at psi_j^(2i+1) (psi_j the smallest
 * primitive 2n-th root of unity mod q_j) is ((w_{2i+1} << 64) | w_{2i}) mod
 * q_j over the Philox4x64-10 word stream (seed, 9, id, j); e: Gaussian
 * stream (seed, 10, id, 0); id = message * k_t + residue.  slots as in
 * lola_encrypt.  keys must hold the secret key (else LOLA_E_STATE). */
int lola_encrypt_symmetric(lola_ctx* ctx, const lola_keys* keys, const int64_t* slots, size_t n_msg, uint64_t seed,
                           lola_ct** out);
/* Upload the c0 halves of seeded symmetric ciphertexts and regenerate their
 * c1 on the device: host_c0 [n_msg][k_t][L][n] (NTT form, the c0 limbs of
 * lola_encrypt_symmetric's output; pinned memory for an asynchronous copy),
 * ct at the full level, seed and ids as at encryption.  Stream-ordered on
 * `stream`.  Errors: LOLA_E_PARAM, LOLA_E_CUDA. */
int lola_ct_upload_seeded(lola_ctx* ctx, lola_ct* ct, const uint64_t* host_c0, uint64_t seed, void* stream);
/* Decrypt and recombine the k_t residues by CRT (Sec. 4.4) into signed
 * values in (-T/2, T/2], T = prod t_i.  out: host, n_msg x n pairs of int64
 * (low word, high word) of a signed 128-bit integer.
 * Errors: LOLA_E_STATE (no secret key). */
int lola_decrypt(lola_ctx* ctx, const lola_keys* keys, const lola_ct* ct, int64_t* out);
/* Decrypt without CRT: out host [n_msg][k_t][n], slot values in [0, t_i). */
int lola_decrypt_residues(lola_ctx* ctx, const lola_keys* keys, const lola_ct* ct, uint64_t* out);
int lola_ct_create(lola_ctx* ctx, size_t n_msg, lola_ct** out); /* all-zero ciphertexts */
size_t lola_ct_messages(const lola_ct* ct);
/* Device bytes the handle holds (its capacity at the context's full level). */
size_t lola_ct_bytes(const lola_ct* ct);
/* Device pointer to the ciphertext words ([n_msg][k_t][2][L][n], NTT form);
 * valid until lola_ct_destroy. */
uint64_t* lola_ct_data(lola_ct* ct);
/* Copy n messages (all k_t residues) from src starting at message src_off
 * to dst starting at dst_off, device to device on `stream` (batch assembly
 * and result scatter for request batching).  A copy that fills all of dst
 * gives dst the level of src; otherwise both must be at the same level.
 * Errors: LOLA_E_PARAM (range, levels). */
int lola_ct_copy_messages(lola_ctx* ctx, lola_ct* dst, size_t dst_off, const lola_ct* src, size_t src_off,
                          size_t n, void* stream);
/* Ciphertext primes of the ciphertexts in `ct`: L, or fewer for the output
 * of a network that switches modulus (0 for a NULL handle).  The words of a
 * ciphertext at level L' are [2][L'][n] over the first L' primes of Q; a
 * handle keeps the capacity of level L. */
uint32_t lola_ct_level(const lola_ct* ct);
/* Coefficient-form exchange, host [n_msg][k_t][2][L'][n] at the handle's
 * level L' (import: level L). */
int lola_ct_export(lola_ctx* ctx, const lola_ct* ct, uint64_t* host);
int lola_ct_import(lola_ctx* ctx, const uint64_t* host, size_t n_msg, lola_ct** out);
/* Asynchronous host<->device copies of the NTT-form words (pinned host memory
 * recommended); bytes = lola_ct_messages * k_t * 2 * lola_ct_level * n * 8. */
int lola_ct_upload(lola_ctx* ctx, lola_ct* ct, const uint64_t* host, void* stream);
int lola_ct_download(lola_ctx* ctx, const lola_ct* ct, uint64_t* host, void* stream);
void lola_ct_destroy(lola_ct* ct);

/* ------------------------------------------------------------ primitives
 * Batched ciphertext primitives on caller-owned device buffers in the
 * device layout (NTT form).  count = number of ciphertexts.  t_index[i]
 * (host; NULL = all 0) selects the plaintext modulus of ciphertext i where
 * the operation depends on it.  Output buffers must not alias inputs.
 * Errors: LOLA_E_PARAM, LOLA_E_NOKEY, LOLA_E_CUDA, LOLA_E_NOMEM (scratch). */

/* In-place forward / inverse negacyclic NTT of n_polys polynomials of
 * n_limbs limbs each (limb j uses prime q_j), device layout. */
int lola_ntt_forward(lola_ctx* ctx, uint64_t* data, size_t n_polys, uint32_t n_limbs, void* stream);
int lola_ntt_inverse(lola_ctx* ctx, uint64_t* data, size_t n_polys, uint32_t n_limbs, void* stream);
/* out = a + b (Sec. 3.1 operator (+)). */
int lola_add(lola_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t count, void* stream);
/* Rotation (Sec. 3.1): out_i = rotate(in_i, steps[i]) with steps host, 0 < step < n/2
 * a right shift of each slot row, step = 0 the row swap. */
int lola_rotate(lola_ctx* ctx, const lola_keys* keys, const uint64_t* in, uint64_t* out, size_t count,
                const int32_t* steps, void* stream);
/* ct (x) ct with BFV scaling and relinearisation (Sec. 3.1 operator (x)):
 * out_i = relin(round(t/Q * a_i (x) b_i)).  b may equal a (square). */
int lola_multiply(lola_ctx* ctx, const lola_keys* keys, const uint64_t* a, const uint64_t* b, uint64_t* out,
                  size_t count, const uint32_t* t_index, void* stream);
/* Rotation that allocates no device memory, for callers that cannot call
 * cudaMalloc / cudaMallocAsync: applications whose memory manager owns the
 * device and forbids allocation after start-up, hosts that budget every byte
 * of device memory up front, latency-critical loops that cannot afford an
 * allocation or its possible implicit synchronisation.  The paper has no
 * counterpart: this is a library facility.  out_i = rotate(in_i, step) for
 * i < count, one step for all (0 < step < n/2 right shift of each slot row,
 * 0 = row swap), device layout, NTT form; the result is identical to
 * lola_rotate's.  Scratch comes from a static device array of
 * LOLA_ROTATE_NOALLOC_SCRATCH_BYTES compiled into the library, which every
 * GPU that loads the library keeps until the process exits.  The first call
 * with a context looks up that array's address on the context's device
 * (cudaGetSymbolAddress) and keeps it in the context, so make that first
 * call before any stream capture.  Calls share the array: calls that overlap
 * on the GPU race and must be serialised by the caller.  No part of the
 * array needs clearing between calls.  A count whose scratch does not fit
 * returns LOLA_E_PARAM; the scratch is count * (L + D*(L+K) + 2K) * n words
 * (D = key-switching digits, ceil(L / alpha)), plus count * 2 * (L+K) * n
 * words when D = 1 (a separate inner-product area); missing key:
 * LOLA_E_NOKEY. */
#define LOLA_ROTATE_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int lola_rotate_noalloc(lola_ctx* ctx, const lola_keys* keys, const uint64_t* in, uint64_t* out, size_t count,
                        int32_t step, void* stream);
/* Hoisted rotations (several rotations of the same ciphertexts, Sec. 3.1
 * rot; a batching of the rotate-and-sum building block of Sec. 4.1): every
 * one of `count` ciphertexts in `in` (device, [count][2][L][n]) is rotated
 * by each of the n_steps steps (0 = row swap); out (device, caller-owned,
 * [n_steps][count][2][L][n], must not overlap in) receives step-major
 * results.  The digits [c1]_{q_i} are computed and raised to Q*P once; the
 * rotation by g uses the digits tau_g([c1]_{q_i}) taken over Z (congruent
 * to tau_g(c1) mod q_i), so results decrypt like lola_rotate's but differ
 * from them in the key-switching noise.  Errors: LOLA_E_NOKEY,
 * LOLA_E_PARAM, LOLA_E_CUDA, LOLA_E_NOMEM (scratch is allocated per call). */
int lola_rotate_hoisted(lola_ctx* ctx, const lola_keys* keys, const uint64_t* in, uint64_t* out, size_t count,
                        const int32_t* steps, size_t n_steps, void* stream);
/* Rotate-sum (the rotate-and-sum of Sec. 4.1 with several doubling steps in
 * one key switch; not in the paper, which takes one rotation per step):
 * out_i = in_i + sum_s rot(in_i, steps[s]) for each of `count` ciphertexts
 * (device, [count][2][L][n], NTT form; out caller-owned, same layout, must
 * not overlap in).  Steps: 0 < step < n/2 right shifts of each slot row, 0 =
 * row swap, repeats allowed, at most 64; two doubling steps x + rot(x, a),
 * then + rot(., b), are steps {a, b, a + b}.  The digits of c1 are raised
 * to Q*P once; the inner products with every step's key (digits permuted as
 * in lola_rotate_hoisted) are added over Q*P and brought down by one
 * mod-down, so the result decrypts to the sum of the rotations and differs
 * from adding lola_rotate_hoisted's outputs by the rounding of one mod-down
 * instead of one per step.  n_steps = 0 copies in to out.  Errors:
 * LOLA_E_NOKEY, LOLA_E_PARAM, LOLA_E_CUDA, LOLA_E_NOMEM (scratch is
 * allocated per call: count * (L + D*(L+K) + 2(L+K) + 2K) * n words, D the
 * key-switching digits). */
int lola_rotate_sum(lola_ctx* ctx, const lola_keys* keys, const uint64_t* in, uint64_t* out, size_t count,
                    const int32_t* steps, size_t n_steps, void* stream);
/* Modulus switching (BFV; not in the paper, which leaves SEAL's modulus
 * management unstated): every ciphertext of in (device, [count][2][L_from][n]
 * over q_0..q_{L_from-1}) becomes one over the first L_to primes, out
 * (device, [count][2][L_to][n], must not overlap in).  Primes are dropped
 * from the top one at a time: coefficient x mod Q becomes round(x / q_l)
 * mod Q / q_l, computed exactly as (c_j - x~) q_l^-1 mod q_j with x~ the
 * centered residue of x mod q_l.  Decryption is unchanged (the noise shrinks
 * with Q, plus a rounding term), and every later operation costs less: a
 * key switch at L' primes runs L'(L'+1) + 2L' + 2 limb transforms (K = 1).  Keys
 * need no change (a level uses the entries of its digits and primes).
 * 1 <= L_to <= L_from <= L.  Errors: LOLA_E_PARAM, LOLA_E_NOMEM (scratch). */
int lola_mod_switch(lola_ctx* ctx, const uint64_t* in, uint64_t* out, size_t count, uint32_t L_from, uint32_t L_to,
                    void* stream);
/* Decrypt ciphertexts at level L' (device, [n_msg][k_t][2][L'][n], e.g. the
 * output of lola_mod_switch) without CRT: out host [n_msg][k_t][n]. */
int lola_decrypt_residues_level(lola_ctx* ctx, const lola_keys* keys, const uint64_t* d_ct, size_t n_msg,
                                uint32_t level, uint64_t* out);
/* ct x plaintext: out_i = in_i * encode(slots_i) (slots host [count][n]
 * int64, centered lift mod t). */
int lola_mul_plain(lola_ctx* ctx, const uint64_t* in, const int64_t* slots, uint64_t* out, size_t count,
                   const uint32_t* t_index, void* stream);

/* ---------------------------------------------------------------- tuning
 * Launch geometry of the key-switch transforms (kernel 0 decompose, 1 mod-up,
 * 2 INTT mod P, 3 mod-down) for each of LOLA_TUNE_BUCKETS launch sizes
 * (limb transforms per launch: < 64, < 256, < 1024, < 4096, < 16384, more):
 * 0 = one CTA per limb, 1 = a 2-CTA cluster per limb with 16 words per
 * thread, 2 = a 2-CTA cluster with 32 words per thread, 3 = a 4-CTA cluster
 * with 16 words per thread (1-3 at n = 16384 only).  Every geometry computes the same words.  Without tuning the
 * library uses clusters for kernels 1-3 at n = 16384 (16 words below 400
 * limb transforms, else 32) and one CTA for decompose.
 * lola_autotune times whole rotations (CUDA events, zero-filled buffers
 * and key, 1 to 256 ciphertexts: about 1.9 GB at n = 16384, L = 5, freed on
 * return) with each kernel's entry for the bucket its launch falls in set
 * to each geometry in turn, keeps a geometry other than the default only
 * when the rotations get more than 3 % faster, and installs the table for
 * the context and all of its modulus-switching levels (a fraction of a
 * second); run it while nothing else uses the context.  lola_tune_get copies the table (4 x 6 bytes, kernel-major) and,
 * if us is not NULL, the measured microseconds per launch (4 x 6 x 4 floats,
 * 0 where not run); LOLA_E_STATE when no table is installed.  lola_tune_set
 * installs a table (e.g. from a cache file); NULL restores the defaults.
 * Errors: LOLA_E_PARAM (bad entry), LOLA_E_NOMEM, LOLA_E_CUDA. */
#define LOLA_TUNE_KERNELS 4
#define LOLA_TUNE_BUCKETS 6
#define LOLA_TUNE_VARIANTS 4
int lola_autotune(lola_ctx* ctx, void* stream);
int lola_tune_get(const lola_ctx* ctx, uint8_t* table, float* us);
int lola_tune_set(lola_ctx* ctx, const uint8_t* table);

/* ------------------------------------------------------------ networks
 * Message representations (Sec. 4.2.1). */
typedef enum {
  LOLA_REPR_DENSE = 1,       /* m_i = v_i (message 0) */
  LOLA_REPR_SPARSE = 2,      /* k messages, message i constant v_i */
  LOLA_REPR_STACKED = 3,     /* copies of v every 2^d slots */
  LOLA_REPR_INTERLEAVED = 4, /* m_sigma(i) = v_i */
  LOLA_REPR_CONVOLUTION = 5  /* r messages, m^j_i = v_sigma_i(j) */
} lola_repr;

/* Layers (Sec. 4.2.2 matrix-vector algorithms, Sec. 3.2 square, Sec. 4.3
 * combine).  Weights are host int64, row-major rows x cols, copied. */
typedef enum {
  LOLA_LAYER_CONV_ROWMAJOR = 1,        /* convolution -> dense messages (one per row of W) */
  LOLA_LAYER_COMBINE = 2,              /* k dense messages -> 1: message m rotated by m*stride, or by
                                          weights[m] (1 x k, weights[0] = 0) when weights is given */
  LOLA_LAYER_SQUARE = 3,               /* elementwise square (ct (x) ct) */
  LOLA_LAYER_STACK = 4,                /* dense -> stacked: copies every 2^d slots */
  LOLA_LAYER_STACKED_ROWMAJOR = 5,     /* stacked -> interleaved (mask + combine rounds) */
  LOLA_LAYER_INTERLEAVED_ROWMAJOR = 6, /* interleaved/dense -> sparse (one message per row) */
  LOLA_LAYER_DENSE_ROWMAJOR = 7,       /* dense -> sparse */
  LOLA_LAYER_SPARSE_COLMAJOR = 8,      /* sparse (one message per element) -> dense: sum_i v_i * column_i */
  LOLA_LAYER_MASKED_SHIFTS = 9,        /* dense -> convolution by masking (App. C, LoLa-Dense): weights
                                          rows x cols = messages x elements, entry = input element index
                                          held by message r at element e (-1 = zero); message r must be a
                                          single shift off_r of message 0 (x * mask_r, rotated left by off_r) */
  LOLA_LAYER_PLACE = 10,               /* k dense messages -> 1 with element e at slot weights[e] (one target
                                          per element, both slot rows; Sec. 6.2 combine of 83 maps); the
                                          messages must hold zeros outside their elements' slots */
  LOLA_LAYER_MOD_SWITCH = 11,          /* modulus switching to the first d primes of Q (lola_mod_switch);
                                          no slot changes, later layers run on d primes; not in the paper */
  LOLA_LAYER_INTERLEAVED_ROWMAJOR_SUPPORT = 12
                                       /* interleaved/dense -> one message per row, each dot product summed
                                          over the vector's occupied slots only: when they form one cyclic run
                                          of 2^k slots modulo a period 2^p in each row, rotations 1 .. 2^(k-1),
                                          then 2^p .. n/4, then the row swap if both rows are occupied (the
                                          fewest such steps; the full support gives the interleaved row-major
                                          product's); output r at the one slot holding the whole sum */
} lola_layer_op;

typedef struct {
  lola_layer_op op;
  lola_repr in_repr;      /* checked against the running representation */
  lola_repr out_repr;     /* checked against what the layer produces */
  uint32_t rows, cols;    /* weight shape (CONV: maps x window size) */
  const int64_t* weights; /* host, rows * cols; NULL for SQUARE/STACK, optional for COMBINE */
  uint32_t d;             /* STACK / STACKED_ROWMAJOR: block size 2^d; MOD_SWITCH: primes kept */
  uint32_t copies;        /* STACK / STACKED_ROWMAJOR: number of copies (power of two) */
  uint32_t stride;        /* COMBINE: slot offset between consecutive messages */
  uint32_t hoist;         /* STACK, STACKED_ROWMAJOR, INTERLEAVED_ROWMAJOR(_SUPPORT), DENSE_ROWMAJOR:
                             rotate-and-sum doubling steps per key switch.  0 or 1: one rotation per
                             step (the paper's).  m > 1: each run of up to m consecutive nonzero
                             shifts a_1 .. a_r (r > 1) is one lola_rotate_sum over the 2^r - 1 subset
                             sums of the a_i (mod n/2, ascending bit mask); a row swap, a lone shift
                             or a run with a subset sum of 0 mod n/2 stays one rotation per step.
                             The network then needs the keys of those subset sums. */
} lola_layer;

/* Input description: n_msgs messages per request, n_elems vector elements
 * (CONVOLUTION: windows per message), element i in slot slot[i] of message 0
 * (NULL = slot i).  STACKED inputs also give d and copies. */
typedef struct {
  lola_repr repr;
  uint32_t n_msgs;
  uint32_t n_elems;
  const uint32_t* slot;
  uint32_t d, copies;
} lola_input;

/* Compile a layer list: validates representations, encodes the weight
 * plaintexts for every t_i and uploads them.  Errors: LOLA_E_REPR,
 * LOLA_E_PARAM, LOLA_E_NOMEM. */
int lola_net_create(lola_ctx* ctx, const lola_input* input, const lola_layer* layers, size_t n_layers,
                    lola_net** out);
void lola_net_destroy(lola_net* net);
/* Rotation steps whose Galois keys the network needs (0 = row swap);
 * steps may be NULL to query the count. */
int lola_net_rotation_steps(const lola_net* net, int32_t* steps, size_t* count);
/* Output element o is in output message msg[o] at slot slot[o]. */
int lola_net_output_map(const lola_net* net, uint32_t* msg, uint32_t* slot, size_t* count);
/* Messages per request at the input and the output. */
int lola_net_shape(const lola_net* net, uint32_t* in_msgs, uint32_t* out_msgs);
/* Evaluate on a batch: `in` holds B * in_msgs messages (request-major), `out`
 * must hold B * out_msgs.  The first call for a batch size B builds and
 * caches the executor (scratch + CUDA graph); later calls replay it.
 * Errors: LOLA_E_NOKEY, LOLA_E_PARAM, LOLA_E_NOMEM, LOLA_E_CUDA. */
int lola_eval_network(lola_ctx* ctx, const lola_keys* keys, lola_net* net, const lola_ct* in, lola_ct* out,
                      void* stream);
/* Same, without CUDA graph capture (plain launches on `stream`). */
int lola_eval_network_eager(lola_ctx* ctx, const lola_keys* keys, lola_net* net, const lola_ct* in,
                            lola_ct* out, void* stream);

/* ------------------------------------------------------------ client packing
 * Convolution representation (Sec. 4.2.1 footnote): image h x w (host int64,
 * row-major), window kh x kw, stride s; windows with upper-left corner
 * (s*i, s*j), padded with zeros bottom/right to ceil((h-kh)/s)+1 windows per
 * axis.  out: host [kh*kw][n]; message r = dr*kw + dc holds pixel
 * (s*i+dr, s*j+dc) at slot i*ow + j.  *windows_out = oh*ow. */
int lola_pack_convolution(const int64_t* image, uint32_t h, uint32_t w, uint32_t kh, uint32_t kw, uint32_t s,
                          uint32_t n, int64_t* out, uint32_t* windows_out);
/* Stacked representation: `copies` copies of vec (length k <= 2^d) every 2^d slots. */
int lola_pack_stacked(const int64_t* vec, uint32_t k, uint32_t d, uint32_t copies, uint32_t n, int64_t* out);

/* ------------------------------------------------------------- profiling
 * CUDA events around every launch of the enabled kernels (events are
 * recorded only on eager launches; lola_eval_network runs eagerly while any
 * kernel is being profiled).  kind = kernel id in [0, lola_profile_kinds()),
 * or -1 in lola_profile_enable for all of them.  Read returns the summed
 * device milliseconds, the launch count and the work units processed since
 * the last enable: limb-polynomials (one n-word limb) for transform kernels,
 * 64-bit words or coefficient positions for element-wise kernels, 64 x
 * 64-bit products for the rotate-sum inner product (ks_ip_sum). */
int lola_profile_enable(lola_ctx* ctx, int kind, int on);
int lola_profile_read(lola_ctx* ctx, int kind, double* ms, uint64_t* launches, uint64_t* units);
int lola_profile_kinds(void);
const char* lola_profile_name(int kind);
/* Integer-unit microbenchmarks on the context's device, the measured peaks
 * the transforms' rates are stated against (the paper has no counterpart:
 * its transforms ran on a CPU).  Each kernel runs a fixed count of operations
 * per thread on register data, 8 CTAs of 256 threads per SM, timed with CUDA
 * events (best of three after one warm-up; about 0.1 s each).  kind:
 *   LOLA_ALU_FWD_BUTTERFLY   forward butterflies of the transforms (lazy,
 *                            32-bit-halves Shoup product) per second
 *   LOLA_ALU_INV_BUTTERFLY   inverse butterflies per second
 *   LOLA_ALU_FWD_BUTTERFLY_C forward butterflies with the product in the
 *                            compiler's 64-bit arithmetic, per second
 *   LOLA_ALU_MAD_LO_U32, LOLA_ALU_MAD_WIDE_U32, LOLA_ALU_MUL_HI_U32
 *                            instructions per second
 *   LOLA_ALU_MMA_S8          int8 tensor-core operations (mma.sync m16n8k32,
 *                            2 * 16 * 8 * 32 per instruction) per second
 *   LOLA_ALU_FWD_BUTTERFLY_SPARSE  forward butterflies for a prime of the
 *                            form 2^60 - c 2^32 + 1, whose product qh q
 *                            needs one 32-bit multiply, per second
 *   LOLA_ALU_MAC64           the key-switch inner products' operation: 64 x
 *                            64 -> 128-bit products of 60-bit words summed four
 *                            at a time and reduced (REDC), products per second
 * per_second and ms (best kernel time) may be NULL.  Errors: LOLA_E_PARAM
 * (unknown kind), LOLA_E_CUDA, LOLA_E_NOMEM. */
#define LOLA_ALU_FWD_BUTTERFLY 0
#define LOLA_ALU_INV_BUTTERFLY 1
#define LOLA_ALU_FWD_BUTTERFLY_C 2
#define LOLA_ALU_MAD_LO_U32 3
#define LOLA_ALU_MAD_WIDE_U32 4
#define LOLA_ALU_MUL_HI_U32 5
#define LOLA_ALU_MMA_S8 6
#define LOLA_ALU_FWD_BUTTERFLY_SPARSE 7
#define LOLA_ALU_MAC64 8
int lola_alu_rate(lola_ctx* ctx, int kind, double* per_second, double* ms);
/* Kernel launches issued by the library since context creation (launches
 * inside a replayed CUDA graph are counted once, when captured). */
uint64_t lola_launch_count(const lola_ctx* ctx);

const char* lola_last_error(void);
const char* lola_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LOLA_H */
