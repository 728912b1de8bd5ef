/*
 * Oracle ring helpers: plain, slow, obviously-correct arithmetic in
 * Z_q[x]/(x^n + 1) for one prime q at a time.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the CPU oracle that the
 * parity tests use to check the CUDA path.  Nothing in the product library
 * links, includes or calls it.
 *
 * The ring is the BFV plaintext/ciphertext ring R = Z_p[x]/(x^n+1) with n a
 * power of two (paper Sec. 3.1 and App. A).  Every residue handled here is a
 * canonical representative in [0, q).  Products use unsigned __int128 and a
 * plain `%`, nothing cleverer.
 *
 * The negacyclic product is offered twice:
 *   - ora_poly_mul_schoolbook: the definition, O(n^2): coefficient k of a*b
 *     is sum_{i+j=k} a_i b_j - sum_{i+j=k+n} a_i b_j  (x^n = -1).
 *   - ora_poly_mul_ntt: the same product through a textbook transform:
 *     twist by psi^i (psi a primitive 2n-th root of unity), a cyclic
 *     radix-2 DFT over Z_q with omega = psi^2 in natural order, pointwise
 *     product, inverse DFT, untwist by psi^-i and scale by n^-1.
 * Tests pin the second against the first.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

uint64_t ora_mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * (u128)b) % (u128)q);
}

static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) {
    u128 s = (u128)a + b;
    return (uint64_t)(s % q);
}

static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : (uint64_t)((u128)a + q - b);
}

uint64_t ora_powmod(uint64_t b, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = ora_mulmod(r, b, q);
        b = ora_mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

/* Inverse by Fermat: q is prime. */
uint64_t ora_invmod(uint64_t a, uint64_t q) { return ora_powmod(a, q - 2, q); }

void ora_vec_mulmod(const uint64_t* a, const uint64_t* b, uint64_t* out, size_t len, uint64_t q) {
    for (size_t i = 0; i < len; i++) out[i] = ora_mulmod(a[i], b[i], q);
}

void ora_vec_scalar_mulmod(const uint64_t* a, uint64_t s, uint64_t* out, size_t len, uint64_t q) {
    for (size_t i = 0; i < len; i++) out[i] = ora_mulmod(a[i], s, q);
}

void ora_vec_addmod(const uint64_t* a, const uint64_t* b, uint64_t* out, size_t len, uint64_t q) {
    for (size_t i = 0; i < len; i++) out[i] = addmod(a[i], b[i], q);
}

void ora_vec_submod(const uint64_t* a, const uint64_t* b, uint64_t* out, size_t len, uint64_t q) {
    for (size_t i = 0; i < len; i++) out[i] = submod(a[i], b[i], q);
}

/* out = a mod q for arbitrary 64-bit a */
void ora_vec_reduce(const uint64_t* a, uint64_t* out, size_t len, uint64_t q) {
    for (size_t i = 0; i < len; i++) out[i] = a[i] % q;
}

/* Negacyclic product by the definition (x^n = -1). O(n^2). */
void ora_poly_mul_schoolbook(const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n, uint64_t q) {
    for (size_t k = 0; k < n; k++) {
        uint64_t pos = 0, neg = 0;
        for (size_t i = 0; i <= k; i++) pos = addmod(pos, ora_mulmod(a[i], b[k - i], q), q);
        for (size_t i = k + 1; i < n; i++) neg = addmod(neg, ora_mulmod(a[i], b[n + k - i], q), q);
        out[k] = submod(pos, neg, q);
    }
}

/* One coefficient of the negacyclic product (for spot checks at large n). */
uint64_t ora_poly_mul_coeff(const uint64_t* a, const uint64_t* b, size_t n, uint64_t q, size_t k) {
    uint64_t pos = 0, neg = 0;
    for (size_t i = 0; i <= k; i++) pos = addmod(pos, ora_mulmod(a[i], b[k - i], q), q);
    for (size_t i = k + 1; i < n; i++) neg = addmod(neg, ora_mulmod(a[i], b[n + k - i], q), q);
    return submod(pos, neg, q);
}

static size_t bitrev(size_t x, int logn) {
    size_t r = 0;
    for (int i = 0; i < logn; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* Cyclic DFT over Z_q, natural order in and out: A_j = sum_i a_i w^(i j).
 * Iterative radix-2: bit-reversal permutation, then log n butterfly levels. */
static void cyclic_dft(uint64_t* a, size_t n, uint64_t q, uint64_t w) {
    int logn = 0;
    while (((size_t)1 << logn) < n) logn++;
    for (size_t i = 0; i < n; i++) {
        size_t j = bitrev(i, logn);
        if (j > i) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        uint64_t wl = ora_powmod(w, n / len, q); /* primitive len-th root */
        for (size_t s = 0; s < n; s += len) {
            uint64_t wk = 1;
            for (size_t k = 0; k < len / 2; k++) {
                uint64_t u = a[s + k];
                uint64_t v = ora_mulmod(a[s + k + len / 2], wk, q);
                a[s + k] = addmod(u, v, q);
                a[s + k + len / 2] = submod(u, v, q);
                wk = ora_mulmod(wk, wl, q);
            }
        }
    }
}

/* Negacyclic evaluation: A_j = a(psi^(2j+1)) = sum_i (a_i psi^i) (psi^2)^(ij). */
void ora_negacyclic_forward(uint64_t* a, size_t n, uint64_t q, uint64_t psi) {
    uint64_t p = 1;
    for (size_t i = 0; i < n; i++) { a[i] = ora_mulmod(a[i], p, q); p = ora_mulmod(p, psi, q); }
    cyclic_dft(a, n, q, ora_mulmod(psi, psi, q));
}

/* Inverse of ora_negacyclic_forward: interpolation from values at psi^(2j+1). */
void ora_negacyclic_inverse(uint64_t* a, size_t n, uint64_t q, uint64_t psi) {
    uint64_t psi_inv = ora_invmod(psi, q);
    cyclic_dft(a, n, q, ora_mulmod(psi_inv, psi_inv, q));
    uint64_t n_inv = ora_invmod((uint64_t)(n % q), q);
    uint64_t p = n_inv;
    for (size_t i = 0; i < n; i++) { a[i] = ora_mulmod(a[i], p, q); p = ora_mulmod(p, psi_inv, q); }
}

/* Negacyclic product through the transform above. */
void ora_poly_mul_ntt(const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n, uint64_t q, uint64_t psi) {
    uint64_t* fa = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint64_t* fb = (uint64_t*)malloc(n * sizeof(uint64_t));
    memcpy(fa, a, n * sizeof(uint64_t));
    memcpy(fb, b, n * sizeof(uint64_t));
    ora_negacyclic_forward(fa, n, q, psi);
    ora_negacyclic_forward(fb, n, q, psi);
    for (size_t i = 0; i < n; i++) fa[i] = ora_mulmod(fa[i], fb[i], q);
    ora_negacyclic_inverse(fa, n, q, psi);
    memcpy(out, fa, n * sizeof(uint64_t));
    free(fa);
    free(fb);
}

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies by the
 * published multipliers, with the key bumped by the published Weyl
 * constants between rounds. */
void ora_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        u128 p0 = (u128)M0 * x0;
        u128 p1 = (u128)M1 * x2;
        uint64_t y0 = (uint64_t)(p1 >> 64) ^ x1 ^ k0;
        uint64_t y1 = (uint64_t)p1;
        uint64_t y2 = (uint64_t)(p0 >> 64) ^ x3 ^ k1;
        uint64_t y3 = (uint64_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Words 0..nwords-1 of the stream (seed, tag, a, b): word w is element
 * w % 4 of Philox(counter = (w / 4, tag, a, b), key = (seed, 0)). */
void ora_philox_words(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b,
                      uint64_t first_word, uint64_t* out, size_t nwords) {
    uint64_t key[2] = {seed, 0};
    uint64_t blk[4];
    uint64_t cur = ~(uint64_t)0;
    for (size_t i = 0; i < nwords; i++) {
        uint64_t w = first_word + i;
        if (w / 4 != cur) {
            uint64_t ctr[4] = {w / 4, tag, a, b};
            ora_philox4x64_10(ctr, key, blk);
            cur = w / 4;
        }
        out[i] = blk[w % 4];
    }
}
