"""Pins for the oracle's BFV scheme and batch encoding (CPU only).

Pinned against: the homomorphic identities the paper states (Sec. 3.1:
D(E(x1) (+) E(x2)) = x1 + x2, D(E(x1) (x) E(x2)) = x1 x2), the slot-matrix
rotation semantics (Sec. 3.1), brute-force evaluation of the encoded
polynomial, and a brute-force tensor product over Z with exact rational
rounding on tiny rings.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import workloads as W
from oracle import bfv, encoding, ring


def mkparams(n, L=3, K=1, t=65537):
    ps = W.params_small(n, L=L, K=K, t=[t])
    return bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)


def row_shift(v, k):
    h = len(v) // 2
    return np.concatenate([np.roll(v[:h], k), np.roll(v[h:], k)])


# ------------------------------------------------------------------ encoding

@pytest.mark.parametrize("n,t", [(8, 65537), (32, 65537), (64, W.T30[0])])
def test_decode_is_evaluation_at_slot_points(n, t):
    m = np.random.default_rng(n).integers(0, t, n, dtype=np.uint64)
    slots = encoding.decode(m, t)
    exps = encoding.slot_exponents(n)
    for j in range(n):
        assert int(slots[j]) == encoding.evaluate(m, t, exps[j])
    # slot points are the n distinct primitive 2n-th roots psi^(odd)
    assert sorted(exps) == list(range(1, 2 * n, 2))


@pytest.mark.parametrize("n,t", [(16, 65537), (4096, 65537), (16384, W.T30[2])])
def test_encode_decode_round_trip_and_multiplicativity(n, t):
    g = np.random.default_rng(n)
    a = g.integers(0, t, n)
    b = g.integers(0, t, n)
    ma, mb = encoding.encode(a, t), encoding.encode(b, t)
    assert np.array_equal(encoding.decode(ma, t), a)
    if n <= 4096:
        prod = ring.poly_mul(ma, mb, t)
        assert np.array_equal(encoding.decode(prod, t), (a * b) % t)


def test_constant_polynomial_is_all_equal_slots():
    # Sec. 4.2.1 footnote: a vector with the same value in every coordinate
    # is the constant polynomial.
    n, t = 32, 65537
    m = encoding.encode([7] * n, t)
    assert int(m[0]) == 7 and not m[1:].any()


@pytest.mark.parametrize("k", [1, 2, 5, 15])
def test_galois_element_rotates_rows_right(k):
    # Sec. 3.1: rotating the columns of the 2 x n/2 matrix by one to the right
    # sends m_1 ... m_{n/2} to m_{n/2}, m_1, ..., m_{n/2-1}.
    n, t = 32, 65537
    v = np.arange(n) + 100
    m = encoding.encode(v, t)
    g = bfv.galois_for_rotation(n, k)
    out = encoding.decode(ring.automorphism(m, g, t), t)
    assert np.array_equal(out, row_shift(v, k))
    out = encoding.decode(ring.automorphism(m, bfv.galois_row_swap(n), t), t)
    assert np.array_equal(out, np.concatenate([v[n // 2:], v[:n // 2]]))


# ----------------------------------------------------------------- BFV scheme

@pytest.fixture(scope="module")
def small():
    P = mkparams(32)
    keys = bfv.keygen(P, 3, rotations=[1, 2, 4, 7], relin=True, row_swap=True)
    return P, keys


def enc(P, keys, v, seed=1, ct_id=0):
    t = P.t[0]
    return bfv.encrypt(P, keys.pk, encoding.encode(v, t), t, seed, ct_id)


def dec(P, keys, ct):
    return encoding.decode(bfv.decrypt(P, keys.sk, ct), ct.t)


def test_encrypt_decrypt(small):
    P, keys = small
    v = np.random.default_rng(0).integers(0, 65537, P.n)
    assert np.array_equal(dec(P, keys, enc(P, keys, v)), v)


def test_homomorphic_add_and_mul(small):
    P, keys = small
    g = np.random.default_rng(1)
    a, b = g.integers(0, 65537, P.n), g.integers(0, 65537, P.n)
    ca, cb = enc(P, keys, a, 1, 0), enc(P, keys, b, 1, 1)
    assert np.array_equal(dec(P, keys, bfv.add(P, ca, cb)), (a + b) % 65537)
    assert np.array_equal(dec(P, keys, bfv.sub(P, ca, cb)), (a - b) % 65537)
    prod3 = bfv.multiply(P, ca, cb)
    assert len(prod3.c) == 3
    assert np.array_equal(dec(P, keys, prod3), (a * b) % 65537)
    rel = bfv.relinearize(P, keys, prod3)
    assert len(rel.c) == 2
    assert np.array_equal(dec(P, keys, rel), (a * b) % 65537)
    assert np.array_equal(dec(P, keys, bfv.square(P, keys, ca)), (a * a) % 65537)


def test_mul_plain_and_scalar(small):
    P, keys = small
    g = np.random.default_rng(2)
    a = g.integers(0, 16, P.n)
    w = g.integers(-3, 4, P.n)
    ca = enc(P, keys, a)
    assert np.array_equal(dec(P, keys, bfv.mul_plain(P, ca, encoding.encode(w, 65537))), (a * w) % 65537)
    assert np.array_equal(dec(P, keys, bfv.mul_scalar(P, ca, -3)), (-3 * a) % 65537)


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_rotation_semantics(small, k):
    P, keys = small
    v = np.random.default_rng(k).integers(0, 65537, P.n)
    assert np.array_equal(dec(P, keys, bfv.rotate(P, keys, enc(P, keys, v), k)), row_shift(v, k))


def test_row_swap(small):
    P, keys = small
    v = np.random.default_rng(9).integers(0, 65537, P.n)
    h = P.n // 2
    assert np.array_equal(dec(P, keys, bfv.rotate_rows(P, keys, enc(P, keys, v))),
                          np.concatenate([v[h:], v[:h]]))


def test_hoisted_rotations_decrypt_to_rotated_slots(small):
    P, keys = small
    v = np.random.default_rng(11).integers(0, 65537, P.n)
    ct = enc(P, keys, v)
    h = P.n // 2
    outs = bfv.rotate_hoisted(P, keys, ct, [1, 7, 0, 4])
    for k, o in zip([1, 7, 0, 4], outs):
        want = np.concatenate([v[h:], v[:h]]) if k == 0 else row_shift(v, k)
        assert np.array_equal(dec(P, keys, o), want), k
        # a different, equally small key-switching noise than the plain rotation
        plain = bfv.rotate_rows(P, keys, ct) if k == 0 else bfv.rotate(P, keys, ct, k)
        m = encoding.encode(want, 65537)
        assert abs(bfv.noise_margin_bits(P, keys.sk, o, m) - bfv.noise_margin_bits(P, keys.sk, plain, m)) < 3


def test_hoisted_digits_are_congruent_to_the_rotated_polynomial(small):
    # tau_g over Z of the digit [c1]_{q_i} reduces mod q_i to tau_g(c1) mod q_i
    P, keys = small
    c1 = enc(P, keys, np.arange(P.n) % 65537).c[1]
    for g in (bfv.galois_for_rotation(P.n, 3), bfv.galois_row_swap(P.n)):
        for i, qi in enumerate(P.q[:P.L]):
            e = ring.automorphism_int(c1[i].astype(np.int64), g)
            assert all(-qi < int(x) < qi for x in e)
            assert np.array_equal(np.mod(e, qi).astype(np.uint64), ring.automorphism(c1[i], g, qi))


def test_hoisted_equals_plain_rotation_when_no_coefficient_changes_sign(small):
    # With c1 zero at every position tau_g maps past x^n, the integer digits
    # tau_g(d_i) are the plain digits [tau_g(c1)]_{q_i}: both definitions agree.
    P, keys = small
    n, k = P.n, 2
    g = bfv.galois_for_rotation(n, k)
    ct = enc(P, keys, np.random.default_rng(5).integers(0, 65537, n))
    keep = np.array([(a * g) % (2 * n) < n for a in range(n)])
    c1 = ct.c[1].copy()
    c1[:, ~keep] = 0
    ct2 = bfv.Ciphertext([ct.c[0], c1], ct.t)
    hz = bfv.rotate_hoisted(P, keys, ct2, [k])[0]
    pl = bfv.rotate(P, keys, ct2, k)
    assert np.array_equal(hz.c[0], pl.c[0]) and np.array_equal(hz.c[1], pl.c[1])
    # and they differ on a generic ciphertext (the definitions are not the same)
    hz2 = bfv.rotate_hoisted(P, keys, ct, [k])[0]
    assert not np.array_equal(hz2.c[1], bfv.rotate(P, keys, ct, k).c[1])


def test_keys_do_not_depend_on_t():
    # BFV keys involve only s and Q*P; the same keys serve every t_i.
    P1, P2 = mkparams(32, t=65537), mkparams(32, t=W.T30[0])
    k1, k2 = bfv.keygen(P1, 5, rotations=[1]), bfv.keygen(P2, 5, rotations=[1])
    assert np.array_equal(k1.pk.p0, k2.pk.p0)
    g = bfv.galois_for_rotation(32, 1)
    assert np.array_equal(k1.galois[g].b, k2.galois[g].b)


def test_key_switch_k0(small):
    P = mkparams(32, L=3, K=0)
    keys = bfv.keygen(P, 4, rotations=[3], relin=True)
    v = np.random.default_rng(4).integers(0, 65537, P.n)
    c = enc(P, keys, v)
    assert np.array_equal(dec(P, keys, bfv.rotate(P, keys, c, 3)), row_shift(v, 3))
    assert np.array_equal(dec(P, keys, bfv.square(P, keys, c)), (v * v) % 65537)


def test_moddown_is_exact_division():
    # (x - x~) / P is an integer for every x mod QP, and equals round(x/P)
    # up to the choice of representative: check on random bignums.
    P = mkparams(16)
    Pm, Q = P.P, P.Q
    g = np.random.default_rng(5)
    for _ in range(200):
        x = int(g.integers(0, 2**62)) * int(g.integers(0, 2**62)) * int(g.integers(1, 2**62)) % (Q * Pm)
        xt = bfv.centered(x, Pm)
        assert (x - xt) % Pm == 0
        y = (x - xt) // Pm
        assert abs(Fraction(x, Pm) - y) <= Fraction(1, 2)


def test_multiply_matches_bruteforce_tensor():
    # Tiny ring: compute the tensor product over Z by a double loop on Python
    # integers and round t*d/Q with exact fractions; the oracle's multiply
    # (CRT-based product over Z) must agree coefficient by coefficient.
    P = mkparams(8, L=2, K=1)
    keys = bfv.keygen(P, 6, rotations=[], relin=False)
    g = np.random.default_rng(6)
    ca = enc(P, keys, g.integers(0, 65537, 8), 2, 0)
    cb = enc(P, keys, g.integers(0, 65537, 8), 2, 1)
    out = bfv.multiply(P, ca, cb)
    Q, t, n = P.Q, 65537, 8
    lift = lambda c: [bfv.centered(v, Q) for v in P.qbasis.lift(c)]
    a0, a1, b0, b1 = lift(ca.c[0]), lift(ca.c[1]), lift(cb.c[0]), lift(cb.c[1])

    def negacyclic(x, y):
        r = [0] * n
        for i in range(n):
            for j in range(n):
                if i + j < n:
                    r[i + j] += x[i] * y[j]
                else:
                    r[i + j - n] -= x[i] * y[j]
        return r

    d0 = negacyclic(a0, b0)
    d1 = [u + v for u, v in zip(negacyclic(a0, b1), negacyclic(a1, b0))]
    d2 = negacyclic(a1, b1)
    for k, d in enumerate((d0, d1, d2)):
        want = []
        for v in d:
            f = Fraction(t * v, Q)
            r = f.numerator // f.denominator
            if f - r > Fraction(1, 2):
                r += 1
            assert f - r != Fraction(1, 2)     # never a tie
            want.append(r)
        got = P.qbasis.lift(out.c[k])
        assert got == [w % Q for w in want]


def test_noise_margin_positive_and_shrinks(small):
    P, keys = small
    v = np.random.default_rng(7).integers(0, 16, P.n)
    c = enc(P, keys, v)
    m = encoding.encode(v, 65537)
    fresh = bfv.noise_margin_bits(P, keys.sk, c, m)
    sq = bfv.square(P, keys, c)
    after = bfv.noise_margin_bits(P, keys.sk, sq, encoding.encode(v * v, 65537))
    assert fresh > after > 0


def test_full_size_rotation_and_square():
    """n = 16384, L = 5, K = 1: the MNIST-network parameters."""
    ps = W.params_mnist()
    P = bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)
    keys = bfv.keygen(P, 8, rotations=[1], relin=True)
    t = ps.t[0]
    v = np.random.default_rng(8).integers(0, 16, P.n)
    c = bfv.encrypt(P, keys.pk, encoding.encode(v, t), t, 3, 0)
    r = bfv.rotate(P, keys, c, 1)
    assert np.array_equal(encoding.decode(bfv.decrypt(P, keys.sk, r), t), row_shift(v, 1))
    s = bfv.square(P, keys, c)
    assert np.array_equal(encoding.decode(bfv.decrypt(P, keys.sk, s), t), v * v)


# --------------------------------------------------------- modulus switching

def test_mod_switch_is_rounded_division_by_the_dropped_prime():
    # Each coefficient x mod Q must become round(x / q_l) mod Q / q_l,
    # checked with bignums on the CRT lift (random residues, and the two
    # residues next to the rounding boundary q_l / 2)
    P = mkparams(16, L=3)
    ql = P.q[P.L - 1]
    g = np.random.default_rng(11)
    res = np.stack([g.integers(0, q, 16, dtype=np.uint64) for q in P.q[:P.L]])
    res[2, 0], res[2, 1] = (ql - 1) // 2, (ql + 1) // 2
    ct = bfv.Ciphertext([res, res.copy()], P.t[0])
    out = bfv.mod_switch(P, ct)
    P2 = bfv.params_at_level(P, 2)
    assert out.c[0].shape == (2, 16) and P2.Q * ql == P.Q
    for x, y in zip(P.qbasis.lift(res), P2.qbasis.lift(out.c[0])):
        assert y == ((2 * x + ql) // (2 * ql)) % P2.Q


def test_mod_switch_keeps_the_message_and_lower_levels_compute(small):
    # decryption is unchanged at every level; at level 2 and 1 the restricted
    # keys still rotate and relinearise correctly (Sec. 3.1 semantics)
    P, keys = small
    v = np.random.default_rng(12).integers(0, 16, P.n)
    c = enc(P, keys, v)
    for Lv in (2, 1):
        cl = bfv.mod_switch_to(P, c, Lv)
        Pl, kl = bfv.params_at_level(P, Lv), bfv.keys_at_level(keys, Lv)
        assert np.array_equal(dec(Pl, kl, cl), v)
        assert np.array_equal(dec(Pl, kl, bfv.rotate(Pl, kl, cl, 7)), row_shift(v, 7))
        assert np.array_equal(dec(Pl, kl, bfv.rotate_rows(Pl, kl, cl)), np.concatenate([v[16:], v[:16]]))
    Pl, kl = bfv.params_at_level(P, 2), bfv.keys_at_level(keys, 2)
    sq = bfv.square(Pl, kl, bfv.mod_switch_to(P, c, 2))
    assert np.array_equal(dec(Pl, kl, sq), (v * v) % 65537)


def test_mod_switch_keeps_the_noise_budget(small):
    # the noise is divided by q_l along with Q, plus a rounding term below
    # (1 + n) / 2 + t: with noise far above q_l n (an error of ~2^100 added to
    # c0) the budget in bits stays; with a fresh ciphertext the rounding term
    # sets the new noise, which still decrypts
    P, keys = small
    g = np.random.default_rng(13)
    v = g.integers(0, 16, P.n)
    m = encoding.encode(v, 65537)
    c = enc(P, keys, v)
    big = [int(x) << 80 for x in g.integers(-2**20, 2**20, P.n)]
    noisy = bfv.Ciphertext([bfv.add(P, c, bfv.Ciphertext([P.qbasis.reduce(big), np.zeros_like(c.c[1])], c.t)).c[0],
                            c.c[1]], c.t)
    before = bfv.noise_margin_bits(P, keys.sk, noisy, m)
    P2 = bfv.params_at_level(P, 2)
    after = bfv.noise_margin_bits(P2, keys.sk, bfv.mod_switch(P, noisy), m)
    assert 30 < before < 70 and abs(before - after) < 0.1
    fresh = bfv.noise_margin_bits(P2, keys.sk, bfv.mod_switch(P, c), m)
    assert fresh > 90        # Q' / 2t ~ 2^103 against a rounding term of a few bits


def test_level_keys_are_restrictions_of_the_full_keys(small):
    P, keys = small
    kl = bfv.keys_at_level(keys, 2)
    g = bfv.galois_for_rotation(P.n, 1)
    kf, kr = keys.galois[g], kl.galois[g]
    assert kr.b.shape == (2, 3, P.n)
    for i in range(2):
        for jl, jf in enumerate([0, 1, P.L]):
            assert np.array_equal(kr.b[i, jl], kf.b[i, jf]) and np.array_equal(kr.a[i, jl], kf.a[i, jf])


# ------------------------------------------- exact pins of the noise margin
#
# For a ciphertext whose phase is [c0 + c1 s]_Q = [Delta m + e]_Q with a
# known error e, the BFV decryption error is t x - Q m = t e - r m (mod tQ),
# r = Q mod t = Q - t Delta, and decryption is right exactly while
# |t e - r m| < Q / 2.  The tests below build such ciphertexts with their
# own schoolbook negacyclic products over Z (no oracle ring code) and check
# noise_margin_bits against log2(Q / 2) - log2(max |t e - r m|).

def schoolbook_negacyclic(a, b):
    n = len(a)
    out = [0] * n
    for i, ai in enumerate(a):
        if not ai:
            continue
        for j, bj in enumerate(b):
            k = i + j
            if k < n:
                out[k] += ai * bj
            else:
                out[k - n] -= ai * bj
    return out


def with_error(P, s, m, e, t, rng):
    """(c0, c1) over Q with c1 uniform and c0 = -c1 s + Delta m + e."""
    Q = P.Q
    a = [int(x) for x in rng.integers(0, 2**62, P.n)]
    a = [x % Q for x in a]
    D = Q // t
    as_ = schoolbook_negacyclic(a, [int(x) for x in s])
    c0 = [(-v + D * int(mi) + int(ei)) % Q for v, mi, ei in zip(as_, m, e)]
    res = lambda xs: np.array([[x % q for x in xs] for q in P.q[:P.L]], dtype=np.uint64)
    return bfv.Ciphertext([res(c0), res(a)], t)


def closed_form_margin(P, t, m, e):
    r = P.Q % t
    worst = max(abs(t * int(ei) - r * int(mi)) for mi, ei in zip(m, e))
    return math.log2(P.Q) - 1 - math.log2(worst)


@pytest.mark.parametrize("t", [65537, W.T30[0]])
@pytest.mark.parametrize("ebits", [3, 40, 90])
def test_noise_margin_equals_closed_form_bfv_error(small, t, ebits):
    P0, keys = small
    P = bfv.Params(P0.n, P0.q, P0.L, P0.K, [t])
    rng = np.random.default_rng(ebits + t % 97)
    m = rng.integers(0, t, P.n)
    e = [(int(x) << max(0, ebits - 40)) + int(y) for x, y in
         zip(rng.integers(-2**min(ebits, 40), 2**min(ebits, 40), P.n), rng.integers(-8, 8, P.n))]
    ct = with_error(P, keys.sk.s, m, e, t, rng)
    got = bfv.noise_margin_bits(P, keys.sk, ct, m)
    assert got == pytest.approx(closed_form_margin(P, t, m, e), abs=1e-9)
    assert np.array_equal(bfv.decrypt(P, keys.sk, ct), m)


def test_noise_margin_sign_is_decryption_correctness(small):
    # one coefficient's error at the decryption boundary |t e - r m| = Q / 2:
    # decryption of that coefficient flips exactly there (exact integers),
    # and the margin (a float of ~2^-20 relative resolution here) is
    # positive a hair inside and negative a hair outside
    P, keys = small
    t = P.t[0]
    Q, r = P.Q, P.Q % t
    rng = np.random.default_rng(21)
    m = rng.integers(0, t, P.n)
    e = [int(x) for x in rng.integers(-8, 8, P.n)]
    for m5 in (0, t - 1):
        m[5] = m5
        hi = (Q // 2 + r * m5) // t            # largest e with t e - r m < Q / 2
        lo = -((Q // 2 - r * m5) // t)         # smallest e with t e - r m > -Q / 2
        eps = hi >> 20
        for e5, ok in ((hi, True), (hi + 1, False), (lo, True), (lo - 1, False),
                       (hi - eps, True), (hi + eps, False), (lo + eps, True), (lo - eps, False)):
            e[5] = e5
            ct = with_error(P, keys.sk.s, m, e, t, rng)
            got = bfv.decrypt(P, keys.sk, ct)
            assert bool(got[5] == m[5]) == ok, (m5, e5)
            assert np.array_equal(np.delete(got, 5), np.delete(m, 5))
            margin = bfv.noise_margin_bits(P, keys.sk, ct, m)
            assert margin == pytest.approx(closed_form_margin(P, t, m, e), abs=1e-9)
            if abs(abs(e5) - abs(hi if e5 > 0 else lo)) > 1:
                assert (margin > 0) == ok, (m5, e5, margin)


def test_fresh_encryption_margin_is_the_public_key_error_term():
    # c = (Delta m + p0 u + e1, p1 u + e2) with p0 = -(a s + e), p1 = a has the
    # phase Delta m + e1 + e2 s - e u: recompute that error from the sampled
    # streams with schoolbook products and compare the margins exactly
    from oracle import sampling
    P = mkparams(32)
    keys = bfv.keygen(P, 3)
    t = P.t[0]
    v = np.random.default_rng(22).integers(0, 16, P.n)
    m = encoding.encode(v, t)
    ct = bfv.encrypt(P, keys.pk, m, t, 9, 4)
    u = sampling.sample_ternary(9, sampling.TAG_ENC_U, 4, 0, P.n)
    e1 = sampling.sample_gaussian(9, sampling.TAG_ENC_E1, 4, 0, P.n)
    e2 = sampling.sample_gaussian(9, sampling.TAG_ENC_E2, 4, 0, P.n)
    epk = sampling.sample_gaussian(3, sampling.TAG_PK_E, 0, 0, P.n)
    s = [int(x) for x in keys.sk.s]
    e2s = schoolbook_negacyclic([int(x) for x in e2], s)
    eu = schoolbook_negacyclic([int(x) for x in epk], [int(x) for x in u])
    err = [int(a) + b - c for a, b, c in zip(e1, e2s, eu)]
    assert bfv.noise_margin_bits(P, keys.sk, ct, m) == pytest.approx(closed_form_margin(P, t, m, err), abs=1e-9)


# ------------------------------------- key switching with grouped digits
#
# Digits of alpha primes each and K = 2 special primes (P = P1 P2 > every
# digit's modulus Q_g): the textbook CRT identity for the digits, exact
# mod-down by a two-prime P, the key-switch result u0 + u1 s = d s' + e with
# a small e, and the negative control that one special prime below the
# digit modulus leaves e of the size of Q_g / P.

def gparams(n=32, L=5, K=2, alpha=2, t=65537):
    ps = W.params_small(n, L=L, K=K, t=[t])
    return bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, alpha)


def test_digit_groups_and_crt_identity():
    P = gparams()
    assert P.groups == [[0, 1], [2, 3], [4]] and P.P == P.q[5] * P.q[6]
    g = np.random.default_rng(31)
    d = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in P.q[:P.L]])
    D = bfv.raise_digits(P, d)
    Q = P.Q
    # d_g in [0, Q_g), congruent to d on its group's primes (own CRT by hand)
    recon = [0] * P.n
    for grp, Dg in zip(P.groups, D):
        Qg = 1
        for i in grp:
            Qg *= P.q[i]
        Mg = Q // Qg
        inv = pow(Mg % Qg, -1, Qg)
        for c in range(P.n):
            # recover d_g from its residues on two primes outside the group
            # is not possible; instead rebuild it from the group's residues
            x = 0
            for i in grp:
                hi = Qg // P.q[i]
                x += int(d[i][c]) * hi * pow(hi % P.q[i], -1, P.q[i])
            x %= Qg
            for j, p in enumerate(P.q):
                assert int(Dg[j][c]) == x % p
            recon[c] += x * Mg * inv
    for c in range(P.n):
        for j in range(P.L):
            assert recon[c] % P.q[j] == int(d[j][c])


def test_mod_down_two_special_primes_is_exact_rounded_division():
    P = gparams(n=16)
    QP, Pm = P.Q * P.P, P.P
    g = np.random.default_rng(32)
    xs = [int(g.integers(0, 2**62)) * int(g.integers(0, 2**62)) * int(g.integers(0, 2**62)) ** 5 % QP
          for _ in range(P.n)]
    xs[0], xs[1] = (Pm - 1) // 2, (Pm + 1) // 2          # either side of the centering boundary
    res = np.array([[x % p for x in xs] for p in P.q], dtype=np.uint64)
    out = bfv.mod_down(P, res)
    for c, x in enumerate(xs):
        xt = x % Pm
        xt = xt - Pm if xt > Pm // 2 else xt
        y = (x - xt) // Pm
        assert (x - xt) % Pm == 0 and abs(Fraction(x, Pm) - y) <= Fraction(1, 2)
        for j in range(P.L):
            assert int(out[j][c]) == y % P.q[j]


def switch_error_bits(P, seed=33):
    """log2 of max |u0 + u1 s - d s'| (centered mod Q) for a random d and a
    relinearisation key (s' = s^2)."""
    keys = bfv.keygen(P, seed, relin=True)
    g = np.random.default_rng(seed)
    d = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in P.q[:P.L]])
    u0, u1 = bfv.key_switch(P, d, keys.relin)
    qs = P.q[:P.L]
    s = bfv._reduce_int_poly(keys.sk.s, qs)
    s2 = np.stack([ring.poly_mul(s[j], s[j], q) for j, q in enumerate(qs)])
    err = []
    for j, q in enumerate(qs):
        lhs = ring.vec_add(u0[j], ring.poly_mul(u1[j], s[j], q), q)
        err.append(ring.vec_sub(lhs, ring.poly_mul(d[j], s2[j], q), q))
    e = P.qbasis.lift_centered(np.stack(err))
    return math.log2(max(abs(v) for v in e) + 1)


@pytest.mark.parametrize("alpha,K", [(1, 1), (2, 2), (1, 2)])
def test_grouped_key_switch_error_is_small(alpha, K):
    # error ~ sum_g d_g e_g / P + rounding: below 2^20 at n = 32 whenever P > Q_g
    P = gparams(alpha=alpha, K=K)
    assert switch_error_bits(P) < 20


@pytest.mark.parametrize("alpha,K", [(2, 1), (3, 2)])
def test_special_primes_below_the_digit_modulus_leave_a_large_error(alpha, K):
    # P (K primes) < Q_g (alpha primes): the error grows to about Q_g / P = 2^60
    P = gparams(alpha=alpha, K=K)
    assert switch_error_bits(P) > 55


def test_grouped_digits_rotate_relinearise_hoist_and_switch_levels():
    P = gparams(n=32, L=5, K=2, alpha=2)
    keys = bfv.keygen(P, 34, rotations=[1, 5], relin=True, row_swap=True)
    t = P.t[0]
    v = np.random.default_rng(34).integers(0, 16, P.n)
    c = bfv.encrypt(P, keys.pk, encoding.encode(v, t), t, 3, 0)
    h = P.n // 2
    for Lv in (5, 4, 3, 2, 1):
        Pl, kl = bfv.params_at_level(P, Lv), bfv.keys_at_level(keys, Lv)
        assert Pl.groups == {5: [[0, 1], [2, 3], [4]], 4: [[0, 1], [2, 3]], 3: [[0, 1], [2]],
                             2: [[0, 1]], 1: [[0]]}[Lv]
        assert kl.relin.b.shape[0] == len(Pl.groups) == (Lv + 1) // 2
        cl = bfv.mod_switch_to(P, c, Lv)
        assert np.array_equal(dec(Pl, kl, bfv.rotate(Pl, kl, cl, 5)), row_shift(v, 5))
        assert np.array_equal(dec(Pl, kl, bfv.rotate_rows(Pl, kl, cl)), np.concatenate([v[h:], v[:h]]))
        outs = bfv.rotate_hoisted(Pl, kl, cl, [1, 0])
        assert np.array_equal(dec(Pl, kl, outs[0]), row_shift(v, 1))
        assert np.array_equal(dec(Pl, kl, outs[1]), np.concatenate([v[h:], v[:h]]))
        if Lv >= 2:
            assert np.array_equal(dec(Pl, kl, bfv.square(Pl, kl, cl)), (v * v) % t)


# ------------------------------------------- seeded symmetric encryption

def test_uniform_wide_is_the_128_bit_word_pair_reduced():
    from oracle import sampling
    q = W.Q60[0]
    w = sampling.Stream(5, sampling.TAG_SYM_A, 3, 1).words(16)
    got = sampling.uniform_wide(5, sampling.TAG_SYM_A, 3, 1, q, 8)
    for i in range(8):
        assert int(got[i]) == (int(w[2 * i]) + int(w[2 * i + 1]) * 2**64) % q


def test_symmetric_encryption_phase_is_delta_m_plus_the_sampled_error():
    from oracle import sampling
    P = mkparams(32)
    keys = bfv.keygen(P, 3)
    t = P.t[0]
    v = np.random.default_rng(41).integers(0, t, P.n)
    m = encoding.encode(v, t)
    ct = bfv.encrypt_symmetric(P, keys.sk, m, t, 7, 5)
    assert np.array_equal(dec(P, keys, ct), v)
    e = sampling.sample_gaussian(7, sampling.TAG_SYM_E, 5, 0, P.n)
    assert bfv.noise_margin_bits(P, keys.sk, ct, m) == pytest.approx(closed_form_margin(P, t, m, e), abs=1e-9)
    # c1's evaluations at psi^(2i+1) are the seeded residues (brute-force evaluation)
    for j, q in enumerate(P.q[:P.L]):
        psi = ring.smallest_primitive_2n_root(q, P.n)
        ev = sampling.uniform_wide(7, sampling.TAG_SYM_A, 5, j, q, P.n)
        for i in (0, 1, 17, P.n - 1):
            x = pow(psi, 2 * i + 1, q)
            assert sum(int(c) * pow(x, k, q) for k, c in enumerate(ct.c[1][j])) % q == int(ev[i])
    # and it is a ciphertext like any other: it rotates and squares
    keys2 = bfv.keygen(P, 3, rotations=[2], relin=True)
    assert np.array_equal(dec(P, keys2, bfv.rotate(P, keys2, ct, 2)), row_shift(v, 2))


# ------------------------------------------- hoisted rotate-and-sum (one mod-down)

def centered_diff(P, a, b):
    """max |a - b| over the coefficients, centered mod Q (a, b: (L, n) mod Q)."""
    qs = P.q[:P.L]
    d = P.qbasis.lift_centered(np.stack([ring.vec_sub(a[j], b[j], q) for j, q in enumerate(qs)]))
    return max(abs(int(x)) for x in d)


@pytest.mark.parametrize("k", [3, 0])
def test_rotate_sum_of_one_step_is_the_ciphertext_plus_its_hoisted_rotation(small, k):
    P, keys = small
    keys3 = bfv.keygen(P, 3, rotations=[1, 2, 3, 4, 7], relin=False, row_swap=True)
    ct = enc(P, keys3, np.random.default_rng(40).integers(0, 65537, P.n))
    got = bfv.rotate_sum_hoisted(P, keys3, ct, [k])
    want = bfv.add(P, ct, bfv.rotate_hoisted(P, keys3, ct, [k])[0])
    assert np.array_equal(got.c[0], want.c[0]) and np.array_equal(got.c[1], want.c[1])


@pytest.mark.parametrize("steps", [[1, 2, 3], [4, 0, 4], [1, 2, 3, 4, 5, 6, 7]])
def test_rotate_sum_decrypts_to_the_sum_of_the_rotations(steps):
    P = mkparams(32)
    keys = bfv.keygen(P, 41, rotations=sorted({s for s in steps if s}), relin=False, row_swap=True)
    v = np.random.default_rng(41).integers(0, 65537, P.n)
    ct = enc(P, keys, v)
    h = P.n // 2
    want = v.copy()
    for s in steps:
        want = want + (np.concatenate([v[h:], v[:h]]) if s == 0 else row_shift(v, s))
    out = bfv.rotate_sum_hoisted(P, keys, ct, steps)
    assert np.array_equal(dec(P, keys, out), want % 65537)


def test_rotate_sum_rounds_once_instead_of_once_per_step():
    # mod_down(sum x_k) - sum mod_down(x_k) = (sum x~_k - (sum x)~) / P: an
    # integer of absolute value at most (G + 1) / 2, and not always 0
    P = mkparams(64)
    steps = [1, 2, 3]
    keys = bfv.keygen(P, 42, rotations=steps, relin=False, row_swap=False)
    ct = enc(P, keys, np.random.default_rng(42).integers(0, 65537, P.n))
    got = bfv.rotate_sum_hoisted(P, keys, ct, steps)
    ref = ct
    for o in bfv.rotate_hoisted(P, keys, ct, steps):
        ref = bfv.add(P, ref, o)
    d0, d1 = centered_diff(P, got.c[0], ref.c[0]), centered_diff(P, got.c[1], ref.c[1])
    assert d0 <= 2 and d1 <= 2
    assert d0 + d1 > 0


def test_rotate_sum_without_special_primes_is_the_sum_of_hoisted_rotations():
    # K = 0: no mod-down, so no rounding to share: the sum is exact
    P = mkparams(32, L=3, K=0)
    steps = [1, 2, 3, 0]
    keys = bfv.keygen(P, 43, rotations=[1, 2, 3], relin=False, row_swap=True)
    ct = enc(P, keys, np.random.default_rng(43).integers(0, 16, P.n))
    got = bfv.rotate_sum_hoisted(P, keys, ct, steps)
    ref = ct
    for o in bfv.rotate_hoisted(P, keys, ct, steps):
        ref = bfv.add(P, ref, o)
    assert np.array_equal(got.c[0], ref.c[0]) and np.array_equal(got.c[1], ref.c[1])


def test_rotate_sum_noise_is_no_worse_than_two_doubling_steps():
    P = mkparams(64)
    keys = bfv.keygen(P, 44, rotations=[1, 2, 3], relin=False)
    v = np.random.default_rng(44).integers(0, 16, P.n)
    ct = enc(P, keys, v)
    seq = bfv.add(P, ct, bfv.rotate(P, keys, ct, 1))
    seq = bfv.add(P, seq, bfv.rotate(P, keys, seq, 2))
    hz = bfv.rotate_sum_hoisted(P, keys, ct, [1, 2, 3])
    want = (v + row_shift(v, 1) + row_shift(v, 2) + row_shift(v, 3)) % 65537
    m = encoding.encode(want, 65537)
    assert np.array_equal(dec(P, keys, hz), want) and np.array_equal(dec(P, keys, seq), want)
    assert bfv.noise_margin_bits(P, keys.sk, hz, m) >= bfv.noise_margin_bits(P, keys.sk, seq, m) - 1


def test_rotate_sum_with_grouped_digits_and_two_special_primes():
    P = gparams(n=32, L=5, K=2, alpha=2)
    keys = bfv.keygen(P, 45, rotations=[1, 2, 3], relin=False, row_swap=True)
    t = P.t[0]
    v = np.random.default_rng(45).integers(0, 16, P.n)
    ct = bfv.encrypt(P, keys.pk, encoding.encode(v, t), t, 3, 0)
    h = P.n // 2
    for Lv in (5, 2):
        Pl, kl = bfv.params_at_level(P, Lv), bfv.keys_at_level(keys, Lv)
        cl = bfv.mod_switch_to(P, ct, Lv)
        out = bfv.rotate_sum_hoisted(Pl, kl, cl, [1, 2, 3, 0])
        want = v + row_shift(v, 1) + row_shift(v, 2) + row_shift(v, 3) + np.concatenate([v[h:], v[:h]])
        assert np.array_equal(dec(Pl, kl, out), want % t)
