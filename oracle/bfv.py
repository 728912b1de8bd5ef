"""Oracle BFV: key generation, encryption, decryption and the homomorphic
operations, each written as its mathematical definition.

TEST INFRASTRUCTURE ONLY (CPU oracle for the parity tests).

The paper fixes the scheme (BFV, Sec. 3.1: E, D, the operators (+) and (x)
with D(E(x1) (+) E(x2)) = x1 + x2 and D(E(x1) (x) E(x2)) = x1 * x2, plus the
row/column rotations) but not SEAL's internals.  The readings used here:

* Keys and ciphertexts live in coefficient form, reduced mod each prime of
  the ciphertext basis Q = q_0 ... q_{L-1}; key-switching keys additionally
  mod the special prime P = q_L when K = 1.
* Public key: p1 = a, p0 = [-(a s + e)]_Q.
* Encryption of m in [0, t)^n:  c = ([Delta m + p0 u + e1]_Q, [p1 u + e2]_Q),
  Delta = floor(Q / t).
* Decryption: x = [c0 + c1 s]_Q in [0, Q), m = round(t x / Q) mod t.
* Plaintext / scalar multiplicands are lifted to the centered range
  [-(t-1)/2, (t-1)/2] before reduction mod q_j.
* ct (x) ct: centered lifts of both ciphertexts to Z, the negacyclic tensor
  product over Z, then [round(t d_k / Q)]_Q for each of the three parts.
* Key switching of a polynomial d from s' to s: the ciphertext primes are
  grouped alpha at a time, G_g = {q_(g alpha), ..., q_(g alpha + alpha - 1)}
  (the last group may be shorter), Q_g their product; digit g is the
  integer polynomial d_g = [d]_(Q_g) with coefficients in [0, Q_g) (the CRT
  lift of d's residues on G_g; alpha = 1: d_i = [d]_(q_i)).  Key row g is
  b_g = -a_g s + e_g + [q_j in G_g] [P]_(q_j) s'  (mod q_j),
  b_g = -a_g s + e_g (mod each special prime); u = sum_g d_g (b_g, a_g) over
  Q*P, P the product of the K special primes; result (x - x~) P^-1 mod Q
  with x~ the centered residue of x mod P.  Since d_g = d mod every prime of
  G_g, the key terms sum to P d s' mod Q.  With K = 0 there is no P and no
  division (alpha = 1 then).
* Rotation by k (0 < k < n/2) is the Galois automorphism x -> x^g with
  g = 3^(n/2 - k) mod 2n followed by a key switch from tau_g(s) to s; it
  shifts each row of the 2 x n/2 slot matrix right by k (Sec. 3.1).  The row
  swap uses g = 2n - 1.
* Modulus switching (not in the paper, which does not say how SEAL's
  modulus is managed; it leaves every decrypted value unchanged): drop the
  last prime q_l of Q, c' = round(c / q_l) mod Q / q_l, one prime at a
  time.  Later operations use the first primes of Q, the same special prime
  and the key entries of the kept digits and primes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache
from math import prod

import numpy as np

from . import ring, sampling
from .ring import Basis
from .sampling import (TAG_ENC_E1, TAG_ENC_E2, TAG_ENC_U, TAG_KSK_A, TAG_KSK_E,
                       TAG_PK_A, TAG_PK_E, TAG_SECRET, TAG_SYM_A, TAG_SYM_E)


@dataclass
class Params:
    n: int
    q: list            # L + K primes, special prime last when K == 1
    L: int
    K: int
    t: list            # plaintext CRT moduli
    alpha: int = 1     # ciphertext primes per key-switching digit

    def __post_init__(self):
        self.q = [int(x) for x in self.q]
        self.t = [int(x) for x in self.t]
        assert len(self.q) == self.L + self.K and self.K in (0, 1, 2)
        assert self.alpha >= 1 and (self.K > 0 or self.alpha == 1)

    @property
    def Q(self) -> int:
        return prod(self.q[:self.L])

    @property
    def P(self) -> int:
        """Product of the special primes (1 when K = 0)."""
        return prod(self.q[self.L:self.L + self.K])

    @property
    def groups(self) -> list:
        """Digit groups: indices of the ciphertext primes of each digit."""
        a = self.alpha
        return [list(range(g, min(g + a, self.L))) for g in range(0, self.L, a)]

    @property
    def qbasis(self) -> Basis:
        return Basis(self.q[:self.L])


def galois_for_rotation(n: int, k: int) -> int:
    """Galois element of the right shift by k within each row (0 < k < n/2)."""
    assert 0 < k < n // 2
    return pow(3, n // 2 - k, 2 * n)


def galois_row_swap(n: int) -> int:
    return 2 * n - 1


# ------------------------------------------------------------------- helpers

def _reduce_int_poly(vals, primes) -> np.ndarray:
    return np.array([[int(v) % p for v in vals] for p in primes], dtype=np.uint64)


def _mul_rns(a: np.ndarray, b: np.ndarray, primes) -> np.ndarray:
    return np.stack([ring.poly_mul(a[j], b[j], p) for j, p in enumerate(primes)])


def _add_rns(a, b, primes):
    return np.stack([ring.vec_add(a[j], b[j], p) for j, p in enumerate(primes)])


def _sub_rns(a, b, primes):
    return np.stack([ring.vec_sub(a[j], b[j], p) for j, p in enumerate(primes)])


def _neg_rns(a, primes):
    return np.stack([ring.vec_neg(a[j], p) for j, p in enumerate(primes)])


def _auto_rns(a, g, primes):
    return np.stack([ring.automorphism(a[j], g, p) for j, p in enumerate(primes)])


def centered(x: int, m: int) -> int:
    """Representative of x mod m in [-(m-1)/2, (m-1)/2] (m odd)."""
    x %= m
    return x - m if x > m // 2 else x


# ---------------------------------------------------------------------- keys

@dataclass
class SecretKey:
    s: list                    # ternary integer coefficients


@dataclass
class PublicKey:
    p0: np.ndarray             # (L, n)
    p1: np.ndarray


@dataclass
class KeySwitchKey:
    b: np.ndarray              # (digits, L+K primes, n)
    a: np.ndarray


@dataclass
class Keys:
    params: Params
    sk: SecretKey
    pk: PublicKey
    relin: KeySwitchKey | None = None
    galois: dict = field(default_factory=dict)    # g -> KeySwitchKey


def gen_secret(params: Params, seed: int) -> SecretKey:
    return SecretKey(sampling.sample_ternary(seed, TAG_SECRET, 0, 0, params.n))


def gen_public(params: Params, sk: SecretKey, seed: int) -> PublicKey:
    n, qs = params.n, params.q[:params.L]
    e = sampling.sample_gaussian(seed, TAG_PK_E, 0, 0, n)
    s = _reduce_int_poly(sk.s, qs)
    er = _reduce_int_poly(e, qs)
    a = np.stack([sampling.sample_uniform(seed, TAG_PK_A, j, 0, q, n) for j, q in enumerate(qs)])
    p0 = _neg_rns(_add_rns(_mul_rns(a, s, qs), er, qs), qs)
    return PublicKey(p0, a)


def gen_switch_key(params: Params, sk: SecretKey, s_from: np.ndarray, key_id: int, seed: int) -> KeySwitchKey:
    """Key that switches a polynomial multiplying s_from (given mod every prime
    of Q*P, shape (L+K, n)) to one multiplying s.  key_id selects the stream
    (0 = relinearisation, else the Galois element).  Row g (digit group G_g)
    carries [P]_(q_j) s_from on the primes of G_g."""
    n, L, K = params.n, params.L, params.K
    primes = params.q
    s = _reduce_int_poly(sk.s, primes)
    P = params.P
    G = params.groups
    b = np.zeros((len(G), L + K, n), dtype=np.uint64)
    a = np.zeros((len(G), L + K, n), dtype=np.uint64)
    for g, grp in enumerate(G):
        e = sampling.sample_gaussian(seed, TAG_KSK_E, key_id, g, n)
        for j, pj in enumerate(primes):
            agj = sampling.sample_uniform(seed, TAG_KSK_A, key_id, g * 256 + j, pj, n)
            v = ring.vec_neg(ring.poly_mul(agj, s[j], pj), pj)
            v = ring.vec_add(v, ring.reduce_signed(e, pj), pj)
            if j in grp:
                v = ring.vec_add(v, ring.vec_scalar_mul(s_from[j], P % pj, pj), pj)
            b[g, j] = v
            a[g, j] = agj
    return KeySwitchKey(b, a)


def keygen(params: Params, seed: int, rotations=(), relin=True, row_swap=False) -> Keys:
    sk = gen_secret(params, seed)
    pk = gen_public(params, sk, seed)
    keys = Keys(params, sk, pk)
    primes = params.q
    s_all = _reduce_int_poly(sk.s, primes)
    if relin:
        s2 = _mul_rns(s_all, s_all, primes)
        keys.relin = gen_switch_key(params, sk, s2, 0, seed)
    gs = [galois_for_rotation(params.n, k) for k in rotations]
    if row_swap:
        gs.append(galois_row_swap(params.n))
    for g in gs:
        if g not in keys.galois:
            keys.galois[g] = gen_switch_key(params, sk, _auto_rns(s_all, g, primes), g, seed)
    return keys


# ---------------------------------------------------------------- ciphertext

@dataclass
class Ciphertext:
    c: list          # 2 (or 3 before relinearisation) arrays of shape (L, n)
    t: int           # plaintext modulus this ciphertext encrypts under

    def copy(self):
        return Ciphertext([x.copy() for x in self.c], self.t)


def delta(params: Params, t: int) -> int:
    return params.Q // t


def encrypt(params: Params, pk: PublicKey, m: np.ndarray, t: int, seed: int, ct_id: int) -> Ciphertext:
    """m: plaintext polynomial coefficients in [0, t)."""
    n, qs = params.n, params.q[:params.L]
    u = _reduce_int_poly(sampling.sample_ternary(seed, TAG_ENC_U, ct_id, 0, n), qs)
    e1 = _reduce_int_poly(sampling.sample_gaussian(seed, TAG_ENC_E1, ct_id, 0, n), qs)
    e2 = _reduce_int_poly(sampling.sample_gaussian(seed, TAG_ENC_E2, ct_id, 0, n), qs)
    D = delta(params, t)
    dm = np.stack([ring.vec_scalar_mul(ring.reduce_signed(m, q), D % q, q) for q in qs])
    c0 = _add_rns(_add_rns(dm, _mul_rns(pk.p0, u, qs), qs), e1, qs)
    c1 = _add_rns(_mul_rns(pk.p1, u, qs), e2, qs)
    return Ciphertext([c0, c1], t)


def seeded_c1(params: Params, seed: int, ct_id: int) -> np.ndarray:
    """The c1 of a seeded symmetric encryption, shape (L, n), coefficient
    form: on prime q_j its evaluations a(psi_j^(2i+1)), i = 0..n-1 (psi_j
    the smallest primitive 2n-th root of unity mod q_j), are the residues
    uniform_wide(seed, TAG_SYM_A, ct_id, j) -- so a server can regenerate c1
    in the evaluation domain from (seed, ct_id) alone."""
    n = params.n
    out = []
    for j, q in enumerate(params.q[:params.L]):
        ev = sampling.uniform_wide(seed, TAG_SYM_A, ct_id, j, q, n)
        out.append(ring.inverse_transform(ev, q, ring.smallest_primitive_2n_root(q, n)))
    return np.stack(out)


def encrypt_symmetric(params: Params, sk: SecretKey, m: np.ndarray, t: int, seed: int, ct_id: int) -> Ciphertext:
    """Symmetric (secret-key) encryption with a seeded c1: c1 = a from
    seeded_c1, c0 = [Delta m + e - a s]_Q with e Gaussian from stream
    (seed, TAG_SYM_E, ct_id, 0).  Decrypts like encrypt's output (phase
    Delta m + e).  The client holds s (Sec. 1: it encrypts and decrypts), so
    it may encrypt this way and send c0 and the seed instead of c1."""
    n, qs = params.n, params.q[:params.L]
    a = seeded_c1(params, seed, ct_id)
    e = _reduce_int_poly(sampling.sample_gaussian(seed, TAG_SYM_E, ct_id, 0, n), qs)
    s = _reduce_int_poly(sk.s, qs)
    D = delta(params, t)
    dm = np.stack([ring.vec_scalar_mul(ring.reduce_signed(m, q), D % q, q) for q in qs])
    c0 = _sub_rns(_add_rns(dm, e, qs), _mul_rns(a, s, qs), qs)
    return Ciphertext([c0, a], t)


def _phase(params: Params, sk: SecretKey, ct: Ciphertext) -> list:
    """[c0 + c1 s (+ c2 s^2)]_Q as ints in [0, Q)."""
    qs = params.q[:params.L]
    s = _reduce_int_poly(sk.s, qs)
    acc = ct.c[0]
    spow = s
    for k in range(1, len(ct.c)):
        acc = _add_rns(acc, _mul_rns(ct.c[k], spow, qs), qs)
        spow = _mul_rns(spow, s, qs)
    return params.qbasis.lift(acc)


def decrypt(params: Params, sk: SecretKey, ct: Ciphertext) -> np.ndarray:
    """m = round(t x / Q) mod t; no ties since Q is odd and coprime to t."""
    Q, t = params.Q, ct.t
    xs = _phase(params, sk, ct)
    return np.array([((2 * t * x + Q) // (2 * Q)) % t for x in xs], dtype=np.uint64)


def noise_margin_bits(params: Params, sk: SecretKey, ct: Ciphertext, m_expected) -> float:
    """log2(Q/2) - log2(max |t x - Q m|), with t x - Q m taken centered mod tQ.

    Decryption returns m_expected exactly when the margin is positive."""
    Q, t = params.Q, ct.t
    xs = _phase(params, sk, ct)
    worst = 0
    for x, m in zip(xs, m_expected):
        w = centered(t * x - Q * int(m), t * Q)
        worst = max(worst, abs(w))
    if worst == 0:
        return float("inf")
    return math.log2(Q) - 1.0 - math.log2(worst)


def add(params: Params, a: Ciphertext, b: Ciphertext) -> Ciphertext:
    qs = params.q[:params.L]
    assert a.t == b.t and len(a.c) == len(b.c)
    return Ciphertext([_add_rns(x, y, qs) for x, y in zip(a.c, b.c)], a.t)


def sub(params: Params, a: Ciphertext, b: Ciphertext) -> Ciphertext:
    qs = params.q[:params.L]
    return Ciphertext([_sub_rns(x, y, qs) for x, y in zip(a.c, b.c)], a.t)


def mul_plain(params: Params, ct: Ciphertext, m: np.ndarray) -> Ciphertext:
    """ct times the plaintext polynomial m (coefficients in [0, t)), centered lift."""
    qs = params.q[:params.L]
    t = ct.t
    p = _reduce_int_poly([centered(int(v), t) for v in m], qs)
    return Ciphertext([_mul_rns(x, p, qs) for x in ct.c], t)


def mul_scalar(params: Params, ct: Ciphertext, w: int) -> Ciphertext:
    """ct times the constant polynomial w (any integer; centered lift mod t)."""
    qs = params.q[:params.L]
    wc = centered(int(w), ct.t)
    return Ciphertext([np.stack([ring.vec_scalar_mul(x[j], wc % q, q) for j, q in enumerate(qs)])
                       for x in ct.c], ct.t)


def raise_digits(params: Params, d: np.ndarray) -> list:
    """The digits of d (shape (L, n), mod Q) raised to Q*P: entry g is the
    (L+K, n) array of the integer digit d_g = [d]_(Q_g) in [0, Q_g) reduced
    mod every prime (for a single-prime group, d_i itself on its prime)."""
    out = []
    for grp in params.groups:
        if len(grp) == 1:
            vals = d[grp[0]].astype(np.int64)
            out.append(np.stack([np.mod(vals, np.int64(p)).astype(np.uint64) for p in params.q]))
        else:
            ints = Basis([params.q[i] for i in grp]).lift(d[grp])      # [0, Q_g)
            out.append(np.stack([np.array([v % p for v in ints], dtype=np.uint64) for p in params.q]))
    return out


def mod_down(params: Params, x: np.ndarray) -> np.ndarray:
    """(x - x~) P^-1 mod Q for x given mod every prime of Q*P (shape
    (L+K, n)), x~ the centered residue of x mod P; identity when K = 0."""
    L, K = params.L, params.K
    if K == 0:
        return x[:L]
    P = params.P
    xt = Basis(params.q[L:L + K]).lift_centered(x[L:L + K])
    res = []
    for j in range(L):
        qj = params.q[j]
        pinv = pow(P, -1, qj)
        res.append(np.array([((int(x[j][c]) - xt[c]) * pinv) % qj for c in range(params.n)], dtype=np.uint64))
    return np.stack(res)


def key_switch_inner(params: Params, D: list, ksk: KeySwitchKey) -> list:
    """The key-switch inner products sum_g D_g * ksk_g over Q * P, one
    (L+K, n) array per key component (b, a), for raised digits D
    (raise_digits, possibly permuted); no mod-down."""
    out = []
    for comp in (ksk.b, ksk.a):
        acc = []
        for j, pj in enumerate(params.q):
            s = np.zeros(params.n, dtype=np.uint64)
            for g in range(len(D)):
                s = ring.vec_add(s, ring.poly_mul(D[g][j], comp[g, j], pj), pj)
            acc.append(s)
        out.append(np.stack(acc))
    return out


def key_switch_raised(params: Params, D: list, ksk: KeySwitchKey):
    """The key-switch inner product sum_g D_g * ksk_g over Q * P and the
    mod-down, for raised digits D (raise_digits, possibly permuted)."""
    acc = key_switch_inner(params, D, ksk)
    return mod_down(params, acc[0]), mod_down(params, acc[1])


def key_switch(params: Params, d: np.ndarray, ksk: KeySwitchKey):
    """Switch d (shape (L, n), mod Q) from s' to s; returns (u0, u1) mod Q."""
    return key_switch_raised(params, raise_digits(params, d), ksk)


def apply_galois(params: Params, ct: Ciphertext, g: int, ksk: KeySwitchKey) -> Ciphertext:
    qs = params.q[:params.L]
    c0 = _auto_rns(ct.c[0], g, qs)
    c1 = _auto_rns(ct.c[1], g, qs)
    u0, u1 = key_switch(params, c1, ksk)
    return Ciphertext([_add_rns(c0, u0, qs), u1], ct.t)


def rotate(params: Params, keys: Keys, ct: Ciphertext, k: int) -> Ciphertext:
    g = galois_for_rotation(params.n, k)
    return apply_galois(params, ct, g, keys.galois[g])


def rotate_hoisted(params: Params, keys: Keys, ct: Ciphertext, steps) -> list:
    """Rotations of one ciphertext by several steps sharing one digit
    decomposition (hoisting; step 0 = row swap).  The digits of c1 are raised
    to Q*P once (raise_digits: the integer digits d_g in [0, Q_g)); rotation
    g switches tau_g(c1) with the digits tau_g(d_g) taken over Z
    (coefficients in (-Q_g, Q_g)), which are congruent to tau_g(c1) mod the
    primes of G_g, then adds tau_g(c0).  tau_g of an integer polynomial
    reduced mod p is tau_g of its residues mod p, so the raised digits are
    permuted prime by prime.  At g = 1 the digits are those of key_switch;
    for other g the result differs from apply_galois by a different (equally
    valid) key-switching noise."""
    qs = params.q[:params.L]
    D = raise_digits(params, ct.c[1])
    out = []
    for k in steps:
        g = galois_row_swap(params.n) if k == 0 else galois_for_rotation(params.n, k)
        c0 = _auto_rns(ct.c[0], g, qs)
        Dg = [np.stack([ring.automorphism(Dd[j], g, p) for j, p in enumerate(params.q)]) for Dd in D]
        u0, u1 = key_switch_raised(params, Dg, keys.galois[g])
        out.append(Ciphertext([_add_rns(c0, u0, qs), u1], ct.t))
    return out


def rotate_sum_hoisted(params: Params, keys: Keys, ct: Ciphertext, steps) -> Ciphertext:
    """ct plus its rotations by every step of `steps` (step 0 = row swap; a
    step may repeat) with one digit raising and one mod-down.

    Reading (not in the paper, whose rotate-and-sum takes one rotation per
    doubling step, Sec. 4.1): two doubling steps x + rot(x, a), then
    + rot(., b), equal x + rot(x, a) + rot(x, b) + rot(x, a + b), rotations of
    one ciphertext.  Their digits are raised once and permuted per step as in
    rotate_hoisted; the inner products with each step's key are added over
    Q * P and brought down by a single mod-down, and tau_g(c0) of every step
    is added to c0 (c1 keeps its own term).  The result decrypts to the sum
    of the rotations; against adding the hoisted rotations one by one it
    differs by the rounding of one mod-down instead of one per step: at most
    (len(steps) + 1) / 2 per coefficient in absolute value."""
    qs = params.q[:params.L]
    D = raise_digits(params, ct.c[1])
    c0 = ct.c[0].copy()
    acc = None
    for k in steps:
        g = galois_row_swap(params.n) if k == 0 else galois_for_rotation(params.n, k)
        c0 = _add_rns(c0, _auto_rns(ct.c[0], g, qs), qs)
        Dg = [np.stack([ring.automorphism(Dd[j], g, p) for j, p in enumerate(params.q)]) for Dd in D]
        ip = key_switch_inner(params, Dg, keys.galois[g])
        acc = ip if acc is None else [_add_rns(acc[c], ip[c], params.q) for c in range(2)]
    u0, u1 = mod_down(params, acc[0]), mod_down(params, acc[1])
    return Ciphertext([_add_rns(c0, u0, qs), _add_rns(ct.c[1], u1, qs)], ct.t)


def rotate_rows(params: Params, keys: Keys, ct: Ciphertext) -> Ciphertext:
    g = galois_row_swap(params.n)
    return apply_galois(params, ct, g, keys.galois[g])


# ------------------------------------------------------ modulus switching

def params_at_level(params: Params, Lv: int) -> Params:
    """Parameters of a ciphertext that keeps the first Lv primes of Q (after
    modulus switching); the special primes, the digit size and the plaintext
    moduli stay (the digit groups are those of the first Lv primes)."""
    assert 1 <= Lv <= params.L
    return Params(params.n, params.q[:Lv] + params.q[params.L:], Lv, params.K, params.t, params.alpha)


def keys_at_level(keys: Keys, Lv: int) -> Keys:
    """The key set restricted to level Lv: public key on q_0..q_{Lv-1};
    switching keys on the digit groups that meet q_0..q_{Lv-1} and on those
    primes plus the special primes.  Every kept entry is unchanged, and it is
    what gen_switch_key defines for the level's groups (a group cut short by
    the level keeps [P]_(q_j) s' exactly on its remaining primes), so the
    restriction is a key set of params_at_level."""
    full = keys.params
    sel = list(range(Lv)) + list(range(full.L, full.L + full.K))
    nd = len(params_at_level(full, Lv).groups)

    def cut(k):
        return None if k is None else KeySwitchKey(k.b[:nd][:, sel], k.a[:nd][:, sel])

    return Keys(params_at_level(full, Lv), keys.sk, PublicKey(keys.pk.p0[:Lv], keys.pk.p1[:Lv]),
                cut(keys.relin), {g: cut(k) for g, k in keys.galois.items()})


def mod_switch(params: Params, ct: Ciphertext) -> Ciphertext:
    """Modulus switching from Q to Q' = Q / q_l, q_l the last prime of Q:
    every coefficient x mod Q becomes round(x / q_l) mod Q'.  In RNS this is
    exact: x - x~ is divisible by q_l when x~ is the centered residue of x
    mod q_l, so c'_j = (c_j - x~) q_l^-1 mod q_j for every other prime.  The
    result decrypts under params_at_level(params, L - 1) to the same message
    (Delta' = floor(Q'/t); the noise is divided by q_l and gains a rounding
    term below (1 + n) / 2 + t)."""
    L = params.L
    assert L >= 2 and all(x.shape[0] == L for x in ct.c)
    ql = params.q[L - 1]
    out = []
    for x in ct.c:
        top = x[L - 1].astype(np.int64)
        xt = np.where(top > ql // 2, top - ql, top)            # centered residue mod q_l
        limbs = []
        for j in range(L - 1):
            qj = params.q[j]
            v = np.mod(x[j].astype(np.int64) - xt, np.int64(qj)).astype(np.uint64)
            limbs.append(ring.vec_scalar_mul(v, pow(ql, -1, qj), qj))
        out.append(np.stack(limbs))
    return Ciphertext(out, ct.t)


def mod_switch_to(params: Params, ct: Ciphertext, Lv: int) -> Ciphertext:
    """Drop primes from the top one at a time until Lv remain."""
    p = params
    while p.L > Lv:
        ct = mod_switch(p, ct)
        p = params_at_level(p, p.L - 1)
    return ct


@lru_cache(maxsize=None)
def _aux_primes(n: int, bits_needed: int) -> list:
    """The oracle's own auxiliary primes (= 1 mod 2n, descending below 2^61)
    whose product exceeds 2^bits_needed; used only to compute products over Z."""
    out, x = [], ((1 << 61) - 1) // (2 * n) * (2 * n) + 1
    while sum(p.bit_length() - 1 for p in out) < bits_needed:
        if x < (1 << 61) and ring.is_prime(x):
            out.append(x)
        x -= 2 * n
    return tuple(out)


def poly_mul_over_Z(a: list, b: list, n: int, bound_bits: int) -> list:
    """Exact negacyclic product of two integer polynomials whose product
    coefficients are below 2^bound_bits in magnitude: computed mod enough
    primes and lifted back by CRT (centered)."""
    aux = _aux_primes(n, bound_bits + 2)
    basis = Basis(aux)
    ar = _reduce_int_poly(a, aux)
    br = _reduce_int_poly(b, aux)
    return basis.lift_centered(_mul_rns(ar, br, aux))


def multiply(params: Params, x: Ciphertext, y: Ciphertext) -> Ciphertext:
    """ct (x) ct without relinearisation: three parts, each
    [round(t * d_k / Q)]_Q of the tensor product over Z of centered lifts."""
    assert x.t == y.t
    n, Q, t = params.n, params.Q, x.t
    qb = params.qbasis
    a0, a1 = qb.lift_centered(x.c[0]), qb.lift_centered(x.c[1])
    b0, b1 = qb.lift_centered(y.c[0]), qb.lift_centered(y.c[1])
    bound = 2 * (Q.bit_length()) + n.bit_length() + 1
    d0 = poly_mul_over_Z(a0, b0, n, bound)
    d1a = poly_mul_over_Z(a0, b1, n, bound)
    d1b = poly_mul_over_Z(a1, b0, n, bound)
    d2 = poly_mul_over_Z(a1, b1, n, bound)
    d1 = [u + v for u, v in zip(d1a, d1b)]
    qs = params.q[:params.L]
    # round(t d / Q) = floor((2 t d + Q) / (2 Q)); never a tie (Q odd, gcd(Q, t) = 1)
    parts = [[(2 * t * v + Q) // (2 * Q) for v in d] for d in (d0, d1, d2)]
    return Ciphertext([_reduce_int_poly(p, qs) for p in parts], t)


def relinearize(params: Params, keys: Keys, ct: Ciphertext) -> Ciphertext:
    qs = params.q[:params.L]
    assert len(ct.c) == 3
    u0, u1 = key_switch(params, ct.c[2], keys.relin)
    return Ciphertext([_add_rns(ct.c[0], u0, qs), _add_rns(ct.c[1], u1, qs)], ct.t)


def square(params: Params, keys: Keys, ct: Ciphertext) -> Ciphertext:
    return relinearize(params, keys, multiply(params, ct, ct))
