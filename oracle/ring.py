"""Oracle ring arithmetic in R_q = Z_q[x]/(x^n+1) and CRT helpers.

TEST INFRASTRUCTURE ONLY (CPU oracle for the parity tests).

Paper Sec. 3.1: the BFV ring is Z_p[x]/(x^n+1) with n a power of two; App. A
recalls that every element has a unique representative of degree < n.  An
element is held here as a numpy uint64 vector of its n coefficients in [0, q).
A polynomial over an RNS basis (q_0, ..., q_{k-1}) is a (k, n) uint64 array:
row j holds the coefficients reduced mod q_j.  CRT lifting to Python integers
is done coefficient by coefficient with Python's arbitrary-precision ints.
"""
from __future__ import annotations

from functools import lru_cache
from math import prod

import numpy as np

from . import _native
from ._native import ptr, u64


def is_prime(x: int) -> bool:
    """Deterministic Miller-Rabin for x < 3.3e24 (first 13 prime bases)."""
    if x < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)
    for p in small:
        if x % p == 0:
            return x == p
    d, s = x - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        y = pow(a, d, x)
        if y in (1, x - 1):
            continue
        for _ in range(s - 1):
            y = y * y % x
            if y == x - 1:
                break
        else:
            return False
    return True


@lru_cache(maxsize=None)
def smallest_primitive_2n_root(q: int, n: int) -> int:
    """Smallest (by value) primitive 2n-th root of unity mod the prime q.

    All primitive 2n-th roots are the odd powers of any one of them, so we
    find one (x with x^n = -1) and take the minimum over its odd powers.
    """
    assert (q - 1) % (2 * n) == 0, "q must be 1 mod 2n"
    for g in range(2, q):
        x = pow(g, (q - 1) // (2 * n), q)
        if pow(x, n, q) == q - 1:
            break
    else:  # pragma: no cover
        raise ValueError("no primitive root found")
    best, x2, cur = x, x * x % q, x
    for _ in range(n - 1):
        cur = cur * x2 % q
        best = min(best, cur)
    return best


def poly_mul(a: np.ndarray, b: np.ndarray, q: int) -> np.ndarray:
    """Negacyclic product mod q (through the textbook transform in C)."""
    n = a.shape[-1]
    a, b = u64(a), u64(b)
    out = np.empty(n, dtype=np.uint64)
    _native.lib().ora_poly_mul_ntt(ptr(a), ptr(b), ptr(out), n, q, smallest_primitive_2n_root(q, n))
    return out


def poly_mul_schoolbook(a: np.ndarray, b: np.ndarray, q: int) -> np.ndarray:
    n = a.shape[-1]
    a, b = u64(a), u64(b)
    out = np.empty(n, dtype=np.uint64)
    _native.lib().ora_poly_mul_schoolbook(ptr(a), ptr(b), ptr(out), n, q)
    return out


def poly_mul_coeff(a: np.ndarray, b: np.ndarray, q: int, k: int) -> int:
    a, b = u64(a), u64(b)
    return int(_native.lib().ora_poly_mul_coeff(ptr(a), ptr(b), a.shape[-1], q, k))


def vec_mul(a, b, q: int) -> np.ndarray:
    a, b = u64(a), u64(b)
    out = np.empty_like(a)
    _native.lib().ora_vec_mulmod(ptr(a), ptr(b), ptr(out), a.size, q)
    return out


def vec_scalar_mul(a, s: int, q: int) -> np.ndarray:
    a = u64(a)
    out = np.empty_like(a)
    _native.lib().ora_vec_scalar_mulmod(ptr(a), s % q, ptr(out), a.size, q)
    return out


def vec_add(a, b, q: int) -> np.ndarray:
    a, b = u64(a), u64(b)
    out = np.empty_like(a)
    _native.lib().ora_vec_addmod(ptr(a), ptr(b), ptr(out), a.size, q)
    return out


def vec_sub(a, b, q: int) -> np.ndarray:
    a, b = u64(a), u64(b)
    out = np.empty_like(a)
    _native.lib().ora_vec_submod(ptr(a), ptr(b), ptr(out), a.size, q)
    return out


def vec_neg(a, q: int) -> np.ndarray:
    return vec_sub(np.zeros_like(u64(a)), a, q)


def reduce_signed(values, q: int) -> np.ndarray:
    """Python/numpy signed integers -> canonical residues mod q."""
    return u64([int(v) % q for v in values])


def forward_transform(a: np.ndarray, q: int, psi: int) -> np.ndarray:
    """A_k = a(psi^(2k+1)), k = 0..n-1 (natural order)."""
    a = u64(a).copy()
    _native.lib().ora_negacyclic_forward(ptr(a), a.size, q, psi)
    return a


def inverse_transform(a: np.ndarray, q: int, psi: int) -> np.ndarray:
    a = u64(a).copy()
    _native.lib().ora_negacyclic_inverse(ptr(a), a.size, q, psi)
    return a


def automorphism_int(a: np.ndarray, g: int) -> np.ndarray:
    """tau_g over Z: a(x) -> a(x^g) mod x^n + 1 for an integer polynomial
    (int64 coefficients, |a_i| < 2^62); x^(n+r) = -x^r."""
    a = np.asarray(a, dtype=np.int64)
    n = a.shape[-1]
    e = (np.arange(n, dtype=np.int64) * g) % (2 * n)
    out = np.zeros(n, dtype=np.int64)
    out[e % n] = np.where(e >= n, -a, a)
    return out


def automorphism(a: np.ndarray, g: int, q: int) -> np.ndarray:
    """tau_g: a(x) -> a(x^g) in Z_q[x]/(x^n+1), g odd.

    x^(i*g) = x^((i*g) mod 2n), and x^(n+r) = -x^r: coefficient i moves to
    (i g mod 2n) mod n, negated mod q when i g mod 2n >= n.
    """
    a = np.asarray(a, dtype=np.uint64)
    n = a.shape[-1]
    e = (np.arange(n, dtype=np.int64) * int(g)) % (2 * n)
    neg = np.where(a == 0, np.uint64(0), np.uint64(q) - a)
    out = np.zeros(n, dtype=np.uint64)
    out[e % n] = np.where(e >= n, neg, a)
    return out


class Basis:
    """An RNS basis: CRT constants for lifting residues to Z."""

    def __init__(self, primes):
        self.primes = [int(p) for p in primes]
        self.M = prod(self.primes)
        self.hats = [self.M // p for p in self.primes]
        self.hat_invs = [pow(h % p, -1, p) for h, p in zip(self.hats, self.primes)]

    def lift(self, res: np.ndarray) -> list:
        """(k, n) residues -> list of n ints in [0, M)."""
        k, n = res.shape
        M = self.M
        coef = [h * hi for h, hi in zip(self.hats, self.hat_invs)]
        rows = [[int(x) for x in res[j]] for j in range(k)]
        return [sum(coef[j] * rows[j][i] for j in range(k)) % M for i in range(n)]

    def lift_centered(self, res: np.ndarray) -> list:
        """(k, n) residues -> list of n ints in (-M/2, M/2] (M odd: [-(M-1)/2, (M-1)/2])."""
        M, half = self.M, self.M // 2
        return [x - M if x > half else x for x in self.lift(res)]

    def reduce(self, values) -> np.ndarray:
        """Python ints (any sign) -> (k, n) canonical residues."""
        return np.array([[int(v) % p for v in values] for p in self.primes], dtype=np.uint64)
