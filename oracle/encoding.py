"""Oracle batch encoding: slot vectors <-> plaintext polynomials mod t.

TEST INFRASTRUCTURE ONLY (CPU oracle for the parity tests).

Sec. 3.1: when Z_t has an order-2n root of unity, an element of
Z_t[x]/(x^n+1) can be viewed as an n-vector over Z_t with componentwise
addition and multiplication; the rotations act on it viewed as a
2 x (n/2) matrix.  The paper does not fix which evaluation point carries
which slot.  Reading used here (and by the CUDA path):

* psi = the smallest primitive 2n-th root of unity mod t;
* slot j (row 0, j < n/2) holds m(psi^(3^j mod 2n));
* slot n/2 + j (row 1) holds m(psi^(-3^j mod 2n)).

Decoding evaluates m at those points; encoding interpolates.  Both go
through the oracle's textbook transform (values at psi^(2k+1) in natural
order k), then pick or place slot j at k = (e_j - 1) / 2.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

from . import ring


@lru_cache(maxsize=None)
def slot_exponents(n: int) -> tuple:
    """e_j such that slot j = m(psi^e_j)."""
    half = n // 2
    row0 = [pow(3, j, 2 * n) for j in range(half)]
    row1 = [(2 * n - e) % (2 * n) for e in row0]
    return tuple(row0 + row1)


def decode(m: np.ndarray, t: int) -> np.ndarray:
    n = m.shape[-1]
    psi = ring.smallest_primitive_2n_root(t, n)
    vals = ring.forward_transform(m, t, psi)
    idx = np.array([(e - 1) // 2 for e in slot_exponents(n)], dtype=np.int64)
    return vals[idx]


def encode(slots, t: int) -> np.ndarray:
    """slots: length-n integers (any sign) -> polynomial coefficients in [0, t)."""
    slots = [int(v) % t for v in slots]
    n = len(slots)
    psi = ring.smallest_primitive_2n_root(t, n)
    vals = np.zeros(n, dtype=np.uint64)
    for j, e in enumerate(slot_exponents(n)):
        vals[(e - 1) // 2] = slots[j]
    return ring.inverse_transform(vals, t, psi)


def evaluate(m, t: int, e: int) -> int:
    """m(psi^e) by Horner's rule (brute force, for pins)."""
    n = len(m)
    psi = ring.smallest_primitive_2n_root(t, n)
    x = pow(psi, e, t)
    acc = 0
    for c in reversed([int(v) for v in m]):
        acc = (acc * x + c) % t
    return acc
