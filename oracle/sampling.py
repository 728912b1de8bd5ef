"""Oracle sampler: Philox4x64-10 word streams and the three BFV distributions.

TEST INFRASTRUCTURE ONLY (CPU oracle for the parity tests).

The paper uses SEAL's BFV and does not describe its randomness (Sec. 3.1,
footnote on SEAL 2.3.1).  Bit-exact parity between two independent
implementations needs one fixed definition, which is this one:

* Stream (seed, tag, a, b) is the word sequence w_0, w_1, ... where word w is
  element (w mod 4) of Philox4x64-10(counter = (w div 4, tag, a, b),
  key = (seed, 0)).  Philox4x64-10 is the counter-based generator of Salmon
  et al., SC'11; the oracle's copy is plain C.
* uniform mod q: per coefficient, draw words until (w AND (2^bitlen(q) - 1)) < q.
* ternary {-1, 0, 1}: draw words until w < 3 * floor(2^64 / 3); then w mod 3
  maps 0 -> 0, 1 -> 1, 2 -> -1.
* discrete Gaussian, sigma = 3.2, support |k| <= 19: one word w per
  coefficient; sign = top bit; u = low 63 bits; |e| = the least k with
  u < T[k], where T[k] = floor(2^63 * (rho(0) + 2 sum_{j=1..k} rho(j)) / S),
  rho(j) = exp(-j^2 / (2 sigma^2)), S = rho(0) + 2 sum_{j=1..19} rho(j),
  and T[19] = 2^63.  The thresholds are computed here with Python's decimal
  module at 80 significant digits.
"""
from __future__ import annotations

from decimal import Decimal, localcontext
from functools import lru_cache

import numpy as np

from . import _native
from ._native import ptr

SIGMA = Decimal("3.2")
GAUSS_BOUND = 19

# stream tags
TAG_SECRET = 1
TAG_PK_A = 2
TAG_PK_E = 3
TAG_KSK_A = 4
TAG_KSK_E = 5
TAG_ENC_U = 6
TAG_ENC_E1 = 7
TAG_ENC_E2 = 8
TAG_SYM_A = 9      # seeded c1 of symmetric encryption (evaluation values)
TAG_SYM_E = 10     # error of symmetric encryption


class Stream:
    """Sequential reader over one Philox word stream."""

    CHUNK = 1 << 14

    def __init__(self, seed: int, tag: int, a: int = 0, b: int = 0):
        self.key = (seed & (2**64 - 1), tag, a, b)
        self.pos = 0
        self.buf = np.empty(0, dtype=np.uint64)
        self.buf_start = 0

    def _fill(self, first: int, count: int):
        out = np.empty(count, dtype=np.uint64)
        s, t, a, b = self.key
        _native.lib().ora_philox_words(s, t, a, b, first, ptr(out), count)
        self.buf, self.buf_start = out, first

    def words(self, count: int) -> np.ndarray:
        out = np.empty(count, dtype=np.uint64)
        done = 0
        while done < count:
            off = self.pos - self.buf_start
            if off < 0 or off >= self.buf.size:
                self._fill(self.pos, max(self.CHUNK, count - done))
                off = 0
            take = min(count - done, self.buf.size - off)
            out[done:done + take] = self.buf[off:off + take]
            done += take
            self.pos += take
        return out

    def next(self) -> int:
        return int(self.words(1)[0])


def philox_block(ctr, key):
    c = np.array(ctr, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    _native.lib().ora_philox4x64_10(ptr(c), ptr(k), ptr(out))
    return [int(x) for x in out]


def uniform_mod(stream: Stream, q: int, n: int) -> np.ndarray:
    """The first n words whose low bitlen(q) bits are < q, masked."""
    mask = np.uint64((1 << q.bit_length()) - 1)
    got = []
    need = n
    while need > 0:
        w = stream.words(need + need // 4 + 16) & mask
        acc = w[w < np.uint64(q)][:need]
        got.append(acc)
        need -= acc.size
    return np.concatenate(got).astype(np.uint64)


def ternary(stream: Stream, n: int) -> list:
    """The first n words below 3*floor(2^64/3), mapped by w mod 3."""
    bound = np.uint64(3 * ((1 << 64) // 3))
    got = []
    need = n
    while need > 0:
        w = stream.words(need + 16)
        acc = w[w < bound][:need]
        got.append(acc)
        need -= acc.size
    r = (np.concatenate(got) % np.uint64(3)).astype(np.int64)
    return [(0, 1, -1)[int(x)] for x in r]


@lru_cache(maxsize=None)
def gaussian_thresholds() -> tuple:
    with localcontext() as ctx:
        ctx.prec = 80
        two_s2 = 2 * SIGMA * SIGMA
        rho = [(-(Decimal(j) ** 2) / two_s2).exp() for j in range(GAUSS_BOUND + 1)]
        S = rho[0] + 2 * sum(rho[1:])
        T, acc = [], rho[0]
        scale = Decimal(2) ** 63
        for k in range(GAUSS_BOUND + 1):
            if k > 0:
                acc += 2 * rho[k]
            T.append(int((scale * acc / S).to_integral_value(rounding="ROUND_FLOOR")))
    T[GAUSS_BOUND] = 1 << 63
    return tuple(T)


def gaussian(stream: Stream, n: int) -> list:
    T = gaussian_thresholds()
    out = []
    for w in stream.words(n):
        w = int(w)
        sign = w >> 63
        u = w & ((1 << 63) - 1)
        k = 0
        while u >= T[k]:
            k += 1
        out.append(-k if sign else k)
    return out


def uniform_wide(seed, tag, a, b, q, n) -> np.ndarray:
    """n residues mod q, residue i = ((w_{2i+1} << 64) | w_{2i}) mod q over the
    stream's words (no rejection; the distance from uniform is below
    q / 2^128)."""
    w = Stream(seed, tag, a, b).words(2 * n)
    return np.array([((int(w[2 * i + 1]) << 64) | int(w[2 * i])) % q for i in range(n)], dtype=np.uint64)


def sample_uniform(seed, tag, a, b, q, n) -> np.ndarray:
    return uniform_mod(Stream(seed, tag, a, b), q, n)


def sample_ternary(seed, tag, a, b, n) -> list:
    return ternary(Stream(seed, tag, a, b), n)


def sample_gaussian(seed, tag, a, b, n) -> list:
    return gaussian(Stream(seed, tag, a, b), n)
