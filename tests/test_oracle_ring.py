"""Pins for the oracle's ring arithmetic and sampler (CPU only).

Each test checks the oracle against something other than itself: the O(n^2)
definition of the negacyclic product, numpy's Philox, sympy's primality
test, floating-point evaluation of the Gaussian, or an algebraic identity.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import ring, sampling


@pytest.mark.parametrize("n", [2, 4, 16, 64, 256])
@pytest.mark.parametrize("q", [W.Q60[0], W.Q60[5], W.Q36[1], 65537])
def test_ntt_product_equals_schoolbook(n, q):
    if (q - 1) % (2 * n):
        pytest.skip("q not NTT friendly for n")
    g = np.random.default_rng(n * 7 + q % 1000)
    a = g.integers(0, q, n, dtype=np.uint64)
    b = g.integers(0, q, n, dtype=np.uint64)
    assert np.array_equal(ring.poly_mul(a, b, q), ring.poly_mul_schoolbook(a, b, q))


def test_schoolbook_small_by_hand():
    # (1 + x) * (1 + x) = 1 + 2x + x^2 ; with n = 2, x^2 = -1 -> 2x
    q = 17
    assert list(ring.poly_mul_schoolbook(np.array([1, 1], np.uint64), np.array([1, 1], np.uint64), q)) == [0, 2]
    # x^(n-1) * x = x^n = -1
    n = 8
    a = np.zeros(n, np.uint64); a[n - 1] = 1
    b = np.zeros(n, np.uint64); b[1] = 1
    out = ring.poly_mul_schoolbook(a, b, q)
    assert out[0] == q - 1 and not out[1:].any()


def test_ntt_product_full_size_spot_coefficients():
    n, q = 16384, W.Q60[2]
    g = np.random.default_rng(3)
    a = g.integers(0, q, n, dtype=np.uint64)
    b = g.integers(0, q, n, dtype=np.uint64)
    c = ring.poly_mul(a, b, q)
    for k in (0, 1, 777, n // 2, n - 1):
        # coefficient k straight from the definition, in Python integers
        pos = sum(int(a[i]) * int(b[k - i]) for i in range(k + 1))
        neg = sum(int(a[i]) * int(b[n + k - i]) for i in range(k + 1, n))
        assert int(c[k]) == (pos - neg) % q


@pytest.mark.parametrize("n", [8, 1024, 16384])
def test_transform_round_trip_and_points(n):
    q = W.Q60[1]
    psi = ring.smallest_primitive_2n_root(q, n)
    assert pow(psi, n, q) == q - 1
    a = np.random.default_rng(n).integers(0, q, n, dtype=np.uint64)
    A = ring.forward_transform(a, q, psi)
    assert np.array_equal(ring.inverse_transform(A, q, psi), a)
    for k in (0, 3, n - 1):
        x = pow(psi, 2 * k + 1, q)
        assert int(A[k]) == sum(int(c) * pow(x, i, q) for i, c in enumerate(a)) % q


def test_smallest_root_is_smallest():
    for q, n in ((65537, 8), (257, 16), (W.T30[0], 16384), (W.T30[1], 16384)):
        psi = ring.smallest_primitive_2n_root(q, n)
        assert pow(psi, n, q) == q - 1        # primitive: psi^n = -1
        assert not any(pow(x, n, q) == q - 1 for x in range(2, psi))


def test_automorphism_is_ring_homomorphism():
    n, q = 64, W.Q60[0]
    g = np.random.default_rng(5)
    a = g.integers(0, q, n, dtype=np.uint64)
    b = g.integers(0, q, n, dtype=np.uint64)
    for gal in (3, 5, 2 * n - 1, pow(3, 7, 2 * n)):
        lhs = ring.automorphism(ring.poly_mul(a, b, q), gal, q)
        rhs = ring.poly_mul(ring.automorphism(a, gal, q), ring.automorphism(b, gal, q), q)
        assert np.array_equal(lhs, rhs)
    # tau_g o tau_h = tau_{gh}
    g1, g2 = 3, 2 * n - 1
    assert np.array_equal(ring.automorphism(ring.automorphism(a, g1, q), g2, q),
                          ring.automorphism(a, g1 * g2 % (2 * n), q))


def test_crt_lift_round_trip():
    primes = W.Q60[:4]
    basis = ring.Basis(primes)
    vals = [0, 1, -1, basis.M // 2, -(basis.M // 2), 123456789 ** 7]
    res = basis.reduce(vals)
    lifted = basis.lift_centered(res)
    assert lifted == vals


# ------------------------------------------------------------------ sampling

def test_philox_matches_numpy():
    # numpy's Philox is Philox4x64-10; it pre-increments its counter, so its
    # first block is the generator at counter (1, 0, 0, 0).
    for key in ((0, 0), (20181225, 0), (2**64 - 1, 12345)):
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.zeros(4, dtype=np.uint64))
        ref = [int(x) for x in bg.random_raw(12)]
        ours = []
        for blk in (1, 2, 3):
            ours += sampling.philox_block((blk, 0, 0, 0), key)
        assert ours == ref


def test_philox_known_answer_zero():
    # Random123's published answer for counter = key = 0
    assert sampling.philox_block((0, 0, 0, 0), (0, 0)) == [
        0x16554D9ECA36314C, 0xDB20FE9D672D0FDC, 0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]


def test_stream_layout():
    s = sampling.Stream(99, 4, 5, 6)
    w = s.words(10)
    blocks = sampling.philox_block((0, 4, 5, 6), (99, 0)) + sampling.philox_block((1, 4, 5, 6), (99, 0)) \
        + sampling.philox_block((2, 4, 5, 6), (99, 0))
    assert [int(x) for x in w] == blocks[:10]


def test_uniform_rejection_definition():
    q = 1000003
    vals = sampling.sample_uniform(1, 2, 3, 4, q, 500)
    # redo the definition word by word in Python
    words = [int(x) for x in sampling.Stream(1, 2, 3, 4).words(5000)]
    mask = (1 << q.bit_length()) - 1
    ref = [w & mask for w in words if (w & mask) < q][:500]
    assert [int(v) for v in vals] == ref
    assert vals.max() < q


def test_ternary_distribution():
    v = np.array(sampling.sample_ternary(5, 1, 0, 0, 30000))
    assert set(np.unique(v)) == {-1, 0, 1}
    for x in (-1, 0, 1):
        assert abs((v == x).mean() - 1 / 3) < 0.02


def test_gaussian_thresholds_vs_float():
    T = sampling.gaussian_thresholds()
    sigma = 3.2
    rho = [math.exp(-k * k / (2 * sigma * sigma)) for k in range(20)]
    S = rho[0] + 2 * sum(rho[1:])
    acc = 0.0
    for k in range(20):
        acc += rho[k] if k == 0 else 2 * rho[k]
        assert abs(T[k] / 2**63 - acc / S) < 1e-12
    assert list(T) == sorted(T) and T[-1] == 2**63


def test_gaussian_moments():
    v = np.array(sampling.sample_gaussian(11, 3, 0, 0, 200000), dtype=np.float64)
    assert abs(v.mean()) < 0.05
    assert abs(v.var() - 3.2 ** 2) < 0.15
    assert np.abs(v).max() <= 19


# ---------------------------------------------------------------- parameters

def test_parameter_primes():
    sympy = pytest.importorskip("sympy")
    for p in W.Q60 + W.Q36 + W.T30:
        assert sympy.isprime(p) and ring.is_prime(p)
    assert all(p % (1 << 15) == 1 and p < 2**60 for p in W.Q60)
    assert all(p % (1 << 13) == 1 and p < 2**36 for p in W.Q36)
    assert all(p % (1 << 15) == 1 and p < 2**30 for p in W.T30)
    assert W.Q60 == sorted(W.Q60, reverse=True) and len(set(W.Q60)) == len(W.Q60)


def test_parameter_security_budgets():
    # 128-bit security caps (homomorphic encryption standard, cited by the
    # paper's Sec. 3.1 footnote): log2(QP) <= 109 at n=4096, <= 438 at n=16384
    p1 = W.params_dense64()
    assert sum(math.log2(q) for q in p1.q) <= 109
    p2 = W.params_mnist()
    assert sum(math.log2(q) for q in p2.q) <= 438


def test_paper_plaintext_primes():
    import json, os
    from conftest import GOLDEN
    g = json.load(open(os.path.join(GOLDEN, "plaintext_primes.json")))
    for f in g["factors"]:
        assert ring.is_prime(f) and f % (2 * g["n"]) == 1
