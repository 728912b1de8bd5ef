"""Edge cases of the CUDA path against the oracle:

* empty batches (count 0) are no-ops for every batched entry point;
* the smallest ring the library accepts (n = 16) and the largest prime
  counts (L = 12 without a special prime, L = 11 with one; k_t = 4
  plaintext moduli): encryption, rotation, ct x ct + relinearisation
  bit-exact, decryption exact;
* ragged batch sizes (7 ciphertexts) and the degenerate messages (all zero,
  all t - 1).
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import ct_stack, lib, make_ctx, need_gpu, oracle_params, torch_u64
from oracle import bfv, encoding

pytestmark = pytest.mark.gpu


def test_empty_batches_are_no_ops():
    need_gpu()
    Lb = lib()
    ps = W.params_small(256, L=3)
    ctx = make_ctx(ps)
    try:
        sk, ev = Lb.lola_keygen(ctx, 1, [1], Lb.LOLA_KEY_RELIN)
        buf = torch_u64(np.zeros((1, 2, ps.L, ps.n), np.uint64))
        Lb.lola_ntt_forward(ctx, buf, 0, ps.L)
        Lb.lola_ntt_inverse(ctx, buf, 0, ps.L)
        Lb.lola_add(ctx, buf, buf, buf, 0)
        Lb.lola_rotate(ctx, ev, buf, buf, 0, [])
        Lb.lola_rotate_hoisted(ctx, ev, buf, buf, 0, [1])
        Lb.lola_multiply(ctx, ev, buf, buf, buf, 0)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
    finally:
        Lb.lola_ctx_destroy(ctx)


def run_primitives_vs_oracle(ps, slots, steps, seed, decrypt_square=True):
    """Encrypt with the oracle's keys (same seed on both sides), rotate and
    multiply on the GPU and in the oracle, compare every word (and decrypt
    the squares unless the parameters leave them no noise budget)."""
    Lb = lib()
    P = oracle_params(ps)
    kt, n = len(ps.t), ps.n
    okeys = bfv.keygen(P, seed, rotations=[s for s in steps if s], relin=True, row_swap=0 in steps)
    ctx = make_ctx(ps)
    try:
        flags = Lb.LOLA_KEY_RELIN | (Lb.LOLA_KEY_ROW_SWAP if 0 in steps else 0)
        sk, ev = Lb.lola_keygen(ctx, seed, [s for s in steps if s], flags)
        cts = [bfv.encrypt(P, okeys.pk, encoding.encode(v, t), t, seed + 1, m * kt + ti)
               for m, v in enumerate(slots) for ti, t in enumerate(ps.t)]
        gct = Lb.lola_encrypt(ctx, sk, np.asarray(slots, np.int64), seed + 1)
        got = Lb.lola_ct_export(ctx, gct, (kt, 2, ps.L, n)).reshape(-1, 2, ps.L, n)
        for i, c in enumerate(cts):
            assert np.array_equal(got[i, 0], c.c[0]) and np.array_equal(got[i, 1], c.c[1]), ("encrypt", i)
        cnt = len(cts)
        src = Lb.lola_ct_data(gct)
        # rotations: ciphertext i by steps[i % len(steps)]
        per = [steps[i % len(steps)] for i in range(cnt)]
        dst = Lb.lola_ct_create(ctx, len(slots))
        Lb.lola_rotate(ctx, ev, src, Lb.lola_ct_data(dst), cnt, per)
        rot = Lb.lola_ct_export(ctx, dst, (kt, 2, ps.L, n)).reshape(-1, 2, ps.L, n)
        for i, c in enumerate(cts):
            ref = bfv.rotate_rows(P, okeys, c) if per[i] == 0 else bfv.rotate(P, okeys, c, per[i])
            assert np.array_equal(rot[i, 0], ref.c[0]) and np.array_equal(rot[i, 1], ref.c[1]), ("rotate", i)
        # squares with relinearisation
        sq = Lb.lola_ct_create(ctx, len(slots))
        Lb.lola_multiply(ctx, ev, src, src, Lb.lola_ct_data(sq), cnt, [i % kt for i in range(cnt)])
        got_sq = Lb.lola_ct_export(ctx, sq, (kt, 2, ps.L, n)).reshape(-1, 2, ps.L, n)
        for i in (0, cnt - 1):
            ref = bfv.relinearize(P, okeys, bfv.multiply(P, cts[i], cts[i]))
            assert np.array_equal(got_sq[i, 0], ref.c[0]) and np.array_equal(got_sq[i, 1], ref.c[1]), ("square", i)
        res = Lb.lola_decrypt_residues(ctx, sk, sq, kt, n)
        for m, v in (enumerate(slots) if decrypt_square else ()):
            for ti, t in enumerate(ps.t):
                want = (np.asarray(v, dtype=object) ** 2) % t
                assert [int(x) for x in res[m, ti]] == [int(x) for x in want], (m, ti)
        for h in (gct, dst, sq):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_smallest_ring():
    need_gpu()
    n = 16
    ps = W.ParamSet("n16", n, W.Q60[:4], 3, 1, [97])        # 97 = 1 mod 2n
    g = np.random.default_rng(1)
    slots = [g.integers(0, 97, n), np.zeros(n, np.int64), np.full(n, 96)]
    run_primitives_vs_oracle(ps, slots, [1, 3, 0], 31)


@pytest.mark.parametrize("L,K", [(12, 0), (11, 1)])
def test_largest_prime_counts_and_plaintext_moduli(L, K):
    need_gpu()
    n = 1024
    ps = W.ParamSet(f"max_L{L}_K{K}", n, W.Q60[:L + K], L, K, W.T30[:4])    # k_t = 4
    g = np.random.default_rng(L)
    slots = [g.integers(0, 1 << 20, n), np.full(n, W.T30[3] - 1)]
    run_primitives_vs_oracle(ps, slots, [5, 0], 37)


def test_ragged_batch():
    need_gpu()
    n = 4096
    ps = W.params_small(n, L=3, K=1, t=W.T30[:1])
    g = np.random.default_rng(7)
    slots = [g.integers(0, 1 << 12, n) for _ in range(7)]
    run_primitives_vs_oracle(ps, slots, [1, 2, 3, 0, 100, 2047, 5], 41)


def test_single_ciphertext_prime():
    # L = 1: the key switch's inner products live in scratch of their own
    need_gpu()
    n = 1024
    ps = W.ParamSet("L1", n, W.Q60[:2], 1, 1, [65537])
    g = np.random.default_rng(3)
    slots = [g.integers(0, 256, n), g.integers(0, 256, n)]
    run_primitives_vs_oracle(ps, slots, [1, 0], 43)


def test_hoisted_rotation_in_step_chunks():
    """150 ciphertexts x 12 steps: the inner product runs in chunks of
    floor(1024 / 150) = 6 steps; every output equals the oracle's hoisted
    rotation."""
    need_gpu()
    Lb = lib()
    n = 256
    ps = W.params_small(n, L=3, K=1, t=W.T30[:1])
    P = oracle_params(ps)
    t = ps.t[0]
    steps = list(range(1, 12)) + [0]
    okeys = bfv.keygen(P, 47, rotations=steps[:-1], relin=False, row_swap=True)
    ctx = make_ctx(ps)
    try:
        sk, ev = Lb.lola_keygen(ctx, 47, steps[:-1], Lb.LOLA_KEY_ROW_SWAP)
        count = 150
        slots = np.random.default_rng(9).integers(0, 1000, (count, n))
        ct = Lb.lola_encrypt(ctx, sk, slots, 48)
        out = Lb.lola_ct_create(ctx, count * len(steps))
        Lb.lola_rotate_hoisted(ctx, ev, Lb.lola_ct_data(ct), Lb.lola_ct_data(out), count, steps)
        got = Lb.lola_ct_export(ctx, out, (1, 2, ps.L, n)).reshape(len(steps), count, 2, ps.L, n)
        for i in (0, 77, count - 1):
            c = bfv.encrypt(P, okeys.pk, encoding.encode(slots[i], t), t, 48, i)
            refs = bfv.rotate_hoisted(P, okeys, c, steps)
            for si in (0, 5, 6, len(steps) - 1):                  # both sides of the chunk boundary
                assert np.array_equal(got[si, i, 0], refs[si].c[0]) and np.array_equal(got[si, i, 1], refs[si].c[1]), (i, si)
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
    finally:
        Lb.lola_ctx_destroy(ctx)


@pytest.mark.parametrize("L,K,alpha", [(1, 1, 1), (2, 1, 1), (5, 1, 1), (2, 2, 2), (5, 2, 2), (4, 2, 1)])
def test_key_switch_at_full_ring(L, K, alpha):
    # n = 16384 with special primes (cluster transforms): rotation and
    # relinearisation (one digit: inner products in scratch of their own;
    # two or more: in place over the digit rows); alpha = 2: digits of two
    # primes with two special primes (L = 2: one digit; L = 5: 2 + 2 + 1)
    need_gpu()
    n = 16384
    ps = W.ParamSet(f"full_ring_L{L}_K{K}_a{alpha}", n, W.Q60[:L + K], L, K, [W.T30[0]], alpha)
    g = np.random.default_rng(100 + L)
    slots = [g.integers(0, 1 << 12, n), g.integers(0, 1 << 12, n)]
    # one 60-bit prime at n = 16384 has no noise budget for a square: words only
    run_primitives_vs_oracle(ps, slots, [7, 0], 53 + L, decrypt_square=L > 1)
