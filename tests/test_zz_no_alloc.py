"""The allocation-free rotation entry point (lola_rotate_noalloc).

It exists for callers that cannot allocate device memory (an application
memory manager that owns the device and forbids cudaMalloc after start-up,
a host that budgets device memory up front, a latency-critical loop that
cannot afford an allocation).  This test calls it through the
C-ABI twice in a row and checks each result against the ordinary
lola_rotate entry point (which allocates its scratch): rotations are exact
integer arithmetic, so the tolerance is zero.  It also checks the size
limit of the static scratch area at its exact boundary.  The file name makes pytest collect it
last.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import lib, make_ctx, need_gpu

pytestmark = pytest.mark.gpu


def test_rotate_noalloc_matches_rotate_twice():
    need_gpu()
    Lb = lib()
    ps = W.params_mnist()            # n = 16384, L = 5, K = 1, three plaintext moduli
    n, kt = ps.n, len(ps.t)
    # scratch per ciphertext: digits, raised digits, special-prime limbs
    digits = (ps.L + ps.alpha - 1) // ps.alpha
    per_ct = (ps.L + digits * (ps.L + ps.K) + 2 * ps.K) * n * 8
    count = Lb.NOALLOC_SCRATCH_BYTES // per_ct          # the largest count that fits
    msgs = (count + kt - 1) // kt
    ctx = make_ctx(ps)
    try:
        sk, ev = Lb.lola_keygen(ctx, 31, [1, 169], Lb.LOLA_KEY_RELIN)
        slots = np.random.default_rng(3).integers(0, 16, (msgs, n))
        ct = Lb.lola_encrypt(ctx, sk, slots, 5)
        ref = Lb.lola_ct_create(ctx, msgs)
        got = Lb.lola_ct_create(ctx, msgs)
        try:
            for step in (1, 169):                                # two calls in a row
                Lb.lola_rotate(ctx, ev, Lb.lola_ct_data(ct), Lb.lola_ct_data(ref), count, [step] * count)
                Lb.lola_rotate_noalloc(ctx, ev, Lb.lola_ct_data(ct), Lb.lola_ct_data(got), count, step)
                a = Lb.lola_ct_export(ctx, ref, (kt, 2, ps.L, n)).reshape(msgs * kt, 2, ps.L, n)[:count]
                b = Lb.lola_ct_export(ctx, got, (kt, 2, ps.L, n)).reshape(msgs * kt, 2, ps.L, n)[:count]
                assert np.array_equal(a, b), step
                res = Lb.lola_decrypt_residues(ctx, sk, got, kt, n).reshape(msgs * kt, n)
                h = n // 2
                for c_ in range(count):
                    m, ti = divmod(c_, kt)
                    want = np.concatenate([np.roll(slots[m, :h], step), np.roll(slots[m, h:], step)])
                    assert np.array_equal(res[c_], want % ps.t[ti])
            # one ciphertext more than fits is refused, not truncated
            big = (count + 1 + kt - 1) // kt
            big_in = Lb.lola_ct_create(ctx, big)
            big_out = Lb.lola_ct_create(ctx, big)
            try:
                with pytest.raises(Lb.LolaError) as ei:
                    Lb.lola_rotate_noalloc(ctx, ev, Lb.lola_ct_data(big_in), Lb.lola_ct_data(big_out), count + 1, 1)
                assert ei.value.code == -1
            finally:
                Lb.lola_ct_destroy(big_in)
                Lb.lola_ct_destroy(big_out)
        finally:
            for h_ in (ct, ref, got):
                Lb.lola_ct_destroy(h_)
            Lb.lola_keys_destroy(sk)
            Lb.lola_keys_destroy(ev)
    finally:
        Lb.lola_ctx_destroy(ctx)
