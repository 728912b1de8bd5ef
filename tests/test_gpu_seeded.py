"""Seeded symmetric encryption on the GPU against the oracle's definition:
lola_encrypt_symmetric's ciphertexts equal oracle bfv.encrypt_symmetric word
for word (n = 1024 and the MNIST parameters at n = 16384, several CRT
residues, so the ciphertext ids message * k_t + residue are exercised), and
lola_ct_upload_seeded rebuilds the same ciphertexts from their c0 halves
and the seed; the result decrypts and evaluates like a public-key one."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import lib, make_ctx, need_gpu, oracle_params
from oracle import bfv, encoding

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,L,kt", [(1024, 3, 1), (1024, 2, 3), (16384, 5, 3)])
def test_symmetric_encryption_matches_oracle_and_seeded_upload(n, L, kt):
    need_gpu()
    Lb = lib()
    ps = W.params_mnist(L) if n == 16384 else W.params_small(n, L=L, K=1, t=W.T30[:kt])
    P = oracle_params(ps)
    ctx = make_ctx(ps)
    try:
        sk, ev = Lb.lola_keygen(ctx, 51, [3], Lb.LOLA_KEY_RELIN)
        msgs = 2
        slots = np.random.default_rng(n + L).integers(0, 1 << 20, (msgs, n))
        seed = 77
        ct = Lb.lola_encrypt_symmetric(ctx, sk, slots, seed)
        got = Lb.lola_ct_export(ctx, ct, (kt, 2, L, n))
        ok = bfv.keygen(P, 51)
        for m in range(msgs):
            for ti in ([0, kt - 1] if n == 16384 else range(kt)):
                t = ps.t[ti]
                o = bfv.encrypt_symmetric(P, ok.sk, encoding.encode(slots[m] % t, t), t, seed, m * kt + ti)
                assert np.array_equal(got[m, ti, 0], o.c[0]) and np.array_equal(got[m, ti, 1], o.c[1]), (m, ti)
        # device layout: c0 halves to the host, then rebuilt by the seeded upload
        words = msgs * kt * 2 * L * n
        full = torch.empty(words, dtype=torch.int64, pin_memory=True)
        Lb.lola_ct_download(ctx, ct, full.data_ptr())
        torch.cuda.synchronize()
        c0 = full.view(msgs * kt, 2, L * n)[:, 0].contiguous().pin_memory()
        ct2 = Lb.lola_ct_create(ctx, msgs)
        Lb.lola_ct_upload_seeded(ctx, ct2, c0.data_ptr(), seed)
        torch.cuda.synchronize()
        assert np.array_equal(Lb.lola_ct_export(ctx, ct2, (kt, 2, L, n)), got)
        dec = Lb.lola_decrypt_residues(ctx, sk, ct2, kt, n)
        for ti in range(kt):
            assert np.array_equal(dec[:, ti], slots % ps.t[ti])
        # a rotation of the rebuilt ciphertext decrypts to the shifted slots
        out = Lb.lola_ct_create(ctx, msgs)
        Lb.lola_rotate(ctx, ev, Lb.lola_ct_data(ct2), Lb.lola_ct_data(out), msgs * kt, [3] * (msgs * kt))
        dec = Lb.lola_decrypt_residues(ctx, sk, out, kt, n)
        h = n // 2
        for m in range(msgs):
            want = np.concatenate([np.roll(slots[m, :h], 3), np.roll(slots[m, h:], 3)])
            for ti in range(kt):
                assert np.array_equal(dec[m, ti], want % ps.t[ti])
        # evaluation keys alone cannot encrypt symmetrically
        with pytest.raises(Lb.LolaError):
            Lb.lola_encrypt_symmetric(ctx, ev, slots, seed)
        for hnd in (ct, ct2, out):
            Lb.lola_ct_destroy(hnd)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
    finally:
        Lb.lola_ctx_destroy(ctx)
