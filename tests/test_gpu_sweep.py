"""Batched primitive sweep (n in {8192, 16384}, 4..8 ciphertext primes of 60
bits plus a special prime, uniform random residues): one launch carries many
ciphertexts.  NTT/INTT round trip of the whole batch; rotations by random
steps in [1, n/2) drawn per ciphertext (one Galois key per distinct step) and
ct x ct + relinearisation, both compared bit-exactly with the oracle on
sampled ciphertexts of the batch."""
import numpy as np
import pytest

import workloads as W
from gpu_util import host_u64, lib, make_ctx, need_gpu, oracle_params, torch_u64
from oracle import bfv, ring

pytestmark = pytest.mark.gpu


def brev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2)


@pytest.mark.parametrize("n,L,B", [(8192, 4, 64), (8192, 8, 16), (16384, 4, 32), (16384, 8, 8)])
def test_sweep_primitives(n, L, B):
    need_gpu()
    Lb = lib()
    ps = W.params_sweep(n, L)
    P = oracle_params(ps)
    ctx = make_ctx(ps)
    try:
        seed = 1000 + n + L
        cts = W.random_residues(seed, (B, 2), ps.q[:L], n)            # [B][2][L][n] coefficient form
        # --- NTT / INTT of the whole batch, spot-checked against the oracle transform
        d = torch_u64(cts)
        Lb.lola_ntt_forward(ctx, d, B * 2, L)
        fwd = host_u64(d).reshape(cts.shape)
        perm = np.array([brev(k, n.bit_length() - 1) for k in range(n)])
        for b, c, j in ((0, 0, 0), (B - 1, 1, L - 1)):
            q = ps.q[j]
            ref = ring.forward_transform(cts[b, c, j], q, ring.smallest_primitive_2n_root(q, n))
            assert np.array_equal(fwd[b, c, j], ref[perm])
        Lb.lola_ntt_inverse(ctx, d, B * 2, L)
        assert np.array_equal(host_u64(d).reshape(cts.shape), cts)
        # --- rotations by random steps, one launch
        steps = [int(s) for s in W.rotation_steps(seed, B, n)]
        sk, ev = Lb.lola_keygen(ctx, seed, sorted(set(steps)), Lb.LOLA_KEY_RELIN)
        src = Lb.lola_ct_import(ctx, cts[:, None])                    # k_t = 1
        dst = Lb.lola_ct_create(ctx, B)
        Lb.lola_rotate(ctx, ev, Lb.lola_ct_data(src), Lb.lola_ct_data(dst), B, steps)
        got = Lb.lola_ct_export(ctx, dst, (1, 2, L, n))[:, 0]
        sample = [0, B // 2, B - 1]
        okeys = bfv.keygen(P, seed, rotations=sorted(set(steps[i] for i in sample)), relin=True)
        for i in sample:
            ref = bfv.rotate(P, okeys, bfv.Ciphertext([cts[i, 0], cts[i, 1]], ps.t[0]), steps[i])
            assert np.array_equal(got[i, 0], ref.c[0]) and np.array_equal(got[i, 1], ref.c[1]), (i, steps[i])
        # --- ct x ct + relinearisation, pairs (i, i+1), one launch
        half = B // 2
        a = Lb.lola_ct_import(ctx, cts[:half, None])
        b2 = Lb.lola_ct_import(ctx, cts[half:2 * half, None])
        out = Lb.lola_ct_create(ctx, half)
        Lb.lola_multiply(ctx, ev, Lb.lola_ct_data(a), Lb.lola_ct_data(b2), Lb.lola_ct_data(out), half)
        gm = Lb.lola_ct_export(ctx, out, (1, 2, L, n))[:, 0]
        for i in (0, half - 1):
            x = bfv.Ciphertext([cts[i, 0], cts[i, 1]], ps.t[0])
            y = bfv.Ciphertext([cts[half + i, 0], cts[half + i, 1]], ps.t[0])
            ref = bfv.relinearize(P, okeys, bfv.multiply(P, x, y))
            assert np.array_equal(gm[i, 0], ref.c[0]) and np.array_equal(gm[i, 1], ref.c[1]), i
        for h in (src, dst, a, b2, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
    finally:
        Lb.lola_ctx_destroy(ctx)
