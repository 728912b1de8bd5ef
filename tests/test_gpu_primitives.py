"""GPU parity of the BFV primitives against the CPU oracle, bit-exact.

Every ciphertext the CUDA path produces is exported in coefficient form and
compared word for word with the oracle's result on the same inputs and keys
(both sides derive keys and encryption randomness from the same seeds with
their own implementations of the same sampler definition).
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import ct_from_arrays, ct_stack, host_u64, lib, make_ctx, need_gpu, oracle_params, torch_u64
from oracle import bfv, encoding, ring

pytestmark = pytest.mark.gpu


def brev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


@pytest.mark.parametrize("n,L", [(16, 2), (32, 3), (256, 3), (1024, 4), (4096, 3), (8192, 4), (16384, 6)])
def test_ntt_matches_oracle_transform(n, L):
    need_gpu()
    Lb = lib()
    ps = W.params_small(n, L=L - 1, K=1)
    ctx = make_ctx(ps)
    try:
        polys = 3
        host = W.random_residues(n * 31 + L, (polys,), ps.q[:L], n)      # [polys][L][n]
        d = torch_u64(host)
        Lb.lola_ntt_forward(ctx, d, polys, L)
        fwd = host_u64(d).reshape(host.shape)
        logn = n.bit_length() - 1
        perm = np.array([brev(k, logn) for k in range(n)])
        for p in range(polys):
            for j in range(L):
                q = ps.q[j]
                ref = ring.forward_transform(host[p, j], q, ring.smallest_primitive_2n_root(q, n))
                assert np.array_equal(fwd[p, j], ref[perm]), (p, j)
        Lb.lola_ntt_inverse(ctx, d, polys, L)
        assert np.array_equal(host_u64(d).reshape(host.shape), host)
    finally:
        Lb.lola_ctx_destroy(ctx)


# K1 / K0: one digit per prime with one / no special prime; K2a2: digits of
# two primes (the last single for odd L) with two special primes; K2a1: one
# digit per prime with two special primes
@pytest.fixture(scope="module", params=[("K1", 32, 3, 1, 1), ("K0", 32, 3, 0, 1), ("K1big", 1024, 4, 1, 1),
                                        ("K2a2", 32, 5, 2, 2), ("K2a2big", 1024, 4, 2, 2), ("K2a1", 32, 3, 2, 1)])
def setup(request):
    need_gpu()
    _, n, L, K, alpha = request.param
    ps = W.params_small(n, L=L, K=K, t=[65537, W.T30[0]], alpha=alpha)
    P = oracle_params(ps)
    steps = [1, 3, n // 4]
    seed = 4242
    okeys = bfv.keygen(P, seed, rotations=steps, relin=True, row_swap=True)
    Lb = lib()
    ctx = make_ctx(ps)
    sk, ev = Lb.lola_keygen(ctx, seed, steps, Lb.LOLA_KEY_RELIN | Lb.LOLA_KEY_ROW_SWAP)
    yield dict(ps=ps, P=P, okeys=okeys, ctx=ctx, sk=sk, ev=ev, steps=steps, L=Lb)
    Lb.lola_keys_destroy(sk)
    Lb.lola_keys_destroy(ev)
    Lb.lola_ctx_destroy(ctx)


def test_keys_match_oracle(setup):
    S = setup
    Lb, ctx, sk, ok, P = S["L"], S["ctx"], S["sk"], S["okeys"], S["P"]
    s = Lb.lola_keys_export(ctx, sk, 0).view(np.int64)
    assert list(s) == list(ok.sk.s)
    pk = Lb.lola_keys_export(ctx, sk, 1).reshape(2, P.L, P.n)
    assert np.array_equal(pk[0], ok.pk.p0) and np.array_equal(pk[1], ok.pk.p1)
    D = len(P.groups)
    rk = Lb.lola_keys_export(ctx, sk, 2).reshape(2, D, P.L + P.K, P.n)
    assert np.array_equal(rk[0], ok.relin.b) and np.array_equal(rk[1], ok.relin.a)
    for step in S["steps"] + [0]:
        g = bfv.galois_row_swap(P.n) if step == 0 else bfv.galois_for_rotation(P.n, step)
        gk = Lb.lola_keys_export(ctx, sk, 3, step).reshape(2, D, P.L + P.K, P.n)
        assert np.array_equal(gk[0], ok.galois[g].b) and np.array_equal(gk[1], ok.galois[g].a), step
    # the evaluation-only handle holds no secret or public key
    with pytest.raises(Lb.LolaError):
        Lb.lola_keys_export(ctx, S["ev"], 0)


def oracle_encrypt_all(S, slots, seed):
    P, ok = S["P"], S["okeys"]
    kt = len(P.t)
    cts = []
    for m, v in enumerate(slots):
        for ti, t in enumerate(P.t):
            cts.append(bfv.encrypt(P, ok.pk, encoding.encode(v, t), t, seed, m * kt + ti))
    return cts


def test_encrypt_and_decrypt_match_oracle(setup):
    S = setup
    Lb, ctx, sk, P = S["L"], S["ctx"], S["sk"], S["P"]
    kt, n = len(P.t), P.n
    slots = np.random.default_rng(1).integers(-3000, 3000, (3, n))
    ct = Lb.lola_encrypt(ctx, sk, slots, 77)
    try:
        got = Lb.lola_ct_export(ctx, ct, (kt, 2, P.L, n))
        ref = ct_stack(oracle_encrypt_all(S, slots, 77), kt)
        assert np.array_equal(got, ref)
        res = Lb.lola_decrypt_residues(ctx, sk, ct, kt, n)
        for m in range(3):
            for ti, t in enumerate(P.t):
                assert np.array_equal(res[m, ti], slots[m] % t)
        dec = Lb.lola_decrypt(ctx, sk, ct, n)
        assert np.array_equal(dec.astype(np.int64), slots)
    finally:
        Lb.lola_ct_destroy(ct)


def test_decrypt_oracle_ciphertext_after_square(setup):
    S = setup
    Lb, ctx, sk, P, ok = S["L"], S["ctx"], S["sk"], S["P"], S["okeys"]
    kt, n = len(P.t), P.n
    slots = np.random.default_rng(2).integers(0, 100, (1, n))
    cts = [bfv.square(P, ok, c) for c in oracle_encrypt_all(S, slots, 5)]
    ct = Lb.lola_ct_import(ctx, ct_stack(cts, kt))
    try:
        res = Lb.lola_decrypt_residues(ctx, sk, ct, kt, n)
        for ti, (c, t) in enumerate(zip(cts, P.t)):
            assert np.array_equal(res[0, ti], encoding.decode(bfv.decrypt(P, ok.sk, c), t))
    finally:
        Lb.lola_ct_destroy(ct)


def test_rotation_matches_oracle(setup):
    S = setup
    Lb, ctx, ev, P, ok = S["L"], S["ctx"], S["ev"], S["P"], S["okeys"]
    kt, n = len(P.t), P.n
    steps_per_ct = S["steps"] + [0]
    slots = np.random.default_rng(3).integers(0, 1000, (len(steps_per_ct), n))
    cts = oracle_encrypt_all(S, slots, 9)
    src = Lb.lola_ct_import(ctx, ct_stack(cts, kt))
    dst = Lb.lola_ct_create(ctx, len(steps_per_ct))
    try:
        per_ct = [s for s in steps_per_ct for _ in range(kt)]
        Lb.lola_rotate(ctx, ev, Lb.lola_ct_data(src), Lb.lola_ct_data(dst), len(per_ct), per_ct)
        got = Lb.lola_ct_export(ctx, dst, (kt, 2, P.L, n)).reshape(-1, 2, P.L, n)
        for i, (c, s) in enumerate(zip(cts, per_ct)):
            ref = bfv.rotate_rows(P, ok, c) if s == 0 else bfv.rotate(P, ok, c, s)
            assert np.array_equal(got[i, 0], ref.c[0]) and np.array_equal(got[i, 1], ref.c[1]), (i, s)
    finally:
        Lb.lola_ct_destroy(src)
        Lb.lola_ct_destroy(dst)


def test_hoisted_rotations_match_oracle(setup):
    """Every ciphertext rotated by several steps with one shared
    decomposition: bit-exact against the oracle's hoisted rotation, and
    decrypting to the rotated slots."""
    S = setup
    Lb, ctx, ev, sk, P, ok = S["L"], S["ctx"], S["ev"], S["sk"], S["P"], S["okeys"]
    kt, n = len(P.t), P.n
    steps = S["steps"][:3] + [0]
    slots = np.random.default_rng(13).integers(0, 1000, (2, n))
    cts = oracle_encrypt_all(S, slots, 14)                       # 2 messages x kt residues
    src = Lb.lola_ct_import(ctx, ct_stack(cts, kt))
    dst = Lb.lola_ct_create(ctx, 2 * len(steps))
    try:
        cnt = 2 * kt
        Lb.lola_rotate_hoisted(ctx, ev, Lb.lola_ct_data(src), Lb.lola_ct_data(dst), cnt, steps)
        got = Lb.lola_ct_export(ctx, dst, (kt, 2, P.L, n)).reshape(len(steps), cnt, 2, P.L, n)
        for i, c in enumerate(cts):
            refs = bfv.rotate_hoisted(P, ok, c, steps)
            for si, ref in enumerate(refs):
                assert np.array_equal(got[si, i, 0], ref.c[0]) and np.array_equal(got[si, i, 1], ref.c[1]), (i, si)
        h = n // 2
        dec = Lb.lola_decrypt_residues(ctx, sk, dst, kt, n)
        for si, k in enumerate(steps):
            for m in range(2):
                v = slots[m] % P.t[0]
                want = np.concatenate([v[h:], v[:h]]) if k == 0 else \
                    np.concatenate([np.roll(v[:h], k), np.roll(v[h:], k)])
                assert np.array_equal(dec[si * 2 + m, 0], want), (si, m)
    finally:
        Lb.lola_ct_destroy(src)
        Lb.lola_ct_destroy(dst)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_rotate_sum_matches_oracle(setup, which):
    """x plus its rotations by several steps in one key switch (one raising,
    one inner product over every step's key, one mod-down): bit-exact against
    the oracle's rotate_sum_hoisted, and decrypting to the summed slots."""
    S = setup
    Lb, ctx, ev, sk, P, ok = S["L"], S["ctx"], S["ev"], S["sk"], S["P"], S["okeys"]
    kt, n = len(P.t), P.n
    steps = [[1], [1, 3], [3, 0, n // 4, 1, 1]][which]
    slots = np.random.default_rng(17 + which).integers(0, 1000, (3, n))
    cts = oracle_encrypt_all(S, slots, 18)                       # 3 messages x kt residues
    src = Lb.lola_ct_import(ctx, ct_stack(cts, kt))
    dst = Lb.lola_ct_create(ctx, 3)
    try:
        Lb.lola_rotate_sum(ctx, ev, Lb.lola_ct_data(src), Lb.lola_ct_data(dst), 3 * kt, steps)
        got = Lb.lola_ct_export(ctx, dst, (kt, 2, P.L, n)).reshape(-1, 2, P.L, n)
        for i, c in enumerate(cts):
            ref = bfv.rotate_sum_hoisted(P, ok, c, steps)
            assert np.array_equal(got[i, 0], ref.c[0]) and np.array_equal(got[i, 1], ref.c[1]), i
        h = n // 2
        dec = Lb.lola_decrypt_residues(ctx, sk, dst, kt, n)
        for m in range(3):
            for ti, t in enumerate(P.t):
                v = slots[m] % t
                want = v.copy()
                for k in steps:
                    want = want + (np.concatenate([v[h:], v[:h]]) if k == 0 else
                                   np.concatenate([np.roll(v[:h], k), np.roll(v[h:], k)]))
                assert np.array_equal(dec[m, ti], want % t), (m, ti)
    finally:
        Lb.lola_ct_destroy(src)
        Lb.lola_ct_destroy(dst)


def test_rotate_sum_rejects_overlap_and_missing_keys(setup):
    S = setup
    Lb, ctx, ev = S["L"], S["ctx"], S["ev"]
    src = Lb.lola_ct_create(ctx, 1)
    dst = Lb.lola_ct_create(ctx, 1)
    try:
        with pytest.raises(Lb.LolaError) as ei:
            Lb.lola_rotate_sum(ctx, ev, Lb.lola_ct_data(src), Lb.lola_ct_data(dst), 1, [1, 2])
        assert ei.value.code == -3
        with pytest.raises(Lb.LolaError) as ei:
            Lb.lola_rotate_sum(ctx, ev, Lb.lola_ct_data(src), Lb.lola_ct_data(src), 1, [1])
        assert ei.value.code == -1
    finally:
        Lb.lola_ct_destroy(src)
        Lb.lola_ct_destroy(dst)


def test_rotation_missing_key_is_an_error(setup):
    S = setup
    Lb, ctx, ev = S["L"], S["ctx"], S["ev"]
    src = Lb.lola_ct_create(ctx, 1)
    dst = Lb.lola_ct_create(ctx, 1)
    try:
        with pytest.raises(Lb.LolaError) as ei:
            Lb.lola_rotate(ctx, ev, Lb.lola_ct_data(src), Lb.lola_ct_data(dst), 1, [2])
        assert ei.value.code == -3
    finally:
        Lb.lola_ct_destroy(src)
        Lb.lola_ct_destroy(dst)


@pytest.mark.parametrize("square", [True, False])
def test_multiply_relin_matches_oracle(setup, square):
    S = setup
    Lb, ctx, ev, P, ok = S["L"], S["ctx"], S["ev"], S["P"], S["okeys"]
    kt, n = len(P.t), P.n
    rng = np.random.default_rng(4 + square)
    a = rng.integers(0, 200, (2, n))
    b = rng.integers(0, 200, (2, n))
    ca, cb = oracle_encrypt_all(S, a, 11), oracle_encrypt_all(S, b, 12)
    A = Lb.lola_ct_import(ctx, ct_stack(ca, kt))
    Bc = A if square else Lb.lola_ct_import(ctx, ct_stack(cb, kt))
    out = Lb.lola_ct_create(ctx, 2)
    try:
        tidx = [i % kt for i in range(2 * kt)]
        Lb.lola_multiply(ctx, ev, Lb.lola_ct_data(A), Lb.lola_ct_data(Bc), Lb.lola_ct_data(out), 2 * kt, tidx)
        got = Lb.lola_ct_export(ctx, out, (kt, 2, P.L, n)).reshape(-1, 2, P.L, n)
        for i in range(2 * kt):
            x = ca[i]
            y = ca[i] if square else cb[i]
            ref = bfv.relinearize(P, ok, bfv.multiply(P, x, y))
            assert np.array_equal(got[i, 0], ref.c[0]) and np.array_equal(got[i, 1], ref.c[1]), i
    finally:
        Lb.lola_ct_destroy(A)
        if not square:
            Lb.lola_ct_destroy(Bc)
        Lb.lola_ct_destroy(out)


def test_mul_plain_and_add_match_oracle(setup):
    S = setup
    Lb, ctx, P = S["L"], S["ctx"], S["P"]
    kt, n = len(P.t), P.n
    rng = np.random.default_rng(6)
    a = rng.integers(0, 50, (1, n))
    w = rng.integers(-3, 4, (kt, n))
    ca = oracle_encrypt_all(S, a, 13)
    A = Lb.lola_ct_import(ctx, ct_stack(ca, kt))
    out = Lb.lola_ct_create(ctx, 1)
    out2 = Lb.lola_ct_create(ctx, 1)
    try:
        Lb.lola_mul_plain(ctx, Lb.lola_ct_data(A), w, Lb.lola_ct_data(out), kt, list(range(kt)))
        got = Lb.lola_ct_export(ctx, out, (kt, 2, P.L, n)).reshape(-1, 2, P.L, n)
        for i, t in enumerate(P.t):
            ref = bfv.mul_plain(P, ca[i], encoding.encode(w[i], t))
            assert np.array_equal(got[i, 0], ref.c[0]) and np.array_equal(got[i, 1], ref.c[1])
        Lb.lola_add(ctx, Lb.lola_ct_data(A), Lb.lola_ct_data(out), Lb.lola_ct_data(out2), kt)
        got2 = Lb.lola_ct_export(ctx, out2, (kt, 2, P.L, n)).reshape(-1, 2, P.L, n)
        for i, t in enumerate(P.t):
            ref = bfv.add(P, ca[i], bfv.mul_plain(P, ca[i], encoding.encode(w[i], t)))
            assert np.array_equal(got2[i, 0], ref.c[0]) and np.array_equal(got2[i, 1], ref.c[1])
    finally:
        for h in (A, out, out2):
            Lb.lola_ct_destroy(h)


def test_adversarial_lifts_near_half_q(setup):
    """ct x ct on ciphertexts whose coefficients sit at +-(Q-1)/2 and 0, the
    edges of the centered lift; compared with the oracle's bignum definition."""
    S = setup
    Lb, ctx, ev, P, ok = S["L"], S["ctx"], S["ev"], S["P"], S["okeys"]
    kt, n = len(P.t), P.n
    Q = P.Q
    vals = [0, 1, Q - 1, (Q - 1) // 2, (Q + 1) // 2, (Q - 3) // 2]
    rng = np.random.default_rng(7)
    cts = []
    for m in range(kt):
        polys = []
        for _ in range(2):
            ints = [vals[i] for i in rng.integers(0, len(vals), n)]
            polys.append(P.qbasis.reduce(ints))
        cts.append(bfv.Ciphertext(polys, P.t[m % kt]))
    A = Lb.lola_ct_import(ctx, ct_stack(cts, kt))
    out = Lb.lola_ct_create(ctx, 1)
    try:
        Lb.lola_multiply(ctx, ev, Lb.lola_ct_data(A), Lb.lola_ct_data(A), Lb.lola_ct_data(out), kt, list(range(kt)))
        got = Lb.lola_ct_export(ctx, out, (kt, 2, P.L, n)).reshape(-1, 2, P.L, n)
        for i in range(kt):
            ref = bfv.relinearize(P, ok, bfv.multiply(P, cts[i], cts[i]))
            assert np.array_equal(got[i, 0], ref.c[0]) and np.array_equal(got[i, 1], ref.c[1])
    finally:
        Lb.lola_ct_destroy(A)
        Lb.lola_ct_destroy(out)


@pytest.mark.parametrize("n,L,levels", [(32, 3, [(3, 2), (3, 1), (2, 1)]), (1024, 5, [(5, 4), (5, 2), (4, 2)]),
                                        (16384, 5, [(5, 4), (5, 2)])])
def test_mod_switch_matches_oracle(n, L, levels):
    """Modulus switching of random ciphertexts (uniform residues, so the
    centered residues of the dropped primes take both signs) and of
    encryptions: every word equal to the oracle's, the encryptions still
    decrypting to their slots at the lower level."""
    need_gpu()
    Lb = lib()
    ps = W.params_small(n, L=L, K=1, t=[W.T30[0]])
    P = oracle_params(ps)
    t = ps.t[0]
    ctx = make_ctx(ps)
    sk, _ = Lb.lola_keygen(ctx, 77, [], 0)
    okeys = bfv.keygen(P, 77, rotations=[], relin=False)
    try:
        cnt = 3
        host = W.random_residues(n + L, (cnt, 2), ps.q[:L], n)                # coefficient form
        slots = np.random.default_rng(n).integers(0, 1 << 20, (2, n))
        encs = [bfv.encrypt(P, okeys.pk, encoding.encode(v, t), t, 5, i) for i, v in enumerate(slots)]
        arr = np.concatenate([host, ct_stack(encs)[:, 0]])                    # [cnt + 2][2][L][n]
        src = Lb.lola_ct_import(ctx, arr[:, None])
        for L1, L2 in levels:
            if L1 < L:      # start from the oracle's level-L1 ciphertexts, in NTT form
                start = [bfv.mod_switch_to(P, bfv.Ciphertext([a[0], a[1]], t), L1) for a in arr]
                base = torch_u64(np.stack([np.stack(c.c) for c in start]))
                Lb.lola_ntt_forward(ctx, base, len(arr) * 2, L1)
            else:
                base = Lb.lola_ct_data(src)
            out = torch_u64(np.zeros((len(arr), 2, L2, n), np.uint64))
            Lb.lola_mod_switch(ctx, base, out, len(arr), L1, L2)
            Lb.lola_ntt_inverse(ctx, out, len(arr) * 2, L2)
            got = host_u64(out).reshape(len(arr), 2, L2, n)
            P1 = bfv.params_at_level(P, L1)
            for i, a in enumerate(arr):
                c = bfv.Ciphertext([a[0], a[1]], t)
                if L1 < L:
                    c = bfv.mod_switch_to(P, c, L1)
                ref = bfv.mod_switch_to(P1, c, L2)
                assert np.array_equal(got[i, 0], ref.c[0]) and np.array_equal(got[i, 1], ref.c[1]), (L1, L2, i)
            # the encryptions decrypt at level L2 (device layout, NTT form)
            Lb.lola_ntt_forward(ctx, out, len(arr) * 2, L2)
            res = Lb.lola_decrypt_residues_level(ctx, sk, out[cnt:], 2, L2, 1, n)
            for m in range(2):
                assert np.array_equal(res[m, 0], slots[m] % t), (L1, L2, m)
        Lb.lola_ct_destroy(src)
    finally:
        Lb.lola_keys_destroy(sk)
        Lb.lola_ctx_destroy(ctx)


def test_mod_switch_rejects_bad_levels_and_overlap():
    need_gpu()
    Lb = lib()
    ps = W.params_small(256, L=3, K=1)
    ctx = make_ctx(ps)
    try:
        buf = torch_u64(np.zeros((2, 2, 3, 256), np.uint64))
        out = torch_u64(np.zeros((2, 2, 3, 256), np.uint64))
        for lf, lt in ((3, 4), (4, 2), (2, 3), (3, 0)):
            with pytest.raises(Lb.LolaError):
                Lb.lola_mod_switch(ctx, buf, out, 2, lf, lt)
        with pytest.raises(Lb.LolaError):
            Lb.lola_mod_switch(ctx, buf, buf, 2, 3, 2)
        Lb.lola_mod_switch(ctx, buf, out, 0, 3, 2)          # empty batch: no-op
    finally:
        Lb.lola_ctx_destroy(ctx)
