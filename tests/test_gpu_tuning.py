"""Launch-geometry tuning of the key-switch transforms: every geometry (one
CTA per limb, 2-CTA clusters with 16 or 32 words per thread) produces the
same words, the autotuner installs a valid table, and results after tuning
are unchanged (and equal to the oracle's)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import lib, make_ctx, need_gpu, oracle_params
from oracle import bfv, encoding

pytestmark = pytest.mark.gpu


def run_ops(Lb, ctx, ev, src, ps, steps):
    """rotations of every ciphertext (one step each) and squares + relinearisation"""
    cnt = Lb.lola_ct_messages(src)
    rot = Lb.lola_ct_create(ctx, cnt)
    sq = Lb.lola_ct_create(ctx, cnt)
    Lb.lola_rotate(ctx, ev, Lb.lola_ct_data(src), Lb.lola_ct_data(rot), cnt, steps)
    Lb.lola_multiply(ctx, ev, Lb.lola_ct_data(src), Lb.lola_ct_data(src), Lb.lola_ct_data(sq), cnt)
    shape = (1, 2, ps.L, ps.n)
    out = (Lb.lola_ct_export(ctx, rot, shape), Lb.lola_ct_export(ctx, sq, shape))
    Lb.lola_ct_destroy(rot)
    Lb.lola_ct_destroy(sq)
    return out


def test_every_geometry_and_the_autotuned_table_give_the_same_words():
    need_gpu()
    Lb = lib()
    n = 16384
    ps = W.params_small(n, L=3, K=1, t=[W.T30[0]])
    P = oracle_params(ps)
    t = ps.t[0]
    steps = [1, 5, 4096, 0]
    ctx = make_ctx(ps)
    try:
        sk, ev = Lb.lola_keygen(ctx, 61, [s for s in steps if s], Lb.LOLA_KEY_RELIN | Lb.LOLA_KEY_ROW_SWAP)
        slots = np.random.default_rng(61).integers(0, 1 << 16, (len(steps), n))
        src = Lb.lola_encrypt(ctx, sk, slots, 62)
        base = run_ops(Lb, ctx, ev, src, ps, steps)            # library defaults
        for g in range(Lb.TUNE_VARIANTS):                     # incl. the 4-CTA clusters
            Lb.lola_tune_set(ctx, [[g] * 6 for _ in range(4)])
            got = run_ops(Lb, ctx, ev, src, ps, steps)
            assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1]), g
        Lb.lola_tune_set(ctx, None)
        res = Lb.lola_autotune(ctx)
        assert len(res["table"]) == 4 and all(len(r) == 6 and all(v in range(Lb.TUNE_VARIANTS) for v in r)
                                         for r in res["table"])
        assert sum(1 for k in range(4) for b in range(6) if all(x > 0 for x in res["us"][k][b])) >= 10
        got = run_ops(Lb, ctx, ev, src, ps, steps)
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1])
        # and the words are the oracle's (first ciphertext: rotation by 1, square)
        ok = bfv.keygen(P, 61, rotations=[1], relin=True)
        c = bfv.encrypt(P, ok.pk, encoding.encode(slots[0], t), t, 62, 0)
        r = bfv.rotate(P, ok, c, 1)
        assert np.array_equal(base[0][0, 0, 0], r.c[0]) and np.array_equal(base[0][0, 0, 1], r.c[1])
        s2 = bfv.relinearize(P, ok, bfv.multiply(P, c, c))
        assert np.array_equal(base[1][0, 0, 0], s2.c[0]) and np.array_equal(base[1][0, 0, 1], s2.c[1])
        Lb.lola_ct_destroy(src)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_tune_table_checks():
    need_gpu()
    Lb = lib()
    ctx = make_ctx(W.params_small(1024, L=3, K=1))
    try:
        with pytest.raises(Lb.LolaError):
            Lb.lola_tune_get(ctx)                              # nothing installed yet
        with pytest.raises(Lb.LolaError):
            Lb.lola_tune_set(ctx, [[1] * 6 for _ in range(4)])  # clusters exist at n = 16384 only
        with pytest.raises(Lb.LolaError):
            Lb.lola_tune_set(ctx, [[3] * 6 for _ in range(4)])
        with pytest.raises(Lb.LolaError):
            Lb.lola_tune_set(ctx, [[Lb.TUNE_VARIANTS] * 6 for _ in range(4)])   # no such geometry
        res = Lb.lola_autotune(ctx)                            # one geometry: all entries 0
        assert res["table"] == [[0] * 6 for _ in range(4)]
        Lb.lola_tune_set(ctx, None)
        with pytest.raises(Lb.LolaError):
            Lb.lola_tune_get(ctx)
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_autotune_cache_file(tmp_path):
    """autotune_cached runs the tuner once per key and then installs the
    stored table from the JSON file."""
    need_gpu()
    Lb = lib()
    ps = W.params_small(16384, L=2, K=1)
    ctx = make_ctx(ps)
    try:
        path = str(tmp_path / "tune.json")
        key = {"n": ps.n, "L": ps.L, "device": "test"}
        first = Lb.autotune_cached(ctx, path, key)
        assert first["cached"] is False
        Lb.lola_tune_set(ctx, None)
        second = Lb.autotune_cached(ctx, path, key)
        assert second["cached"] is True and second["table"] == first["table"]
        assert Lb.lola_tune_get(ctx)["table"] == first["table"]
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_alu_microbenchmarks_report_positive_rates():
    # the measured integer peaks the transforms' roofline is stated against:
    # every kind runs and returns a positive rate; unknown kinds are refused
    need_gpu()
    Lb = lib()
    ctx = make_ctx(W.params_small(1024, L=2))
    try:
        rates = {k: Lb.lola_alu_rate(ctx, k) for k in Lb.ALU_KINDS}
        for k, (r, ms) in rates.items():
            assert r > 0 and ms > 0, k
        # a butterfly needs about a dozen 32-bit multiply-class instructions:
        # its rate must sit far below the mad.lo.u32 instruction rate
        assert rates["fwd_butterfly"][0] < rates["mad_lo_u32"][0] / 4
        with pytest.raises(Lb.LolaError):
            Lb.lola_alu_rate(ctx, 99)
    finally:
        Lb.lola_ctx_destroy(ctx)
