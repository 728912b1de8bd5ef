"""GPU parity of whole LoLa networks.

* single dense layer + square (n = 4096) and a reduced MNIST-shaped network
  (n = 1024): every output ciphertext bit-exact against the oracle running
  the same layer list on the same encrypted input with the same keys;
* the full MNIST-shaped network (n = 16384, three CRT moduli) and the
  transfer-learning head at full size, batched: decrypted outputs equal the
  integer network exactly (after CRT), graph replay equal to eager launch.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import ct_stack, lib, make_ctx, need_gpu, oracle_params
from oracle import bfv, encoding, lola as OL

pytestmark = pytest.mark.gpu


def gpu_keys(Lb, ctx, net, seed):
    steps = net.rotation_steps()
    flags = Lb.LOLA_KEY_RELIN | (Lb.LOLA_KEY_ROW_SWAP if 0 in steps else 0)
    return Lb.lola_keygen(ctx, seed, [s for s in steps if s], flags)


def oracle_keys(P, net, seed):
    steps = net.rotation_steps()
    return bfv.keygen(P, seed, rotations=[s for s in steps if s], relin=True, row_swap=0 in steps)


def mnist_int(net, img):
    x = OL.int_conv(img, net.conv_w, net.kh, net.kw, net.stride)
    x = OL.int_dense(OL.int_square(x), net.dense1_w)
    return OL.int_dense(OL.int_square(x), net.dense2_w)


def test_dense64_bit_exact_vs_oracle():
    need_gpu()
    Lb = lib()
    ps = W.params_dense64()
    P = oracle_params(ps)
    n, t = ps.n, ps.t[0]
    Wd, x = W.dense_weights(), W.dense_vector()
    copies = W.dense64_input_copies(Wd)
    layers = W.layers_dense64(Wd, n)
    ctx = make_ctx(ps)
    try:
        net = Lb.lola_net_create(ctx, {"repr": "stacked", "n_msgs": 1, "n_elems": 64, "d": 6, "copies": copies}, layers)
        sk, ev = gpu_keys(Lb, ctx, net, W.DEFAULT_SEED)
        packed = Lb.lola_pack_stacked(x, 6, copies, n)
        ct = Lb.lola_encrypt(ctx, sk, packed[None], 3)
        out = Lb.lola_ct_create(ctx, 1)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        got = Lb.lola_ct_export(ctx, out, (1, 2, P.L, n))[0, 0]
        # oracle: same keys, same ciphertext, same layer list
        ok = oracle_keys(P, net, W.DEFAULT_SEED)
        oct_ = bfv.encrypt(P, ok.pk, encoding.encode(packed, t), t, 3, 0)
        st = OL.run_network(OL.HEEval(P, ok, t), layers, OL.State([oct_], [(0, i) for i in range(64)], 64, copies))
        assert np.array_equal(got[0], st.msgs[0].c[0]) and np.array_equal(got[1], st.msgs[0].c[1])
        dec = Lb.lola_decrypt_residues(ctx, sk, out, 1, n)[0, 0]
        want = [v % t for v in OL.int_square(OL.int_dense(x, Wd))]
        assert [int(dec[s]) for _, s in net.output_map()] == want
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


@pytest.mark.parametrize("levels,K,alpha,support,hoist", [
    (None, 1, 1, False, 1), ((4, 2), 1, 1, False, 1), ((3, 1), 1, 1, False, 1), ((4, 2), 2, 2, False, 1),
    ((3, 1), 2, 2, False, 1), ((4, 2), 1, 1, True, 1), (None, 2, 2, True, 1), ((4, 2), 1, 1, True, (2, 2, 3)),
    ((4, 2), 1, 1, False, (2, 3, 2)), (None, 2, 2, True, (3, 3, 4))])
def test_mini_mnist_bit_exact_vs_oracle(levels, K, alpha, support, hoist):
    # levels: modulus switching after each square (every later ciphertext,
    # including the relinearisation at level 4 or 3, compared word for word);
    # K = 2, alpha = 2: key-switching digits of two primes; hoist: rotate-and-
    # sum doubling steps per key switch in the stack, the stacked row-major
    # and the last layer (rotate-sums next to single rotations)
    need_gpu()
    Lb = lib()
    n = 1024
    ps = W.params_small(n, L=5, K=K, t=W.T30[:1], alpha=alpha)
    P = oracle_params(ps)
    t = ps.t[0]
    mnet = W.mnist_net(seed=7, maps=2, hidden=12, classes=3, h=12, w=12, k=3, stride=2)
    img = W.image(seed=7, h=12, w=12)
    layers = W.layers_mnist(mnet, n, levels, support_sum=support, hoist=hoist)
    ctx = make_ctx(ps)
    try:
        msgs, win = Lb.lola_pack_convolution(img, 3, 3, 2, n)
        net = Lb.lola_net_create(ctx, {"repr": "convolution", "n_msgs": 9, "n_elems": win}, layers)
        sk, ev = gpu_keys(Lb, ctx, net, 11)
        ct = Lb.lola_encrypt(ctx, sk, msgs, 5)
        out = Lb.lola_ct_create(ctx, 3)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        got = Lb.lola_ct_export(ctx, out, (1, 2, P.L, n))[:, 0]
        assert Lb.lola_ct_level(out) == (levels[1] if levels else P.L)
        ok = oracle_keys(P, net, 11)
        octs = [bfv.encrypt(P, ok.pk, encoding.encode(m, t), t, 5, i) for i, m in enumerate(msgs)]
        st = OL.run_network(OL.HEEval(P, ok, t), layers, OL.State(octs, [(0, i) for i in range(win)]))
        assert [(int(m), int(s)) for m, s in net.output_map()] == [(int(m), int(s)) for m, s in st.pos]
        for o in range(3):
            assert np.array_equal(got[o, 0], st.msgs[o].c[0]) and np.array_equal(got[o, 1], st.msgs[o].c[1]), o
        if levels != (3, 1):     # one 60-bit prime leaves no noise budget for the last layer (oracle: -15 bits)
            res = Lb.lola_decrypt_residues(ctx, sk, out, 1, n)
            assert [int(res[m, 0, s]) for m, s in net.output_map()] == [v % t for v in mnist_int(mnet, img)]
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_full_mnist_batched_decrypts_to_integer_network():
    need_gpu()
    Lb = lib()
    ps = W.params_mnist()
    n = ps.n
    mnet = W.mnist_net()
    layers = W.layers_mnist(mnet, n, W.MNIST_LEVELS)
    ctx = make_ctx(ps)
    try:
        B = 2
        imgs = [W.image(idx=i) for i in range(B)]
        packed = [Lb.lola_pack_convolution(im, 5, 5, 2, n) for im in imgs]
        win = packed[0][1]
        net = Lb.lola_net_create(ctx, {"repr": "convolution", "n_msgs": 25, "n_elems": win}, layers)
        assert sorted(net.rotation_steps()) == sorted([0, 1, 2, 3, 4, 5, 6, 169, 338, 507, 676] +
                                                      [1 << j for j in range(3, 13)])
        sk, ev = gpu_keys(Lb, ctx, net, W.DEFAULT_SEED)
        ct = Lb.lola_encrypt(ctx, sk, np.concatenate([p[0] for p in packed]), 21)
        out = Lb.lola_ct_create(ctx, B * 10)
        out2 = Lb.lola_ct_create(ctx, B * 10)
        Lb.lola_eval_network(ctx, ev, net, ct, out)                   # first call: eager + capture
        Lb.lola_eval_network(ctx, ev, net, ct, out2)                  # graph replay
        a = Lb.lola_ct_export(ctx, out, (3, 2, ps.L, n))
        b = Lb.lola_ct_export(ctx, out2, (3, 2, ps.L, n))
        assert a.shape[3] == W.MNIST_LEVELS[1] and np.array_equal(a, b)
        dec = Lb.lola_decrypt(ctx, sk, out, n)
        omap = net.output_map()
        for r in range(B):
            got = [int(dec[r * 10 + m, s]) for m, s in omap]
            assert got == mnist_int(mnet, imgs[r]), r
            # sparse output: every slot of the message holds the value
            assert all(int(dec[r * 10 + m, 77]) == g for (m, _), g in zip(omap, got))
        for h in (ct, out, out2):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_head_batched_decrypts_to_integer_network():
    need_gpu()
    Lb = lib()
    ps = W.params_head()
    n, t = ps.n, ps.t[0]
    Wh = W.head_weights()
    layers = W.layers_head(Wh, n)
    ctx = make_ctx(ps)
    try:
        B = 3
        xs = [W.feature_vector(idx=i) for i in range(B)]
        net = Lb.lola_net_create(ctx, {"repr": "dense", "n_msgs": 1, "n_elems": 4096}, layers)
        sk, ev = gpu_keys(Lb, ctx, net, 99)
        slots = np.zeros((B, n), dtype=np.int64)
        for i, x in enumerate(xs):
            slots[i, :4096] = x
        ct = Lb.lola_encrypt(ctx, sk, slots, 8)
        out = Lb.lola_ct_create(ctx, B)
        Lb.lola_eval_network(ctx, ev, net, ct, out, graph=False)
        dec = Lb.lola_decrypt(ctx, sk, out, n)
        for r in range(B):
            got = [int(dec[r, s]) for _, s in net.output_map()]
            assert got == OL.int_dense(xs[r], Wh)
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_representation_mismatch_rejected():
    need_gpu()
    Lb = lib()
    ps = W.params_small(1024, L=3)
    ctx = make_ctx(ps)
    try:
        with pytest.raises(Lb.LolaError) as ei:
            Lb.lola_net_create(ctx, {"repr": "dense", "n_msgs": 1, "n_elems": 10},
                               [{"op": "stacked_rowmajor", "weights": np.ones((2, 10), np.int64), "d": 4, "copies": 2}])
        assert ei.value.code == -4
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_dense_rowmajor_sparse_colmajor_bit_exact_vs_oracle():
    """Dense vector - row major (Sec. 4.2.2, the transfer-learning head's
    variant) followed by sparse vector - column major, on the GPU and on the
    oracle with the same keys and ciphertext."""
    need_gpu()
    Lb = lib()
    n = 256
    ps = W.params_small(n, L=3, K=1, t=W.T30[:1])
    P = oracle_params(ps)
    t = ps.t[0]
    g = np.random.default_rng(4)
    x = g.integers(0, 16, 40)
    W1 = g.integers(-3, 4, (6, 40))
    W2 = g.integers(-3, 4, (9, 6))
    layers = [{"op": "dense_rowmajor", "weights": W1}, {"op": "sparse_colmajor", "weights": W2}]
    ctx = make_ctx(ps)
    try:
        net = Lb.lola_net_create(ctx, {"repr": "dense", "n_msgs": 1, "n_elems": 40}, layers)
        sk, ev = gpu_keys(Lb, ctx, net, 21)
        v = np.zeros((1, n), np.int64)
        v[0, :40] = x
        ct = Lb.lola_encrypt(ctx, sk, v, 4)
        out = Lb.lola_ct_create(ctx, 1)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        got = Lb.lola_ct_export(ctx, out, (1, 2, P.L, n))[0, 0]
        ok = oracle_keys(P, net, 21)
        oct_ = bfv.encrypt(P, ok.pk, encoding.encode(v[0], t), t, 4, 0)
        st = OL.run_network(OL.HEEval(P, ok, t), layers, OL.State([oct_], [(0, i) for i in range(40)]))
        assert np.array_equal(got[0], st.msgs[0].c[0]) and np.array_equal(got[1], st.msgs[0].c[1])
        dec = Lb.lola_decrypt(ctx, sk, out, n)
        assert [int(dec[m, s]) for m, s in net.output_map()] == OL.int_dense(OL.int_dense(x, W1), W2)
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


def lola_dense_input(net, width):
    return {"repr": "dense", "n_msgs": 1, "n_elems": net.h * net.w,
            "slot": W.dense_image_slots(net.h, net.w, width)}


@pytest.mark.parametrize("levels", [None, (4, 2)])
def test_mini_lola_dense_bit_exact_vs_oracle(levels):
    """LoLa-Dense (App. C) on a reduced network: the dense image message is
    masked into the convolution representation on the server; every output
    ciphertext bit-exact against the oracle with the same keys and input
    (levels: modulus switching after the squares)."""
    need_gpu()
    Lb = lib()
    n = 1024
    ps = W.params_small(n, L=5, K=1, t=W.T30[:1])
    P = oracle_params(ps)
    t = ps.t[0]
    mnet = W.mnist_net(seed=7, maps=2, hidden=12, classes=3, h=12, w=12, k=3, stride=2)
    img = W.image(seed=7, h=12, w=12)
    width = 13
    layers = W.layers_lola_dense(mnet, n, width, levels)
    ctx = make_ctx(ps)
    try:
        net = Lb.lola_net_create(ctx, lola_dense_input(mnet, width), layers)
        sk, ev = gpu_keys(Lb, ctx, net, 13)
        v, _ = OL.pack_image_rows(img, width, n)
        ct = Lb.lola_encrypt(ctx, sk, np.array([v], np.int64), 6)
        out = Lb.lola_ct_create(ctx, 3)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        got = Lb.lola_ct_export(ctx, out, (1, 2, P.L, n))[:, 0]
        ok = oracle_keys(P, net, 13)
        oct_ = bfv.encrypt(P, ok.pk, encoding.encode(v, t), t, 6, 0)
        st = OL.run_network(OL.HEEval(P, ok, t), layers, OL.State([oct_], OL.pack_image_rows(img, width, n)[1]))
        for o in range(3):
            assert np.array_equal(got[o, 0], st.msgs[o].c[0]) and np.array_equal(got[o, 1], st.msgs[o].c[1]), o
        res = Lb.lola_decrypt_residues(ctx, sk, out, 1, n)
        assert [int(res[m, 0, s]) for m, s in net.output_map()] == [x % t for x in mnist_int(mnet, img)]
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_full_lola_dense_batched_decrypts_to_integer_network():
    need_gpu()
    Lb = lib()
    ps = W.params_lola_dense(6)
    n = ps.n
    mnet = W.mnist_net()
    layers = W.layers_lola_dense(mnet, n, levels=W.LOLA_DENSE_LEVELS)
    ctx = make_ctx(ps)
    try:
        B = 2
        imgs = [W.image(idx=10 + i) for i in range(B)]
        net = Lb.lola_net_create(ctx, lola_dense_input(mnet, W.DENSE_IMAGE_WIDTH), layers)
        sk, ev = gpu_keys(Lb, ctx, net, W.DEFAULT_SEED)
        slots = np.array([OL.pack_image_rows(im, W.DENSE_IMAGE_WIDTH, n)[0] for im in imgs], np.int64)
        ct = Lb.lola_encrypt(ctx, sk, slots, 31)
        out = Lb.lola_ct_create(ctx, B * 10)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        dec = Lb.lola_decrypt(ctx, sk, out, n)
        for r in range(B):
            assert [int(dec[r * 10 + m, s]) for m, s in net.output_map()] == mnist_int(mnet, imgs[r]), r
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_masked_shifts_rejects_a_non_shift_gather():
    need_gpu()
    Lb = lib()
    ps = W.params_small(256, L=3)
    ctx = make_ctx(ps)
    try:
        with pytest.raises(Lb.LolaError) as ei:
            Lb.lola_net_create(ctx, {"repr": "dense", "n_msgs": 1, "n_elems": 8},
                               [{"op": "masked_shifts", "weights": np.array([[0, 1], [2, 4]])}])
        assert ei.value.code == -1
    finally:
        Lb.lola_ctx_destroy(ctx)


# ------------------------------------------------------ CIFAR-shaped (Sec. 6.2)

def test_place_layer_bit_exact_vs_oracle():
    """Three dense messages combined over both slot rows (in-row shifts, a
    row change, a message split by masks): bit-exact against the oracle."""
    need_gpu()
    Lb = lib()
    n = 256
    ps = W.params_small(n, L=3, K=1, t=W.T30[:1])
    P = oracle_params(ps)
    t = ps.t[0]
    h = n // 2
    T = list(range(9)) + [h + e for e in range(9)] + [20 + e for e in range(4)] + [h + 40 + e for e in range(5)]
    layers = [{"op": "conv", "weights": np.eye(3, dtype=np.int64)},
              {"op": "place", "weights": np.array([T], dtype=np.int64)}]
    g = np.random.default_rng(5)
    msgs = np.zeros((3, n), np.int64)
    msgs[:, :9] = g.integers(0, 1000, (3, 9))
    ctx = make_ctx(ps)
    try:
        net = Lb.lola_net_create(ctx, {"repr": "convolution", "n_msgs": 3, "n_elems": 9}, layers)
        sk, ev = gpu_keys(Lb, ctx, net, 23)
        ct = Lb.lola_encrypt(ctx, sk, msgs, 2)
        out = Lb.lola_ct_create(ctx, 1)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        got = Lb.lola_ct_export(ctx, out, (1, 2, P.L, n))[0, 0]
        ok = oracle_keys(P, net, 23)
        octs = [bfv.encrypt(P, ok.pk, encoding.encode(m, t), t, 2, i) for i, m in enumerate(msgs)]
        st = OL.run_network(OL.HEEval(P, ok, t), layers, OL.State(octs, [(0, e) for e in range(9)]))
        assert np.array_equal(got[0], st.msgs[0].c[0]) and np.array_equal(got[1], st.msgs[0].c[1])
        dec = Lb.lola_decrypt_residues(ctx, sk, out, 1, n)[0, 0]
        assert [int(dec[s]) for _, s in net.output_map()] == [int(msgs[m, e]) for m in range(3) for e in range(9)]
        for hdl in (ct, out):
            Lb.lola_ct_destroy(hdl)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


def cifar_int(net, img):
    x = OL.int_conv(W.cifar_padded(img, net.pad), net.w1, net.k1, net.k1, net.stride)
    x = np.array(OL.int_square(x), dtype=np.int64)
    x = W.cifar_dense2(net) @ x
    x = OL.int_square([int(v) for v in x])
    return OL.int_dense(x, net.w3)


@pytest.mark.parametrize("levels,hoist,support", [(None, 1, False), ((4, 2), 1, False), ((4, 2), 3, True),
                                                  (None, (1, 2, 4), True)])
def test_mini_cifar_bit_exact_vs_oracle(levels, hoist, support):
    # hoist / support: the two row-major products' rotate-and-sums hoisted,
    # and the last one summed over its occupied slots, as bench.py runs them
    need_gpu()
    Lb = lib()
    n = 1024
    ps = W.params_small(n, L=5, K=1, t=W.T30[:1])
    P = oracle_params(ps)
    t = ps.t[0]
    net_ = W.cifar_net(seed=9, C=2, h=8, w=8, pad=2, k1=4, maps1=6, k2=2, maps2=3, classes=2)
    img = W.cifar_image(seed=9, C=2, h=8, w=8)
    layers = W.layers_cifar(net_, n, levels=levels, hoist=hoist, support_sum=support)
    msgs, pos = OL.pack_convolution(W.cifar_padded(img, net_.pad), net_.k1, net_.k1, net_.stride, n)
    ctx = make_ctx(ps)
    try:
        net = Lb.lola_net_create(ctx, {"repr": "convolution", "n_msgs": len(msgs), "n_elems": len(pos)}, layers)
        sk, ev = gpu_keys(Lb, ctx, net, 17)
        ct = Lb.lola_encrypt(ctx, sk, np.array(msgs, np.int64), 8)
        out = Lb.lola_ct_create(ctx, 2)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        got = Lb.lola_ct_export(ctx, out, (1, 2, P.L, n))[:, 0]
        ok = oracle_keys(P, net, 17)
        octs = [bfv.encrypt(P, ok.pk, encoding.encode(m, t), t, 8, i) for i, m in enumerate(msgs)]
        st = OL.run_network(OL.HEEval(P, ok, t), layers, OL.State(octs, pos))
        for o in range(2):
            assert np.array_equal(got[o, 0], st.msgs[o].c[0]) and np.array_equal(got[o, 1], st.msgs[o].c[1]), o
        res = Lb.lola_decrypt_residues(ctx, sk, out, 1, n)
        assert [int(res[m, 0, s]) for m, s in net.output_map()] == [x % t for x in cifar_int(net_, img)]
        for hdl in (ct, out):
            Lb.lola_ct_destroy(hdl)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


@pytest.mark.slow
def test_full_cifar_decrypts_to_integer_network():
    """The CIFAR-shaped network at full size (n = 16384, three ~30-bit t_i):
    the decrypted outputs equal the integer network modulo each t_i."""
    need_gpu()
    Lb = lib()
    ps = W.params_cifar()
    n = ps.n
    net_ = W.cifar_net()
    img = W.cifar_image(idx=3)
    layers = W.layers_cifar(net_, n, levels=W.CIFAR_LEVELS)
    msgs, win = Lb.lola_pack_convolution_channels(W.cifar_padded(img, net_.pad), net_.k1, net_.k1, net_.stride, n)
    ctx = make_ctx(ps)
    try:
        net = Lb.lola_net_create(ctx, {"repr": "convolution", "n_msgs": len(msgs), "n_elems": win}, layers)
        sk, ev = gpu_keys(Lb, ctx, net, W.DEFAULT_SEED)
        ct = Lb.lola_encrypt(ctx, sk, msgs, 41)
        out = Lb.lola_ct_create(ctx, 10)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        res = Lb.lola_decrypt_residues(ctx, sk, out, len(ps.t), n)
        want = cifar_int(net_, img)
        for ti, t in enumerate(ps.t):
            assert [int(res[m, ti, s]) for m, s in net.output_map()] == [x % t for x in want], ti
        for hdl in (ct, out):
            Lb.lola_ct_destroy(hdl)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_large_nonuniform_rotation_wave_is_chunked_exactly():
    """A combine of 9 messages rotates 8 of them by different steps; at 200
    requests the wave holds 1600 ciphertexts, more than one launch takes, so
    it runs in chunks of whole messages.  Every request's output must equal
    its single-request evaluation bit for bit and decrypt to the combined
    vector."""
    need_gpu()
    Lb = lib()
    n = 256
    ps = W.params_small(n, L=3, K=1, t=W.T30[:1])
    t = ps.t[0]
    layers = [{"op": "conv", "weights": np.eye(9, dtype=np.int64)},
              {"op": "combine", "stride": 10}]
    g = np.random.default_rng(8)
    B = 200
    msgs = np.zeros((B, 9, n), np.int64)
    msgs[:, :, :10] = g.integers(0, 1000, (B, 9, 10))
    ctx = make_ctx(ps)
    try:
        net = Lb.lola_net_create(ctx, {"repr": "convolution", "n_msgs": 9, "n_elems": 10}, layers)
        sk, ev = gpu_keys(Lb, ctx, net, 29)
        ct = Lb.lola_encrypt(ctx, sk, msgs.reshape(B * 9, n), 4)
        out = Lb.lola_ct_create(ctx, B)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        allw = Lb.lola_ct_export(ctx, out, (1, 2, ps.L, n))
        for r in (0, 57, B - 1):
            one_in = Lb.lola_ct_create(ctx, 9)
            Lb.lola_ct_copy_messages(ctx, one_in, 0, ct, r * 9, 9)
            one_out = Lb.lola_ct_create(ctx, 1)
            Lb.lola_eval_network(ctx, ev, net, one_in, one_out)
            single = Lb.lola_ct_export(ctx, one_out, (1, 2, ps.L, n))
            assert np.array_equal(allw[r], single[0]), r
            Lb.lola_ct_destroy(one_in)
            Lb.lola_ct_destroy(one_out)
        dec = Lb.lola_decrypt_residues(ctx, sk, out, 1, n)
        omap = net.output_map()
        for r in (0, B - 1):
            assert [int(dec[r, 0, s]) for _, s in omap] == [int(msgs[r, m, e]) % t for m in range(9) for e in range(10)]
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)
