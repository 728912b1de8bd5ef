"""Continuous-batching server: every request's output ciphertext is the same
whether it is evaluated alone or batched with others in the mix (bit-exact:
all operations act on each ciphertext independently), with two networks of
different sizes served together and arrivals interleaved with running
batches."""
import numpy as np
import pytest

import workloads as W
from gpu_util import lib, make_ctx, need_gpu

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone_results():
    need_gpu()
    Lb = lib()
    from paper_1812_10659_gb300 import serve
    import torch
    n = 1024
    ps = W.params_small(n, L=5, K=1, t=W.T30[:2])
    ctx = make_ctx(ps)
    try:
        mnet = W.mnist_net(seed=7, maps=2, hidden=12, classes=3, h=12, w=12, k=3, stride=2)
        Wh = W.head_weights(classes=6, dim=64)
        nets = {
            "mnist": ({"repr": "convolution", "n_msgs": 9, "n_elems": 36}, W.layers_mnist(mnet, n)),
            "head": ({"repr": "dense", "n_msgs": 1, "n_elems": 64}, W.layers_head(Wh, n)),
        }
        steps = set()
        for d, layers in nets.values():
            h = Lb.lola_net_create(ctx, d, layers)
            steps |= set(h.rotation_steps())
            h.destroy()
        sk, ev = Lb.lola_keygen(ctx, 5, sorted(s for s in steps if s), Lb.LOLA_KEY_RELIN | Lb.LOLA_KEY_ROW_SWAP)
        rng = np.random.default_rng(0)
        inputs = []
        for i in range(12):
            if i % 3 == 2:
                x = np.zeros((1, n), np.int64)
                x[0, :64] = rng.integers(0, 16, 64)
                inputs.append(("head", Lb.lola_encrypt(ctx, sk, x, 100 + i)))
            else:
                img = W.image(seed=50 + i, h=12, w=12)
                inputs.append(("mnist", Lb.lola_encrypt(ctx, sk, Lb.lola_pack_convolution(img, 3, 3, 2, n)[0], 100 + i)))
        # alone: one request per batch, eager launches
        alone = []
        for kind, ct in inputs:
            h = Lb.lola_net_create(ctx, *nets[kind])
            out = Lb.lola_ct_create(ctx, h.shape()[1])
            Lb.lola_eval_network(ctx, ev, h, ct, out, graph=False)
            alone.append(Lb.lola_ct_export(ctx, out, (2, 2, ps.L, n)))
            Lb.lola_ct_destroy(out)
            h.destroy()
        # in the mix: two slots, batches up to 4, arrivals interleaved with running batches
        srv = serve.Server(ctx, ev, nets, slots=2, max_batch={"mnist": 4, "head": 4})
        srv.warm()
        ids = []
        for i, (kind, ct) in enumerate(inputs):
            ids.append(srv.submit(kind, ct))
            if i % 4 == 3:
                srv.step()
        srv.drain()
        batches = set()
        for rid, want in zip(ids, alone):
            got = Lb.lola_ct_export(ctx, srv.poll(rid), (2, 2, ps.L, n))
            assert np.array_equal(got, want), rid
            batches.add(srv.requests[rid].batch)
        assert max(batches) > 1           # some requests really were batched
        st = srv.stats()
        assert st["all"]["n"] == len(inputs)
        srv.close()
        for _, ct in inputs:
            Lb.lola_ct_destroy(ct)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
    finally:
        Lb.lola_ctx_destroy(ctx)
