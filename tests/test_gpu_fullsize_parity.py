"""Word-for-word GPU parity at full size, in the configuration bench.py times.

The MNIST-shaped network (n = 16384, five 60-bit primes switched to four and
two after the squares, key-switching digits of two primes with two special
primes, three CRT plaintext moduli, the last layer summed
over the occupied slots, the rotate-and-sums hoisted several doubling steps
per key switch, batch of 16 requests, autotuned launch geometry,
CUDA-graph replay) and the transfer-learning head
(n = 16384, three primes, one plaintext modulus, hoisted rotate-and-sums,
batch of 64): for one
sampled request and one CRT residue the oracle runs the same layer list on
the same encrypted input with the same keys, and every output ciphertext
must match the GPU's word for word.  The oracle runs (a minute or two each
on one core) start in spawned worker processes when the module's first test
begins and overlap the GPU work.
"""
import multiprocessing
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import oracle_jobs as J
import workloads as W
from gpu_util import lib, make_ctx, need_gpu

pytestmark = pytest.mark.gpu

MNIST_B, MNIST_REQ, MNIST_TI = 16, 5, 1
HEAD_B, HEAD_REQ = 64, 17
KEY_SEED, ENC_SEED = W.DEFAULT_SEED, 21
HEAD_KEY_SEED, HEAD_ENC_SEED = 99, 8


@pytest.fixture(scope="module")
def oracle_runs():
    need_gpu()
    ex = ProcessPoolExecutor(max_workers=2, mp_context=multiprocessing.get_context("spawn"))
    futs = {"mnist": ex.submit(J.mnist_residue, MNIST_TI, KEY_SEED, ENC_SEED, MNIST_REQ, MNIST_REQ * 25),
            "head": ex.submit(J.head, HEAD_KEY_SEED, HEAD_ENC_SEED, HEAD_REQ)}
    yield futs
    ex.shutdown(cancel_futures=True)


def gpu_keys(Lb, ctx, net, seed):
    steps = net.rotation_steps()
    flags = Lb.LOLA_KEY_RELIN | (Lb.LOLA_KEY_ROW_SWAP if 0 in steps else 0)
    return Lb.lola_keygen(ctx, seed, [s for s in steps if s], flags)


def test_full_mnist_batch16_every_output_ciphertext_matches_oracle(oracle_runs):
    Lb = lib()
    ps = W.params_mnist_grouped()
    n = ps.n
    mnet = W.mnist_net()
    layers = J.mnist_layers()
    ctx = make_ctx(ps)
    try:
        Lb.lola_autotune(ctx)                 # the geometry table bench.py times with
        packed = [Lb.lola_pack_convolution(W.image(idx=i), 5, 5, 2, n) for i in range(MNIST_B)]
        net = Lb.lola_net_create(ctx, {"repr": "convolution", "n_msgs": 25, "n_elems": packed[0][1]}, layers)
        assert sorted(s for s in net.rotation_steps() if s) == J.mnist_steps()
        sk, ev = gpu_keys(Lb, ctx, net, KEY_SEED)
        ct = Lb.lola_encrypt(ctx, sk, np.concatenate([p[0] for p in packed]), ENC_SEED)
        out = Lb.lola_ct_create(ctx, MNIST_B * 10)
        Lb.lola_eval_network(ctx, ev, net, ct, out)          # eager + capture
        Lb.lola_eval_network(ctx, ev, net, ct, out)          # graph replay (what the bench times)
        got = Lb.lola_ct_export(ctx, out, (3, 2, ps.L, n))   # [request * 10 + o][t_i][2][L_out][n]
        assert got.shape[3] == W.MNIST_LEVELS[1]
        want, pos = oracle_runs["mnist"].result(timeout=1800)
        assert want.shape == (10, 2, W.MNIST_LEVELS[1], n)
        assert pos == [(m, s) for m, s in net.output_map()]
        for o in range(10):
            g = got[MNIST_REQ * 10 + o, MNIST_TI]
            assert np.array_equal(g, want[o]), f"output ciphertext {o} differs"
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)


def test_full_head_batch64_every_output_ciphertext_matches_oracle(oracle_runs):
    Lb = lib()
    ps = W.params_head()
    n = ps.n
    Wh = W.head_weights()
    layers = W.layers_head(Wh, n, W.HEAD_HOIST)
    ctx = make_ctx(ps)
    try:
        Lb.lola_autotune(ctx)
        net = Lb.lola_net_create(ctx, {"repr": "dense", "n_msgs": 1, "n_elems": 4096}, layers)
        sk, ev = gpu_keys(Lb, ctx, net, HEAD_KEY_SEED)
        slots = np.zeros((HEAD_B, n), dtype=np.int64)
        for i in range(HEAD_B):
            slots[i, :4096] = W.feature_vector(idx=i)
        ct = Lb.lola_encrypt(ctx, sk, slots, HEAD_ENC_SEED)
        n_out = net.shape()[1]
        out = Lb.lola_ct_create(ctx, HEAD_B * n_out)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        Lb.lola_eval_network(ctx, ev, net, ct, out)
        got = Lb.lola_ct_export(ctx, out, (1, 2, ps.L, n))[:, 0]
        want, pos, steps = oracle_runs["head"].result(timeout=1800)
        assert steps == sorted(net.rotation_steps())
        assert pos == [(m, s) for m, s in net.output_map()]
        for o in range(want.shape[0]):
            assert np.array_equal(got[HEAD_REQ * n_out + o], want[o]), f"output ciphertext {o} differs"
        for h in (ct, out):
            Lb.lola_ct_destroy(h)
        Lb.lola_keys_destroy(sk)
        Lb.lola_keys_destroy(ev)
        net.destroy()
    finally:
        Lb.lola_ctx_destroy(ctx)
