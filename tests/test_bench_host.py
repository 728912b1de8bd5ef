"""Host-side pieces of bench.py: the plain integer network its output check
uses (its own numpy code, no oracle import) equals the oracle's integer
network on the MNIST-shaped weights and images."""
import os
import sys

import numpy as np
import pytest

import workloads as W
from oracle import lola as OL

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_plain_network_matches_oracle_integer_network():
    mnet = W.mnist_net()
    for idx in (0, 3):
        img = W.image(idx=idx)
        x = OL.int_conv(img, mnet.conv_w, 5, 5, 2)
        assert [int(v) for v in bench.plain_conv(img, mnet.conv_w)] == x
        x = OL.int_dense(OL.int_square(x), mnet.dense1_w)
        want = OL.int_dense(OL.int_square(x), mnet.dense2_w)
        assert bench.plain_mnist(img, mnet) == want


def test_plain_dense_matches_oracle():
    Wh = W.head_weights()
    f = W.feature_vector(idx=1)
    assert bench.plain_dense(f, Wh) == OL.int_dense(f, Wh)


def test_plain_cifar_matches_oracle_integer_network():
    net = W.cifar_net()
    img = W.cifar_image(idx=5)
    x = OL.int_conv(W.cifar_padded(img, net.pad), net.w1, net.k1, net.k1, net.stride)
    x = OL.int_square(x)
    x = OL.int_square(OL.int_dense(x, W.cifar_dense2(net)))
    assert bench.plain_cifar(img, net) == OL.int_dense(x, net.w3)


@pytest.mark.parametrize("workload", ["mnist", "mnist_paper", "lola_dense", "lola_dense_paper", "cifar", "head"])
def test_op_counts_by_level_match_the_plan(workload):
    """bench.py's per-level operation counts (used to scale the oracle's
    per-operation times) are the plan's, counted on slot vectors with the
    modulus switches in place."""
    lola = OL

    class LevelCount(lola.SlotEval):
        def __init__(self, n, t, L):
            super().__init__(n, t)
            self.level, self.c = L, {}

        def _k(self, op):
            d = self.c.setdefault(self.level, {"rot": 0, "square": 0, "mul_plain": 0, "mul_scalar": 0, "add": 0})
            d[op] += 1

        def add(self, a, b):
            self._k("add")
            return super().add(a, b)

        def rot(self, a, k):
            self._k("rot")
            return super().rot(a, k)

        def rot_rows(self, a):
            self._k("rot")
            return super().rot_rows(a)

        def rot_hoisted(self, a, steps):
            return [self.rot_rows(a) if k == 0 else self.rot(a, k) for k in steps]

        def mul_plain(self, a, v):
            self._k("mul_plain")
            return super().mul_plain(a, v)

        def mul_scalar(self, a, w):
            self._k("mul_scalar")
            return super().mul_scalar(a, w)

        def square(self, a):
            self._k("square")
            return super().square(a)

        def mod_switch(self, msgs, Lv):
            self.level = Lv
            return msgs

    n, t = 16384, W.T30[0]
    net = W.mnist_net()
    if workload.startswith("mnist"):
        ev = LevelCount(n, t, 5)
        msgs, pos = lola.pack_convolution(W.image(), net.kh, net.kw, net.stride, n)
        layers = W.layers_mnist(net, n, W.MNIST_LEVELS, support_sum=not workload.endswith("_paper"))
    elif workload.startswith("lola_dense"):
        ev = LevelCount(n, t, 6)
        v, pos = lola.pack_image_rows(W.image(), W.DENSE_IMAGE_WIDTH, n)
        msgs = [v]
        layers = W.layers_lola_dense(net, n, levels=W.LOLA_DENSE_LEVELS, support_sum=not workload.endswith("_paper"))
    elif workload == "head":
        ev = LevelCount(n, t, 3)
        Wh = W.head_weights()
        v = np.zeros(n, np.int64)
        v[:Wh.shape[1]] = W.feature_vector()
        msgs, pos = [v], [(0, i) for i in range(Wh.shape[1])]
        layers = W.layers_head(Wh, n)
    else:
        ev = LevelCount(n, t, 6)
        cnet = W.cifar_net()
        msgs, pos = lola.pack_convolution(W.cifar_padded(W.cifar_image(), cnet.pad), cnet.k1, cnet.k1, cnet.stride, n)
        layers = W.layers_cifar(cnet, n, levels=W.CIFAR_LEVELS)
    lola.run_network(ev, layers, lola.State([np.array(m, np.int64) % t for m in msgs], pos))
    assert ev.c == bench.OP_COUNTS_LEVELS.get(workload, {3: bench.OP_COUNTS[workload]})
    for op in ("rot", "square", "mul_plain", "mul_scalar", "add"):
        assert sum(c[op] for c in ev.c.values()) == bench.OP_COUNTS[workload][op]


def test_oracle_end_to_end_inference_dense64():
    """The CPU baseline's end-to-end oracle inference (spawned worker per
    residue) runs the single dense layer + square, decrypts to the integer
    network mod t and counts the plan's operations."""
    r = bench.oracle_e2e_inference("dense64", 3, None)
    assert r["ok"] and r["residues"] == 1 and r["eval_s"] > 0
    assert r["ops_per_residue"]["rot"] == bench.OP_COUNTS["dense64"]["rot"]
    assert r["ops_per_residue"]["square"] == 1
    obj = bench.cpu_baseline_obj("dense64", 3, None)
    assert obj["kind"] == "oracle end-to-end" and obj["cores"] == 1 and obj["value"] > 0


def test_plan_counts_without_hoisting_are_the_op_count_tables():
    for workload in ("mnist", "lola_dense"):
        for paper in (False, True):
            c = bench.plan_counts(workload, {"mnist": 5}.get(workload, 6),
                                  W.MNIST_LEVELS if workload == "mnist" else W.LOLA_DENSE_LEVELS, paper, (1, 1, 1))
            want = bench.OP_COUNTS_LEVELS[bench.counts_key(workload, paper)]
            assert {lv: {k: v for k, v in d.items() if k != "rot_sum"} for lv, d in c.items()} == want
            assert all(d["rot_sum"] == {} for d in c.values())


def test_plan_counts_of_the_hoisted_mnist_plan():
    # at 4 primes: the stack's [1024, 2048 | 4096 | row swap] and 7 rounds of
    # [1, 2 | 4, 8 | ... | 256, 512] -> 1 + 35 rotate-sums of 3 rotations, 2
    # single rotations + 6 for the rounds' combine; at 2 primes 10 outputs x
    # [1, 2, 4 | 1024, 2048, 4096 | row swap] -> 20 rotate-sums of 7, 10 single
    c = bench.plan_counts("mnist", 5, W.MNIST_LEVELS, False, (2, 2, 3))
    assert {lv: (d["rot"], d["rot_sum"]) for lv, d in c.items()} == {5: (4, {}), 4: (8, {3: 36}), 2: (10, {7: 20})}
    # three steps per key switch everywhere: the stack's [1024, 2048, 4096 |
    # row swap], 7 rounds of [1, 2, 4 | 8, 16, 32 | 64, 128, 256 | 512]
    c = bench.plan_counts("mnist", 5, W.MNIST_LEVELS, False, (3, 3, 3))
    assert {lv: (d["rot"], d["rot_sum"]) for lv, d in c.items()} == {5: (4, {}), 4: (14, {7: 22}), 2: (10, {7: 20})}


def test_plan_counts_of_the_hoisted_head_and_cifar_plans():
    # head: stack [4096 | row swap] and 26 rounds of [1, 2, 4 | ... | 512, 1024, 2048],
    # 25 round shifts -> 27 single rotations and 26 x 4 rotate-sums of 7;
    # CIFAR: 4075 outputs of [1, 2, 4 | ... | 512, 1024, 2048 | 4096 | row swap] at 4 primes
    # (4 rotate-sums, then the last shift and the row swap alone) and the last product's 10
    # outputs summed over 4075 slots ([1, 2, 4 | ... | 512, 1024, 2048]: 4 rotate-sums) at 2
    c = bench.plan_counts("head", 3, None, False, (3, 3, 3))
    assert {lv: (d["rot"], d["rot_sum"]) for lv, d in c.items()} == {3: (27, {7: 104})}
    c = bench.plan_counts("cifar", 6, W.CIFAR_LEVELS, False, (3, 3, 3))
    assert {lv: (d["rot"], d["rot_sum"]) for lv, d in c.items()} == {6: (83, {}), 4: (8150, {7: 16300}),
                                                                     2: (0, {7: 40})}
