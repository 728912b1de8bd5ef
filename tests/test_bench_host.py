"""Host-side pieces of bench.py: the plain integer network its output check
uses (its own numpy code, no oracle import) equals the oracle's integer
network on the MNIST-shaped weights and images."""
import os
import sys

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
