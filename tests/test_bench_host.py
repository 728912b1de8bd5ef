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
