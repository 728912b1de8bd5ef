"""Oracle runs of whole networks at full size, as plain functions so that a
spawned worker process can run them while the GPU test waits (each takes a
minute or more on one core).  CPU oracle only; no CUDA."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import bfv, encoding, lola as OL  # noqa: E402

def rotation_steps(layers, n, t, st):
    """Rotation steps the plan uses (0 = row swap), from a slot-level run."""
    seen = set()

    class Rec(OL.SlotEval):
        def rot(self, a, k):
            seen.add(k)
            return super().rot(a, k)

        def rot_rows(self, a):
            seen.add(0)
            return super().rot_rows(a)

        def rot_hoisted(self, a, steps):
            seen.update(steps)
            return super().rot_hoisted(a, steps)

    OL.run_network(Rec(n, t), layers, st)
    return sorted(seen)


def mnist_layers():
    """The MNIST-shaped layer list bench.py runs: modulus switching, the last
    layer summed over the occupied slots, hoisted rotate-and-sums (on the
    parameters of params_mnist_grouped, key-switching digits of two primes)."""
    return W.layers_mnist(W.mnist_net(), W.params_mnist().n, W.MNIST_LEVELS, support_sum=True, hoist=W.MNIST_HOIST)


def mnist_steps():
    """Nonzero rotation steps of that plan (its Galois keys besides the row swap)."""
    ps = W.params_mnist_grouped()
    net = W.mnist_net()
    msgs, pos = OL.pack_convolution(W.image(), net.kh, net.kw, net.stride, ps.n)
    t = ps.t[0]
    st = OL.State([np.asarray(m, np.int64) % t for m in msgs], pos)
    return [s for s in rotation_steps(mnist_layers(), ps.n, t, st) if s]


def mnist_residue(ti: int, key_seed: int, enc_seed: int, img_idx: int = 0, msg0: int = 0):
    """Full MNIST-shaped network (n = 16384, L = 5 -> 4 -> 2, the plan of
    mnist_layers as bench.py runs it) for CRT residue
    ti of image img_idx, whose 25 messages are messages msg0 ... msg0 + 24 of
    a batch encrypted with k_t = len(t) residues per message (ciphertext id =
    message * k_t + ti).  Returns the output ciphertexts as an array
    [message][2][L_out][n] and the output positions (message, slot)."""
    ps = W.params_mnist_grouped()
    P = bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)
    kt, t = len(ps.t), ps.t[ti]
    net, img = W.mnist_net(), W.image(idx=img_idx)
    layers = mnist_layers()
    keys = bfv.keygen(P, key_seed, rotations=mnist_steps(), relin=True, row_swap=True)
    msgs, pos = OL.pack_convolution(img, net.kh, net.kw, net.stride, ps.n)
    cts = [bfv.encrypt(P, keys.pk, encoding.encode(m, t), t, enc_seed, (msg0 + i) * kt + ti)
           for i, m in enumerate(msgs)]
    ev = OL.HEEval(P, keys, t)
    st = OL.run_network(ev, layers, OL.State(cts, pos))
    out = np.stack([np.stack([c.c[0], c.c[1]]) for c in st.msgs])
    return out, [(int(m), int(s)) for m, s in st.pos]


def head(key_seed: int, enc_seed: int, idx: int = 0):
    """Transfer-learning head (n = 16384, L = 3, one t; rotate-and-sums hoisted
    as bench.py runs them) on feature vector idx,
    encrypted as message idx of a batch (ciphertext id idx).  Returns the
    output ciphertexts [message][2][L][n], output positions and the plan's
    rotation steps."""
    ps = W.params_head()
    P = bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)
    n, t = ps.n, ps.t[0]
    Wh = W.head_weights()
    layers = W.layers_head(Wh, n, W.HEAD_HOIST)
    steps = rotation_steps(layers, n, t, OL.State([np.zeros(n, np.int64)], [(0, i) for i in range(4096)]))
    keys = bfv.keygen(P, key_seed, rotations=[s for s in steps if s], relin=True, row_swap=0 in steps)
    v = np.zeros(n, np.int64)
    v[:4096] = W.feature_vector(idx=idx)
    ct = bfv.encrypt(P, keys.pk, encoding.encode(v, t), t, enc_seed, idx)
    st = OL.run_network(OL.HEEval(P, keys, t), layers, OL.State([ct], [(0, i) for i in range(4096)]))
    out = np.stack([np.stack([c.c[0], c.c[1]]) for c in st.msgs])
    return out, [(int(m), int(s)) for m, s in st.pos], steps
