"""Pins for the oracle's LoLa layers (CPU only).

* the paper's worked footnote examples (tests/golden/*.json);
* the slot simulator against the integer network over Z (reduced mod t and,
  for several t_i, recombined by CRT) at the full MNIST / head shapes;
* operation counts stated in the paper (Table 1, App. C) and derived in the
  plan;
* encrypted runs of the oracle whose decryptions equal the integer network,
  with the measured noise margin.
"""
import json
import os
from math import prod

import numpy as np
import pytest

import workloads as W
from conftest import GOLDEN
from oracle import bfv, encoding, lola


class Counting(lola.SlotEval):
    def __init__(self, n, t):
        super().__init__(n, t)
        self.c = {"rot": 0, "mul_plain": 0, "mul_scalar": 0, "square": 0}

    def rot(self, a, k):
        self.c["rot"] += 1
        return super().rot(a, k)

    def rot_rows(self, a):
        self.c["rot"] += 1
        return super().rot_rows(a)

    def mul_plain(self, a, s):
        self.c["mul_plain"] += 1
        return super().mul_plain(a, s)

    def mul_scalar(self, a, w):
        self.c["mul_scalar"] += 1
        return super().mul_scalar(a, w)

    def square(self, a):
        self.c["square"] += 1
        return super().square(a)


def load(name):
    return json.load(open(os.path.join(GOLDEN, name)))


# ------------------------------------------------------------ golden examples

def test_dot_product_footnote():
    g = load("dot_product_footnote.json")
    n, t = 8, 65537          # one row of the 2 x 4 slot matrix holds the 4-vector
    ev = lola.SlotEval(n, t)
    tags = [10 ** i for i in range(1, 5)]        # v_i w_i := 10^i, decodable sums
    x = np.array(tags + [0] * 4, dtype=np.int64) % t
    x1 = ev.add(x, ev.rot(x, 1))
    x2 = ev.add(x1, ev.rot(x1, 2))

    def decode(v):
        return sorted(i for i in range(1, 5) if (v // 10 ** i) % 10)

    assert [decode(int(v)) for v in x1[:4]] == [sorted(s) for s in g["after_rot1_add"]]
    assert [decode(int(v)) for v in x2[:4]] == [sorted(s) for s in g["after_rot2_add"]]


def test_stacked_2x2_footnote():
    g = load("stacked_2x2_footnote.json")
    n, t = 8, 65537
    Wm = g["W"]
    v = [5, 7]
    ev = lola.SlotEval(n, t)
    x, pos = lola.pack_stacked(v, 1, 2, n)
    st = lola.State([np.array(x, dtype=np.int64)], pos, 2, 2)
    out = lola.layer_stacked_rowmajor(ev, st, Wm, 1, 2)
    for entry, terms in g["result_entries_1based"].items():
        want = sum(Wm[r - 1][c - 1] * v[c - 1] for r, c in terms)
        assert int(out.msgs[0][int(entry) - 1]) == want
    assert [s for _, s in out.pos] == [int(e) - 1 for e in g["result_entries_1based"]]


def test_conv_representation_footnote():
    g = load("conv_representation_footnote.json")
    h, w = g["image_shape"]
    img = np.array([[10 * (r + 1) + (c + 1) for c in range(w)] for r in range(h)])   # a_{r,c} -> "rc"
    msgs, pos = lola.pack_convolution(img, *g["kernel"], g["stride"], 16)
    assert len(msgs) == len(g["messages_1based"]) and len(pos) == 4
    for m, want in zip(msgs, g["messages_1based"]):
        assert m[:4] == [10 * r + c for r, c in want]


# ------------------------------------------------- plan vs integer network

def mnist_slot_run(n, t, net, img, ev_cls=lola.SlotEval):
    ev = ev_cls(n, t)
    msgs, pos = lola.pack_convolution(img, net.kh, net.kw, net.stride, n)
    st = lola.State([np.array(m, dtype=np.int64) % t for m in msgs], pos)
    return ev, lola.run_network(ev, W.layers_mnist(net, n), st)


def mnist_int(net, img):
    x = lola.int_conv(img, net.conv_w, net.kh, net.kw, net.stride)
    x = lola.int_square(x)
    x = lola.int_dense(x, net.dense1_w)
    x = lola.int_square(x)
    return lola.int_dense(x, net.dense2_w)


def crt(residues, moduli):
    T = prod(moduli)
    x = sum(r * (T // m) * pow(T // m, -1, m) for r, m in zip(residues, moduli)) % T
    return x - T if x > T // 2 else x


def test_mnist_plan_matches_integer_network_with_crt():
    n = 16384
    net = W.mnist_net()
    img = W.image()
    want = mnist_int(net, img)
    # no-wrap bound: the largest possible |output| must fit in prod(t_i)/2
    bound = 100 * 3 * (845 * 3 * (25 * 15 * 3) ** 2) ** 2
    assert max(abs(v) for v in want) <= bound < prod(W.T30[:3]) // 2
    per_t = []
    for t in W.T30[:3]:
        ev, st = mnist_slot_run(n, t, net, img, Counting)
        assert ev.c == {"rot": 224, "mul_plain": 24, "mul_scalar": 125, "square": 2}
        per_t.append([int(st.msgs[m][s]) for m, s in st.pos])
        # the output is sparse: every slot of message o holds output o
        assert all(len(set(int(v) for v in msg)) == 1 for msg in st.msgs)
    got = [crt([r[o] for r in per_t], W.T30[:3]) for o in range(10)]
    assert got == want


def test_table1_operation_counts():
    # Table 1 / Sec. 4.3: 5 maps combined with 4 rotations; App. C: at
    # n = 16384 the 845-vector takes 16 stacked copies and 7 rounds.
    n = 16384
    L = W.layers_mnist(W.mnist_net(), n)
    assert L[3]["copies"] == 16 and L[3]["d"] == 10
    assert -(-100 // L[4]["copies"]) == 7
    ev = Counting(n, 65537)
    st = lola.State([np.zeros(n, np.int64) for _ in range(5)], [(m, w) for m in range(5) for w in range(169)])
    lola.layer_combine(ev, st, 169)
    assert ev.c["rot"] == 4
    # Table 1's n = 8192 variant: 8 copies, 13 rounds
    L8 = W.layers_mnist(W.mnist_net(), 8192)
    assert L8[3]["copies"] == 8 and -(-100 // L8[4]["copies"]) == 13


def test_head_plan_matches_integer_network():
    n, t = 16384, W.T30[0]
    Wh = W.head_weights()
    x = W.feature_vector()
    want = lola.int_dense(x, Wh)
    assert max(abs(v) for v in want) < t // 2
    ev = Counting(n, t)
    v, pos = lola.pack_dense(x, n)
    st = lola.run_network(ev, W.layers_head(Wh, n), lola.State([np.array(v, np.int64) % t], pos))
    assert ev.c["rot"] == 2 + 26 * 12 + 25 and ev.c["mul_plain"] == 26 + 26
    got = [int(st.msgs[m][s]) for m, s in st.pos]
    assert [g - t if g > t // 2 else g for g in got] == want


def test_dense64_plan_wraps_mod_t():
    # the square of a 64-term dot product can exceed t = 65537: compare mod t
    n, t = 4096, 65537
    Wd, x = W.dense_weights(), W.dense_vector()
    want = [v % t for v in lola.int_square(lola.int_dense(x, Wd))]
    ev = Counting(n, t)
    v, pos = lola.pack_stacked(x, 6, W.dense64_input_copies(Wd), n)
    st = lola.run_network(ev, W.layers_dense64(Wd, n), lola.State([np.array(v, np.int64)], pos, 64, 16))
    assert ev.c == {"rot": 6, "mul_plain": 1, "mul_scalar": 0, "square": 1}
    assert [int(st.msgs[m][s]) for m, s in st.pos] == want


# --------------------------------------------------------- encrypted runs

def test_dense64_encrypted_oracle_run():
    ps = W.params_dense64()
    P = bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)
    keys = bfv.keygen(P, W.DEFAULT_SEED, rotations=[1, 2, 4, 8, 16, 32], relin=True)
    t = 65537
    Wd, x = W.dense_weights(), W.dense_vector()
    v, pos = lola.pack_stacked(x, 6, 16, ps.n)
    ct = bfv.encrypt(P, keys.pk, encoding.encode(v, t), t, 1, 0)
    ev = lola.HEEval(P, keys, t)
    st = lola.run_network(ev, W.layers_dense64(Wd, ps.n), lola.State([ct], pos, 64, 16))
    slots = encoding.decode(bfv.decrypt(P, keys.sk, st.msgs[0]), t)
    want = [v % t for v in lola.int_square(lola.int_dense(x, Wd))]
    assert [int(slots[s]) for _, s in st.pos] == want
    # the margin left after the square (recorded in the design notes)
    sim = lola.run_network(lola.SlotEval(ps.n, t), W.layers_dense64(Wd, ps.n),
                           lola.State([np.array(v, np.int64)], pos, 64, 16))
    margin = bfv.noise_margin_bits(P, keys.sk, st.msgs[0], encoding.encode(sim.msgs[0], t))
    assert margin > 8


def mini_mnist():
    # a reduced MNIST-shaped network: 12x12 image, 3x3 stride-2 conv, 2 maps,
    # 12 hidden (two stacked rounds, so masks + combine run), 3 outputs
    net = W.mnist_net(seed=7, maps=2, hidden=12, classes=3, h=12, w=12, k=3, stride=2)
    return net, W.image(seed=7, h=12, w=12)


def test_mini_mnist_encrypted_oracle_run():
    n = 1024
    ps = W.params_small(n, L=5, K=1, t=W.T30[:1])
    P = bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)
    net, img = mini_mnist()
    layers = W.layers_mnist(net, n)
    assert layers[3]["copies"] == 8 and -(-12 // 8) == 2
    steps = sorted({36, 128, 256, 1, 2, 4, 8, 16, 32, 64} | set(1 << j for j in range(9)))
    keys = bfv.keygen(P, 11, rotations=steps, relin=True, row_swap=True)
    t = ps.t[0]
    msgs, pos = lola.pack_convolution(img, net.kh, net.kw, net.stride, n)
    cts = [bfv.encrypt(P, keys.pk, encoding.encode(m, t), t, 5, i) for i, m in enumerate(msgs)]
    ev = lola.HEEval(P, keys, t)
    st = lola.run_network(ev, layers, lola.State(cts, pos))
    got = [int(encoding.decode(bfv.decrypt(P, keys.sk, st.msgs[m]), t)[s]) for m, s in st.pos]
    # one ~30-bit modulus: the outputs wrap, so compare mod t
    assert got == [v % t for v in mnist_int(net, img)]
    assert ev.counts["rot"] == 1 + 3 + 2 * 7 + 1 + 3 * 10


def test_dense_rowmajor_then_sparse_colmajor_chain():
    # M1 (dense -> sparse) then M2 (sparse -> dense), checked against the
    # integer product W2 (W1 x) on the slot simulator
    n, t = 256, W.T30[0]
    g = np.random.default_rng(4)
    x = g.integers(0, 16, 40)
    W1 = g.integers(-3, 4, (6, 40))
    W2 = g.integers(-3, 4, (9, 6))
    layers = [{"op": "dense_rowmajor", "weights": W1}, {"op": "sparse_colmajor", "weights": W2}]
    ev = Counting(n, t)
    v, pos = lola.pack_dense(x, n)
    st = lola.run_network(ev, layers, lola.State([np.array(v, np.int64)], pos))
    want = lola.int_dense(lola.int_dense(x, W1), W2)
    got = [int(st.msgs[m][s]) for m, s in st.pos]
    assert [v2 - t if v2 > t // 2 else v2 for v2 in got] == want
    # M1: log2(n) rotations per output (7 within a row of 128, then the row swap); M2: none
    assert ev.c["rot"] == 6 * 8 and ev.c["mul_plain"] == 6 + 6


# ------------------------------------------------------------- LoLa-Dense (App. C)

def lola_dense_slot_run(n, t, net, img, ev_cls=lola.SlotEval, width=W.DENSE_IMAGE_WIDTH):
    ev = ev_cls(n, t)
    v, pos = lola.pack_image_rows(img, width, n)
    st = lola.State([np.array(v, dtype=np.int64) % t], pos)
    return ev, lola.run_network(ev, W.layers_lola_dense(net, n, width), st)


def test_masked_shifts_equal_convolution_representation():
    # App. C: masking the dense image gives the convolution representation;
    # message r = dr*kw + dc holds pixel (2i+dr, 2j+dc) of window (i, j),
    # zero in the padding, brute-forced from the image itself.
    n, t = 4096, 65537
    net = W.mnist_net()
    img = W.image(idx=4)
    v, pos = lola.pack_image_rows(img, W.DENSE_IMAGE_WIDTH, n)
    ev = lola.SlotEval(n, t)
    st = lola.layer_masked_shifts(ev, lola.State([np.array(v, np.int64)], pos), W.conv_gather(net))
    assert len(st.msgs) == 25 and len(st.pos) == 169
    for r in range(25):
        dr, dc = divmod(r, 5)
        for e, (_, slot) in enumerate(st.pos):
            i, j = divmod(e, 13)
            assert slot == 2 * W.DENSE_IMAGE_WIDTH * i + 2 * j
            rr, cc = 2 * i + dr, 2 * j + dc
            want = int(img[rr, cc]) if rr < 28 and cc < 28 else 0
            assert int(st.msgs[r][slot]) == want, (r, e)
    # and only those slots of each message are nonzero
    live = {slot for _, slot in st.pos}
    for m in st.msgs:
        assert all(int(x) == 0 for s, x in enumerate(m) if s not in live)


def test_masked_shifts_rejects_a_non_shift_gather():
    n = 256
    st = lola.State([np.zeros(n, np.int64)], [(0, s) for s in range(8)])
    with pytest.raises(AssertionError):
        lola.layer_masked_shifts(lola.SlotEval(n, 17), st, [[0, 1], [2, 4]])


def test_lola_dense_plan_matches_integer_network_with_crt():
    n = 16384
    net = W.mnist_net()
    img = W.image(idx=1)
    want = mnist_int(net, img)
    layers = W.layers_lola_dense(net, n)
    # 845 values combined by shifts [0, 1, 26, 27, 748] span 1469 slots, so
    # 2048-slot blocks: 8 copies, 13 rounds (the paper's 16 copies need a
    # span below 1024, which no placement of 5 shifted corner grids reaches)
    assert layers[2]["shifts"] == [0, 1, 26, 27, 748]
    assert layers[4]["d"] == 11 and layers[4]["copies"] == 8
    per_t = []
    for t in W.T30[:3]:
        ev, st = lola_dense_slot_run(n, t, net, img, Counting)
        # 24 alignment + 4 combine + 3 stack + 13*11 + 12 stacked + 10*14 interleaved
        assert ev.c == {"rot": 24 + 4 + 3 + 13 * 11 + 12 + 140, "mul_plain": 25 + 13 + 13 + 10,
                        "mul_scalar": 125, "square": 2}
        per_t.append([int(st.msgs[m][s]) for m, s in st.pos])
    assert [crt([r[o] for r in per_t], W.T30[:3]) for o in range(10)] == want


def mini_lola_dense_layers(n):
    net, img = mini_mnist()
    width = 13                                   # 12 pixels per line + 1 padding column
    return net, img, width, W.layers_lola_dense(net, n, width)


def test_mini_lola_dense_encrypted_oracle_run():
    n = 1024
    ps = W.params_small(n, L=5, K=1, t=W.T30[:1])
    P = bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)
    net, img, width, layers = mini_lola_dense_layers(n)
    t = ps.t[0]

    class Rec(lola.SlotEval):
        def __init__(self, n, t):
            super().__init__(n, t)
            self.steps = set()

        def rot(self, a, k):
            self.steps.add(k)
            return super().rot(a, k)

    v, pos = lola.pack_image_rows(img, width, n)
    rec = Rec(n, t)
    sim = lola.run_network(rec, layers, lola.State([np.array(v, np.int64) % t], pos))
    keys = bfv.keygen(P, 13, rotations=sorted(rec.steps), relin=True, row_swap=True)
    ct = bfv.encrypt(P, keys.pk, encoding.encode(v, t), t, 6, 0)
    ev = lola.HEEval(P, keys, t)
    st = lola.run_network(ev, layers, lola.State([ct], pos))
    got = [int(encoding.decode(bfv.decrypt(P, keys.sk, st.msgs[m]), t)[s]) for m, s in st.pos]
    assert got == [int(sim.msgs[m][s]) for m, s in sim.pos] == [x % t for x in mnist_int(net, img)]
    assert min(bfv.noise_margin_bits(P, keys.sk, c, encoding.encode(s, t)) for c, s in zip(st.msgs, sim.msgs)) > 4


# ------------------------------------------------------ CIFAR-shaped (Sec. 6.2)

def place_case(n):
    """Three messages of 9 values at slots 0..8; targets exercise no move, an
    in-row shift, a row change without shift, and a message split over both rows."""
    h = n // 2
    T = [e for e in range(9)]                                  # message 0 stays
    T += [h + e for e in range(9)]                             # message 1: row swap only
    T += [20 + e for e in range(4)] + [h + 40 + e for e in range(5)]   # message 2: split
    return T


def test_place_layer_puts_every_element_at_its_target():
    n, t = 256, 257
    rng = np.random.default_rng(3)
    vals = rng.integers(0, t, size=(3, 9))
    msgs = [np.zeros(n, np.int64) for _ in range(3)]
    for m in range(3):
        msgs[m][:9] = vals[m]
    st = lola.State(msgs, [(m, e) for m in range(3) for e in range(9)])
    T = place_case(n)
    ev = Counting(n, t)
    out = lola.layer_place(ev, st, T)
    want = np.zeros(n, np.int64)
    for idx, (m, e) in enumerate(st.pos):
        want[T[idx]] = vals[m][e]
    assert np.array_equal(out.msgs[0] % t, want) and out.pos == [(0, x) for x in T]
    # message 2 has two groups (masked); groups: m1 swap k=0, m2 (k=20, k=40 swap); one row swap
    assert ev.c["mul_plain"] == 2 and ev.c["rot"] == 2 + 1


def cifar_int(net, img):
    """Integer network: conv (padded image), square, second conv as its dense
    matrix, square, dense; exact over Z (Python ints after the first square)."""
    x = lola.int_conv(W.cifar_padded(img, net.pad), net.w1, net.k1, net.k1, net.stride)
    x = np.array(lola.int_square(x), dtype=np.int64)
    x = W.cifar_dense2(net) @ x                                 # |x| < 2^43: exact in int64
    x = lola.int_square([int(v) for v in x])
    return lola.int_dense(x, net.w3)


def mini_cifar():
    net = W.cifar_net(seed=9, C=2, h=8, w=8, pad=2, k1=4, maps1=6, k2=2, maps2=3, classes=2)
    return net, W.cifar_image(seed=9, C=2, h=8, w=8)


def test_mini_cifar_encrypted_oracle_run():
    n = 1024
    ps = W.params_small(n, L=5, K=1, t=W.T30[:1])
    P = bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)
    net, img = mini_cifar()
    layers = W.layers_cifar(net, n)
    t = ps.t[0]
    msgs, pos = lola.pack_convolution(W.cifar_padded(img, net.pad), net.k1, net.k1, net.stride, n)
    assert len(msgs) == 2 * 16 and len(pos) == 16
    rec = Counting(n, t)
    sim = lola.run_network(rec, layers, lola.State([np.array(m, np.int64) % t for m in msgs], pos))
    want = [x % t for x in cifar_int(net, img)]
    assert [int(sim.msgs[m][s]) for m, s in sim.pos] == want
    steps = set()

    class Rec(lola.SlotEval):
        def rot(self, a, k):
            steps.add(k)
            return super().rot(a, k)
    lola.run_network(Rec(n, t), layers, lola.State([np.array(m, np.int64) % t for m in msgs], pos))
    keys = bfv.keygen(P, 17, rotations=sorted(steps), relin=True, row_swap=True)
    cts = [bfv.encrypt(P, keys.pk, encoding.encode(m, t), t, 8, i) for i, m in enumerate(msgs)]
    st = lola.run_network(lola.HEEval(P, keys, t), layers, lola.State(cts, pos))
    got = [int(encoding.decode(bfv.decrypt(P, keys.sk, st.msgs[m]), t)[s]) for m, s in st.pos]
    assert got == want


def test_cifar_plan_matches_integer_network():
    n, t = 16384, W.T30[0]
    net = W.cifar_net()
    img = W.cifar_image(idx=2)
    layers = W.layers_cifar(net, n)
    msgs, pos = lola.pack_convolution(W.cifar_padded(img, net.pad), net.k1, net.k1, net.stride, n)
    assert len(msgs) == 192 and len(pos) == 196          # Sec. 6.2: 3 x 8 x 8 messages
    ev = Counting(n, t)
    st = lola.run_network(ev, layers, lola.State([np.array(m, np.int64) % t for m in msgs], pos))
    assert [int(st.msgs[m][s]) for m, s in st.pos] == [x % t for x in cifar_int(net, img)]
    # place: 40 + 40 + 2 shifted groups + 1 row swap; 4075 + 10 outputs x 14 rotations
    assert ev.c == {"rot": 83 + 4085 * 14, "mul_plain": 2 + 4075 + 4075 + 10, "mul_scalar": 83 * 192,
                    "square": 2}


def test_cifar_second_convolution_matrix_is_the_convolution():
    # the dense matrix the second layer is evaluated as equals a direct
    # 6x6x83 stride-2 convolution of the 14x14x83 first-layer output
    net = W.cifar_net()
    D = W.cifar_dense2(net)
    maps1, o1, o2, k2, s = net.w1.shape[0], net.o1, net.o2, net.k2, net.stride
    h1 = np.random.default_rng(6).integers(-50, 50, size=(maps1, o1, o1))
    direct = []
    for o in range(net.w2.shape[0]):
        K = net.w2[o].reshape(maps1, k2, k2)
        for i in range(o2):
            for j in range(o2):
                direct.append(int((K * h1[:, s * i:s * i + k2, s * j:s * j + k2]).sum()))
    assert [int(v) for v in D @ h1.reshape(-1)] == direct


@pytest.mark.slow
def test_full_mnist_with_modulus_switching_keeps_its_noise_margin():
    """The MNIST-shaped network at full size (n = 16384, L = 5) with the
    modulus switches of workloads.MNIST_LEVELS (4 primes after the first
    square, 2 after the second), encrypted in the oracle for one CRT
    residue: the output decrypts to the integer network mod t with more than
    20 bits of noise margin (about a minute on one core)."""
    n = 16384
    ps = W.params_mnist()
    P = bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)
    t = ps.t[0]
    net, img = W.mnist_net(), W.image()
    layers = W.layers_mnist(net, n, W.MNIST_LEVELS)
    steps = sorted({169, 338, 507, 676} | {1 << j for j in range(13)} | set(range(1, 7)))
    keys = bfv.keygen(P, W.DEFAULT_SEED, rotations=steps, relin=True, row_swap=True)
    msgs, pos = lola.pack_convolution(img, net.kh, net.kw, net.stride, n)
    cts = [bfv.encrypt(P, keys.pk, encoding.encode(m, t), t, 5, i) for i, m in enumerate(msgs)]
    ev = lola.HEEval(P, keys, t)
    st = lola.run_network(ev, layers, lola.State(cts, pos))
    assert ev.p.L == W.MNIST_LEVELS[1] and all(len(c.c[0]) == ev.p.L for c in st.msgs)
    want = [v % t for v in mnist_int(net, img)]
    got = [int(encoding.decode(bfv.decrypt(ev.p, keys.sk, st.msgs[m]), t)[s]) for m, s in st.pos]
    assert got == want
    for m in range(2):
        vals = np.zeros(n, dtype=np.int64)
        vals[:] = want[m]                       # sparse output: the value in every slot
        margin = bfv.noise_margin_bits(ev.p, keys.sk, st.msgs[m], encoding.encode(vals, t))
        assert margin > 20, margin


# ------------------------------- row-major product summed over the support

def test_support_sum_shifts_against_brute_force():
    # for random supports built as (run mod period) lattices, and a few
    # irregular ones, the chosen shifts are the fewest of every (period, run)
    # choice checked by brute force, and the result slot holds every
    # occupied slot exactly once
    import itertools
    n = 64
    h = n // 2
    g = np.random.default_rng(9)
    cases = [list(range(n)), [5], [3, 40], [1, 2, 9, 10, 17, 18, 25, 26]]
    for _ in range(20):
        lp = int(g.integers(0, 6))
        per = 1 << lp
        run = int(g.integers(1, per + 1))
        o = int(g.integers(0, per))
        rows = [0] if g.random() < 0.5 else [0, 1]
        cols = [c for c in range(h) if (c - o) % per < run and g.random() < 0.8] or [o]
        cases.append([r * h + c for r in rows for c in cols])
    for slots in cases:
        shifts, p = lola.support_sum_shifts(slots, n)
        # exactly-once coverage at p, by brute force over subset sums
        cover = {}
        rowswap = 0 in shifts
        row_shifts = [s for s in shifts if s]
        for sub in itertools.product([0, 1], repeat=len(row_shifts)):
            off = sum(s for s, b in zip(row_shifts, sub) if b)
            for sw in ([0, 1] if rowswap else [0]):
                src_row = (p // h) ^ sw
                src = src_row * h + ((p % h) - off) % h
                cover[src] = cover.get(src, 0) + 1
        assert all(cover.get(s, 0) == 1 for s in set(slots)), (slots, shifts, p)
        # no (period, run) choice does it in fewer steps
        logh = h.bit_length() - 1
        best = min(k + (logh - q) + (1 if len({s // h for s in slots}) > 1 else 0)
                   for q in range(logh + 1) for k in range(q + 1)
                   if any(all(((c % h) - o2) % (1 << q) < (1 << k) for c in slots) for o2 in range(1 << q)))
        assert len(shifts) == best


def test_mnist_support_sum_plan_matches_integer_network():
    # the MNIST-shaped plan with the support-summed last layer: 7 rotations
    # per output instead of 14 (154 per residue instead of 224), same outputs
    n = 16384
    net, img = W.mnist_net(), W.image(idx=4)
    want = mnist_int(net, img)
    layers = W.layers_mnist(net, n, W.MNIST_LEVELS, support_sum=True)
    msgs, pos = lola.pack_convolution(img, net.kh, net.kw, net.stride, n)
    for t in W.T30[:3]:
        ev = Counting(n, t)
        st = lola.run_network(ev, layers, lola.State([np.array(m, np.int64) % t for m in msgs], pos))
        assert ev.c["rot"] == 224 - 70 and ev.c["square"] == 2
        assert [int(st.msgs[m][s]) for m, s in st.pos] == [v % t for v in want]
        assert len({s for _, s in st.pos}) == 1                 # one result slot for all outputs


def test_support_sum_on_ciphertexts_small():
    # the same layer on oracle ciphertexts (n = 64): decrypts to the dot products
    n, t = 64, W.T30[0]
    P = bfv.Params(n, W.Q60[:4], 3, 1, [t])
    keys = bfv.keygen(P, 3, rotations=[1, 2, 4, 8, 16], relin=False, row_swap=True)
    g = np.random.default_rng(10)
    slots = [0, 1, 2, 16, 17, 18, 32, 33, 34, 48, 49, 50]     # runs of 3 every 16 slots, both rows
    x = g.integers(0, 16, len(slots))
    Wm = g.integers(-3, 4, (3, len(slots)))
    v = np.zeros(n, np.int64)
    v[slots] = x
    ct = bfv.encrypt(P, keys.pk, encoding.encode(v, t), t, 4, 0)
    st = lola.run_network(lola.HEEval(P, keys, t), [{"op": "interleaved_rowmajor_support", "weights": Wm}],
                          lola.State([ct], [(0, s) for s in slots]))
    for o, (m, s) in enumerate(st.pos):
        dec = encoding.decode(bfv.decrypt(P, keys.sk, st.msgs[m]), t)
        assert int(dec[s]) == int(np.dot(Wm[o], x)) % t


# ------------------------------------------------ hoisted rotate-and-sum groups

def test_hoist_groups_examples():
    n = 64                                       # rows of 32 slots
    assert lola.hoist_groups([1, 2, 4, 8, 16], 1, n) == [[1], [2], [4], [8], [16]]
    assert lola.hoist_groups([1, 2, 4, 8, 16], 2, n) == [[1, 2, 3], [4, 8, 12], [16]]
    assert lola.hoist_groups([1, 2, 4, 0, 8], 3, n) == [[1, 2, 3, 4, 5, 6, 7], [0], [8]]
    assert lola.hoist_groups([16, 16], 2, n) == [[16], [16]]          # 16 + 16 = 0 mod 32: no rotation
    assert lola.hoist_groups([8, 16], 2, n) == [[8, 16, 24]]


@pytest.mark.parametrize("m", [2, 3, 4])
def test_hoisted_rotate_and_sum_equals_the_doubling_steps(m):
    # brute force on slot vectors: every grouping gives the sequential sum
    n, t = 64, 65537
    g = np.random.default_rng(m)
    ev = lola.SlotEval(n, t)
    for trial in range(20):
        shifts = [int(x) for x in g.integers(0, n // 2, g.integers(1, 8))]
        x = g.integers(0, t, n)
        assert np.array_equal(lola.rotate_and_sum(ev, x, shifts, m), lola.rotate_and_sum(ev, x, shifts, 1)), shifts


def test_mini_mnist_hoisted_encrypted_oracle_run():
    # the reduced MNIST-shaped network with the rotate-and-sums hoisted two
    # steps per key switch (three in the last layer): same outputs, fewer
    # key switches
    n = 1024
    ps = W.params_small(n, L=5, K=1, t=W.T30[:1])
    P = bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)
    net, img = mini_mnist()
    layers = W.layers_mnist(net, n, support_sum=True, hoist=(2, 2, 3))
    t = ps.t[0]
    msgs, pos = lola.pack_convolution(img, net.kh, net.kw, net.stride, n)
    steps = set()

    class Rec(lola.SlotEval):
        def rot(self, a, k):
            steps.add(k)
            return super().rot(a, k)

        def rot_rows(self, a):
            steps.add(0)
            return super().rot_rows(a)
    lola.run_network(Rec(n, t), layers, lola.State([np.array(m, np.int64) % t for m in msgs], pos))
    keys = bfv.keygen(P, 12, rotations=sorted(s for s in steps if s), relin=True, row_swap=0 in steps)
    cts = [bfv.encrypt(P, keys.pk, encoding.encode(m, t), t, 5, i) for i, m in enumerate(msgs)]
    ev = lola.HEEval(P, keys, t)
    st = lola.run_network(ev, layers, lola.State(cts, pos))
    got = [int(encoding.decode(bfv.decrypt(P, keys.sk, st.msgs[m]), t)[s]) for m, s in st.pos]
    assert got == [v % t for v in mnist_int(net, img)]
    # key switches: combine 1; stack [128, 256 | row swap] 1 + 1; stacked
    # row-major 2 rounds x [1, 2 | 4, 8 | 16, 32 | 64] 2 x (3 + 1); round
    # combine 1; last layer 3 outputs x 4 support steps as 3 + 1: 3 x (1 + 1)
    # -> 8 single rotations and 10 rotate-sums (31 rotations without hoisting)
    assert (ev.counts["rot"], ev.counts["rot_sum"]) == (8, 10)


def test_hoisted_head_and_cifar_plans_match_integer_network():
    # the plans bench.py runs: the head's stack and stacked row-major and
    # CIFAR's two row-major products hoisted three doubling steps per key
    # switch, CIFAR's last product summed over its 4075 occupied slots
    n, t = 16384, W.T30[0]
    Wh, x = W.head_weights(), W.feature_vector()
    v, pos = lola.pack_dense(x, n)
    st = lola.run_network(lola.SlotEval(n, t), W.layers_head(Wh, n, W.HEAD_HOIST),
                          lola.State([np.array(v, np.int64) % t], pos))
    got = [int(st.msgs[m][s]) for m, s in st.pos]
    assert [g - t if g > t // 2 else g for g in got] == lola.int_dense(x, Wh)
    net, img = W.cifar_net(), W.cifar_image(idx=2)
    msgs, pos = lola.pack_convolution(W.cifar_padded(img, net.pad), net.k1, net.k1, net.stride, n)
    st = lola.run_network(lola.SlotEval(n, t), W.layers_cifar(net, n, hoist=W.CIFAR_HOIST, support_sum=True),
                          lola.State([np.array(m, np.int64) % t for m in msgs], pos))
    assert [int(st.msgs[m][s]) for m, s in st.pos] == [x % t for x in cifar_int(net, img)]
