"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module holds parameter tables (literal prime lists) and seeded input
generators only: no part of the method's arithmetic.  It is the one module
that both the CUDA path's callers and the CPU oracle import.

The paper evaluates on MNIST, CIFAR-10 and CalTech-101 features with trained
weights; none of those are available, so every input here is synthetic with
the paper's shapes (Sec. 4.3 MNIST network, Sec. 5 transfer-learning head):
pixel / feature values uniform in [0, 15] and weights uniform in [-3, 3],
drawn from numpy's Philox generator seeded per purpose.

Prime lists: NTT-friendly primes (= 1 mod 2n), listed in descending order
below 2^60 (ciphertext primes), 2^36 (n = 4096 set) and 2^30 (plaintext
CRT moduli).  Each side validates them with its own code.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 20181225

# primes = 1 mod 2^15 below 2^60, descending
Q60 = [
    1152921504606748673, 1152921504606683137, 1152921504606584833,
    1152921504605962241, 1152921504604979201, 1152921504600260609,
    1152921504599080961, 1152921504598720513, 1152921504597114881,
    1152921504597016577, 1152921504596525057, 1152921504595968001,
]
# primes = 1 mod 2^13 below 2^36, descending
Q36 = [68719403009, 68719230977, 68719206401, 68719190017]
# plaintext CRT moduli: primes = 1 mod 2^15 below 2^30, descending
T30 = [1073643521, 1073479681, 1073184769, 1073053697]


@dataclass
class ParamSet:
    name: str
    n: int
    q: list          # L + K primes, special primes last
    L: int
    K: int
    t: list
    alpha: int = 1   # ciphertext primes per key-switching digit

    def as_dict(self):
        return dict(n=self.n, q=list(self.q), L=self.L, K=self.K, t=list(self.t), alpha=self.alpha)


def params_dense64() -> ParamSet:
    """Single encrypted dense layer: n = 4096, three ~36-bit primes, no
    special prime, t = 65537."""
    return ParamSet("dense64_n4096", 4096, Q36[:3], 3, 0, [65537])


def params_mnist(L: int = 5) -> ParamSet:
    """MNIST-shaped network: n = 16384, L ciphertext primes of 60 bits plus
    one 60-bit special prime, one-prime key-switching digits, three ~30-bit
    plaintext CRT moduli.  bench.py runs the network on params_mnist_grouped
    (digits of two primes): with the hoisted rotate-and-sums the inner
    products weigh more than the second special prime's transforms, 492.7
    against 462.8 inferences/s (without hoisting it was the other way,
    262.9 against 269.0)."""
    return ParamSet(f"mnist_n16384_L{L}", 16384, Q60[:L + 1], L, 1, T30[:3])


def params_mnist_grouped(L: int = 5) -> ParamSet:
    """The MNIST-shaped network's parameters with key-switching digits of two
    primes (the last one single when L is odd) and two 60-bit special
    primes (420 bits at L = 5, within the 438-bit budget; +25.2 bits of
    noise margin at the output of the oracle's full-size run, against +24.2
    with one-prime digits).  The parameter set bench.py times."""
    return ParamSet(f"mnist_grouped_n16384_L{L}", 16384, Q60[:L + 2], L, 2, T30[:3], alpha=2)


def params_lola_dense(L: int = 6) -> ParamSet:
    """LoLa-Dense (App. C): n = 16384, six 60-bit primes plus one 60-bit
    special prime (420 bits, within the 438-bit budget; a second special
    prime would exceed it), one-prime key-switching digits, three ~30-bit
    plaintext CRT moduli."""
    return ParamSet(f"lola_dense_n16384_L{L}", 16384, Q60[:L + 1], L, 1, T30[:3])


def params_cifar(L: int = 6) -> ParamSet:
    """CIFAR-shaped network (Sec. 6.2): n = 16384, L 60-bit primes plus a
    60-bit special prime, three ~30-bit plaintext CRT moduli."""
    return ParamSet(f"cifar_n16384_L{L}", 16384, Q60[:L + 1], L, 1, T30[:3])


def params_head(L: int = 3) -> ParamSet:
    """Transfer-learning head: 60-bit primes as params_mnist, one plaintext
    modulus.  The head is linear (no square), so three primes suffice: the
    oracle's exact noise measurement at n = 16384 ends at +40.5 bits (two
    primes: -14.8)."""
    return ParamSet(f"head_n16384_L{L}", 16384, Q60[:L + 1], L, 1, T30[:1])


def params_sweep(n: int, L: int, alpha: int = 1) -> ParamSet:
    """Batched primitive sweep: n in {8192, 16384}, L in 4..8 primes of 60
    bits plus a special prime, or two with key-switching digits of two primes
    (alpha = 2); security not considered: random residues."""
    K = 2 if alpha == 2 else 1
    return ParamSet(f"sweep_n{n}_L{L}_a{alpha}", n, Q60[:L + K], L, K, T30[:1], alpha)


def params_small(n: int, L: int = 3, K: int = 1, t=None, alpha: int = 1) -> ParamSet:
    """Reduced ring sizes for fast parity tests (same 60-bit primes)."""
    return ParamSet(f"small_n{n}_L{L}_K{K}_a{alpha}", n, Q60[:L + K], L, K, list(t or T30[:1]), alpha)


def rng(seed: int, purpose: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & (2**64 - 1), purpose]))


# purposes
P_IMAGE, P_CONV_W, P_DENSE1_W, P_DENSE2_W, P_FEAT, P_HEAD_W, P_VEC, P_DENSE_W, \
    P_RESIDUES, P_STEPS, P_ENC, P_KEY, P_CIFAR_IMG, P_CIFAR_W1, P_CIFAR_W2, P_CIFAR_W3 = range(1, 17)


def image(seed=DEFAULT_SEED, idx: int = 0, h: int = 28, w: int = 28) -> np.ndarray:
    return rng(seed + idx, P_IMAGE).integers(0, 16, size=(h, w), dtype=np.int64)


def int_weights(seed, purpose, shape) -> np.ndarray:
    return rng(seed, purpose).integers(-3, 4, size=shape, dtype=np.int64)


@dataclass
class MnistNet:
    conv_w: np.ndarray = field(repr=False)     # (maps, kh*kw)
    dense1_w: np.ndarray = field(repr=False)   # (hidden, maps*oh*ow)
    dense2_w: np.ndarray = field(repr=False)   # (classes, hidden)
    kh: int = 5
    kw: int = 5
    stride: int = 2
    h: int = 28
    w: int = 28


def mnist_net(seed=DEFAULT_SEED, maps=5, hidden=100, classes=10, h=28, w=28, k=5, stride=2) -> MnistNet:
    oh = -(-(h - k) // stride) + 1
    ow = -(-(w - k) // stride) + 1
    return MnistNet(int_weights(seed, P_CONV_W, (maps, k * k)),
                    int_weights(seed, P_DENSE1_W, (hidden, maps * oh * ow)),
                    int_weights(seed, P_DENSE2_W, (classes, hidden)), k, k, stride, h, w)


@dataclass
class CifarNet:
    """Sec. 6.2 / App. D, after collapsing adjacent linear layers: k1 x k1 x C
    convolution, stride 2, maps1 maps; square; k2 x k2 x maps1 convolution,
    stride 2, maps2 maps (evaluated as a dense layer); square; dense layer
    with `classes` outputs.  The image is zero-padded bottom/right by `pad`
    (34 x 34 from 32 x 32 gives the paper's 14 x 14 windows: 83 * 196 = 16268
    first-layer nodes, 163 * 25 = 4075 second-layer nodes)."""
    w1: np.ndarray = field(repr=False)     # (maps1, C*k1*k1)
    w2: np.ndarray = field(repr=False)     # (maps2, maps1*k2*k2)
    w3: np.ndarray = field(repr=False)     # (classes, maps2*o2*o2)
    C: int = 3
    h: int = 32
    w: int = 32
    pad: int = 2
    k1: int = 8
    k2: int = 6
    stride: int = 2

    @property
    def o1(self) -> int:
        return -(-(self.h + self.pad - self.k1) // self.stride) + 1

    @property
    def o2(self) -> int:
        return (self.o1 - self.k2) // self.stride + 1


def cifar_net(seed=DEFAULT_SEED, C=3, h=32, w=32, pad=2, k1=8, maps1=83, k2=6, maps2=163, classes=10,
              stride=2) -> CifarNet:
    o1 = -(-(h + pad - k1) // stride) + 1
    o2 = (o1 - k2) // stride + 1
    return CifarNet(int_weights(seed, P_CIFAR_W1, (maps1, C * k1 * k1)),
                    int_weights(seed, P_CIFAR_W2, (maps2, maps1 * k2 * k2)),
                    int_weights(seed, P_CIFAR_W3, (classes, maps2 * o2 * o2)), C, h, w, pad, k1, k2, stride)


def cifar_image(seed=DEFAULT_SEED, idx: int = 0, C=3, h=32, w=32) -> np.ndarray:
    return rng(seed + idx, P_CIFAR_IMG).integers(0, 16, size=(C, h, w), dtype=np.int64)


def cifar_padded(img: np.ndarray, pad: int) -> np.ndarray:
    """Zero rows and columns appended bottom/right (the client pads before packing)."""
    C, h, w = img.shape
    out = np.zeros((C, h + pad, w + pad), dtype=np.int64)
    out[:, :h, :w] = img
    return out


def cifar_dense2(net: CifarNet) -> np.ndarray:
    """The second convolution as the dense matrix it is evaluated as: row
    (o, i, j) (map-major, windows row-major) over the first layer's outputs
    (map-major, windows row-major)."""
    maps2, maps1 = net.w2.shape[0], net.w1.shape[0]
    o1, o2, k2, s = net.o1, net.o2, net.k2, net.stride
    M = np.zeros((maps2 * o2 * o2, maps1 * o1 * o1), dtype=np.int64)
    # column of kernel entry (ch, dr, dc), in the kernel's own order, for window (0, 0)
    ch, dr, dc = np.meshgrid(np.arange(maps1), np.arange(k2), np.arange(k2), indexing="ij")
    off = (ch * o1 * o1 + dr * o1 + dc).reshape(-1)
    for o in range(maps2):
        for i in range(o2):
            for j in range(o2):
                M[(o * o2 + i) * o2 + j, s * i * o1 + s * j + off] = net.w2[o]
    return M


def feature_vector(seed=DEFAULT_SEED, idx: int = 0, dim: int = 4096) -> np.ndarray:
    return rng(seed + idx, P_FEAT).integers(0, 16, size=dim, dtype=np.int64)


def head_weights(seed=DEFAULT_SEED, classes: int = 101, dim: int = 4096) -> np.ndarray:
    return int_weights(seed, P_HEAD_W, (classes, dim))


def dense_vector(seed=DEFAULT_SEED, dim: int = 64) -> np.ndarray:
    return rng(seed, P_VEC).integers(0, 16, size=dim, dtype=np.int64)


def dense_weights(seed=DEFAULT_SEED, rows: int = 10, dim: int = 64) -> np.ndarray:
    return int_weights(seed, P_DENSE_W, (rows, dim))


def random_residues(seed, shape_prefix, primes, n) -> np.ndarray:
    """Uniform residues: array of shape shape_prefix + (len(primes), n), row j mod primes[j]."""
    g = rng(seed, P_RESIDUES)
    out = np.empty(tuple(shape_prefix) + (len(primes), n), dtype=np.uint64)
    for j, p in enumerate(primes):
        out[..., j, :] = g.integers(0, p, size=tuple(shape_prefix) + (n,), dtype=np.uint64)
    return out


def rotation_steps(seed, count: int, n: int) -> np.ndarray:
    """Random rotation steps in [1, n/2)."""
    return rng(seed, P_STEPS).integers(1, n // 2, size=count, dtype=np.int64)


# ----------------------------------------------------------- layer lists
# Network descriptions (weights + representation choices), consumed by both
# the oracle's plan and the library's layer-list API.

def _ceil_log2(k: int) -> int:
    return max(0, (k - 1).bit_length())


# Rotate-and-sum doubling steps per key switch (stack, stacked row-major,
# last layer) of the MNIST-shaped network and LoLa-Dense, and of the single
# dense layer: three steps (seven rotations) per key switch, the fastest of
# the groupings measured on the MNIST network (1, 2, 3, (2, 3, 3), (3, 3, 4)).
MNIST_HOIST = (3, 3, 3)
LOLA_DENSE_HOIST = (3, 3, 3)
DENSE64_HOIST = 3
HEAD_HOIST = 3
CIFAR_HOIST = (3, 3, 3)

# Ciphertext primes kept after each square of the MNIST-shaped network at
# L = 5: the oracle's exact noise measurement (full network, n = 16384)
# leaves a 23-bit margin at the output either way, because modulus switching
# divides the noise with Q while it is far above the rounding term.
MNIST_LEVELS = (4, 2)


def _hoist3(hoist) -> tuple:
    """(stack, stacked row-major, last layer) rotate-and-sum steps per key switch."""
    h = (hoist,) * 3 if isinstance(hoist, int) else tuple(hoist)
    assert len(h) == 3
    return h


def _with_hoist(layer: dict, m: int) -> dict:
    return {**layer, "hoist": m} if m > 1 else layer


def layers_mnist(net: MnistNet, n: int, levels=None, support_sum: bool = False, hoist=1) -> list:
    """Sec. 4.3 / Table 1: conv (convolution representation) -> combine maps
    -> square -> stack -> stacked row-major dense -> square -> interleaved
    row-major dense.  levels = (L1, L2): switch modulus to L1 primes after the
    first square and to L2 after the second (None: no switching).
    support_sum: the last layer sums each dot product over the interleaved
    vector's occupied slots only (7 rotations per output at n = 16384
    instead of the paper's 14; output o at one slot of message o).
    hoist: rotate-and-sum doubling steps per key switch in the stack, the
    stacked row-major and the last layer (an int for all three, or a
    3-tuple; 1 = one key switch per step)."""
    hs, hr, hl = _hoist3(hoist)
    maps, hidden = net.conv_w.shape[0], net.dense1_w.shape[0]
    oh = -(-(net.h - net.kh) // net.stride) + 1
    ow = -(-(net.w - net.kw) // net.stride) + 1
    k1 = maps * oh * ow
    d = _ceil_log2(k1)
    copies = n >> d
    ms = ([{"op": "mod_switch", "L": levels[0]}], [{"op": "mod_switch", "L": levels[1]}]) if levels else ([], [])
    return [
        {"op": "conv", "weights": net.conv_w},
        {"op": "combine", "stride": oh * ow},
        {"op": "square"},
        *ms[0],
        _with_hoist({"op": "stack", "d": d, "copies": copies}, hs),
        _with_hoist({"op": "stacked_rowmajor", "weights": net.dense1_w, "d": d, "copies": copies}, hr),
        {"op": "square"},
        *ms[1],
        _with_hoist({"op": "interleaved_rowmajor_support" if support_sum else "interleaved_rowmajor",
                     "weights": net.dense2_w}, hl),
    ]


DENSE_IMAGE_WIDTH = 29   # line length of the dense image message: 28 pixels + 1 padding column


def dense_image_slots(h: int = 28, w: int = 28, width: int = DENSE_IMAGE_WIDTH) -> list:
    """Slots of the pixels of a dense image message, line after line (App. C)."""
    return [r * width + c for r in range(h) for c in range(w)]


def conv_gather(net: MnistNet) -> np.ndarray:
    """[kh*kw][windows] pixel index (row-major) that window offset r = dr*kw
    + dc reads at window (i, j); -1 in the zero padding."""
    oh = -(-(net.h - net.kh) // net.stride) + 1
    ow = -(-(net.w - net.kw) // net.stride) + 1
    G = np.full((net.kh * net.kw, oh * ow), -1, dtype=np.int64)
    for dr in range(net.kh):
        for dc in range(net.kw):
            for i in range(oh):
                for j in range(ow):
                    r, c = net.stride * i + dr, net.stride * j + dc
                    if r < net.h and c < net.w:
                        G[dr * net.kw + dc, i * ow + j] = r * net.w + c
    return G


def combine_shifts(slots, k: int) -> list:
    """Smallest right shifts, message by message, that place k copies of the
    slot pattern `slots` without collisions (shift 0 for message 0)."""
    base = sorted(slots)
    placed, shifts = set(base), [0]
    for _ in range(1, k):
        s = 1
        while any(p + s in placed for p in base):
            s += 1
        shifts.append(s)
        placed |= {p + s for p in base}
    return shifts


# LoLa-Dense and the CIFAR-shaped network at L = 6: primes kept after each
# square (oracle's exact noise measurement at n = 16384: +30.3 bits at the
# LoLa-Dense output, +32.7 at the CIFAR output of the 8-output reduction;
# the switch to 4 primes costs 17.5 bits because the noise falls to the
# rounding term there).
LOLA_DENSE_LEVELS = (4, 2)
CIFAR_LEVELS = (4, 2)


def _with_levels(layers: list, after_squares, levels) -> list:
    """Insert a modulus switch after the given layer indices (the squares)."""
    if not levels:
        return layers
    out = []
    for i, Ly in enumerate(layers):
        out.append(Ly)
        if i in after_squares:
            out.append({"op": "mod_switch", "L": levels[after_squares.index(i)]})
    return out


def layers_lola_dense(net: MnistNet, n: int, width: int = DENSE_IMAGE_WIDTH, levels=None,
                      support_sum: bool = False, hoist=1) -> list:
    """LoLa-Dense (App. C, Table 3): one dense image message masked into the
    convolution representation (window (i, j) at the slot of its upper-left
    pixel), convolution row-major, maps combined by collision-free shifts,
    square, stack, stacked row-major, square, interleaved row-major.
    levels = (L1, L2): modulus switching after the two squares; support_sum
    and hoist as in layers_mnist."""
    hs, hr, hl = _hoist3(hoist)
    G = conv_gather(net)
    slots = dense_image_slots(net.h, net.w, width)
    corner = [slots[int(g)] for g in G[0]]
    maps, hidden = net.conv_w.shape[0], net.dense1_w.shape[0]
    shifts = combine_shifts(corner, maps)
    span = max(corner) + shifts[-1] + 1
    d = _ceil_log2(span)
    copies = n >> d
    return _with_levels([
        {"op": "masked_shifts", "weights": G},
        {"op": "conv", "weights": net.conv_w},
        {"op": "combine", "shifts": shifts},
        {"op": "square"},
        _with_hoist({"op": "stack", "d": d, "copies": copies}, hs),
        _with_hoist({"op": "stacked_rowmajor", "weights": net.dense1_w, "d": d, "copies": copies}, hr),
        {"op": "square"},
        _with_hoist({"op": "interleaved_rowmajor_support" if support_sum else "interleaved_rowmajor",
                     "weights": net.dense2_w}, hl),
    ], [3, 6], levels)


def cifar_place_targets(maps: int, per_map: int, n: int) -> list:
    """Target slots for combining `maps` messages of `per_map` values (at
    slots 0..per_map-1) into one message over both slot rows: whole maps fill
    row 0 then row 1, a map that does not fit in what is left of row 0 is split
    between the tail of row 0 and the tail of row 1."""
    h = n // 2
    per_row = h // per_map
    assert maps * per_map <= n
    T = []
    for m in range(maps):
        for e in range(per_map):
            if m < per_row:
                t = m * per_map + e
            elif m < 2 * per_row:
                t = h + (m - per_row) * per_map + e
            else:                                   # split maps: row 0 tail, then row 1 tail
                k = (m - 2 * per_row) * per_map + e
                tail0 = h - per_row * per_map
                t = per_row * per_map + k if k < tail0 else h + per_row * per_map + (k - tail0)
            T.append(t)
    assert len(set(T)) == len(T) and max(T) < n
    return T


def layers_cifar(net: CifarNet, n: int, dense2: np.ndarray | None = None, levels=None, hoist=1,
                 support_sum: bool = False) -> list:
    """Sec. 6.2: convolution row-major on the convolution representation
    (C*k1*k1 messages), the maps combined into one message, square, the
    second convolution as dense row-major (sparse output), sparse -> dense by
    masks and additions (column-major with the identity), square, dense
    row-major.  levels = (L1, L2): modulus switching after the two squares.
    hoist: rotate-and-sum doubling steps per key switch in the two row-major
    products (an int, or a 3-tuple whose last two entries are used, as in
    layers_mnist); support_sum: the last product summed over the occupied
    slots of its dense input (output o at one slot of message o)."""
    _, h2, h3 = _hoist3(hoist)
    maps1 = net.w1.shape[0]
    per = net.o1 * net.o1
    D2 = cifar_dense2(net) if dense2 is None else dense2
    k2 = D2.shape[0]
    return _with_levels([
        {"op": "conv", "weights": net.w1},
        {"op": "place", "weights": np.array([cifar_place_targets(maps1, per, n)], dtype=np.int64)},
        {"op": "square"},
        _with_hoist({"op": "dense_rowmajor", "weights": D2}, h2),
        {"op": "sparse_colmajor", "weights": np.eye(k2, dtype=np.int64)},
        {"op": "square"},
        _with_hoist({"op": "interleaved_rowmajor_support" if support_sum else "dense_rowmajor",
                     "weights": net.w3}, h3),
    ], [2, 5], levels)


def layers_head(Wh: np.ndarray, n: int, hoist: int = 1) -> list:
    """Sec. 5 transfer-learning head as stacked row-major: dense input
    stacked n / 2^d times, then rounds of stacked row-major products.
    hoist: rotate-and-sum doubling steps per key switch."""
    d = _ceil_log2(Wh.shape[1])
    copies = n >> d
    return [
        _with_hoist({"op": "stack", "d": d, "copies": copies}, hoist),
        _with_hoist({"op": "stacked_rowmajor", "weights": Wh, "d": d, "copies": copies}, hoist),
    ]


def layers_dense64(Wd: np.ndarray, n: int, hoist: int = 1) -> list:
    """Single dense layer + square; the input arrives already stacked
    (one copy per output row) so no server-side stacking rotations.
    hoist: rotate-and-sum doubling steps per key switch."""
    d = _ceil_log2(Wd.shape[1])
    copies = 1 << _ceil_log2(Wd.shape[0])
    return [
        _with_hoist({"op": "stacked_rowmajor", "weights": Wd, "d": d, "copies": copies}, hoist),
        {"op": "square"},
    ]


def dense64_input_copies(Wd: np.ndarray) -> int:
    return 1 << _ceil_log2(Wd.shape[0])
