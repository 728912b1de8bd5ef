"""Oracle LoLa layers: the paper's message representations and matrix-vector
algorithms, run either on oracle BFV ciphertexts or on plain slot vectors.

TEST INFRASTRUCTURE ONLY (CPU oracle for the parity tests).

One plan, two evaluators: ``HEEval`` runs every step with the oracle's BFV
(``oracle.bfv``); ``SlotEval`` runs the same steps on plain Z_t slot vectors
with the rotation semantics of Sec. 3.1 (the slot simulator).  The integer
network (``int_network``) evaluates the same layers over Z with no
encryption at all.  Every rotation, add and multiply below is in the order
the paper's algorithms state it; the readings where the paper is silent are
listed in each function.

Layer list entries (dicts):
  {"op": "conv", "weights": W[maps][r]}                 Sec. 4.2.2 convolution vector - row major
  {"op": "combine", "stride": s}                        Sec. 4.3 / App. C: combine messages
  {"op": "square"}                                      Sec. 3.2 square activation
  {"op": "stack", "d": d, "copies": c}                  Sec. 4.2.1 stacked representation
  {"op": "stacked_rowmajor", "weights": W, "d": d, "copies": c}
                                                        Sec. 4.2.2 stacked vector - row major
  {"op": "interleaved_rowmajor", "weights": W}          Sec. 4.2.2 interleaved vector - row major
  {"op": "interleaved_rowmajor_support", "weights": W}  the same product, each dot product summed
                                                        over the vector's occupied slots only
  {"op": "dense_rowmajor", "weights": W}                Sec. 4.2.2 dense vector - row major
  {"op": "sparse_colmajor", "weights": W}               Sec. 4.2.2 sparse vector - column major
  {"op": "mod_switch", "L": Lv}                         keep the first Lv primes of Q (modulus
                                                        switching; no change to any slot value)
The layers with a rotate-and-sum (stack, stacked_rowmajor, interleaved_rowmajor(_support),
dense_rowmajor) take an optional "hoist": m, the doubling steps summed per key switch
(rotate_and_sum, hoist_groups; 1 = the paper's one rotation per step).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import bfv, encoding


# ----------------------------------------------------------------- evaluators

class SlotEval:
    """Plain slot vectors mod t with the paper's rotation semantics."""

    def __init__(self, n: int, t: int):
        self.n, self.t = n, t

    def add(self, a, b):
        return (a + b) % self.t

    def rot(self, a, k):
        """Right shift by k within each row of the 2 x n/2 slot matrix (Sec. 3.1)."""
        h = self.n // 2
        return np.concatenate([np.roll(a[:h], k), np.roll(a[h:], k)])

    def rot_hoisted(self, a, steps):
        """Several rotations of one message (slot semantics of rot / rot_rows)."""
        return [self.rot_rows(a) if k == 0 else self.rot(a, k) for k in steps]

    def rot_rows(self, a):
        h = self.n // 2
        return np.concatenate([a[h:], a[:h]])

    def rot_sum(self, a, steps):
        """a plus its rotations by every step (0 = row swap)."""
        out = a
        for k in steps:
            out = self.add(out, self.rot_rows(a) if k == 0 else self.rot(a, k))
        return out

    def mul_plain(self, a, slots):
        return (a * (np.asarray(slots, dtype=np.int64) % self.t)) % self.t

    def mul_scalar(self, a, w):
        return (a * (int(w) % self.t)) % self.t

    def square(self, a):
        return (a * a) % self.t

    def mod_switch(self, msgs, Lv):
        return msgs


class HEEval:
    """The same steps on oracle ciphertexts."""

    def __init__(self, params: bfv.Params, keys: bfv.Keys, t: int):
        self.p, self.keys, self.t = params, keys, t
        self.full_keys = keys
        self.n = params.n
        self.counts = {"rot": 0, "rot_sum": 0, "mul_plain": 0, "mul_scalar": 0, "square": 0, "add": 0}

    def add(self, a, b):
        self.counts["add"] += 1
        return bfv.add(self.p, a, b)

    def rot(self, a, k):
        self.counts["rot"] += 1
        return bfv.rotate(self.p, self.keys, a, k)

    def rot_rows(self, a):
        self.counts["rot"] += 1
        return bfv.rotate_rows(self.p, self.keys, a)

    def rot_hoisted(self, a, steps):
        self.counts["rot"] += len(steps)
        return bfv.rotate_hoisted(self.p, self.keys, a, steps)

    def rot_sum(self, a, steps):
        """One key switch (one mod-down) for all of the steps' rotations."""
        self.counts["rot_sum"] += 1
        return bfv.rotate_sum_hoisted(self.p, self.keys, a, steps)

    def mul_plain(self, a, slots):
        self.counts["mul_plain"] += 1
        return bfv.mul_plain(self.p, a, encoding.encode(slots, self.t))

    def mul_scalar(self, a, w):
        self.counts["mul_scalar"] += 1
        return bfv.mul_scalar(self.p, a, w)

    def square(self, a):
        self.counts["square"] += 1
        return bfv.square(self.p, self.keys, a)

    def mod_switch(self, msgs, Lv):
        """Every message to level Lv; later steps run at that level."""
        out = [bfv.mod_switch_to(self.p, m, Lv) for m in msgs]
        self.p = bfv.params_at_level(self.p, Lv)
        self.keys = bfv.keys_at_level(self.full_keys, Lv)
        return out


# ------------------------------------------------------------------ the plan

@dataclass
class State:
    msgs: list          # messages (ciphertexts or slot vectors)
    pos: list           # element i -> (message index, slot)
    block: int = 0      # stacked block size (0 if not stacked)
    copies: int = 0


def hoist_groups(shifts, m: int, n: int) -> list:
    """The rotate-and-sum steps `shifts` (0 = row swap) taken up to m at a
    time: each run of up to m consecutive nonzero shifts a_1 .. a_r becomes
    the rotation steps of the 2^r - 1 nonempty subsets, sum_{i in S} a_i mod
    n/2 (subset S as a bit mask, ascending), whose rotations added to x give
    the r doubling steps at once; a row swap is a group of its own.  A run
    with a subset sum of 0 mod n/2 (no rotation) is left as single steps.
    m <= 1: every shift is a group of its own."""
    h = n // 2
    groups, run = [], []

    def flush():
        if not run:
            return
        sums = [sum(a for i, a in enumerate(run) if mask >> i & 1) % h for mask in range(1, 1 << len(run))]
        if len(run) == 1 or 0 in sums:
            groups.extend([a] for a in run)
        else:
            groups.append(sums)
        run.clear()
    for s in shifts:
        if s == 0:
            flush()
            groups.append([0])
            continue
        run.append(s)
        if len(run) >= max(m, 1):
            flush()
    flush()
    return groups


def rotate_and_sum(ev, x, shifts, hoist: int = 1):
    """x <- x + rot(x, s) for s in shifts, in order (Sec. 4.1 and its
    footnote; s = 0 is the row swap).  With hoist = m > 1, each group of
    hoist_groups with more than one step is one hoisted rotate-sum (x plus
    its rotations by all of the group's steps, one key switch); single steps
    stay x + rot(x, s)."""
    for grp in hoist_groups(shifts, hoist, ev.n):
        if len(grp) > 1:
            x = ev.rot_sum(x, grp)
        else:
            s = grp[0]
            x = ev.add(x, ev.rot_rows(x) if s == 0 else ev.rot(x, s))
    return x


def layer_conv(ev, st: State, W) -> State:
    """Convolution vector - row major (Sec. 4.2.2): map m = sum_j W[m][j] * M^j,
    scalar weights (sparse representation of w).  Output: one dense message
    per map; element (m, w) sits at message m, in the slot window w has in
    the input messages."""
    R = len(st.msgs)
    out = []
    for m in range(len(W)):
        acc = ev.mul_scalar(st.msgs[0], W[m][0])
        for j in range(1, R):
            acc = ev.add(acc, ev.mul_scalar(st.msgs[j], W[m][j]))
        out.append(acc)
    pos = [(m, slot) for m in range(len(W)) for (_, slot) in st.pos]
    return State(out, pos)


def layer_combine(ev, st: State, stride: int = 0, shifts=None) -> State:
    """Combine k messages into one (Sec. 4.3, App. C): message m is rotated
    right by shifts[m] (default m * stride; shifts[0] = 0) so active slots do
    not collide, then all are added."""
    h = ev.n // 2
    k = len(st.msgs)
    if shifts is None:
        shifts = [m * stride for m in range(k)]
    assert len(shifts) == k and shifts[0] == 0 and all(0 < s < h for s in shifts[1:])
    acc = st.msgs[0]
    for m in range(1, k):
        acc = ev.add(acc, ev.rot(st.msgs[m], shifts[m]))
    pos = []
    for (m, slot) in st.pos:
        assert slot + shifts[m] < h, "combine must not wrap a row"
        pos.append((0, slot + shifts[m]))
    assert len(set(pos)) == len(pos), "combine positions collide"
    return State([acc], pos)


def masked_shift_plan(st: State, G, n: int):
    """Slots S_e of the output elements and the offset of each message for
    layer_masked_shifts; checks that every message is one shift of message 0."""
    h = n // 2
    slot_of = [slot for (_, slot) in st.pos]
    assert all(m == 0 for (m, _) in st.pos)
    R, E = len(G), len(G[0])
    assert all(int(G[0][e]) >= 0 for e in range(E)), "message 0 must hold every element"
    S = [slot_of[int(G[0][e])] for e in range(E)]
    offs = []
    for r in range(R):
        d = {slot_of[int(G[r][e])] - S[e] for e in range(E) if int(G[r][e]) >= 0}
        assert len(d) == 1, "message %d is not a single shift of message 0" % r
        off = d.pop()
        assert 0 <= off < h and (r == 0) == (off == 0)
        assert all(S[e] + off < h for e in range(E))
        offs.append(off)
    assert len(set(offs)) == R
    return S, offs


def layer_masked_shifts(ev, st: State, G) -> State:
    """Dense -> convolution representation by masking (App. C, LoLa-Dense;
    Table 3: mask the input to create 25 messages).  G[r][e] is the input
    element that message r holds at element e (-1: zero padding).  Reading:
    message 0 keeps element G[0][e] at its input slot S_e; message r is the
    input rotated left by off_r (right by n/2 - off_r; the masks are shifts
    of each other, so one rotation per message aligns it), then multiplied
    by the 0/1 mask of the slots S_e of its elements.  The R - 1 rotations
    all rotate the one input, so they share one decomposition (hoisted)."""
    n, h = ev.n, ev.n // 2
    S, offs = masked_shift_plan(st, G, n)
    x = st.msgs[0]
    ys = [x] + ev.rot_hoisted(x, [h - off for off in offs[1:]])
    out = []
    for r, y in enumerate(ys):
        mask = [0] * n
        for e in range(len(S)):
            if int(G[r][e]) >= 0:
                mask[S[e]] = 1
        out.append(ev.mul_plain(y, mask))
    return State(out, [(0, s) for s in S])


def place_groups(st: State, T, n: int):
    """For layer_place: per message, its elements grouped by the within-row
    right shift and the row change that carry them from their slot to T[e]."""
    h = n // 2
    assert len(T) == len(st.pos) and len(set(T)) == len(T) and all(0 <= t < n for t in T)
    groups = {}
    for e, ((m, s), t) in enumerate(zip(st.pos, T)):
        k = (t % h - s % h) % h
        swap = (s // h) != (t // h)
        groups.setdefault(m, {}).setdefault((swap, k), []).append(e)
    return groups


def layer_place(ev, st: State, T) -> State:
    """Combine k messages into one with element e at slot T[e], over both
    slot rows (Sec. 6.2: the 83 convolution maps of the CIFAR-shaped network
    combined into one message of 16268 values, more than one row holds).
    Each message's elements are grouped by the right shift within a row and
    by whether they change row; a message with several groups is multiplied
    by the 0/1 mask of each group's slots; every group is rotated right by
    its shift; the groups that change row are summed and row-swapped once.
    The messages must hold zeros outside their elements' slots."""
    n = ev.n
    groups = place_groups(st, T, n)
    acc = {False: None, True: None}
    for m in sorted(groups):
        gs = groups[m]
        for (swap, k) in sorted(gs):
            y = st.msgs[m]
            if len(gs) > 1:
                mask = [0] * n
                for e in gs[(swap, k)]:
                    mask[st.pos[e][1]] = 1
                y = ev.mul_plain(y, mask)
            if k:
                y = ev.rot(y, k)
            acc[swap] = y if acc[swap] is None else ev.add(acc[swap], y)
    out = acc[False]
    if acc[True] is not None:
        z = ev.rot_rows(acc[True])
        out = z if out is None else ev.add(out, z)
    return State([out], [(0, t) for t in T])


def layer_square(ev, st: State) -> State:
    return State([ev.square(x) for x in st.msgs], st.pos, st.block, st.copies)


def layer_mod_switch(ev, st: State, Lv: int) -> State:
    """Modulus switching of every message to the first Lv primes of Q: the
    same slots, less work for every later step (not in the paper)."""
    return State(ev.mod_switch(st.msgs, Lv), st.pos, st.block, st.copies)


def layer_stack(ev, st: State, d: int, copies: int, hoist: int = 1) -> State:
    """Stacked representation (Sec. 4.2.1): copies of the vector every 2^d
    slots.  Built by x <- x + rot(x, s) for s = 2^d, 2^(d+1), ... within a
    row, then x <- x + rot_rows(x) when the copies fill both rows."""
    n, h, s = ev.n, ev.n // 2, 1 << d
    assert len(st.msgs) == 1 and all(m == 0 and slot < s for m, slot in st.pos)
    assert copies & (copies - 1) == 0 and copies * s <= n
    per_row = min(copies, h // s)
    shifts = []
    shift = s
    while shift < per_row * s:
        shifts.append(shift)
        shift *= 2
    if copies > per_row:
        shifts.append(0)
    x = rotate_and_sum(ev, st.msgs[0], shifts, hoist)
    return State([x], st.pos, s, copies)


def stacked_output_slot(n: int, s: int, b: int, r: int) -> int:
    h = n // 2
    base = b * s + s - 1
    row, col = divmod(base, h)
    return row * h + (col + r) % h


def layer_stacked_rowmajor(ev, st: State, W, d: int, copies: int, hoist: int = 1) -> State:
    """Stacked vector - row major (Sec. 4.2.2 and its footnote).

    Round r multiplies the stacked vector by rows r*c .. r*c+c-1 of W
    concatenated (block b holds row r*c+b), then sums each block with right
    rotations 1, 2, ..., 2^(d-1); row r*c+b ends at the last slot of block b.
    With more than one round, each round's result is multiplied by a 0/1
    mask of its valid block ends (rotate-and-sum leaves partial sums in the
    other slots), rotated right by r and added (App. C: message i shifted by
    i-1 positions)."""
    n, s = ev.n, 1 << d
    assert st.block == s and st.copies == copies
    rows, k = len(W), len(W[0])
    assert k == len(st.pos)
    R = -(-rows // copies)
    assert R <= s
    x = st.msgs[0]
    outs = []
    for r in range(R):
        P = [0] * n
        for b in range(copies):
            row = r * copies + b
            if row >= rows:
                continue
            for i, (_, slot) in enumerate(st.pos):
                P[b * s + slot] = int(W[row][i])
        y = ev.mul_plain(x, P)
        y = rotate_and_sum(ev, y, [1 << j for j in range(d)], hoist)
        outs.append(y)
    if R == 1:
        pos = [(0, stacked_output_slot(n, s, b, 0)) for b in range(rows)]
        return State([outs[0]], pos)
    acc = None
    for r, y in enumerate(outs):
        mask = [0] * n
        for b in range(copies):
            if r * copies + b < rows:
                mask[b * s + s - 1] = 1
        z = ev.mul_plain(y, mask)
        if r > 0:
            z = ev.rot(z, r)
        acc = z if acc is None else ev.add(acc, z)
    pos = [(0, stacked_output_slot(n, s, o % copies, o // copies)) for o in range(rows)]
    return State([acc], pos)


def layer_interleaved_rowmajor(ev, st: State, W, hoist: int = 1) -> State:
    """Interleaved vector - row major (Sec. 4.2.2): the dense row-major dot
    product with the columns of W placed at the vector's slots.  Each output
    sums all n slots: right rotations 1, 2, ..., n/4 within the rows, then
    the row swap; every slot then holds the result (sparse representation)."""
    n = ev.n
    assert len(st.msgs) == 1 and len(W[0]) == len(st.pos)
    shifts = [1 << j for j in range((n // 2).bit_length() - 1)]
    outs = []
    slots = np.array([slot for (_, slot) in st.pos], dtype=np.int64)
    for o in range(len(W)):
        V = np.zeros(n, dtype=np.int64)
        V[slots] = np.asarray(W[o], dtype=np.int64)     # column i of W at element i's slot
        y = ev.mul_plain(st.msgs[0], V)
        y = rotate_and_sum(ev, y, shifts + [0], hoist)
        outs.append(y)
    return State(outs, [(o, 0) for o in range(len(W))])


def support_sum_shifts(slots, n: int):
    """Rotate-and-sum steps that add up every slot of `slots` (occupied slot
    positions of one message) into one slot, and that slot.

    Reading (not in the paper, whose interleaved row-major product sums all
    n slots with log2(n) rotations): when the occupied slots of each row lie
    in one cyclic run of 2^k slots modulo a period 2^p, the run shifts 1, 2,
    ..., 2^(k-1), then the period shifts 2^p, ..., n/4 (right rotations
    within the rows), then the row swap if both rows are occupied, add every
    occupied slot exactly once into one slot.  The pair (p, k) with the
    fewest steps is taken, the smallest p on ties; the full support (p = 0)
    gives the paper's 1, 2, ..., n/4 and the row swap.  The result slot is
    the smallest slot whose sum covers every occupied slot, found by running
    the steps on occupancy counts."""
    h = n // 2
    logh = h.bit_length() - 1
    rows = sorted({s // h for s in slots})
    cols = sorted({s % h for s in slots})
    best = None
    for lp in range(logh + 1):
        per = 1 << lp
        res = sorted({c % per for c in cols})
        for k in range(lp + 1):
            run = 1 << k
            if any(all((c - o) % per < run for c in res) for o in res):
                cand = (k + (logh - lp) + (1 if len(rows) > 1 else 0), lp, k)
                if best is None or cand < best:
                    best = cand
                break
    _, lp, k = best
    shifts = [1 << j for j in range(k)] + [1 << j for j in range(lp, logh)] + ([0] if len(rows) > 1 else [])
    cnt = np.zeros(n, dtype=np.int64)
    cnt[list(slots)] = 1
    for sh in shifts:
        if sh == 0:
            cnt = cnt + np.concatenate([cnt[h:], cnt[:h]])
        else:
            cnt = cnt + np.concatenate([np.roll(cnt[:h], sh), np.roll(cnt[h:], sh)])
    full = np.nonzero(cnt == len(set(slots)))[0]
    return shifts, int(full[0])


def layer_interleaved_rowmajor_support(ev, st: State, W, hoist: int = 1) -> State:
    """Interleaved vector - row major with each dot product summed over the
    vector's occupied slots only (support_sum_shifts): the products are
    those of layer_interleaved_rowmajor (column i of W at element i's
    slot), the rotate-and-sum uses the support's shifts, and output o is
    message o at the one slot that holds the whole sum."""
    n = ev.n
    assert len(st.msgs) == 1 and len(W[0]) == len(st.pos)
    slots = np.array([slot for (_, slot) in st.pos], dtype=np.int64)
    shifts, p = support_sum_shifts([int(x) for x in slots], n)
    outs = []
    for o in range(len(W)):
        V = np.zeros(n, dtype=np.int64)
        V[slots] = np.asarray(W[o], dtype=np.int64)
        y = ev.mul_plain(st.msgs[0], V)
        y = rotate_and_sum(ev, y, shifts, hoist)
        outs.append(y)
    return State(outs, [(o, p) for o in range(len(W))])


def layer_sparse_colmajor(ev, st: State, W) -> State:
    """Sparse vector - column major (Sec. 4.2.2): W v = sum_i v_i c^i.
    Message i holds v_i in every slot (sparse representation); multiply it
    by column i of W laid out densely and add the products in order i = 0,
    1, ...; the result is dense (output o at slot o)."""
    n = ev.n
    k, rows = len(st.msgs), len(W)
    assert len(W[0]) == k and rows <= n
    acc = None
    Wa = np.asarray(W, dtype=np.int64)
    for i in range(k):
        col = np.zeros(n, dtype=np.int64)
        col[:rows] = Wa[:, i]                             # column i, output o at slot o
        y = ev.mul_plain(st.msgs[i], col)
        acc = y if acc is None else ev.add(acc, y)
    return State([acc], [(0, o) for o in range(rows)])


def run_network(ev, layers, st: State) -> State:
    for L in layers:
        op = L["op"]
        if op == "conv":
            st = layer_conv(ev, st, L["weights"])
        elif op == "masked_shifts":
            st = layer_masked_shifts(ev, st, L["weights"])
        elif op == "place":
            st = layer_place(ev, st, [int(t) for t in np.asarray(L["weights"]).reshape(-1)])
        elif op == "combine":
            st = layer_combine(ev, st, L.get("stride", 0), L.get("shifts"))
        elif op == "square":
            st = layer_square(ev, st)
        elif op == "stack":
            st = layer_stack(ev, st, L["d"], L["copies"], L.get("hoist", 1))
        elif op == "stacked_rowmajor":
            st = layer_stacked_rowmajor(ev, st, L["weights"], L["d"], L["copies"], L.get("hoist", 1))
        elif op in ("interleaved_rowmajor", "dense_rowmajor"):
            st = layer_interleaved_rowmajor(ev, st, L["weights"], L.get("hoist", 1))
        elif op == "interleaved_rowmajor_support":
            st = layer_interleaved_rowmajor_support(ev, st, L["weights"], L.get("hoist", 1))
        elif op == "sparse_colmajor":
            st = layer_sparse_colmajor(ev, st, L["weights"])
        elif op == "mod_switch":
            st = layer_mod_switch(ev, st, L["L"])
        else:
            raise ValueError(op)
    return st


# ---------------------------------------------------------- input packing

def conv_windows(h: int, w: int, kh: int, kw: int, stride: int):
    """Window upper-left corners, row-major.  Reading of Sec. 4.3 (845 = 5*13*13
    on a 28x28 image): pad bottom/right with zeros so that
    ceil((h - kh) / stride) + 1 windows fit per axis."""
    oh = -(-(h - kh) // stride) + 1
    ow = -(-(w - kw) // stride) + 1
    return oh, ow


def pack_convolution(img, kh: int, kw: int, stride: int, n: int):
    """Convolution representation (Sec. 4.2.1 and its footnote): message
    r = dr*kw + dc (window offset, row-major) holds, at slot i*ow + j, the
    pixel at (stride*i + dr, stride*j + dc) (zero in the padding).  A
    multi-channel image (channels, h, w) gives messages r = ch*kh*kw +
    dr*kw + dc (Sec. 6.2: 3 x 8 x 8 = 192 messages)."""
    img = np.asarray(img)
    chans = img[None] if img.ndim == 2 else img
    _, h, w = chans.shape
    oh, ow = conv_windows(h, w, kh, kw, stride)
    msgs = []
    for ch in range(chans.shape[0]):
        for dr in range(kh):
            for dc in range(kw):
                v = [0] * n
                for i in range(oh):
                    for j in range(ow):
                        r, c = stride * i + dr, stride * j + dc
                        v[i * ow + j] = int(chans[ch, r, c]) if (r < h and c < w) else 0
                msgs.append(v)
    return msgs, [(0, i) for i in range(oh * ow)]


def pack_dense(vec, n: int):
    v = [0] * n
    for i, x in enumerate(vec):
        v[i] = int(x)
    return v, [(0, i) for i in range(len(vec))]


def pack_image_rows(img, width: int, n: int):
    """Dense message of an image, line after line (App. C): pixel (r, c) at
    slot r * width + c; width > the image width leaves zero columns (the
    convolution's right padding)."""
    img = np.asarray(img)
    h, w = img.shape
    assert width >= w and h * width <= n // 2
    v = [0] * n
    pos = []
    for r in range(h):
        for c in range(w):
            v[r * width + c] = int(img[r, c])
            pos.append((0, r * width + c))
    return v, pos


def pack_stacked(vec, d: int, copies: int, n: int):
    s = 1 << d
    v = [0] * n
    for b in range(copies):
        for i, x in enumerate(vec):
            v[b * s + i] = int(x)
    return v, [(0, i) for i in range(len(vec))]


# ------------------------------------------------------- integer network

def int_conv(img, W, kh: int, kw: int, stride: int):
    """Convolution over Z with bottom/right zero padding; a multi-channel
    image (channels, h, w) pairs weight index ch*kh*kw + dr*kw + dc with
    channel ch.  Output map-major, windows row-major."""
    img = np.asarray(img)
    chans = img[None] if img.ndim == 2 else img
    C, h, w = chans.shape
    oh, ow = conv_windows(h, w, kh, kw, stride)
    out = []
    for m in range(len(W)):
        for i in range(oh):
            for j in range(ow):
                acc = 0
                for ch in range(C):
                    for dr in range(kh):
                        for dc in range(kw):
                            r, c = stride * i + dr, stride * j + dc
                            if r < h and c < w:
                                acc += int(W[m][(ch * kh + dr) * kw + dc]) * int(chans[ch, r, c])
                out.append(acc)
    return out


def int_dense(x, W):
    return [sum(int(W[o][i]) * int(x[i]) for i in range(len(x))) for o in range(len(W))]


def int_square(x):
    return [int(v) * int(v) for v in x]
