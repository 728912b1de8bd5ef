"""Continuous-batching server for encrypted LoLa inference on one GPU.

The paper's service model (Sec. 1): clients send encrypted inputs, the
server evaluates the network without the secret key and returns encrypted
outputs.  This module serves a stream of such requests for several networks
at once (e.g. the MNIST-shaped network and the transfer-learning head):

* requests queue per network, first come first served;
* each of `slots` execution slots owns a CUDA stream and its own compiled
  copy of every network (so batches on different slots never share
  registers or scratch), and runs one batch at a time;
* whenever a slot is free, the network with the oldest waiting request is
  served: the largest power-of-two batch of its waiting requests that fits
  the batch cap and the free device memory is copied into the slot's input
  buffer, evaluated (CUDA-graph replay) and scattered into per-request
  output ciphertexts, which are taken from a pool (or allocated) only at
  admission, so a backlog of queued requests holds no device memory;
* requests that arrive while others run are admitted as soon as a slot and
  memory free up, and their batches overlap on the device with the batches
  already running on other slots.

Each request's output is exactly what evaluating it alone would give: every
operation of the network acts on each ciphertext independently.

The server only marshals handles and streams; all arithmetic runs in the
CUDA library.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

from . import lola as L


@dataclass
class Request:
    rid: int
    kind: str
    ct_in: object
    t_arrival: float
    t_admit: float = 0.0
    t_done: float = 0.0
    ct_out: object = None
    batch: int = 0


@dataclass
class _Batch:
    kind: str
    reqs: list
    event: object
    t_launch: float


@dataclass
class _Slot:
    stream: object
    nets: dict
    bufs: dict = field(default_factory=dict)      # (kind, B) -> (ct_in, ct_out)
    busy: _Batch | None = None


class Server:
    def __init__(self, ctx, keys, networks: dict, slots: int = 2, max_batch: dict | None = None,
                 memory_reserve: int = 2 << 30, graph: bool = True):
        """networks: kind -> (input_desc, layers) evaluated with (ctx, keys), or
        kind -> (input_desc, layers, ctx, keys) for a network with its own
        context (e.g. fewer plaintext moduli)."""
        import torch
        self.torch = torch
        self.graph = graph
        self.kinds = list(networks)
        self.kctx = {k: (v[2] if len(v) > 2 else ctx) for k, v in networks.items()}
        self.kkeys = {k: (v[3] if len(v) > 3 else keys) for k, v in networks.items()}
        self.max_batch = {k: (max_batch or {}).get(k, 8) for k in self.kinds}
        self.memory_reserve = memory_reserve
        self.slots = []
        for _ in range(slots):
            nets = {k: L.lola_net_create(self.kctx[k], v[0], v[1]) for k, v in networks.items()}
            self.slots.append(_Slot(torch.cuda.Stream(), nets))
        self.free_outputs = {k: [] for k in self.kinds}
        self.shape = {k: self.slots[0].nets[k].shape() for k in self.kinds}
        self.queues = {k: collections.deque() for k in self.kinds}
        self.requests = {}
        self.next_id = 0
        self.done = []
        self.bytes_per_request = {}                  # measured executor footprint per request
        self.out_bytes = {}                          # device bytes of one output handle

    # ---------------------------------------------------------------- API
    def submit(self, kind: str, ct_in, t_arrival: float | None = None) -> int:
        """Queue an encrypted input (a lola_ct with the network's input
        message count).  The caller keeps ct_in alive until the request is done."""
        rid = self.next_id
        self.next_id += 1
        r = Request(rid, kind, ct_in, time.perf_counter() if t_arrival is None else t_arrival)
        self.requests[rid] = r
        self.queues[kind].append(r)
        return rid

    def poll(self, rid: int):
        """The encrypted output (lola_ct) once the request is done, else None."""
        r = self.requests[rid]
        return r.ct_out if r.t_done else None

    def release(self, rid: int):
        """Return a finished request's output handle to the server's pool."""
        r = self.requests.pop(rid)
        if r.ct_out is not None:
            self.free_outputs[r.kind].append(r.ct_out)
            r.ct_out = None

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values()) + sum(1 for s in self.slots if s.busy)

    def _retire(self, wait: bool = False) -> bool:
        changed = False
        for s in self.slots:
            if s.busy and wait:
                s.busy.event.synchronize()
            if s.busy and s.busy.event.query():
                now = time.perf_counter()
                for r in s.busy.reqs:
                    r.t_done = now
                    self.done.append(r)
                s.busy = None
                changed = True
        return changed

    def settle(self):
        """Wait for the batches already running and retire them; queued
        requests stay queued (e.g. to stop a saturated run)."""
        self._retire(wait=True)

    def step(self) -> bool:
        """Retire finished batches and admit new ones; True if anything changed."""
        changed = self._retire()
        for s in self.slots:
            if s.busy:
                continue
            kind = self._next_kind()
            if kind is None:
                break
            B = self._admit_size(s, kind)
            if B == 0:
                break
            self._launch(s, kind, [self.queues[kind].popleft() for _ in range(B)])
            changed = True
        return changed

    def drain(self, poll_s: float = 2e-4):
        while self.pending():
            if not self.step():
                time.sleep(poll_s)

    def warm(self, sizes=None, outputs: int = 0):
        """Build executors (scratch + CUDA graph) for every slot, network and
        power-of-two batch size up to the cap, and `outputs` pooled output
        handles per network, outside any timed region."""
        for k in self.kinds:
            while len(self.free_outputs[k]) < outputs:
                self.free_outputs[k].append(L.lola_ct_create(self.kctx[k], self.shape[k][1]))
        for s in self.slots:
            for k in self.kinds:
                B = 1
                while B <= self.max_batch[k]:
                    if sizes is None or B in sizes:
                        self._prepare(s, k, B)
                    B *= 2
        self.torch.cuda.synchronize()

    def stats(self) -> dict:
        import statistics
        out = {}
        for k in self.kinds + ["all"]:
            rs = [r for r in self.done if k == "all" or r.kind == k]
            if not rs:
                continue
            lat = sorted((r.t_done - r.t_arrival) * 1000 for r in rs)
            out[k] = {"n": len(rs), "p50_ms": statistics.median(lat), "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                      "mean_batch": sum(r.batch for r in rs) / len(rs)}
        return out

    # -------------------------------------------------------------- internals
    def _next_kind(self):
        best, t = None, None
        for k, q in self.queues.items():
            if q and (t is None or q[0].t_arrival < t):
                best, t = k, q[0].t_arrival
        return best

    def _out_bytes(self, kind: str) -> int:
        """Device bytes of one request's output handle."""
        if kind not in self.out_bytes:
            h = self._output(kind)
            self.out_bytes[kind] = L.lola_ct_bytes(h)
            self.free_outputs[kind].append(h)
        return self.out_bytes[kind]

    def _admit_size(self, s: _Slot, kind: str) -> int:
        """Largest power-of-two batch of waiting requests within the cap whose
        executor (if not built yet) and new output handles fit the free
        device memory above the reserve; 0 = wait for memory."""
        n = min(len(self.queues[kind]), self.max_batch[kind])
        B = 1
        while B * 2 <= n:
            B *= 2
        free = None
        while B >= 1:
            need = max(0, B - len(self.free_outputs[kind])) * self._out_bytes(kind)
            if (kind, B) not in s.bufs:
                need += (self.bytes_per_request.get(kind) or 0) * B
            if need == 0:
                return B
            if free is None:
                free, _ = self.torch.cuda.mem_get_info()
            if free - self.memory_reserve >= need:
                return B
            B //= 2
        return 0

    def _output(self, kind: str):
        """An output handle from the pool, or a new one (allocated at
        admission, so queued requests hold no device memory)."""
        if self.free_outputs[kind]:
            return self.free_outputs[kind].pop()
        h = L.lola_ct_create(self.kctx[kind], self.shape[kind][1])
        # a new handle is zero-filled on the default stream; finish that
        # before a slot stream writes into it
        self.torch.cuda.default_stream().synchronize()
        return h

    def _prepare(self, s: _Slot, kind: str, B: int):
        if (kind, B) in s.bufs:
            return s.bufs[(kind, B)]
        n_in, n_out = self.shape[kind]
        free0, _ = self.torch.cuda.mem_get_info()
        ctx = self.kctx[kind]
        ci = L.lola_ct_create(ctx, B * n_in)
        co = L.lola_ct_create(ctx, B * n_out)
        self.torch.cuda.default_stream().synchronize()
        # one evaluation builds the executor (scratch + graph) for this batch size
        L.lola_eval_network(ctx, self.kkeys[kind], s.nets[kind], ci, co, s.stream, graph=self.graph)
        s.stream.synchronize()
        free1, _ = self.torch.cuda.mem_get_info()
        per = max(0, free0 - free1) / B
        self.bytes_per_request[kind] = max(self.bytes_per_request.get(kind, 0), per)
        s.bufs[(kind, B)] = (ci, co)
        return ci, co

    def _launch(self, s: _Slot, kind: str, reqs: list):
        B = len(reqs)
        n_in, n_out = self.shape[kind]
        ci, co = self._prepare(s, kind, B)
        now = time.perf_counter()
        ctx = self.kctx[kind]
        for i, r in enumerate(reqs):
            r.t_admit = now
            r.batch = B
            r.ct_out = self._output(kind)
            L.lola_ct_copy_messages(ctx, ci, i * n_in, r.ct_in, 0, n_in, s.stream)
        L.lola_eval_network(ctx, self.kkeys[kind], s.nets[kind], ci, co, s.stream, graph=self.graph)
        for i, r in enumerate(reqs):
            L.lola_ct_copy_messages(ctx, r.ct_out, 0, co, i * n_out, n_out, s.stream)
        ev = self.torch.cuda.Event()
        ev.record(s.stream)
        s.busy = _Batch(kind, reqs, ev, now)

    def close(self):
        self.torch.cuda.synchronize()
        for s in self.slots:
            for ci, co in s.bufs.values():
                L.lola_ct_destroy(ci)
                L.lola_ct_destroy(co)
            for net in s.nets.values():
                net.destroy()
        for r in self.requests.values():
            if r.ct_out is not None:
                L.lola_ct_destroy(r.ct_out)
        for lst in self.free_outputs.values():
            for h in lst:
                L.lola_ct_destroy(h)
        self.slots = []
