"""Python binding of the C-ABI in include/lola.h (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library.  The functions keep the C names; a few helpers convert layer lists
and numpy arrays.  Importing works without a GPU; creating a context needs
one, and every call raises LolaError when the library reports an error.
There is no fallback path: if the compiled library is missing, loading fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LOLA_OK = 0
ERRORS = {-1: "E_PARAM", -2: "E_NOMEM", -3: "E_NOKEY", -4: "E_REPR", -5: "E_CUDA", -6: "E_TIMEOUT", -7: "E_STATE"}

LOLA_KEY_RELIN = 1
LOLA_KEY_ROW_SWAP = 2

REPR = {"dense": 1, "sparse": 2, "stacked": 3, "interleaved": 4, "convolution": 5}
LAYER = {"conv": 1, "combine": 2, "square": 3, "stack": 4, "stacked_rowmajor": 5,
         "interleaved_rowmajor": 6, "dense_rowmajor": 7, "sparse_colmajor": 8, "masked_shifts": 9, "place": 10,
         "interleaved_rowmajor_support": 12,
         "mod_switch": 11}
# representation each layer consumes / produces (0 = not checked)
LAYER_REPR = {"conv": (5, 1), "combine": (1, 1), "square": (0, 0), "stack": (1, 3),
              "stacked_rowmajor": (3, 4), "interleaved_rowmajor": (4, 2), "dense_rowmajor": (1, 2),
              "interleaved_rowmajor_support": (0, 1),   # interleaved or dense input (checked by the library)
              "sparse_colmajor": (2, 1), "masked_shifts": (1, 5), "place": (1, 1), "mod_switch": (0, 0)}


class LolaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class lola_params(C.Structure):
    _fields_ = [("n", C.c_uint32), ("L", C.c_uint32), ("K", C.c_uint32), ("q", C.POINTER(C.c_uint64)),
                ("k_t", C.c_uint32), ("t", C.POINTER(C.c_uint64)), ("alpha", C.c_uint32)]


class lola_layer(C.Structure):
    _fields_ = [("op", C.c_int), ("in_repr", C.c_int), ("out_repr", C.c_int), ("rows", C.c_uint32),
                ("cols", C.c_uint32), ("weights", C.POINTER(C.c_int64)), ("d", C.c_uint32),
                ("copies", C.c_uint32), ("stride", C.c_uint32), ("hoist", C.c_uint32)]


class lola_input(C.Structure):
    _fields_ = [("repr", C.c_int), ("n_msgs", C.c_uint32), ("n_elems", C.c_uint32),
                ("slot", C.POINTER(C.c_uint32)), ("d", C.c_uint32), ("copies", C.c_uint32)]


_lib = None
P = C.c_void_p
U64P = C.POINTER(C.c_uint64)
I64P = C.POINTER(C.c_int64)
U32P = C.POINTER(C.c_uint32)
I32P = C.POINTER(C.c_int32)

_SIGS = {
    "lola_ctx_create": (C.c_int, [C.POINTER(lola_params), C.c_int, C.POINTER(P)]),
    "lola_ctx_destroy": (None, [P]),
    "lola_ctx_aux_primes": (C.c_int, [P, U64P, U32P]),
    "lola_keygen": (C.c_int, [P, C.c_uint64, I32P, C.c_size_t, C.c_uint32, C.POINTER(P), C.POINTER(P)]),
    "lola_keys_destroy": (None, [P]),
    "lola_keys_export": (C.c_int, [P, P, C.c_int, C.c_int32, U64P, C.POINTER(C.c_size_t)]),
    "lola_encrypt": (C.c_int, [P, P, I64P, C.c_size_t, C.c_uint64, C.POINTER(P)]),
    "lola_decrypt": (C.c_int, [P, P, P, I64P]),
    "lola_decrypt_residues": (C.c_int, [P, P, P, U64P]),
    "lola_ct_create": (C.c_int, [P, C.c_size_t, C.POINTER(P)]),
    "lola_ct_messages": (C.c_size_t, [P]),
    "lola_ct_data": (P, [P]),
    "lola_ct_export": (C.c_int, [P, P, U64P]),
    "lola_ct_level": (C.c_uint32, [P]),
    "lola_autotune": (C.c_int, [P, P]),
    "lola_tune_get": (C.c_int, [P, C.POINTER(C.c_uint8), C.POINTER(C.c_float)]),
    "lola_tune_set": (C.c_int, [P, C.POINTER(C.c_uint8)]),
    "lola_mod_switch": (C.c_int, [P, P, P, C.c_size_t, C.c_uint32, C.c_uint32, P]),
    "lola_decrypt_residues_level": (C.c_int, [P, P, P, C.c_size_t, C.c_uint32, U64P]),
    "lola_ct_import": (C.c_int, [P, U64P, C.c_size_t, C.POINTER(P)]),
    "lola_ct_copy_messages": (C.c_int, [P, P, C.c_size_t, P, C.c_size_t, C.c_size_t, P]),
    "lola_ct_upload": (C.c_int, [P, P, P, P]),
    "lola_ct_download": (C.c_int, [P, P, P, P]),
    "lola_ct_destroy": (None, [P]),
    "lola_ntt_forward": (C.c_int, [P, P, C.c_size_t, C.c_uint32, P]),
    "lola_ntt_inverse": (C.c_int, [P, P, C.c_size_t, C.c_uint32, P]),
    "lola_add": (C.c_int, [P, P, P, P, C.c_size_t, P]),
    "lola_rotate": (C.c_int, [P, P, P, P, C.c_size_t, I32P, P]),
    "lola_multiply": (C.c_int, [P, P, P, P, P, C.c_size_t, U32P, P]),
    "lola_mul_plain": (C.c_int, [P, P, I64P, P, C.c_size_t, U32P, P]),
    "lola_rotate_noalloc": (C.c_int, [P, P, P, P, C.c_size_t, C.c_int32, P]),
    "lola_rotate_hoisted": (C.c_int, [P, P, P, P, C.c_size_t, I32P, C.c_size_t, P]),
    "lola_rotate_sum": (C.c_int, [P, P, P, P, C.c_size_t, I32P, C.c_size_t, P]),
    "lola_net_create": (C.c_int, [P, C.POINTER(lola_input), C.POINTER(lola_layer), C.c_size_t, C.POINTER(P)]),
    "lola_net_destroy": (None, [P]),
    "lola_net_rotation_steps": (C.c_int, [P, I32P, C.POINTER(C.c_size_t)]),
    "lola_net_output_map": (C.c_int, [P, U32P, U32P, C.POINTER(C.c_size_t)]),
    "lola_net_shape": (C.c_int, [P, U32P, U32P]),
    "lola_eval_network": (C.c_int, [P, P, P, P, P, P]),
    "lola_eval_network_eager": (C.c_int, [P, P, P, P, P, P]),
    "lola_pack_convolution": (C.c_int, [I64P, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                        C.c_uint32, I64P, U32P]),
    "lola_pack_stacked": (C.c_int, [I64P, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, I64P]),
    "lola_profile_enable": (C.c_int, [P, C.c_int, C.c_int]),
    "lola_profile_read": (C.c_int, [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_uint64),
                                    C.POINTER(C.c_uint64)]),
    "lola_profile_kinds": (C.c_int, []),
    "lola_alu_rate": (C.c_int, [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lola_encrypt_symmetric": (C.c_int, [P, P, I64P, C.c_size_t, C.c_uint64, C.POINTER(P)]),
    "lola_ct_upload_seeded": (C.c_int, [P, P, C.c_void_p, C.c_uint64, P]),
    "lola_ct_bytes": (C.c_size_t, [P]),
    "lola_profile_name": (C.c_char_p, [C.c_int]),
    "lola_launch_count": (C.c_uint64, [P]),
    "lola_last_error": (C.c_char_p, []),
    "lola_version": (C.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if asked and needed)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"CUDA library not built: {path}")
            _build.build()
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc):
    if rc != LOLA_OK:
        raise LolaError(rc, load().lola_last_error().decode())


def _u64(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    return a, a.ctypes.data_as(U64P)


def _i64(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    return a, a.ctypes.data_as(I64P)


def dptr(t) -> int:
    """Device pointer of a torch tensor (or an int)."""
    return t if isinstance(t, int) else t.data_ptr()


def stream_handle(stream) -> int | None:
    if stream is None:
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


# ------------------------------------------------------------------ context

def lola_ctx_create(n, q, L, K, t, device=0, alpha=1):
    """alpha: ciphertext primes per key-switching digit (1 or 2)."""
    lib = load()
    q_arr, qp = _u64(q)
    t_arr, tp = _u64(t)
    p = lola_params(n, L, K, qp, len(t_arr), tp, alpha)
    out = P()
    _check(lib.lola_ctx_create(C.byref(p), device, C.byref(out)))
    return out


def lola_ctx_destroy(ctx):
    load().lola_ctx_destroy(ctx)


def lola_ctx_aux_primes(ctx):
    lib = load()
    cnt = C.c_uint32()
    _check(lib.lola_ctx_aux_primes(ctx, None, C.byref(cnt)))
    arr = np.zeros(cnt.value, dtype=np.uint64)
    _check(lib.lola_ctx_aux_primes(ctx, arr.ctypes.data_as(U64P), C.byref(cnt)))
    return [int(x) for x in arr]


def lola_keygen(ctx, seed, rot_steps=(), flags=LOLA_KEY_RELIN, want_eval=True):
    lib = load()
    steps = np.ascontiguousarray(np.asarray(list(rot_steps), dtype=np.int32))
    sk, ev = P(), P()
    _check(lib.lola_keygen(ctx, seed, steps.ctypes.data_as(I32P), len(steps), flags, C.byref(sk),
                           C.byref(ev) if want_eval else None))
    return (sk, ev) if want_eval else sk


def lola_keys_destroy(keys):
    load().lola_keys_destroy(keys)


def lola_keys_export(ctx, keys, what, step=0):
    lib = load()
    words = C.c_size_t()
    _check(lib.lola_keys_export(ctx, keys, what, step, None, C.byref(words)))
    out = np.zeros(words.value, dtype=np.uint64)
    _check(lib.lola_keys_export(ctx, keys, what, step, out.ctypes.data_as(U64P), C.byref(words)))
    return out


# -------------------------------------------------------------- ciphertexts

def lola_encrypt(ctx, keys, slots, seed):
    lib = load()
    s, sp = _i64(np.atleast_2d(slots))
    out = P()
    _check(lib.lola_encrypt(ctx, keys, sp, s.shape[0], seed, C.byref(out)))
    return out


def lola_encrypt_symmetric(ctx, keys, slots, seed):
    """Seeded symmetric encryption with the secret key (c1 regenerable from the seed)."""
    lib = load()
    s, sp = _i64(np.atleast_2d(slots))
    out = P()
    _check(lib.lola_encrypt_symmetric(ctx, keys, sp, s.shape[0], seed, C.byref(out)))
    return out


def lola_ct_upload_seeded(ctx, ct, host_c0_ptr: int, seed, stream=None):
    """Copy the c0 halves [n_msg][k_t][L][n] at host address host_c0_ptr into
    ct and regenerate c1 from the seed on the device (stream-ordered)."""
    _check(load().lola_ct_upload_seeded(ctx, ct, C.c_void_p(host_c0_ptr), seed, stream_handle(stream)))


def lola_ct_bytes(ct) -> int:
    """Device bytes held by a ciphertext handle."""
    return int(load().lola_ct_bytes(ct))


def lola_ct_messages(ct) -> int:
    return int(load().lola_ct_messages(ct))


def lola_ct_data(ct) -> int:
    return int(load().lola_ct_data(ct))


def lola_ct_create(ctx, n_msg):
    out = P()
    _check(load().lola_ct_create(ctx, n_msg, C.byref(out)))
    return out


def lola_ct_destroy(ct):
    load().lola_ct_destroy(ct)


def lola_ct_level(ct) -> int:
    return int(load().lola_ct_level(ct))


def lola_ct_export(ctx, ct, shape_tail):
    """shape_tail = (k_t, 2, L, n); returns [n_msg][k_t][2][L'][n] coefficient form,
    L' = the handle's level (L unless a network switched modulus)."""
    m = lola_ct_messages(ct)
    tail = list(shape_tail)
    tail[2] = lola_ct_level(ct)
    out = np.zeros((m,) + tuple(tail), dtype=np.uint64)
    _check(load().lola_ct_export(ctx, ct, out.ctypes.data_as(U64P)))
    return out


def lola_ct_import(ctx, host):
    a, ap = _u64(host)
    out = P()
    _check(load().lola_ct_import(ctx, ap, a.shape[0], C.byref(out)))
    return out


def lola_ct_copy_messages(ctx, dst, dst_off, src, src_off, n, stream=None):
    _check(load().lola_ct_copy_messages(ctx, dst, dst_off, src, src_off, n, stream_handle(stream)))


def lola_ct_upload(ctx, ct, host_ptr: int, stream=None):
    _check(load().lola_ct_upload(ctx, ct, host_ptr, stream_handle(stream)))


def lola_ct_download(ctx, ct, host_ptr: int, stream=None):
    _check(load().lola_ct_download(ctx, ct, host_ptr, stream_handle(stream)))


def lola_decrypt(ctx, keys, ct, n):
    """Signed CRT-recombined slot values as Python ints, shape [n_msg][n]."""
    m = lola_ct_messages(ct)
    out = np.zeros((m, n, 2), dtype=np.int64)
    _check(load().lola_decrypt(ctx, keys, ct, out.ctypes.data_as(I64P)))
    lo = out[..., 0].astype(np.uint64).astype(object)
    hi = out[..., 1].astype(object)
    return hi * (1 << 64) + lo


def lola_decrypt_residues(ctx, keys, ct, k_t, n):
    m = lola_ct_messages(ct)
    out = np.zeros((m, k_t, n), dtype=np.uint64)
    _check(load().lola_decrypt_residues(ctx, keys, ct, out.ctypes.data_as(U64P)))
    return out


def lola_decrypt_residues_level(ctx, keys, d_ct, n_msg, level, k_t, n):
    """Decrypt device ciphertexts [n_msg][k_t][2][level][n] (e.g. lola_mod_switch output)."""
    out = np.zeros((n_msg, k_t, n), dtype=np.uint64)
    _check(load().lola_decrypt_residues_level(ctx, keys, dptr(d_ct), n_msg, level, out.ctypes.data_as(U64P)))
    return out


# --------------------------------------------------------------- primitives

def lola_ntt_forward(ctx, data, n_polys, n_limbs, stream=None):
    _check(load().lola_ntt_forward(ctx, dptr(data), n_polys, n_limbs, stream_handle(stream)))


def lola_ntt_inverse(ctx, data, n_polys, n_limbs, stream=None):
    _check(load().lola_ntt_inverse(ctx, dptr(data), n_polys, n_limbs, stream_handle(stream)))


def lola_add(ctx, a, b, out, count, stream=None):
    _check(load().lola_add(ctx, dptr(a), dptr(b), dptr(out), count, stream_handle(stream)))


def lola_rotate(ctx, keys, inp, out, count, steps, stream=None):
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.int32))
    assert st.size == count
    _check(load().lola_rotate(ctx, keys, dptr(inp), dptr(out), count, st.ctypes.data_as(I32P),
                              stream_handle(stream)))


def lola_rotate_hoisted(ctx, keys, inp, out, count, steps, stream=None):
    """Rotate each of `count` ciphertexts by every step in `steps` (one
    shared decomposition); out holds len(steps) * count ciphertexts, step-major."""
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.int32))
    _check(load().lola_rotate_hoisted(ctx, keys, dptr(inp), dptr(out), count, st.ctypes.data_as(I32P), st.size,
                                      stream_handle(stream)))


def lola_rotate_sum(ctx, keys, inp, out, count, steps, stream=None):
    """out_i = in_i + sum of its rotations by every step in `steps`, one key
    switch per ciphertext (see include/lola.h)."""
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.int32))
    _check(load().lola_rotate_sum(ctx, keys, dptr(inp), dptr(out), count, st.ctypes.data_as(I32P), st.size,
                                  stream_handle(stream)))


def lola_rotate_noalloc(ctx, keys, inp, out, count, step, stream=None):
    """Rotation of `count` ciphertexts by one step using the library's static
    scratch area (no device allocation); see include/lola.h."""
    _check(load().lola_rotate_noalloc(ctx, keys, dptr(inp), dptr(out), count, int(step), stream_handle(stream)))


NOALLOC_SCRATCH_BYTES = 32 << 20


TUNE_KERNELS, TUNE_BUCKETS, TUNE_VARIANTS = 4, 6, 4
TUNE_NAMES = ("ks_decompose", "ks_modup", "ks_intt_p", "ks_moddown")
TUNE_GEOMETRY = ("cta", "cluster16", "cluster32", "cluster4x16")


def lola_autotune(ctx, stream=None) -> dict:
    """Time the key-switch transforms' launch geometries on this device and
    install the fastest per kernel and launch-size bucket; returns the table."""
    _check(load().lola_autotune(ctx, stream_handle(stream)))
    return lola_tune_get(ctx)


def lola_tune_get(ctx) -> dict:
    """{"table": [[geometry per bucket] per kernel], "us": [[[us per geometry]]]}"""
    t = (C.c_uint8 * (TUNE_KERNELS * TUNE_BUCKETS))()
    us = (C.c_float * (TUNE_KERNELS * TUNE_BUCKETS * TUNE_VARIANTS))()
    _check(load().lola_tune_get(ctx, t, us))
    tab = [[int(t[k * TUNE_BUCKETS + b]) for b in range(TUNE_BUCKETS)] for k in range(TUNE_KERNELS)]
    tim = [[[round(float(us[(k * TUNE_BUCKETS + b) * TUNE_VARIANTS + v]), 2) for v in range(TUNE_VARIANTS)]
            for b in range(TUNE_BUCKETS)]
           for k in range(TUNE_KERNELS)]
    return {"table": tab, "us": tim}


def lola_tune_set(ctx, table=None):
    """Install a table (list of 4 lists of 6 geometry ids), or None for the defaults."""
    if table is None:
        _check(load().lola_tune_set(ctx, None))
        return
    flat = [int(x) for row in table for x in row]
    assert len(flat) == TUNE_KERNELS * TUNE_BUCKETS
    arr = (C.c_uint8 * len(flat))(*flat)
    _check(load().lola_tune_set(ctx, arr))


def autotune_cached(ctx, path, key: dict, stream=None) -> dict:
    """Load the table for `key` (device name and parameters) from the JSON
    cache at `path`, or run lola_autotune and store its result there."""
    import json
    cache = {}
    if os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    k = json.dumps(key, sort_keys=True)
    if k in cache:
        lola_tune_set(ctx, cache[k]["table"])
        return dict(cache[k], cached=True)
    res = lola_autotune(ctx, stream)
    cache[k] = res
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f)
    os.replace(tmp, path)
    return dict(res, cached=False)


def lola_mod_switch(ctx, inp, out, count, L_from, L_to, stream=None):
    """Modulus switching of `count` ciphertexts [2][L_from][n] to [2][L_to][n]."""
    _check(load().lola_mod_switch(ctx, dptr(inp), dptr(out), count, L_from, L_to, stream_handle(stream)))


def lola_multiply(ctx, keys, a, b, out, count, t_index=None, stream=None):
    ti = None
    if t_index is not None:
        ti_arr = np.ascontiguousarray(np.asarray(t_index, dtype=np.uint32))
        ti = ti_arr.ctypes.data_as(U32P)
    _check(load().lola_multiply(ctx, keys, dptr(a), dptr(b), dptr(out), count, ti, stream_handle(stream)))


def lola_mul_plain(ctx, inp, slots, out, count, t_index=None, stream=None):
    s, sp = _i64(np.atleast_2d(slots))
    ti = None
    if t_index is not None:
        ti_arr = np.ascontiguousarray(np.asarray(t_index, dtype=np.uint32))
        ti = ti_arr.ctypes.data_as(U32P)
    _check(load().lola_mul_plain(ctx, dptr(inp), sp, dptr(out), count, ti, stream_handle(stream)))


# ------------------------------------------------------------------ networks

class Network:
    """Holds the C net handle and the host arrays its creation referenced."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def rotation_steps(self):
        lib = load()
        cnt = C.c_size_t()
        _check(lib.lola_net_rotation_steps(self.handle, None, C.byref(cnt)))
        arr = np.zeros(cnt.value, dtype=np.int32)
        _check(lib.lola_net_rotation_steps(self.handle, arr.ctypes.data_as(I32P), C.byref(cnt)))
        return [int(x) for x in arr]

    def output_map(self):
        lib = load()
        cnt = C.c_size_t()
        _check(lib.lola_net_output_map(self.handle, None, None, C.byref(cnt)))
        m = np.zeros(cnt.value, dtype=np.uint32)
        s = np.zeros(cnt.value, dtype=np.uint32)
        _check(lib.lola_net_output_map(self.handle, m.ctypes.data_as(U32P), s.ctypes.data_as(U32P), C.byref(cnt)))
        return list(zip(m.tolist(), s.tolist()))

    def shape(self):
        a, b = C.c_uint32(), C.c_uint32()
        _check(load().lola_net_shape(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    def destroy(self):
        if self.handle:
            load().lola_net_destroy(self.handle)
            self.handle = None


def lola_net_create(ctx, input_desc: dict, layers: list) -> Network:
    """input_desc: {"repr", "n_msgs", "n_elems", "slot"=None, "d"=0, "copies"=0};
    layers: dicts as produced by workloads.layers_* ({"op", "weights", "d", "copies", "stride", "hoist"})."""
    keep = []
    slot = input_desc.get("slot")
    if slot is not None:
        sa = np.ascontiguousarray(np.asarray(slot, dtype=np.uint32))
        keep.append(sa)
        sp = sa.ctypes.data_as(U32P)
    else:
        sp = None
    inp = lola_input(REPR[input_desc["repr"]], input_desc["n_msgs"], input_desc["n_elems"], sp,
                     input_desc.get("d", 0), input_desc.get("copies", 0))
    arr = (lola_layer * max(1, len(layers)))()
    for i, Ld in enumerate(layers):
        op = Ld["op"]
        w = Ld.get("weights")
        if op == "combine" and Ld.get("shifts") is not None:
            w = [list(Ld["shifts"])]
        rows = cols = 0
        wp = None
        if w is not None:
            wa = np.ascontiguousarray(np.asarray(w, dtype=np.int64))
            keep.append(wa)
            rows, cols = wa.shape
            wp = wa.ctypes.data_as(I64P)
        rin, rout = LAYER_REPR[op]
        d = Ld["L"] if op == "mod_switch" else Ld.get("d", 0)
        arr[i] = lola_layer(LAYER[op], rin, rout, rows, cols, wp, d, Ld.get("copies", 0), Ld.get("stride", 0),
                            Ld.get("hoist", 0))
    out = P()
    _check(load().lola_net_create(ctx, C.byref(inp), arr, len(layers), C.byref(out)))
    return Network(out, keep)


def lola_eval_network(ctx, keys, net: Network, ct_in, ct_out, stream=None, graph=True):
    fn = load().lola_eval_network if graph else load().lola_eval_network_eager
    _check(fn(ctx, keys, net.handle, ct_in, ct_out, stream_handle(stream)))


def lola_pack_convolution(image, kh, kw, stride, n):
    img, ip = _i64(image)
    h, w = img.shape
    out = np.zeros((kh * kw, n), dtype=np.int64)
    win = C.c_uint32()
    _check(load().lola_pack_convolution(ip, h, w, kh, kw, stride, n, out.ctypes.data_as(I64P), C.byref(win)))
    return out, win.value


def lola_pack_convolution_channels(image, kh, kw, stride, n):
    """Multi-channel image (channels, h, w): the convolution representation
    of each channel, concatenated channel by channel (message ch*kh*kw +
    dr*kw + dc), through lola_pack_convolution."""
    img = np.asarray(image)
    parts = [lola_pack_convolution(img[ch], kh, kw, stride, n) for ch in range(img.shape[0])]
    return np.concatenate([p[0] for p in parts]), parts[0][1]


def lola_pack_stacked(vec, d, copies, n):
    v, vp = _i64(vec)
    out = np.zeros(n, dtype=np.int64)
    _check(load().lola_pack_stacked(vp, v.size, d, copies, n, out.ctypes.data_as(I64P)))
    return out


def lola_profile_enable(ctx, kind, on=True):
    _check(load().lola_profile_enable(ctx, kind, 1 if on else 0))


def lola_profile_read(ctx, kind):
    """(milliseconds, launches, work units) since the last enable."""
    ms, cnt, units = C.c_double(), C.c_uint64(), C.c_uint64()
    _check(load().lola_profile_read(ctx, kind, C.byref(ms), C.byref(cnt), C.byref(units)))
    return ms.value, cnt.value, units.value


ALU_KINDS = {"fwd_butterfly": 0, "inv_butterfly": 1, "fwd_butterfly_c": 2, "mad_lo_u32": 3,
             "mad_wide_u32": 4, "mul_hi_u32": 5, "mma_s8": 6, "fwd_butterfly_sparse": 7, "mac64": 8}


def lola_alu_rate(ctx, kind) -> tuple:
    """(operations per second, best kernel ms) of integer-unit microbenchmark
    `kind` (a name of ALU_KINDS or its number) on the context's device."""
    k = ALU_KINDS[kind] if isinstance(kind, str) else int(kind)
    rate, ms = C.c_double(), C.c_double()
    _check(load().lola_alu_rate(ctx, k, C.byref(rate), C.byref(ms)))
    return rate.value, ms.value


def lola_profile_kinds() -> int:
    return int(load().lola_profile_kinds())


def lola_profile_name(kind) -> str:
    return load().lola_profile_name(kind).decode()


def lola_launch_count(ctx) -> int:
    return int(load().lola_launch_count(ctx))


def lola_version() -> str:
    return load().lola_version().decode()
