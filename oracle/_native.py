"""Build and load the oracle's plain-C ring helper (``oracle/c/oracle_ring.c``).

TEST INFRASTRUCTURE ONLY: the CPU oracle that the parity tests, the smoke check
and the CPU-baseline leg of the benchmark use.  The product library never
imports this package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c", "oracle_ring.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_ring.so")

_lock = threading.Lock()
_lib = None

U64P = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the C helper with gcc (no GPU needed). Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u64, sz = ctypes.c_uint64, ctypes.c_size_t
            L.ora_mulmod.restype = u64
            L.ora_mulmod.argtypes = [u64, u64, u64]
            L.ora_powmod.restype = u64
            L.ora_powmod.argtypes = [u64, u64, u64]
            L.ora_invmod.restype = u64
            L.ora_invmod.argtypes = [u64, u64]
            for name in ("ora_vec_mulmod", "ora_vec_addmod", "ora_vec_submod"):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [U64P, U64P, U64P, sz, u64]
            L.ora_vec_scalar_mulmod.restype = None
            L.ora_vec_scalar_mulmod.argtypes = [U64P, u64, U64P, sz, u64]
            L.ora_vec_reduce.restype = None
            L.ora_vec_reduce.argtypes = [U64P, U64P, sz, u64]
            L.ora_poly_mul_schoolbook.restype = None
            L.ora_poly_mul_schoolbook.argtypes = [U64P, U64P, U64P, sz, u64]
            L.ora_poly_mul_coeff.restype = u64
            L.ora_poly_mul_coeff.argtypes = [U64P, U64P, sz, u64, sz]
            L.ora_poly_mul_ntt.restype = None
            L.ora_poly_mul_ntt.argtypes = [U64P, U64P, U64P, sz, u64, u64]
            L.ora_negacyclic_forward.restype = None
            L.ora_negacyclic_forward.argtypes = [U64P, sz, u64, u64]
            L.ora_negacyclic_inverse.restype = None
            L.ora_negacyclic_inverse.argtypes = [U64P, sz, u64, u64]
            L.ora_philox4x64_10.restype = None
            L.ora_philox4x64_10.argtypes = [U64P, U64P, U64P]
            L.ora_philox_words.restype = None
            L.ora_philox_words.argtypes = [u64, u64, u64, u64, u64, U64P, sz]
            _lib = L
    return _lib


def ptr(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(U64P)


def u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
