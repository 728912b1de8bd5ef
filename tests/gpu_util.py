"""Shared helpers for the GPU parity tests: contexts from workload parameter
sets, oracle <-> library ciphertext layout conversion."""
import numpy as np
import pytest

import workloads as W
from oracle import bfv

try:
    import torch
    HAVE_CUDA = torch.cuda.is_available()
except Exception:  # pragma: no cover
    HAVE_CUDA = False


def need_gpu():
    if not HAVE_CUDA:
        pytest.skip("no CUDA device")


def lib():
    from paper_1812_10659_gb300 import lola as L
    L.load()
    return L


def oracle_params(ps: W.ParamSet) -> bfv.Params:
    return bfv.Params(ps.n, ps.q, ps.L, ps.K, ps.t, ps.alpha)


def make_ctx(ps: W.ParamSet):
    L = lib()
    return L.lola_ctx_create(ps.n, ps.q, ps.L, ps.K, ps.t, alpha=ps.alpha, device=0)


def ct_stack(cts, kt=1):
    """oracle ciphertexts (message-major, then t_i) -> [n_msg][kt][2][L][n]"""
    arr = np.stack([np.stack([c.c[0], c.c[1]]) for c in cts])
    return arr.reshape((len(cts) // kt, kt) + arr.shape[1:])


def ct_from_arrays(arr, t):
    return bfv.Ciphertext([arr[0].copy(), arr[1].copy()], t)


def torch_u64(host: np.ndarray):
    """host uint64 array -> CUDA tensor holding the same words (int64 view)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(host).view(np.int64)).cuda()


def host_u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def galois_steps_for(steps):
    return sorted(set(s for s in steps if s != 0))
