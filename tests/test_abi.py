"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/lola.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def header_functions():
    src = open(os.path.join(ROOT, "include", "lola.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(lola_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_parses():
    names = header_functions()
    assert "lola_eval_network" in names and "lola_keygen" in names and len(names) > 30


def test_library_exports_every_declared_symbol():
    from paper_1812_10659_gb300 import lola as L
    lib = L.load()
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing
    raw = ctypes.CDLL(L.library_path())
    for n in header_functions():
        getattr(raw, n)
    # and the binding wraps each of them under the same name
    assert sorted(header_functions()) == sorted(L.exported_symbols())


def test_no_device_error_is_reported():
    from paper_1812_10659_gb300 import lola as L
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(L.LolaError) as ei:
        L.lola_ctx_create(32, [1152921504606748673], 1, 0, [65537])
    assert ei.value.code == -5


def test_pack_convolution_matches_footnote():
    import numpy as np
    from paper_1812_10659_gb300 import lola as L
    img = np.array([[10 * (r + 1) + (c + 1) for c in range(4)] for r in range(4)])
    out, win = L.lola_pack_convolution(img, 2, 2, 2, 16)
    assert win == 4
    assert out[:, :4].tolist() == [[11, 13, 31, 33], [12, 14, 32, 34], [21, 23, 41, 43], [22, 24, 42, 44]]


def test_pack_matches_oracle_packer():
    import numpy as np
    import workloads as W
    from oracle import lola as OL
    from paper_1812_10659_gb300 import lola as L
    img = W.image()
    out, win = L.lola_pack_convolution(img, 5, 5, 2, 16384)
    ref, pos = OL.pack_convolution(img, 5, 5, 2, 16384)
    assert win == 169 == len(pos)
    assert np.array_equal(out, np.array(ref, dtype=np.int64))
    v = W.dense_vector()
    assert np.array_equal(L.lola_pack_stacked(v, 6, 16, 4096), np.array(OL.pack_stacked(v, 6, 16, 4096)[0]))


def test_bad_parameters_rejected_before_device_use():
    from paper_1812_10659_gb300 import lola as L
    with pytest.raises(L.LolaError):
        L.lola_pack_convolution([[1, 2], [3, 4]], 3, 3, 1, 16)


def test_autotune_cache_helper_runs_the_tuner_once_per_key(tmp_path, monkeypatch):
    """Host logic of lola.autotune_cached (the device calls replaced by
    recorders): the first call for a key tunes and stores the table, the
    next installs the stored one, another key tunes again."""
    from paper_1812_10659_gb300 import lola as L
    calls = {"tune": 0, "set": []}
    table = [[1, 0, 0, 0, 0, 0], [1, 1, 1, 2, 2, 2], [1, 1, 1, 2, 2, 2], [1, 1, 1, 2, 2, 2]]

    def fake_autotune(ctx, stream=None):
        calls["tune"] += 1
        return {"table": table, "us": []}

    monkeypatch.setattr(L, "lola_autotune", fake_autotune)
    monkeypatch.setattr(L, "lola_tune_set", lambda ctx, t=None: calls["set"].append(t))
    path = str(tmp_path / "tune.json")
    a = L.autotune_cached(None, path, {"n": 16384, "L": 5})
    b = L.autotune_cached(None, path, {"n": 16384, "L": 5})
    c = L.autotune_cached(None, path, {"n": 16384, "L": 6})
    assert (a["cached"], b["cached"], c["cached"]) == (False, True, False)
    assert calls["tune"] == 2 and calls["set"] == [table]
    assert b["table"] == table
