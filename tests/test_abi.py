"""CPU-side checks of the boundary: the library builds, loads, and exports every declared entry point."""
import ctypes
import os
import re

import numpy as np

import paper_2601_03187_b300 as tg
from paper_2601_03187_b300 import build as tgbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tang.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tang_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = tgbuild.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers every declared entry point with the same name
    assert set(names) <= set(tg.EXPORTED)


def test_no_gpu_context_creation_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    try:
        tg.Context(0)
    except tg.TangError as e:
        assert e.code == -5  # TANG_EDEVICE
    else:
        raise AssertionError("context creation without a GPU must fail")


def test_model_blob_round_trip():
    rng = np.random.default_rng(0)
    p = {"W0": rng.normal(size=(7, 16)).astype(np.float32), "b0": rng.normal(size=16).astype(np.float32),
         "W1": [rng.normal(size=(16, 16)).astype(np.float32) for _ in range(2)],
         "b1": [rng.normal(size=16).astype(np.float32) for _ in range(2)],
         "W2": [rng.normal(size=(16, 16)).astype(np.float32) for _ in range(2)],
         "b2": [rng.normal(size=16).astype(np.float32) for _ in range(2)],
         "Wc": rng.normal(size=(16, 5)).astype(np.float32), "bc": rng.normal(size=5).astype(np.float32)}
    amax = np.arange(1, 6, dtype=np.float32)
    blob = tg.pack_model(p, amax)
    assert len(blob) == 64 + 4 * 5 + 4 * (7 * 16 + 16 + 2 * (2 * 256 + 32) + 80 + 5)
    q, a = tg.unpack_model(blob)
    assert (a == amax).all()
    assert (q["W0"] == p["W0"]).all() and (q["Wc"] == p["Wc"]).all()
    assert all((x == y).all() for x, y in zip(q["W2"], p["W2"]))
