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


def header_constants():
    src = open(os.path.join(ROOT, "include", "tang.h")).read()
    out = {}
    for name, val in re.findall(r"^#define (TANG_[A-Z0-9_]+) \(?(-?(?:0x[0-9A-Fa-f]+|[0-9]+))u?\)?", src, flags=re.M):
        out[name] = int(val, 0)
    return out


def test_binding_constants_match_the_header():
    """The binding's flag and code values are the header's (a drift would send wrong flags)."""
    from paper_2601_03187_b300 import _native as nat
    h = header_constants()
    pairs = {
        "TANG_OK": nat.OK, "TANG_EINVAL": nat.EINVAL, "TANG_ENOMEM": nat.ENOMEM, "TANG_ETABLEFULL": nat.ETABLEFULL,
        "TANG_ENOTFOUND": nat.ENOTFOUND, "TANG_EDEVICE": nat.EDEVICE, "TANG_ETIMEOUT": nat.ETIMEOUT,
        "TANG_EUNSUPPORTED": nat.EUNSUPPORTED, "TANG_EEXIST": nat.EEXIST, "TANG_EAGAIN": nat.EAGAIN,
        "TANG_NO_MATCH": nat.NO_MATCH, "TANG_FP32": nat.FP32, "TANG_BF16": nat.BF16, "TANG_FP8": nat.FP8,
        "TANG_PATH_FUSED_BF16": nat.PATHS["fused_bf16"], "TANG_PATH_FUSED_FP8": nat.PATHS["fused_fp8"],
        "TANG_PATH_PLAIN_FP32": nat.PATHS["plain_fp32"], "TANG_PATH_STAGED_BF16": nat.PATHS["staged_bf16"],
        "TANG_PATH_NO_NN": nat.PATHS["no_nn"], "TANG_PATH_STAGED_FP8": nat.PATHS["staged_fp8"],
        "TANG_MEM_DEVICE": nat.MEM_DEVICE, "TANG_MEM_HOST": nat.MEM_HOST, "TANG_GRAPH": nat.GRAPH,
        "TANG_FUSED_N256": nat.VARIANTS["n256"], "TANG_FUSED_PAIR": nat.VARIANTS["pair"],
        "TANG_FUSED_SPLIT": nat.VARIANTS["split"], "TANG_SEARCH_PAPER": nat.SEARCH_PAPER,
        "TANG_SEARCH_SERIAL": nat.SEARCH_SERIAL, "TANG_MODEL_MAGIC": nat.MODEL_MAGIC,
        "TANG_DU_NONE": nat.DU_NONE, "TANG_DU_INCREMENTAL": nat.DU_INCREMENTAL, "TANG_DU_RETRAIN": nat.DU_RETRAIN,
    }
    wrong = {k: (h.get(k), v) for k, v in pairs.items() if h.get(k) != v}
    assert not wrong, wrong
    # every variant flag lies inside the variant mask, and the split form is both bits
    for k in ("TANG_FUSED_N256", "TANG_FUSED_PAIR", "TANG_FUSED_SPLIT"):
        assert h[k] & ~h["TANG_VARIANT_MASK"] == 0, k
    assert h["TANG_FUSED_SPLIT"] == h["TANG_FUSED_N256"] | h["TANG_FUSED_PAIR"]
