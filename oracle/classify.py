"""ORACLE (test infrastructure): §2.1 classification by linear scan, via oracle/liboracle.so."""
import ctypes
import os

import numpy as np

from workloads import HEADER_DTYPE, RULE_DTYPE, NO_MATCH  # noqa: F401  (input layouts only)
from .build import build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_classify.restype = ctypes.c_int
        _lib.oracle_classify.argtypes = [
            ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
        ]
    return _lib


def classify(rules: np.ndarray, headers: np.ndarray, threads: int | None = None, return_index: bool = False):
    """Rule id of the highest-priority match per header (0xFFFFFFFF if none).

    With return_index, also the matched rule's position in `rules` (-1 if none).
    """
    rules = np.ascontiguousarray(rules, dtype=RULE_DTYPE)
    headers = np.ascontiguousarray(headers, dtype=HEADER_DTYPE)
    n = len(headers)
    ids = np.empty(n, dtype=np.uint32)
    idx = np.empty(n, dtype=np.int64) if return_index else None
    if threads is None:
        threads = os.cpu_count() or 1
    rc = _load().oracle_classify(
        rules.ctypes.data, len(rules), headers.ctypes.data, n, ids.ctypes.data,
        idx.ctypes.data if idx is not None else None, int(threads),
    )
    if rc != 0:
        raise MemoryError("oracle_classify failed")
    return (ids, idx) if return_index else ids


def paper_classify(rules: np.ndarray, headers: np.ndarray, predicted, tuple_of_rule, threads: int | None = None):
    """§5.1.1's post-verification exactly as the paper states it (it is not exact).

    Per packet: if some rule stored in the predicted tuple matches, the answer is the
    highest-priority such rule (the search stays in that tuple, even when a better rule of another
    tuple also matches: the first scenario of §5.1.1, left uncorrected per §8). Otherwise the
    ordered search over the remaining tuples runs, and since the predicted tuple holds no match
    its result is the highest-priority match over all rules, i.e. the §2.1 answer.
    predicted[i] outside [0, T) means no prediction. tuple_of_rule[j] is the tuple rules[j] is
    stored in. Written as that definition over the linear scan, not as the search procedure.
    """
    rules = np.ascontiguousarray(rules, dtype=RULE_DTYPE)
    headers = np.ascontiguousarray(headers, dtype=HEADER_DTYPE)
    pred = np.asarray(predicted, dtype=np.int64)
    tor = np.asarray(tuple_of_rule, dtype=np.int64)
    out = classify(rules, headers, threads)
    for t in np.unique(pred):
        members = rules[tor == t]
        if t < 0 or len(members) == 0:
            continue
        sel = np.nonzero(pred == t)[0]
        inside = classify(members, headers[sel], threads)
        hit = inside != NO_MATCH
        out[sel[hit]] = inside[hit]
    return out
