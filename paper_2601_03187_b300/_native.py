"""ctypes binding of libtang.so: argument marshalling only, every step runs in the library.

Names mirror the C ABI in include/tang.h (tang_load_ruleset -> Context.load_ruleset, ...).
Device buffers are torch CUDA tensors (their data pointers are passed through); host buffers
are numpy arrays. There is no CPU fallback: if the library is missing, importing fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import struct

import numpy as np

from workloads import HEADER_DTYPE, RULE_DTYPE

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("TANG_LIBRARY") or os.path.join(_HERE, "libtang.so")

# constants of include/tang.h
NO_MATCH = 0xFFFFFFFF
OK, EINVAL, ENOMEM, ETABLEFULL, ENOTFOUND, EDEVICE, ETIMEOUT, EUNSUPPORTED, EEXIST, EAGAIN = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
FP32, BF16, FP8 = 0, 1, 2
PATH_FUSED_BF16, PATH_FUSED_FP8, PATH_PLAIN_FP32, PATH_STAGED_BF16, PATH_NO_NN, PATH_STAGED_FP8 = 0, 1, 2, 3, 4, 5
PATHS = {
    "fused_bf16": PATH_FUSED_BF16, "fused_fp8": PATH_FUSED_FP8, "plain_fp32": PATH_PLAIN_FP32,
    "staged_bf16": PATH_STAGED_BF16, "no_nn": PATH_NO_NN, "staged_fp8": PATH_STAGED_FP8,
}
MEM_DEVICE, MEM_HOST, GRAPH = 0x00, 0x10, 0x100
FUSED_N256, FUSED_PAIR, FUSED_SPLIT = 0x2000, 0x1000, 0x3000
VARIANTS = {None: 0, "n256": FUSED_N256, "pair": FUSED_PAIR, "split": FUSED_SPLIT}
SEARCH_PAPER = 0x4000
SEARCH_SERIAL = 0x8000
DU_NONE, DU_INCREMENTAL, DU_RETRAIN = 0, 1, 2
DU_DECISIONS = {DU_NONE: "none", DU_INCREMENTAL: "incremental", DU_RETRAIN: "retrain"}
MODEL_MAGIC = 0x474E4154
MODEL_HEADER_BYTES = 64


class TangError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("tang error %d: %s" % (code, msg))
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("packets", "matched", "nn_correct", "pred_hit", "fallback", "probes", "rule_reads", "slot_reads")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class RulesetInfo(ctypes.Structure):
    _fields_ = [("n_rules", ctypes.c_uint32), ("n_tuples", ctypes.c_uint32), ("conflict_words", ctypes.c_uint32),
                ("n_keys", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64), ("build_ms", ctypes.c_double)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("blocks", ctypes.c_uint32), ("batch", ctypes.c_uint32),
                ("epochs", ctypes.c_uint32), ("max_rounds", ctypes.c_uint32), ("decay_every", ctypes.c_uint32),
                ("lr", ctypes.c_float), ("decay", ctypes.c_float), ("alpha", ctypes.c_uint32),
                ("beta", ctypes.c_float), ("holdout", ctypes.c_float), ("time_budget_s", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class TrainReport(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("epochs_run", ctypes.c_uint32), ("samples_labelled", ctypes.c_uint32),
                ("samples_trained", ctypes.c_uint32), ("classes_empty", ctypes.c_uint32),
                ("alpha_final", ctypes.c_uint32), ("final_loss", ctypes.c_float),
                ("holdout_accuracy", ctypes.c_float), ("train_seconds", ctypes.c_float)]


class DuCfg(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("theta", ctypes.c_uint64)]


class DuWindow(ctypes.Structure):
    _fields_ = [("window", ctypes.c_uint64), ("th_cur", ctypes.c_double), ("th_base", ctypes.c_double),
                ("suboptimal", ctypes.c_uint64), ("decision", ctypes.c_int)]


class HybridCfg(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_uint32), ("streams", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("precision", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 3)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_uint32), ("max_batch", ctypes.c_uint32), ("path", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class ServeInfo(ctypes.Structure):
    _fields_ = [("slots_max", ctypes.c_uint32), ("slots_admitted", ctypes.c_uint32),
                ("slots_admitted_peak", ctypes.c_uint32), ("slots_busy", ctypes.c_uint32),
                ("admissions_refused", ctypes.c_uint64), ("launches", ctypes.c_uint64), ("packets", ctypes.c_uint64),
                ("slot_bytes", ctypes.c_uint64), ("queued", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ReqStats(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("done_s", ctypes.c_double)]


_P, _U32, _U64, _I, _F, _SZ = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
_SIGS = {
    "tang_create": (_I, [_I, _SZ, ctypes.POINTER(_P)]),
    "tang_destroy": (None, [_P]),
    "tang_last_error": (ctypes.c_char_p, [_P]),
    "tang_memory_usage": (_I, [_P, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "tang_load_ruleset": (_I, [_P, _P, _U32, ctypes.POINTER(_U32)]),
    "tang_unload_ruleset": (_I, [_P, _U32]),
    "tang_ruleset_info_get": (_I, [_P, _U32, ctypes.POINTER(RulesetInfo)]),
    "tang_tuple_get": (_I, [_P, _U32, _U32] + [ctypes.POINTER(_U32)] * 4),
    "tang_rule_conflicts": (_I, [_P, _U32, _U32, ctypes.POINTER(_U32), _P]),
    "tang_load_model": (_I, [_P, _U32, _P, _SZ]),
    "tang_classify": (_I, [_P, _U32, _P, _U32, _P, _U32, _P, ctypes.POINTER(Stats)]),
    "tang_infer": (_I, [_P, _U32, _P, _U32, _P, _P, _I, _P]),
    "tang_search": (_I, [_P, _U32, _P, _P, _U32, _P, _P, ctypes.POINTER(Stats)]),
    "tang_insert_rule": (_I, [_P, _U32, _P]),
    "tang_delete_rule": (_I, [_P, _U32, _U32]),
    "tang_suboptimal_count": (_I, [_P, _U32, ctypes.POINTER(_U64)]),
    "tang_train": (_I, [_P, _U32, _P, _U32, ctypes.POINTER(TrainCfg), _P, ctypes.POINTER(_SZ), ctypes.POINTER(TrainReport)]),
    "tang_loss_grad": (_I, [_P, _U32, _U32, _U32, _U32, _P, _P, _P, _U32, _F, ctypes.POINTER(_F), _P]),
    "tang_adam_step": (_I, [_P, _P, _P, _P, _P, _U64, _U32, _F, _F, _F, _F]),
    "tang_autotune": (_I, [_P, _U32, _P, _U32, _U32]),
    "tang_serve_start": (_I, [_P, ctypes.POINTER(ServeCfg)]),
    "tang_serve_submit": (_I, [_P, _U32, _P, _U32, _P, ctypes.POINTER(_U64)]),
    "tang_serve_poll": (_I, [_P, _U64, _I, ctypes.POINTER(ReqStats)]),
    "tang_serve_stop": (_I, [_P]),
    "tang_serve_info_get": (_I, [_P, ctypes.POINTER(ServeInfo)]),
    "tang_now": (ctypes.c_double, []),
    "tang_classify_noalloc": (_I, [_P, _U32, _P, _U32, _P, _P]),
    "tang_search_ex": (_I, [_P, _U32, _P, _P, _U32, _P, _U32, _P, ctypes.POINTER(Stats)]),
    "tang_graph_count": (_I, [_P, ctypes.POINTER(_U32)]),
    "tang_du_decide": (_I, [ctypes.POINTER(DuCfg), ctypes.c_double, ctypes.c_double, _U64]),
    "tang_du_observe": (_I, [_P, _U32, _U64, ctypes.c_double]),
    "tang_du_close_window": (_I, [_P, _U32, ctypes.POINTER(DuCfg), ctypes.POINTER(DuWindow)]),
    "tang_finetune": (_I, [_P, _U32, _P, _U32, ctypes.POINTER(TrainCfg), _P, ctypes.POINTER(_SZ), ctypes.POINTER(TrainReport)]),
    "tang_rebuild_ruleset": (_I, [_P, _U32, ctypes.POINTER(_I)]),
    "tang_du_apply": (_I, [_P, _U32, _I, _P, _U32, ctypes.POINTER(TrainCfg), ctypes.POINTER(TrainReport)]),
    "tang_classify_hybrid": (_I, [_P, _U32, _P, _U32, _P, ctypes.POINTER(HybridCfg), ctypes.POINTER(Stats)]),
    "tang_autotune_get": (_I, [_P, _U32, _U32] + [ctypes.POINTER(_I)] * 4 + [ctypes.POINTER(_F)]),
    "tang_selftest_wait_timeout": (_I, [_P, _U32, ctypes.POINTER(_F)]),
    "tang_export_rules": (_I, [_P, _U32, _P, _U32, ctypes.POINTER(_U32)]),
    "tang_checked_build": (_I, []),
    "tang_autotune_set": (_I, [_P, _U32, _U32, _I, _I, _I, _I]),
    "tang_debug_set_pool_view": (_I, [_P, _U32, _U32]),
}


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libtang.so is not built (run paper_2601_03187_b300.build.build()); no fallback exists")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


class _Lib:
    """The loaded library, opened on first use (so the build step can import this package before
    libtang.so exists); a missing library raises at that first use."""

    _real = None

    def __getattr__(self, name):
        if _Lib._real is None:
            _Lib._real = load_library()
        return getattr(_Lib._real, name)


lib = _Lib()

# Extra entry points that a build may add beside the ones above.
EXPORTED = sorted(_SIGS)


def _ptr(x):
    """Device pointer of a torch tensor, host pointer of a numpy array, or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError("expected a torch tensor, numpy array or int pointer, got %r" % type(x))


CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy


def _stream(s):
    """cudaStream_t for a device-mode call: the given torch stream (or raw handle), else torch's
    current stream, so that torch work queued afterwards is ordered after the library's kernels."""
    if s is None:
        import torch
        s = torch.cuda.current_stream()
    h = s.cuda_stream if hasattr(s, "cuda_stream") else int(s)
    return h if h != 0 else CUDA_STREAM_LEGACY


def _n_headers(h):
    if isinstance(h, np.ndarray):
        if h.dtype != HEADER_DTYPE:
            raise TypeError("host headers must use HEADER_DTYPE")
        return len(h)
    if not h.is_contiguous():
        raise ValueError("headers tensor must be contiguous")
    return h.numel() * h.element_size() // 16


def pack_model(p: dict, amax=None) -> bytes:
    """Model blob of include/tang.h from float parameters (x.W convention, W: (in, out))."""
    S, N = p["W0"].shape
    blocks = len(p["W1"])
    C = p["Wc"].shape[1]
    if amax is None:
        amax = np.zeros(2 * blocks + 1, dtype=np.float32)
    head = struct.pack("<6I10I", MODEL_MAGIC, 1, S, N, blocks, C, *([0] * 10))
    parts = [np.asarray(p["W0"]), np.asarray(p["b0"])]
    for k in range(blocks):
        parts += [np.asarray(p["W1"][k]), np.asarray(p["b1"][k]), np.asarray(p["W2"][k]), np.asarray(p["b2"][k])]
    parts += [np.asarray(p["Wc"]), np.asarray(p["bc"])]
    body = b"".join(np.ascontiguousarray(a, dtype=np.float32).tobytes() for a in parts)
    return head + np.asarray(amax, dtype=np.float32).tobytes() + body


def unpack_model(blob: bytes):
    """(params dict of float32 arrays, amax) from a model blob."""
    magic, ver, S, N, blocks, C = struct.unpack_from("<6I", blob, 0)
    if magic != MODEL_MAGIC or ver != 1:
        raise ValueError("not a TaNG model blob")
    off = MODEL_HEADER_BYTES
    amax = np.frombuffer(blob, dtype=np.float32, count=2 * blocks + 1, offset=off).copy()
    off += 4 * (2 * blocks + 1)

    def take(*shape):
        nonlocal off
        cnt = int(np.prod(shape))
        a = np.frombuffer(blob, dtype=np.float32, count=cnt, offset=off).reshape(shape).copy()
        off += 4 * cnt
        return a

    p = {"W0": take(S, N), "b0": take(N), "W1": [], "b1": [], "W2": [], "b2": []}
    for _ in range(blocks):
        p["W1"].append(take(N, N))
        p["b1"].append(take(N))
        p["W2"].append(take(N, N))
        p["b2"].append(take(N))
    p["Wc"] = take(N, C)
    p["bc"] = take(C)
    return p, amax


class Context:
    """One tang_ctx on one CUDA device."""

    def __init__(self, device: int = 0, pool_bytes: int = 0):
        h = ctypes.c_void_p()
        rc = lib.tang_create(device, pool_bytes, ctypes.byref(h))
        if rc != OK:
            raise TangError(rc, "tang_create(device=%d) failed" % device)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib.tang_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, rc, what):
        if rc != OK:
            raise TangError(rc, "%s: %s" % (what, lib.tang_last_error(self._h).decode(errors="replace")))
        return rc

    @property
    def handle(self):
        return self._h

    def memory_usage(self):
        u, c = ctypes.c_size_t(), ctypes.c_size_t()
        self._ck(lib.tang_memory_usage(self._h, ctypes.byref(u), ctypes.byref(c)), "memory_usage")
        return u.value, c.value

    # -- rulesets ---------------------------------------------------------------------------
    def load_ruleset(self, rules: np.ndarray) -> int:
        rules = np.ascontiguousarray(rules, dtype=RULE_DTYPE)
        rs = ctypes.c_uint32()
        self._ck(lib.tang_load_ruleset(self._h, rules.ctypes.data if len(rules) else None, len(rules), ctypes.byref(rs)),
                 "load_ruleset")
        return rs.value

    def unload_ruleset(self, rs: int):
        self._ck(lib.tang_unload_ruleset(self._h, rs), "unload_ruleset")

    def ruleset_info(self, rs: int) -> dict:
        info = RulesetInfo()
        self._ck(lib.tang_ruleset_info_get(self._h, rs, ctypes.byref(info)), "ruleset_info")
        return {k: getattr(info, k) for k, _ in info._fields_}

    def tuple_get(self, rs: int, t: int):
        v = [ctypes.c_uint32() for _ in range(4)]
        self._ck(lib.tang_tuple_get(self._h, rs, t, *[ctypes.byref(x) for x in v]), "tuple_get")
        return tuple(x.value for x in v)

    def rule_conflicts(self, rs: int, rule_id: int):
        words = np.zeros(self.ruleset_info(rs)["conflict_words"], dtype=np.uint32)
        t = ctypes.c_uint32()
        self._ck(lib.tang_rule_conflicts(self._h, rs, rule_id, ctypes.byref(t), words.ctypes.data), "rule_conflicts")
        return t.value, words

    def load_model(self, rs: int, blob: bytes):
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        self._ck(lib.tang_load_model(self._h, rs, buf, len(blob)), "load_model")

    # -- classification ---------------------------------------------------------------------
    def classify(self, rs: int, headers, ids, path="fused_bf16", graph=False, stream=None, stats=False, variant=None,
                 paper=False, serial=False):
        """ids[i] = matching rule id. numpy headers/ids -> host mode; torch CUDA tensors -> device mode.
        variant: None (tuned / default), "n256" or "pair" tensor-core kernel, or "split" (fused paths:
        the network kernel, then the search kernel in place in ids). paper: the paper's
        non-exact post-verification (TANG_SEARCH_PAPER), for measurement. serial: one thread per
        rule run (TANG_SEARCH_SERIAL), for measurement."""
        host = isinstance(headers, np.ndarray)
        flags = (PATHS[path] if isinstance(path, str) else int(path)) | VARIANTS[variant]
        flags |= MEM_HOST if host else MEM_DEVICE
        if graph:
            flags |= GRAPH
        if paper:
            flags |= SEARCH_PAPER
        if serial:
            flags |= SEARCH_SERIAL
        n = _n_headers(headers)
        st = Stats()
        self._ck(lib.tang_classify(self._h, rs, _ptr(headers), n, _ptr(ids), flags,
                                   None if host else _stream(stream),
                                   ctypes.byref(st) if stats else None), "classify")
        return st.as_dict() if stats else None

    def infer(self, rs: int, headers, logits=None, tuples=None, precision=BF16, stream=None, variant=None):
        n = _n_headers(headers)
        self._ck(lib.tang_infer(self._h, rs, _ptr(headers), n, _ptr(logits), _ptr(tuples),
                                precision | VARIANTS[variant], _stream(stream)), "infer")

    def search(self, rs: int, headers, tuples, ids, stream=None, stats=False, paper=False, serial=False):
        n = _n_headers(headers)
        st = Stats()
        self._ck(lib.tang_search_ex(self._h, rs, _ptr(headers), _ptr(tuples), n, _ptr(ids),
                                    (SEARCH_PAPER if paper else 0) | (SEARCH_SERIAL if serial else 0), _stream(stream),
                                    ctypes.byref(st) if stats else None), "search")
        return st.as_dict() if stats else None

    def graph_count(self) -> int:
        c = ctypes.c_uint32()
        self._ck(lib.tang_graph_count(self._h, ctypes.byref(c)), "graph_count")
        return c.value

    def classify_hybrid(self, rs: int, headers: np.ndarray, ids: np.ndarray, batch=8192, streams=4, threads=0,
                        precision=BF16, paper=False, stats=False):
        """The paper's CPU-GPU pipeline (tang_classify_hybrid): network on the GPU, search on host threads."""
        if not isinstance(headers, np.ndarray) or headers.dtype != HEADER_DTYPE:
            raise TypeError("host headers (HEADER_DTYPE) required")
        if not isinstance(ids, np.ndarray) or ids.dtype != np.uint32 or len(ids) < len(headers):
            raise TypeError("host uint32 ids of at least len(headers) required")
        c = HybridCfg(batch=batch, streams=streams, threads=threads, precision=precision,
                      flags=SEARCH_PAPER if paper else 0)
        st = Stats()
        self._ck(lib.tang_classify_hybrid(self._h, rs, headers.ctypes.data, len(headers), ids.ctypes.data,
                                          ctypes.byref(c), ctypes.byref(st) if stats else None), "classify_hybrid")
        return st.as_dict() if stats else None

    def classify_noalloc(self, rs: int, headers, ids, stream=None):
        """Staged BF16 classify whose inter-kernel scratch is a static device array (no allocation)."""
        n = _n_headers(headers)
        self._ck(lib.tang_classify_noalloc(self._h, rs, _ptr(headers), n, _ptr(ids), _stream(stream)),
                 "classify_noalloc")

    # -- updates ----------------------------------------------------------------------------
    def insert_rule(self, rs: int, rule):
        r = np.ascontiguousarray(np.asarray(rule, dtype=RULE_DTYPE).reshape(1))
        self._ck(lib.tang_insert_rule(self._h, rs, r.ctypes.data), "insert_rule")

    def delete_rule(self, rs: int, rule_id: int):
        self._ck(lib.tang_delete_rule(self._h, rs, int(rule_id)), "delete_rule")

    def export_rules(self, rs: int) -> np.ndarray:
        """The live rules in ascending (priority, id) (tang_export_rules)."""
        n = ctypes.c_uint32()
        self._ck(lib.tang_export_rules(self._h, rs, None, 0, ctypes.byref(n)), "export_rules")
        out = np.zeros(n.value, dtype=RULE_DTYPE)
        if n.value:
            self._ck(lib.tang_export_rules(self._h, rs, out.ctypes.data, n.value, ctypes.byref(n)), "export_rules")
        return out

    def suboptimal_count(self, rs: int) -> int:
        c = ctypes.c_uint64()
        self._ck(lib.tang_suboptimal_count(self._h, rs, ctypes.byref(c)), "suboptimal_count")
        return c.value

    # -- training ---------------------------------------------------------------------------
    @staticmethod
    def _train_cfg(cfg):
        c = TrainCfg(N=512, blocks=6, batch=8192, epochs=1000, max_rounds=3, decay_every=200, lr=1e-3, decay=0.1,
                     alpha=1000, beta=0.95, holdout=0.1, time_budget_s=0.0, seed=0)
        for k, v in cfg.items():
            setattr(c, k, v)
        return c

    def _train_call(self, fn, what, rs, samples, c):
        samples = np.ascontiguousarray(samples, dtype=HEADER_DTYPE)
        size = ctypes.c_size_t(0)
        rep = TrainReport()
        # size query first (blob == NULL), then the real call into a buffer of that size
        buf = None
        for _ in range(2):
            self._ck(fn(self._h, rs, samples.ctypes.data, len(samples), ctypes.byref(c), buf, ctypes.byref(size),
                        ctypes.byref(rep)), what)
            if buf is not None:
                break
            buf = ctypes.create_string_buffer(size.value)
        return buf.raw[: size.value], {k: getattr(rep, k) for k, _ in rep._fields_}

    def train(self, rs: int, samples: np.ndarray, **cfg):
        c = self._train_cfg(cfg)
        T = self.ruleset_info(rs)["n_tuples"]
        nparams = 7 * c.N + c.N + c.blocks * (2 * c.N * c.N + 2 * c.N) + c.N * T + T
        size = ctypes.c_size_t(MODEL_HEADER_BYTES + 4 * (2 * c.blocks + 1) + 4 * nparams)
        buf = ctypes.create_string_buffer(size.value)
        rep = TrainReport()
        samples = np.ascontiguousarray(samples, dtype=HEADER_DTYPE)
        self._ck(lib.tang_train(self._h, rs, samples.ctypes.data, len(samples), ctypes.byref(c), buf,
                                ctypes.byref(size), ctypes.byref(rep)), "train")
        return buf.raw[: size.value], {k: getattr(rep, k) for k, _ in rep._fields_}

    def finetune(self, rs: int, samples: np.ndarray, **cfg):
        """Incremental training from the ruleset's loaded model (tang_finetune): (blob, report)."""
        return self._train_call(lib.tang_finetune, "finetune", rs, samples, self._train_cfg(cfg))

    # -- deferred update (§5.2.2) -----------------------------------------------------------
    def rebuild_ruleset(self, rs: int) -> bool:
        """Rebuild the tuple space over the live rules; True if the loaded model was kept."""
        kept = ctypes.c_int()
        self._ck(lib.tang_rebuild_ruleset(self._h, rs, ctypes.byref(kept)), "rebuild_ruleset")
        return bool(kept.value)

    def du_observe(self, rs: int, packets: int, cost: float):
        self._ck(lib.tang_du_observe(self._h, rs, int(packets), float(cost)), "du_observe")

    def du_close_window(self, rs: int, tau: float = 0.05, theta: int = 10000) -> dict:
        c = DuCfg(tau=tau, theta=theta)
        w = DuWindow()
        self._ck(lib.tang_du_close_window(self._h, rs, ctypes.byref(c), ctypes.byref(w)), "du_close_window")
        return {"window": w.window, "th_cur": w.th_cur, "th_base": w.th_base, "suboptimal": w.suboptimal,
                "decision": DU_DECISIONS[w.decision]}

    def du_apply(self, rs: int, decision, samples: np.ndarray, **cfg) -> dict:
        d = {v: k for k, v in DU_DECISIONS.items()}[decision] if isinstance(decision, str) else int(decision)
        c = self._train_cfg(cfg)
        samples = np.ascontiguousarray(samples, dtype=HEADER_DTYPE)
        rep = TrainReport()
        self._ck(lib.tang_du_apply(self._h, rs, d, samples.ctypes.data, len(samples), ctypes.byref(c),
                                   ctypes.byref(rep)), "du_apply")
        return {k: getattr(rep, k) for k, _ in rep._fields_}

    def loss_grad(self, S, N, blocks, C, params: np.ndarray, headers: np.ndarray, labels: np.ndarray, input_scale=1.0):
        params = np.ascontiguousarray(params, dtype=np.float32)
        headers = np.ascontiguousarray(headers, dtype=HEADER_DTYPE)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        grads = np.empty_like(params)
        loss = ctypes.c_float()
        self._ck(lib.tang_loss_grad(self._h, S, N, blocks, C, params.ctypes.data, headers.ctypes.data,
                                    labels.ctypes.data, len(labels), input_scale, ctypes.byref(loss),
                                    grads.ctypes.data), "loss_grad")
        return float(loss.value), grads

    def adam_step(self, params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        for a in (params, grads, m, v):
            assert a.dtype == np.float32 and a.flags.c_contiguous
        self._ck(lib.tang_adam_step(self._h, params.ctypes.data, grads.ctypes.data, m.ctypes.data, v.ctypes.data,
                                    params.size, t, lr, beta1, beta2, eps), "adam_step")

    # -- tuning / serving -------------------------------------------------------------------
    def autotune(self, rs: int, headers, path="fused_bf16"):
        n = _n_headers(headers)
        flags = PATHS[path] if isinstance(path, str) else int(path)
        self._ck(lib.tang_autotune(self._h, rs, _ptr(headers), n, flags), "autotune")

    def autotune_get(self, rs: int, path="fused_bf16") -> dict:
        v = [ctypes.c_int() for _ in range(4)]
        ms = ctypes.c_float()
        self._ck(lib.tang_autotune_get(self._h, rs, PATHS[path] if isinstance(path, str) else int(path),
                                       *[ctypes.byref(x) for x in v], ctypes.byref(ms)), "autotune_get")
        names = {0: "default", 5: "n256", 6: "pair", 7: "split"}
        return {"variant": names.get(v[0].value, str(v[0].value)), "grid": v[1].value, "search_threads": v[2].value,
                "search_bps": v[3].value, "ms": round(ms.value, 4)}

    def autotune_set(self, rs: int, path="fused_bf16", variant="default", grid=0, search_threads=0, search_bps=0):
        """Set (rs, path)'s launch shape, e.g. a dict saved from autotune_get (tang_autotune_set)."""
        names = {"default": 0, "n256": 5, "pair": 6, "split": 7}
        v = names[variant] if isinstance(variant, str) else int(variant)
        self._ck(lib.tang_autotune_set(self._h, rs, PATHS[path] if isinstance(path, str) else int(path), v, int(grid),
                                       int(search_threads), int(search_bps)), "autotune_set")

    def selftest_wait_timeout(self, limit_ms: int = 50):
        """(return code, kernel ms) of tang_selftest_wait_timeout; TANG_ETIMEOUT is the designed outcome."""
        ms = ctypes.c_float()
        rc = lib.tang_selftest_wait_timeout(self._h, int(limit_ms), ctypes.byref(ms))
        return rc, float(ms.value)

    def debug_set_pool_view(self, rs: int, n=None):
        """Test hook of checked builds: the ruleset's device descriptor states a rule-pool size of n
        (None: the real size again); see tang_debug_set_pool_view."""
        self._ck(lib.tang_debug_set_pool_view(self._h, rs, 0xFFFFFFFF if n is None else int(n)), "debug_set_pool_view")

    def serve_start(self, max_inflight=8, max_batch=262144, path="fused_bf16"):
        c = ServeCfg(max_inflight=max_inflight, max_batch=max_batch,
                     path=PATHS[path] if isinstance(path, str) else int(path))
        self._ck(lib.tang_serve_start(self._h, ctypes.byref(c)), "serve_start")

    def serve_submit(self, rs: int, headers: np.ndarray, ids: np.ndarray) -> int:
        req = ctypes.c_uint64()
        self._ck(lib.tang_serve_submit(self._h, rs, headers.ctypes.data, len(headers), ids.ctypes.data,
                                       ctypes.byref(req)), "serve_submit")
        return req.value

    def serve_poll(self, req: int, wait_ms: int = 0):
        st = ReqStats()
        rc = lib.tang_serve_poll(self._h, req, wait_ms, ctypes.byref(st))
        if rc == EAGAIN:
            return None
        self._ck(rc, "serve_poll")
        return {"submit_s": st.submit_s, "start_s": st.start_s, "done_s": st.done_s}

    def serve_info(self) -> dict:
        """Counters of the running serving engine (tang_serve_info_get)."""
        i = ServeInfo()
        self._ck(lib.tang_serve_info_get(self._h, ctypes.byref(i)), "serve_info")
        return {k: getattr(i, k) for k, _ in ServeInfo._fields_ if k != "reserved"}

    def serve_stop(self):
        self._ck(lib.tang_serve_stop(self._h), "serve_stop")


def now() -> float:
    return lib.tang_now()


def checked_build() -> bool:
    """True when the loaded library was built with TANG_CHECKED (tang_checked_build)."""
    return bool(lib.tang_checked_build())


def du_decide(tau: float, theta: int, th_base: float, th_cur: float, suboptimal: int) -> str:
    """The deferred-update rule of §5.2.2 (tang_du_decide): "none", "incremental" or "retrain"."""
    c = DuCfg(tau=tau, theta=theta)
    rc = lib.tang_du_decide(ctypes.byref(c), float(th_base), float(th_cur), int(suboptimal))
    if rc < 0:
        raise TangError(rc, "tang_du_decide: bad configuration")
    return DU_DECISIONS[rc]
