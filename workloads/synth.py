"""Seeded synthetic rulesets, packet traces, update streams and serving arrivals.

Record layouts are the 16-byte header and 32-byte rule of the C ABI (include/tang.h):

    header: sip u32, dip u32, sp u16, dp u16, proto u8, 3 pad bytes
    rule:   sip u32, dip u32, sp_lo u16, sp_hi u16, dp_lo u16, dp_hi u16,
            sip_len u8, dip_len u8, proto u8, proto_wild u8, priority u32, id u32, reserved u32

Rules follow the 5-field model of §2.1: SIP/DIP prefixes, SP/DP inclusive ranges, protocol
exact or wildcard, one priority per rule (smaller value = higher priority, Table 1).
Prefix values are stored already truncated to their length (low bits zero).

Everything here is random-number drawing only; no classification arithmetic lives here.
"""
from __future__ import annotations

import numpy as np

HEADER_DTYPE = np.dtype(
    [("sip", "<u4"), ("dip", "<u4"), ("sp", "<u2"), ("dp", "<u2"), ("proto", "u1"), ("pad", "u1", (3,))]
)
RULE_DTYPE = np.dtype(
    [
        ("sip", "<u4"), ("dip", "<u4"),
        ("sp_lo", "<u2"), ("sp_hi", "<u2"), ("dp_lo", "<u2"), ("dp_hi", "<u2"),
        ("sip_len", "u1"), ("dip_len", "u1"), ("proto", "u1"), ("proto_wild", "u1"),
        ("priority", "<u4"), ("id", "<u4"), ("reserved", "<u4"),
    ]
)
assert HEADER_DTYPE.itemsize == 16 and RULE_DTYPE.itemsize == 32

NO_MATCH = 0xFFFFFFFF

LEN_CHOICES = np.array([0, 8, 16, 24, 32], dtype=np.int64)
LEN_WEIGHTS_DEFAULT = np.array([0.10, 0.15, 0.25, 0.30, 0.20])
LEN_WEIGHTS_SKEWED = np.array([0.25, 0.30, 0.25, 0.15, 0.05])
PROTO_CHOICES = np.array([6, 17, 1], dtype=np.uint8)


def _prefix_bits(lengths: np.ndarray) -> np.ndarray:
    """uint32 masks with the top `len` bits set (len 0 -> 0), built without a 32-bit shift."""
    lengths = lengths.astype(np.uint64)
    full = np.uint64(0xFFFFFFFF)
    return ((full << (np.uint64(32) - lengths)) & full).astype(np.uint32)


def _ports(rng: np.random.Generator, n: int, p_wild: float, p_exact: float):
    kind = rng.random(n)
    a = rng.integers(0, 65536, n)
    b = rng.integers(0, 65536, n)
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    wild = kind < p_wild
    exact = (~wild) & (kind < p_wild + p_exact)
    lo = np.where(wild, 0, np.where(exact, a, lo))
    hi = np.where(wild, 65535, np.where(exact, a, hi))
    return lo.astype(np.uint16), hi.astype(np.uint16)


def gen_rules(
    n: int,
    seed: int,
    len_weights=LEN_WEIGHTS_DEFAULT,
    port_wild: float = 0.5,
    port_exact: float = 0.3,
    proto_wild: float = 0.5,
    first_priority: int = 0,
    first_id: int = 0,
) -> np.ndarray:
    """Draw `n` rules. Priority and id both equal `first_* + index` (priority = rule index)."""
    rng = np.random.default_rng(seed)
    w = np.asarray(len_weights, dtype=np.float64)
    w = w / w.sum()
    r = np.zeros(n, dtype=RULE_DTYPE)
    sl = rng.choice(LEN_CHOICES, size=n, p=w)
    dl = rng.choice(LEN_CHOICES, size=n, p=w)
    r["sip_len"] = sl
    r["dip_len"] = dl
    r["sip"] = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32) & _prefix_bits(sl)
    r["dip"] = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32) & _prefix_bits(dl)
    r["sp_lo"], r["sp_hi"] = _ports(rng, n, port_wild, port_exact)
    r["dp_lo"], r["dp_hi"] = _ports(rng, n, port_wild, port_exact)
    wild = rng.random(n) < proto_wild
    r["proto_wild"] = wild.astype(np.uint8)
    r["proto"] = np.where(wild, 0, rng.choice(PROTO_CHOICES, size=n))
    r["priority"] = np.arange(first_priority, first_priority + n, dtype=np.uint64).astype(np.uint32)
    r["id"] = np.arange(first_id, first_id + n, dtype=np.uint64).astype(np.uint32)
    return r


def gen_clustered_rules(
    n: int,
    seed: int,
    n_blocks: int = 64,
    p_block_len: float = 0.97,
    first_id: int = 0,
    priority_range: int | None = None,
    lengths=(8, 16, 24, 32),
) -> np.ndarray:
    """Rules clustered in address blocks, each block with its own typical prefix lengths.

    n_blocks distinct (SIP /8, DIP /8) pairs are drawn; every block gets a (SIP length, DIP
    length) pair uniform over lengths^2 (default {8,16,24,32}^2; all lengths must be >= 8). A rule picks a block uniformly, takes the block's
    lengths with probability p_block_len (else uniform lengths from the same set), and random
    address bits below the block's /8. Ports and protocol as gen_rules' defaults. Priorities are
    uniform draws from [0, priority_range) (default: a permutation of 0..n-1); ids are
    first_id + index. This stands in for rulesets whose address structure ties regions of the
    header space to tuples (as ClassBench-ng rulesets do), which a network can learn; rules of
    "another ruleset" are the same draw with another seed.
    """
    rng = np.random.default_rng(seed)
    pairs = rng.choice(1 << 16, n_blocks, replace=False)
    b_sip = (pairs >> 8).astype(np.uint32) << np.uint32(24)
    b_dip = (pairs & 0xFF).astype(np.uint32) << np.uint32(24)
    lens = np.array(lengths, dtype=np.int64)
    assert lens.min() >= 8 and lens.max() <= 32
    b_ls = rng.choice(lens, n_blocks)
    b_ld = rng.choice(lens, n_blocks)
    blk = rng.integers(0, n_blocks, n)
    own = rng.random(n) < p_block_len
    sl = np.where(own, b_ls[blk], rng.choice(lens, n))
    dl = np.where(own, b_ld[blk], rng.choice(lens, n))
    r = np.zeros(n, dtype=RULE_DTYPE)
    r["sip_len"] = sl
    r["dip_len"] = dl
    low_s = rng.integers(0, 1 << 24, n, dtype=np.uint64).astype(np.uint32)
    low_d = rng.integers(0, 1 << 24, n, dtype=np.uint64).astype(np.uint32)
    r["sip"] = (b_sip[blk] | low_s) & _prefix_bits(sl)
    r["dip"] = (b_dip[blk] | low_d) & _prefix_bits(dl)
    r["sp_lo"], r["sp_hi"] = _ports(rng, n, 0.5, 0.3)
    r["dp_lo"], r["dp_hi"] = _ports(rng, n, 0.5, 0.3)
    wild = rng.random(n) < 0.5
    r["proto_wild"] = wild.astype(np.uint8)
    r["proto"] = np.where(wild, 0, rng.choice(PROTO_CHOICES, size=n))
    if priority_range is None:
        r["priority"] = rng.permutation(n).astype(np.uint32)
    else:
        r["priority"] = rng.integers(0, max(1, priority_range), n).astype(np.uint32)
    r["id"] = np.arange(first_id, first_id + n, dtype=np.uint64).astype(np.uint32)
    return r


def sample_inside(rules: np.ndarray, idx: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """One header drawn uniformly inside each rule `rules[idx[i]]` (wildcard protocol -> 0..255)."""
    sel = rules[idx]
    n = len(idx)
    h = np.zeros(n, dtype=HEADER_DTYPE)
    ms = _prefix_bits(sel["sip_len"])
    md = _prefix_bits(sel["dip_len"])
    h["sip"] = (sel["sip"] & ms) | (rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32) & ~ms)
    h["dip"] = (sel["dip"] & md) | (rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32) & ~md)
    h["sp"] = rng.integers(sel["sp_lo"].astype(np.int64), sel["sp_hi"].astype(np.int64) + 1)
    h["dp"] = rng.integers(sel["dp_lo"].astype(np.int64), sel["dp_hi"].astype(np.int64) + 1)
    h["proto"] = np.where(sel["proto_wild"] != 0, rng.integers(0, 256, n), sel["proto"])
    return h


def uniform_headers(n: int, rng: np.random.Generator) -> np.ndarray:
    h = np.zeros(n, dtype=HEADER_DTYPE)
    h["sip"] = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    h["dip"] = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    h["sp"] = rng.integers(0, 65536, n)
    h["dp"] = rng.integers(0, 65536, n)
    h["proto"] = rng.integers(0, 256, n)
    return h


def zipf_ranks(n_items: int, alpha: float, size: int, rng: np.random.Generator) -> np.ndarray:
    """0-based ranks k with P(k) proportional to (k+1)^-alpha, by inverse CDF over all items."""
    w = np.arange(1, n_items + 1, dtype=np.float64) ** (-float(alpha))
    cdf = np.cumsum(w)
    u = rng.random(size) * cdf[-1]
    return np.minimum(np.searchsorted(cdf, u, side="right"), n_items - 1)


def gen_trace(rules: np.ndarray, parts, seed: int) -> np.ndarray:
    """Concatenate trace parts, then shuffle them with a seeded permutation.

    `parts` is a list of tuples:
      ("inside", count)          - uniformly chosen rule, header uniform inside it
      ("zipf", count, alpha)     - Zipf(alpha) rule popularity over a seeded rank permutation
      ("random", count)          - uniform random header
    """
    rng = np.random.default_rng(seed)
    chunks = []
    perm = None
    for p in parts:
        kind, count = p[0], int(p[1])
        if count == 0:
            continue
        if kind == "inside":
            chunks.append(sample_inside(rules, rng.integers(0, len(rules), count), rng))
        elif kind == "zipf":
            if perm is None:
                perm = rng.permutation(len(rules))
            chunks.append(sample_inside(rules, perm[zipf_ranks(len(rules), p[2], count, rng)], rng))
        elif kind == "random":
            chunks.append(uniform_headers(count, rng))
        else:
            raise ValueError(kind)
    h = np.concatenate(chunks) if chunks else np.zeros(0, dtype=HEADER_DTYPE)
    return h[rng.permutation(len(h))]


# ---------------------------------------------------------------------------------------------
# The five workload configurations (sizes and mixes), each with its seeds.
# ---------------------------------------------------------------------------------------------

CONFIGS = {
    0: dict(rules=1024, len_weights=LEN_WEIGHTS_DEFAULT, port_wild=0.5, port_exact=0.3,
            trace=[("inside", 90_000), ("random", 10_000)], rule_seed=0, trace_seed=0),
    1: dict(rules=65_536, len_weights=LEN_WEIGHTS_SKEWED, port_wild=0.7, port_exact=0.18,
            trace=[("zipf", 1_000_000, 1.0)], rule_seed=0, trace_seed=1),
    2: dict(rules=524_288, len_weights=LEN_WEIGHTS_DEFAULT, port_wild=0.5, port_exact=0.3,
            trace=[("inside", 8_388_608), ("zipf", 8_388_608, 1.2)], rule_seed=0, trace_seed=1),
    4: dict(rules=1_048_576, len_weights=LEN_WEIGHTS_DEFAULT, port_wild=0.5, port_exact=0.3,
            trace=[("inside", 131_072), ("zipf", 131_072, 1.2)], rule_seed=0, trace_seed=1),
}


def rules_for_config(cfg: int, n_rules: int | None = None, seed: int | None = None) -> np.ndarray:
    c = CONFIGS[cfg]
    return gen_rules(
        c["rules"] if n_rules is None else n_rules,
        c["rule_seed"] if seed is None else seed,
        len_weights=c["len_weights"], port_wild=c["port_wild"], port_exact=c["port_exact"],
    )


def trace_for_config(cfg: int, rules: np.ndarray, scale: float = 1.0, seed: int | None = None) -> np.ndarray:
    """The configuration's trace mix; `scale` shrinks every part by the same factor."""
    c = CONFIGS[cfg]
    parts = []
    for p in c["trace"]:
        q = list(p)
        q[1] = max(1, int(round(q[1] * scale)))
        parts.append(tuple(q))
    return gen_trace(rules, parts, c["trace_seed"] if seed is None else seed)


def gen_update_stream(rules: np.ndarray, n_ops: int, seed: int, update_frac: float = 0.10,
                      batch_lo: int = 4096, batch_hi: int = 262_144):
    """Operation stream over a live ruleset: ('insert', rule) / ('delete', id) / ('lookup', n, seed).

    Updates are half inserts (fresh rules from an independently seeded generator, new ids from a
    counter, priority uniform over the current priority range) and half deletes of a uniformly
    chosen live id. Lookup batch sizes are log-uniform in [batch_lo, batch_hi].
    """
    rng = np.random.default_rng(seed)
    live = list(int(i) for i in rules["id"])
    pos = {v: i for i, v in enumerate(live)}
    next_id = int(rules["id"].max()) + 1 if len(rules) else 0
    pmax = int(rules["priority"].max()) if len(rules) else 0
    fresh = gen_rules(max(16, n_ops), seed + 1000003)
    fi = 0
    ops = []
    for _ in range(n_ops):
        if rng.random() < update_frac:
            if rng.random() < 0.5 or not live:
                r = fresh[fi % len(fresh)].copy()
                fi += 1
                r["id"] = next_id
                r["priority"] = int(rng.integers(0, pmax + 1))
                next_id += 1
                pos[int(r["id"])] = len(live)
                live.append(int(r["id"]))
                ops.append(("insert", r))
            else:
                k = int(rng.integers(0, len(live)))
                victim = live[k]
                last = live[-1]
                live[k] = last
                pos[last] = k
                live.pop()
                del pos[victim]
                ops.append(("delete", victim))
        else:
            n = int(np.exp(rng.uniform(np.log(batch_lo), np.log(batch_hi + 1))))
            ops.append(("lookup", min(n, batch_hi), int(rng.integers(0, 1 << 31))))
    return ops


def gen_serving_arrivals(n_requests: int, n_rulesets: int, rate_per_s: float, seed: int,
                         batch_lo: int = 1, batch_hi: int = 65_536):
    """Poisson arrivals: (arrival_time_s, ruleset_index, batch_size, trace_seed) per request."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    t = np.cumsum(gaps)
    rs = rng.integers(0, n_rulesets, n_requests)
    sizes = np.exp(rng.uniform(np.log(batch_lo), np.log(batch_hi + 1), n_requests)).astype(np.int64)
    sizes = np.clip(sizes, batch_lo, batch_hi)
    seeds = rng.integers(0, 1 << 31, n_requests)
    return [(float(t[i]), int(rs[i]), int(sizes[i]), int(seeds[i])) for i in range(n_requests)]


def table1_rules() -> np.ndarray:
    """The eight two-field rules of Table 1, X -> top 3 bits of SIP, Y -> top 3 bits of DIP.

    Ports and protocol are wildcards. Priority is the table's priority column; id = priority.
    """
    rows = [  # (X pattern, Y pattern)
        ("000", "011"), ("000", "101"), ("00*", "11*"), ("110", "***"),
        ("111", "***"), ("***", "011"), ("***", "010"), ("0**", "0**"),
    ]
    r = np.zeros(len(rows), dtype=RULE_DTYPE)
    for i, (x, y) in enumerate(rows):
        for fld, pat in (("sip", x), ("dip", y)):
            bits = pat.rstrip("*")
            r[fld + "_len"][i] = len(bits)
            r[fld][i] = (int(bits, 2) << (32 - len(bits))) if bits else 0
    r["sp_lo"], r["sp_hi"], r["dp_lo"], r["dp_hi"] = 0, 65535, 0, 65535
    r["proto_wild"] = 1
    r["priority"] = np.arange(1, len(rows) + 1)
    r["id"] = np.arange(1, len(rows) + 1)
    return r
