"""Pins for the oracle's §2.1 linear scan, each against something other than the oracle itself."""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import classify as oc
from golden_io import table1, worked_examples

def _points_3bit():
    """All 64 headers of Table 1's 3-bit (X, Y) space, X/Y in the top bits of SIP/DIP."""
    h = np.zeros(64, dtype=wl.HEADER_DTYPE)
    for k, (x, y) in enumerate(itertools.product(range(8), range(8))):
        h["sip"][k] = x << 29
        h["dip"][k] = y << 29
    return h


def _pattern_set(pat):
    """Explicit set of 3-bit values a pattern like '0**' covers (string matching, no masks)."""
    return {v for v in range(8) if format(v, "03b").startswith(pat.rstrip("*"))}


def test_table1_map_matches_set_expansion():
    """Every point of Table 1's field space: oracle vs. assigning each point by explicit rule sets."""
    rules, names, _, _, patterns = table1()
    h = _points_3bit()
    got = oc.classify(rules, h, threads=1)
    for k, (x, y) in enumerate(itertools.product(range(8), range(8))):
        owners = [i for i, (px, py) in enumerate(patterns) if x in _pattern_set(px) and y in _pattern_set(py)]
        want = min(owners, key=lambda i: int(rules["priority"][i])) if owners else None
        assert got[k] == (wl.NO_MATCH if want is None else rules["id"][want]), (x, y)


def test_table1_paper_point():
    """§4.2: the area R1 shares with R6 and R8 belongs to R1."""
    rules, names, *_ = table1()
    ex = [e for e in worked_examples() if e[0] == "classify"]
    assert ex
    for _, kv, expected, _ in ex:
        h = np.zeros(1, dtype=wl.HEADER_DTYPE)
        h["sip"] = int(kv["X"], 2) << 29
        h["dip"] = int(kv["Y"], 2) << 29
        got = oc.classify(rules, h, threads=1)[0]
        assert names[list(rules["id"]).index(got)] == expected


def _interval(value, length):
    """A prefix as the closed integer interval it covers (no bit masks)."""
    span = 1 << (32 - int(length))
    lo = (int(value) // span) * span
    return lo, lo + span - 1


def _small_ruleset(rng, n):
    r = wl.gen_rules(n, int(rng.integers(1 << 30)))
    # short, coarse prefixes so that rules overlap often
    for f in ("sip", "dip"):
        L = rng.choice([0, 1, 2, 3, 32], size=n)
        r[f + "_len"] = L
        top = rng.integers(0, 8, size=n).astype(np.uint64) << np.uint64(29)
        vals = (top | rng.integers(0, 1 << 29, size=n).astype(np.uint64)).astype(np.uint32)
        r[f] = np.array([_interval(v, l)[0] for v, l in zip(vals, L)], dtype=np.uint32)
    r["priority"] = rng.permutation(n)
    return r


def test_elementary_cells_exhaustive():
    """Random <=6-rule rulesets: every elementary cell of the 5-D header space.

    Per field, the rules' interval endpoints lo and hi+1 cut the axis into cells on which every
    rule condition is constant; the oracle is checked on both corners of every cell against
    interval containment (a formulation with no prefix masks).
    """
    rng = np.random.default_rng(7)
    for trial in range(12):
        n = int(rng.integers(1, 7))
        r = _small_ruleset(rng, n)
        iv = {
            "sip": [_interval(r["sip"][i], r["sip_len"][i]) for i in range(n)],
            "dip": [_interval(r["dip"][i], r["dip_len"][i]) for i in range(n)],
            "sp": [(int(r["sp_lo"][i]), int(r["sp_hi"][i])) for i in range(n)],
            "dp": [(int(r["dp_lo"][i]), int(r["dp_hi"][i])) for i in range(n)],
        }
        top = {"sip": (1 << 32) - 1, "dip": (1 << 32) - 1, "sp": 65535, "dp": 65535}
        cells = {}
        for f in iv:
            cuts = sorted({0} | {lo for lo, _ in iv[f]} | {hi + 1 for _, hi in iv[f] if hi + 1 <= top[f]})
            ends = cuts[1:] + [top[f] + 1]
            cells[f] = [(a, b - 1) for a, b in zip(cuts, ends)]
        protos = sorted({int(p) for p, w in zip(r["proto"], r["proto_wild"]) if not w} | {250})
        pts = []
        for cs, cd, cp, cq in itertools.product(cells["sip"], cells["dip"], cells["sp"], cells["dp"]):
            for corner in (0, 1):
                for pr in protos:
                    pts.append((cs[corner], cd[corner], cp[corner], cq[corner], pr))
        h = np.zeros(len(pts), dtype=wl.HEADER_DTYPE)
        arr = np.array(pts, dtype=np.int64)
        h["sip"], h["dip"], h["sp"], h["dp"], h["proto"] = arr.T
        got = oc.classify(r, h, threads=2)
        for k, (s, d, p, q, pr) in enumerate(pts):
            owners = [
                i for i in range(n)
                if iv["sip"][i][0] <= s <= iv["sip"][i][1] and iv["dip"][i][0] <= d <= iv["dip"][i][1]
                and iv["sp"][i][0] <= p <= iv["sp"][i][1] and iv["dp"][i][0] <= q <= iv["dp"][i][1]
                and (r["proto_wild"][i] or int(r["proto"][i]) == pr)
            ]
            want = min(owners, key=lambda i: (int(r["priority"][i]), int(r["id"][i]))) if owners else None
            assert got[k] == (wl.NO_MATCH if want is None else r["id"][want]), (trial, pts[k])


def test_inside_rule_invariant_and_default():
    """A packet drawn inside rule r returns a rule no worse than r; a packet matching nothing -> default."""
    rules = wl.rules_for_config(0)
    rng = np.random.default_rng(3)
    idx = rng.integers(0, len(rules), 20000)
    h = wl.sample_inside(rules, idx, rng)
    ids, pos = oc.classify(rules, h, return_index=True)
    assert (pos >= 0).all()
    assert (rules["priority"][pos] <= rules["priority"][idx]).all()
    # a ruleset with no wildcards at all: most random headers match nothing
    exact = wl.gen_rules(256, 11, len_weights=[0, 0, 0, 0, 1], port_wild=0.0, port_exact=1.0, proto_wild=0.0)
    rand = wl.uniform_headers(5000, rng)
    out, pos = oc.classify(exact, rand, return_index=True)
    assert ((out == wl.NO_MATCH) == (pos < 0)).all()
    assert (out == wl.NO_MATCH).mean() > 0.99
    # the header of an exact rule matches exactly that rule (or a better duplicate)
    inside = wl.sample_inside(exact, np.arange(256), rng)
    out = oc.classify(exact, inside)
    assert (out != wl.NO_MATCH).all()


def test_threads_agree_and_empty_inputs():
    rules = wl.rules_for_config(0)
    h = wl.trace_for_config(0, rules, scale=0.05)
    a = oc.classify(rules, h, threads=1)
    b = oc.classify(rules, h, threads=7)
    assert (a == b).all()
    assert len(oc.classify(rules, h[:0])) == 0
    assert (oc.classify(rules[:0], h[:10]) == wl.NO_MATCH).all()


def test_priority_ties_break_by_id():
    """Equal priorities: the smaller id wins (reading for ties; the order of input is irrelevant)."""
    r = np.zeros(2, dtype=wl.RULE_DTYPE)
    r["sp_hi"] = r["dp_hi"] = 65535
    r["proto_wild"] = 1
    r["priority"] = 5
    r["id"] = [9, 4]
    h = np.zeros(1, dtype=wl.HEADER_DTYPE)
    assert oc.classify(r, h)[0] == 4
    assert oc.classify(r[::-1].copy(), h)[0] == 4
