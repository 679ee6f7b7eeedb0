"""Pins for the oracle's tuple space (§4.3), restricted insertion (§5.2.1) and conflict sets."""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import classify as oc
from oracle import tss
from golden_io import table1, worked_examples, pattern_to_prefix

def test_table1_tuples():
    """Tuple construction on Table 1 reproduces T1..T5 and their members (plus the appended (0,0))."""
    rules, names, tnames, tlens, _ = table1()
    tuples, tor = tss.build_tuples(rules)
    assert tuples[:5] == [(3, 3), (2, 2), (3, 0), (0, 3), (1, 1)]
    assert tuples[5:] == [(0, 0)]
    for i, tn in enumerate(tnames):
        assert tor[i] == int(tn[1:]) - 1
        assert tuples[tor[i]] == tlens[i]


def test_table1_buckets_hold_every_rule_once():
    rules, *_ = table1()
    tuples, tor = tss.build_tuples(rules)
    b = tss.tuple_buckets(rules, tuples, tor)
    members = sorted(i for t in b for k in t for i in t[k])
    assert members == list(range(len(rules)))
    # T3 = (3, 0): R4 and R5 differ in X, so two keys
    assert len(b[2]) == 2


def _tname(t):
    return "T%d" % (t + 1)


def test_worked_examples():
    rules, *_ = table1()
    tuples, _ = tss.build_tuples(rules)
    seen = set()
    for kind, kv, expected, src in worked_examples():
        if kind == "truncate":
            bits = int(kv["bits"])
            v, _ = pattern_to_prefix(kv["value"])
            got = tss.truncate(v, int(kv["len"])) >> (32 - bits)
            assert format(got, "0%db" % bits) == expected, src
        elif kind == "insert":
            ls, ld = (int(x) for x in kv["lengths"].split(","))
            assert _tname(tss.restricted_insert_tuple(tuples, ls, ld)) == expected, src
        elif kind == "candidates":
            ls, ld = (int(x) for x in kv["lengths"].split(","))
            cands = [_tname(t) for t in tss.insertion_candidates(tuples, ls, ld) if t < 5]
            assert cands == expected.split(","), src
            assert "T4" not in cands  # (0,3) is not <= (3,1): the stated rule excludes it
        seen.add(kind)
    assert seen == {"truncate", "insert", "candidates", "classify", "paper"}


def test_insert_without_candidate_and_ties():
    assert tss.restricted_insert_tuple([(8, 8)], 0, 32) is None
    # equal sums: the first tuple wins
    assert tss.restricted_insert_tuple([(8, 16), (16, 8), (0, 0)], 24, 24) == 0
    assert tss.restricted_insert_tuple([(0, 0), (16, 8), (8, 16)], 24, 24) == 1


def _point_sets_3bit(patterns):
    return [
        {(x, y) for x in range(8) for y in range(8)
         if format(x, "03b").startswith(px.rstrip("*")) and format(y, "03b").startswith(py.rstrip("*"))}
        for px, py in patterns
    ]


def test_table1_conflicts_by_point_sets():
    """conflict(r) on Table 1 vs. explicit point-set intersection (no overlap arithmetic)."""
    rules, names, tnames, _, patterns = table1()
    tuples, tor = tss.build_tuples(rules)
    sets = _point_sets_3bit(patterns)
    want = [
        {int(tor[j]) for j in range(len(rules)) if rules["priority"][j] < rules["priority"][i] and sets[i] & sets[j]}
        for i in range(len(rules))
    ]
    assert tss.conflict_sets(rules, tor) == want
    words = tss.conflict_words(rules, tor, len(tuples))
    for i in range(len(rules)):
        assert {t for t in range(len(tuples)) if words[i, 0] >> t & 1} == want[i]
    # two entries spelled out: R6 = (***, 011) is beaten in part by R1 (T1) and R4, R5 (T3)
    assert want[5] == {0, 2}
    # R8 = (0**, 0**) is beaten in part by R1 (T1) and R6, R7 (T4)
    assert want[7] == {0, 3}
    assert want[0] == set()


def _cell_overlap(a, b):
    """Do two rules share a header? By explicit interval intersection of each field."""
    def iv(v, l):
        span = 1 << (32 - int(l))
        lo = (int(v) // span) * span
        return lo, lo + span - 1
    for f in ("sip", "dip"):
        (a0, a1), (b0, b1) = iv(a[f], a[f + "_len"]), iv(b[f], b[f + "_len"])
        if a1 < b0 or b1 < a0:
            return False
    for f in ("sp", "dp"):
        if int(a[f + "_hi"]) < int(b[f + "_lo"]) or int(b[f + "_hi"]) < int(a[f + "_lo"]):
            return False
    pa = set(range(256)) if a["proto_wild"] else {int(a["proto"])}
    pb = set(range(256)) if b["proto_wild"] else {int(b["proto"])}
    return bool(pa & pb)


def test_conflicts_random_vs_interval_overlap():
    rng = np.random.default_rng(5)
    r = wl.gen_rules(160, 9, len_weights=[0.3, 0.3, 0.2, 0.1, 0.1])
    r["priority"] = rng.permutation(len(r))
    tuples, tor = tss.build_tuples(r)
    words = tss.conflict_words(r, tor, len(tuples))
    for i in range(len(r)):
        want = set()
        for j in range(len(r)):
            if (r["priority"][j], r["id"][j]) < (r["priority"][i], r["id"][i]) and _cell_overlap(r[i], r[j]):
                want.add(int(tor[j]))
        got = {t for t in range(len(tuples)) if words[i, t // 32] >> (t % 32) & 1}
        assert got == want, i


@pytest.mark.parametrize("seed", [0, 1])
def test_exact_two_stage_search_equals_linear_scan(seed):
    """The conflict-set certificate: any predicted tuple yields the linear-scan answer."""
    rng = np.random.default_rng(seed)
    r = wl.gen_rules(120, 20 + seed, len_weights=[0.3, 0.3, 0.2, 0.1, 0.1])
    r["priority"] = rng.permutation(len(r))
    tuples, tor = tss.build_tuples(r)
    h = wl.gen_trace(r, [("inside", 150), ("random", 30)], seed)
    want, pos = oc.classify(r, h, return_index=True)
    s = tss.TwoStageSearch(r, tuples, tor)
    for k in range(len(h)):
        for pred in (None, int(rng.integers(0, len(tuples))), int(tor[pos[k]]) if pos[k] >= 0 else 0):
            got, probes = s.search(h[k], pred)
            assert got == pos[k], (k, pred)
            assert 0 <= probes <= len(tuples)
