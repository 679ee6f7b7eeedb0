"""Pins for the oracle's paper-mode post-verification (§5.1.1 as printed) and for the host-side
deferred-update rule (§5.2.2), against values the paper prints (Table 1 packet of §4.2, the
dynamic experiment of §7.3) and invariants that hold for any prediction."""
import numpy as np

import paper_2601_03187_b300 as tg
import workloads as wl
from golden_io import GOLDEN, pattern_to_prefix, table1, worked_examples
from oracle import classify as oc
from oracle import tss


def _header(x, y):
    h = np.zeros(1, dtype=wl.HEADER_DTYPE)
    h["sip"], _ = pattern_to_prefix(x)
    h["dip"], _ = pattern_to_prefix(y)
    return h


def test_table1_paper_mode_examples():
    """§5.1.1's two scenarios on the §4.2 packet: a wrong tuple with a match keeps its (lower-priority)
    rule; a wrong tuple without one falls back to the ordered search, which finds R1."""
    rules, names, *_ = table1()
    tuples, tor = tss.build_tuples(rules)
    rows = [e for e in worked_examples() if e[0] == "paper"]
    assert len(rows) == 4
    for _, kv, expected, src in rows:
        h = _header(kv["X"], kv["Y"])
        pred = int(kv["predicted"][1:]) - 1
        got = oc.paper_classify(rules, h, [pred], tor)[0]
        assert names[list(rules["id"]).index(got)] == expected, src
        # the exact answer is R1 whatever the prediction
        assert names[list(rules["id"]).index(oc.classify(rules, h)[0])] == "R1"


def test_paper_mode_invariants_random():
    """For any prediction: exact when the prediction is the answer's tuple or absent; otherwise a
    rule of the predicted tuple that matches the packet and is no better than the exact answer,
    and the default id exactly when nothing matches."""
    rng = np.random.default_rng(5)
    rules = wl.gen_rules(300, seed=11)
    tuples, tor = tss.build_tuples(rules)
    T = len(tuples)
    h = wl.gen_trace(rules, [("inside", 3000), ("random", 500)], seed=12)
    exact, pos = oc.classify(rules, h, return_index=True)
    true_t = np.where(pos >= 0, tor[np.maximum(pos, 0)], -1)
    assert (oc.paper_classify(rules, h, true_t, tor) == exact).all()
    assert (oc.paper_classify(rules, h, np.full(len(h), -1), tor) == exact).all()
    assert (oc.paper_classify(rules, h, np.full(len(h), T + 3), tor) == exact).all()
    pred = rng.integers(0, T, len(h))
    got = oc.paper_classify(rules, h, pred, tor)
    assert ((got == wl.NO_MATCH) == (exact == wl.NO_MATCH)).all()
    key = {int(r["id"]): (int(r["priority"]), int(r["id"])) for r in rules}
    row = {int(r["id"]): j for j, r in enumerate(rules)}
    differ = 0
    for i in np.nonzero(got != exact)[0]:
        differ += 1
        j = row[int(got[i])]
        assert tor[j] == pred[i] != true_t[i]
        assert key[int(got[i])] > key[int(exact[i])]
        # the returned rule contains the packet (interval arithmetic, no masks)
        r = rules[j]
        for f in ("sip", "dip"):
            span = 1 << (32 - int(r[f + "_len"]))
            lo = (int(r[f]) // span) * span
            assert lo <= int(h[f][i]) < lo + span
        assert r["sp_lo"] <= h["sp"][i] <= r["sp_hi"] and r["dp_lo"] <= h["dp"][i] <= r["dp_hi"]
        assert r["proto_wild"] or r["proto"] == h["proto"][i]
    assert differ > 0  # random predictions do land on lower-priority matches here


def _golden_du():
    out = []
    with open(GOLDEN + "/deferred_update.txt") as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                kind, inputs, expected, src = [s.strip() for s in line.split("|")]
                out.append((kind, dict(t.split("=") for t in inputs.split()), expected, src))
    return out


def test_du_decide_paper_values():
    """§7.3's printed windows (tau = 5 %, theta = 10,000) through the library's decision rule."""
    rows = _golden_du()
    assert {r[0] for r in rows} == {"decide", "drop"}
    for kind, kv, expected, src in rows:
        base, cur = float(kv["base"]), float(kv["cur"])
        if kind == "decide":
            got = tg.du_decide(float(kv["tau"]), int(kv["theta"]), base, cur, int(kv["suboptimal"]))
            assert got == expected, src
        else:
            # the printed percentage sits between two tau values: the rule fires below it only
            drop = float(expected)
            assert tg.du_decide(drop - 0.0006, 10, base, cur, 0) == "incremental", src
            assert tg.du_decide(drop + 0.0006, 10, base, cur, 0) == "none", src


def test_du_decide_boundaries():
    assert tg.du_decide(0.05, 10, 100.0, 96.0, 0) == "none"          # 4 % drop
    assert tg.du_decide(0.05, 10, 100.0, 94.0, 10) == "incremental"  # counter not above theta
    assert tg.du_decide(0.05, 10, 100.0, 94.0, 11) == "retrain"
    assert tg.du_decide(0.05, 10, 100.0, 120.0, 99) == "none"        # throughput rose
    assert tg.du_decide(0.0, 10, 100.0, 100.0, 99) == "none"         # "exceeds" is strict
    assert tg.du_decide(0.05, 10, 0.0, 50.0, 0) == "none"            # no baseline yet
    try:
        tg.du_decide(-0.1, 10, 100.0, 50.0, 0)
    except tg.TangError:
        pass
    else:
        raise AssertionError("a negative tau must be refused")
