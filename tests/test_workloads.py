"""The seeded input generators against the recipe they state (CPU only).

Every parity case and the benchmark draw their rulesets and traces from `workloads/`. These tests
check that the draws have the stated shape: prefix-length mix, port and protocol kinds, priority
and id order, trace mix sizes, Zipf popularity, the clustered generator's block structure, and
reproducibility from the seed.
"""
import numpy as np
import pytest

import workloads as wl
from workloads import synth


def _mask(lengths):
    lengths = lengths.astype(np.uint64)
    return ((np.uint64(0xFFFFFFFF) << (np.uint64(32) - lengths)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


@pytest.mark.parametrize("cfg", [2, 1])
def test_rule_mix_follows_the_stated_weights(cfg):
    c = synth.CONFIGS[cfg]
    r = wl.rules_for_config(cfg, n_rules=200_000)
    n = len(r)
    w = np.asarray(c["len_weights"]) / np.sum(c["len_weights"])
    for f in ("sip", "dip"):
        lens = r[f + "_len"].astype(np.int64)
        assert set(np.unique(lens)) <= {0, 8, 16, 24, 32}
        freq = np.array([(lens == L).mean() for L in (0, 8, 16, 24, 32)])
        assert np.abs(freq - w).max() < 0.005, (f, freq, w)
        # prefix values carry no bits below their length
        assert ((r[f] & ~_mask(lens)) == 0).all()
    for f in ("sp", "dp"):
        lo, hi = r[f + "_lo"].astype(np.int64), r[f + "_hi"].astype(np.int64)
        assert (lo <= hi).all()
        wild = (lo == 0) & (hi == 65535)
        exact = lo == hi
        assert abs(wild.mean() - c["port_wild"]) < 0.005
        assert abs(exact.mean() - c["port_exact"]) < 0.005
        assert abs((~wild & ~exact).mean() - (1 - c["port_wild"] - c["port_exact"])) < 0.005
    pw = r["proto_wild"] != 0
    assert abs(pw.mean() - 0.5) < 0.005
    assert (r["proto"][pw] == 0).all()
    assert set(np.unique(r["proto"][~pw])) == {1, 6, 17}
    assert (r["priority"] == np.arange(n)).all() and (r["id"] == np.arange(n)).all()


def test_config_sizes_and_trace_mix():
    assert synth.CONFIGS[0]["rules"] == 1024 and sum(p[1] for p in synth.CONFIGS[0]["trace"]) == 100_000
    assert synth.CONFIGS[1]["rules"] == 65_536 and sum(p[1] for p in synth.CONFIGS[1]["trace"]) == 1_000_000
    assert synth.CONFIGS[2]["rules"] == 524_288 and sum(p[1] for p in synth.CONFIGS[2]["trace"]) == 16_777_216
    assert synth.CONFIGS[4]["rules"] == 1_048_576
    rules = wl.rules_for_config(0)
    h = wl.trace_for_config(0, rules)
    assert len(h) == 100_000 and h.dtype == wl.HEADER_DTYPE
    # scaling shrinks every part by the same factor
    assert len(wl.trace_for_config(2, wl.rules_for_config(2, n_rules=4096), scale=1 / 1024)) == 16_384


def test_inside_headers_lie_in_their_rule():
    rules = wl.rules_for_config(0)
    rng = np.random.default_rng(3)
    idx = rng.integers(0, len(rules), 50_000)
    h = synth.sample_inside(rules, idx, rng)
    sel = rules[idx]
    for f in ("sip", "dip"):
        m = _mask(sel[f + "_len"])
        assert ((h[f] & m) == (sel[f] & m)).all()
    for f in ("sp", "dp"):
        assert ((h[f] >= sel[f + "_lo"]) & (h[f] <= sel[f + "_hi"])).all()
    fixed = sel["proto_wild"] == 0
    assert (h["proto"][fixed] == sel["proto"][fixed]).all()
    # wildcard bits are drawn, not left at zero
    free = sel["sip_len"] < 32
    assert (h["sip"][free] & ~_mask(sel["sip_len"][free])).any()


@pytest.mark.parametrize("alpha", [1.0, 1.2])
def test_zipf_ranks_follow_the_power_law(alpha):
    rng = np.random.default_rng(4)
    k = synth.zipf_ranks(100_000, alpha, 2_000_000, rng)
    assert k.min() >= 0 and k.max() < 100_000
    counts = np.bincount(k, minlength=100_000).astype(np.float64)
    # P(k) / P(0) = (k + 1)^-alpha for the head ranks
    for j in (1, 3, 9):
        ratio = counts[j] / counts[0]
        assert abs(ratio - (j + 1) ** -alpha) < 0.03 * (j + 1) ** -alpha + 0.01, (j, ratio)


def test_traces_are_reproducible_from_the_seed():
    rules = wl.rules_for_config(0)
    parts = [("inside", 5000), ("zipf", 5000, 1.2), ("random", 1000)]
    a = wl.gen_trace(rules, parts, 7)
    b = wl.gen_trace(rules, parts, 7)
    c = wl.gen_trace(rules, parts, 8)
    assert len(a) == 11_000
    assert (a.view(np.uint8) == b.view(np.uint8)).all()
    assert not (a.view(np.uint8) == c.view(np.uint8)).all()
    assert (wl.gen_rules(1000, 5) == wl.gen_rules(1000, 5)).all()


def test_clustered_rules_tie_address_blocks_to_lengths():
    r = wl.gen_clustered_rules(65_536, 70)
    blocks = (r["sip"] >> 24).astype(np.int64) * 256 + (r["dip"] >> 24).astype(np.int64)
    ub, inv = np.unique(blocks, return_inverse=True)
    assert len(ub) == 64
    assert set(np.unique(r["sip_len"])) <= {8, 16, 24, 32} and set(np.unique(r["dip_len"])) <= {8, 16, 24, 32}
    # per block, the most common (SIP length, DIP length) pair covers about 97 % + 3 % / 16 of it
    pair = r["sip_len"].astype(np.int64) * 64 + r["dip_len"].astype(np.int64)
    share = []
    for b in range(len(ub)):
        p = pair[inv == b]
        share.append(np.bincount(p).max() / len(p))
    assert np.median(share) > 0.95
    assert (np.sort(r["priority"]) == np.arange(len(r))).all()
    for f in ("sip", "dip"):
        assert ((r[f] & ~_mask(r[f + "_len"])) == 0).all()
