"""ORACLE (test infrastructure): tuple space, restricted insertion and overlap-conflict sets.

Sources in the paper:
  §4.3  tuples group rules by their prefix-length vector; for 5-field rules the tuples are built
        from SIP and DIP lengths only; a rule is truncated to its tuple's lengths (zero the bits
        below the length) and stored in that tuple's hash table under the truncated key.
  §5.2.1 restricted insertion: use the tuple whose lengths equal the rule's; otherwise, among the
        tuples whose lengths are all <= the rule's, the first one with the largest length sum.
  §5.1.1 post-verification searches the remaining tuples when the predicted tuple has no match,
        and (§5.1.1, §8) leaves a lower-priority hit in a wrong tuple uncorrected. The conflict
        sets below close that gap: conflict(r) holds the tuple of every rule that beats r and
        shares at least one header with r. If P matches r, the true answer lies in r's tuple or
        in a tuple of conflict(r), because the true answer also contains P.

Readings where the paper is silent: tuple indices are given in order of first appearance over
rules sorted by (priority, id); a (0, 0) tuple is appended when absent so that every insertion
has a candidate; "first" among equal sums means the lowest tuple index.
"""
from __future__ import annotations

import numpy as np


def prefix_mask(length: int) -> int:
    """Top `length` bits of a 32-bit word; length 0 -> 0."""
    return 0 if length == 0 else ((0xFFFFFFFF << (32 - length)) & 0xFFFFFFFF)


def truncate(value: int, length: int) -> int:
    """§4.3 truncation of a prefix value to a tuple's length."""
    return value & prefix_mask(length)


def priority_order(rules: np.ndarray) -> np.ndarray:
    """Indices of `rules` in ascending (priority, id)."""
    return np.lexsort((rules["id"].astype(np.int64), rules["priority"].astype(np.int64)))


def build_tuples(rules: np.ndarray, ensure_zero_tuple: bool = True):
    """§4.3 tuple construction. Returns (tuples, tuple_of_rule).

    tuples[t] = (sip_len, dip_len); tuple_of_rule[i] = t for rules[i].
    """
    tuples: list[tuple[int, int]] = []
    index: dict[tuple[int, int], int] = {}
    tor = np.empty(len(rules), dtype=np.int64)
    for i in priority_order(rules):
        key = (int(rules["sip_len"][i]), int(rules["dip_len"][i]))
        if key not in index:
            index[key] = len(tuples)
            tuples.append(key)
        tor[i] = index[key]
    if ensure_zero_tuple and (0, 0) not in index:
        tuples.append((0, 0))
    return tuples, tor


def tuple_buckets(rules: np.ndarray, tuples, tuple_of_rule):
    """Per tuple, the hash table contents: {(sip_key, dip_key): [rule positions in (prio, id) order]}."""
    buckets = [dict() for _ in tuples]
    for i in priority_order(rules):
        t = int(tuple_of_rule[i])
        ls, ld = tuples[t]
        key = (truncate(int(rules["sip"][i]), ls), truncate(int(rules["dip"][i]), ld))
        buckets[t].setdefault(key, []).append(int(i))
    return buckets


def restricted_insert_tuple(tuples, sip_len: int, dip_len: int):
    """§5.2.1: exact-length tuple if present, else the first tuple with l^T <= l^R of maximal sum.

    Returns the tuple index, or None when no tuple satisfies l^T <= l^R.
    """
    for t, (ls, ld) in enumerate(tuples):
        if ls == sip_len and ld == dip_len:
            return t
    best, best_sum = None, -1
    for t, (ls, ld) in enumerate(tuples):
        if ls <= sip_len and ld <= dip_len and ls + ld > best_sum:
            best, best_sum = t, ls + ld
    return best


def insertion_candidates(tuples, sip_len: int, dip_len: int):
    """All tuples with l^T <= l^R componentwise (§5.2.1)."""
    return [t for t, (ls, ld) in enumerate(tuples) if ls <= sip_len and ld <= dip_len]


def overlap(a, b) -> bool:
    """Two rules share at least one header: prefixes agree on the shorter length, both port ranges
    intersect, and protocols agree or one is a wildcard."""
    for f in ("sip", "dip"):
        m = prefix_mask(min(int(a[f + "_len"]), int(b[f + "_len"])))
        if (int(a[f]) ^ int(b[f])) & m:
            return False
    for f in ("sp", "dp"):
        if int(a[f + "_hi"]) < int(b[f + "_lo"]) or int(b[f + "_hi"]) < int(a[f + "_lo"]):
            return False
    if not a["proto_wild"] and not b["proto_wild"] and int(a["proto"]) != int(b["proto"]):
        return False
    return True


def conflict_sets(rules: np.ndarray, tuple_of_rule) -> list[set]:
    """conflict(r) = {tuple(r') : (prio', id') < (prio, id) and overlap(r, r')}, brute force O(n^2)."""
    n = len(rules)
    out = [set() for _ in range(n)]
    key = [(int(rules["priority"][i]), int(rules["id"][i])) for i in range(n)]
    for i in range(n):
        for j in range(n):
            if key[j] < key[i] and overlap(rules[i], rules[j]):
                out[i].add(int(tuple_of_rule[j]))
    return out


def conflict_words(rules: np.ndarray, tuple_of_rule, n_tuples: int) -> np.ndarray:
    """conflict_sets() as bitsets, vectorised over the better rules; shape (n, ceil(T/32)) uint32."""
    n = len(rules)
    words = max(1, (n_tuples + 31) // 32)
    out = np.zeros((n, words), dtype=np.uint32)
    pr = rules["priority"].astype(np.int64)
    rid = rules["id"].astype(np.int64)
    sl = rules["sip_len"].astype(np.int64)
    dl = rules["dip_len"].astype(np.int64)
    sip = rules["sip"].astype(np.int64)
    dip = rules["dip"].astype(np.int64)
    masks = np.array([prefix_mask(k) for k in range(33)], dtype=np.int64)
    tor = np.asarray(tuple_of_rule, dtype=np.int64)
    for i in range(n):
        better = (pr < pr[i]) | ((pr == pr[i]) & (rid < rid[i]))
        ms = masks[np.minimum(sl, sl[i])]
        md = masks[np.minimum(dl, dl[i])]
        ok = better & (((sip ^ sip[i]) & ms) == 0) & (((dip ^ dip[i]) & md) == 0)
        ok &= (rules["sp_hi"] >= rules["sp_lo"][i]) & (rules["sp_lo"] <= rules["sp_hi"][i])
        ok &= (rules["dp_hi"] >= rules["dp_lo"][i]) & (rules["dp_lo"] <= rules["dp_hi"][i])
        ok &= (rules["proto_wild"] != 0) | (rules["proto_wild"][i] != 0) | (rules["proto"] == rules["proto"][i])
        for t in np.unique(tor[ok]):
            out[i, t // 32] |= np.uint32(1 << (t % 32))
    return out


class TwoStageSearch:
    """Two-stage search of §5.1.1 made exact with the conflict sets (a plain restatement).

    1. Probe the predicted tuple: truncate the header to the tuple's lengths, look up that key,
       compare the bucket's rules one by one; the first match is the tuple's best.
    2. On a hit r, probe every other tuple in conflict(r); on a miss (or with no prediction),
       probe every other tuple. Tuples are visited in ascending order of their best
       (priority, id); a tuple whose best is worse than the current answer cannot improve it,
       and neither can any later one, so the search stops there. Inside a bucket the rules are
       in (priority, id) order, so a bucket scan stops at the first rule worse than the answer.
    """

    def __init__(self, rules: np.ndarray, tuples, tuple_of_rule):
        self.rules = rules
        self.tuples = tuples
        self.buckets = tuple_buckets(rules, tuples, tuple_of_rule)
        words = conflict_words(rules, tuple_of_rule, len(tuples))
        self.conflicts = [{t for t in range(len(tuples)) if words[i, t // 32] >> (t % 32) & 1}
                          for i in range(len(rules))]
        self.tmin = [None] * len(tuples)
        for i in range(len(rules)):
            t = int(tuple_of_rule[i])
            k = self.key_of(i)
            if self.tmin[t] is None or k < self.tmin[t]:
                self.tmin[t] = k

    def key_of(self, i):
        return (int(self.rules["priority"][i]), int(self.rules["id"][i]))

    def matches(self, i, header) -> bool:
        r = self.rules[i]
        return (
            ((int(header["sip"]) ^ int(r["sip"])) & prefix_mask(int(r["sip_len"]))) == 0
            and ((int(header["dip"]) ^ int(r["dip"])) & prefix_mask(int(r["dip_len"]))) == 0
            and int(r["sp_lo"]) <= int(header["sp"]) <= int(r["sp_hi"])
            and int(r["dp_lo"]) <= int(header["dp"]) <= int(r["dp_hi"])
            and bool(r["proto_wild"] or int(r["proto"]) == int(header["proto"]))
        )

    def probe(self, t, header, best):
        ls, ld = self.tuples[t]
        k = (truncate(int(header["sip"]), ls), truncate(int(header["dip"]), ld))
        for i in self.buckets[t].get(k, []):
            if best is not None and self.key_of(i) >= self.key_of(best):
                break
            if self.matches(i, header):
                return i
        return None

    def search(self, header, predicted):
        """(rule position or -1, tuples probed)."""
        best = None
        probes = 0
        if predicted is not None:
            probes += 1
            best = self.probe(predicted, header, None)
        rest = sorted((t for t in range(len(self.tuples)) if t != predicted and self.tmin[t] is not None),
                      key=lambda t: self.tmin[t])
        if best is not None:
            rest = [t for t in rest if t in self.conflicts[best]]
        for t in rest:
            if best is not None and self.tmin[t] > self.key_of(best):
                break
            probes += 1
            hit = self.probe(t, header, best)
            if hit is not None:
                best = hit
        return (-1 if best is None else best), probes
