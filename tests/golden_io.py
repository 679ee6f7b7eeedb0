"""Readers for the text fixtures under tests/golden/."""
import os

import numpy as np

from workloads import RULE_DTYPE

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


def pattern_to_prefix(pat: str):
    """3-bit pattern like '0**' -> (value placed in the top bits of a 32-bit word, length)."""
    bits = pat.rstrip("*")
    return ((int(bits, 2) << (32 - len(bits))) if bits else 0), len(bits)


def table1():
    """(rules as RULE_DTYPE, names, tuple names, tuple lengths) from Table 1."""
    rows = [l.split() for l in _lines("table1.txt")]
    r = np.zeros(len(rows), dtype=RULE_DTYPE)
    names, tnames, tlens = [], [], []
    for i, (name, prio, x, y, tname, lx, ly) in enumerate(rows):
        r["sip"][i], r["sip_len"][i] = pattern_to_prefix(x)
        r["dip"][i], r["dip_len"][i] = pattern_to_prefix(y)
        r["priority"][i] = int(prio)
        r["id"][i] = int(prio)
        names.append(name)
        tnames.append(tname)
        tlens.append((int(lx), int(ly)))
    r["sp_lo"], r["sp_hi"], r["dp_lo"], r["dp_hi"] = 0, 65535, 0, 65535
    r["proto_wild"] = 1
    patterns = [(row[2], row[3]) for row in rows]
    return r, names, tnames, tlens, patterns


def worked_examples():
    out = []
    for l in _lines("worked_examples.txt"):
        kind, inputs, expected, source = [s.strip() for s in l.split("|")]
        kv = dict(tok.split("=") for tok in inputs.split())
        out.append((kind, kv, expected, source))
    return out
