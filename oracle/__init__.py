"""ORACLE -- test infrastructure, not product code.

A plain, slow, obviously correct CPU restatement of what the packet-classification path
computes, written from the paper and shared with nothing in the CUDA path:

  linear_scan.c / classify.py  §2.1 definition: highest-priority matching rule (linear scan)
  tss.py                       §4.3 tuple construction and truncation, §5.2.1 restricted
                               insertion, and the overlap-conflict sets that make the
                               post-verification of §5.1.1 exact
  mlp.py                       §6.1 residual MLP (Eq. 1-2) forward and backward in float64,
                               §6.2 feature encoding, cross-entropy and Adam (§6.2 training)
  quant.py                     BF16 and FP8 E4M3 round-to-nearest-even encoders written from
                               the formats' definitions

Only tests, the smoke check and the benchmark's CPU-baseline leg may import this package.

Parity status: every function here is pinned by a test in tests/test_oracle_*.py against values
the paper prints (Table 1, §4.3 and §5.2.1 worked examples), closed forms, finite differences,
library routines for special cases, or brute force on tiny inputs. None is "parity unpinned".
"""
