"""Seeded synthetic inputs for the packet classifier: rulesets, traces, update streams.

This package only draws random inputs (rules, packet headers, arrivals). It holds none of
the classification arithmetic, so both the CPU oracle and the CUDA path can consume it.
"""
from .synth import (  # noqa: F401
    HEADER_DTYPE,
    RULE_DTYPE,
    NO_MATCH,
    LEN_CHOICES,
    LEN_WEIGHTS_DEFAULT,
    LEN_WEIGHTS_SKEWED,
    gen_rules,
    gen_clustered_rules,
    sample_inside,
    uniform_headers,
    zipf_ranks,
    gen_trace,
    trace_for_config,
    rules_for_config,
    gen_update_stream,
    gen_serving_arrivals,
    table1_rules,
)
