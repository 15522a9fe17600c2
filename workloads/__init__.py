"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This package only draws random bytes and patterns; it holds none of the
matching arithmetic (no hashing, no comparison of windows).
"""

from .gen import (  # noqa: F401
    Workload,
    ZIPF_ORDER,
    dna_single,
    zipf_large,
    signature_set,
    random_small,
    make_config,
    Batch,
    batched,
    serving_tables,
    serving_texts,
)
