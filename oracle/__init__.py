"""CPU oracle of the estimator's hot path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` and ``--impl reference`` legs) may import this package.  The
library under ``paper_2509_19974_gb300`` never does; it has no CPU fallback.
"""
from .oracle import (  # noqa: F401
    build, quantize, rank_thresholds, xcorr, xcorr_at, argmax, estimate,
    num_threads, full_lag_range, real_ccf, refine,
)
