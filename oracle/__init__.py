"""FP64 CPU oracle for the wind-tunnel FW-H integral (TEST INFRASTRUCTURE ONLY).

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline
leg may import this package.  The product library never calls it.
"""
from .oracle import Oracle, build_oracle, load_oracle

__all__ = ["Oracle", "build_oracle", "load_oracle"]
