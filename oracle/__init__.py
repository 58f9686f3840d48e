"""FP64 CPU oracle for the LOPe stencil hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs use this package.  The library in ``paper_1502_03504_gb300``
never imports it.  See ``lope_oracle.c`` for the paper passages each function
follows.
"""
from .oracle import (  # noqa: F401
    BC_DIRICHLET,
    BC_PERIODIC,
    KIND,
    adjoint,
    apply,
    apply_source,
    build,
    max_threads,
    vjp,
    weights,
)
