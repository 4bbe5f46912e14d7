"""FP64 CPU oracle for AIDW (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. The product library never does, and this package imports nothing from it.
"""
from .oracle import (  # noqa: F401
    build,
    load_library,
    default_threads,
    r_exp,
    mu_of_R,
    alpha_of_mu,
    knn,
    interpolate,
    idw,
)
