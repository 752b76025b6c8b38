"""FP64 CPU oracle of the PDHCG-II iteration (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, loads or calls it.
"""
from .oracle import (  # noqa: F401
    OracleParams,
    OracleResult,
    build,
    default_params,
    inner_solve,
    kkt,
    norm_estimate,
    pid_update,
    ruiz,
    solve,
    STATUS_NAMES,
)
