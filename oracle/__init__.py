"""CPU oracle for the J/K build (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never touches the CUDA library and
shares no code with it; both sides read the same seeded arrays from
``workloads``.

The arithmetic lives in ``eri_oracle.c`` (Obara-Saika + Head-Gordon-Pople in
FP64, own Boys function, J/K by definition); ``brute.py`` holds an
independent numerical-integration check for low angular momentum.
"""

from .oracle import (  # noqa: F401
    build_oracle,
    boys,
    normalise,
    shell_quartet,
    schwarz,
    jk,
    jk_blocks,
    jk_sample,
    count_quartets,
    max_threads,
    OracleBasis,
    OPS_PHASES,
    quartet_ops,
    class_ops,
)
