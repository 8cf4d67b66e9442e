"""CPU oracle of BDDC-preconditioned CG — test infrastructure only.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package. The CUDA library never calls it.
"""
from .bddc_oracle import (ALL_GLOBS, CORNER, EDGE, FACE, Oracle, dirichlet_mask,  # noqa: F401
                          element_nodes, q1_element_matrices)
