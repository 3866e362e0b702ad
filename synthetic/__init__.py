"""Seeded synthetic inputs shared by the tests, the oracle and the benchmark.

This package only builds matrices (CSR arrays) and their parameters; it holds
none of the kernel polynomial method's arithmetic.  Both the CUDA path and the
CPU oracle read the very same arrays, so the generators need not be
bit-reproducible across implementations.
"""
from .matrices import (  # noqa: F401
    CSR,
    laplacian_2d,
    anderson_3d,
    chung_lu_normalized_laplacian,
    random_symmetric,
    diagonal,
    batched_anderson,
    concat_block_diagonal,
)
