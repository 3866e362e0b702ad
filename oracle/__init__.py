"""CPU oracle for the KPM density-of-states path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct FP64 implementations of what the GPU library
computes, written from the paper (Lin, Saad, Yang, arXiv:1308.5467).  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference
leg may import this package; the library never does, and nothing here imports
the library.

Modules:
  kpm     -- start vectors and the Chebyshev moment sweep (C, kpm_oracle.c)
  bounds  -- Gershgorin and k-step Lanczos spectrum bounds (Section 3.1)
  dos     -- Jackson damping, reconstruction and the smoothed error metric
  mlp     -- FP64 forward/backward of the moments-to-DOS network

Pinned by tests/test_oracle_*.py against dense eigendecompositions, the
closed-form Laplacian spectrum, special cases and invariants (no pin compares
the oracle with itself).
"""
