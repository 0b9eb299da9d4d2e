"""FP64 CPU oracle of the EPIC imaging path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline/reference
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library: ``epic_oracle.c`` restates the paper's Eq. 1-2 in plain loops with its
own geometry, unpacking and radix-2 transform, and ``bruteforce.py`` evaluates
the same image through explicit pairwise correlations (the O(N^2) correlator
route the method avoids, paper Sec. 1-2).

Parity of every function here is pinned by the ``-m "not gpu"`` tests against
facts the mathematics fixes (exhaustive unpack table, naive DFT and numpy's
inverse FFT, Parseval, closed-form one- and two-element images, point-source
localisation, time linearity, and the pairwise-correlation brute force).
"""
from .oracle import (  # noqa: F401
    GCF_GAUSSIAN, GCF_TABLE, build, lib, unpack_table, unpack8_pairs, fft2, footprint, grid_frame, image, image_cfg, max_threads,
    OracleError,
)
