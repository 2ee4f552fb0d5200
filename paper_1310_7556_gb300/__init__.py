"""GB300-native Hough-transform track finding (Halyo et al., arXiv:1310.7556).

The hot path -- hit staging, stage-1 (q/pT, phi0) vote, peak search, candidate
membership and the stage-2 (cot theta, z0) vote -- runs as hand-written CUDA
kernels for sm_103a behind the C ABI declared in ``include/hough.h``.
``binding`` is the thin ctypes layer over that library; ``eventgen`` holds the
seeded synthetic workloads.  Importing the package loads nothing: the CUDA
library is opened on first use and its absence is an error, never a fallback.
"""
