"""GB300 (sm_103a) SpAMM and SP2: the hot path of the O(N) spectral-projection
solver of Bock, Challacombe and Kale (arXiv:1403.7458).

`spamm` is the Python binding of the C ABI declared in `include/spamm.h`;
`synth` draws the seeded synthetic inputs; `build` compiles the CUDA library.
"""
__all__ = ["spamm", "synth", "build"]
