"""GB300-native DSPS photometry hot path (Hearin et al. 2021, arXiv:2112.06830).

The compute path is the CUDA library ``libdsps.so`` behind the C ABI declared in
``include/dsps.h``; ``paper_2112_06830_gb300.dsps`` is its thin ctypes binding.
Importing this package loads nothing; the library is loaded on first use.
"""
__all__ = ["synth"]
