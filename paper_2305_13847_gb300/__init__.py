"""GB300-native moist DG right-hand side and SSPRK(4,3) step (arXiv 2305.13847).

The compute path is the CUDA library ``libdgmoist.so`` (sources in ``csrc/``,
C interface in ``include/dgmoist.h``); ``dgmoist`` is its thin ctypes binding.
Importing this package loads nothing; the library is loaded on first use of
``paper_2305_13847_gb300.dgmoist`` and a missing library is an error.
"""
