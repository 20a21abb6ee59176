"""GB300-native hybrid tree force path (Watanabe & Nakasato, hybrid tree algorithm).

The compute path is the CUDA library ``libhybrid.so`` behind a C-ABI
(``include/hybrid.h``); :mod:`paper_1406_6158_gb300.hybrid` is its thin ctypes
binding. :mod:`paper_1406_6158_gb300.ics` holds the seeded input generators.
"""
__all__ = ["hybrid", "ics"]
