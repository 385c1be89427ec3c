"""B300-native CSPH-TVD gas dynamics (Khrapov, Khoperskov & Khoperskov, arXiv 1912.04855).

``cspht`` is the thin ctypes binding of the CUDA library ``libcspht.so`` (C ABI
declared in ``include/cspht.h``); ``workloads`` holds the seeded initial
conditions of the paper's test problems.
"""
