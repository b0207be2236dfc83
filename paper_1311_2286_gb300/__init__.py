"""GB300-native (sm_103a) curvilinear particle-in-cell hot path (CPIC, arXiv 1311.2286).

Importing the package loads nothing: the CUDA library is loaded by
``paper_1311_2286_gb300.cpic`` (the thin ctypes binding of include/cpic.h), which fails
loudly when the compiled library is missing.
"""
