"""GB300-native approximate LDM^t factorization with HSS-compressed Schur
complements over a nested-dissection tree, applied as a preconditioner in
flexible GMRES (Gatto & Hesthaven, arXiv 1508.07798).

Submodules:
  dg_inputs   seeded synthetic SIPG DG system matrices (inputs only)
  hssnd       ctypes binding of the CUDA C-ABI library libhssnd.so
"""
__version__ = "0.1.0"
