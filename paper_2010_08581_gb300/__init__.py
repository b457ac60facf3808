"""GB300-native TR-ALS-Sampled (Malik & Becker, Alg. 2 with Alg. 3 and Alg. 4): sm_103a
CUDA kernels behind a C ABI (``libtrals.so``), with a thin ctypes binding in
:mod:`paper_2010_08581_gb300.trals`.

Importing the package does not load the CUDA library; :mod:`.trals` loads it on first
use and raises if it has not been built.
"""
