"""libcbp: check-belief propagation (CBP) decoding of QC-LDPC codes on GB300 (sm_103a).

The decoder kernels live in ``csrc/`` behind the C ABI declared in ``include/cbp.h``;
``cbp`` is the thin ctypes binding and ``inputs`` the seeded input generators.
Importing the package loads nothing: ``from paper_2305_05286_gb300 import cbp`` does.
"""
