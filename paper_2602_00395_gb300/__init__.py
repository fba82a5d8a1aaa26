"""GB300-native hot path of the 3DGS^2-TR optimiser (arXiv 2602.00395).

The compute lives in the CUDA library ``libgs3dtr.so`` (sources in ``csrc/``,
C ABI in ``include/gs3dtr.h``); ``gs3dtr`` is its thin Python binding and
``synth`` the seeded synthetic-input generators.
"""
