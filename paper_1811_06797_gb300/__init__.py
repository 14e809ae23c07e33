"""GB300-native low-rank isogeometric optimal control (Buenger, Dolgov, Stoll).

The compute path lives in the CUDA library ``libiga.so`` (sources in
``csrc/``, C ABI in ``include/iga.h``); ``iga`` is its ctypes binding.
Importing this package does not load the library; the first call through
``paper_1811_06797_gb300.iga`` does, and raises if it is missing.
"""
