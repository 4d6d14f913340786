"""GB300-native VESIS hot path (arXiv 2208.05524).

The compute lives in the CUDA shared library `libvesis.so` (C ABI declared
in include/vesis.h); `paper_2208_05524_gb300.vesis` is its thin ctypes
binding and `paper_2208_05524_gb300.synth` draws seeded synthetic inputs.
Importing this package loads nothing.
"""
