"""GB300-native fused image-kernel chains (arXiv 1509.04394).

libkfuse.so (include/kfuse.h) holds the partitioner and the CUDA kernels; `kfuse` is
its ctypes binding. Build it with `python -m paper_1509_04394_gb300.build`.
"""
from . import kfuse  # noqa: F401
