"""GB300-native ASKIT evaluation (March, Xiao & Biros, arXiv:1410.0260).

``askit`` is the Python binding of the C ABI (include/askit.h) implemented in
``csrc/`` as CUDA for sm_103a; ``workloads`` draws seeded synthetic inputs.
"""
__all__ = ["askit", "workloads", "build"]
