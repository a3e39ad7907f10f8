"""GB300 (sm_103a) kernel-independent treecode of arXiv 1902.02250.

``kitc`` is the Python binding of the C ABI in include/kitc.h (libkitc.so,
built in-tree by ``build``); ``workloads`` draws the seeded synthetic inputs.
"""
from . import kitc, workloads  # noqa: F401
