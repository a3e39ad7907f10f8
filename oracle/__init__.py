"""FP64 CPU oracle of the kernel-independent treecode (arXiv 1902.02250).

Test infrastructure only: the test suite, the smoke check and the
benchmark's CPU-baseline leg use it; the library under
``paper_1902_02250_gb300`` never imports it.
"""
from .oracle import *  # noqa: F401,F403
