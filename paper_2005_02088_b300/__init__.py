"""B300-native Camelot query-pipeline runtime (ctypes binding of libcamelot.so).

``camelot`` holds the C-ABI wrappers; ``pipelines`` builds the synthetic
pipelines (plain 2-stage FP32, 3-stage BF16) from weight tensors.
"""
from . import camelot  # noqa: F401
from .camelot import CamelotError  # noqa: F401
