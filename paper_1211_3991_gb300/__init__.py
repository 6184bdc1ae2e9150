"""GB300-native Monte Carlo of the XY model on dilute Levy graphs.

The compute lives in ``libxyl.so`` (CUDA for sm_103a + host C++), reached
through the C ABI declared in ``include/xyl.h``; ``xyl`` is its ctypes binding.
"""
from . import xyl  # noqa: F401
from .xyl import (FP32_BATCHED, FP32_PLAIN, FP64_PLAIN, OP_MEASURE, OP_MET, OP_OR, OP_PT, Graph, Plan,  # noqa: F401
                  XylError, build_graph_csr, graph_from_edges)
