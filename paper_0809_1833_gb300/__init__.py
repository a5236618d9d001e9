"""GB300-native Matching Pursuit decoder (sm_103a).

The compute path lives in the CUDA library ``libmpgb.so`` built from
``csrc/``; ``binding`` is a thin ctypes layer over its C ABI.  Importing this
package does not load the library; ``binding.lib()`` does, and raises if the
library has not been built.
"""
__all__ = ["binding", "workloads"]
