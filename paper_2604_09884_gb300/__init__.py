"""GB300-native memory-efficient INR gradients for CT (arXiv 2604.09884).

The compute path lives in the CUDA library ``libinrct.so`` (sources in
``csrc/``, C-ABI in ``include/inrct.h``); ``inrct`` is its thin ctypes
binding.  Importing this package does not load the library; the first call
into ``inrct`` does, and raises if the library is missing.
"""
__all__ = ["inrct", "synth"]
