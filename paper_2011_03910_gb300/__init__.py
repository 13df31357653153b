"""GB300-native JDE detect-and-track: CUDA library ``libjde`` (sm_103a) and its Python binding.

The compute path is ``libjde.so`` (C ABI, ``include/jde.h``); ``jde`` is a thin
ctypes binding with the same function names.  Build with
``python -m paper_2011_03910_gb300._build``.
"""
