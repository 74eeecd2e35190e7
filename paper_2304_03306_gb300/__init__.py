"""GB300 (sm_103a) solver for the confined Toner-Tu-Swift-Hohenberg active-fluid model.

The compute path is libttsh.so (hand-written CUDA, C ABI in include/ttsh.h); ``ttsh`` is
its ctypes binding and ``build`` compiles it in-tree.
"""
