"""DSES (Direct Semi-Exhaustive Search, arXiv 2502.00115) on B300 / sm_103a.

The registration path lives in libdses.so (csrc/, C ABI in include/dses.h);
`capi` is its ctypes binding, `synth` the seeded synthetic inputs, `build`
compiles the library.
"""
