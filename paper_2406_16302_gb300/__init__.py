"""Residual path integrals for re-rendering (arXiv 2406.16302) on GB300.

``scenes``  seeded procedural scenes and edits (input data)
``rp``      ctypes binding of librp.so, the CUDA implementation
``build``   in-tree nvcc build of librp.so for sm_103a
"""
