"""GB300-native solve phase of the edge-matrix AMG (Kogler & Schoeberl).

``amg`` is the ctypes binding of libamg (include/amg.h); ``build`` compiles
the CUDA sources for sm_103a in-tree.
"""
