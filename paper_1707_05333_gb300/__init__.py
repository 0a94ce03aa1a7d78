"""GB300-native moving-mesh hot path (Voronoi tessellation + MUSCL-Hancock/HLLC).

The compute path lives in the CUDA library under ``csrc/``; ``binding`` loads
it through its C ABI.  Importing this package does not load the library.
"""
