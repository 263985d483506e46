"""GB300-native exhaustive flux-balanced pathway enumeration.

Hot path of "A system architecture for parallel analysis of flux-balanced
metabolic pathways" (Arabzadeh et al.): the data-parallel traversal of the
metabolic AND/OR graph, as hand-written sm_103a CUDA behind a C-ABI
(include/efmgraph.h).

Submodules:
  efmgraph -- ctypes binding of the C-ABI (loads libefmgraph.so, no fallback)
  build    -- compiles the library in-tree (nvcc, sm_103a)
  synth    -- seeded synthetic networks (input generator only)
"""
