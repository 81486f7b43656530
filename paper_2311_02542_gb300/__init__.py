"""GB300-native per-ray renderer of VR-NeRF's field (hash grid + LOD + MLP +
PQ colour), as a C-ABI CUDA library for sm_103a.

Submodules:
  vrnerf  -- thin ctypes binding of the C-ABI (loads the CUDA library; fails
             loudly when it is missing)
  synth   -- seeded synthetic scenes, cameras and parameter blobs
  build   -- compiles the CUDA library in-tree with nvcc
"""
__all__ = ["vrnerf", "synth", "build"]
