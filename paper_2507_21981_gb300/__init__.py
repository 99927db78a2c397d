"""GB300-native batched 3D Gaussian Splatting RGB + depth renderer (DISCOVERSE, arXiv 2507.21981).

Modules:
  scenes  seeded synthetic scenes (inputs only)
  build   builds libdgs.so in-tree for sm_103a
  dgs     ctypes binding of the C ABI (include/dgs.h), same names
  render  torch-facing DeviceScene / Renderer (device memory and streams from PyTorch)

Importing the package loads nothing; `render` and `dgs` load libdgs.so on first use and raise
if it is missing.
"""
