"""GB300-native MBE(3)-OSV-MP2 energies and OSV-space analytical gradients (arXiv 2106.06149).

The compute path is the C-ABI library libosvmbe.so (CUDA, sm_103a); `osvmbe` is its thin ctypes binding.
Importing this package does not load the library; `synth` (seeded inputs) needs no GPU.
"""
