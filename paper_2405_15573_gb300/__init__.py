"""GB300-native uniform H-matrix (UH) matrix-vector product.

The compute path is the C-ABI library built from `csrc/` (CUDA for sm_103a); `uh` holds the thin
ctypes binding. `inputs` generates the seeded synthetic workloads.
"""
