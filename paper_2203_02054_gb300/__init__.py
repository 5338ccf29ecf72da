"""GB300-native collision-aware local-global soft-robot simulation.

``casim``  -- Python binding of the CUDA library's C ABI (include/casim.h).
``synth``  -- seeded synthetic voxel-finger inputs (no method arithmetic).
``build``  -- nvcc build of libcasim.so for sm_103a.
"""
