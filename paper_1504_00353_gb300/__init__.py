"""GB300-native (sm_103a) Fast-SSC decoder for systematic polar codes.

The decoder runs in hand-written CUDA kernels inside ``libpolar_gb300.so``,
reached through the C ABI declared in ``include/polar_gb300.h``. The Python
binding in :mod:`paper_1504_00353_gb300.polar` only marshals arguments
(tensor data pointers, sizes, the CUDA stream) into that ABI.
:mod:`paper_1504_00353_gb300.synth` draws the seeded synthetic workloads.
"""
