"""GB300-native made-to-measure (M2M) particle-model training step.

The compute path is the C-ABI library ``libm2m.so`` (hand-written sm_103a
CUDA kernels, built in-tree by :mod:`paper_1207_6403_gb300.build`); the
Python binding in :mod:`paper_1207_6403_gb300.m2m` only marshals arguments.
:mod:`paper_1207_6403_gb300.inputs` holds the seeded synthetic workloads.
Importing this package loads nothing; the library is loaded on first use.
"""
