"""GB300 (sm_103a) boundary-MPS environments of finite PEPS.

The compute path is the C-ABI library ``libpeps.so`` (hand-written CUDA
kernels); :mod:`paper_1311_6696_gb300.peps` is a thin ctypes binding with the
same names.  :mod:`paper_1311_6696_gb300.synth` draws seeded inputs.
"""
