"""CPU oracle (FP64) for the boundary-MPS PEPS environments.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import, call or execute anything in
this package.  It shares no code with the CUDA path, and the CUDA path never
routes through it.

* :mod:`oracle.peps_oracle` -- the method of the paper, step by step.
* :mod:`oracle.bruteforce` -- state vectors of small PEPS (the plain
  definition), used to pin the oracle.
* :mod:`oracle.update_oracle` -- the tensor update of the full / cluster
  update (reduced-tensor ALS, Section 2) and its imaginary-time driver.
"""
