"""GB300-native ghost-cell multigrid for the Poisson equation on {phi < 0}.

The solver lives in the CUDA shared library ``libgcmg.so`` built from
``csrc/``; ``gcmg`` is its thin ctypes binding.  ``inputs`` holds seeded
synthetic problems.  Importing this package loads nothing compiled.
"""
