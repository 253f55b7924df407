"""GB300-native multigrid waveform relaxation (MGWR) for the time-fractional
heat equation D_t^alpha u - Laplace u = f (Gaspar & Rodrigo, arXiv 1608.05400).

* ``inputs``  -- seeded synthetic workloads (numpy only)
* ``mgwr``    -- ctypes binding of the CUDA library ``libmgwr.so`` (include/mgwr.h)
* ``_build``  -- in-tree nvcc build of ``libmgwr.so`` for sm_103a

Importing the package loads nothing; ``mgwr.load()`` loads the CUDA library
and raises if it is missing.
"""
