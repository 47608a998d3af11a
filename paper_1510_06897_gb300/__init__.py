"""GB300 (sm_103a) implementation of the overlap Dirac operator hot path
(Cundy & Lee, "Overlap fermions on GPUs", arXiv:1510.06897).

The compute path lives in the C-ABI shared library built from ``csrc/``;
``binding`` marshals arguments to it.  Importing the package does not load
the library: ``binding.lib()`` does, and raises if it has not been built.
"""
