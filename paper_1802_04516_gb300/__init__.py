"""GB300 (sm_103a) implementation of the staggered space-time DG scheme for
velocity-stress linear elasticity (Tavelli & Dumbser, arXiv:1802.04516).

The compute path is the CUDA library libstdg.so (C ABI in include/stdg.h);
``binding`` marshals arguments to it and ``build`` compiles it in-tree.  Importing
this package does not load the library; ``binding.load()`` does, and raises if it is
missing.
"""
__all__ = ["binding", "build"]
