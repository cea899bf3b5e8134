"""GB300-native scale-based collision avoidance (arXiv 2406.07048).

The compute path is the CUDA library ``liboca.so`` behind the C-ABI in
``include/oca.h``; :mod:`paper_2406_07048_gb300.binding` marshals arguments
to it.  Importing this package does not load the library.
"""
__all__ = ["synth"]
