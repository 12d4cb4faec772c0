"""GB300-native shift-and-invert eigensolver for arrowhead matrices.

Implements the method of Jakovcevic Stor, Slapnicar & Barlow, "Accurate
eigenvalue decomposition of arrowhead matrices and applications": for each
eigenvalue, shift to the nearest pole, invert the shifted arrowhead (one
element in double-double), bisect for the inverse's extreme eigenvalue, and
form the componentwise-accurate eigenvector -- one warp per eigenpair on the
GPU.  The compute path is a C-ABI CUDA library (``include/arrowhead.h``);
``paper_1302_7203_gb300.arrowhead`` is its thin Python binding.
"""

__all__ = ["arrowhead", "workloads"]
