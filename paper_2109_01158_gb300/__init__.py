"""GB300-native evaluation of nonlinear FEM energies and their gradients over P1
triangles and tetrahedra (Moskovka & Valdman, arXiv 2109.01158).

The compute path is the CUDA library ``libfemenergy.so`` (C ABI, ``include/femenergy.h``);
``paper_2109_01158_gb300.fem`` is its thin Python binding.
"""
