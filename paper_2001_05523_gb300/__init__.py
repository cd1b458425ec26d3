"""GB300-native H^2-matrix BEM matvec (Laplace single and double layer).

The compute path is the CUDA library libh2bem.so (C ABI in include/h2bem.h);
``h2bem`` is its thin Python binding and ``inputs`` the seeded synthetic
meshes and right-hand sides.
"""
