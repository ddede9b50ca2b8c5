"""GB300-native adaptive-resolution WCSPH (Muta & Ramachandran, arXiv
2107.01276): hand-written CUDA kernels for sm_103a behind a C ABI.

``paper_2107_01276_gb300.sph`` is the Python binding of that C ABI;
``paper_2107_01276_gb300.workloads`` holds the seeded input generators.
Importing the package itself loads nothing.
"""
