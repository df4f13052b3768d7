"""GB300 (sm_103a) sparse-wavefunction circuit solver: the data-parallel hot
path of ADAPT-VQE with a sparse determinant state (arXiv 2411.07920, Sec. II).

Importing the package loads nothing; ``paper_2411_07920_gb300.swcs`` binds the
CUDA library (and fails loudly when it has not been built).
"""
