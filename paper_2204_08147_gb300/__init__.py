"""GB300-native typicality + block-Lanczos estimator of the equilibrium-reduced
density matrix rho*_s = tr_b(exp(-beta H_t))/Z_t and the mean-force Hamiltonian
(Chen & Cheng, arXiv:2204.08147).

The compute path is ``librdm.so`` (hand-written sm_103a CUDA + C++ host code) behind
the C ABI in ``include/rdm.h``; ``paper_2204_08147_gb300.rdm`` is its Python binding.
Import ``rdm`` explicitly: it loads the library and fails if it is not built.
"""
