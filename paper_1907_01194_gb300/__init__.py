"""GB300-native kernels for the spin-F BEC ground-state hot path of
arXiv:1907.01194 (Fourier-pseudospectral Gross-Pitaevskii energy, gradients,
Hessian-vector products and retractions behind the C-ABI library libsbec).

The CUDA binding lives in :mod:`paper_1907_01194_gb300.sbec`; importing it
loads the compiled library and raises if it is missing.  The seeded workload
generators are in :mod:`paper_1907_01194_gb300.workloads`.
"""
