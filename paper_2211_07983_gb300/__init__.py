"""GB300-native differentiable MPS simulator for VQE (arXiv:2211.07983).

The computation lives in libmps.so (CUDA for sm_103a + C++ host builders, C ABI in
include/mps.h).  This package holds its ctypes binding (`api`), the autograd wrapper
(`autograd.MPSEnergy`), the build script (`build`) and the multi-rank sharding helpers
(`parallel`).  Importing the package does not load the library; the first call does,
and fails loudly if the library was not built.
"""
from .api import (Circuit, Hamiltonian, State, apply_circuit, apply_circuit_host, build_hamiltonian,
                  compile_excitations, energy, energy_cotangent, energy_grad, energy_grad_host, energy_grad_multi, energy_host,
                  kernel_launches, svd)

__all__ = ["Circuit", "Hamiltonian", "State", "apply_circuit", "apply_circuit_host", "build_hamiltonian",
           "compile_excitations", "energy", "energy_cotangent", "energy_grad", "energy_grad_host", "energy_grad_multi", "energy_host",
           "kernel_launches", "svd"]
